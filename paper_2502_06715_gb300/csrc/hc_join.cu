// Generic Join over CoCo indexes, one logical worker per HyperCube cell
// (Sec. 5 "Executor"; Listing C of Fig. "algo-comp").
//
// GPU mapping.  Loop 1 of every cell (the intersection of the top levels of
// the atoms holding X_sigma(1), Sec. 5) runs as a flat data-parallel pass: one
// thread per value of the cell's shortest top-level list, probing the others.
// Its surviving bindings ("entries") are the roots of the cells' search
// trees.  The rest of the loops run in a persistent kernel: a warp takes a
// work item (a range of loop-2 candidates of one or more entries, handed out
// by an atomic counter), and walks the remaining loops depth first.  At each
// loop the warp holds a batch of at most 32 parent bindings, one per lane,
// and flattens the candidates of all of them over its lanes: a candidate is
// an element of its parent's shortest list (the paper's choice: iterate the
// smallest set, search the others, Sec. 5.2), searched in the parent's other
// lists by binary search (the "search(V, x)" primitive of Sec. 5); matches are
// compacted with ballots into the next batch.  At the last loop a match is
// counted (count mode) or written (materialize mode).
#include <algorithm>
#include <vector>

#include "hc_internal.cuh"

namespace hc {

constexpr int MAXSRC = 4;   // lists intersected by one loop
constexpr int MAXOPEN = 4;  // atoms whose first variable one loop binds

// One atom as the kernels see it.  Unpartitioned atoms (one share for both
// variables) are read in place: their level 1 is [0, l1_whole).
struct DAtom {
    const uint32_t* v1;
    const uint32_t* o1;
    const uint32_t* v2;
    const uint32_t* l1s;  // level-1 start of each partition, [np + 1]; NULL when whole
    uint32_t l1_whole;
    uint32_t pb;                                     // shares of the second variable
    uint32_t stride_f, share_f, stride_s, share_s;  // cell -> partition identifiers
    int lev_first, lev_second, slot;                // slot among atoms opened at lev_first
};

// The query plan: loops, the lists each loop intersects (top-level lists of
// the atoms it opens first, in slot order, then sub-lists R[x] of atoms
// opened earlier), and the variable each loop binds.
struct DPlan {
    int nlev, natoms, nv;
    uint32_t ncells;
    DAtom atom[HC_MAX_ATOMS];
    int nsrc[HC_MAX_VARS];
    int src_atom[HC_MAX_VARS][MAXSRC];
    int src_top[HC_MAX_VARS][MAXSRC];
    int nopen[HC_MAX_VARS];
    int var_of_level[HC_MAX_VARS];
};

struct JoinCtl {
    uint32_t err;
    uint32_t item_ctr[2];
    uint32_t n_entries;  // loop-1 bindings, written by the loop-1 pass
    uint64_t total;      // |Q|
    uint64_t work;       // work counter (stats)
    uint64_t n_items;
};

__device__ __forceinline__ void load_plan(DPlan& dst, const DPlan* __restrict__ src) {
    const uint32_t* s = (const uint32_t*)src;
    uint32_t* d = (uint32_t*)&dst;
    for (uint32_t i = threadIdx.x; i < sizeof(DPlan) / 4; i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

__device__ __forceinline__ void top_range(const DAtom& a, uint32_t cell, uint32_t& lo, uint32_t& hi) {
    if (a.l1s == nullptr) {
        lo = 0;
        hi = a.l1_whole;
        return;
    }
    const uint32_t sf = (cell / a.stride_f) % a.share_f;
    const uint32_t ss = (cell / a.stride_s) % a.share_s;
    const uint32_t pid = sf * a.pb + ss;
    lo = a.l1s[pid];
    hi = a.l1s[pid + 1];
}

// ------------------------------------------------------------------ loop 1
// Per cell: length of the shortest top-level list of loop 1.
__global__ void l0_count_kernel(const DPlan* __restrict__ gP, uint32_t* __restrict__ cand, JoinCtl* ctl, int stats) {
    __shared__ DPlan P;
    load_plan(P, gP);
    uint64_t work = 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < P.ncells; c += gridDim.x * blockDim.x) {
        uint32_t m = 0xFFFFFFFFu;
        for (int q = 0; q < P.nsrc[0]; ++q) {
            uint32_t lo, hi;
            top_range(P.atom[P.src_atom[0][q]], c, lo, hi);
            m = min(m, hi - lo);
        }
        cand[c] = m;
        work += (uint64_t)P.nsrc[0] * m;
    }
    if (stats) {
        work = warp_sum64(work);
        if (lane_id() == 0 && work) atomicAdd((unsigned long long*)&ctl->work, (unsigned long long)work);
    }
}

// Candidate t -> (cell, value of the cell's shortest loop-1 list); probe the
// other loop-1 lists.  WRITE=false stores the match flag (0 past the last
// candidate); WRITE=true writes each matching candidate as an entry at its
// compacted slot, with the ranges of the atoms it opens and its number of
// loop-2 candidates.
template <bool WRITE>
__global__ void l0_probe_kernel(const DPlan* __restrict__ gP, const uint64_t* __restrict__ candoff, uint64_t tmax,
                                uint32_t* __restrict__ flags, const uint64_t* __restrict__ flagoff,
                                uint32_t* __restrict__ e_cell, uint32_t* __restrict__ e_x,
                                uint32_t* __restrict__ e_rng, uint32_t* __restrict__ e_units) {
    __shared__ DPlan P;
    load_plan(P, gP);
    const uint64_t T = min(tmax, candoff[P.ncells]);
    const int n0 = P.nsrc[0];
    const uint64_t tend = WRITE ? T : tmax;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < tend; t += (uint64_t)gridDim.x * blockDim.x) {
        if (!WRITE && t >= T) {
            flags[t] = 0;
            continue;
        }
        if (WRITE && flags[t] == 0) continue;
        uint32_t lo = 0, hi = P.ncells;  // last cell c with candoff[c] <= t
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (candoff[mid] <= t)
                lo = mid;
            else
                hi = mid;
        }
        const uint32_t c = lo;
        const uint32_t k = (uint32_t)(t - candoff[c]);
        uint32_t rlo[MAXOPEN], rhi[MAXOPEN];
        uint32_t best = 0, bestlen = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < MAXOPEN; ++q) {
            rlo[q] = rhi[q] = 0;
            if (q < n0) {
                top_range(P.atom[P.src_atom[0][q]], c, rlo[q], rhi[q]);
                if (rhi[q] - rlo[q] < bestlen) {
                    bestlen = rhi[q] - rlo[q];
                    best = q;
                }
            }
        }
        uint32_t x = 0;
#pragma unroll
        for (int q = 0; q < MAXOPEN; ++q)
            if (q == (int)best) x = P.atom[P.src_atom[0][q]].v1[rlo[q] + k];
        bool ok = true;
        uint32_t pos[MAXOPEN];
#pragma unroll
        for (int q = 0; q < MAXOPEN; ++q) {
            pos[q] = 0;
            if (q < n0) {
                const DAtom& a = P.atom[P.src_atom[0][q]];
                uint32_t p = (q == (int)best) ? rlo[q] + k : lower_bound_u32(a.v1, rlo[q], rhi[q], x);
                ok = ok && p < rhi[q] && a.v1[p] == x;
                pos[q] = p;
            }
        }
        if (!WRITE) {
            flags[t] = ok ? 1u : 0u;
            continue;
        }
        const uint64_t e = flagoff[t];
        e_cell[e] = c;
        e_x[e] = x;
#pragma unroll
        for (int q = 0; q < MAXOPEN; ++q) {
            uint32_t a0 = 0, a1 = 0;
            if (q < n0) {
                const DAtom& a = P.atom[P.src_atom[0][q]];
                a0 = a.o1[pos[q]];
                a1 = a.o1[pos[q] + 1];
            }
            rlo[q] = a0;
            rhi[q] = a1;
            e_rng[e * (2 * MAXOPEN) + 2 * q] = a0;
            e_rng[e * (2 * MAXOPEN) + 2 * q + 1] = a1;
        }
        uint32_t m = 1;  // a one-loop query: the entry is the output
        if (P.nlev > 1) {
            m = 0xFFFFFFFFu;
            for (int q = 0; q < P.nsrc[1]; ++q) {
                const DAtom& a = P.atom[P.src_atom[1][q]];
                uint32_t len = 0;
                if (P.src_top[1][q]) {
                    uint32_t l0, l1;
                    top_range(a, c, l0, l1);
                    len = l1 - l0;
                } else {
#pragma unroll
                    for (int s = 0; s < MAXOPEN; ++s)
                        if (s == a.slot) len = rhi[s] - rlo[s];
                }
                m = min(m, len);
            }
        }
        e_units[e] = m;
    }
}

__global__ void entries_total_kernel(const uint64_t* __restrict__ flagoff, const uint64_t* __restrict__ candoff,
                                     uint32_t ncells, uint64_t tmax, JoinCtl* ctl) {
    const uint64_t T = min(tmax, candoff[ncells]);
    ctl->n_entries = (uint32_t)flagoff[T];
}

// ---------------------------------------------------------- search loops
// Bindings of the batches of loops 2.. (index = loop), one per lane.
struct Frame {
    uint32_t val[HC_MAX_VARS];
    uint32_t par[HC_MAX_VARS];
    uint32_t olo[HC_MAX_VARS][MAXOPEN];
    uint32_t ohi[HC_MAX_VARS][MAXOPEN];
};

// The loop-1 binding a work item is under (lane-uniform).
struct EntryCtx {
    uint32_t cell, x;
    uint32_t r0lo[MAXOPEN], r0hi[MAXOPEN];          // atoms opened by loop 1
    uint32_t tlo[HC_MAX_ATOMS], thi[HC_MAX_ATOMS];  // partition top-level range per atom
};

struct Acc {
    uint64_t count;    // matches at the last loop (lane-uniform)
    uint64_t work;     // per-lane work counter
    uint64_t out_pos;  // next output slot (materialize)
    uint32_t* out;
    int stats;
};

// Position of the r-th (0-based) set bit of m (r < popc(m)).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t w = 16; w >= 1; w >>= 1) {
        uint32_t c = __popc(m & ((1u << (pos + w)) - 1u));  // set bits below pos + w
        if (c <= r) pos += w;
    }
    return pos;
}

// Range of source q of loop L for the binding of loop L-1 held by lane
// `lane_of` (every lane calls with its own lane_of; all lanes take part).
template <int L>
__device__ __forceinline__ void src_range(const DPlan& P, const Frame& F, const EntryCtx& E, int q, uint32_t lane_of,
                                          uint32_t& lo, uint32_t& hi) {
    const int j = P.src_atom[L][q];
    const DAtom& a = P.atom[j];
    lo = 0;
    hi = 0;
    if (P.src_top[L][q]) {
#pragma unroll
        for (int jj = 0; jj < HC_MAX_ATOMS; ++jj)
            if (jj == j) {
                lo = E.tlo[jj];
                hi = E.thi[jj];
            }
        return;
    }
    const int f = a.lev_first, s = a.slot;
    if (f == 0) {
#pragma unroll
        for (int ss = 0; ss < MAXOPEN; ++ss)
            if (ss == s) {
                lo = E.r0lo[ss];
                hi = E.r0hi[ss];
            }
        return;
    }
    uint32_t anc = lane_of;  // ancestor at loop f of the loop L-1 binding
#pragma unroll
    for (int g = L - 1; g >= 1; --g)
        if (g > f) anc = __shfl_sync(0xffffffffu, F.par[g], anc);
    uint32_t mylo = 0, myhi = 0;
#pragma unroll
    for (int g = 1; g < L; ++g)
#pragma unroll
        for (int ss = 0; ss < MAXOPEN; ++ss)
            if (g == f && ss == s) {
                mylo = F.olo[g][ss];
                myhi = F.ohi[g][ss];
            }
    lo = __shfl_sync(0xffffffffu, mylo, anc);
    hi = __shfl_sync(0xffffffffu, myhi, anc);
}

__device__ __forceinline__ const uint32_t* src_list(const DPlan& P, int L, int q) {
    const DAtom& a = P.atom[P.src_atom[L][q]];
    return P.src_top[L][q] ? a.v1 : a.v2;
}

// Search candidate v (element kpos of source `best`) in the other lists of
// loop L.  A top-level list that holds v opens its atom: the o1 range of v's
// position is the atom's sub-list for the next loops.
template <int L>
__device__ __forceinline__ bool probe(const DPlan& P, int best, const uint32_t (&rlo)[MAXSRC],
                                      const uint32_t (&rhi)[MAXSRC], uint32_t kpos, uint32_t v, bool active,
                                      uint32_t (&nlo)[MAXOPEN], uint32_t (&nhi)[MAXOPEN]) {
    bool ok = active;
#pragma unroll
    for (int q = 0; q < MAXSRC; ++q) {
        if (q < P.nsrc[L]) {
            const uint32_t* list = src_list(P, L, q);
            uint32_t p = kpos;
            if (q != best) {
                p = ok ? lower_bound_u32(list, rlo[q], rhi[q], v) : rhi[q];
                ok = ok && p < rhi[q] && list[p] == v;
            }
            if (q < MAXOPEN && P.src_top[L][q] && ok) {
                const DAtom& a = P.atom[P.src_atom[L][q]];
                nlo[q] = a.o1[p];
                nhi[q] = a.o1[p + 1];
            }
        }
    }
    return ok;
}

template <int L, int NL, bool MAT>
__device__ __forceinline__ void run_level(const DPlan& P, Frame& F, const EntryCtx& E, Acc& A, uint32_t nb);

// Last loop: count the matches, or write them as output tuples.
template <int L, int NL, bool MAT>
__device__ __forceinline__ void finish_round(const DPlan& P, const Frame& F, const EntryCtx& E, Acc& A, bool ok,
                                             uint32_t v, uint32_t parent) {
    const uint32_t ball = __ballot_sync(0xffffffffu, ok);
    if constexpr (MAT) {
        uint32_t vals[HC_MAX_VARS];
        uint32_t anc = parent;
#pragma unroll
        for (int g = L - 1; g >= 1; --g) {
            vals[g] = __shfl_sync(0xffffffffu, F.val[g], anc);
            anc = __shfl_sync(0xffffffffu, F.par[g], anc);
        }
        if (ok) {
            const uint64_t slot = A.out_pos + __popc(ball & lanemask_lt());
            uint32_t* o = A.out + slot * (uint64_t)P.nv;
            o[P.var_of_level[L]] = v;
            o[P.var_of_level[0]] = E.x;
#pragma unroll
            for (int g = L - 1; g >= 1; --g) o[P.var_of_level[g]] = vals[g];
        }
    }
    A.count += __popc(ball);
    A.out_pos += __popc(ball);
}

// Compact this round's matches into the batch of loop L and descend.
template <int L, int NL, bool MAT>
__device__ __forceinline__ void descend(const DPlan& P, Frame& F, const EntryCtx& E, Acc& A, bool ok, uint32_t v,
                                        uint32_t parent, const uint32_t (&nlo)[MAXOPEN],
                                        const uint32_t (&nhi)[MAXOPEN]) {
    const uint32_t ball = __ballot_sync(0xffffffffu, ok);
    const uint32_t nnew = __popc(ball);
    if (nnew == 0) return;
    const uint32_t lane = lane_id();
    const uint32_t src = lane < nnew ? nth_set_bit(ball, lane) : 0;
    F.val[L] = __shfl_sync(0xffffffffu, v, src);
    F.par[L] = __shfl_sync(0xffffffffu, parent, src);
#pragma unroll
    for (int s = 0; s < MAXOPEN; ++s) {
        F.olo[L][s] = __shfl_sync(0xffffffffu, nlo[s], src);
        F.ohi[L][s] = __shfl_sync(0xffffffffu, nhi[s], src);
    }
    run_level<L + 1, NL, MAT>(P, F, E, A, nnew);
}

// Loop L >= 2 (index): the parents are the nb bindings of loop L-1 held by
// lanes 0..nb-1; their candidates are flattened over the lanes, 32 a round.
template <int L, int NL, bool MAT>
__device__ __forceinline__ void run_level(const DPlan& P, Frame& F, const EntryCtx& E, Acc& A, uint32_t nb) {
    if constexpr (L < NL) {
        const uint32_t lane = lane_id();
        const int ns = P.nsrc[L];
        uint32_t mlo[MAXSRC], mhi[MAXSRC];
        uint32_t best = 0, bestlen = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < MAXSRC; ++q) {
            mlo[q] = mhi[q] = 0;
            if (q < ns) {
                src_range<L>(P, F, E, q, lane < nb ? lane : 0, mlo[q], mhi[q]);
                const uint32_t len = mhi[q] - mlo[q];
                if (len < bestlen) {
                    bestlen = len;
                    best = q;
                }
            }
        }
        const uint32_t cnt = lane < nb ? bestlen : 0;
        if (A.stats) A.work += (uint64_t)ns * cnt;
        const uint32_t incl = warp_incl_scan(cnt);
        const uint32_t excl = incl - cnt;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t t0 = 0; t0 < total; t0 += 32) {
            const uint32_t t = t0 + lane;
            const bool active = t < total;
            uint32_t p = 0;  // parent of candidate t: the last lane p < nb with excl_p <= t
#pragma unroll
            for (uint32_t step = 16; step >= 1; step >>= 1) {
                const uint32_t c = p + step;
                const uint32_t ex = __shfl_sync(0xffffffffu, excl, c & 31u);
                if (c < nb && ex <= t) p = c;
            }
            const uint32_t k = t - __shfl_sync(0xffffffffu, excl, p);
            const uint32_t pbest = __shfl_sync(0xffffffffu, best, p);
            uint32_t rlo[MAXSRC], rhi[MAXSRC];
#pragma unroll
            for (int q = 0; q < MAXSRC; ++q) {
                rlo[q] = __shfl_sync(0xffffffffu, mlo[q], p);
                rhi[q] = __shfl_sync(0xffffffffu, mhi[q], p);
            }
            uint32_t v = 0, kpos = 0;
#pragma unroll
            for (int q = 0; q < MAXSRC; ++q)
                if (q == (int)pbest && active) {
                    kpos = rlo[q] + k;
                    v = src_list(P, L, q)[kpos];
                }
            uint32_t nlo[MAXOPEN] = {0, 0, 0, 0}, nhi[MAXOPEN] = {0, 0, 0, 0};
            const bool ok = probe<L>(P, (int)pbest, rlo, rhi, kpos, v, active, nlo, nhi);
            if constexpr (L == NL - 1)
                finish_round<L, NL, MAT>(P, F, E, A, ok, v, p);
            else
                descend<L, NL, MAT>(P, F, E, A, ok, v, p, nlo, nhi);
        }
    }
}

// Loop 2 (index 1) of one entry, candidates [k0, k1) of its shortest list.
template <int NL, bool MAT>
__device__ __forceinline__ void run_entry(const DPlan& P, Frame& F, const EntryCtx& E, Acc& A, uint32_t k0,
                                          uint32_t k1) {
    const uint32_t lane = lane_id();
    const int ns = P.nsrc[1];
    uint32_t rlo[MAXSRC], rhi[MAXSRC];
    uint32_t best = 0, bestlen = 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < MAXSRC; ++q) {
        rlo[q] = rhi[q] = 0;
        if (q < ns) {
            const int j = P.src_atom[1][q];
            const DAtom& a = P.atom[j];
            if (P.src_top[1][q]) {
#pragma unroll
                for (int jj = 0; jj < HC_MAX_ATOMS; ++jj)
                    if (jj == j) {
                        rlo[q] = E.tlo[jj];
                        rhi[q] = E.thi[jj];
                    }
            } else {
#pragma unroll
                for (int s = 0; s < MAXOPEN; ++s)
                    if (s == a.slot) {
                        rlo[q] = E.r0lo[s];
                        rhi[q] = E.r0hi[s];
                    }
            }
            if (rhi[q] - rlo[q] < bestlen) {
                bestlen = rhi[q] - rlo[q];
                best = q;
            }
        }
    }
    if (A.stats && k0 == 0 && lane == 0) A.work += (uint64_t)ns * bestlen;
    for (uint32_t t0 = k0; t0 < k1; t0 += 32) {
        const uint32_t k = t0 + lane;
        const bool active = k < k1;
        uint32_t v = 0, kpos = 0;
#pragma unroll
        for (int q = 0; q < MAXSRC; ++q)
            if (q == (int)best && active) {
                kpos = rlo[q] + k;
                v = src_list(P, 1, q)[kpos];
            }
        uint32_t nlo[MAXOPEN] = {0, 0, 0, 0}, nhi[MAXOPEN] = {0, 0, 0, 0};
        const bool ok = probe<1>(P, (int)best, rlo, rhi, kpos, v, active, nlo, nhi);
        if constexpr (NL == 2)
            finish_round<1, NL, MAT>(P, F, E, A, ok, v, 0);
        else
            descend<1, NL, MAT>(P, F, E, A, ok, v, 0, nlo, nhi);
    }
}

// Persistent search kernel.  Work item i covers loop-2 candidates
// [i*grain, (i+1)*grain) of the concatenation of all entries' candidates.
// pass 0 counts (and, with item_counts, records each item's count); pass 1
// writes tuples at item_base[item].
template <int NL, bool MAT>
__global__ void __launch_bounds__(256) gj_kernel(const DPlan* __restrict__ gP, const uint32_t* __restrict__ e_cell,
                                                 const uint32_t* __restrict__ e_x, const uint32_t* __restrict__ e_rng,
                                                 const uint64_t* __restrict__ uoff, uint32_t grain, JoinCtl* ctl,
                                                 int pass, uint64_t* __restrict__ cell_counts,
                                                 uint64_t* __restrict__ item_counts,
                                                 const uint64_t* __restrict__ item_base, uint32_t* __restrict__ out,
                                                 int stats) {
    __shared__ DPlan P;
    load_plan(P, gP);
    const uint32_t lane = lane_id();
    const uint32_t E_n = ctl->n_entries;
    const uint64_t U = uoff[E_n];
    const uint64_t nitems = (U + grain - 1) / grain;
    Frame F;
    Acc A;
    A.count = 0;
    A.work = 0;
    A.out_pos = 0;
    A.out = out;
    A.stats = stats && pass == 0;
    uint64_t total = 0;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&ctl->item_ctr[pass], 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        uint64_t u0 = (uint64_t)item * grain;
        const uint64_t u1 = min(U, u0 + grain);
        uint32_t lo = 0, hi = E_n;  // last entry e with uoff[e] <= u0
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (uoff[mid] <= u0)
                lo = mid;
            else
                hi = mid;
        }
        uint32_t e = lo;
        A.out_pos = MAT ? item_base[item] : 0;
        uint64_t item_count = 0;
        while (u0 < u1 && e < E_n) {
            const uint64_t eb = uoff[e], ee = uoff[e + 1];
            if (ee <= u0) {
                ++e;
                continue;
            }
            const uint32_t k0 = (uint32_t)(u0 - eb);
            const uint32_t k1 = (uint32_t)(min(u1, ee) - eb);
            EntryCtx E;
            E.cell = e_cell[e];
            E.x = e_x[e];
#pragma unroll
            for (int s = 0; s < MAXOPEN; ++s) {
                E.r0lo[s] = e_rng[(uint64_t)e * (2 * MAXOPEN) + 2 * s];
                E.r0hi[s] = e_rng[(uint64_t)e * (2 * MAXOPEN) + 2 * s + 1];
            }
#pragma unroll
            for (int j = 0; j < HC_MAX_ATOMS; ++j) {
                E.tlo[j] = E.thi[j] = 0;
                if (j < P.natoms && P.atom[j].lev_first >= 1) top_range(P.atom[j], E.cell, E.tlo[j], E.thi[j]);
            }
            const uint64_t before = A.count;
            run_entry<NL, MAT>(P, F, E, A, k0, k1);
            const uint64_t got = A.count - before;
            if (pass == 0 && cell_counts && got && lane == 0)
                atomicAdd((unsigned long long*)&cell_counts[E.cell], (unsigned long long)got);
            item_count += got;
            u0 = eb + k1;
            ++e;
        }
        if (pass == 0 && item_counts && lane == 0) item_counts[item] = item_count;
        total += item_count;
    }
    if (pass == 0 && lane == 0 && total) atomicAdd((unsigned long long*)&ctl->total, (unsigned long long)total);
    if (A.stats) {
        const uint64_t w = warp_sum64(A.work);
        if (lane == 0 && w) atomicAdd((unsigned long long*)&ctl->work, (unsigned long long)w);
    }
}

// A query with one loop per variable has at least two loops; NL = 2..5 are
// instantiated.
template <int NL>
int gj_grid(bool mat, int threads) {
    const void* kern = mat ? (const void*)gj_kernel<NL, true> : (const void*)gj_kernel<NL, false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms();
}

struct GjArgs {
    const DPlan* plan;
    const uint32_t *e_cell, *e_x, *e_rng;
    const uint64_t* uoff;
    uint32_t grain;
    JoinCtl* ctl;
    int pass;
    uint64_t* cell_counts;
    uint64_t* item_counts;
    const uint64_t* item_base;
    uint32_t* out;
    int stats;
    int threads;
};

template <int NL>
hc_status launch_gj(bool mat, const GjArgs& g, cudaStream_t s) {
    const int grid = gj_grid<NL>(mat, g.threads);
    if (mat)
        gj_kernel<NL, true><<<grid, g.threads, 0, s>>>(g.plan, g.e_cell, g.e_x, g.e_rng, g.uoff, g.grain, g.ctl, g.pass,
                                                       g.cell_counts, g.item_counts, g.item_base, g.out, g.stats);
    else
        gj_kernel<NL, false><<<grid, g.threads, 0, s>>>(g.plan, g.e_cell, g.e_x, g.e_rng, g.uoff, g.grain, g.ctl,
                                                        g.pass, g.cell_counts, g.item_counts, g.item_base, g.out,
                                                        g.stats);
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

hc_status launch_any(int nl, bool mat, const GjArgs& g, cudaStream_t s) {
    switch (nl) {
        case 2: return launch_gj<2>(mat, g, s);
        case 3: return launch_gj<3>(mat, g, s);
        case 4: return launch_gj<4>(mat, g, s);
        case 5: return launch_gj<5>(mat, g, s);
        default: return fail(HC_ERR_CAPACITY, "run_join: queries of 2 to 5 variables are built in");
    }
}

}  // namespace hc

// ------------------------------------------------------------------ host
struct hc_result {
    cudaStream_t stream = nullptr;
    uint32_t n_vars = 0;
    uint64_t n_cells = 0;
    hc::JoinCtl* d_ctl = nullptr;
    uint64_t* d_cell_counts = nullptr;
    uint32_t* d_tuples = nullptr;
    uint64_t n_tuples = 0;
    uint64_t n_items = 0;
    bool materialized = false;
    bool done = false;
    hc::JoinCtl h_ctl{};
    std::vector<hc_partitioned*> parts;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int n_timed = 0;  // search launches bracketed by ev[2i], ev[2i+1]
};

namespace hc {

namespace {

struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* p : ptrs) dev_free(p, s);
    }
    template <typename T>
    hc_status get(T** p, size_t count) {
        void* v = nullptr;
        HC_TRY(dev_alloc(&v, std::max<size_t>(count, 1) * sizeof(T), s));
        ptrs.push_back(v);
        *p = (T*)v;
        return HC_OK;
    }
};

hc_status read_ctl(hc_result* R) {
    HC_CUDA_TRY(cudaMemcpyAsync(&R->h_ctl, R->d_ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, R->stream));
    HC_CUDA_TRY(cudaStreamSynchronize(R->stream));
    if (R->h_ctl.err & DEV_ERR_TIMEOUT) return fail(HC_ERR_TIMEOUT, "run_join: a bounded device wait gave up");
    return HC_OK;
}

}  // namespace

void result_release(hc_result* r) {
    if (!r) return;
    cudaStream_t s = r->stream;
    for (auto* p : r->parts) partitioned_release(p, s);
    dev_free(r->d_ctl, s);
    dev_free(r->d_cell_counts, s);
    dev_free(r->d_tuples, s);
    for (auto& e : r->ev)
        if (e) cudaEventDestroy(e);
    delete r;
}

hc_status result_get(hc_result* R, hc_result_view* v) {
    if (!R || !v) return fail(HC_ERR_ARG, "result_get: NULL argument");
    if (!R->done) {
        HC_TRY(read_ctl(R));
        R->done = true;
    }
    memset(v, 0, sizeof(*v));
    v->count = R->h_ctl.total;
    v->n_tuples = R->materialized ? R->n_tuples : 0;
    v->d_tuples = R->materialized ? R->d_tuples : nullptr;
    v->n_cells = R->n_cells;
    v->d_cell_counts = R->d_cell_counts;
    v->work = R->h_ctl.work;
    v->n_items = R->n_items;
    v->n_join_launches = R->materialized ? 2 : 1;
    float total_ms = 0.f;
    for (int i = 0; i < R->n_timed; ++i) {
        float ms = 0.f;
        HC_CUDA_TRY(cudaEventElapsedTime(&ms, R->ev[2 * i], R->ev[2 * i + 1]));
        total_ms += ms;
    }
    v->ms_join_kernel = total_ms;
    return HC_OK;
}

hc_status run_join_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm, cudaStream_t s,
                        hc_result** out) {
    if (!out) return fail(HC_ERR_ARG, "run_join: out is NULL");
    *out = nullptr;
    if (!q || !idx || !prm) return fail(HC_ERR_ARG, "run_join: NULL argument");
    const int nv = (int)q->n_vars, na = (int)q->n_atoms;
    if (nv < 2 || nv > HC_MAX_VARS || na < 1 || na > HC_MAX_ATOMS)
        return fail(HC_ERR_ARG, "run_join: need 2..8 variables and 1..8 atoms");
    if (nv > 5) return fail(HC_ERR_CAPACITY, "run_join: queries of 2 to 5 variables are built in");
    if (prm->mode > HC_MODE_MATERIALIZE) return fail(HC_ERR_ARG, "run_join: unknown mode");
    int rank[HC_MAX_VARS];
    bool seen[HC_MAX_VARS] = {false};
    for (int i = 0; i < nv; ++i) {
        const int v = q->order[i];
        if (v >= nv || seen[v]) return fail(HC_ERR_ARG, "run_join: order must list every variable once");
        seen[v] = true;
        rank[v] = i;
    }
    bool covered[HC_MAX_VARS] = {false};
    for (int j = 0; j < na; ++j) {
        const int a = q->atoms[j].var0, b = q->atoms[j].var1;
        if (a >= nv || b >= nv || a == b) return fail(HC_ERR_ARG, "run_join: atom variables out of range or equal");
        if (!idx[j]) return fail(HC_ERR_ARG, "run_join: missing index for an atom");
        if (idx[j]->stats_only) return fail(HC_ERR_ARG, "run_join: a statistics-only index has no data");
        covered[a] = covered[b] = true;
    }
    for (int v = 0; v < nv; ++v)
        if (!covered[v]) return fail(HC_ERR_ARG, "run_join: a variable occurs in no atom");
    uint64_t ncells = 1;
    for (int v = 0; v < nv; ++v) {
        if (prm->shares[v] < 1) return fail(HC_ERR_ARG, "run_join: shares must be >= 1");
        ncells *= prm->shares[v];
        if (ncells > (1ull << 24)) return fail(HC_ERR_CAPACITY, "run_join: more than 2^24 cells");
    }
    uint64_t stride[HC_MAX_VARS];
    {
        uint64_t st = 1;
        for (int v = nv - 1; v >= 0; --v) {
            stride[v] = st;
            st *= prm->shares[v];
        }
    }
    const uint32_t grain = prm->item_grain ? prm->item_grain : 64;
    const int threads = prm->block_threads ? (int)prm->block_threads : 128;
    if (threads % 32 != 0 || threads < 32 || threads > 256)
        return fail(HC_ERR_ARG, "run_join: block_threads must be a multiple of 32 in [32, 256]");

    hc_result* R = new hc_result();
    R->stream = s;
    R->n_vars = nv;
    R->n_cells = ncells;
    auto bail = [&](hc_status st) {
        result_release(R);
        return st;
    };

    DPlan P;
    memset(&P, 0, sizeof(P));
    P.nlev = nv;
    P.natoms = na;
    P.nv = nv;
    P.ncells = (uint32_t)ncells;
    for (int i = 0; i < nv; ++i) P.var_of_level[i] = q->order[i];
    for (int j = 0; j < na; ++j) {
        const hc_index* ix = idx[j];
        const int a = q->atoms[j].var0, b = q->atoms[j].var1;
        const int first = rank[a] < rank[b] ? a : b, second = first == a ? b : a;
        const uint32_t need_ao = rank[a] < rank[b] ? 0u : 1u;
        if (ix->attr_order != need_ao)
            return bail(fail(HC_ERR_ARG, "run_join: an index's attr_order does not sort its atom in loop order"));
        DAtom& d = P.atom[j];
        const uint32_t pa = prm->shares[first], pb = prm->shares[second];
        d.pb = pb;
        d.stride_f = (uint32_t)stride[first];
        d.share_f = pa;
        d.stride_s = (uint32_t)stride[second];
        d.share_s = pb;
        d.lev_first = rank[first];
        d.lev_second = rank[second];
        if ((uint64_t)pa * pb == 1) {
            d.v1 = ix->d_v1;
            d.o1 = ix->d_o1;
            d.v2 = ix->d_v2;
            d.l1s = nullptr;
            d.l1_whole = (uint32_t)ix->l1;
        } else {
            hc_partitioned* part = nullptr;
            const hc_status st = partition_impl(ix, prm->seeds[first], pa, prm->seeds[second], pb, s, &part);
            if (st != HC_OK) return bail(st);
            R->parts.push_back(part);
            d.v1 = part->d_v1;
            d.o1 = part->d_o1;
            d.v2 = part->d_v2;
            d.l1s = part->d_lvl1_start;
        }
    }
    for (int L = 0; L < nv; ++L) {
        for (int j = 0; j < na; ++j) {
            if (P.atom[j].lev_first == L) {
                if (P.nopen[L] >= MAXOPEN || P.nsrc[L] >= MAXSRC)
                    return bail(fail(HC_ERR_CAPACITY, "run_join: a loop intersects more than 4 lists"));
                P.atom[j].slot = P.nopen[L]++;
                P.src_atom[L][P.nsrc[L]] = j;
                P.src_top[L][P.nsrc[L]] = 1;
                P.nsrc[L]++;
            }
        }
        for (int j = 0; j < na; ++j) {
            if (P.atom[j].lev_second == L) {
                if (P.nsrc[L] >= MAXSRC)
                    return bail(fail(HC_ERR_CAPACITY, "run_join: a loop intersects more than 4 lists"));
                P.src_atom[L][P.nsrc[L]] = j;
                P.src_top[L][P.nsrc[L]] = 0;
                P.nsrc[L]++;
            }
        }
    }
    // loop-1 candidates are bounded by any loop-1 atom's rows times the
    // number of cells that read each of its partitions
    uint64_t cand_bound = UINT64_MAX;
    for (int q0 = 0; q0 < P.nsrc[0]; ++q0) {
        const int j = P.src_atom[0][q0];
        const DAtom& d = P.atom[j];
        const uint64_t rep = ncells / ((uint64_t)d.share_f * d.share_s);
        const uint64_t rows = d.l1s ? idx[j]->n : idx[j]->l1;
        cand_bound = std::min<uint64_t>(cand_bound, rep * rows);
    }
    cand_bound = std::max<uint64_t>(cand_bound, 1);
    if (cand_bound >= 0xFFFFFFFFull) return bail(fail(HC_ERR_CAPACITY, "run_join: too many loop-1 candidates"));

    {
        void* p;
        if (dev_alloc(&p, sizeof(JoinCtl), s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_ctl = (JoinCtl*)p;
    }
    JoinCtl* ctl = R->d_ctl;
    if (cudaMemsetAsync(ctl, 0, sizeof(JoinCtl), s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    const int stats = (prm->flags & HC_FLAG_STATS) ? 1 : 0;
    if (prm->flags & HC_FLAG_CELL_COUNTS) {
        void* p;
        if (dev_alloc(&p, ncells * 8, s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_cell_counts = (uint64_t*)p;
        if (cudaMemsetAsync(p, 0, ncells * 8, s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    }

    Scratch tmp(s);
    DPlan* d_plan;
    uint32_t *cand, *flags, *e_cell, *e_x, *e_rng, *e_units;
    uint64_t *candoff, *flagoff, *uoff;
    hc_status st;
    if ((st = tmp.get(&d_plan, 1)) != HC_OK) return bail(st);
    if (cudaMemcpyAsync(d_plan, &P, sizeof(DPlan), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "plan copy"));
    if ((st = tmp.get(&cand, ncells)) != HC_OK) return bail(st);
    if ((st = tmp.get(&candoff, ncells + 1)) != HC_OK) return bail(st);
    if ((st = tmp.get(&flags, cand_bound)) != HC_OK) return bail(st);
    if ((st = tmp.get(&flagoff, cand_bound + 1)) != HC_OK) return bail(st);
    if ((st = tmp.get(&e_cell, cand_bound)) != HC_OK) return bail(st);
    if ((st = tmp.get(&e_x, cand_bound)) != HC_OK) return bail(st);
    if ((st = tmp.get(&e_rng, cand_bound * 2 * MAXOPEN)) != HC_OK) return bail(st);
    if ((st = tmp.get(&e_units, cand_bound)) != HC_OK) return bail(st);
    if ((st = tmp.get(&uoff, cand_bound + 1)) != HC_OK) return bail(st);

    const int tpb = 256;
    l0_count_kernel<<<(unsigned)std::min<uint64_t>((ncells + tpb - 1) / tpb, 4096), tpb, 0, s>>>(d_plan, cand, ctl,
                                                                                                 stats);
    if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "l0_count_kernel"));
    if ((st = exclusive_scan_u32_to_u64(cand, candoff, ncells, nullptr, &ctl->err, s)) != HC_OK) return bail(st);
    const unsigned pgrid =
        (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((cand_bound + tpb - 1) / tpb, (uint64_t)num_sms() * 16));
    l0_probe_kernel<false><<<pgrid, tpb, 0, s>>>(d_plan, candoff, cand_bound, flags, nullptr, nullptr, nullptr, nullptr,
                                                 nullptr);
    if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "l0_probe_kernel"));
    if ((st = exclusive_scan_u32_to_u64(flags, flagoff, cand_bound, nullptr, &ctl->err, s)) != HC_OK) return bail(st);
    l0_probe_kernel<true><<<pgrid, tpb, 0, s>>>(d_plan, candoff, cand_bound, flags, flagoff, e_cell, e_x, e_rng, e_units);
    if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "l0_probe_kernel"));
    entries_total_kernel<<<1, 1, 0, s>>>(flagoff, candoff, (uint32_t)ncells, cand_bound, ctl);
    if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "entries_total_kernel"));
    if ((st = exclusive_scan_u32_to_u64(e_units, uoff, cand_bound, &ctl->n_entries, &ctl->err, s)) != HC_OK)
        return bail(st);

    GjArgs g{d_plan, e_cell, e_x, e_rng, uoff, grain, ctl, 0, R->d_cell_counts, nullptr, nullptr, nullptr, stats, threads};
    const bool timed = (prm->flags & HC_FLAG_TIME_KERNELS) != 0;
    if (timed)
        for (auto& e : R->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    // one search launch, bracketed by events when timed
    auto search = [&](bool mat) -> hc_status {
        if (timed && cudaEventRecord(R->ev[2 * R->n_timed], s) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
        HC_TRY(launch_any(nv, mat, g, s));
        if (timed) {
            if (cudaEventRecord(R->ev[2 * R->n_timed + 1], s) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
            R->n_timed++;
        }
        return HC_OK;
    };
    if (prm->mode == HC_MODE_COUNT) {
        if ((st = search(false)) != HC_OK) return bail(st);
        *out = R;
        return HC_OK;
    }
    // materialize: count each item, place items by a scan, then write
    if ((st = read_ctl(R)) != HC_OK) return bail(st);
    uint64_t hU = 0;
    if (cudaMemcpyAsync(&hU, uoff + R->h_ctl.n_entries, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "read units"));
    const uint64_t nitems = (hU + grain - 1) / grain;
    R->n_items = nitems;
    uint64_t *item_counts, *item_base;
    if ((st = tmp.get(&item_counts, nitems)) != HC_OK) return bail(st);
    if ((st = tmp.get(&item_base, nitems + 1)) != HC_OK) return bail(st);
    g.item_counts = item_counts;
    if ((st = search(false)) != HC_OK) return bail(st);
    if ((st = exclusive_scan_u64(item_counts, item_base, nitems, nullptr, &ctl->err, s)) != HC_OK) return bail(st);
    uint64_t total = 0;
    if (cudaMemcpyAsync(&total, item_base + nitems, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "read total"));
    {
        void* p;
        if (dev_alloc(&p, std::max<uint64_t>(total, 1) * nv * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_tuples = (uint32_t*)p;
    }
    g.pass = 1;
    g.item_counts = nullptr;
    g.item_base = item_base;
    g.out = R->d_tuples;
    g.cell_counts = nullptr;
    if ((st = search(true)) != HC_OK) return bail(st);
    R->n_tuples = total;
    R->materialized = true;
    *out = R;
    return HC_OK;
}

}  // namespace hc
