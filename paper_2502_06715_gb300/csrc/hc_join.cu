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
#include <type_traits>
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
    const uint32_t* l1s;    // level-1 start of each partition, [np + 1]; NULL when whole
    const uint32_t* v1pos;  // value -> position in v1 (V1POS_NONE if absent), or NULL
    uint32_t v1pos_n;       // values covered by v1pos
    const uint4* g1;        // bucket directory of v1's top-level runs, or NULL
    const uint4* g2;        // bucket directory of v2's runs, or NULL
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
    // per loop and source: 1 when the list depends only on the loop-1
    // binding (a top-level list, or the sub-list of an atom loop 1 opens);
    // otherwise the loop f that opens the atom and its slot there
    int src_ec[HC_MAX_VARS][MAXSRC];
    int src_f[HC_MAX_VARS][MAXSRC];
    int src_slot[HC_MAX_VARS][MAXSRC];
    // last loop: a parent whose two lists are both >= merge_min long and
    // within merge_ratio of each other takes the block-merge path; of the
    // others, one whose shorter list has >= pair_min values is searched by
    // the whole warp (probe_pair); the rest are flattened over the lanes
    uint32_t merge_min, merge_ratio, pair_min;
    // searches of runs at least dir_min long go through their bucket
    // directory (0xFFFFFFFF: never)
    uint32_t dir_min;
    // queries of 4+ loops: an entry whose loop-3 lists (those fixed by the
    // entry) exceed slice_grain is cut into slices of about that many loop-3
    // candidates per loop-2 candidate (0: no slicing)
    uint32_t slice_grain;
    // query rewriting (Sec. 5.1): the sources of the last loop that do not
    // depend on the binding of the loop before it (bit q of far_mask) are
    // intersected once per binding of loop nlev-3, into the warp's arena of
    // arena_words words; the last loop reads that list in place of source
    // far0 and skips the other far sources.  lift = 0: off.
    int lift, far0;
    uint32_t far_mask, arena_words;
};

constexpr uint32_t LIFT_ARENA_WORDS = 16384;  // per warp, by default

// Single-pass materialize: each warp writes its tuples into chunks of
// OUT_CHUNK tuples taken from an output pool with one atomic per chunk.
constexpr uint32_t OUT_CHUNK = 2048;
constexpr uint32_t NO_CHUNK = 0xFFFFFFFFu;
// Materializing search: the last loop's per-binding path stages its matches
// (the last variable's values) in a per-warp shared-memory buffer of OBUF
// values and writes them out 32 tuples at a time.
constexpr uint32_t OBUF = 256;

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
__global__ void l0_count_kernel(const DPlan* __restrict__ gP, uint32_t* __restrict__ cand, JoinCtl* ctl, int stats,
                                uint64_t* __restrict__ cprof) {
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
        if (cprof) cprof[2 * (uint64_t)c] += (uint64_t)P.nsrc[0] * m;  // one thread per cell; zeroed before
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
// Nothing runs once the join's error word is set (a scan before it gave up
// a wait, so its offsets are not valid).
template <bool WRITE>
__global__ void l0_probe_kernel(const DPlan* __restrict__ gP, const uint64_t* __restrict__ candoff, uint64_t tmax,
                                uint32_t* __restrict__ flags, const uint64_t* __restrict__ flagoff,
                                uint32_t* __restrict__ e_cell, uint32_t* __restrict__ e_x,
                                uint32_t* __restrict__ e_rng, uint64_t* __restrict__ e_units,
                                uint32_t* __restrict__ e_split, const JoinCtl* __restrict__ ctl) {
    __shared__ DPlan P;
    load_plan(P, gP);
    if (dev_err_set(&ctl->err)) return;
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
                uint32_t p;
                if (q == (int)best) {
                    p = rlo[q] + k;
                } else if (a.v1pos != nullptr) {  // direct position of x in V1
                    p = x < a.v1pos_n ? a.v1pos[x] : V1POS_NONE;
                    ok = ok && p >= rlo[q] && p < rhi[q];
                } else {
                    ok = dir_find(a.v1, a.g1, rlo[q], rhi[q], x, P.dir_min, p) && ok;
                }
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
        // work units of the entry: loop-2 candidates, each cut into slices of
        // its loop-3 candidates when the entry fixes a long loop-3 list
        uint32_t split = 1;
        if (P.nlev >= 4 && P.slice_grain > 0) {
            uint32_t w = 0xFFFFFFFFu;
            for (int q = 0; q < P.nsrc[2]; ++q) {
                const DAtom& a = P.atom[P.src_atom[2][q]];
                uint32_t len = 0xFFFFFFFFu;
                if (P.src_top[2][q]) {
                    uint32_t l0, l1;
                    top_range(a, c, l0, l1);
                    len = l1 - l0;
                } else if (a.lev_first == 0) {
#pragma unroll
                    for (int s = 0; s < MAXOPEN; ++s)
                        if (s == a.slot) len = rhi[s] - rlo[s];
                }
                w = min(w, len);
            }
            if (w != 0xFFFFFFFFu) split = max(1u, (w + P.slice_grain - 1) / P.slice_grain);
        }
        e_units[e] = (uint64_t)m * split;
        e_split[e] = split;
    }
}

__global__ void entries_total_kernel(const uint64_t* __restrict__ flagoff, const uint64_t* __restrict__ candoff,
                                     uint32_t ncells, uint64_t tmax, JoinCtl* ctl) {
    const uint64_t T = min(tmax, candoff[ncells]);
    ctl->n_entries = (uint32_t)flagoff[T];
}

// ---------------------------------------------------------- search loops
// Shapes are compiled per (NL loops, S lists per loop, O atoms opened per
// loop) so that per-lane state stays in registers.

// The loop-1 binding a work item is under (lane-uniform): the value, its
// cell, and for every later loop the ranges of its lists that depend only on
// this binding (top-level lists of the cell's partitions, and sub-lists of
// atoms opened by loop 1).
template <int NL, int S>
struct Entry {
    uint32_t cell, x;
    uint32_t (*lo)[S];  // [NL][S] in the warp's shared memory (lane-uniform)
    uint32_t (*hi)[S];
    uint32_t k0, k1;      // the work item's subrange of loop 1's shortest list
    uint32_t best1, len1;  // that list (source index) and its full length
    uint32_t j0, j1, ns;   // slices [j0, j1) of ns of the loop-2 binding's loop-3 candidates
};

// Batch bindings of loops 1..NL-2 (index = loop), one per lane.
template <int NL, int O>
struct Frame {
    uint32_t val[NL];
    uint32_t par[NL];
    uint32_t olo[NL][O];
    uint32_t ohi[NL][O];
    // lifted list of the loop nlev-3 binding held by this lane: arena[tlo, thi)
    uint32_t tlo, thi;
    bool lifted;  // the current batch's lifted lists fit the arena (lane-uniform)
};

struct Acc {
    uint64_t count;    // matches at the last loop (lane-uniform)
    uint64_t work;     // per-lane work counter
    uint64_t out_pos;  // next output slot (two-pass materialize)
    uint32_t* out;
    int stats;
    // single-pass materialize (pool != 0): the warp's current chunk and fill
    int pool;
    uint32_t chunk, fill, n_chunks;
    uint32_t* chunk_fill;
    JoinCtl* ctl;
    uint32_t* arena;  // the warp's arena for lifted lists (query rewriting), or NULL
    uint32_t* obuf;   // the warp's staging buffer of OBUF values (materialize), or NULL
    uint64_t* cprof;  // per-cell profile [cells][2] (work units, SM cycles), or NULL
};

// Output slot of the lane holding rank r among the k = popc(ball) matches
// of this round (all lanes call).  Two-pass mode: consecutive slots from
// out_pos.  Pool mode: the rest of the warp's chunk, then a new chunk; a slot
// of ~0 means the pool is exhausted and the tuple is not written.
__device__ __forceinline__ uint64_t out_reserve(Acc& A, uint32_t ball) {
    const uint32_t r = __popc(ball & lanemask_lt());
    const uint32_t k = __popc(ball);
    if (!A.pool) {
        const uint64_t slot = A.out_pos + r;
        A.out_pos += k;
        return slot;
    }
    if (k == 0) return ~0ull;
    const uint32_t room = OUT_CHUNK - A.fill;
    uint64_t slot;
    if (k <= room) {
        slot = A.chunk == NO_CHUNK ? ~0ull : (uint64_t)A.chunk * OUT_CHUNK + A.fill + r;
        A.fill += k;
        return slot;
    }
    uint32_t nc = 0;
    if (lane_id() == 0) {
        if (A.chunk != NO_CHUNK) A.chunk_fill[A.chunk] = OUT_CHUNK;
        nc = atomicAdd(&A.ctl->chunk_ctr, 1u);
        if (nc >= A.n_chunks) atomicOr(&A.ctl->overflow, 1u);
    }
    nc = __shfl_sync(0xffffffffu, nc, 0);
    if (nc >= A.n_chunks) nc = NO_CHUNK;
    if (r < room)
        slot = A.chunk == NO_CHUNK ? ~0ull : (uint64_t)A.chunk * OUT_CHUNK + A.fill + r;
    else
        slot = nc == NO_CHUNK ? ~0ull : (uint64_t)nc * OUT_CHUNK + (r - room);
    A.chunk = nc;
    A.fill = k - room;
    return slot;
}

// Reserve n <= OUT_CHUNK consecutive output slots for the warp (all lanes
// call, n lane-uniform).  Tuple t of the n goes to slot s0 + t when t < room,
// else to s1 + (t - room); a base of ~0 means the pool is exhausted and those
// tuples are not written (the overflow flag makes the join rerun them).
__device__ __forceinline__ void out_reserve_n(Acc& A, uint32_t n, uint64_t& s0, uint32_t& room, uint64_t& s1) {
    s1 = ~0ull;
    if (!A.pool) {
        s0 = A.out_pos;
        room = n;
        A.out_pos += n;
        return;
    }
    room = OUT_CHUNK - A.fill;
    s0 = A.chunk == NO_CHUNK ? ~0ull : (uint64_t)A.chunk * OUT_CHUNK + A.fill;
    if (n <= room) {
        room = n;
        A.fill += n;
        return;
    }
    uint32_t nc = 0;
    if (lane_id() == 0) {
        if (A.chunk != NO_CHUNK) A.chunk_fill[A.chunk] = OUT_CHUNK;
        nc = atomicAdd(&A.ctl->chunk_ctr, 1u);
        if (nc >= A.n_chunks) atomicOr(&A.ctl->overflow, 1u);
    }
    nc = __shfl_sync(0xffffffffu, nc, 0);
    if (nc >= A.n_chunks) nc = NO_CHUNK;
    s1 = nc == NO_CHUNK ? ~0ull : (uint64_t)nc * OUT_CHUNK;
    A.chunk = nc;
    A.fill = n - room;
}

// Position of the r-th (0-based) set bit of m (r < popc(m)).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t w = 16; w >= 1; w >>= 1) {
        const uint32_t c = __popc(m & ((1u << (pos + w)) - 1u));  // set bits below pos + w
        if (c <= r) pos += w;
    }
    return pos;
}

// Range of source q of loop L for the binding of loop L-1 held by lane
// `lane_of` (all lanes call together: ranges of atoms opened by loops >= 1
// are fetched from the holder of the opening binding by shuffles).
template <int L, int NL, int S, int O>
__device__ __forceinline__ void src_range(const DPlan& P, const Frame<NL, O>& F, const Entry<NL, S>& E, int q,
                                          uint32_t lane_of, uint32_t& lo, uint32_t& hi) {
    if (P.src_ec[L][q]) {
        lo = E.lo[L][q];
        hi = E.hi[L][q];
        return;
    }
    const int f = P.src_f[L][q], s = P.src_slot[L][q];
    uint32_t anc = lane_of;  // ancestor at loop f of the loop L-1 binding
#pragma unroll
    for (int g = L - 1; g >= 1; --g)
        if (g > f) anc = __shfl_sync(0xffffffffu, F.par[g], anc);
    uint32_t mylo = 0, myhi = 0;
#pragma unroll
    for (int g = 1; g < L; ++g)
#pragma unroll
        for (int ss = 0; ss < O; ++ss)
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

// The list of source q of loop L, where source lift_q reads the arena.
__device__ __forceinline__ const uint32_t* src_list_l(const DPlan& P, const Acc& A, int L, int q, int lift_q) {
    return q == lift_q ? A.arena : src_list(P, L, q);
}

// Search candidate v (element kpos of source `best`) in the other lists of
// loop L ("search(V, x)", Sec. 5: first position >= x, by binary search).  A
// top-level list holding v opens its atom: the o1 range at v's position is
// the atom's sub-list for later loops (Sec. 5 level restriction).
template <int L, int S, int O>
__device__ __forceinline__ bool probe(const DPlan& P, int best, const uint32_t (&rlo)[S], const uint32_t (&rhi)[S],
                                      uint32_t kpos, uint32_t v, bool active, uint32_t (&nlo)[O],
                                      uint32_t (&nhi)[O], uint32_t use = 0xFFFFFFFFu,
                                      const uint32_t* lift_list = nullptr, int lift_q = -1) {
    bool ok = active;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        if (q < P.nsrc[L] && ((use >> q) & 1u)) {
            const uint32_t* list = q == lift_q ? lift_list : src_list(P, L, q);
            const DAtom& aq = P.atom[P.src_atom[L][q]];
            uint32_t p = kpos;
            if (q != best) {
                if (q != lift_q && P.src_top[L][q] && aq.v1pos != nullptr) {  // direct position of v in V1
                    p = (ok && v < aq.v1pos_n) ? __ldg(aq.v1pos + v) : V1POS_NONE;
                    ok = ok && p >= rlo[q] && p < rhi[q];
                } else if (q == lift_q) {  // the arena, written by this kernel: coherent loads
                    uint32_t* al = const_cast<uint32_t*>(list);
                    ok = ok && rhi[q] > rlo[q] && find_u32(al, rlo[q], rhi[q], v, p);
                } else {
                    ok = ok && dir_find(list, P.src_top[L][q] ? aq.g1 : aq.g2, rlo[q], rhi[q], v, P.dir_min, p);
                }
            }
            if (q < O && q != lift_q && P.src_top[L][q] && ok) {  // top sources come first, slot == q
                const DAtom& a = P.atom[P.src_atom[L][q]];
                nlo[q] = a.o1[p];
                nhi[q] = a.o1[p + 1];
            }
        }
    }
    return ok;
}

// Range of source q of loop L for the loop L-2 binding held by lane
// `lane_of` (all lanes call together): the source is fixed by the entry or
// opened by loop L-2 or an earlier loop.
template <int L, int NL, int S, int O>
__device__ __forceinline__ void far_range(const DPlan& P, const Frame<NL, O>& F, const Entry<NL, S>& E, int q,
                                          uint32_t lane_of, uint32_t& lo, uint32_t& hi) {
    if (P.src_ec[L][q]) {
        lo = E.lo[L][q];
        hi = E.hi[L][q];
        return;
    }
    const int f = P.src_f[L][q], s = P.src_slot[L][q];
    uint32_t anc = lane_of;  // ancestor at loop f of the loop L-2 binding
#pragma unroll
    for (int g = L - 2; g >= 1; --g)
        if (g > f) anc = __shfl_sync(0xffffffffu, F.par[g], anc);
    uint32_t mylo = 0, myhi = 0;
#pragma unroll
    for (int g = 1; g <= L - 2; ++g)
#pragma unroll
        for (int ss = 0; ss < O; ++ss)
            if (g == f && ss == s) {
                mylo = F.olo[g][ss];
                myhi = F.ohi[g][ss];
            }
    lo = __shfl_sync(0xffffffffu, mylo, anc);
    hi = __shfl_sync(0xffffffffu, myhi, anc);
}

// Query rewriting (Sec. 5.1), at the start of loop NL-2: for each parent (a
// loop NL-3 binding, lanes < nb) intersect the last loop's far sources once
// and store the result, sorted, in the warp's arena at [F.tlo, F.thi) of the
// parent's lane.  The parents' candidates are flattened over the lanes as in
// run_level; a round's matches of one parent occupy consecutive lanes and are
// written in lane order after those of earlier rounds.  Returns false (and
// writes nothing) when the parents' lists could exceed the arena.
template <int NL, int S, int O>
__device__ __forceinline__ bool lift_compute(const DPlan& P, Frame<NL, O>& F, const Entry<NL, S>& E, const Acc& A,
                                             uint32_t nb) {
    constexpr int L = NL - 1;
    const uint32_t lane = lane_id();
    const int ns = P.nsrc[L];
    uint32_t flo[S], fhi[S];
    uint32_t best = 0, bestlen = 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        flo[q] = fhi[q] = 0;
        if (q < ns && ((P.far_mask >> q) & 1u)) {
            far_range<L, NL, S, O>(P, F, E, q, lane < nb ? lane : 0, flo[q], fhi[q]);
            const uint32_t len = fhi[q] - flo[q];
            if (len < bestlen) {
                bestlen = len;
                best = q;
            }
        }
    }
    const uint32_t cnt = lane < nb ? bestlen : 0;  // candidates, and a bound on the parent's list
    // each bound fits the arena (arena_words <= 2^26), so their sum cannot wrap
    if (__any_sync(0xffffffffu, cnt > P.arena_words)) return false;
    const uint32_t incl = warp_incl_scan(cnt);
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > P.arena_words) return false;
    uint32_t filled = 0;  // entries written for this lane's parent
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + lane;
        const bool active = t < total;
        uint32_t p = 0;  // parent of candidate t: the last lane p < nb with excl_p <= t
        if (nb > 1) {
#pragma unroll
            for (uint32_t step = 16; step >= 1; step >>= 1) {
                const uint32_t c = p + step;
                const uint32_t ex = __shfl_sync(0xffffffffu, excl, c & 31u);
                if (c < nb && ex <= t) p = c;
            }
        }
        const uint32_t pex = __shfl_sync(0xffffffffu, excl, p);
        const uint32_t pbest = __shfl_sync(0xffffffffu, best, p);
        const uint32_t pfill = __shfl_sync(0xffffffffu, filled, p);
        uint32_t rlo[S], rhi[S];
#pragma unroll
        for (int q = 0; q < S; ++q) {
            rlo[q] = __shfl_sync(0xffffffffu, flo[q], p);
            rhi[q] = __shfl_sync(0xffffffffu, fhi[q], p);
        }
        uint32_t v = 0;
#pragma unroll
        for (int q = 0; q < S; ++q)
            if (q == (int)pbest && active) v = src_list(P, L, q)[rlo[q] + (t - pex)];
        bool ok = active;
#pragma unroll
        for (int q = 0; q < S; ++q) {
            if (q < ns && ((P.far_mask >> q) & 1u) && q != (int)pbest) {
                const uint32_t* list = src_list(P, L, q);
                const DAtom& aq = P.atom[P.src_atom[L][q]];
                uint32_t pos;
                ok = ok && dir_find(list, P.src_top[L][q] ? aq.g1 : aq.g2, rlo[q], rhi[q], v, P.dir_min, pos);
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, ok);
        const uint32_t seg = pex > t0 ? pex - t0 : 0u;  // first lane of this round holding the parent
        const uint32_t rank = __popc(ball & lanemask_lt() & ~((1u << seg) - 1u));
        if (ok) A.arena[pex + pfill + rank] = v;
        // a parent's matches in this round: rank + ok of its last lane here
        const uint32_t mine = rank + (ok ? 1u : 0u);
        uint32_t src = lane;
        bool here = false;
        if (lane < nb && cnt > 0 && excl < t0 + 32 && excl + cnt > t0) {
            here = true;
            src = min(excl + cnt, t0 + 32) - 1 - t0;
        }
        const uint32_t got = __shfl_sync(0xffffffffu, mine, src);
        if (here) filled += got;
    }
    __syncwarp();
    F.tlo = excl;
    F.thi = excl + filled;
    return true;
}

// Values bound by loops 1..L-1 for the binding of loop L-1 held by lane
// `parent` (all lanes call together).
template <int L, int NL, int O>
__device__ __forceinline__ void prefix_values(const Frame<NL, O>& F, uint32_t parent, uint32_t (&vals)[NL]) {
    uint32_t anc = parent;
#pragma unroll
    for (int g = L - 1; g >= 1; --g) {
        vals[g] = __shfl_sync(0xffffffffu, F.val[g], anc);
        anc = __shfl_sync(0xffffffffu, F.par[g], anc);
    }
}

template <int L, int NL>
__device__ __forceinline__ void write_tuple(const DPlan& P, uint32_t* o, uint32_t x, const uint32_t (&vals)[NL],
                                            uint32_t v) {
    o[P.var_of_level[L]] = v;
    o[P.var_of_level[0]] = x;
#pragma unroll
    for (int g = L - 1; g >= 1; --g) o[P.var_of_level[g]] = vals[g];
}

template <int L, int NL, int S, int O, bool MAT>
__device__ __forceinline__ void run_level(const DPlan& P, Frame<NL, O>& F, const Entry<NL, S>& E, Acc& A,
                                          uint32_t nb);

// Last loop, flattened path: count the round's matches, or write them.
template <int L, int NL, int S, int O, bool MAT>
__device__ __forceinline__ void finish_round(const DPlan& P, const Frame<NL, O>& F, const Entry<NL, S>& E, Acc& A,
                                             bool ok, uint32_t v, uint32_t parent) {
    const uint32_t ball = __ballot_sync(0xffffffffu, ok);
    if constexpr (MAT) {
        uint32_t vals[NL];
        prefix_values<L, NL, O>(F, parent, vals);
        const uint64_t slot = out_reserve(A, ball);
        if (ok && slot != ~0ull) write_tuple<L, NL>(P, A.out + slot * (uint64_t)P.nv, E.x, vals, v);
    }
    A.count += __popc(ball);
}

// Last loop, merge-path for one parent whose two lists are long and of
// similar length.  The longer list B is cut into 32 equal chunks, one per
// lane; each lane finds the matching range of the shorter list A by two
// binary searches (the A values in [B[j0], B[j1]) ) and walks both ranges as
// a sequential merge, so an equal pair is met by exactly one lane (the lane
// owning its B position).  Count mode walks lanes independently; materialize
// mode steps the lanes together and writes each step's matches in lane order.
// LP is const uint32_t* for index lists (read through the read-only path)
// and uint32_t* when a list is in the arena this kernel writes.
template <int L, int NL, int S, int O, bool MAT, typename LP>
__device__ __forceinline__ void merge_pair(const DPlan& P, const Entry<NL, S>& E, Acc& A, LP la, uint32_t a0,
                                           uint32_t a1, LP lb, uint32_t b0, uint32_t b1,
                                           const uint32_t (&vals)[NL]) {
    const uint32_t lane = lane_id();
    if (a1 - a0 > b1 - b0) {  // B is the longer list
        LP t = la;
        la = lb;
        lb = t;
        uint32_t u = a0;
        a0 = b0;
        b0 = u;
        u = a1;
        a1 = b1;
        b1 = u;
    }
    const uint32_t n = b1 - b0;
    const uint32_t j0 = b0 + (uint32_t)(((uint64_t)n * lane) >> 5);
    const uint32_t j1 = b0 + (uint32_t)(((uint64_t)n * (lane + 1)) >> 5);
    uint32_t i = a1, i1 = a1;
    if (j0 < j1) {
        i = lower_bound_u32(la, a0, a1, lb[j0]);
        i1 = j1 < b1 ? lower_bound_u32(la, i, a1, lb[j1]) : a1;
    }
    uint32_t j = j0;
    // branch-free merge step: both heads are compared, the equal pair is
    // counted, and each side advances when its head is not the larger one
    if constexpr (!MAT) {
        // software-pipelined: the heads x, y and the next elements xn, yn are
        // in registers; each step issues the loads two positions ahead, so
        // a step waits on no load issued in the same step
        uint32_t cnt = 0;
        if (i < i1 && j < j1) {
            uint32_t x = load_ro(la + i), y = load_ro(lb + j);
            uint32_t xn = load_ro(la + min(i + 1, i1 - 1)), yn = load_ro(lb + min(j + 1, j1 - 1));
            for (;;) {
                cnt += x == y ? 1u : 0u;
                const bool ax = x <= y, ay = y <= x;
                i += ax ? 1u : 0u;
                j += ay ? 1u : 0u;
                if (i >= i1 || j >= j1) break;
                const uint32_t xnn = load_ro(la + min(i + 1, i1 - 1));
                const uint32_t ynn = load_ro(lb + min(j + 1, j1 - 1));
                x = ax ? xn : x;
                xn = ax ? xnn : xn;
                y = ay ? yn : y;
                yn = ay ? ynn : yn;
            }
        }
        A.count += __reduce_add_sync(0xffffffffu, cnt);
    } else {
        for (;;) {
            const bool live = i < i1 && j < j1;
            if (!__any_sync(0xffffffffu, live)) break;
            uint32_t x = 0, y = 1;
            if (live) {
                x = la[i];
                y = lb[j];
                i += x <= y ? 1u : 0u;
                j += y <= x ? 1u : 0u;
            }
            const bool m = live && x == y;
            const uint32_t ball = __ballot_sync(0xffffffffu, m);
            const uint64_t slot = out_reserve(A, ball);
            if (m && slot != ~0ull) write_tuple<L, NL>(P, A.out + slot * (uint64_t)P.nv, E.x, vals, x);
            A.count += __popc(ball);
        }
    }
}

// Last loop, one parent whose shorter list A has many values: the warp takes
// A's values 128 at a time, lane l the values l, l + 32, l + 64, l + 96 of
// the round (so each load instruction reads 32 consecutive values, whose
// buckets in B lie close together), and each lane searches its values in the
// longer list B ("search(V, x)", Sec. 5) through B's bucket directory, the
// four directory reads issued together (index lists; a list in the arena is
// read one value per lane).  B's range, bounds and bucket width are the same for every value,
// so they are read once per parent.  Count mode counts per lane;
// materialize mode writes each slot's matches in lane order.
template <int L, int NL, int S, int O, bool MAT>
__device__ __forceinline__ void pair_match(const DPlan& P, const Entry<NL, S>& E, Acc& A, bool ok, uint32_t v,
                                           const uint32_t (&vals)[NL], uint32_t& cnt) {
    if constexpr (MAT) {
        const uint32_t ball = __ballot_sync(0xffffffffu, ok);
        const uint64_t slot = out_reserve(A, ball);
        if (ok && slot != ~0ull) write_tuple<L, NL>(P, A.out + slot * (uint64_t)P.nv, E.x, vals, v);
        A.count += __popc(ball);
    } else {
        cnt += ok ? 1u : 0u;
    }
}

// Write the n staged values of the warp's buffer as tuples (E.x, the
// parent's values, value) at freshly reserved slots; lane i writes tuples
// i, i + 32, ... (all lanes call, n lane-uniform).
template <int L, int NL, int S>
__device__ __forceinline__ void flush_staged(const DPlan& P, const Entry<NL, S>& E, Acc& A, uint32_t n,
                                             const uint32_t (&vals)[NL]) {
    if (n == 0) return;
    __syncwarp();
    uint64_t s0, s1;
    uint32_t room;
    out_reserve_n(A, n, s0, room, s1);
    for (uint32_t t = lane_id(); t < n; t += 32) {
        const uint64_t base = t < room ? s0 : s1;
        if (base != ~0ull) {
            const uint64_t slot = base + (t < room ? t : t - room);
            write_tuple<L, NL>(P, A.out + slot * (uint64_t)P.nv, E.x, vals, A.obuf[t]);
        }
    }
    __syncwarp();
    A.count += n;
}

template <int L, int NL, int S, int O, bool MAT, typename LP>
__device__ __forceinline__ void probe_pair(const DPlan& P, const Entry<NL, S>& E, Acc& A, LP la,
                                           const uint4* ga, uint32_t a0, uint32_t a1, LP lb,
                                           const uint4* gb, uint32_t b0, uint32_t b1,
                                           const uint32_t (&vals)[NL]) {
    constexpr bool VEC = std::is_same<LP, const uint32_t*>::value;  // an index list (read-only path)
    const uint32_t lane = lane_id();
    if (a1 - a0 > b1 - b0) {  // A is the shorter list
        LP t = la;
        la = lb;
        lb = t;
        const uint4* tg = ga;
        ga = gb;
        gb = tg;
        uint32_t u = a0;
        a0 = b0;
        b0 = u;
        u = a1;
        a1 = b1;
        b1 = u;
    }
    const uint32_t nbv = b1 - b0;
    if (nbv == 0 || a1 == a0) return;
    const uint32_t vmin = load_ro(lb + b0), vmax = load_ro(lb + b1 - 1);
    const bool dir = gb != nullptr && nbv >= P.dir_min;
    const uint32_t sh = dir ? dir_shift(nbv, vmax - vmin) : 0u;
    const uint4* gd = gb + b0;
    uint32_t cnt = 0;
    uint32_t staged = 0;  // values in the warp's buffer (materialize, VEC)
    if constexpr (VEC) {
        for (uint32_t t0 = a0; t0 < a1; t0 += 128) {
            uint32_t vv[4];
            bool okv[4];
            uint4 ev[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t t = t0 + 32 * j + lane;
                vv[j] = t < a1 ? load_ro(la + t) : 0u;
                okv[j] = t < a1 && vv[j] - vmin <= vmax - vmin;  // x in [vmin, vmax], one compare
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                ev[j] = (okv[j] && dir) ? dir_load(gd, (vv[j] - vmin) >> sh) : make_uint4(0u, 0u, 0u, 0u);
            uint32_t mine = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t pos;
                if (okv[j]) okv[j] = dir ? dir_walk_find(lb, ev[j], b1, vv[j], pos) : find_u32(lb, b0, b1, vv[j], pos);
                mine += okv[j] ? 1u : 0u;
            }
            if constexpr (MAT) {
                // stage this round's matches: lane l's go after those of lanes < l
                const uint32_t incl = warp_incl_scan(mine);
                const uint32_t k = __shfl_sync(0xffffffffu, incl, 31);
                if (staged + k > OBUF) {
                    flush_staged<L, NL, S>(P, E, A, staged, vals);
                    staged = 0;
                }
                uint32_t at = staged + incl - mine;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (okv[j]) A.obuf[at++] = vv[j];
                staged += k;
            } else {
                cnt += mine;
            }
        }
        if constexpr (MAT) flush_staged<L, NL, S>(P, E, A, staged, vals);
    } else {
        for (uint32_t t0 = a0; t0 < a1; t0 += 32) {
            const uint32_t t = t0 + lane;
            const uint32_t v = t < a1 ? load_ro(la + t) : 0u;
            bool ok = t < a1 && v >= vmin && v <= vmax;
            if (ok) {
                uint32_t pos;
                ok = dir ? dir_walk_find(lb, dir_load(gd, (v - vmin) >> sh), b1, v, pos) : find_u32(lb, b0, b1, v, pos);
            }
            pair_match<L, NL, S, O, MAT>(P, E, A, ok, v, vals, cnt);
        }
    }
    if constexpr (!MAT) A.count += __reduce_add_sync(0xffffffffu, cnt);
}

// Compact this round's matches into the batch of loop L and descend.
template <int L, int NL, int S, int O, bool MAT>
__device__ __forceinline__ void descend(const DPlan& P, Frame<NL, O>& F, const Entry<NL, S>& E, Acc& A, bool ok,
                                        uint32_t v, uint32_t parent, const uint32_t (&nlo)[O],
                                        const uint32_t (&nhi)[O]) {
    const uint32_t ball = __ballot_sync(0xffffffffu, ok);
    const uint32_t nnew = __popc(ball);
    if (nnew == 0) return;
    const uint32_t lane = lane_id();
    const uint32_t src = lane < nnew ? nth_set_bit(ball, lane) : 0;
    F.val[L] = __shfl_sync(0xffffffffu, v, src);
    F.par[L] = __shfl_sync(0xffffffffu, parent, src);
#pragma unroll
    for (int s = 0; s < O; ++s) {
        F.olo[L][s] = __shfl_sync(0xffffffffu, nlo[s], src);
        F.ohi[L][s] = __shfl_sync(0xffffffffu, nhi[s], src);
    }
    run_level<L + 1, NL, S, O, MAT>(P, F, E, A, nnew);
}

// Loop L >= 1 (index): the parents are the nb bindings of loop L-1 held by
// lanes 0..nb-1 (for L == 1 the entry itself, nb == 1, candidates limited to
// the work item's subrange via E.lo/hi of its shortest list); their
// candidates are flattened over the lanes, 32 a round.
template <int L, int NL, int S, int O, bool MAT>
__device__ __forceinline__ void run_level(const DPlan& P, Frame<NL, O>& F, const Entry<NL, S>& E, Acc& A,
                                          uint32_t nb) {
    if constexpr (L < NL) {
        const uint32_t lane = lane_id();
        const int ns = P.nsrc[L];
        // query rewriting: the last loop's far sources, once per parent of this loop
        if constexpr (L == NL - 2 && NL >= 4) {
            if (P.lift) F.lifted = lift_compute<NL, S, O>(P, F, E, A, nb);
        }
        bool lifted = false;
        if constexpr (L == NL - 1 && NL >= 4) lifted = P.lift && F.lifted;
        const uint32_t use = lifted ? ~(P.far_mask & ~(1u << P.far0)) : 0xFFFFFFFFu;  // sources read
        const int lift_q = lifted ? P.far0 : -1;                                     // reads the arena
        uint32_t mlo[S], mhi[S];
        uint32_t best = 0, bestlen = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < S; ++q) {
            mlo[q] = mhi[q] = 0;
            if (q < ns && ((use >> q) & 1u)) {
                if (q == lift_q) {  // the lifted list of the parent's loop NL-3 ancestor
                    const uint32_t anc = __shfl_sync(0xffffffffu, F.par[L - 1], lane < nb ? lane : 0);
                    mlo[q] = __shfl_sync(0xffffffffu, F.tlo, anc);
                    mhi[q] = __shfl_sync(0xffffffffu, F.thi, anc);
                } else {
                    src_range<L, NL, S, O>(P, F, E, q, lane < nb ? lane : 0, mlo[q], mhi[q]);
                }
                const uint32_t len = mhi[q] - mlo[q];
                if (len < bestlen) {
                    bestlen = len;
                    best = q;
                }
            }
        }
        if constexpr (L == 1) {
            // loop 1 of a work item: its subrange [k0, k1) of the entry's shortest list
            best = E.best1;
            bestlen = E.k1 - E.k0;
#pragma unroll
            for (int q = 0; q < S; ++q)
                if (q == (int)best) {
                    const uint32_t base = mlo[q];
                    mlo[q] = base + E.k0;
                    mhi[q] = base + E.k1;
                }
        }
        if constexpr (L == 2 && NL >= 4) {
            // a sliced work unit: one loop-2 binding (lane 0), slices [j0, j1)
            if (E.ns > 1 && lane == 0 && nb == 1) {
#pragma unroll
                for (int q = 0; q < S; ++q)
                    if (q == (int)best) {
                        const uint32_t base = mlo[q];
                        mlo[q] = base + (uint32_t)(((uint64_t)bestlen * E.j0) / E.ns);
                        mhi[q] = base + (uint32_t)(((uint64_t)bestlen * E.j1) / E.ns);
                    }
            }
        }
        bool merge_class = false, pair_class = false;
        int qa = 0, qb = 1;  // the two lists of a merge pair
        if constexpr (L == NL - 1 && S >= 2) {
            const uint32_t um = use & ((1u << ns) - 1u);
            if (__popc(um) == 2) {
                qa = __ffs(um) - 1;
                qb = __ffs(um & (um - 1u)) - 1;
                if (lane < nb) {
                    uint32_t l0 = 0, l1 = 0;
#pragma unroll
                    for (int q = 0; q < S; ++q) {
                        if (q == qa) l0 = mhi[q] - mlo[q];
                        if (q == qb) l1 = mhi[q] - mlo[q];
                    }
                    const uint32_t mn = min(l0, l1), mx = max(l0, l1);
                    merge_class = mn >= P.merge_min && (uint64_t)mx <= (uint64_t)P.merge_ratio * mn;
                    pair_class = !merge_class && mn >= P.pair_min;
                }
            }
        }
        if (A.stats && lane < nb) {
            if (L > 2 || (L == 2 && E.j0 == 0))
                A.work += (uint64_t)ns * bestlen;  // once per binding, before slicing
            else if (L == 1 && E.k0 == 0 && E.j0 == 0)
                A.work += (uint64_t)ns * E.len1;  // once per loop-1 binding
        }
        if constexpr (L == 2 && NL >= 4) {
            if (E.ns > 1 && lane == 0 && nb == 1) {
#pragma unroll
                for (int q = 0; q < S; ++q)
                    if (q == (int)best) bestlen = mhi[q] - mlo[q];
            }
        }
        const uint32_t cnt = (lane < nb && !merge_class && !pair_class) ? bestlen : 0;
        const uint32_t incl = warp_incl_scan(cnt);
        const uint32_t excl = incl - cnt;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t t0 = 0; t0 < total; t0 += 32) {
            const uint32_t t = t0 + lane;
            const bool active = t < total;
            uint32_t p = 0;  // parent of candidate t: the last lane p < nb with excl_p <= t
            if (nb > 1) {
#pragma unroll
                for (uint32_t step = 16; step >= 1; step >>= 1) {
                    const uint32_t c = p + step;
                    const uint32_t ex = __shfl_sync(0xffffffffu, excl, c & 31u);
                    if (c < nb && ex <= t) p = c;
                }
            }
            const uint32_t k = t - __shfl_sync(0xffffffffu, excl, p);
            const uint32_t pbest = __shfl_sync(0xffffffffu, best, p);
            uint32_t rlo[S], rhi[S];
#pragma unroll
            for (int q = 0; q < S; ++q) {
                rlo[q] = __shfl_sync(0xffffffffu, mlo[q], p);
                rhi[q] = __shfl_sync(0xffffffffu, mhi[q], p);
            }
            uint32_t v = 0, kpos = 0;
#pragma unroll
            for (int q = 0; q < S; ++q)
                if (q == (int)pbest && active) {
                    kpos = rlo[q] + k;
                    v = src_list_l(P, A, L, q, lift_q)[kpos];
                }
            uint32_t nlo[O], nhi[O];
#pragma unroll
            for (int s = 0; s < O; ++s) nlo[s] = nhi[s] = 0;
            const bool ok = probe<L, S, O>(P, (int)pbest, rlo, rhi, kpos, v, active, nlo, nhi, use, A.arena, lift_q);
            if constexpr (L == NL - 1)
                finish_round<L, NL, S, O, MAT>(P, F, E, A, ok, v, p);
            else
                descend<L, NL, S, O, MAT>(P, F, E, A, ok, v, p, nlo, nhi);
        }
        if constexpr (L == NL - 1 && S >= 2) {
            uint32_t mball = __ballot_sync(0xffffffffu, merge_class);
            uint32_t xa0 = 0, xa1 = 0, xb0 = 0, xb1 = 0;
#pragma unroll
            for (int q = 0; q < S; ++q) {
                if (q == qa) {
                    xa0 = mlo[q];
                    xa1 = mhi[q];
                }
                if (q == qb) {
                    xb0 = mlo[q];
                    xb1 = mhi[q];
                }
            }
            while (mball) {
                const uint32_t p = __ffs(mball) - 1;
                mball &= mball - 1;
                const uint32_t a0 = __shfl_sync(0xffffffffu, xa0, p), a1 = __shfl_sync(0xffffffffu, xa1, p);
                const uint32_t b0 = __shfl_sync(0xffffffffu, xb0, p), b1 = __shfl_sync(0xffffffffu, xb1, p);
                uint32_t vals[NL];
                if constexpr (MAT) prefix_values<L, NL, O>(F, p, vals);
                if (qa == lift_q || qb == lift_q)  // a list in the arena: coherent loads
                    merge_pair<L, NL, S, O, MAT>(P, E, A, const_cast<uint32_t*>(src_list_l(P, A, L, qa, lift_q)), a0,
                                                 a1, const_cast<uint32_t*>(src_list_l(P, A, L, qb, lift_q)), b0, b1,
                                                 vals);
                else
                    merge_pair<L, NL, S, O, MAT>(P, E, A, src_list(P, L, qa), a0, a1, src_list(P, L, qb), b0, b1,
                                                 vals);
            }
            uint32_t pball = __ballot_sync(0xffffffffu, pair_class);
            if (pball) {
                const DAtom& da = P.atom[P.src_atom[L][qa]];
                const DAtom& db = P.atom[P.src_atom[L][qb]];
                const uint4* ga = qa == lift_q ? nullptr : (P.src_top[L][qa] ? da.g1 : da.g2);
                const uint4* gb = qb == lift_q ? nullptr : (P.src_top[L][qb] ? db.g1 : db.g2);
                while (pball) {
                    const uint32_t p = __ffs(pball) - 1;
                    pball &= pball - 1;
                    const uint32_t a0 = __shfl_sync(0xffffffffu, xa0, p), a1 = __shfl_sync(0xffffffffu, xa1, p);
                    const uint32_t b0 = __shfl_sync(0xffffffffu, xb0, p), b1 = __shfl_sync(0xffffffffu, xb1, p);
                    uint32_t vals[NL];
                    if constexpr (MAT) prefix_values<L, NL, O>(F, p, vals);
                    if (qa == lift_q || qb == lift_q)  // a list in the arena: coherent loads
                        probe_pair<L, NL, S, O, MAT>(P, E, A, const_cast<uint32_t*>(src_list_l(P, A, L, qa, lift_q)),
                                                     ga, a0, a1, const_cast<uint32_t*>(src_list_l(P, A, L, qb, lift_q)),
                                                     gb, b0, b1, vals);
                    else
                        probe_pair<L, NL, S, O, MAT>(P, E, A, src_list(P, L, qa), ga, a0, a1, src_list(P, L, qb), gb,
                                                     b0, b1, vals);
                }
            }
        }
    }
}

// One work item: units [item*grain, (item+1)*grain) of the concatenation of
// all entries' units (a unit is a loop-2 candidate, or a slice of one for
// deep queries).  Returns the item's count; cell counts are added when
// requested.  elo/ehi are the warp's shared-memory rows for entry ranges.
template <int NL, int S, int O, bool MAT>
__device__ __forceinline__ uint64_t search_item(const DPlan& P, Frame<NL, O>& F, Acc& A, uint32_t (*elo)[S],
                                                uint32_t (*ehi)[S], uint64_t item, uint32_t grain, uint32_t E_n,
                                                uint64_t U, const uint32_t* __restrict__ e_cell,
                                                const uint32_t* __restrict__ e_x, const uint32_t* __restrict__ e_rng,
                                                const uint32_t* __restrict__ e_split,
                                                const uint64_t* __restrict__ uoff, uint64_t* __restrict__ cell_counts,
                                                int pass) {
    const uint32_t lane = lane_id();
    uint64_t u0 = item * grain;
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
    uint64_t item_count = 0;
    while (u0 < u1 && e < E_n) {
        const uint64_t eb = uoff[e], ee = uoff[e + 1];
        if (ee <= u0) {
            ++e;
            continue;
        }
        const uint64_t ku0 = u0 - eb, ku1 = min(u1, ee) - eb;
        Entry<NL, S> E;
        E.lo = elo;
        E.hi = ehi;
        __syncwarp();  // the previous entry's ranges are no longer read
        E.cell = e_cell[e];
        E.x = e_x[e];
        uint32_t r0lo[MAXOPEN], r0hi[MAXOPEN];
#pragma unroll
        for (int s = 0; s < MAXOPEN; ++s) {
            r0lo[s] = s < P.nopen[0] ? e_rng[(uint64_t)e * (2 * MAXOPEN) + 2 * s] : 0;
            r0hi[s] = s < P.nopen[0] ? e_rng[(uint64_t)e * (2 * MAXOPEN) + 2 * s + 1] : 0;
        }
        uint32_t best1 = 0, len1 = 0xFFFFFFFFu;
#pragma unroll
        for (int L = 1; L < NL; ++L)
#pragma unroll
            for (int q = 0; q < S; ++q) {
                uint32_t lo2 = 0, hi2 = 0;
                if (q < P.nsrc[L] && P.src_ec[L][q]) {
                    const DAtom& a = P.atom[P.src_atom[L][q]];
                    if (P.src_top[L][q]) {
                        top_range(a, E.cell, lo2, hi2);
                    } else {
#pragma unroll
                        for (int s = 0; s < MAXOPEN; ++s)
                            if (s == a.slot) {
                                lo2 = r0lo[s];
                                hi2 = r0hi[s];
                            }
                    }
                }
                if (L == 1 && q < P.nsrc[1] && hi2 - lo2 < len1) {
                    len1 = hi2 - lo2;
                    best1 = q;
                }
                if (lane == 0) {
                    E.lo[L][q] = lo2;
                    E.hi[L][q] = hi2;
                }
            }
        __syncwarp();
        E.best1 = best1;
        E.len1 = len1;
        const uint64_t before = A.count;
        const uint64_t work0 = A.work;
        const long long clk0 = A.cprof ? clock64() : 0;
        const uint32_t split = e_split[e];
        // units are (loop-2 candidate k, slice j) pairs, k-major; an
        // unsliced entry (split 1) is one call over its candidate range
        for (uint64_t u = ku0; u < ku1;) {
            if (split == 1) {
                E.k0 = (uint32_t)u;
                E.k1 = (uint32_t)ku1;
                E.j0 = 0;
                E.j1 = 1;
                u = ku1;
            } else {
                const uint32_t j0 = (uint32_t)(u % split);
                const uint64_t jend = j0 + (ku1 - u);
                E.k0 = (uint32_t)(u / split);
                E.k1 = E.k0 + 1;
                E.j0 = j0;
                E.j1 = jend < split ? (uint32_t)jend : split;
                u += E.j1 - j0;
            }
            E.ns = split;
            run_level<1, NL, S, O, MAT>(P, F, E, A, 1);
        }
        const uint64_t got = A.count - before;
        if (pass == 0 && cell_counts && got && lane == 0)
            atomicAdd((unsigned long long*)&cell_counts[E.cell], (unsigned long long)got);
        if (A.cprof) {  // this entry's share of its cell's work and of the warps' time on it
            const uint64_t dw = warp_sum64(A.work - work0);
            const unsigned long long dt = (unsigned long long)(clock64() - clk0);
            if (lane == 0) {
                if (dw) atomicAdd((unsigned long long*)&A.cprof[2 * (uint64_t)E.cell], (unsigned long long)dw);
                atomicAdd((unsigned long long*)&A.cprof[2 * (uint64_t)E.cell + 1], dt);
            }
        }
        item_count += got;
        u0 = eb + ku1;
        ++e;
    }
    return item_count;
}

// Persistent search kernel of one query.  Warps take work items from an
// atomic counter.  pass 0 counts (and, with item_counts, records each item's
// count; materialize writes into pool chunks); pass 1 writes tuples at
// item_base[item].
template <int NL, int S, int O, bool MAT>
__global__ void __launch_bounds__(128, (NL <= 3 ? 16 : 12)) gj_kernel(const DPlan* __restrict__ gP, const uint32_t* __restrict__ e_cell,
                                                    const uint32_t* __restrict__ e_x,
                                                    const uint32_t* __restrict__ e_rng,
                                                    const uint32_t* __restrict__ e_split,
                                                    const uint64_t* __restrict__ uoff, uint32_t grain, JoinCtl* ctl,
                                                    int pass, uint64_t* __restrict__ cell_counts,
                                                    uint64_t* __restrict__ item_counts,
                                                    const uint64_t* __restrict__ item_base, uint32_t* __restrict__ out,
                                                    int stats, uint32_t* __restrict__ chunk_fill, uint32_t n_chunks,
                                                    uint32_t* __restrict__ arena, uint32_t item_lo, uint32_t item_hi,
                                                    uint32_t* __restrict__ item_ctr, uint64_t* __restrict__ cell_prof) {
    __shared__ DPlan P;
    __shared__ uint32_t s_elo[4][NL][S], s_ehi[4][NL][S];  // per warp (blocks of <= 128 threads)
    __shared__ uint32_t s_obuf[MAT ? 4 : 1][MAT ? OBUF : 1];
    load_plan(P, gP);
    if (dev_err_set(&ctl->err)) return;  // a scan of the loop-1 pass gave up a wait
    const uint32_t lane = lane_id();
    const uint32_t E_n = ctl->n_entries;
    const uint64_t U = uoff[E_n];
    const uint64_t nitems = (U + grain - 1) / grain;
    Frame<NL, O> F;
    F.lifted = false;
    Acc A;
    A.count = 0;
    A.work = 0;
    A.out_pos = 0;
    A.out = out;
    A.stats = stats && pass == 0;
    A.pool = MAT && pass == 0;  // single pass: count and write into pool chunks
    A.chunk = NO_CHUNK;
    A.fill = OUT_CHUNK;
    A.n_chunks = n_chunks;
    A.chunk_fill = chunk_fill;
    A.ctl = ctl;
    A.arena = arena ? arena + (uint64_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * P.arena_words
                    : nullptr;
    A.obuf = MAT ? s_obuf[MAT ? (threadIdx.x >> 5) : 0] : nullptr;
    A.cprof = pass == 0 ? cell_prof : nullptr;
    uint64_t total = 0;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = item_lo + atomicAdd(item_ctr, 1u);  // items [item_lo, item_hi) of this launch
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= item_hi || item >= nitems) break;
        A.out_pos = (MAT && !A.pool) ? item_base[item] : 0;
        const uint64_t item_count =
            search_item<NL, S, O, MAT>(P, F, A, s_elo[threadIdx.x >> 5], s_ehi[threadIdx.x >> 5], item, grain, E_n, U,
                                       e_cell, e_x, e_rng, e_split, uoff, cell_counts, pass);
        if (pass == 0 && item_counts && lane == 0) item_counts[item] = item_count;
        total += item_count;
    }
    if (pass == 0 && lane == 0 && total) atomicAdd((unsigned long long*)&ctl->total, (unsigned long long)total);
    if (A.pool && lane == 0 && A.chunk != NO_CHUNK) chunk_fill[A.chunk] = A.fill;
    if (A.stats) {
        const uint64_t w = warp_sum64(A.work);
        if (lane == 0 && w) atomicAdd((unsigned long long*)&ctl->work, (unsigned long long)w);
    }
}

// ------------------------------------------------------------ batched launch
// Many queries in one persistent launch (count mode).  Each query keeps its
// own plan, entries and unit offsets; the work items of all queries form one
// space (item_off: prefix of the per-query item counts) handed out by one
// atomic counter, so warps move on to whichever query still has work.  A
// warp keeps the plan of the query it is working on in shared memory.
struct BQuery {
    const DPlan* plan;
    const uint32_t *e_cell, *e_x, *e_rng, *e_split;
    const uint64_t* uoff;
    JoinCtl* ctl;
    uint32_t grain;
    uint32_t shape;  // 0: the kernel's first shape, 1: its second (all-shapes kernel: the shape class)
};

__global__ void batch_items_kernel(const BQuery* __restrict__ qs, uint32_t n, uint64_t* __restrict__ items) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const BQuery& b = qs[i];
        const uint64_t U = b.uoff[b.ctl->n_entries];
        items[i] = (U + b.grain - 1) / b.grain;
    }
}

template <int NLA, int SA, int OA, int NLB, int SB, int OB>
__global__ void __launch_bounds__(128, ((NLA <= 3 && NLB <= 3) ? 16 : 12))
    gj_batch_kernel(const BQuery* __restrict__ qs, uint32_t n, const uint64_t* __restrict__ item_off,
                    uint32_t* __restrict__ ctr, uint32_t* __restrict__ arena, uint32_t arena_stride) {
    constexpr int NLM = NLA > NLB ? NLA : NLB;
    constexpr int SM = SA > SB ? SA : SB;
    __shared__ DPlan wplan[4];
    __shared__ uint32_t s_e[4][2 * NLM * SM];
    const uint32_t w = threadIdx.x >> 5, lane = lane_id();
    if (dev_err_set(&qs[0].ctl->err)) return;  // the item-offset scan gave up a wait
    const uint64_t total_items = item_off[n];
    uint32_t cur = 0xFFFFFFFFu;
    Acc A;
    A.count = 0;
    A.work = 0;
    A.out_pos = 0;
    A.out = nullptr;
    A.stats = 0;
    A.pool = 0;
    A.chunk = NO_CHUNK;
    A.fill = OUT_CHUNK;
    A.n_chunks = 0;
    A.chunk_fill = nullptr;
    A.ctl = nullptr;
    A.arena = arena ? arena + (uint64_t)(blockIdx.x * 4 + w) * arena_stride : nullptr;
    A.obuf = nullptr;
    A.cprof = nullptr;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(ctr, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total_items) break;
        uint32_t lo = 0, hi = n;  // query holding item it: last q with item_off[q] <= it
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= it)
                lo = mid;
            else
                hi = mid;
        }
        const uint32_t q = lo;
        const BQuery& b = qs[q];
        if (dev_err_set(&b.ctl->err)) continue;  // a scan of this query's loop-1 pass gave up a wait
        if (q != cur) {
            __syncwarp();
            const uint32_t* src = (const uint32_t*)b.plan;
            uint32_t* dst = (uint32_t*)&wplan[w];
            for (uint32_t i = lane; i < sizeof(DPlan) / 4; i += 32) dst[i] = src[i];
            __syncwarp();
            cur = q;
        }
        const DPlan& P = wplan[w];
        const uint32_t E_n = b.ctl->n_entries;
        const uint64_t U = b.uoff[E_n];
        const uint64_t local = it - item_off[q];
        uint64_t c;
        if (b.shape == 0) {
            Frame<NLA, OA> F;
            F.lifted = false;
            c = search_item<NLA, SA, OA, false>(P, F, A, (uint32_t(*)[SA])s_e[w], (uint32_t(*)[SA])(s_e[w] + NLA * SA),
                                                local, b.grain, E_n, U, b.e_cell, b.e_x, b.e_rng, b.e_split, b.uoff,
                                                nullptr, 0);
        } else {
            Frame<NLB, OB> F;
            F.lifted = false;
            c = search_item<NLB, SB, OB, false>(P, F, A, (uint32_t(*)[SB])s_e[w], (uint32_t(*)[SB])(s_e[w] + NLB * SB),
                                                local, b.grain, E_n, U, b.e_cell, b.e_x, b.e_rng, b.e_split, b.uoff,
                                                nullptr, 0);
        }
        if (lane == 0 && c) atomicAdd((unsigned long long*)&b.ctl->total, (unsigned long long)c);
    }
}

// Batches of more than two query shapes: one launch over the four built-in
// shape classes (3 loops with 2 or 4 lists and opened atoms per loop, 4 loops
// likewise); each query's item runs the search compiled for its class.
__global__ void __launch_bounds__(128, 12)
    gj_batch_all_kernel(const BQuery* __restrict__ qs, uint32_t n, const uint64_t* __restrict__ item_off,
                        uint32_t* __restrict__ ctr, uint32_t* __restrict__ arena, uint32_t arena_stride) {
    __shared__ DPlan wplan[4];
    __shared__ uint32_t s_e[4][2 * 4 * 4];
    const uint32_t w = threadIdx.x >> 5, lane = lane_id();
    if (dev_err_set(&qs[0].ctl->err)) return;  // the item-offset scan gave up a wait
    const uint64_t total_items = item_off[n];
    uint32_t cur = 0xFFFFFFFFu;
    Acc A;
    A.count = 0;
    A.work = 0;
    A.out_pos = 0;
    A.out = nullptr;
    A.stats = 0;
    A.pool = 0;
    A.chunk = NO_CHUNK;
    A.fill = OUT_CHUNK;
    A.n_chunks = 0;
    A.chunk_fill = nullptr;
    A.ctl = nullptr;
    A.arena = arena ? arena + (uint64_t)(blockIdx.x * 4 + w) * arena_stride : nullptr;
    A.obuf = nullptr;
    A.cprof = nullptr;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(ctr, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total_items) break;
        uint32_t lo = 0, hi = n;  // query holding item it: last q with item_off[q] <= it
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= it)
                lo = mid;
            else
                hi = mid;
        }
        const uint32_t q = lo;
        const BQuery& b = qs[q];
        if (dev_err_set(&b.ctl->err)) continue;  // a scan of this query's loop-1 pass gave up a wait
        if (q != cur) {
            __syncwarp();
            const uint32_t* src = (const uint32_t*)b.plan;
            uint32_t* dst = (uint32_t*)&wplan[w];
            for (uint32_t i = lane; i < sizeof(DPlan) / 4; i += 32) dst[i] = src[i];
            __syncwarp();
            cur = q;
        }
        const DPlan& P = wplan[w];
        const uint32_t E_n = b.ctl->n_entries;
        const uint64_t U = b.uoff[E_n];
        const uint64_t local = it - item_off[q];
        uint64_t c = 0;
        switch (b.shape) {
            case 0: {
                Frame<3, 2> F;
                F.lifted = false;
                c = search_item<3, 2, 2, false>(P, F, A, (uint32_t(*)[2])s_e[w], (uint32_t(*)[2])(s_e[w] + 3 * 2),
                                                local, b.grain, E_n, U, b.e_cell, b.e_x, b.e_rng, b.e_split, b.uoff,
                                                nullptr, 0);
                break;
            }
            case 1: {
                Frame<3, 4> F;
                F.lifted = false;
                c = search_item<3, 4, 4, false>(P, F, A, (uint32_t(*)[4])s_e[w], (uint32_t(*)[4])(s_e[w] + 3 * 4),
                                                local, b.grain, E_n, U, b.e_cell, b.e_x, b.e_rng, b.e_split, b.uoff,
                                                nullptr, 0);
                break;
            }
            case 2: {
                Frame<4, 2> F;
                F.lifted = false;
                c = search_item<4, 2, 2, false>(P, F, A, (uint32_t(*)[2])s_e[w], (uint32_t(*)[2])(s_e[w] + 4 * 2),
                                                local, b.grain, E_n, U, b.e_cell, b.e_x, b.e_rng, b.e_split, b.uoff,
                                                nullptr, 0);
                break;
            }
            default: {
                Frame<4, 4> F;
                F.lifted = false;
                c = search_item<4, 4, 4, false>(P, F, A, (uint32_t(*)[4])s_e[w], (uint32_t(*)[4])(s_e[w] + 4 * 4),
                                                local, b.grain, E_n, U, b.e_cell, b.e_x, b.e_rng, b.e_split, b.uoff,
                                                nullptr, 0);
                break;
            }
        }
        if (lane == 0 && c) atomicAdd((unsigned long long*)&b.ctl->total, (unsigned long long)c);
    }
}

// Single-pass materialize: the pool becomes the output in place.  A search
// launch (a segment of the work items) fills the chunk range [cb, ce) of the
// pool; every chunk of it is full except each warp's last one, so the n_full
// full chunks are arranged to fill slots [cb, cb + n_full) and the partial
// chunks' tuples follow them: a partial chunk in that prefix (a hole)
// receives a full chunk from above it (a donor), k-th hole from k-th donor.
// Only the partial chunks' tuples and the donors move (at most a chunk per
// resident warp each), not the whole output.  The range comes from the device
// (seg_mark_kernel); local chunk index i stands for chunk cb + i.
//   seg_mark_kernel       seg = {cb, ce, ce - cb}, cb = the previous segment's ce
//   chunk_class_kernel    is_partial[i], fill of partial chunks (0 for full)
//   (two exclusive scans: prank = partials before i, poff = their tuples)
//   save_partials_kernel  partial chunks' tuples -> tmp at poff; pslot[prank] = i
//   move_donors_kernel    donor of rank r -> local slot pslot[r]
//   place_partials_kernel tmp -> after the n_full full chunks; seg.tuples
struct Seg {
    uint32_t cb, ce, n, pad;
    uint64_t tuples;  // tuples of the segment, contiguous from chunk cb after compaction
};

__global__ void seg_mark_kernel(const JoinCtl* __restrict__ ctl, uint32_t n_chunks, const Seg* __restrict__ prev,
                                Seg* __restrict__ seg) {
    const uint32_t cb = prev ? prev->ce : 0u;
    const uint32_t ce = max(cb, min(ctl->chunk_ctr, n_chunks));
    seg->cb = cb;
    seg->ce = ce;
    seg->n = ce - cb;
    seg->tuples = 0;
}

__global__ void chunk_class_kernel(const uint32_t* __restrict__ chunk_fill, const Seg* __restrict__ seg,
                                   uint32_t* __restrict__ is_partial, uint32_t* __restrict__ pfill) {
    const uint32_t cb = seg->cb, n = seg->n;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t f = chunk_fill[cb + i];
        is_partial[i] = f < OUT_CHUNK ? 1u : 0u;
        pfill[i] = f < OUT_CHUNK ? f : 0u;
    }
}

__global__ void save_partials_kernel(const uint32_t* __restrict__ pool, const uint32_t* __restrict__ chunk_fill,
                                     const Seg* __restrict__ seg, const uint64_t* __restrict__ prank,
                                     const uint64_t* __restrict__ poff, uint32_t nv, uint32_t* __restrict__ tmp,
                                     uint32_t* __restrict__ pslot, const uint32_t* __restrict__ err) {
    if (dev_err_set(err)) return;  // the scans gave up a wait: their offsets are not valid
    const uint32_t cb = seg->cb, n = seg->n;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t f = chunk_fill[cb + i];
        if (f >= OUT_CHUNK) continue;
        if (threadIdx.x == 0) pslot[prank[i]] = i;
        const uint64_t words = (uint64_t)f * nv;
        const uint32_t* src = pool + (uint64_t)(cb + i) * OUT_CHUNK * nv;
        uint32_t* dst = tmp + poff[i] * nv;
        for (uint64_t w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
}

__global__ void move_donors_kernel(uint32_t* __restrict__ pool, const uint32_t* __restrict__ chunk_fill,
                                   const Seg* __restrict__ seg, const uint64_t* __restrict__ prank,
                                   const uint32_t* __restrict__ pslot, uint32_t nv, const uint32_t* __restrict__ err) {
    if (dev_err_set(err)) return;
    const uint32_t cb = seg->cb, n = seg->n;
    const uint32_t n_full = n - (uint32_t)prank[n];
    for (uint32_t i = n_full + blockIdx.x; i < n; i += gridDim.x) {
        if (chunk_fill[cb + i] < OUT_CHUNK) continue;
        // full chunks in [n_full, i), i.e. this donor's rank among donors
        const uint64_t r = (uint64_t)(i - n_full) - (prank[i] - prank[n_full]);
        const uint32_t dst_slot = cb + pslot[r];  // the r-th partial chunk of the segment, a hole
        const uint4* src = reinterpret_cast<const uint4*>(pool + (uint64_t)(cb + i) * OUT_CHUNK * nv);
        uint4* dst = reinterpret_cast<uint4*>(pool + (uint64_t)dst_slot * OUT_CHUNK * nv);
        const uint32_t vecs = OUT_CHUNK * nv / 4;  // a chunk is a multiple of 16 bytes
        for (uint32_t w = threadIdx.x; w < vecs; w += blockDim.x) dst[w] = src[w];
    }
}

__global__ void place_partials_kernel(uint32_t* __restrict__ pool, const uint32_t* __restrict__ tmp,
                                      Seg* __restrict__ seg, const uint64_t* __restrict__ prank,
                                      const uint64_t* __restrict__ poff, uint32_t nv, const uint32_t* __restrict__ err) {
    if (dev_err_set(err)) return;
    const uint32_t cb = seg->cb, n = seg->n;
    const uint32_t n_full = n - (uint32_t)prank[n];
    const uint64_t words = poff[n] * nv;
    uint32_t* dst = pool + (uint64_t)(cb + n_full) * OUT_CHUNK * nv;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x)
        dst[w] = tmp[w];
    if (blockIdx.x == 0 && threadIdx.x == 0) seg->tuples = (uint64_t)n_full * OUT_CHUNK + poff[n];
}

// Search kernels are compiled for NL = 2..5 loops and for S (lists per
// loop) and O (atoms opened per loop) of 2 or 4.
template <int NL, int S, int O>
int gj_grid(bool mat, int threads) {
    const void* kern = mat ? (const void*)gj_kernel<NL, S, O, true> : (const void*)gj_kernel<NL, S, O, false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms();
}

struct GjArgs {
    const DPlan* plan;
    const uint32_t *e_cell, *e_x, *e_rng, *e_split;
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
    uint32_t* chunk_fill;
    uint32_t n_chunks;
    uint32_t* arena;  // lifted lists, P.arena_words per warp of the launch
    // work items [item_lo, item_hi) taken through item_ctr (NULL: the join's
    // counter of the pass, all items)
    uint32_t item_lo = 0, item_hi = 0xFFFFFFFFu;
    uint32_t* item_ctr = nullptr;
    uint64_t* cell_prof = nullptr;  // per-cell profile (HC_FLAG_CELL_PROFILE)
};

template <int NL, int S, int O>
hc_status launch_gj(bool mat, const GjArgs& g, cudaStream_t s) {
    const int grid = gj_grid<NL, S, O>(mat, g.threads);
    uint32_t* ctr = g.item_ctr ? g.item_ctr : &g.ctl->item_ctr[g.pass];
    if (mat)
        gj_kernel<NL, S, O, true><<<grid, g.threads, 0, s>>>(g.plan, g.e_cell, g.e_x, g.e_rng, g.e_split, g.uoff,
                                                             g.grain, g.ctl,
                                                             g.pass, g.cell_counts, g.item_counts, g.item_base, g.out,
                                                             g.stats, g.chunk_fill, g.n_chunks, g.arena, g.item_lo,
                                                             g.item_hi, ctr, g.cell_prof);
    else
        gj_kernel<NL, S, O, false><<<grid, g.threads, 0, s>>>(g.plan, g.e_cell, g.e_x, g.e_rng, g.e_split, g.uoff,
                                                              g.grain,
                                                              g.ctl, g.pass, g.cell_counts, g.item_counts, g.item_base,
                                                              g.out, g.stats, g.chunk_fill, g.n_chunks, g.arena,
                                                              g.item_lo, g.item_hi, ctr, g.cell_prof);
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

template <int NL>
hc_status launch_nl(int S, int O, bool mat, const GjArgs& g, cudaStream_t s) {
    if (S <= 2 && O <= 2) return launch_gj<NL, 2, 2>(mat, g, s);
    if (S <= 2) return launch_gj<NL, 2, 4>(mat, g, s);
    if (O <= 2) return launch_gj<NL, 4, 2>(mat, g, s);
    return launch_gj<NL, 4, 4>(mat, g, s);
}

template <int NL>
int gj_grid_nl(int S, int O, bool mat, int threads) {
    if (S <= 2 && O <= 2) return gj_grid<NL, 2, 2>(mat, threads);
    if (S <= 2) return gj_grid<NL, 2, 4>(mat, threads);
    if (O <= 2) return gj_grid<NL, 4, 2>(mat, threads);
    return gj_grid<NL, 4, 4>(mat, threads);
}

int gj_grid_any(int nl, int S, int O, bool mat, int threads) {
    switch (nl) {
        case 2: return gj_grid_nl<2>(S, O, mat, threads);
        case 3: return gj_grid_nl<3>(S, O, mat, threads);
        case 4: return gj_grid_nl<4>(S, O, mat, threads);
        default: return gj_grid_nl<5>(S, O, mat, threads);
    }
}

hc_status launch_any(int nl, int S, int O, bool mat, const GjArgs& g, cudaStream_t s) {
    switch (nl) {
        case 2: return launch_nl<2>(S, O, mat, g, s);
        case 3: return launch_nl<3>(S, O, mat, g, s);
        case 4: return launch_nl<4>(S, O, mat, g, s);
        case 5: return launch_nl<5>(S, O, mat, g, s);
        default: return fail(HC_ERR_CAPACITY, "run_join: queries of 2 to 5 variables are built in");
    }
}

}  // namespace hc

// ------------------------------------------------------------------ host
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
    dev_free(r->d_cell_prof, s);
    dev_free(r->d_tuples, s);
    for (auto& e : r->ev)
        if (e) cudaEventDestroy(e);
    delete r;
}

hc_status time_mark(hc_result* R, bool end, cudaStream_t s) {
    const size_t i = 2 * (size_t)R->n_timed + (end ? 1 : 0);
    if (R->ev.size() <= i) R->ev.resize(i + 1, nullptr);
    if (!R->ev[i]) HC_CUDA_TRY(cudaEventCreate(&R->ev[i]));
    HC_CUDA_TRY(cudaEventRecord(R->ev[i], s));
    if (end) R->n_timed++;
    return HC_OK;
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
    v->d_cell_profile = R->d_cell_prof;
    v->work = R->h_ctl.work;
    v->n_items = R->n_items;
    v->n_join_launches = (uint32_t)R->n_search;
    float total_ms = 0.f;
    for (int i = 0; i < R->n_timed; ++i) {
        float ms = 0.f;
        HC_CUDA_TRY(cudaEventElapsedTime(&ms, R->ev[2 * i], R->ev[2 * i + 1]));
        total_ms += ms;
    }
    v->ms_join_kernel = total_ms;
    return HC_OK;
}

// ------------------------------------------------------------ query plans
// Host-side plan of one query: validation, loop order, the lists of every
// loop, and the atoms it partitions (enqueued on `s`, owned by the caller).
struct QueryPlan {
    DPlan P;
    int nv = 0, shape_s = 2, shape_o = 2, threads = 128, stats = 0;
    uint32_t grain = 64;
    uint64_t ncells = 1, cand_bound = 1;
    std::vector<hc_partitioned*> parts;
    std::vector<const hc_index*> part_src;  // the index each partitioned copy was made from
};

static void release_parts(std::vector<hc_partitioned*>& parts, cudaStream_t s) {
    for (auto* p : parts) partitioned_release(p, s);
    parts.clear();
}

hc_status plan_query(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm, cudaStream_t s,
                     QueryPlan* out, uint64_t* partition_bytes = nullptr) {
    if (!q || !idx || !prm || !out) return fail(HC_ERR_ARG, "run_join: NULL argument");
    const int nv = (int)q->n_vars, na = (int)q->n_atoms;
    if (nv < 2 || nv > HC_MAX_VARS || na < 1 || na > HC_MAX_ATOMS)
        return fail(HC_ERR_ARG, "run_join: need 2..8 variables and 1..12 atoms");
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
        if (a >= nv || (b >= nv && b != (int)HC_UNARY) || a == b)
            return fail(HC_ERR_ARG, "run_join: atom variables out of range or equal");
        if (!idx[j]) return fail(HC_ERR_ARG, "run_join: missing index for an atom");
        // a size estimate (partition_bytes given) needs no data
        if (idx[j]->stats_only && !partition_bytes)
            return fail(HC_ERR_ARG, "run_join: a statistics-only index has no data");
        covered[a] = true;
        if (b != (int)HC_UNARY) covered[b] = true;
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
    out->grain = prm->item_grain ? prm->item_grain : 64;
    out->threads = prm->block_threads ? (int)prm->block_threads : 128;
    if (out->threads % 32 != 0 || out->threads < 32 || out->threads > 128)
        return fail(HC_ERR_ARG, "run_join: block_threads must be a multiple of 32 in [32, 128]");
    out->nv = nv;
    out->ncells = ncells;
    out->stats = (prm->flags & (HC_FLAG_STATS | HC_FLAG_CELL_PROFILE)) ? 1 : 0;

    DPlan& P = out->P;
    memset(&P, 0, sizeof(P));
    P.nlev = nv;
    P.natoms = na;
    P.nv = nv;
    P.ncells = (uint32_t)ncells;
    for (int i = 0; i < nv; ++i) P.var_of_level[i] = q->order[i];
    auto bail = [&](hc_status st) {
        release_parts(out->parts, s);
        return st;
    };
    for (int j = 0; j < na; ++j) {
        const hc_index* ix = idx[j];
        const int a = q->atoms[j].var0, b = q->atoms[j].var1;
        const bool unary = b == (int)HC_UNARY;
        const int first = (unary || rank[a] < rank[b]) ? a : b, second = unary ? -1 : (first == a ? b : a);
        const uint32_t need_ao = (unary || rank[a] < rank[b]) ? 0u : 1u;
        if (ix->attr_order != need_ao)
            return bail(fail(HC_ERR_ARG, "run_join: an index's attr_order does not sort its atom in loop order"));
        DAtom& d = P.atom[j];
        const uint32_t pa = prm->shares[first], pb = unary ? 1u : prm->shares[second];
        d.pb = pb;
        d.stride_f = (uint32_t)stride[first];
        d.share_f = pa;
        d.stride_s = unary ? 1u : (uint32_t)stride[second];
        d.share_s = pb;
        d.lev_first = rank[first];
        d.lev_second = unary ? -1 : rank[second];
        if ((uint64_t)pa * pb == 1) {
            d.v1 = ix->d_v1;
            d.o1 = ix->d_o1;
            d.v2 = ix->d_v2;
            d.l1s = nullptr;
            d.l1_whole = (uint32_t)ix->l1;
            d.v1pos = ix->d_v1pos;
            d.v1pos_n = ix->v1pos_n;
            d.g1 = ix->d_g1;
            d.g2 = ix->d_g2;
        } else if (partition_bytes) {
            // estimate only: keys, levels and directory of the partitioned copy,
            // its V1 position map, plus the radix pass temporaries
            const uint64_t n = ix->n, np = (uint64_t)pa * pb;
            *partition_bytes += n * (8 + 8 + 4 + 4 + 4) + (np + 1) * 8 + ((n + 4095) / 4096) * 256 * 8 + 4096;
            const bool map = pb == 1 && v1pos_eligible(n, ix->max_first);
            if (map) *partition_bytes += ((uint64_t)ix->max_first + 1) * 4;
            *partition_bytes += n * 16 * (map ? 1 : 2);  // bucket directories of V2 (and V1 without a map)
            d.l1s = nullptr;
        } else {
            // atoms of one index with the same shares and hash seeds on both
            // attributes (a seed is immaterial under one share) read one
            // partitioned copy: e.g. the triangle's R(x,y) and T(x,z) on E+
            const uint32_t seed_a = prm->seeds[first], seed_b = (unary || pb == 1) ? 0u : prm->seeds[second];
            hc_partitioned* part = nullptr;
            for (size_t k = 0; k < out->parts.size() && !part; ++k) {
                hc_partitioned* c = out->parts[k];
                if (out->part_src[k] == ix && c->pa == pa && c->pb == pb && c->seed_a == seed_a &&
                    c->seed_b == seed_b)
                    part = c;
            }
            if (!part) {
                const hc_status st = partition_impl(ix, seed_a, pa, seed_b, pb, s, &part);
                if (st != HC_OK) return bail(st);
                out->parts.push_back(part);
                out->part_src.push_back(ix);
            }
            d.v1 = part->d_v1;
            d.o1 = part->d_o1;
            d.v2 = part->d_v2;
            d.l1s = part->d_lvl1_start;
            d.v1pos = part->d_v1pos;
            d.v1pos_n = part->v1pos_n;
            d.g1 = part->d_g1;
            d.g2 = part->d_g2;
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
    for (int L = 0; L < nv; ++L) {
        out->shape_s = std::max(out->shape_s, P.nsrc[L]);
        if (L >= 1) out->shape_o = std::max(out->shape_o, P.nopen[L]);
        for (int qq = 0; qq < P.nsrc[L]; ++qq) {
            const DAtom& a = P.atom[P.src_atom[L][qq]];
            P.src_ec[L][qq] = (P.src_top[L][qq] || a.lev_first == 0) ? 1 : 0;
            P.src_f[L][qq] = a.lev_first;
            P.src_slot[L][qq] = a.slot;
        }
    }
    // the search kernels sum up to 32 bindings' candidate counts in 32 bits:
    // at every loop after the first, the shortest of its lists must stay
    // below 2^27 (a top-level list is at most the relation's l1 long, a
    // sub-list at most its longest run)
    for (int L = 1; L < nv; ++L) {
        uint64_t bound = UINT64_MAX;
        for (int qq = 0; qq < P.nsrc[L]; ++qq) {
            const hc_index* ix = idx[P.src_atom[L][qq]];
            bound = std::min<uint64_t>(bound, P.src_top[L][qq] ? ix->l1 : ix->max_run);
        }
        if (P.nsrc[L] > 0 && bound >= MAX_LIST_LEN)
            return bail(fail(HC_ERR_CAPACITY, "run_join: a loop's shortest list can reach 2^27 values (a key with "
                                              "2^27 or more rows), beyond the search kernels' 32-bit candidate "
                                              "counts"));
    }
    P.dir_min = prm->dir_min == 0 ? DIR_MIN : std::max(prm->dir_min, DIR_MIN);
    P.merge_min = prm->merge_min ? prm->merge_min : 32;
    P.pair_min = prm->pair_min ? prm->pair_min : 32;
    P.merge_ratio = prm->merge_ratio ? prm->merge_ratio : 4;
    P.slice_grain = prm->slice_grain == 0xFFFFFFFFu ? 0 : (prm->slice_grain ? prm->slice_grain : 256);
    // query rewriting (Sec. 5.1): the last loop's lists fixed before the loop
    // above it ("far": top lists, lists of atoms opened by loop 1 or at least
    // two loops up) are intersected once per binding of loop nv-3
    P.lift = 0;
    P.far0 = -1;
    P.far_mask = 0;
    P.arena_words = 0;
    if (nv >= 4 && !out->stats && !(prm->flags & HC_FLAG_NO_LIFT)) {
        const int Ls = nv - 1;
        int nfar = 0;
        for (int qq = 0; qq < P.nsrc[Ls]; ++qq) {
            if (P.src_ec[Ls][qq] || P.src_f[Ls][qq] <= Ls - 2) {
                P.far_mask |= 1u << qq;
                if (P.far0 < 0) P.far0 = qq;
                ++nfar;
            }
        }
        if (nfar >= 2) {
            P.lift = 1;
            P.arena_words = std::min<uint32_t>(prm->lift_arena ? prm->lift_arena : LIFT_ARENA_WORDS, 1u << 26);
        } else {
            P.far0 = -1;
            P.far_mask = 0;
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
    out->cand_bound = cand_bound;
    return HC_OK;
}

// Device buffers of one query's loop-1 pass.  The first group is needed by
// the search; the second only during the loop-1 pass.
struct Level1 {
    DPlan* d_plan = nullptr;
    uint32_t *e_cell = nullptr, *e_x = nullptr, *e_rng = nullptr, *e_split = nullptr;
    uint64_t* uoff = nullptr;
    uint32_t *cand = nullptr, *flags = nullptr;
    uint64_t *candoff = nullptr, *flagoff = nullptr, *e_units = nullptr;
};

template <class Alloc>
hc_status alloc_level1_keep(const QueryPlan& qp, Alloc& a, Level1* L) {
    const uint64_t cb = qp.cand_bound;
    HC_TRY(a.get(&L->d_plan, 1));
    HC_TRY(a.get(&L->e_cell, cb));
    HC_TRY(a.get(&L->e_x, cb));
    HC_TRY(a.get(&L->e_rng, cb * 2 * MAXOPEN));
    HC_TRY(a.get(&L->e_split, cb));
    HC_TRY(a.get(&L->uoff, cb + 1));
    return HC_OK;
}

template <class Alloc>
hc_status alloc_level1_temp(const QueryPlan& qp, Alloc& a, Level1* L) {
    const uint64_t cb = qp.cand_bound;
    HC_TRY(a.get(&L->cand, qp.ncells));
    HC_TRY(a.get(&L->candoff, qp.ncells + 1));
    HC_TRY(a.get(&L->flags, cb));
    HC_TRY(a.get(&L->flagoff, cb + 1));
    HC_TRY(a.get(&L->e_units, cb));
    return HC_OK;
}

// Loop 1 of every cell (enqueued, no host waits): candidates per cell, the
// flat probe, compaction into entries and the entries' unit offsets.  The
// plan must already be in L.d_plan.
hc_status enqueue_level1(const QueryPlan& qp, const Level1& L, JoinCtl* ctl, cudaStream_t s,
                         uint64_t* cell_prof = nullptr) {
    const int tpb = 256;
    const uint64_t ncells = qp.ncells, cb = qp.cand_bound;
    l0_count_kernel<<<(unsigned)std::min<uint64_t>((ncells + tpb - 1) / tpb, 4096), tpb, 0, s>>>(L.d_plan, L.cand, ctl,
                                                                                                 qp.stats, cell_prof);
    if (cudaError_t le = launch_check()) return cuda_fail(le, "l0_count_kernel");
    HC_TRY(exclusive_scan_u32_to_u64(L.cand, L.candoff, ncells, nullptr, &ctl->err, s));
    const unsigned pgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((cb + tpb - 1) / tpb, (uint64_t)num_sms() * 16));
    l0_probe_kernel<false><<<pgrid, tpb, 0, s>>>(L.d_plan, L.candoff, cb, L.flags, nullptr, nullptr, nullptr, nullptr,
                                                 nullptr, nullptr, ctl);
    if (cudaError_t le = launch_check()) return cuda_fail(le, "l0_probe_kernel");
    HC_TRY(exclusive_scan_u32_to_u64(L.flags, L.flagoff, cb, nullptr, &ctl->err, s));
    l0_probe_kernel<true><<<pgrid, tpb, 0, s>>>(L.d_plan, L.candoff, cb, L.flags, L.flagoff, L.e_cell, L.e_x, L.e_rng,
                                                L.e_units, L.e_split, ctl);
    if (cudaError_t le = launch_check()) return cuda_fail(le, "l0_probe_kernel");
    entries_total_kernel<<<1, 1, 0, s>>>(L.flagoff, L.candoff, (uint32_t)ncells, cb, ctl);
    if (cudaError_t le = launch_check()) return cuda_fail(le, "entries_total_kernel");
    HC_TRY(exclusive_scan_u64(L.e_units, L.uoff, cb, &ctl->n_entries, &ctl->err, s));
    return HC_OK;
}

// Words of the lifted-list arena of a search launch: arena_words for every
// warp either kind of search kernel (count or write) keeps resident.
static uint64_t lift_arena_words(const QueryPlan& qp) {
    if (!qp.P.lift) return 0;
    const uint64_t blocks = (uint64_t)std::max(gj_grid_any(qp.nv, qp.shape_s, qp.shape_o, false, qp.threads),
                                               gj_grid_any(qp.nv, qp.shape_s, qp.shape_o, true, qp.threads));
    return blocks * (uint64_t)(qp.threads / 32) * qp.P.arena_words;
}

hc_status join_footprint_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm,
                              uint64_t* bytes) {
    if (!bytes) return fail(HC_ERR_ARG, "join_footprint: NULL argument");
    QueryPlan qp;
    uint64_t part_bytes = 0;
    HC_TRY(plan_query(q, idx, prm, nullptr, &qp, &part_bytes));
    // with partitioned atoms the bound uses their row counts (as run_join does)
    uint64_t cb = 1;
    {
        uint64_t c = UINT64_MAX;
        for (int q0 = 0; q0 < qp.P.nsrc[0]; ++q0) {
            const int j = qp.P.src_atom[0][q0];
            const DAtom& d = qp.P.atom[j];
            const uint64_t rep = qp.ncells / ((uint64_t)d.share_f * d.share_s);
            const uint64_t rows = ((uint64_t)d.share_f * d.share_s > 1) ? idx[j]->n : idx[j]->l1;
            c = std::min<uint64_t>(c, rep * rows);
        }
        cb = std::max<uint64_t>(c, 1);
    }
    // loop-1 buffers (kept and temporary), per-cell arrays, scan look-back
    // words and the control block
    const uint64_t per_cand = 4 + 4 + 4 * 2 * MAXOPEN + 4 + 8 + 4 + 8 + 8;
    *bytes = part_bytes + cb * per_cand + qp.ncells * (4 + 8 + 8) + ((cb + 2047) / 2048) * 8 * 3 + 65536 +
             4 * lift_arena_words(qp);
    return HC_OK;
}

// Host delivery of a materialized result (hc_run_join_to_host).
struct HostOut {
    uint32_t* h_tuples;
    uint64_t capacity;
    uint64_t* count_out;
};

// Search launches of a host-delivered join (consecutive item ranges).
constexpr uint64_t HOST_SEGMENTS = 16;

// Per-call host side of the segments: a stream for the copies to the host,
// one event per segment, and pinned host copies of the segments' ranges.
struct HostSegs {
    cudaStream_t copy = nullptr;
    std::vector<cudaEvent_t> ev;
    Seg* h = nullptr;
    ~HostSegs() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (copy) cudaStreamDestroy(copy);
        if (h) cudaFreeHost(h);
    }
    hc_status init(uint32_t n) {
        HC_CUDA_TRY(cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking));
        HC_CUDA_TRY(cudaMallocHost((void**)&h, n * sizeof(Seg)));
        ev.assign(n, nullptr);
        for (auto& e : ev) HC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return HC_OK;
    }
    // after segment k's compaction on s: its range to the host, then the event
    hc_status mark(uint32_t k, const Seg* d, cudaStream_t s) {
        HC_CUDA_TRY(cudaMemcpyAsync(h + k, d, sizeof(Seg), cudaMemcpyDeviceToHost, s));
        HC_CUDA_TRY(cudaEventRecord(ev[k], s));
        return HC_OK;
    }
    hc_status wait(uint32_t k, Seg* out) {
        HC_CUDA_TRY(cudaEventSynchronize(ev[k]));
        *out = h[k];
        return HC_OK;
    }
};

hc_status run_join_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm, cudaStream_t s,
                        hc_result** out, const HostOut* host) {
    if (!out) return fail(HC_ERR_ARG, "run_join: out is NULL");
    *out = nullptr;
    QueryPlan qp;
    HC_TRY(plan_query(q, idx, prm, s, &qp));
    const int nv = qp.nv, shape_s = qp.shape_s, shape_o = qp.shape_o, threads = qp.threads, stats = qp.stats;
    const uint32_t grain = qp.grain;
    const uint64_t ncells = qp.ncells;

    hc_result* R = new hc_result();
    R->stream = s;
    R->n_vars = nv;
    R->n_cells = ncells;
    R->parts = qp.parts;
    qp.parts.clear();
    auto bail = [&](hc_status st) {
        result_release(R);
        return st;
    };
    {
        void* p;
        if (dev_alloc(&p, sizeof(JoinCtl), s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_ctl = (JoinCtl*)p;
    }
    JoinCtl* ctl = R->d_ctl;
    if (cudaMemsetAsync(ctl, 0, sizeof(JoinCtl), s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    if (prm->flags & HC_FLAG_CELL_COUNTS) {
        void* p;
        if (dev_alloc(&p, ncells * 8, s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_cell_counts = (uint64_t*)p;
        if (cudaMemsetAsync(p, 0, ncells * 8, s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    }
    if (prm->flags & HC_FLAG_CELL_PROFILE) {
        void* p;
        if (dev_alloc(&p, ncells * 16, s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_cell_prof = (uint64_t*)p;
        if (cudaMemsetAsync(p, 0, ncells * 16, s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    }

    Scratch tmp(s);
    Level1 L;
    hc_status st;
    if ((st = alloc_level1_keep(qp, tmp, &L)) != HC_OK) return bail(st);
    if ((st = alloc_level1_temp(qp, tmp, &L)) != HC_OK) return bail(st);
    if (cudaMemcpyAsync(L.d_plan, &qp.P, sizeof(DPlan), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "plan copy"));
    if ((st = enqueue_level1(qp, L, ctl, s, R->d_cell_prof)) != HC_OK) return bail(st);
    const uint64_t* uoff = L.uoff;

    GjArgs g{L.d_plan, L.e_cell, L.e_x,   L.e_rng, L.e_split, uoff,    grain,   ctl, 0, R->d_cell_counts,
             nullptr,  nullptr,  nullptr, stats,   threads,   nullptr, 0};
    if (const uint64_t aw = lift_arena_words(qp)) {
        if ((st = tmp.get(&g.arena, aw)) != HC_OK) return bail(st);
    }
    g.cell_prof = R->d_cell_prof;
    const bool timed = (prm->flags & HC_FLAG_TIME_KERNELS) != 0;
    // one search launch, bracketed by events when timed
    auto search = [&](bool mat) -> hc_status {
        if (timed) HC_TRY(time_mark(R, false, s));
        HC_TRY(launch_any(nv, shape_s, shape_o, mat, g, s));
        R->n_search++;
        if (timed) HC_TRY(time_mark(R, true, s));
        return HC_OK;
    };
    if (prm->mode == HC_MODE_COUNT && !host) {
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
    uint64_t total = 0;
    bool written = false;
    if (prm->out_capacity > 0 || host) {
        // single pass into pool chunks, in nseg search launches over
        // consecutive item ranges, each followed by the in-place compaction
        // of the chunks it filled; the slack covers every warp's last, partly
        // filled chunk of every launch
        const uint64_t warps = (uint64_t)gj_grid_any(nv, shape_s, shape_o, true, threads) * (threads / 32);
        const uint32_t nseg =
            host ? (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(HOST_SEGMENTS, nitems / 64)) : 1u;
        const uint64_t cap = host ? host->capacity : prm->out_capacity;
        const uint64_t n_chunks64 = (cap + OUT_CHUNK - 1) / OUT_CHUNK + (uint64_t)nseg * warps;
        if (n_chunks64 >= 0xFFFFFFFFull) return bail(fail(HC_ERR_CAPACITY, "run_join: output capacity too large"));
        const uint32_t n_chunks = (uint32_t)n_chunks64;
        uint32_t *pool = nullptr, *chunk_fill, *is_partial, *pfill, *pslot, *ptmp, *seg_ctr;
        uint64_t *prank, *poff;
        Seg* d_seg;
        {
            void* pp;
            if (dev_alloc(&pp, (size_t)n_chunks * OUT_CHUNK * nv * 4, s) != HC_OK) return bail(HC_ERR_OOM);
            pool = (uint32_t*)pp;
        }
        auto bail_pool = [&](hc_status e) {
            dev_free(pool, s);
            return bail(e);
        };
        if ((st = tmp.get(&chunk_fill, n_chunks)) != HC_OK || (st = tmp.get(&is_partial, n_chunks)) != HC_OK ||
            (st = tmp.get(&pfill, n_chunks)) != HC_OK || (st = tmp.get(&prank, (size_t)n_chunks + 1)) != HC_OK ||
            (st = tmp.get(&poff, (size_t)n_chunks + 1)) != HC_OK || (st = tmp.get(&pslot, warps + 1)) != HC_OK ||
            (st = tmp.get(&ptmp, (size_t)warps * OUT_CHUNK * nv)) != HC_OK || (st = tmp.get(&d_seg, nseg)) != HC_OK ||
            (st = tmp.get(&seg_ctr, nseg)) != HC_OK)
            return bail_pool(st);
        if (cudaMemsetAsync(seg_ctr, 0, nseg * sizeof(uint32_t), s) != cudaSuccess)
            return bail_pool(cuda_fail(cudaGetLastError(), "memset"));
        HostSegs hs;
        if (host && (st = hs.init(nseg)) != HC_OK) return bail_pool(st);
        g.out = pool;
        g.chunk_fill = chunk_fill;
        g.n_chunks = n_chunks;
        const unsigned cgrid = std::min<uint32_t>((n_chunks + 255) / 256, (uint32_t)num_sms() * 8);
        const unsigned bgrid = std::min<uint32_t>(n_chunks, (uint32_t)num_sms() * 16);
        for (uint32_t k = 0; k < nseg; ++k) {
            g.item_lo = (uint32_t)(nitems * k / nseg);
            g.item_hi = (uint32_t)(nitems * (k + 1) / nseg);
            g.item_ctr = seg_ctr + k;
            if ((st = search(true)) != HC_OK) return bail_pool(st);
            Seg* sk = d_seg + k;
            seg_mark_kernel<<<1, 1, 0, s>>>(ctl, n_chunks, k ? d_seg + k - 1 : nullptr, sk);
            if (cudaError_t le = launch_check()) return bail_pool(cuda_fail(le, "seg_mark_kernel"));
            chunk_class_kernel<<<cgrid, 256, 0, s>>>(chunk_fill, sk, is_partial, pfill);
            if (cudaError_t le = launch_check()) return bail_pool(cuda_fail(le, "chunk_class_kernel"));
            if ((st = exclusive_scan_u32_to_u64(is_partial, prank, n_chunks, &sk->n, &ctl->err, s)) != HC_OK ||
                (st = exclusive_scan_u32_to_u64(pfill, poff, n_chunks, &sk->n, &ctl->err, s)) != HC_OK)
                return bail_pool(st);
            save_partials_kernel<<<bgrid, 256, 0, s>>>(pool, chunk_fill, sk, prank, poff, (uint32_t)nv, ptmp, pslot,
                                                       &ctl->err);
            if (cudaError_t le = launch_check()) return bail_pool(cuda_fail(le, "save_partials_kernel"));
            move_donors_kernel<<<bgrid, 256, 0, s>>>(pool, chunk_fill, sk, prank, pslot, (uint32_t)nv, &ctl->err);
            if (cudaError_t le = launch_check()) return bail_pool(cuda_fail(le, "move_donors_kernel"));
            place_partials_kernel<<<(unsigned)num_sms() * 4, 256, 0, s>>>(pool, ptmp, sk, prank, poff, (uint32_t)nv,
                                                                          &ctl->err);
            if (cudaError_t le = launch_check()) return bail_pool(cuda_fail(le, "place_partials_kernel"));
            if (host && (st = hs.mark(k, sk, s)) != HC_OK) return bail_pool(st);
        }
        if (host) {
            // each segment's tuples go to the host as soon as its compaction is
            // done, on a second stream, while later segments run
            uint64_t off = 0;
            bool room = true;
            for (uint32_t k = 0; k < nseg; ++k) {
                Seg sk;
                if ((st = hs.wait(k, &sk)) != HC_OK) return bail_pool(st);
                if (off + sk.tuples > host->capacity) room = false;
                if (room && sk.tuples > 0 &&
                    cudaMemcpyAsync(host->h_tuples + off * nv, pool + (uint64_t)sk.cb * OUT_CHUNK * nv,
                                    sk.tuples * nv * 4, cudaMemcpyDeviceToHost, hs.copy) != cudaSuccess)
                    return bail_pool(cuda_fail(cudaGetLastError(), "result copy to host"));
                off += sk.tuples;
            }
            if (cudaStreamSynchronize(hs.copy) != cudaSuccess) return bail_pool(cuda_fail(cudaGetLastError(), "copy"));
            if ((st = read_ctl(R)) != HC_OK) return bail_pool(st);
            *host->count_out = R->h_ctl.total;
            dev_free(pool, s);
            result_release(R);
            if (!room || off != *host->count_out)
                return fail(HC_ERR_CAPACITY, "run_join_to_host: " + std::to_string(*host->count_out) +
                                                 " tuples do not fit a host buffer of " +
                                                 std::to_string(host->capacity));
            return HC_OK;
        }
        st = read_ctl(R);
        if (st != HC_OK) return bail_pool(st);
        total = R->h_ctl.total;
        if (!R->h_ctl.overflow) {
            R->d_tuples = pool;  // compacted in place: tuples [0, total) from chunk 0
            written = true;
        } else {
            // on overflow the item counts of the single pass place the tuples
            // of a second, deterministic emitting pass
            dev_free(pool, s);
        }
    } else {
        if ((st = search(false)) != HC_OK) return bail(st);
    }
    if (!written) {
        if ((st = exclusive_scan_u64(item_counts, item_base, nitems, nullptr, &ctl->err, s)) != HC_OK) return bail(st);
        if (cudaMemcpyAsync(&total, item_base + nitems, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "read total"));
        void* p;
        if (dev_alloc(&p, std::max<uint64_t>(total, 1) * nv * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_tuples = (uint32_t*)p;
    }
    if (written) {
        R->n_tuples = total;
        R->materialized = true;
        *out = R;
        return HC_OK;
    }
    g.pass = 1;
    g.chunk_fill = nullptr;
    g.n_chunks = 0;
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

hc_status run_join_to_host_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm,
                                uint32_t* h_tuples, uint64_t capacity, uint64_t* count_out, cudaStream_t s) {
    if (!count_out || (capacity > 0 && !h_tuples)) return fail(HC_ERR_ARG, "run_join_to_host: NULL argument");
    *count_out = 0;
    HostOut host{h_tuples, capacity, count_out};
    hc_result* R = nullptr;
    return run_join_impl(q, idx, prm, s, &R, &host);
}

// -------------------------------------------------------------- batches
// Shape classes of the batched kernel: (loops, lists per loop, atoms opened
// per loop) rounded up to the instantiated widths.
enum ShapeClass { SC_T = 0, SC_T4 = 1, SC_C = 2, SC_K = 3, SC_NONE = 4 };

static int shape_class(const QueryPlan& qp) {
    const bool wide = qp.shape_s > 2 || qp.shape_o > 2;
    if (qp.nv == 3) return wide ? SC_T4 : SC_T;
    if (qp.nv == 4) return wide ? SC_K : SC_C;
    return SC_NONE;
}

template <int NLA, int SA, int OA, int NLB, int SB, int OB>
hc_status launch_batch_kernel(const BQuery* q, uint32_t n, const uint64_t* item_off, uint32_t* ctr, uint32_t* arena,
                              uint32_t stride, cudaStream_t s) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_batch_kernel<NLA, SA, OA, NLB, SB, OB>, 128, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    gj_batch_kernel<NLA, SA, OA, NLB, SB, OB><<<per_sm * num_sms(), 128, 0, s>>>(q, n, item_off, ctr, arena, stride);
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

// (a, b) with a <= b; the kernel's shape 0 is class a, shape 1 class b.
static hc_status launch_batch_pair(int a, int b, const BQuery* q, uint32_t n, const uint64_t* item_off, uint32_t* ctr,
                                   uint32_t* arena, uint32_t stride, cudaStream_t s) {
    switch (a * 8 + b) {
        case SC_T * 8 + SC_T: return launch_batch_kernel<3, 2, 2, 3, 2, 2>(q, n, item_off, ctr, arena, stride, s);
        case SC_T4 * 8 + SC_T4: return launch_batch_kernel<3, 4, 4, 3, 4, 4>(q, n, item_off, ctr, arena, stride, s);
        case SC_C * 8 + SC_C: return launch_batch_kernel<4, 2, 2, 4, 2, 2>(q, n, item_off, ctr, arena, stride, s);
        case SC_K * 8 + SC_K: return launch_batch_kernel<4, 4, 4, 4, 4, 4>(q, n, item_off, ctr, arena, stride, s);
        case SC_T * 8 + SC_K: return launch_batch_kernel<3, 2, 2, 4, 4, 4>(q, n, item_off, ctr, arena, stride, s);
        case SC_T * 8 + SC_C: return launch_batch_kernel<3, 2, 2, 4, 2, 2>(q, n, item_off, ctr, arena, stride, s);
        case SC_C * 8 + SC_K: return launch_batch_kernel<4, 2, 2, 4, 4, 4>(q, n, item_off, ctr, arena, stride, s);
        case SC_T4 * 8 + SC_K: return launch_batch_kernel<3, 4, 4, 4, 4, 4>(q, n, item_off, ctr, arena, stride, s);
        default: return fail(HC_ERR_CAPACITY, "batch: this pair of query shapes is not built in");
    }
}

// Owned device memory with plain (non stream-ordered) allocation, so that a
// captured graph can replay the batch for as long as the batch lives.
struct OwnedAlloc {
    std::vector<void*>* list;
    template <typename T>
    hc_status get(T** p, size_t count) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(HC_ERR_OOM, "batch: device allocation failed");
        }
        list->push_back(v);
        *p = (T*)v;
        return HC_OK;
    }
};

}  // namespace hc

struct hc_batch {
    uint32_t n = 0;
    std::vector<hc::QueryPlan> plans;
    std::vector<hc::Level1> l1;
    std::vector<void*> mem;
    hc::JoinCtl* d_ctl = nullptr;
    hc::BQuery* d_q = nullptr;
    uint64_t* d_items = nullptr;
    uint64_t* d_item_off = nullptr;
    uint32_t* d_ctr = nullptr;
    hc::Level1 temp;  // loop-1 temporaries shared by the queries (sized by the largest)
    int class_a = 0, class_b = 0;
    bool all_shapes = false;  // more than two shape classes: gj_batch_all_kernel
    uint32_t* d_arena = nullptr;  // lifted lists (query rewriting), arena_stride words per warp
    uint32_t arena_stride = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
};

namespace hc {

void batch_release(hc_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaDeviceSynchronize();
    for (auto& qp : b->plans) release_parts(qp.parts, nullptr);
    for (void* p : b->mem) cudaFree(p);
    delete b;
}

hc_status batch_create(const hc_query* qs, const hc_index* const* idx_flat, const hc_join_params* prm, uint32_t n,
                       cudaStream_t s, hc_batch** out) {
    if (!out) return fail(HC_ERR_ARG, "batch: out is NULL");
    *out = nullptr;
    if (!qs || !idx_flat || !prm || n == 0 || n > 65536) return fail(HC_ERR_ARG, "batch: need 1..65536 queries");
    hc_batch* B = new hc_batch();
    B->n = n;
    B->plans.resize(n);
    B->l1.resize(n);
    auto bail = [&](hc_status st) {
        batch_release(B);
        return st;
    };
    OwnedAlloc A{&B->mem};
    size_t off = 0;
    int classes[2] = {-1, -1};
    uint64_t max_cb = 1, max_cells = 1;
    std::vector<BQuery> hq(n);
    for (uint32_t i = 0; i < n; ++i) {
        if (prm[i].mode != HC_MODE_COUNT) return bail(fail(HC_ERR_ARG, "batch: queries run in count mode"));
        hc_status st = plan_query(&qs[i], idx_flat + off, &prm[i], s, &B->plans[i]);
        if (st != HC_OK) return bail(st);
        if (B->plans[i].P.lift) B->arena_stride = std::max(B->arena_stride, B->plans[i].P.arena_words);
        off += qs[i].n_atoms;
        const int c = shape_class(B->plans[i]);
        if (c == SC_NONE) return bail(fail(HC_ERR_CAPACITY, "batch: queries of 3 or 4 variables are built in"));
        if (classes[0] < 0 || classes[0] == c)
            classes[0] = c;
        else if (classes[1] < 0 || classes[1] == c)
            classes[1] = c;
        else
            B->all_shapes = true;  // three or four shape classes: the all-shapes kernel
        if ((st = alloc_level1_keep(B->plans[i], A, &B->l1[i])) != HC_OK) return bail(st);
        max_cb = std::max(max_cb, B->plans[i].cand_bound);
        max_cells = std::max(max_cells, B->plans[i].ncells);
        if (cudaMemcpy(B->l1[i].d_plan, &B->plans[i].P, sizeof(DPlan), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "batch plan copy"));
    }
    if (classes[1] < 0) classes[1] = classes[0];
    B->class_a = std::min(classes[0], classes[1]);
    B->class_b = std::max(classes[0], classes[1]);
    {
        QueryPlan big;
        big.cand_bound = max_cb;
        big.ncells = max_cells;
        hc_status st = alloc_level1_temp(big, A, &B->temp);
        if (st != HC_OK) return bail(st);
    }
    hc_status st;
    if (B->arena_stride) {  // one arena per warp of the largest batched grid (16 blocks of 4 warps per SM)
        if ((st = A.get(&B->d_arena, (size_t)num_sms() * 16 * 4 * B->arena_stride)) != HC_OK) return bail(st);
    }
    if ((st = A.get(&B->d_ctl, n)) != HC_OK || (st = A.get(&B->d_q, n)) != HC_OK ||
        (st = A.get(&B->d_items, n)) != HC_OK || (st = A.get(&B->d_item_off, (size_t)n + 1)) != HC_OK ||
        (st = A.get(&B->d_ctr, 1)) != HC_OK)
        return bail(st);
    for (uint32_t i = 0; i < n; ++i) {
        const Level1& L = B->l1[i];
        const int cls = shape_class(B->plans[i]);
        hq[i] = BQuery{L.d_plan, L.e_cell, L.e_x, L.e_rng, L.e_split, L.uoff, B->d_ctl + i, B->plans[i].grain,
                       (uint32_t)(B->all_shapes ? cls : (cls == B->class_a ? 0 : 1))};
    }
    if (cudaMemcpy(B->d_q, hq.data(), n * sizeof(BQuery), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "batch table copy"));
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "batch partition sync"));
    *out = B;
    return HC_OK;
}

static hc_status batch_enqueue(hc_batch* B, cudaStream_t s) {
    HC_CUDA_TRY(cudaMemsetAsync(B->d_ctl, 0, B->n * sizeof(JoinCtl), s));
    HC_CUDA_TRY(cudaMemsetAsync(B->d_ctr, 0, sizeof(uint32_t), s));
    for (uint32_t i = 0; i < B->n; ++i) {
        Level1 L = B->l1[i];
        L.cand = B->temp.cand;
        L.candoff = B->temp.candoff;
        L.flags = B->temp.flags;
        L.flagoff = B->temp.flagoff;
        L.e_units = B->temp.e_units;
        HC_TRY(enqueue_level1(B->plans[i], L, B->d_ctl + i, s));
    }
    batch_items_kernel<<<(B->n + 255) / 256, 256, 0, s>>>(B->d_q, B->n, B->d_items);
    HC_CUDA_TRY(launch_check());
    HC_TRY(exclusive_scan_u64(B->d_items, B->d_item_off, B->n, nullptr, &B->d_ctl[0].err, s));
    if (B->all_shapes) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_batch_all_kernel, 128, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        gj_batch_all_kernel<<<per_sm * num_sms(), 128, 0, s>>>(B->d_q, B->n, B->d_item_off, B->d_ctr, B->d_arena,
                                                               B->arena_stride);
        HC_CUDA_TRY(launch_check());
        return HC_OK;
    }
    return launch_batch_pair(B->class_a, B->class_b, B->d_q, B->n, B->d_item_off, B->d_ctr, B->d_arena,
                             B->arena_stride, s);
}

hc_status batch_launch(hc_batch* B, cudaStream_t s) {
    if (!B) return fail(HC_ERR_ARG, "batch: NULL");
    B->last_stream = s;
    if (B->exec) {
        HC_CUDA_TRY(cudaGraphLaunch(B->exec, s));
        return HC_OK;
    }
    return batch_enqueue(B, s);
}

hc_status batch_capture(hc_batch* B, cudaStream_t s) {
    if (!B) return fail(HC_ERR_ARG, "batch: NULL");
    if (s == nullptr) return fail(HC_ERR_ARG, "batch: graph capture needs a created (non-default) stream");
    if (B->exec) return HC_OK;
    HC_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    hc_status st = batch_enqueue(B, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != HC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&B->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    B->graph = g;
    return HC_OK;
}

hc_status batch_counts(hc_batch* B, uint64_t* counts) {
    if (!B || !counts) return fail(HC_ERR_ARG, "batch: NULL argument");
    std::vector<JoinCtl> h(B->n);
    HC_CUDA_TRY(cudaStreamSynchronize(B->last_stream));
    HC_CUDA_TRY(cudaMemcpy(h.data(), B->d_ctl, B->n * sizeof(JoinCtl), cudaMemcpyDeviceToHost));
    for (uint32_t i = 0; i < B->n; ++i) {
        if (h[i].err & DEV_ERR_TIMEOUT) return fail(HC_ERR_TIMEOUT, "batch: a bounded device wait gave up");
        counts[i] = h[i].total;
    }
    return HC_OK;
}

}  // namespace hc
