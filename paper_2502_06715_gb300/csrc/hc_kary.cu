// Relations of arity 1..3: the k-level CoCo index (Sec. 4, one level
// (V_r, O_r) per attribute) and Generic Join over it (Sec. 5), for
// hypergraph queries such as LW and CT (Table "Queries").
//
// Build.  The rows are sorted lexicographically in level order, then one
// scan over the sorted rows writes every level: row i opens an entry of
// level d when its prefix of length d+1 differs from row i-1's, so each
// level's entries are counted with ballots and placed by a decoupled
// look-back (one per level with offsets).  When the levels' value bits add
// up to at most 64, a row is one packed 64-bit key and the sort is the
// library's LSD radix sort of 64-bit keys (the binary index builder, with
// the key's high and low words as first and second attribute).  Otherwise
// the rows are sorted one level at a time, last level first: each pass
// sorts (level value, position in the previous order) pairs, which orders
// by the level value and keeps the previous order among equal values.
//
// Partitioning (Sec. 4, "Preprocessor").  With HyperCube shares the rows
// are sorted by partition id first (the mixed radix of the columns' hash
// identifiers), and a change of partition opens an entry of every level, so
// the levels are the partitions' tries concatenated; the scan records where
// each partition starts in the rows (B^pref) and in level 0.
//
// Join.  Loop 0 intersects the top levels of the atoms holding its variable
// in a flat pass over the loop-0 candidates of all HyperCube cells (in each
// cell the shortest list of the partitions its coordinates select), one
// thread per candidate; every match ("entry") records its cell, the
// level-1 ranges of the atoms it opens and its number of loop-1
// candidates.  The later loops run in a persistent kernel: a warp takes a
// work item (a range of loop-1 candidates, over consecutive entries) from
// an atomic counter and walks the remaining loops depth first.  At each
// loop it holds up to 32 parent bindings and flattens their candidates
// over its lanes, 32 a round; a candidate is an element of its parent's
// shortest list (Sec. 5.2: iterate the smallest set, search the others)
// and is searched in the parent's other lists through their bucket
// directories (or a direct position map of a top level); matches are
// compacted into the next loop's bindings.  At the last loop a parent with
// many candidates is searched by the whole warp instead, 128 candidates an
// iteration with its lists' bounds read once (kpair).  A binding keeps, for
// each list it matched that has a deeper level, the range of its children
// there (the level restriction of Sec. 5), and the index of its parent, so
// that a later loop finds the range an earlier loop opened by walking up
// the parents.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/honeycomb_kary.h"
#include "hc_internal.cuh"

struct hc_kindex {
    uint64_t n = 0;
    uint32_t arity = 0;
    uint8_t level_cols[HC_KMAX_ARITY] = {0, 0, 0};
    bool packed = false;
    uint64_t len[HC_KMAX_ARITY] = {0, 0, 0};
    uint32_t maxv[HC_KMAX_ARITY] = {0, 0, 0};  // largest value of each level
    uint32_t* d_v[HC_KMAX_ARITY] = {nullptr, nullptr, nullptr};
    uint32_t* d_o[HC_KMAX_ARITY] = {nullptr, nullptr, nullptr};
    // level-0 position map: pos[v] = position of v in V_0, or V1POS_NONE
    uint32_t* d_v0pos = nullptr;
    uint32_t v0pos_n = 0;
    // bucket directory of each level's runs (level 0: one run, built when
    // there is no position map; level d >= 1: the runs of O_{d-1})
    uint4* d_g[HC_KMAX_ARITY] = {nullptr, nullptr, nullptr};
    // HyperCube partitions (Sec. 4, "Preprocessor"): the share and seed of
    // each column, n_parts their product.  Partitioned (n_parts > 1), the
    // levels concatenate the partitions' tries in partition order; d_bpref[p]
    // is partition p's first row (B^pref) and d_l0start[p] its first level-0
    // entry, both [n_parts + 1]; h_l0start is the host copy of d_l0start.
    uint32_t n_parts = 1;
    uint32_t pshare[HC_KMAX_ARITY] = {1, 1, 1};
    uint32_t pseed[HC_KMAX_ARITY] = {0, 0, 0};
    uint32_t* d_bpref = nullptr;
    uint32_t* d_l0start = nullptr;
    std::vector<uint32_t> h_l0start;
    float ms_sort = 0.f, ms_levels = 0.f;
    bool stats_only = false;  // sizes only (planning), no device arrays
};

namespace hc {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

// Device allocations released (stream-ordered) when the holder goes.
struct KScratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit KScratch(cudaStream_t st) : s(st) {}
    ~KScratch() {
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

int grid_of(uint64_t n, int threads, int per_sm) {
    const uint64_t want = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)num_sms() * per_sm;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, cap));
}

uint32_t bit_width(uint32_t v) { return v == 0 ? 0 : 32 - __builtin_clz(v); }

// ==================================================================== build

struct KBuildCtl {
    uint32_t err;
    uint32_t dup;
    uint32_t maxv[HC_KMAX_ARITY];  // per column of the rows
    uint32_t tile_counter;
    uint32_t len[HC_KMAX_ARITY - 1];  // l_d of the levels with offsets
};

// Where level d of a row comes from: column col[d] of the row, or bits
// [shift[d], shift[d] + width) of a packed key (mask[d] = 2^width - 1).
struct KLayout {
    uint32_t k;
    uint32_t col[HC_KMAX_ARITY];
    uint32_t shift[HC_KMAX_ARITY];
    uint64_t mask[HC_KMAX_ARITY];
};

// Partition id of a row from its level values (Sec. 4): the mixed-radix
// number of the columns' identifiers s_c = h_c(x_c), column 0 most
// significant; by level d, weight[d] is the radix weight of level d's column.
struct KPart {
    uint32_t np;
    uint32_t share[HC_KMAX_ARITY], seed[HC_KMAX_ARITY], weight[HC_KMAX_ARITY];
};

template <int K>
__host__ __device__ __forceinline__ uint32_t kpid(const KPart& P, const uint32_t (&c)[K]) {
    uint32_t p = 0;
#pragma unroll
    for (int d = 0; d < K; ++d) p += share_of(c[d], P.seed[d], P.share[d]) * P.weight[d];
    return p;
}

__global__ void kcolmax_kernel(const uint32_t* __restrict__ rows, uint64_t n, uint32_t k, KBuildCtl* ctl) {
    uint32_t m[HC_KMAX_ARITY] = {0, 0, 0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t* r = rows + i * k;
#pragma unroll
        for (int c = 0; c < HC_KMAX_ARITY; ++c)
            if (c < (int)k) m[c] = max(m[c], r[c]);
    }
#pragma unroll
    for (int c = 0; c < HC_KMAX_ARITY; ++c) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) m[c] = max(m[c], __shfl_xor_sync(FULL, m[c], d));
        if (lane_id() == 0 && c < (int)k) atomicMax(&ctl->maxv[c], m[c]);
    }
}

// Rows -> packed keys, stored as (high word, low word) pairs; a partitioned
// build puts the row's partition id above the levels, at bit pid_shift.
__global__ void kpack_kernel(const uint32_t* __restrict__ rows, uint64_t n, KLayout L, KPart Pt, uint32_t pid_shift,
                             uint2* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t* r = rows + i * L.k;
        uint64_t key = 0;
        uint32_t pid = 0;
#pragma unroll
        for (int d = 0; d < HC_KMAX_ARITY; ++d)
            if (d < (int)L.k) {
                const uint32_t x = r[L.col[d]];
                key |= (uint64_t)x << L.shift[d];
                if (Pt.np > 1) pid += share_of(x, Pt.seed[d], Pt.share[d]) * Pt.weight[d];
            }
        if (Pt.np > 1) key |= (uint64_t)pid << pid_shift;
        out[i] = make_uint2((uint32_t)(key >> 32), (uint32_t)key);
    }
}

// Pairs (value of column `col` of row perm[i], i) for one level pass of the
// unpacked sort (perm NULL: the identity).
__global__ void kperm_pairs_kernel(const uint32_t* __restrict__ rows, uint64_t n, uint32_t k, uint32_t col,
                                   const uint32_t* __restrict__ perm, uint2* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = perm ? perm[i] : i;
        out[i] = make_uint2(rows[r * k + col], (uint32_t)i);
    }
}

// Pairs (partition id of row perm[i], i): the last, most significant pass of
// a partitioned unpacked sort.
__global__ void kpid_pairs_kernel(const uint32_t* __restrict__ rows, uint64_t n, KLayout L, KPart Pt,
                                  const uint32_t* __restrict__ perm, uint2* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = perm ? perm[i] : i;
        uint32_t pid = 0;
#pragma unroll
        for (int d = 0; d < HC_KMAX_ARITY; ++d)
            if (d < (int)L.k) pid += share_of(rows[r * L.k + L.col[d]], Pt.seed[d], Pt.share[d]) * Pt.weight[d];
        out[i] = make_uint2(pid, (uint32_t)i);
    }
}

// After a pass sorted the pairs: the new order is the old order read at the
// positions the sorted keys carry in their low words.
__global__ void kperm_compose_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ perm_old,
                                     uint32_t* __restrict__ perm_new, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)keys[i];
        perm_new[i] = perm_old ? perm_old[j] : j;
    }
}

// The sorted rows: packed keys, or the rows read through the sorted order.
struct KSorted {
    const uint64_t* keys;
    const uint32_t* rows;
    const uint32_t* perm;
    KLayout L;
    KPart part;        // np > 1: rows are sorted by partition first
    uint32_t* bpref;   // partitioned: first row of each partition (others untouched)
    uint32_t* l0start; // partitioned: first level-0 entry of each partition
};

template <int K, bool PACKED>
__device__ __forceinline__ void load_levels(const KSorted& s, uint64_t i, uint32_t (&c)[K]) {
    if (PACKED) {
        const uint64_t key = s.keys[i];
#pragma unroll
        for (int d = 0; d < K; ++d) c[d] = (uint32_t)((key >> s.L.shift[d]) & s.L.mask[d]);
    } else {
        const uint64_t r = s.perm[i];
#pragma unroll
        for (int d = 0; d < K; ++d) c[d] = s.rows[r * K + s.L.col[d]];
    }
}

// Level scan.  A partitioned build (rows sorted by partition id first)
// treats a change of partition like a change at level 0: the row opens an
// entry of every level, and records itself as its partition's first row and
// that entry as the partition's first level-0 entry.  Rows are warp-striped as in the binary run-boundary scan:
// item j of lane q of warp w is row tile * KL_TILE + w * 32 * KL_ITEMS +
// 32 j + q, so the row before a lane-0 row is lane 31's row of the previous
// item.  fd = the first level at which a row differs from the row before
// (0 for row 0, K for an equal row: a repeat).  Row i opens an entry of
// every level d >= fd; an opened entry of level d < K-1 points at the row's
// entry of level d+1 (opened too), or at the row itself for d = K-2.
// Level K-1 is the last column of every row.  Warp d of each tile runs the
// look-back of level d; the tile holding the last row closes every level
// with O_d[l_d] = l_{d+1}.
constexpr int KL_THREADS = 256;
constexpr int KL_WARPS = KL_THREADS / 32;
constexpr int KL_ITEMS = 16;
constexpr int KL_TILE = KL_THREADS * KL_ITEMS;

template <int K, bool PACKED>
__global__ void __launch_bounds__(KL_THREADS) klevels_kernel(KSorted src, uint64_t n, uint32_t* __restrict__ v0,
                                                             uint32_t* __restrict__ v1, uint32_t* __restrict__ v2,
                                                             uint32_t* __restrict__ o0, uint32_t* __restrict__ o1,
                                                             uint64_t* __restrict__ status, uint64_t ntiles,
                                                             KBuildCtl* __restrict__ ctl, uint64_t wait_ns) {
    constexpr int NL = K - 1;              // levels with offsets
    constexpr int NLA = NL > 0 ? NL : 1;  // array extent
    __shared__ uint32_t wsum[NLA][KL_WARPS];
    __shared__ uint64_t s_excl[NLA];
    __shared__ uint32_t s_tile;
    uint32_t* const vv[3] = {v0, v1, v2};
    uint32_t* const oo[2] = {o0, o1};
    const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    // nothing once a sort pass before this scan gave up a wait
    if (tid == 0) s_tile = dev_err_set(&ctl->err) ? 0xFFFFFFFFu : atomicAdd(&ctl->tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile == 0xFFFFFFFFu) return;
    const uint64_t base = (uint64_t)tile * KL_TILE + (uint64_t)w * (KL_ITEMS * 32);
    const bool full = base + KL_ITEMS * 32 <= n;

    uint32_t c[KL_ITEMS][K];
#pragma unroll
    for (int j = 0; j < KL_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
        if (full || i < n) {
            load_levels<K, PACKED>(src, i, c[j]);
        } else {
#pragma unroll
            for (int d = 0; d < K; ++d) c[j][d] = 0;
        }
    }
    uint32_t carry[K];
#pragma unroll
    for (int d = 0; d < K; ++d) carry[d] = 0;
    if (lane == 0 && base > 0 && base < n) load_levels<K, PACKED>(src, base - 1, carry);
    const bool parted = src.part.np > 1;
    uint32_t carry_pid = 0;
    if (parted && lane == 0) carry_pid = kpid<K>(src.part, carry);
    uint32_t pchg = 0;  // bit j: item j's row is the first of its partition

    uint32_t ball[KL_ITEMS][NLA];
    uint32_t cnt[NLA];
#pragma unroll
    for (int d = 0; d < NLA; ++d) cnt[d] = 0;
    bool dup = false;
#pragma unroll
    for (int j = 0; j < KL_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
        const bool valid = full || i < n;
        int fd = K;
#pragma unroll
        for (int d = K - 1; d >= 0; --d) {
            uint32_t prev = __shfl_up_sync(FULL, c[j][d], 1);
            if (lane == 0) prev = carry[d];
            if (c[j][d] != prev) fd = d;
        }
        if (i == 0) fd = 0;
        if (parted) {
            const uint32_t pc = kpid<K>(src.part, c[j]);
            uint32_t pp = __shfl_up_sync(FULL, pc, 1);
            if (lane == 0) pp = carry_pid;
            const uint32_t plast = __shfl_sync(FULL, pc, 31);
            if (lane == 0) carry_pid = plast;
            if (pc != pp) fd = 0;
            if (valid && (pc != pp || i == 0)) {
                pchg |= 1u << j;
                src.bpref[pc] = (uint32_t)i;
                if (K == 1) src.l0start[pc] = (uint32_t)i;
            }
        }
        dup |= valid && fd == K;
#pragma unroll
        for (int d = 0; d < NL; ++d) {
            ball[j][d] = __ballot_sync(FULL, valid && fd <= d);
            cnt[d] += __popc(ball[j][d]);
        }
        if (valid) vv[K - 1][i] = c[j][K - 1];  // the last level needs no offset
#pragma unroll
        for (int d = 0; d < K; ++d) {
            const uint32_t last = __shfl_sync(FULL, c[j][d], 31);
            if (lane == 0) carry[d] = last;
        }
    }
    if (__any_sync(FULL, dup) && lane == 0) atomicOr(&ctl->dup, 1u);
    if (NL == 0) return;

    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < NL; ++d) wsum[d][w] = cnt[d];
    }
    __syncthreads();
    if (w < (uint32_t)NL) {
        const int d = (int)w;
        const uint64_t tot = warp_sum64(lane < (uint32_t)KL_WARPS ? wsum[d][lane] : 0u);
        uint64_t* st = status + (uint64_t)d * ntiles + tile;
        if (lane == 0) st_relaxed(st, (tile == 0 ? LB_INC : LB_AGG) | tot);
        uint64_t excl = 0;
        if (tile != 0) {
            excl = warp_lookback(status + (uint64_t)d * ntiles, tile, &ctl->err, wait_ns);
            if (lane == 0) st_relaxed(st, LB_INC | (excl + tot));
        }
        if (lane == 0) s_excl[d] = excl;
    }
    __syncthreads();
    uint64_t pos[NLA];
#pragma unroll
    for (int d = 0; d < NL; ++d) {
        pos[d] = s_excl[d];
        for (uint32_t q = 0; q < w; ++q) pos[d] += wsum[d][q];
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < KL_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
#pragma unroll
        for (int d = 0; d < NL; ++d) {
            if (ball[j][d] >> lane & 1u) {  // flagged rows are valid rows
                const uint64_t e = pos[d] + __popc(ball[j][d] & lt);
                vv[d][e] = c[j][d];
                if (d == 0 && (pchg >> j & 1u)) src.l0start[kpid<K>(src.part, c[j])] = (uint32_t)e;
                const int d1 = d + 1 < NL ? d + 1 : d;
                const uint64_t child = d + 1 < NL ? pos[d1] + __popc(ball[j][d1] & lt) : i;
                oo[d][e] = (uint32_t)child;
            }
        }
#pragma unroll
        for (int d = 0; d < NL; ++d) pos[d] += __popc(ball[j][d]);
    }
    if (tid == 0 && (uint64_t)(tile + 1) * KL_TILE >= n) {
        uint64_t l[NLA + 1];
#pragma unroll
        for (int d = 0; d < NL; ++d) {
            uint64_t t = s_excl[d];
            for (int q = 0; q < KL_WARPS; ++q) t += wsum[d][q];
            l[d] = t;
        }
        l[NL] = n;
#pragma unroll
        for (int d = 0; d < NL; ++d) {
            oo[d][l[d]] = (uint32_t)l[d + 1];
            ctl->len[d] = (uint32_t)l[d];
        }
    }
}

// Level-0 position map: pos[V_0[i]] = i (values distinct, so each entry is
// written at most once).
__global__ void kpos_kernel(const uint32_t* __restrict__ v0, uint64_t l0, uint32_t* __restrict__ pos, uint32_t pos_n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < l0; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = v0[i];
        if (v < pos_n) pos[v] = (uint32_t)i;
    }
}

hc_status launch_levels(int k, bool packed, const KSorted& src, uint64_t n, uint32_t* const* v, uint32_t* const* o,
                        uint64_t* status, uint64_t ntiles, KBuildCtl* ctl, cudaStream_t s) {
    const unsigned grid = (unsigned)ntiles;
#define HC_KLEV(K, P) \
    klevels_kernel<K, P><<<grid, KL_THREADS, 0, s>>>(src, n, v[0], v[1], v[2], o[0], o[1], status, ntiles, ctl, \
                                                     wait_limit_ns())
    if (k == 1) {
        if (packed) HC_KLEV(1, true); else HC_KLEV(1, false);
    } else if (k == 2) {
        if (packed) HC_KLEV(2, true); else HC_KLEV(2, false);
    } else {
        if (packed) HC_KLEV(3, true); else HC_KLEV(3, false);
    }
#undef HC_KLEV
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

}  // namespace

void kindex_release(hc_kindex* x, cudaStream_t s) {
    if (!x) return;
    for (int d = 0; d < HC_KMAX_ARITY; ++d) {
        dev_free(x->d_v[d], s);
        dev_free(x->d_o[d], s);
        dev_free(x->d_g[d], s);
    }
    dev_free(x->d_v0pos, s);
    dev_free(x->d_bpref, s);
    dev_free(x->d_l0start, s);
    delete x;
}

hc_status build_kindex_impl(const uint32_t* d_rows, uint64_t n, uint32_t k, const uint8_t* level_cols,
                            const uint32_t* seeds, const uint32_t* shares, uint32_t flags, cudaStream_t s,
                            hc_kindex** out) {
    if (!out) return fail(HC_ERR_ARG, "build_kindex: out is NULL");
    *out = nullptr;
    if (k < 1 || k > HC_KMAX_ARITY) return fail(HC_ERR_ARG, "build_kindex: arity must be 1, 2 or 3");
    if (n > 0 && !d_rows) return fail(HC_ERR_ARG, "build_kindex: d_rows is NULL");
    if (n >= 0xFFFFFFFFull) return fail(HC_ERR_CAPACITY, "build_kindex: n must be below 2^32 - 1");
    uint8_t cols[HC_KMAX_ARITY] = {0, 1, 2};
    if (level_cols) {
        bool seen[HC_KMAX_ARITY] = {false, false, false};
        for (uint32_t d = 0; d < k; ++d) {
            if (level_cols[d] >= k || seen[level_cols[d]])
                return fail(HC_ERR_ARG, "build_kindex: level_cols must be a permutation of the columns");
            seen[level_cols[d]] = true;
            cols[d] = level_cols[d];
        }
    }
    uint64_t np = 1;
    if (shares) {
        for (uint32_t c = 0; c < k; ++c) {
            if (shares[c] == 0) return fail(HC_ERR_ARG, "build_kindex: shares must be at least 1");
            np *= shares[c];
            if (np > 65536) return fail(HC_ERR_ARG, "build_kindex: the shares' product must be at most 65536");
        }
    }
    hc_kindex* x = new hc_kindex();
    x->n = n;
    x->arity = k;
    for (uint32_t d = 0; d < k; ++d) x->level_cols[d] = cols[d];
    x->n_parts = (uint32_t)np;
    if (np > 1)
        for (uint32_t c = 0; c < k; ++c) {
            x->pshare[c] = shares[c];
            x->pseed[c] = seeds ? seeds[c] : 0u;
        }
    auto bail = [&](hc_status st) {
        kindex_release(x, s);
        return st;
    };
    void* p = nullptr;
    if (np > 1) {
        // every partition starts at 0 until the level scan says otherwise
        if (dev_alloc(&p, (np + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        x->d_bpref = (uint32_t*)p;
        if (dev_alloc(&p, (np + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        x->d_l0start = (uint32_t*)p;
        const int fill = n == 0 ? 0x00 : 0xFF;
        if (cudaMemsetAsync(x->d_bpref, fill, (np + 1) * 4, s) != cudaSuccess ||
            cudaMemsetAsync(x->d_l0start, fill, (np + 1) * 4, s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "memset"));
        x->h_l0start.assign(np + 1, 0u);
    }
    if (n == 0) {
        for (uint32_t d = 0; d < k; ++d) {
            if (dev_alloc(&p, 4, s) != HC_OK) return bail(HC_ERR_OOM);
            x->d_v[d] = (uint32_t*)p;
            if (d + 1 < k) {
                if (dev_alloc(&p, 4, s) != HC_OK) return bail(HC_ERR_OOM);
                x->d_o[d] = (uint32_t*)p;
                if (cudaMemsetAsync(p, 0, 4, s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
            }
        }
        *out = x;
        return HC_OK;
    }

    hc_status st;
    KScratch tmp(s);
    KBuildCtl* ctl;
    if ((st = tmp.get(&ctl, 1)) != HC_OK) return bail(st);
    if (cudaMemsetAsync(ctl, 0, sizeof(KBuildCtl), s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "memset"));
    kcolmax_kernel<<<grid_of(n, 256, 4), 256, 0, s>>>(d_rows, n, k, ctl);
    if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "kcolmax_kernel"));
    KBuildCtl h;
    if (cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "build_kindex: column maxima"));

    KLayout L{};
    L.k = k;
    uint32_t bits[HC_KMAX_ARITY] = {0, 0, 0}, total_bits = 0;
    for (uint32_t d = 0; d < k; ++d) {
        L.col[d] = cols[d];
        x->maxv[d] = h.maxv[cols[d]];
        bits[d] = bit_width(x->maxv[d]);
        total_bits += bits[d];
        L.mask[d] = bits[d] >= 32 ? 0xFFFFFFFFull : ((1ull << bits[d]) - 1);
    }
    for (int d = (int)k - 1, sh = 0; d >= 0; --d) {
        L.shift[d] = bits[d] ? (uint32_t)sh : 0u;  // a level of zeros takes no bits (and no shift of 64)
        sh += (int)bits[d];
    }
    KPart Pt{};
    Pt.np = (uint32_t)np;
    for (uint32_t d = 0; d < k; ++d) {
        Pt.share[d] = x->pshare[cols[d]];
        Pt.seed[d] = x->pseed[cols[d]];
        uint32_t w = 1;
        for (uint32_t c = cols[d] + 1; c < k; ++c) w *= x->pshare[c];
        Pt.weight[d] = w;
    }
    const uint32_t pid_bits = bit_width((uint32_t)(np - 1));

    const bool timed = (flags & HC_BUILD_TIME_KERNELS) != 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    auto destroy_events = [&]() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    };
    if (timed) {
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                destroy_events();
                return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
            }
        cudaEventRecord(ev[0], s);
    }

    // ---- sort
    KSorted src{};
    src.L = L;
    src.part = Pt;
    src.bpref = x->d_bpref;
    src.l0start = x->d_l0start;
    hc_index* sorted = nullptr;  // holds the packed keys, sorted
    auto bail2 = [&](hc_status e) {
        if (sorted) index_release(sorted, s);
        destroy_events();
        return bail(e);
    };
    if (total_bits + pid_bits <= 64) {
        x->packed = true;
        uint2* pk;
        if ((st = tmp.get(&pk, n)) != HC_OK) return bail2(st);
        kpack_kernel<<<grid_of(n, 256, 8), 256, 0, s>>>(d_rows, n, L, Pt, total_bits, pk);
        if (cudaError_t le = launch_check()) return bail2(cuda_fail(le, "kpack_kernel"));
        if ((st = build_index_impl((const uint32_t*)pk, n, 0, BUILD_NO_DIRECTORIES, s, &sorted)) != HC_OK) return bail2(st);
        src.keys = sorted->d_keys;
    } else {
        uint2* pairs;
        uint32_t *pa, *pb;
        if ((st = tmp.get(&pairs, n)) != HC_OK || (st = tmp.get(&pa, n)) != HC_OK || (st = tmp.get(&pb, n)) != HC_OK)
            return bail2(st);
        const uint32_t* cur = nullptr;
        for (int d = (int)k - 1; d >= 0; --d) {
            kperm_pairs_kernel<<<grid_of(n, 256, 8), 256, 0, s>>>(d_rows, n, k, cols[d], cur, pairs);
            if (cudaError_t le = launch_check()) return bail2(cuda_fail(le, "kperm_pairs_kernel"));
            hc_index* pass = nullptr;
            if ((st = build_index_impl((const uint32_t*)pairs, n, 0, BUILD_NO_DIRECTORIES, s, &pass)) != HC_OK) return bail2(st);
            uint32_t* nxt = cur == pa ? pb : pa;
            kperm_compose_kernel<<<grid_of(n, 256, 8), 256, 0, s>>>(pass->d_keys, cur, nxt, n);
            cudaError_t le = launch_check();
            index_release(pass, s);
            if (le) return bail2(cuda_fail(le, "kperm_compose_kernel"));
            cur = nxt;
        }
        if (np > 1) {  // the partition id last: the most significant key
            kpid_pairs_kernel<<<grid_of(n, 256, 8), 256, 0, s>>>(d_rows, n, L, Pt, cur, pairs);
            if (cudaError_t le = launch_check()) return bail2(cuda_fail(le, "kpid_pairs_kernel"));
            hc_index* pass = nullptr;
            if ((st = build_index_impl((const uint32_t*)pairs, n, 0, BUILD_NO_DIRECTORIES, s, &pass)) != HC_OK)
                return bail2(st);
            uint32_t* nxt = cur == pa ? pb : pa;
            kperm_compose_kernel<<<grid_of(n, 256, 8), 256, 0, s>>>(pass->d_keys, cur, nxt, n);
            cudaError_t le = launch_check();
            index_release(pass, s);
            if (le) return bail2(cuda_fail(le, "kperm_compose_kernel"));
            cur = nxt;
        }
        src.rows = d_rows;
        src.perm = cur;
    }
    if (timed) cudaEventRecord(ev[1], s);

    // ---- levels: upper-bound arrays for the levels with offsets, exact for the last
    uint32_t* v[3] = {nullptr, nullptr, nullptr};
    uint32_t* o[2] = {nullptr, nullptr};
    for (uint32_t d = 0; d + 1 < k; ++d) {
        if ((st = tmp.get(&v[d], n)) != HC_OK || (st = tmp.get(&o[d], n + 1)) != HC_OK) return bail2(st);
    }
    if (dev_alloc(&p, n * 4, s) != HC_OK) return bail2(HC_ERR_OOM);
    x->d_v[k - 1] = (uint32_t*)p;
    v[k - 1] = x->d_v[k - 1];
    const uint64_t ntiles = (n + KL_TILE - 1) / KL_TILE;
    uint64_t* status;
    if ((st = tmp.get(&status, (k > 1 ? k - 1 : 1) * ntiles)) != HC_OK) return bail2(st);
    if (cudaMemsetAsync(status, 0, (k > 1 ? k - 1 : 1) * ntiles * sizeof(uint64_t), s) != cudaSuccess)
        return bail2(cuda_fail(cudaGetLastError(), "memset"));
    if ((st = launch_levels((int)k, x->packed, src, n, v, o, status, ntiles, ctl, s)) != HC_OK) return bail2(st);
    if (timed) cudaEventRecord(ev[2], s);
    if (cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return bail2(cuda_fail(cudaGetLastError(), "build_kindex: level scan"));
    if (sorted) {
        index_release(sorted, s);
        sorted = nullptr;
    }
    if (h.err & DEV_ERR_TIMEOUT) return bail2(fail(HC_ERR_TIMEOUT, "build_kindex: a look-back wait gave up"));
    if ((flags & HC_BUILD_CHECK_DUPLICATES) && h.dup)
        return bail2(fail(HC_ERR_DUPLICATE, "build_kindex: the relation holds a repeated row"));
    if (timed) {
        cudaEventElapsedTime(&x->ms_sort, ev[0], ev[1]);
        cudaEventElapsedTime(&x->ms_levels, ev[1], ev[2]);
    }
    destroy_events();

    // exact-size copies of the levels with offsets
    x->len[k - 1] = n;
    for (uint32_t d = 0; d + 1 < k; ++d) {
        const uint64_t l = h.len[d];
        if (l == 0 || l > n) return bail(fail(HC_ERR_CUDA, "build_kindex: level scan gave an invalid level size"));
        x->len[d] = l;
        if (dev_alloc(&p, l * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        x->d_v[d] = (uint32_t*)p;
        if (dev_alloc(&p, (l + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        x->d_o[d] = (uint32_t*)p;
        if (cudaMemcpyAsync(x->d_v[d], v[d], l * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(x->d_o[d], o[d], (l + 1) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "build_kindex: level copy"));
    }
    if (np > 1) {
        // the starts of empty partitions were left unwritten (~0): each takes
        // the start of the next partition, and entry np closes the last one
        std::vector<uint32_t> hb(np + 1);
        if (cudaMemcpyAsync(hb.data(), x->d_bpref, (np + 1) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(x->h_l0start.data(), x->d_l0start, (np + 1) * 4, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "build_kindex: partition starts"));
        hb[np] = (uint32_t)n;
        x->h_l0start[np] = (uint32_t)x->len[0];
        for (int64_t q = (int64_t)np - 1; q >= 0; --q) {
            if (hb[q] == 0xFFFFFFFFu) hb[q] = hb[q + 1];
            if (x->h_l0start[q] == 0xFFFFFFFFu) x->h_l0start[q] = x->h_l0start[q + 1];
        }
        if (cudaMemcpyAsync(x->d_bpref, hb.data(), (np + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(x->d_l0start, x->h_l0start.data(), (np + 1) * 4, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "build_kindex: partition starts"));
    }
    // a level-0 position map needs each level-0 value in one partition: the
    // deeper levels' columns unpartitioned
    bool v0_unique = true;
    for (uint32_t d = 1; d < k; ++d) v0_unique &= x->pshare[cols[d]] == 1;
    if (v0_unique && v1pos_eligible(n, x->maxv[0])) {
        const uint64_t dn = (uint64_t)x->maxv[0] + 1;
        if (dev_alloc(&p, dn * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        x->d_v0pos = (uint32_t*)p;
        x->v0pos_n = (uint32_t)dn;
        if (cudaMemsetAsync(x->d_v0pos, 0xFF, dn * 4, s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "memset"));
        kpos_kernel<<<grid_of(x->len[0], 256, 8), 256, 0, s>>>(x->d_v[0], x->len[0], x->d_v0pos, x->v0pos_n);
        if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "kpos_kernel"));
    }
    // bucket directories: level 0 as one run per partition (without a
    // position map), and every deeper level by the runs its parent level's
    // offsets mark
    if (x->d_v0pos == nullptr &&
        (st = build_directory(x->d_v[0], x->len[0], np > 1 ? x->d_l0start : nullptr, np > 1 ? np : x->len[0],
                              nullptr, nullptr, s, &x->d_g[0])) != HC_OK)
        return bail(st);
    for (uint32_t d = 1; d < k; ++d)
        if ((st = build_directory(x->d_v[d], x->len[d], x->d_o[d - 1], x->len[d - 1], nullptr, nullptr, s,
                                  &x->d_g[d])) != HC_OK)
            return bail(st);
    *out = x;
    return HC_OK;
}

// ===================================================================== join

namespace {

constexpr int KMAXS = 4;          // lists intersected by one loop
constexpr uint64_t KMAX_CELLS = 1ull << 20;
constexpr uint32_t KPAIR_MIN = 32;  // default per-binding threshold of the last loop
// How kpair searches a list: a run holding every integer of [vmin, vmax]
// addresses itself (x can only sit at lo + x - vmin: one 4-byte read);
// else through its bucket directory (low byte: the bucket shift), else, a
// run shorter than DIR_MIN, by binary search.
constexpr uint32_t KP_DIRECT = 0x200u, KP_DIR = 0x100u, KP_POS = 0x400u;  // KP_POS: a top level's position map
constexpr int KJ_MAXT = 128;      // threads per block of the search kernel, at most
constexpr int KJ_WARPS = KJ_MAXT / 32;

// One list of one loop: level `depth` of an atom.  A top level (depth 0) is
// the whole V_0; a deeper level is the range of V_depth that the atom's
// previous level opened at loop from_loop (through the binding's list
// from_src there).  A list with an offset array `o` opens the atom's next
// level at its match.
struct KSrc {
    const uint32_t* v;
    const uint4* g;       // bucket directory of this level's runs, or NULL
    const uint32_t* o;
    const uint32_t* pos;  // depth 0: value -> position in V_0 (V1POS_NONE if absent), or NULL
    const uint32_t* l0s;  // depth 0 of a partitioned atom: first level-0 entry of each partition, else NULL
    uint32_t pos_n;       // values covered by pos
    uint32_t top_len;     // l_0 of the atom
    uint32_t pw[HC_KMAX_ARITY];  // radix weight of each column of the atom in its partition id
    uint8_t pv[HC_KMAX_ARITY];   // variable of each column of the atom
    uint8_t pk;                  // the atom's arity
    int32_t depth;
    int32_t from_loop, from_src;
};

// HyperCube cells (Sec. 4-5): cell id = mixed radix of the variables'
// coordinates, variable 0 most significant; coordinate of variable v in
// cell c = (c / vstride[v]) % vshare[v].
struct KPlan {
    int32_t nv, stats;
    uint32_t n_cells;
    uint32_t pair_min;  // last-loop parents with at least this many candidates take the per-binding path
    int32_t nsrc[HC_KMAX_VARS];
    int32_t var_of_loop[HC_KMAX_VARS];
    uint32_t vshare[HC_KMAX_VARS], vstride[HC_KMAX_VARS];
    KSrc src[HC_KMAX_VARS][KMAXS];
};

// A loop-0 binding: its cell, its value and, per loop-0 list that opens a
// level, the range of its children there.
struct KEntry {
    uint32_t cell;
    uint32_t val;
    uint32_t lo[KMAXS], hi[KMAXS];
};

// A cell with loop-0 candidates: its shortest loop-0 list (drv) and that
// list's range [lo, lo + len) in V_0.
struct KCell {
    uint32_t cell, drv, lo, len;
};

__device__ __forceinline__ void load_kplan(KPlan& dst, const KPlan* __restrict__ src) {
    const uint32_t* sp = (const uint32_t*)src;
    uint32_t* dp = (uint32_t*)&dst;
    for (uint32_t i = threadIdx.x; i < sizeof(KPlan) / 4; i += blockDim.x) dp[i] = sp[i];
    __syncthreads();
}

// The range of a top-level list in a cell: the level 0 of the partition
// that the cell's coordinates select in the list's atom (Sec. 4-5), or all
// of V_0 for an unpartitioned atom.
__device__ __forceinline__ void ktop(const KPlan& P, const KSrc& s, uint32_t cell, uint32_t& lo, uint32_t& hi) {
    if (s.l0s == nullptr) {
        lo = 0;
        hi = s.top_len;
        return;
    }
    uint32_t pid = 0;
#pragma unroll
    for (int c = 0; c < HC_KMAX_ARITY; ++c) {
        if (c < (int)s.pk) {
            const uint32_t v = s.pv[c];
            pid += (cell / P.vstride[v]) % P.vshare[v] * s.pw[c];
        }
    }
    lo = __ldg(s.l0s + pid);
    hi = __ldg(s.l0s + pid + 1);
}

// search(V, x) of Sec. 5 within [lo, hi): the position of v, found or not.
__device__ __forceinline__ uint32_t ksearch(const KSrc& s, uint32_t lo, uint32_t hi, uint32_t v, bool& ok) {
    if (s.depth == 0 && s.pos != nullptr) {
        const uint32_t p = v < s.pos_n ? __ldg(s.pos + v) : V1POS_NONE;
        ok = p != V1POS_NONE && p >= lo && p < hi;
        return p;
    }
    uint32_t p = lo;
    ok = dir_find(s.v, s.g, lo, hi, v, DIR_MIN, p);
    return p;
}

// ----------------------------------------------------------------- loop 0
// The loop-0 candidates of all cells, concatenated: thread t takes
// candidate t, a value of its cell's shortest loop-0 list, and searches it
// in the cell's other loop-0 lists.  n_vars == 1: matches are the result
// (counted, or written with MAT).  Otherwise a match with loop-1 candidates
// becomes an entry.
template <bool MAT>
__global__ void __launch_bounds__(256) kloop0_kernel(const KPlan* __restrict__ gP, const KCell* __restrict__ cells,
                                                     const uint64_t* __restrict__ cell_pref, uint32_t ncell,
                                                     KEntry* __restrict__ entries, uint32_t* __restrict__ units,
                                                     JoinCtl* ctl, uint32_t* __restrict__ out, uint64_t cap,
                                                     uint64_t* __restrict__ cell_counts) {
    __shared__ KPlan P;
    load_kplan(P, gP);
    const uint32_t lane = lane_id();
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool valid = t < cell_pref[ncell];
    KCell C{0, 0, 0, 0};
    uint32_t off = 0;
    if (valid) {
        uint32_t lo = 0, hi = ncell;  // the last cell whose first candidate is <= t
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cell_pref[mid] <= t)
                lo = mid;
            else
                hi = mid;
        }
        C = cells[lo];
        off = (uint32_t)(t - cell_pref[lo]);
    }
    uint32_t v = 0;
    bool ok = valid;
    uint32_t pq[KMAXS];
    if (valid) v = __ldg(P.src[0][C.drv].v + C.lo + off);
#pragma unroll
    for (int q = 0; q < KMAXS; ++q) {
        pq[q] = 0;
        if (q < P.nsrc[0]) {
            if (q == (int)C.drv) {
                pq[q] = C.lo + off;
            } else if (ok) {
                const KSrc& s = P.src[0][q];
                uint32_t lo, hi;
                ktop(P, s, C.cell, lo, hi);
                pq[q] = ksearch(s, lo, hi, v, ok);
            }
        }
    }
    if (!MAT && P.stats && valid && off == 0)
        atomicAdd((unsigned long long*)&ctl->work, (unsigned long long)P.nsrc[0] * C.len);
    if (P.nv == 1) {
        const uint32_t m = __ballot_sync(FULL, ok);
        if (!MAT) {
            if (lane == 0 && m) atomicAdd((unsigned long long*)&ctl->total, (unsigned long long)__popc(m));
            if (cell_counts && ok) atomicAdd((unsigned long long*)&cell_counts[C.cell], 1ull);
            return;
        }
        unsigned long long b = 0;
        if (lane == 0 && m) b = atomicAdd((unsigned long long*)&ctl->written, (unsigned long long)__popc(m));
        b = __shfl_sync(FULL, b, 0);
        if (ok) {
            const uint64_t idx = b + __popc(m & lanemask_lt());
            if (idx < cap)
                out[idx] = v;
            else
                atomicOr(&ctl->overflow, 1u);
        }
        return;
    }
    if (MAT) return;  // entries are made by the counting pass
    uint32_t lo[KMAXS], hi[KMAXS];
#pragma unroll
    for (int q = 0; q < KMAXS; ++q) {
        lo[q] = hi[q] = 0;
        if (ok && q < P.nsrc[0] && P.src[0][q].o != nullptr) {
            const uint32_t* o = P.src[0][q].o;
            lo[q] = __ldg(o + pq[q]);
            hi[q] = __ldg(o + pq[q] + 1);
        }
    }
    uint32_t nu = 0;
    if (ok) {
        nu = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < KMAXS; ++q) {
            if (q < P.nsrc[1]) {
                const KSrc& s = P.src[1][q];
                uint32_t len = 0;
                if (s.depth == 0) {
                    uint32_t lo, hi;
                    ktop(P, s, C.cell, lo, hi);
                    len = hi - lo;
                } else {
#pragma unroll
                    for (int r = 0; r < KMAXS; ++r)
                        if (r == s.from_src) len = hi[r] - lo[r];
                }
                nu = min(nu, len);
            }
        }
        if (nu == 0) ok = false;
    }
    if (P.stats) {
        const uint64_t wk = warp_sum64(ok ? (uint64_t)P.nsrc[1] * nu : 0);
        if (lane == 0 && wk) atomicAdd((unsigned long long*)&ctl->work, (unsigned long long)wk);
    }
    const uint32_t m = __ballot_sync(FULL, ok);
    uint32_t b = 0;
    if (lane == 0 && m) b = atomicAdd(&ctl->n_entries, (uint32_t)__popc(m));
    b = __shfl_sync(FULL, b, 0);
    if (ok) {
        const uint32_t slot = b + __popc(m & lanemask_lt());
        KEntry e;
        e.cell = C.cell;
        e.val = v;
#pragma unroll
        for (int q = 0; q < KMAXS; ++q) {
            e.lo[q] = lo[q];
            e.hi[q] = hi[q];
        }
        entries[slot] = e;
        units[slot] = nu;
    }
}

// ------------------------------------------------------------ search loops
// Per-warp state in shared memory.  Bindings of loops 1..NV-2 (frame f =
// loop - 1), one per lane slot: value, parent slot in the loop above, and
// the children range of each of the loop's lists that opens a level.
// Candidate rounds of loops 1..NV-1 (level li = loop - 1): per parent the
// prefix of candidate counts, the shortest list and its start.
template <int NV>
struct KWarp {
    static constexpr int NF = NV > 2 ? NV - 2 : 1;
    uint64_t pref[NV - 1][33];
    uint64_t round[NV - 1], total[NV - 1];
    uint32_t val[NF][32];
    uint32_t rlo[NF][KMAXS][32];
    uint32_t rhi[NF][KMAXS][32];
    uint32_t dlo[NV - 1][32];
    uint32_t tlo[NV - 1][KMAXS], thi[NV - 1][KMAXS];  // top-level lists of loops 1.. in the entry's cell
    uint32_t e_lo[KMAXS], e_hi[KMAXS];
    uint32_t e_val;
    uint64_t c0[32];    // each lane's count when the entry started (per-cell counts)
    uint32_t llen[32];  // candidates of each last-loop parent on the per-binding path
    uint32_t lmask;     // those parents
    // kpair, per list of the parent: (lo, span or hi, vmin or pos_n, search kind KP_* | bucket
    // shift), the array it reads (the values from lo for KP_DIRECT, the position map for KP_POS),
    // the directory from lo, and hi
    uint4 prec[KMAXS];
    const uint32_t* pptr[KMAXS];
    const uint4* pdir[KMAXS];
    uint32_t phi[KMAXS];
    uint8_t par[NF][32];
    uint8_t drv[NV - 1][32];
};

// Range of list q of loop L for parent slot b (a binding of loop L-1; the
// entry when L == 1).
template <int NV>
__device__ __forceinline__ void krange(const KPlan& P, const KWarp<NV>& S, int L, int q, uint32_t b, uint32_t& lo,
                                       uint32_t& hi) {
    const KSrc& s = P.src[L][q];
    if (s.depth == 0) {
        lo = S.tlo[L - 1][q];
        hi = S.thi[L - 1][q];
        return;
    }
    const int f = s.from_loop, r = s.from_src;
    if (f == 0) {
        lo = S.e_lo[r];
        hi = S.e_hi[r];
        return;
    }
    uint32_t a = b;
    for (int l = L - 1; l > f; --l) a = S.par[l - 1][a];
    lo = S.rlo[f - 1][r][a];
    hi = S.rhi[f - 1][r][a];
}

// Start loop L with parents 0..nb-1: each parent's shortest list and the
// prefix of their candidate counts.  Loop 1 has the entry as its only
// parent and takes candidates [t0, t1) of its shortest list.
template <int NV>
__device__ __forceinline__ void kinit_level(const KPlan& P, KWarp<NV>& S, int L, uint32_t nb, uint32_t t0,
                                            uint32_t t1, uint64_t& work) {
    const uint32_t lane = lane_id();
    const int li = L - 1;
    uint64_t c = 0;
    uint32_t dsel = 0, dlo = 0;
    if (lane < nb) {
        uint32_t best = 0xFFFFFFFFu;
        for (int q = 0; q < P.nsrc[L]; ++q) {
            uint32_t lo, hi;
            krange<NV>(P, S, L, q, lane, lo, hi);
            if (hi - lo < best) {
                best = hi - lo;
                dsel = (uint32_t)q;
                dlo = lo;
            }
        }
        if (L == 1) {
            dlo += t0;
            c = t1 - t0;
        } else {
            c = best;
            if (P.stats) work += (uint64_t)P.nsrc[L] * best;
        }
    }
    // last loop: a parent with many candidates leaves the flattened rounds
    // for the per-binding path (kpair)
    bool lng = false;
    if (L == NV - 1 && lane < nb && c >= P.pair_min) {
        lng = true;
        S.llen[lane] = (uint32_t)c;
        c = 0;
    }
    const uint32_t lm = __ballot_sync(FULL, lng);
    if (lane == 0 && L == NV - 1) S.lmask = lm;
    const uint64_t incl = warp_incl_scan64(c);
    __syncwarp();
    S.pref[li][lane + 1] = incl;
    if (lane == 0) {
        S.pref[li][0] = 0;
        S.round[li] = 0;
    }
    if (lane < nb) {
        S.drv[li][lane] = (uint8_t)dsel;
        S.dlo[li][lane] = dlo;
    }
    if (lane == 31) S.total[li] = incl;
    __syncwarp();
}

// The per-binding path of the last loop: parent b's candidates, the
// elements of its shortest list, 128 per iteration (lane l takes the
// elements l, l + 32, l + 64, l + 96 of each block), searched in each other
// list in turn with the four reads of a lane issued together.  A list's
// range, bounds and search kind (KP_*) are the same for every candidate, so
// one lane per list sets them up once, in one shared-memory record.  The
// last loop's lists are the atoms' last levels (no positions are needed).
template <int NV, bool MAT>
__device__ __forceinline__ void kpair(const KPlan& P, KWarp<NV>& S, uint32_t b, uint64_t& cnt, JoinCtl* ctl,
                                      uint32_t* __restrict__ out, uint64_t cap) {
    constexpr int L = NV - 1, li = NV - 2;
    const uint32_t lane = lane_id();
    const uint32_t d = S.drv[li][b];
    const uint32_t a0 = S.dlo[li][b], a1 = a0 + S.llen[b];
    const uint32_t* __restrict__ va = P.src[L][d].v;
    const int ns = P.nsrc[L];
    if (ns == 1 && !MAT) {  // nothing to search: every candidate is a result
        if (lane == 0) cnt += a1 - a0;
        return;
    }
    // lane q sets up list q once for the whole parent
    __syncwarp();
    if (lane < (uint32_t)ns && lane != d) {
        const KSrc& sq = P.src[L][lane];
        uint32_t lo, hi;
        krange<NV>(P, S, L, (int)lane, b, lo, hi);
        S.phi[lane] = hi;
        if (sq.depth == 0 && sq.pos != nullptr) {
            S.prec[lane] = make_uint4(lo, hi, sq.pos_n, KP_POS);
            S.pptr[lane] = sq.pos;
        } else {
            const uint32_t vmin = __ldg(sq.v + lo), vmax = __ldg(sq.v + hi - 1);
            const bool dir = sq.g != nullptr && hi - lo >= DIR_MIN;
            // distinct ascending values with vmax - vmin = n - 1 are every integer between
            const bool direct = vmax - vmin == hi - lo - 1;
            S.prec[lane] = make_uint4(lo, vmax - vmin, vmin,
                                      direct ? KP_DIRECT : dir ? (KP_DIR | dir_shift(hi - lo, vmax - vmin)) : 0u);
            S.pptr[lane] = direct ? sq.v + lo : sq.v;
            S.pdir[lane] = dir ? sq.g + lo : nullptr;
        }
    }
    __syncwarp();
    for (uint32_t t0 = a0; t0 < a1; t0 += 128) {
        uint32_t vv[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = t0 + 32 * j + lane;
            ok[j] = t < a1;
            vv[j] = ok[j] ? __ldg(va + t) : 0u;
        }
        for (int q = 0; q < ns; ++q) {
            if (q == (int)d) continue;
            const uint4 r = S.prec[q];
            const uint32_t* __restrict__ pq = S.pptr[q];
            if (r.w == KP_DIRECT) {  // x can only be at lo + (x - vmin): read that value
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t dx = vv[j] - r.z;
                    ok[j] = ok[j] && dx <= r.y;
                    const uint32_t w = ok[j] ? __ldg(pq + dx) : 0u;
                    ok[j] = ok[j] && w == vv[j];
                }
                continue;
            }
            if (r.w == KP_POS) {  // a top level's position map, checked against the cell's range
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t p = ok[j] && vv[j] < r.z ? __ldg(pq + vv[j]) : V1POS_NONE;
                    ok[j] = p != V1POS_NONE && p >= r.x && p < r.y;
                }
                continue;
            }
            const uint32_t lo = r.x, span = r.y, vmin = r.z, hi = S.phi[q];
            if (r.w == 0) {  // a short list: binary search
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t pos;
                    if (ok[j]) ok[j] = vv[j] - vmin <= span && find_u32(pq, lo, hi, vv[j], pos);
                }
                continue;
            }
            const uint4* __restrict__ gq = S.pdir[q];
            uint4 ev[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t dx = vv[j] - vmin;  // x in [vmin, vmax] <=> x - vmin <= vmax - vmin
                ok[j] = ok[j] && dx <= span;
                ev[j] = ok[j] ? dir_load(gq, dx >> (r.w & 0xFFu)) : make_uint4(0u, 0u, 0u, 0u);
            }
            // the entry's three values decide, unless x lies beyond them
            // (then the walk of dir_walk_find, which also pulls a position
            // outside the run back to it)
            uint32_t slow = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 e = ev[j];
                const bool hit = (e.y == vv[j]) | (e.z == vv[j]) | (e.w == vv[j]);
                slow |= (ok[j] && vv[j] > e.w ? 1u : 0u) << j;
                ok[j] = ok[j] && hit;
            }
            if (slow) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t pos;
                    if (slow >> j & 1u) ok[j] = dir_walk_find(pq, ev[j], hi, vv[j], pos);
                }
            }
        }
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) mine += ok[j] ? 1u : 0u;
        if (!MAT) {
            cnt += mine;
            continue;
        }
        const uint32_t incl = warp_incl_scan(mine);
        const uint32_t k = __shfl_sync(FULL, incl, 31);
        if (k == 0) continue;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd((unsigned long long*)&ctl->written, (unsigned long long)k);
        base = __shfl_sync(FULL, base, 31);
        uint64_t idx = base + incl - mine;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            if (idx < cap) {
                uint32_t* t = out + idx * (uint64_t)P.nv;
                t[P.var_of_loop[NV - 1]] = vv[j];
                t[P.var_of_loop[0]] = S.e_val;
                uint32_t a = b;
                for (int l = NV - 2; l >= 1; --l) {
                    t[P.var_of_loop[l]] = S.val[l - 1][a];
                    a = S.par[l - 1][a];
                }
            } else {
                atomicOr(&ctl->overflow, 1u);
            }
            ++idx;
        }
    }
}

// Walk loops 1..NV-1 below the entry in S, loop 1 over candidates [t0, t1).
template <int NV, bool MAT>
__device__ void kwalk(const KPlan& P, KWarp<NV>& S, uint32_t t0, uint32_t t1, uint64_t& cnt, uint64_t& work,
                      JoinCtl* ctl, uint32_t* __restrict__ out, uint64_t cap) {
    const uint32_t lane = lane_id();
    kinit_level<NV>(P, S, 1, 1, t0, t1, work);
    int L = 1;
    while (true) {
        const int li = L - 1;
        __syncwarp();
        const uint64_t r = S.round[li], tot = S.total[li];
        __syncwarp();
        if (r * 32 >= tot) {
            if (L == NV - 1) {  // the last loop's long parents, one at a time
                uint32_t lm = S.lmask;
                while (lm) {
                    const uint32_t b = __ffs(lm) - 1;
                    lm &= lm - 1;
                    kpair<NV, MAT>(P, S, b, cnt, ctl, out, cap);
                }
            }
            if (L == 1) break;
            --L;
            continue;
        }
        if (lane == 0) S.round[li] = r + 1;
        const uint64_t g = r * 32 + lane;
        const bool valid = g < tot;
        // parent: the last slot b whose prefix is <= g
        uint32_t b = 0;
        if (L > 1 && valid) {
            uint32_t lo = 0, hi = 32;  // pref[li][b] for b < 32; slots past the parents have prefix == tot > g
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (S.pref[li][mid] <= g)
                    lo = mid;
                else
                    hi = mid;
            }
            b = lo;
        }
        uint32_t v = 0;
        bool ok = valid;
        uint32_t pq[KMAXS];
#pragma unroll
        for (int q = 0; q < KMAXS; ++q) pq[q] = 0;
        if (valid) {
            const uint32_t d = S.drv[li][b];
            const uint32_t pos = S.dlo[li][b] + (uint32_t)(g - S.pref[li][b]);
            v = __ldg(P.src[L][d].v + pos);
#pragma unroll
            for (int q = 0; q < KMAXS; ++q) {
                if (q < P.nsrc[L]) {
                    if (q == (int)d) {
                        pq[q] = pos;
                    } else if (ok) {
                        uint32_t lo, hi;
                        krange<NV>(P, S, L, q, b, lo, hi);
                        pq[q] = ksearch(P.src[L][q], lo, hi, v, ok);
                    }
                }
            }
        }
        const uint32_t m = __ballot_sync(FULL, ok);
        if (L == NV - 1) {
            if (!MAT) {
                cnt += ok ? 1u : 0u;
                continue;
            }
            if (m == 0) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd((unsigned long long*)&ctl->written, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (ok) {
                const uint64_t idx = base + __popc(m & lanemask_lt());
                if (idx < cap) {
                    uint32_t* t = out + idx * (uint64_t)P.nv;
                    t[P.var_of_loop[NV - 1]] = v;
                    uint32_t a = b;
                    for (int l = NV - 2; l >= 1; --l) {
                        t[P.var_of_loop[l]] = S.val[l - 1][a];
                        a = S.par[l - 1][a];
                    }
                    t[P.var_of_loop[0]] = S.e_val;
                } else {
                    atomicOr(&ctl->overflow, 1u);
                }
            }
            continue;
        }
        // compact the matches into the bindings of loop L and descend
        if (ok) {
            const int f = L - 1;
            const uint32_t rk = __popc(m & lanemask_lt());
            S.val[f][rk] = v;
            S.par[f][rk] = (uint8_t)b;
#pragma unroll
            for (int q = 0; q < KMAXS; ++q) {
                if (q < P.nsrc[L] && P.src[L][q].o != nullptr) {
                    const uint32_t* o = P.src[L][q].o;
                    S.rlo[f][q][rk] = __ldg(o + pq[q]);
                    S.rhi[f][q][rk] = __ldg(o + pq[q] + 1);
                }
            }
        }
        __syncwarp();
        if (m) {
            ++L;
            kinit_level<NV>(P, S, L, (uint32_t)__popc(m), 0, 0, work);
        }
    }
}

// Persistent search kernel: warps take work items of `grain` loop-1
// candidates (0: sized so that each warp gets about 8 items) from an atomic
// counter, over the concatenation of all entries' candidates.
template <int NV, bool MAT>
__global__ void __launch_bounds__(KJ_MAXT) kjoin_kernel(const KPlan* __restrict__ gP,
                                                        const KEntry* __restrict__ entries,
                                                        const uint64_t* __restrict__ unit_off, JoinCtl* ctl,
                                                        uint32_t grain_in, uint32_t* __restrict__ out, uint64_t cap,
                                                        uint64_t* __restrict__ cell_counts) {
    __shared__ KPlan P;
    __shared__ KWarp<NV> WS[KJ_WARPS];
    load_kplan(P, gP);
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    KWarp<NV>& S = WS[w];
    if (dev_err_set(&ctl->err)) return;  // the unit-offset scan gave up a wait
    const uint32_t ne = ctl->n_entries;
    const uint64_t total_units = unit_off[ne];
    uint64_t grain = grain_in;
    if (grain == 0) {
        const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
        grain = total_units / (warps * 8);
        if (grain == 0) grain = 1;
    }
    uint64_t cnt = 0, work = 0;
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&ctl->item_ctr[MAT ? 1 : 0], 1u);
        item = __shfl_sync(FULL, item, 0);
        uint64_t u0 = (uint64_t)item * grain;
        if (u0 >= total_units) break;
        const uint64_t u1 = u0 + grain < total_units ? u0 + grain : total_units;
        // the entry holding unit u0: first j in [1, ne] with unit_off[j] > u0, minus one
        uint32_t lo = 1, hi = ne;
        while (lo < hi) {
            const uint32_t mid = lo + ((hi - lo) >> 1);
            if (unit_off[mid] > u0)
                hi = mid;
            else
                lo = mid + 1;
        }
        uint32_t e = lo - 1;
        while (u0 < u1 && e < ne) {
            const uint64_t eb = unit_off[e], ee = unit_off[e + 1];
            if (ee > u0) {
                __syncwarp();
                if (lane == 0) {
                    const KEntry en = entries[e];
                    S.e_val = en.val;
#pragma unroll
                    for (int q = 0; q < KMAXS; ++q) {
                        S.e_lo[q] = en.lo[q];
                        S.e_hi[q] = en.hi[q];
                    }
                }
                if (lane < (uint32_t)((NV - 1) * KMAXS)) {
                    const int L = 1 + (int)lane / KMAXS, q = (int)lane % KMAXS;
                    if (q < P.nsrc[L] && P.src[L][q].depth == 0)
                        ktop(P, P.src[L][q], entries[e].cell, S.tlo[L - 1][q], S.thi[L - 1][q]);
                }
                __syncwarp();
                const uint64_t u_end = u1 < ee ? u1 : ee;
                if (!MAT && cell_counts) S.c0[lane] = cnt;
                kwalk<NV, MAT>(P, S, (uint32_t)(u0 - eb), (uint32_t)(u_end - eb), cnt, work, ctl, out, cap);
                if (!MAT && cell_counts) {
                    const uint64_t dc = warp_sum64(cnt - S.c0[lane]);
                    if (lane == 0 && dc)
                        atomicAdd((unsigned long long*)&cell_counts[entries[e].cell], (unsigned long long)dc);
                }
                u0 = u_end;
            }
            ++e;
        }
    }
    if (!MAT) {
        cnt = warp_sum64(cnt);
        work = warp_sum64(work);
        if (lane == 0) {
            if (cnt) atomicAdd((unsigned long long*)&ctl->total, (unsigned long long)cnt);
            if (work) atomicAdd((unsigned long long*)&ctl->work, (unsigned long long)work);
        }
    }
}

template <int NV, bool MAT>
hc_status launch_kjoin_t(int threads, const KPlan* P, const KEntry* entries, const uint64_t* unit_off, JoinCtl* ctl,
                         uint32_t grain, uint32_t* out, uint64_t cap, uint64_t* cell_counts, cudaStream_t s) {
    int per_sm = 0;
    HC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kjoin_kernel<NV, MAT>, threads, 0));
    const int grid = num_sms() * std::max(1, per_sm);
    kjoin_kernel<NV, MAT><<<grid, threads, 0, s>>>(P, entries, unit_off, ctl, grain, out, cap, cell_counts);
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

template <bool MAT>
hc_status launch_kjoin(int nv, int threads, const KPlan* P, const KEntry* entries, const uint64_t* unit_off,
                       JoinCtl* ctl, uint32_t grain, uint32_t* out, uint64_t cap, uint64_t* cc, cudaStream_t s) {
    switch (nv) {
        case 2: return launch_kjoin_t<2, MAT>(threads, P, entries, unit_off, ctl, grain, out, cap, cc, s);
        case 3: return launch_kjoin_t<3, MAT>(threads, P, entries, unit_off, ctl, grain, out, cap, cc, s);
        case 4: return launch_kjoin_t<4, MAT>(threads, P, entries, unit_off, ctl, grain, out, cap, cc, s);
        case 5: return launch_kjoin_t<5, MAT>(threads, P, entries, unit_off, ctl, grain, out, cap, cc, s);
        case 6: return launch_kjoin_t<6, MAT>(threads, P, entries, unit_off, ctl, grain, out, cap, cc, s);
        default: return fail(HC_ERR_CAPACITY, "run_kjoin: unsupported number of variables");
    }
}

hc_status read_kctl(hc_result* R) {
    HC_CUDA_TRY(cudaMemcpyAsync(&R->h_ctl, R->d_ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, R->stream));
    HC_CUDA_TRY(cudaStreamSynchronize(R->stream));
    if (R->h_ctl.err & DEV_ERR_TIMEOUT) return fail(HC_ERR_TIMEOUT, "run_kjoin: a bounded device wait gave up");
    return HC_OK;
}

// Validation and the lists of every loop (host only).
hc_status make_kplan(const hc_kquery* q, const hc_kindex* const* idx, KPlan& P) {
    memset(&P, 0, sizeof(P));
    const uint32_t nv = q->n_vars, na = q->n_atoms;
    if (nv < 1) return fail(HC_ERR_ARG, "run_kjoin: n_vars must be at least 1");
    if (nv > HC_KMAX_VARS) return fail(HC_ERR_CAPACITY, "run_kjoin: at most 6 variables");
    if (na < 1 || na > HC_MAX_ATOMS) return fail(HC_ERR_ARG, "run_kjoin: n_atoms must be 1..12");
    int rank[HC_MAX_VARS];
    bool seen[HC_MAX_VARS] = {false};
    for (uint32_t i = 0; i < nv; ++i) {
        const uint32_t v = q->order[i];
        if (v >= nv || seen[v]) return fail(HC_ERR_ARG, "run_kjoin: order must list every variable once");
        seen[v] = true;
        rank[v] = (int)i;
        P.var_of_loop[i] = (int32_t)v;
    }
    P.nv = (int32_t)nv;
    uint32_t vseed[HC_KMAX_VARS] = {0};
    for (uint32_t j = 0; j < na; ++j) {
        const hc_katom& a = q->atoms[j];
        const uint32_t k = a.arity;
        if (k < 1 || k > HC_KMAX_ARITY) return fail(HC_ERR_ARG, "run_kjoin: atom arity must be 1, 2 or 3");
        for (uint32_t c = 0; c < k; ++c) {
            if (a.var[c] >= nv) return fail(HC_ERR_ARG, "run_kjoin: atom variable out of range");
            for (uint32_t c2 = 0; c2 < c; ++c2)
                if (a.var[c2] == a.var[c]) return fail(HC_ERR_ARG, "run_kjoin: a variable twice in one atom");
        }
        const hc_kindex* x = idx[j];
        if (!x) return fail(HC_ERR_ARG, "run_kjoin: index is NULL");
        if (x->arity != k) return fail(HC_ERR_ARG, "run_kjoin: index arity differs from the atom's");
        // every atom holding a variable partitions it with the same share
        // and seed, so the cells' coordinates select one partition per atom
        uint32_t pw[HC_KMAX_ARITY] = {1, 1, 1};
        for (int c = (int)k - 2; c >= 0; --c) pw[c] = pw[c + 1] * x->pshare[c + 1];
        for (uint32_t c = 0; c < k; ++c) {
            const uint32_t v = a.var[c], sh = x->pshare[c], sd = sh > 1 ? x->pseed[c] : 0u;
            if (P.vshare[v] == 0) {
                P.vshare[v] = sh;
                vseed[v] = sd;
            } else if (P.vshare[v] != sh || vseed[v] != sd) {
                return fail(HC_ERR_ARG, "run_kjoin: atoms partition a variable with different shares or seeds");
            }
        }
        int prev_loop = -1, prev_src = -1;
        for (uint32_t d = 0; d < k; ++d) {
            const int L = rank[a.var[x->level_cols[d]]];
            if (L <= prev_loop)
                return fail(HC_ERR_ARG, "run_kjoin: the index levels must hold the atom's variables in loop order");
            if (P.nsrc[L] >= KMAXS) return fail(HC_ERR_CAPACITY, "run_kjoin: a variable is in more than 4 atoms");
            const int qn = P.nsrc[L]++;
            KSrc& s = P.src[L][qn];
            s.v = x->d_v[d];
            s.g = x->d_g[d];
            s.o = d + 1 < k ? x->d_o[d] : nullptr;
            s.pos = d == 0 ? x->d_v0pos : nullptr;
            s.pos_n = d == 0 ? x->v0pos_n : 0;
            s.top_len = (uint32_t)x->len[0];
            s.l0s = d == 0 && x->n_parts > 1 ? x->d_l0start : nullptr;
            s.pk = (uint8_t)k;
            for (uint32_t c = 0; c < k; ++c) {
                s.pv[c] = a.var[c];
                s.pw[c] = pw[c];
            }
            s.depth = (int32_t)d;
            s.from_loop = prev_loop;
            s.from_src = prev_src;
            prev_loop = L;
            prev_src = qn;
        }
    }
    for (uint32_t i = 0; i < nv; ++i)
        if (P.nsrc[i] == 0) return fail(HC_ERR_ARG, "run_kjoin: every variable must occur in some atom");
    for (uint32_t j = 0; j < na; ++j)
        if (idx[j]->stats_only) return fail(HC_ERR_ARG, "run_kjoin: a statistics-only index has no data");
    uint64_t cells = 1;
    for (int v = (int)nv - 1; v >= 0; --v) {
        P.vstride[v] = (uint32_t)cells;
        cells *= P.vshare[v];
        if (cells > KMAX_CELLS) return fail(HC_ERR_CAPACITY, "run_kjoin: more than 2^20 HyperCube cells");
    }
    P.n_cells = (uint32_t)cells;
    return HC_OK;
}

// Loop-0 candidates of every cell (host, from the indexes' partition
// starts): per cell, its shortest loop-0 list and that list's range; cells
// with an empty loop-0 list are left out.  pref receives the prefix of the
// candidate counts (size cells.size() + 1).
void kcell_table(const KPlan& P, const hc_kquery* q, const hc_kindex* const* idx, std::vector<KCell>& cells,
                 std::vector<uint64_t>& pref) {
    // the atom behind each loop-0 list
    const hc_kindex* xs[KMAXS] = {nullptr, nullptr, nullptr, nullptr};
    for (int qn = 0; qn < P.nsrc[0]; ++qn)
        for (uint32_t j = 0; j < q->n_atoms; ++j)
            if (idx[j]->d_v[0] == P.src[0][qn].v) xs[qn] = idx[j];
    cells.clear();
    pref.assign(1, 0);
    for (uint32_t c = 0; c < P.n_cells; ++c) {
        KCell best{c, 0, 0, 0xFFFFFFFFu};
        for (int qn = 0; qn < P.nsrc[0]; ++qn) {
            const KSrc& s = P.src[0][qn];
            uint32_t lo = 0, hi = s.top_len;
            if (s.l0s != nullptr) {
                uint32_t pid = 0;
                for (uint32_t k = 0; k < s.pk; ++k) pid += (c / P.vstride[s.pv[k]]) % P.vshare[s.pv[k]] * s.pw[k];
                lo = xs[qn]->h_l0start[pid];
                hi = xs[qn]->h_l0start[pid + 1];
            }
            if (hi - lo < best.len) best = KCell{c, (uint32_t)qn, lo, hi - lo};
        }
        if (best.len == 0) continue;
        cells.push_back(best);
        pref.push_back(pref.back() + best.len);
    }
}

}  // namespace

hc_status run_kjoin_impl(const hc_kquery* q, const hc_kindex* const* idx, const hc_kjoin_params* prm,
                         cudaStream_t s, hc_result** out) {
    if (!out) return fail(HC_ERR_ARG, "run_kjoin: out is NULL");
    *out = nullptr;
    if (!q || !idx) return fail(HC_ERR_ARG, "run_kjoin: NULL argument");
    hc_kjoin_params dp{};
    if (prm) dp = *prm;
    if (dp.mode > HC_MODE_MATERIALIZE) return fail(HC_ERR_ARG, "run_kjoin: unknown mode");
    const int threads = dp.block_threads ? (int)dp.block_threads : KJ_MAXT;
    if (threads % 32 != 0 || threads < 32 || threads > KJ_MAXT)
        return fail(HC_ERR_ARG, "run_kjoin: block_threads must be 32, 64, 96 or 128");
    KPlan P;
    HC_TRY(make_kplan(q, idx, P));
    P.stats = (dp.flags & HC_FLAG_STATS) ? 1 : 0;
    P.pair_min = dp.pair_min ? dp.pair_min : KPAIR_MIN;
    const uint32_t nv = q->n_vars;

    std::vector<KCell> hcells;
    std::vector<uint64_t> hpref;
    kcell_table(P, q, idx, hcells, hpref);
    const uint64_t len0 = hpref.back();  // loop-0 candidates over all cells
    if (len0 >= 0xFFFFFFFFull) return fail(HC_ERR_CAPACITY, "run_kjoin: 2^32 - 1 or more loop-0 candidates");

    hc_result* R = new hc_result();
    R->stream = s;
    R->n_vars = nv;
    R->n_cells = P.n_cells;
    auto bail = [&](hc_status st) {
        result_release(R);
        return st;
    };
    void* p = nullptr;
    if (dev_alloc(&p, sizeof(JoinCtl), s) != HC_OK) return bail(HC_ERR_OOM);
    R->d_ctl = (JoinCtl*)p;
    JoinCtl* ctl = R->d_ctl;
    if (cudaMemsetAsync(ctl, 0, sizeof(JoinCtl), s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    if (dp.flags & HC_FLAG_CELL_COUNTS) {
        if (dev_alloc(&p, (uint64_t)P.n_cells * 8, s) != HC_OK) return bail(HC_ERR_OOM);
        R->d_cell_counts = (uint64_t*)p;
        if (cudaMemsetAsync(R->d_cell_counts, 0, (uint64_t)P.n_cells * 8, s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "memset"));
    }
    uint64_t* cc = R->d_cell_counts;
    const bool timed = (dp.flags & HC_FLAG_TIME_KERNELS) != 0;

    KScratch tmp(s);
    hc_status st;
    KPlan* dP;
    if ((st = tmp.get(&dP, 1)) != HC_OK) return bail(st);
    if (cudaMemcpyAsync(dP, &P, sizeof(KPlan), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "plan copy"));
    const uint32_t ncell = (uint32_t)hcells.size();
    KCell* dcells;
    uint64_t* dpref;
    if ((st = tmp.get(&dcells, ncell)) != HC_OK || (st = tmp.get(&dpref, (size_t)ncell + 1)) != HC_OK)
        return bail(st);
    if ((ncell && cudaMemcpyAsync(dcells, hcells.data(), ncell * sizeof(KCell), cudaMemcpyHostToDevice, s) !=
                      cudaSuccess) ||
        cudaMemcpyAsync(dpref, hpref.data(), (ncell + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cell table copy"));
    KEntry* entries = nullptr;
    uint32_t* units = nullptr;
    uint64_t* unit_off = nullptr;
    const unsigned l0_grid = (unsigned)((len0 + 255) / 256);
    auto search = [&](bool mat, uint32_t* tup, uint64_t cap) -> hc_status {
        if (timed) HC_TRY(time_mark(R, false, s));
        if (nv == 1) {
            if (mat)
                kloop0_kernel<true><<<l0_grid, 256, 0, s>>>(dP, dcells, dpref, ncell, nullptr, nullptr, ctl, tup, cap,
                                                            nullptr);
            else
                kloop0_kernel<false><<<l0_grid, 256, 0, s>>>(dP, dcells, dpref, ncell, nullptr, nullptr, ctl, nullptr,
                                                             0, cc);
            HC_CUDA_TRY(launch_check());
        } else if (mat) {
            HC_TRY(launch_kjoin<true>((int)nv, threads, dP, entries, unit_off, ctl, dp.item_grain, tup, cap, nullptr,
                                      s));
        } else {
            HC_TRY(
                launch_kjoin<false>((int)nv, threads, dP, entries, unit_off, ctl, dp.item_grain, nullptr, 0, cc, s));
        }
        if (timed) HC_TRY(time_mark(R, true, s));
        R->n_search++;
        return HC_OK;
    };
    if (len0 > 0) {
        if (nv > 1) {
            if ((st = tmp.get(&entries, len0)) != HC_OK || (st = tmp.get(&units, len0)) != HC_OK ||
                (st = tmp.get(&unit_off, (size_t)len0 + 1)) != HC_OK)
                return bail(st);
            kloop0_kernel<false><<<l0_grid, 256, 0, s>>>(dP, dcells, dpref, ncell, entries, units, ctl, nullptr, 0,
                                                         nullptr);
            if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "kloop0_kernel"));
            if ((st = exclusive_scan_u32_to_u64(units, unit_off, len0, &ctl->n_entries, &ctl->err, s)) != HC_OK)
                return bail(st);
        }
        if ((st = search(false, nullptr, 0)) != HC_OK) return bail(st);
    }
    if (dp.mode == HC_MODE_MATERIALIZE) {
        if ((st = read_kctl(R)) != HC_OK) return bail(st);
        const uint64_t total = R->h_ctl.total;
        if (total > 0) {
            if (total > (~0ull) / 4 / nv) return bail(fail(HC_ERR_CAPACITY, "run_kjoin: output too large"));
            if (dev_alloc(&p, total * nv * 4, s) != HC_OK) return bail(HC_ERR_OOM);
            R->d_tuples = (uint32_t*)p;
            if ((st = search(true, R->d_tuples, total)) != HC_OK) return bail(st);
            if ((st = read_kctl(R)) != HC_OK) return bail(st);
            if (R->h_ctl.written != total || R->h_ctl.overflow)
                return bail(fail(HC_ERR_CUDA, "run_kjoin: the writing pass disagrees with the count"));
        }
        R->materialized = true;
        R->n_tuples = total;
        R->done = true;
    }
    *out = R;
    return HC_OK;
}

// ------------------------------------------------------------------ planning
// Cost of one loop order (Sec. 5.2, Lemma "cost-ub", one cell): loop i costs
//   C_i = |S(X_i)| * (sum min N) * log2(1 + sum max N / sum min N)
// over the bindings of the prefix query, estimated as for binary atoms: a
// binding's list in atom j at loop i has average length
//   D(bound columns + X_i's column) / D(bound columns)
// where D(C) is the number of distinct value combinations of the column set
// C in the relation (a top level: D of one column), and a k-way intersection
// over a domain of size dom keeps prod(s) / dom^(k-1) values, at most min s.
// D is exact for the prefixes of the index's own level order (l_d) and for
// all columns (n); other sets take the product of single-column counts (the
// first level's l_0, else the value range) bounded by n.
namespace {

double kdistinct(const hc_kindex* x, uint32_t colmask) {
    if (colmask == 0) return 1.0;
    const double n = (double)x->n;
    uint32_t pm = 0;
    for (uint32_t d = 0; d < x->arity; ++d) {
        pm |= 1u << x->level_cols[d];
        if (pm == colmask) return (double)x->len[d];
    }
    double est = 1.0;
    for (uint32_t d = 0; d < x->arity; ++d) {
        if (!(colmask >> x->level_cols[d] & 1u)) continue;
        est *= d == 0 ? (double)x->len[0] : std::min(n, (double)x->maxv[d] + 1.0);
    }
    return std::min(est, n);
}

hc_status kplan_check(const hc_kquery* q, const hc_kindex* const* idx) {
    if (!q || !idx) return fail(HC_ERR_ARG, "kplan: NULL argument");
    const uint32_t nv = q->n_vars, na = q->n_atoms;
    if (nv < 1 || nv > HC_KMAX_VARS || na < 1 || na > HC_MAX_ATOMS)
        return fail(HC_ERR_ARG, "kplan: need 1..6 variables and 1..12 atoms");
    bool cover[HC_MAX_VARS] = {false};
    for (uint32_t j = 0; j < na; ++j) {
        const hc_katom& a = q->atoms[j];
        if (a.arity < 1 || a.arity > HC_KMAX_ARITY) return fail(HC_ERR_ARG, "kplan: atom arity must be 1, 2 or 3");
        if (!idx[j] || idx[j]->arity != a.arity) return fail(HC_ERR_ARG, "kplan: missing index or arity mismatch");
        for (uint32_t c = 0; c < a.arity; ++c) {
            if (a.var[c] >= nv) return fail(HC_ERR_ARG, "kplan: atom variable out of range");
            for (uint32_t c2 = 0; c2 < c; ++c2)
                if (a.var[c2] == a.var[c]) return fail(HC_ERR_ARG, "kplan: a variable twice in one atom");
            cover[a.var[c]] = true;
        }
    }
    for (uint32_t v = 0; v < nv; ++v)
        if (!cover[v]) return fail(HC_ERR_ARG, "kplan: a variable occurs in no atom");
    return HC_OK;
}

// Per-loop costs under `order` (variable ids) and the domain estimates.
void kplan_costs(const hc_kquery* q, const hc_kindex* const* idx, const uint8_t* order, double* cost, double* dom) {
    const int nv = (int)q->n_vars, na = (int)q->n_atoms;
    int rank[HC_MAX_VARS];
    for (int i = 0; i < nv; ++i) rank[order[i]] = i;
    for (int v = 0; v < nv; ++v) dom[v] = INFINITY;
    for (int j = 0; j < na; ++j)
        for (int c = 0; c < q->atoms[j].arity; ++c)
            dom[q->atoms[j].var[c]] = std::min(dom[q->atoms[j].var[c]], kdistinct(idx[j], 1u << c));
    double bindings = 1.0;
    for (int i = 0; i < nv; ++i) {
        const int v = order[i];
        double smin = INFINITY, smax = 0.0, prod = 1.0;
        int k = 0;
        for (int j = 0; j < na; ++j) {
            const hc_katom& a = q->atoms[j];
            int cv = -1;
            uint32_t bound = 0;
            for (int c = 0; c < a.arity; ++c) {
                if (a.var[c] == v) cv = c;
                else if (rank[a.var[c]] < i) bound |= 1u << c;
            }
            if (cv < 0) continue;
            const double below = kdistinct(idx[j], bound);
            const double len = below > 0 ? kdistinct(idx[j], bound | (1u << cv)) / below : 0.0;
            smin = std::min(smin, len);
            smax = std::max(smax, len);
            prod *= len;
            ++k;
        }
        if (k == 0 || !(smin > 0)) {
            cost[i] = 0.0;
            bindings = 0.0;
            continue;
        }
        const double sum_min = bindings * smin, sum_max = bindings * smax;
        cost[i] = (double)k * sum_min * log2(1.0 + sum_max / sum_min);
        const double keep = prod / pow(std::max(1.0, dom[v]), (double)(k - 1));
        bindings *= std::min(keep, smin);
    }
}

}  // namespace

}  // namespace hc

// ------------------------------------------------------------------- C ABI
extern "C" {

hc_status hc_build_kindex(const uint32_t* d_rows, uint64_t n, uint32_t arity, const uint8_t* level_cols,
                          uint32_t flags, void* stream, hc_kindex** out) {
    return hc::build_kindex_impl(d_rows, n, arity, level_cols, nullptr, nullptr, flags, (cudaStream_t)stream, out);
}

hc_status hc_build_kindex_partitioned(const uint32_t* d_rows, uint64_t n, uint32_t arity, const uint8_t* level_cols,
                                      const uint32_t* seeds, const uint32_t* shares, uint32_t flags, void* stream,
                                      hc_kindex** out) {
    if (!shares || !seeds) {
        if (out) *out = nullptr;
        return hc::fail(HC_ERR_ARG, "build_kindex_partitioned: seeds and shares are required");
    }
    return hc::build_kindex_impl(d_rows, n, arity, level_cols, seeds, shares, flags, (cudaStream_t)stream, out);
}

hc_status hc_kindex_free(hc_kindex* index) {
    hc::kindex_release(index, nullptr);  // a statistics-only index holds no device arrays
    return HC_OK;
}

hc_status hc_kindex_get_view(const hc_kindex* x, hc_kindex_view* v) {
    if (!x || !v) return hc::fail(HC_ERR_ARG, "kindex_get_view: NULL argument");
    memset(v, 0, sizeof(*v));
    v->n = x->n;
    v->arity = x->arity;
    v->packed = x->packed ? 1 : 0;
    for (int d = 0; d < HC_KMAX_ARITY; ++d) {
        v->level_cols[d] = (uint32_t)d < x->arity ? x->level_cols[d] : 0;
        v->len[d] = x->len[d];
        v->max_value[d] = x->maxv[d];
        v->d_v[d] = x->d_v[d];
        v->d_o[d] = x->d_o[d];
    }
    v->ms_sort = x->ms_sort;
    v->ms_levels = x->ms_levels;
    v->n_parts = x->n_parts;
    for (int c = 0; c < HC_KMAX_ARITY; ++c) {
        v->shares[c] = (uint32_t)c < x->arity ? x->pshare[c] : 0u;
        v->seeds[c] = (uint32_t)c < x->arity ? x->pseed[c] : 0u;
    }
    v->d_bpref = x->d_bpref;
    v->d_level0_start = x->d_l0start;
    return HC_OK;
}

hc_status hc_run_kjoin(const hc_kquery* q, const hc_kindex* const* idx, const hc_kjoin_params* params, void* stream,
                       hc_result** out) {
    return hc::run_kjoin_impl(q, idx, params, (cudaStream_t)stream, out);
}

hc_status hc_kindex_from_stats(uint64_t n, uint32_t arity, const uint8_t* level_cols, const uint64_t* len,
                               const uint32_t* max_value, hc_kindex** out) {
    if (!out) return hc::fail(HC_ERR_ARG, "kindex_from_stats: out is NULL");
    *out = nullptr;
    if (arity < 1 || arity > HC_KMAX_ARITY || !len || !max_value)
        return hc::fail(HC_ERR_ARG, "kindex_from_stats: arity 1..3 with len and max_value");
    uint8_t cols[HC_KMAX_ARITY] = {0, 1, 2};
    bool seen[HC_KMAX_ARITY] = {false, false, false};
    for (uint32_t d = 0; d < arity; ++d) {
        if (level_cols) cols[d] = level_cols[d];
        if (cols[d] >= arity || seen[cols[d]])
            return hc::fail(HC_ERR_ARG, "kindex_from_stats: level_cols must be a permutation of the columns");
        seen[cols[d]] = true;
    }
    if (len[arity - 1] != n) return hc::fail(HC_ERR_ARG, "kindex_from_stats: the last level holds every row");
    for (uint32_t d = 0; d < arity; ++d) {
        if ((n > 0 && len[d] == 0) || (d > 0 && len[d] < len[d - 1]) || len[d] > n)
            return hc::fail(HC_ERR_ARG, "kindex_from_stats: need 1 <= l_0 <= l_1 <= .. <= n");
    }
    hc_kindex* x = new hc_kindex();
    x->n = n;
    x->arity = arity;
    x->stats_only = true;
    for (uint32_t d = 0; d < arity; ++d) {
        x->level_cols[d] = cols[d];
        x->len[d] = len[d];
        x->maxv[d] = max_value[d];
    }
    *out = x;
    return HC_OK;
}

hc_status hc_kplan_cost(const hc_kquery* q, const hc_kindex* const* idx, double level_cost[HC_MAX_VARS],
                        double dom_out[HC_MAX_VARS]) {
    HC_TRY(hc::kplan_check(q, idx));
    bool seen[HC_MAX_VARS] = {false};
    for (uint32_t i = 0; i < q->n_vars; ++i) {
        if (q->order[i] >= q->n_vars || seen[q->order[i]])
            return hc::fail(HC_ERR_ARG, "kplan_cost: order must list every variable once");
        seen[q->order[i]] = true;
    }
    double cost[HC_MAX_VARS] = {0}, dom[HC_MAX_VARS] = {0};
    hc::kplan_costs(q, idx, q->order, cost, dom);
    for (int v = 0; v < HC_MAX_VARS; ++v) {
        if (level_cost) level_cost[v] = v < (int)q->n_vars ? cost[v] : 0.0;
        if (dom_out) dom_out[v] = v < (int)q->n_vars ? dom[v] : 0.0;
    }
    return HC_OK;
}

hc_status hc_choose_korder(const hc_kquery* q, const hc_kindex* const* idx, uint8_t order_out[HC_MAX_VARS]) {
    HC_TRY(hc::kplan_check(q, idx));
    if (!order_out) return hc::fail(HC_ERR_ARG, "choose_korder: NULL order_out");
    const int nv = (int)q->n_vars;
    uint8_t perm[HC_MAX_VARS], best[HC_MAX_VARS];
    for (int i = 0; i < nv; ++i) perm[i] = best[i] = (uint8_t)i;
    double best_cost = INFINITY;
    do {  // lexicographic order, so a tie keeps the smaller order
        double cost[HC_MAX_VARS], dom[HC_MAX_VARS];
        hc::kplan_costs(q, idx, perm, cost, dom);
        double total = 0.0;
        for (int i = 0; i < nv; ++i) total += cost[i];
        if (total < best_cost - 1e-9 * std::max(1.0, fabs(best_cost)) || best_cost == INFINITY) {
            best_cost = total;
            std::copy(perm, perm + nv, best);
        }
    } while (std::next_permutation(perm, perm + nv));
    for (int i = 0; i < HC_MAX_VARS; ++i) order_out[i] = i < nv ? best[i] : (uint8_t)0xFF;
    return HC_OK;
}

}  // extern "C"
