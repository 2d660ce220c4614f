// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/honeycomb.h"

namespace hc {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
hc_status fail(hc_status s, const std::string& msg);
hc_status cuda_fail(cudaError_t e, const char* what);

#define HC_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return ::hc::cuda_fail(_e, #expr); \
    } while (0)

#define HC_TRY(expr)                    \
    do {                                \
        hc_status _s = (expr);          \
        if (_s != HC_OK) return _s;     \
    } while (0)

// Every kernel launch of the library goes through launch_check(), which
// counts it (hc_kernel_launches) and returns the launch error, if any.
void note_launch();
inline cudaError_t launch_check() {
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------- device memory (stream-ordered)
hc_status dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Device-side error word: bit 0 = a bounded wait gave up.
enum : uint32_t { DEV_ERR_TIMEOUT = 1u };

// Limit of each bounded device-side wait, in nanoseconds, for kernels
// launched from now on (hc_set_wait_limit_ns; default 2 s).
uint64_t wait_limit_ns();

// Level arrays V1 and V2 (of indexes and partitioned copies) are allocated
// with LIST_PAD spare entries, so a 16-byte vector load that starts at a
// multiple of 4 entries inside the array stays inside the allocation.
constexpr uint64_t LIST_PAD = 4;

// Longest list the search kernels may iterate: they sum up to 32 bindings'
// list lengths in 32 bits, so every list they iterate must be shorter than
// 2^27 (checked by run_join against the indexes' longest runs).
constexpr uint64_t MAX_LIST_LEN = 1ull << 27;

// Library-wide per-device scratch holding the error word and work counters.
struct DevScratch {
    uint32_t* err;  // [1]
};
hc_status dev_scratch(DevScratch* out);

// -------------------------------------------------------------- owned objects
}  // namespace hc

struct hc_index {
    uint64_t n = 0, l1 = 0;
    uint32_t attr_order = 0, max_first = 0, max_second = 0;
    uint64_t* d_keys = nullptr;  // [n] sorted (first << 32 | second)
    uint32_t* d_v1 = nullptr;    // [l1]
    uint32_t* d_o1 = nullptr;    // [l1 + 1]
    uint32_t* d_v2 = nullptr;    // [n]
    bool stats_only = false;     // sizes only (planning), no device arrays
    float ms_radix = 0.f, ms_boundary = 0.f;  // with HC_BUILD_TIME_KERNELS
    uint32_t n_radix = 0;
    // V1 position map: v1pos[v] = position of v in V1, or V1POS_NONE; built
    // when the first attribute's values are dense enough (v1pos_n = 0: none)
    uint32_t* d_v1pos = nullptr;
    uint32_t v1pos_n = 0;
    // longest run of V2 (rows of one first-attribute value): exact for a
    // built index, the caller's figure (0 = unknown) for a statistics-only one
    uint64_t max_run = 0;
    // bucket directories (search acceleration, see dir_lower_bound): d_g2
    // parallel to V2 for the runs of O1; d_g1 parallel to V1 for the single
    // run [0, l1) when there is no position map
    uint4* d_g2 = nullptr;
    uint4* d_g1 = nullptr;
};

struct hc_partitioned {
    uint64_t n = 0, l1 = 0, n_parts = 0;
    uint32_t pa = 1, pb = 1, seed_a = 0, seed_b = 0;
    cudaStream_t stream = nullptr;
    uint64_t* d_keys = nullptr;        // [n]
    uint32_t* d_bpref = nullptr;       // [np + 1]
    uint32_t* d_v1 = nullptr;          // [<= n]
    uint32_t* d_o1 = nullptr;          // [<= n + 1]
    uint32_t* d_v2 = nullptr;          // [n]
    uint32_t* d_lvl1_start = nullptr;  // [np + 1]
    uint32_t* d_l1 = nullptr;          // [1] device copy of l1
    bool l1_known = false;
    // V1 position map over the concatenated V1 (partitions on the first
    // attribute only, so that each value sits in one partition)
    uint32_t* d_v1pos = nullptr;
    uint32_t v1pos_n = 0;
    // bucket directories: d_g2 parallel to V2 (runs of O1), d_g1 parallel to
    // V1 (one run per partition, lvl1_start) when there is no position map
    uint4* d_g2 = nullptr;
    uint4* d_g1 = nullptr;
};

namespace hc {

// Device control block of one join (hc_run_join, hc_run_kjoin).
struct JoinCtl {
    uint32_t err;
    uint32_t item_ctr[2];
    uint32_t n_entries;  // loop-1 bindings, written by the loop-1 pass
    uint64_t total;      // |Q|
    uint64_t work;       // work counter (stats)
    uint64_t n_items;
    uint32_t chunk_ctr;  // output chunks handed out (single-pass materialize)
    uint32_t overflow;   // 1 when the output pool ran out of chunks
    uint64_t written;    // tuples given an output slot (k-ary materialize)
};

}  // namespace hc

struct hc_result {
    cudaStream_t stream = nullptr;
    uint32_t n_vars = 0;
    uint64_t n_cells = 0;
    hc::JoinCtl* d_ctl = nullptr;
    uint64_t* d_cell_counts = nullptr;
    uint64_t* d_cell_prof = nullptr;  // [n_cells][2] with HC_FLAG_CELL_PROFILE
    uint32_t* d_tuples = nullptr;
    uint64_t n_tuples = 0;
    uint64_t n_items = 0;
    bool materialized = false;
    bool done = false;
    hc::JoinCtl h_ctl{};
    std::vector<hc_partitioned*> parts;
    std::vector<cudaEvent_t> ev;  // timed search launches: ev[2i] before, ev[2i+1] after launch i
    int n_timed = 0;   // search launches bracketed by ev[2i], ev[2i+1]
    int n_search = 0;  // search launches of this join
};

namespace hc {

// V1 position maps (value -> position in V1, a dense direct-address table in
// place of a binary search of V1).  Built only when the values span at most
// V1POS_ROWS_FACTOR entries per row (plus a fixed allowance), so a map costs
// at most about 4 * V1POS_ROWS_FACTOR bytes per row.  The map's length
// (max_value + 1) is stored in 32 bits, so a relation holding the value
// 0xFFFFFFFF never gets one (its length 2^32 would not fit).
constexpr uint32_t V1POS_NONE = 0xFFFFFFFFu;
constexpr uint64_t V1POS_ROWS_FACTOR = 4;
constexpr uint64_t V1POS_ALLOWANCE = 1ull << 20;
inline bool v1pos_eligible(uint64_t rows, uint32_t max_value) {
    return rows > 0 && max_value < 0xFFFFFFFFu &&
           (uint64_t)max_value + 1 <= V1POS_ROWS_FACTOR * rows + V1POS_ALLOWANCE;
}

// --------------------------------------------------------------- device code
#if defined(__CUDACC__)

// MurmurHash3 32-bit finaliser (Appleby, 2011).
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Share of value x among P buckets: (fmix32(x ^ seed) * P) >> 32.
__host__ __device__ __forceinline__ uint32_t share_of(uint32_t x, uint32_t seed, uint32_t P) {
    return (uint32_t)(((uint64_t)fmix32(x ^ seed) * (uint64_t)P) >> 32);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Look-back status words carry their value in the same 64-bit word as the
// flags, so plain relaxed (coherent, unordered) accesses at GPU scope suffice:
// no other memory is read on the strength of a flag.
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Decoupled look-back status word: 2 flag bits over a 62-bit value.
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_VAL = (1ull << 62) - 1;

// The error word of a launch sequence, read past the caches: set by a wait
// that gave up in this kernel or an earlier one on the same stream.  Kernels
// that consume a look-back's output check it first and do nothing once it is
// set, so offsets from an abandoned look-back are never used.
__device__ __forceinline__ bool dev_err_set(const uint32_t* err) {
    return *(const volatile uint32_t*)err != 0u;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Exclusive prefix of tile `tile` by decoupled look-back (Merrill & Garland,
// 2016) over one status word per tile, by a whole warp: lane q reads the word
// of tile top - q, so each round covers 32 predecessors; the round sums the
// values up to the nearest inclusive word and stops there.  Tile ids are
// taken in launch order, so every predecessor has started and each wait
// ends unless the device stalls; a wait longer than wait_ns nanoseconds
// sets DEV_ERR_TIMEOUT in *err and returns what it has (a prefix no larger
// than the true one).  All 32 lanes call it and all get the result.
__device__ __forceinline__ uint64_t warp_lookback(const uint64_t* status, uint32_t tile, uint32_t* err,
                                                  uint64_t wait_ns) {
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t excl = 0;
    int64_t top = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer_ns();
    while (top >= 0) {
        const int64_t t = top - (int64_t)lane;
        uint64_t x = t >= 0 ? ld_relaxed(status + t) : LB_INC;  // before tile 0: an inclusive zero
        for (uint32_t spins = 0;; ++spins) {
            const bool ready = (x & ~LB_VAL) != 0;
            if (__all_sync(0xffffffffu, ready)) break;
            if (__any_sync(0xffffffffu, globaltimer_ns() - t0 > wait_ns)) {
                if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                return excl;
            }
            if (spins > 16) __nanosleep(32);
            if (!ready) x = ld_relaxed(status + t);
        }
        const uint32_t incm = __ballot_sync(0xffffffffu, (x & LB_INC) != 0);
        const uint32_t upto = incm ? (uint32_t)__ffs(incm) - 1u : 31u;
        excl += warp_sum64(lane <= upto ? (x & LB_VAL) : 0);
        if (incm) break;
        top -= 32;
    }
    return excl;
}

// Warp-wide inclusive scan (sum) of a 32-bit value.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= (uint32_t)d) v += u;
    }
    return v;
}
__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= (uint32_t)d) v += u;
    }
    return v;
}
__device__ __forceinline__ uint32_t load_ro(const uint32_t* p) { return __ldg(p); }
__device__ __forceinline__ uint32_t load_ro(uint32_t* p) { return *p; }

// First index in [lo, hi) of sorted a[] whose value is >= x (hi if none).
// Branch-free halving: each step keeps the upper half when its first
// element is still below x.
template <typename P>
__device__ __forceinline__ uint32_t lower_bound_u32(P a, uint32_t lo, uint32_t hi, uint32_t x) {
    uint32_t len = hi - lo;
    if (len == 0) return lo;
    uint32_t base = lo;
    while (len > 1) {
        const uint32_t half = len >> 1;
        base = load_ro(a + base + half) < x ? base + half : base;
        len -= half;
    }
    return base + (load_ro(a + base) < x ? 1u : 0u);
}

// Membership form of the same search: the last position i in [lo, hi) with
// a[i] <= x (lo if none), its value in w, true when w == x (then i is the
// first position holding x, the lower bound).  The value at the answer comes
// out of the search itself, so no second read is needed.  hi > lo.
template <typename P>
__device__ __forceinline__ bool find_u32(P a, uint32_t lo, uint32_t hi, uint32_t x, uint32_t& pos) {
    uint32_t len = hi - lo, base = lo;
    while (len > 1) {
        const uint32_t half = len >> 1;
        base = load_ro(a + base + half) <= x ? base + half : base;
        len -= half;
    }
    pos = base;
    return load_ro(a + base) == x;
}

// ------------------------------------------------------- bucket directories
// The search primitive of Sec. 5 ("search(V, x)": the first position of a
// sorted list holding a value >= x) over a run a[lo, hi) of n >= DIR_MIN
// distinct ascending values, narrowed by a directory stored in an array g of
// 16-byte entries parallel to a.  With vmin = a[lo], vmax = a[hi-1] the run's
// values fall in nb = ((vmax - vmin) >> s) + 1 buckets of width 2^s, where
// s = dir_shift(n, vmax - vmin) makes nb at most n (one to four values a
// bucket on average).  Entry k of the run, g[lo + k] for k < nb, holds p_k =
// the first position in [lo, hi) whose value is in bucket k or above, and
// the values a[p_k], a[p_k + 1], a[p_k + 2] (~0 past the run); every p_k
// exists, since vmax lies in the last bucket.  A search of x in [vmin, vmax]
// reads the entry of x's bucket k: every value before p_k is below
// vmin + k 2^s <= x, so the answer is the first of p_k, p_k + 1, p_k + 2
// whose value is >= x, and otherwise lies further on (a forward walk that
// stops at the latest at hi - 1, because vmax >= x).  A value of the entry
// past the run is never consulted: it lies beyond hi - 1, where a value
// >= x already ended the search.  The answer is the plain binary search's.
// The paper's fixed-stride ("quadratic") search jumps by strides to reach the
// stride holding x; here that stride is addressed directly, and its first
// three values come with it, so a search is one 16-byte read unless x lies
// beyond the third value of its bucket.
constexpr uint32_t DIR_MIN = 16;  // shorter runs have no directory

// Bucket width exponent for a run of n >= DIR_MIN values spanning `span`:
// with 2^lm <= n < 2^(lm+1) and s the bit length of span >> lm, 2^s > span
// >> lm, so the last bucket index span >> s is below 2^lm <= n; s <= 29.
__device__ __forceinline__ uint32_t dir_shift(uint32_t n, uint32_t span) {
    const uint32_t lm = 31u - __clz(n);
    const uint32_t t = span >> lm;
    return t ? 32u - __clz(t) : 0u;
}

__device__ __forceinline__ uint4 dir_load(const uint4* g, uint64_t i) { return __ldg(g + i); }

// Membership of x in the run a[lo, hi) from the entry e of x's bucket, x in
// [vmin, vmax]: the position of the first value >= x in pos, true when that
// value is x.  A position outside the run (a directory of unsorted input, a
// caller's broken promise) is pulled back to hi - 1, where the walk ends.
template <typename P>
__device__ __forceinline__ bool dir_walk_find(P a, uint4 e, uint32_t hi, uint32_t x, uint32_t& pos) {
    uint32_t p = e.x;
    if (p >= hi) {
        p = hi - 1;
        uint32_t w = load_ro(a + p);
        while (w < x) w = load_ro(a + (++p));
        pos = p;
        return w == x;
    }
    if (e.y >= x) {
        pos = p;
        return e.y == x;
    }
    if (e.z >= x) {
        pos = p + 1;
        return e.z == x;
    }
    if (e.w >= x) {
        pos = p + 2;
        return e.w == x;
    }
    p += 3;
    uint32_t w = load_ro(a + p);
    while (w < x) w = load_ro(a + (++p));
    pos = p;
    return w == x;
}

// Membership of x in the run a[lo, hi) and, when present, its position:
// through the run's directory when g is given and the run has at least dmin
// (>= DIR_MIN) values, else by find_u32.
template <typename P>
__device__ __forceinline__ bool dir_find(P a, const uint4* __restrict__ g, uint32_t lo, uint32_t hi, uint32_t x,
                                         uint32_t dmin, uint32_t& pos) {
    const uint32_t n = hi - lo;
    pos = lo;
    if (n == 0) return false;
    if (g == nullptr || n < dmin) return find_u32(a, lo, hi, x, pos);
    const uint32_t vmin = load_ro(a + lo), vmax = load_ro(a + hi - 1);
    if (x <= vmin) return x == vmin;
    if (x > vmax) return false;
    const uint32_t k = (x - vmin) >> dir_shift(n, vmax - vmin);
    return dir_walk_find(a, dir_load(g, (uint64_t)lo + k), hi, x, pos);
}

#endif  // __CUDACC__

// --------------------------------------------------------------- host entry
// Sorting and CoCo construction (hc_sort.cu).  BUILD_NO_DIRECTORIES (a
// flag of internal callers that only want the sorted keys) skips the
// position map and the bucket directories.
constexpr uint32_t BUILD_NO_DIRECTORIES = 0x80000000u;
hc_status build_index_impl(const uint32_t* d_pairs, uint64_t n, uint32_t attr_order, uint32_t flags,
                           cudaStream_t s, hc_index** out);
hc_status partition_impl(const hc_index* idx, uint32_t seed_a, uint32_t pa, uint32_t seed_b,
                         uint32_t pb, cudaStream_t s, hc_partitioned** out);
void partitioned_release(hc_partitioned* p, cudaStream_t s);
void index_release(hc_index* idx, cudaStream_t s);
hc_status build_unary_impl(const uint32_t* d_values, uint64_t n, uint32_t max_value, cudaStream_t s,
                           hc_index** out);
// Bucket directory g (parallel to a, alen 16-byte entries, allocated here) of the
// runs [o[r], o[r+1]) of a, r < nruns (nruns = min(nruns_max, *d_nruns) when
// d_nruns is given), or with o == NULL of the one run [0, nruns_max);
// nothing is computed once *d_err is set.
hc_status build_directory(const uint32_t* a, uint64_t alen, const uint32_t* o, uint64_t nruns_max,
                          const uint32_t* d_nruns, const uint32_t* d_err, cudaStream_t s, uint4** out_g);

// Device-wide exclusive scan of counts into uint64 offsets; out[n] receives
// the total.  n = min(n_max, *d_n) when d_n is given (a device-side count),
// else n_max.  A timed-out look-back sets DEV_ERR_TIMEOUT in *d_err.
// Temporary memory is stream-ordered.
hc_status exclusive_scan_u32_to_u64(const uint32_t* d_in, uint64_t* d_out, uint64_t n_max, const uint32_t* d_n,
                                    uint32_t* d_err, cudaStream_t s);
hc_status exclusive_scan_u64(const uint64_t* d_in, uint64_t* d_out, uint64_t n_max, const uint32_t* d_n,
                             uint32_t* d_err, cudaStream_t s);
hc_status partitioned_sync(hc_partitioned* p);
void result_release(hc_result* r);
// Record the event that opens (end = false) or closes timed search launch
// R->n_timed on s, creating it first; closing advances n_timed.
hc_status time_mark(hc_result* R, bool end, cudaStream_t s);
struct HostOut;
hc_status run_join_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm, cudaStream_t s,
                        hc_result** out, const HostOut* host = nullptr);
hc_status run_join_to_host_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm,
                                uint32_t* h_tuples, uint64_t capacity, uint64_t* count_out, cudaStream_t s);
hc_status join_footprint_impl(const hc_query* q, const hc_index* const* idx, const hc_join_params* prm,
                              uint64_t* bytes);
hc_status batch_create(const hc_query* qs, const hc_index* const* idx_flat, const hc_join_params* prm, uint32_t n,
                       cudaStream_t s, hc_batch** out);
hc_status batch_launch(hc_batch* b, cudaStream_t s);
hc_status batch_capture(hc_batch* b, cudaStream_t s);
hc_status batch_counts(hc_batch* b, uint64_t* counts);
void batch_release(hc_batch* b);

int num_sms();

}  // namespace hc
