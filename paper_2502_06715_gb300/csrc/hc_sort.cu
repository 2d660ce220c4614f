// CoCo construction on the GPU (Sec. 4 "Construction of CoCo"): an LSD radix
// sort of the rows packed as 64-bit keys (first << 32 | second), then a
// single-pass run-boundary scan that writes the trie levels V1, O1, V2.
// HyperCube partitioning (Sec. 4, partitioning paragraphs) reuses the same
// radix pass with the partition id as the digit (a stable scatter of the
// already sorted rows, so each partition stays sorted) and a segmented
// run-boundary scan that builds one CoCo per partition.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "hc_internal.cuh"

namespace hc {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // 4096 keys per tile
constexpr int RADIX = 256;
constexpr int MAX_PASSES = 8;

// How a pass extracts its 8-bit digit: a byte of the key (mode 0), or a byte
// of the key's HyperCube partition id (mode 1).
struct DigitSpec {
    uint32_t mode, shift;
    uint32_t seed_a, pa, seed_b, pb;
};

__device__ __forceinline__ uint32_t partition_id(uint64_t key, uint32_t seed_a, uint32_t pa,
                                                 uint32_t seed_b, uint32_t pb) {
    return share_of((uint32_t)(key >> 32), seed_a, pa) * pb + share_of((uint32_t)key, seed_b, pb);
}

__device__ __forceinline__ uint32_t digit_of(uint64_t key, const DigitSpec& d) {
    uint64_t v = d.mode == 0 ? key : (uint64_t)partition_id(key, d.seed_a, d.pa, d.seed_b, d.pb);
    return (uint32_t)(v >> d.shift) & 0xFFu;
}

__device__ __forceinline__ uint64_t pack_row(const uint2* pairs, uint64_t i, uint32_t ao) {
    uint2 r = pairs[i];
    uint32_t a = ao ? r.y : r.x, b = ao ? r.x : r.y;
    return ((uint64_t)a << 32) | b;
}

// Per-call control block in device memory.
struct Ctl {
    uint32_t err;
    uint32_t dup;
    uint32_t maxv[2];
    uint32_t l1;
    uint32_t maxrun;  // longest run of the level-1 entries (maxrun_kernel)
    uint32_t tile_counter[MAX_PASSES + 2];
};

// ------------------------------------------------------------ column maxima
__global__ void colmax_kernel(const uint2* __restrict__ pairs, uint64_t n, Ctl* ctl) {
    uint32_t m0 = 0, m1 = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint2 r = pairs[i];
        m0 = max(m0, r.x);
        m1 = max(m1, r.y);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, d));
        m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, d));
    }
    if (lane_id() == 0) {
        atomicMax(&ctl->maxv[0], m0);
        atomicMax(&ctl->maxv[1], m1);
    }
}

// ------------------------------------------------------------- histograms
// Digit histograms of every pass in one read of the input.
template <bool FROM_PAIRS>
__global__ void __launch_bounds__(SORT_THREADS) hist_kernel(const void* __restrict__ in, uint64_t n,
                                                            uint32_t ao, const DigitSpec* __restrict__ ds,
                                                            int npasses, uint32_t* __restrict__ ghist) {
    __shared__ uint32_t sh[MAX_PASSES][RADIX];
    __shared__ DigitSpec sds[MAX_PASSES];
    for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
    if (threadIdx.x < npasses) sds[threadIdx.x] = ds[threadIdx.x];
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = FROM_PAIRS ? pack_row((const uint2*)in, i, ao) : ((const uint64_t*)in)[i];
        for (int p = 0; p < npasses; ++p) atomicAdd(&sh[p][digit_of(k, sds[p])], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x) {
        uint32_t v = (&sh[0][0])[i];
        if (v) atomicAdd(&ghist[i], v);
    }
}

// Exclusive scan of each pass's 256 counters (one block of 256 per pass).
__global__ void digit_scan_kernel(uint32_t* __restrict__ ghist) {
    __shared__ uint32_t wsum[SORT_WARPS];
    uint32_t* h = ghist + blockIdx.x * RADIX;
    uint32_t v = h[threadIdx.x];
    uint32_t inc = warp_incl_scan(v);
    if (lane_id() == 31) wsum[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t add = 0;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) add += wsum[w];
    __syncthreads();
    h[threadIdx.x] = inc - v + add;
}

// --------------------------------------------------------- onesweep pass
// One stable LSD pass over 8 bits (Adinets & Merrill's single-pass "onesweep"
// structure).  A tile of PASS_TILE keys is loaded into registers, every key is
// ranked among the equal digits before it in its warp, the warps' digit
// counts are scanned into the tile's digit runs, and the tile's global digit
// offsets come from a decoupled look-back over the tiles before it.  The keys
// are staged in shared memory in digit order and each digit run is written
// contiguously.  Row counts are below 2^32, so offsets are 32-bit.
//
// Ranking: lanes holding the same digit find each other through a per-warp,
// per-digit word in shared memory that each lane ORs its lane bit into; the
// group's highest lane advances the warp's digit counter by the group size.
// Ranks follow (item, lane) order, which is the tile's row order, so the
// pass is stable.
constexpr int PASS_THREADS = 256;
constexpr int PASS_WARPS = PASS_THREADS / 32;
constexpr int PASS_ITEMS = 24;
constexpr int PASS_TILE = PASS_THREADS * PASS_ITEMS;  // 6144 keys per tile
constexpr int PASS_LOOKBACK = 8;                      // status words read per look-back round

enum : int { SRC_KEYS = 0, SRC_PAIRS = 1 };
enum : int { DIGIT_BYTE = 0, DIGIT_PARTITION = 1 };

template <int DIG>
__device__ __forceinline__ uint32_t pass_digit(uint64_t key, const DigitSpec& d) {
    if (DIG == DIGIT_BYTE) return (uint32_t)(key >> d.shift) & 0xFFu;
    return (partition_id(key, d.seed_a, d.pa, d.seed_b, d.pb) >> d.shift) & 0xFFu;
}

// Exclusive prefix of one digit's count over the tiles before `tile`:
// status[t * RADIX] holds tile t's word for this digit.  Each round reads
// PASS_LOOKBACK words at once and stops at the nearest inclusive one.  A
// wait longer than wait_ns sets DEV_ERR_TIMEOUT in *err and returns the
// prefix summed so far (no larger than the true one).
__device__ __forceinline__ uint64_t digit_lookback(const uint64_t* status, uint32_t tile, uint32_t* err,
                                                   uint64_t wait_ns) {
    uint64_t excl = 0;
    int64_t t = (int64_t)tile - 1;
    while (t >= 0) {
        uint64_t wv[PASS_LOOKBACK];
#pragma unroll
        for (int q = 0; q < PASS_LOOKBACK; ++q)
            wv[q] = (t - q >= 0) ? ld_relaxed(status + (uint64_t)(t - q) * RADIX) : LB_INC;
        bool done = false;
#pragma unroll
        for (int q = 0; q < PASS_LOOKBACK; ++q) {
            if (done) continue;
            uint64_t x = wv[q];
            if ((x & ~LB_VAL) == 0) {
                const uint64_t* p = status + (uint64_t)(t - q) * RADIX;
                const uint64_t t0 = globaltimer_ns();
                uint32_t spins = 0;
                do {
                    if (++spins > 16) __nanosleep(32);
                    x = ld_relaxed(p);
                    if ((x & ~LB_VAL) == 0 && globaltimer_ns() - t0 > wait_ns) {
                        atomicOr(err, DEV_ERR_TIMEOUT);
                        return excl;
                    }
                } while ((x & ~LB_VAL) == 0);
            }
            excl += x & LB_VAL;
            done = (x & LB_INC) != 0;
        }
        if (done) break;
        t -= PASS_LOOKBACK;
    }
    return excl;
}

// A pass does nothing once *err is set (by an earlier pass that gave up a
// wait): its input would not hold the rows its digit counts describe.  With
// `withhold` (testing only) tile 0 never publishes its status words, so every
// wait on them runs out.
template <int SRC, int DIG>
__global__ void __launch_bounds__(PASS_THREADS, 2) onesweep_kernel(
    const void* __restrict__ in, uint64_t* __restrict__ out, uint32_t n, uint32_t ao, DigitSpec ds,
    const uint32_t* __restrict__ gbase, uint64_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
    uint32_t* __restrict__ err, uint64_t wait_ns, uint32_t withhold) {
    constexpr bool KEEP_DIGITS = DIG == DIGIT_PARTITION;  // hashing twice costs more than a byte of smem
    __shared__ uint64_t skeys[PASS_TILE];
    __shared__ uint8_t sdig[KEEP_DIGITS ? PASS_TILE : 1];
    __shared__ uint32_t whist[PASS_WARPS][RADIX];  // per-warp digit counters, later run starts
    __shared__ uint32_t peers_word[PASS_WARPS][RADIX];
    __shared__ uint32_t goff[RADIX];
    __shared__ uint32_t wsum[PASS_WARPS];
    __shared__ uint32_t s_tile;

    const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    if (tid == 0) s_tile = dev_err_set(err) ? 0xFFFFFFFFu : atomicAdd(tile_counter, 1u);
    for (int i = tid; i < PASS_WARPS * RADIX; i += PASS_THREADS) {
        (&whist[0][0])[i] = 0;
        (&peers_word[0][0])[i] = 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile == 0xFFFFFFFFu) return;  // no tile id taken: no later tile waits on this block
    const uint32_t base = tile * (uint32_t)PASS_TILE;
    const uint32_t wb = base + w * (PASS_ITEMS * 32) + lane;  // row of item 0 of this lane
    const bool full = n - base >= (uint32_t)PASS_TILE;

    // all loads first, so that they are in flight together
    uint64_t k[PASS_ITEMS];
    if (full) {
#pragma unroll
        for (int j = 0; j < PASS_ITEMS; ++j)
            k[j] = SRC == SRC_PAIRS ? pack_row((const uint2*)in + wb, j * 32, ao) : ((const uint64_t*)in + wb)[j * 32];
    } else {
#pragma unroll
        for (int j = 0; j < PASS_ITEMS; ++j) {
            const uint32_t i = wb + j * 32;
            k[j] = 0;
            if (i < n) k[j] = SRC == SRC_PAIRS ? pack_row((const uint2*)in, i, ao) : ((const uint64_t*)in)[i];
        }
    }

    const uint32_t lt = lanemask_lt();
    uint32_t rp[PASS_ITEMS];  // rank among the warp's equal digits | digit << 16 (digit RADIX: no row)
#pragma unroll
    for (int j = 0; j < PASS_ITEMS; ++j) {
        const bool valid = full || wb + j * 32 < n;
        const uint32_t d = valid ? pass_digit<DIG>(k[j], ds) : RADIX;
        uint32_t peers = 0, b = 0;
        if (valid) atomicOr(&peers_word[w][d], 1u << lane);
        __syncwarp();
        if (valid) peers = peers_word[w][d];
        __syncwarp();
        const uint32_t below = __popc(peers & lt);
        if (valid && (peers >> lane) == 1u) {  // highest lane of the group
            b = whist[w][d];
            whist[w][d] = b + below + 1u;
            peers_word[w][d] = 0;
        }
        b = __shfl_sync(0xffffffffu, b, valid ? 31u - __clz(peers) : lane);
        rp[j] = (b + below) | (d << 16);
        __syncwarp();
    }
    __syncthreads();

    // per digit (one per thread): warp prefix, tile total, aggregate published
    const uint32_t d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < PASS_WARPS; ++q) {
        const uint32_t c = whist[q][d];
        whist[q][d] = run;
        run += c;
    }
    uint64_t* st = status + (uint64_t)tile * RADIX + d;
    if (!(withhold && tile == 0)) st_relaxed(st, (tile == 0 ? LB_INC : LB_AGG) | run);
    const uint32_t inc = warp_incl_scan(run);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t lstart = inc - run;
#pragma unroll
    for (uint32_t q = 0; q < (uint32_t)PASS_WARPS; ++q) lstart += q < w ? wsum[q] : 0u;
#pragma unroll
    for (int q = 0; q < PASS_WARPS; ++q) whist[q][d] += lstart;
    __syncthreads();

    // stage the tile in digit order (keys leave the registers before the look-back)
#pragma unroll
    for (int j = 0; j < PASS_ITEMS; ++j) {
        const uint32_t dg = rp[j] >> 16;
        if (full || dg < RADIX) {
            const uint32_t pos = whist[w][dg] + (rp[j] & 0xFFFFu);
            skeys[pos] = k[j];
            if (KEEP_DIGITS) sdig[pos] = (uint8_t)dg;
        }
    }
    uint64_t excl = 0;
    if (tile != 0) {
        excl = digit_lookback(status + d, tile, err, wait_ns);
        st_relaxed(st, LB_INC | (excl + run));
    }
    goff[d] = gbase[d] + (uint32_t)excl - lstart;  // mod 2^32; goff + row is below n
    __syncthreads();

    // unrolled for a full tile, so that the shared-memory reads of all items
    // are in flight together
    if (full) {
#pragma unroll
        for (int j = 0; j < PASS_ITEMS; ++j) {
            const uint32_t i = tid + j * PASS_THREADS;
            const uint64_t key = skeys[i];
            const uint32_t dg = KEEP_DIGITS ? sdig[i] : pass_digit<DIG>(key, ds);
            out[goff[dg] + i] = key;
        }
    } else {
        for (uint32_t i = tid; i < n - base; i += PASS_THREADS) {
            const uint64_t key = skeys[i];
            const uint32_t dg = KEEP_DIGITS ? sdig[i] : pass_digit<DIG>(key, ds);
            out[goff[dg] + i] = key;
        }
    }
}

// Pack rows into keys without sorting (a relation with a single key value).
__global__ void pack_kernel(const uint2* __restrict__ pairs, uint64_t* __restrict__ out, uint64_t n, uint32_t ao) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = pack_row(pairs, i, ao);
}

// ------------------------------------------------------ run-boundary scan
// Single pass over the sorted keys.  Row i opens a level-1 entry when its
// first attribute (or, with SEGMENTED, its partition id) differs from row
// i-1.  Flags are counted with ballots, the tile's offset comes from a
// decoupled look-back (one warp reads 32 predecessors per round), and every
// flagged row writes V1[pos] = first value and O1[pos] = i; every row writes
// V2[i] = second value (before the look-back, as it needs no offset).  The last tile writes O1[l1] = n and l1.  Equal
// adjacent keys mark a duplicate row.  Rows are warp-striped: item j of lane
// q of warp w is row tile * SORT_TILE + w * 32 * SORT_ITEMS + 32 j + q, so
// row i-1 of a lane-0 row is lane 31's row of the previous item.
// The scan does nothing once ctl->err is set (a radix pass gave up a wait,
// so the keys are not sorted); `withhold` (testing only) keeps tile 0 from
// publishing its status word, so every wait on it runs out.
template <bool SEGMENTED>
__global__ void __launch_bounds__(SORT_THREADS, 3) boundary_kernel(
    const uint64_t* __restrict__ keys, uint64_t n, uint32_t seed_a, uint32_t pa, uint32_t seed_b,
    uint32_t pb, uint32_t* __restrict__ v1, uint32_t* __restrict__ o1, uint32_t* __restrict__ v2,
    uint64_t* __restrict__ status, uint32_t* __restrict__ tile_counter, Ctl* __restrict__ ctl, uint64_t wait_ns,
    uint32_t withhold) {
    __shared__ uint32_t wsum[SORT_WARPS];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_tile;
    const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    if (tid == 0) s_tile = dev_err_set(&ctl->err) ? 0xFFFFFFFFu : atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile == 0xFFFFFFFFu) return;
    const uint64_t base = (uint64_t)tile * SORT_TILE + (uint64_t)w * (SORT_ITEMS * 32);
    const bool full = base + SORT_ITEMS * 32 <= n;

    uint64_t k[SORT_ITEMS];
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
        k[j] = (full || i < n) ? keys[i] : 0;
    }
    // the row before the warp's first row
    uint64_t carry = (lane == 0 && base > 0 && base < n) ? keys[base - 1] : 0;
    auto pid = [&](uint64_t key) { return partition_id(key, seed_a, pa, seed_b, pb); };
    uint32_t carry_pid = SEGMENTED && lane == 0 && base > 0 && base < n ? pid(carry) : 0;

    uint32_t ball[SORT_ITEMS];
    uint32_t wcount = 0;
    bool dup = false;
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
        const bool valid = full || i < n;
        const uint32_t my_pid = SEGMENTED ? pid(k[j]) : 0;
        uint64_t prev = __shfl_up_sync(0xffffffffu, k[j], 1);
        uint32_t prev_pid = SEGMENTED ? __shfl_up_sync(0xffffffffu, my_pid, 1) : 0;
        if (lane == 0) {
            prev = carry;
            prev_pid = carry_pid;
        }
        bool flag = false;
        if (valid) {
            flag = i == 0 || (prev >> 32) != (k[j] >> 32) || (SEGMENTED && prev_pid != my_pid);
            dup |= i > 0 && prev == k[j];
        }
        ball[j] = __ballot_sync(0xffffffffu, flag);
        wcount += __popc(ball[j]);
        if (valid) v2[i] = (uint32_t)k[j];  // V2 needs no offset: written before the look-back
        // lane 31's row precedes lane 0's row of the next item
        const uint64_t last = __shfl_sync(0xffffffffu, k[j], 31);
        const uint32_t last_pid = SEGMENTED ? __shfl_sync(0xffffffffu, my_pid, 31) : 0;
        if (lane == 0) {
            carry = last;
            carry_pid = last_pid;
        }
    }
    if (__any_sync(0xffffffffu, dup) && lane == 0) atomicOr(&ctl->dup, 1u);
    if (lane == 0) wsum[w] = wcount;
    __syncthreads();
    if (w == 0) {
        const uint32_t tot = warp_sum64(lane < (uint32_t)SORT_WARPS ? wsum[lane] : 0u);
        uint64_t* st = status + tile;
        if (lane == 0 && !(withhold && tile == 0)) st_relaxed(st, (tile == 0 ? LB_INC : LB_AGG) | tot);
        uint64_t excl = 0;
        if (tile != 0) {
            excl = warp_lookback(status, tile, &ctl->err, wait_ns);
            if (lane == 0) st_relaxed(st, LB_INC | (excl + tot));
        }
        if (lane == 0) {
            s_excl = excl;
            const uint64_t tile_end = (uint64_t)tile * SORT_TILE + SORT_TILE;
            if (tile_end >= n) {  // the tile holding the last row closes the arrays
                o1[excl + tot] = (uint32_t)n;
                ctl->l1 = (uint32_t)(excl + tot);
            }
        }
    }
    __syncthreads();
    uint64_t pos = s_excl;
    for (uint32_t q = 0; q < w; ++q) pos += wsum[q];
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * 32 + lane;
        if (ball[j] >> lane & 1u) {  // flagged rows are valid rows
            const uint64_t p = pos + __popc(ball[j] & lanemask_lt());
            v1[p] = (uint32_t)(k[j] >> 32);
            o1[p] = (uint32_t)i;
        }
        pos += __popc(ball[j]);
    }
}

// B^pref and the level-1 directory of a partitioned relation: partition p
// starts at the first row whose partition id is >= p (ids ascend along R~),
// and its level 1 at the first entry whose row offset is >= that start.
__global__ void directory_kernel(const uint64_t* __restrict__ keys, uint64_t n, uint32_t seed_a,
                                 uint32_t pa, uint32_t seed_b, uint32_t pb,
                                 const uint32_t* __restrict__ o1, const Ctl* __restrict__ ctl,
                                 uint32_t* __restrict__ bpref, uint32_t* __restrict__ lvl1_start) {
    const uint32_t np = pa * pb;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p <= np; p += gridDim.x * blockDim.x) {
        uint64_t lo = 0, hi = n;
        while (lo < hi) {
            uint64_t mid = lo + ((hi - lo) >> 1);
            if (partition_id(keys[mid], seed_a, pa, seed_b, pb) < p)
                lo = mid + 1;
            else
                hi = mid;
        }
        bpref[p] = (uint32_t)lo;
        lvl1_start[p] = lower_bound_u32(o1, 0u, ctl->l1, (uint32_t)lo);
    }
}

// V1 position map: pos[V1[i]] = i for i < l1 (l1 from *d_l1 when given).
// V1 values are distinct, so every entry is written at most once.  A value
// at or past the map's length pos_n (a caller's max_value below the data)
// is not written; a lookup of it then misses, as the map's bound check in the
// search tells it to.
__global__ void v1pos_kernel(const uint32_t* __restrict__ v1, uint64_t l1_max, const uint32_t* __restrict__ d_l1,
                             uint32_t* __restrict__ pos, uint32_t pos_n) {
    const uint64_t l1 = d_l1 ? min(l1_max, (uint64_t)*d_l1) : l1_max;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < l1; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = v1[i];
        if (v < pos_n) pos[v] = (uint32_t)i;
    }
}

// Longest run of a CoCo level: max over i < l1 of O1[i+1] - O1[i], with l1
// read from ctl (a device-side count); nothing once ctl->err is set.
__global__ void maxrun_kernel(const uint32_t* __restrict__ o1, uint64_t l1_max, Ctl* __restrict__ ctl) {
    if (dev_err_set(&ctl->err)) return;
    const uint64_t l1 = min(l1_max, (uint64_t)ctl->l1);
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < l1; i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, o1[i + 1] - o1[i]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    if (lane_id() == 0 && m) atomicMax(&ctl->maxrun, m);
}

// Bucket directory of the runs of a level (layout at dir_lower_bound): the
// runs [o[r], o[r+1]) for r < nruns, or with o == NULL the one run
// [0, nruns_max).  Element-parallel: a block takes tiles of DIRB_TILE
// consecutive positions; thread 0 finds the runs that hold the tile's first
// and last positions, and each thread finds the run of its position by a
// binary search of the run starts between them.  The value at position j
// opens the buckets above its predecessor's bucket up to its own and writes
// entry (j, a[j], a[j+1], a[j+2]) for each (~0 past the run).  Buckets are
// clamped to [0, nb - 1], so unsorted input (never produced by the builders
// here) cannot write outside the run.
constexpr uint32_t DIRB_TILE = 2048;

__global__ void __launch_bounds__(256) dir_build_kernel(const uint32_t* __restrict__ a, const uint32_t* __restrict__ o,
                                                        uint64_t nruns_max, const uint32_t* __restrict__ d_nruns,
                                                        uint4* __restrict__ g, const uint32_t* __restrict__ err) {
    __shared__ uint32_t s_r0, s_r1;
    if (err && dev_err_set(err)) return;
    const uint32_t nruns = o == nullptr ? 1u : (uint32_t)(d_nruns ? min(nruns_max, (uint64_t)*d_nruns) : nruns_max);
    const uint32_t total = o == nullptr ? (uint32_t)nruns_max : o[nruns];
    for (uint32_t base = blockIdx.x * DIRB_TILE; base < total; base += gridDim.x * DIRB_TILE) {
        const uint32_t end = min(base + DIRB_TILE, total);
        __syncthreads();  // the previous tile's run bounds are no longer read
        if (threadIdx.x == 0) {
            uint32_t r0 = 0, r1 = 0;
            if (o != nullptr) {
                // last r with o[r] <= base, and last r with o[r] <= end - 1
                uint32_t lo = 0, hi = nruns;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (o[mid] <= base) lo = mid; else hi = mid;
                }
                r0 = lo;
                hi = nruns;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (o[mid] <= end - 1) lo = mid; else hi = mid;
                }
                r1 = lo;
            }
            s_r0 = r0;
            s_r1 = r1;
        }
        __syncthreads();
        const uint32_t r0 = s_r0, r1 = s_r1;
        for (uint32_t j = base + threadIdx.x; j < end; j += blockDim.x) {
            uint32_t lo = 0, hi = total;
            if (o != nullptr) {
                uint32_t rl = r0, rh = r1 + 1;  // last r in [r0, r1] with o[r] <= j
                while (rh - rl > 1) {
                    const uint32_t mid = (rl + rh) >> 1;
                    if (o[mid] <= j) rl = mid; else rh = mid;
                }
                lo = o[rl];
                hi = o[rl + 1];
            }
            if (hi < lo || hi - lo < DIR_MIN) continue;
            const uint32_t vmin = a[lo], vmax = a[hi - 1];
            const uint32_t sh = dir_shift(hi - lo, vmax - vmin);
            const uint32_t kmax = (vmax - vmin) >> sh;  // nb - 1 < hi - lo
            const uint32_t v = a[j];
            const uint32_t k = min((v - vmin) >> sh, kmax);
            const uint32_t k0 = j == lo ? 0u : min((a[j - 1] - vmin) >> sh, kmax) + 1u;
            const uint4 e = make_uint4(j, v, j + 1 < hi ? a[j + 1] : ~0u, j + 2 < hi ? a[j + 2] : ~0u);
            for (uint32_t b = k0; b <= k; ++b) g[lo + b] = e;
        }
    }
}

// ----------------------------------------------------------- device scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of in[0..n) into out[0..n), out[n] = total.  n is read from
// *d_n when given (a count produced on the device), else n_max is used; the
// grid covers n_max elements and tiles past n contribute nothing.  Thread t
// of a tile owns SCAN_ITEMS consecutive elements; with VEC (both arrays
// 16-byte aligned) a full tile moves them as 16-byte vectors.  The tile
// offset comes from a warp-wide decoupled look-back.
// Does nothing once *err is set: its input then comes from a pass that gave
// up a wait.
template <typename T, bool VEC>
__global__ void __launch_bounds__(SCAN_THREADS) scan_kernel(const T* __restrict__ in, uint64_t* __restrict__ out,
                                                            uint64_t n_max, const uint32_t* __restrict__ d_n,
                                                            uint64_t* __restrict__ status,
                                                            uint32_t* __restrict__ tile_counter,
                                                            uint32_t* __restrict__ err, uint64_t wait_ns) {
    __shared__ uint64_t wsum[SCAN_THREADS / 32];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_tile;
    const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    const uint64_t n = d_n ? (n_max < (uint64_t)*d_n ? n_max : (uint64_t)*d_n) : n_max;
    const uint64_t ntiles = (n_max + SCAN_TILE - 1) / SCAN_TILE;
    if (tid == 0) s_tile = dev_err_set(err) ? 0xFFFFFFFFu : atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile == 0xFFFFFFFFu) return;
    const uint64_t base = (uint64_t)tile * SCAN_TILE + (uint64_t)tid * SCAN_ITEMS;
    const bool full = (uint64_t)(tile + 1) * SCAN_TILE <= n;
    uint64_t v[SCAN_ITEMS];
    if (VEC && full) {
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / PER; ++q) {
            const uint4 u = reinterpret_cast<const uint4*>(in + base)[q];
            if (sizeof(T) == 4) {
                v[q * 4 + 0] = u.x;
                v[q * 4 + 1] = u.y;
                v[q * 4 + 2] = u.z;
                v[q * 4 + 3] = u.w;
            } else {
                v[q * 2 + 0] = ((uint64_t)u.y << 32) | u.x;
                v[q * 2 + 1] = ((uint64_t)u.w << 32) | u.z;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) v[j] = base + j < n ? (uint64_t)in[base + j] : 0;
    }
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) sum += v[j];
    const uint64_t inc = warp_incl_scan64(sum);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint64_t tot = warp_sum64(lane < (uint32_t)(SCAN_THREADS / 32) ? wsum[lane] : 0);
        uint64_t* st = status + tile;
        if (lane == 0) st_relaxed(st, (tile == 0 ? LB_INC : LB_AGG) | tot);
        uint64_t excl = 0;
        if (tile != 0) {
            excl = warp_lookback(status, tile, err, wait_ns);
            if (lane == 0) st_relaxed(st, LB_INC | (excl + tot));
        }
        if (lane == 0) {
            s_excl = excl;
            const uint64_t last = ntiles ? (n / SCAN_TILE < ntiles - 1 ? n / SCAN_TILE : ntiles - 1) : 0;
            if (tile == last) out[n] = excl + tot;
        }
    }
    __syncthreads();
    uint64_t run = s_excl + inc - sum;
    for (uint32_t q = 0; q < w; ++q) run += wsum[q];
    if (VEC && full) {
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 2; ++q) {
            const uint64_t a = run;
            const uint64_t b = run + v[2 * q];
            run = b + v[2 * q + 1];
            reinterpret_cast<uint4*>(out + base)[q] =
                make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
        }
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            if (base + j < n) out[base + j] = run;
            run += v[j];
        }
    }
}

int grid_for(uint64_t n, int threads, int per_sm) {
    uint64_t want = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms() * per_sm;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, cap));
}

struct Tmp {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Tmp(cudaStream_t st) : s(st) {}
    ~Tmp() {
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

hc_status check_ctl(const Ctl* d_ctl, cudaStream_t s, Ctl* h) {
    HC_CUDA_TRY(cudaMemcpyAsync(h, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    HC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->err & DEV_ERR_TIMEOUT) return fail(HC_ERR_TIMEOUT, "a look-back wait in the sort gave up");
    return HC_OK;
}

// CUDA events around selected launches (HC_BUILD_TIME_KERNELS): mark()
// before and after each timed launch; sum() after the stream has synchronised.
struct LaunchTimer {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    ~LaunchTimer() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    hc_status mark(cudaStream_t s) {
        if (!on) return HC_OK;
        cudaEvent_t e;
        HC_CUDA_TRY(cudaEventCreate(&e));
        ev.push_back(e);
        HC_CUDA_TRY(cudaEventRecord(e, s));
        return HC_OK;
    }
    uint32_t launches() const { return (uint32_t)(ev.size() / 2); }
    float sum() const {
        float t = 0.f;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) t += ms;
        }
        return t;
    }
};

// Radix passes over the given digit specs; the sorted keys end in `dst`.
hc_status radix_passes(const void* src, bool src_pairs, uint32_t ao, uint64_t n, const std::vector<DigitSpec>& specs,
                       uint64_t* dst, Tmp& tmp, Ctl* d_ctl, cudaStream_t s, LaunchTimer* timer = nullptr,
                       bool withhold_first = false) {
    const int np = (int)specs.size();
    if (np == 0) return fail(HC_ERR_ARG, "internal: no radix passes");
    DigitSpec* d_specs;
    uint32_t* d_hist;
    HC_TRY(tmp.get(&d_specs, np));
    HC_TRY(tmp.get(&d_hist, (size_t)np * RADIX));
    HC_CUDA_TRY(cudaMemcpyAsync(d_specs, specs.data(), np * sizeof(DigitSpec), cudaMemcpyHostToDevice, s));
    HC_CUDA_TRY(cudaMemsetAsync(d_hist, 0, (size_t)np * RADIX * sizeof(uint32_t), s));
    const int hgrid = grid_for(n, SORT_THREADS * 8, 4);
    if (src_pairs)
        hist_kernel<true><<<hgrid, SORT_THREADS, 0, s>>>(src, n, ao, d_specs, np, d_hist);
    else
        hist_kernel<false><<<hgrid, SORT_THREADS, 0, s>>>(src, n, ao, d_specs, np, d_hist);
    HC_CUDA_TRY(launch_check());
    digit_scan_kernel<<<np, RADIX, 0, s>>>(d_hist);
    HC_CUDA_TRY(launch_check());

    if (n >= 0xFFFFFFFFull) return fail(HC_ERR_CAPACITY, "radix sort: n must be below 2^32 - 1");
    const uint64_t ntiles = (n + PASS_TILE - 1) / PASS_TILE;
    uint64_t* status;
    uint64_t* alt = nullptr;
    HC_TRY(tmp.get(&status, ntiles * RADIX));
    if (np > 1 || !src_pairs) HC_TRY(tmp.get(&alt, n));
    // ping-pong so that the last pass writes `dst`
    uint64_t* bufs[2] = {dst, alt};
    int cur = (np % 2 == 1) ? 0 : 1;  // buffer written by pass 0
    const void* in = src;
    const uint32_t n32 = (uint32_t)n;
    for (int p = 0; p < np; ++p) {
        uint64_t* outb = bufs[cur];
        if (outb == nullptr) return fail(HC_ERR_ARG, "internal: radix buffer");
        const bool from_pairs = p == 0 && src_pairs;
        if (from_pairs && specs[p].mode != 0) return fail(HC_ERR_ARG, "internal: partition digits of raw pairs");
        HC_CUDA_TRY(cudaMemsetAsync(status, 0, ntiles * RADIX * sizeof(uint64_t), s));
        auto* kern = from_pairs              ? onesweep_kernel<SRC_PAIRS, DIGIT_BYTE>
                     : specs[p].mode == 0 ? onesweep_kernel<SRC_KEYS, DIGIT_BYTE>
                                          : onesweep_kernel<SRC_KEYS, DIGIT_PARTITION>;
        if (timer) HC_TRY(timer->mark(s));
        kern<<<(unsigned)ntiles, PASS_THREADS, 0, s>>>(in, outb, n32, ao, specs[p], d_hist + p * RADIX, status,
                                                       &d_ctl->tile_counter[p], &d_ctl->err, wait_limit_ns(),
                                                       (withhold_first && p == 0) ? 1u : 0u);
        HC_CUDA_TRY(launch_check());
        if (timer) HC_TRY(timer->mark(s));
        in = outb;
        cur ^= 1;
    }
    return HC_OK;
}

hc_status run_boundary(const uint64_t* keys, uint64_t n, bool segmented, uint32_t seed_a, uint32_t pa,
                       uint32_t seed_b, uint32_t pb, uint32_t* v1, uint32_t* o1, uint32_t* v2, Tmp& tmp,
                       Ctl* d_ctl, cudaStream_t s, bool withhold = false) {
    const uint64_t ntiles = std::max<uint64_t>(1, (n + SORT_TILE - 1) / SORT_TILE);
    uint64_t* status;
    HC_TRY(tmp.get(&status, ntiles));
    HC_CUDA_TRY(cudaMemsetAsync(status, 0, ntiles * sizeof(uint64_t), s));
    uint32_t* tc = &d_ctl->tile_counter[MAX_PASSES];
    if (segmented)
        boundary_kernel<true><<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(keys, n, seed_a, pa, seed_b, pb, v1, o1, v2,
                                                                         status, tc, d_ctl, wait_limit_ns(),
                                                                         withhold ? 1u : 0u);
    else
        boundary_kernel<false><<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(keys, n, 0, 1, 0, 1, v1, o1, v2, status,
                                                                          tc, d_ctl, wait_limit_ns(),
                                                                          withhold ? 1u : 0u);
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

uint32_t bits_of(uint32_t v) { return v == 0 ? 0 : 32 - __builtin_clz(v); }

}  // namespace

hc_status build_directory(const uint32_t* a, uint64_t alen, const uint32_t* o, uint64_t nruns_max,
                          const uint32_t* d_nruns, const uint32_t* d_err, cudaStream_t s, uint4** out_g) {
    *out_g = nullptr;
    if (alen < DIR_MIN || nruns_max == 0) return HC_OK;  // no run can have a directory
    void* p = nullptr;
    HC_TRY(dev_alloc(&p, alen * sizeof(uint4), s));
    // tiles of the level's positions, a few blocks per SM resident
    const uint64_t want = (alen + DIRB_TILE - 1) / DIRB_TILE;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * 8));
    dir_build_kernel<<<grid, 256, 0, s>>>(a, o, nruns_max, d_nruns, (uint4*)p, d_err);
    if (cudaError_t le = launch_check()) {
        dev_free(p, s);
        return cuda_fail(le, "dir_build_kernel");
    }
    *out_g = (uint4*)p;
    return HC_OK;
}

hc_status build_level_directories(hc_index* idx, cudaStream_t s);

void index_release(hc_index* idx, cudaStream_t s) {
    if (!idx) return;
    dev_free(idx->d_keys, s);
    dev_free(idx->d_v1, s);
    dev_free(idx->d_o1, s);
    dev_free(idx->d_v2, s);
    dev_free(idx->d_v1pos, s);
    dev_free(idx->d_g1, s);
    dev_free(idx->d_g2, s);
    delete idx;
}

hc_status build_index_impl(const uint32_t* d_pairs, uint64_t n, uint32_t ao, uint32_t flags, cudaStream_t s,
                           hc_index** out) {
    if (!out) return fail(HC_ERR_ARG, "build_index: out is NULL");
    *out = nullptr;
    if (ao > 1) return fail(HC_ERR_ARG, "build_index: attr_order must be 0 or 1");
    if (n > 0 && !d_pairs) return fail(HC_ERR_ARG, "build_index: d_pairs is NULL");
    if (n >= 0xFFFFFFFFull) return fail(HC_ERR_CAPACITY, "build_index: n must be below 2^32 - 1");
    hc_index* idx = new hc_index();
    idx->n = n;
    idx->attr_order = ao;
    auto bail = [&](hc_status st) {
        index_release(idx, s);
        return st;
    };
    void* p;
    if (dev_alloc(&p, std::max<uint64_t>(n, 1) * 8, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_keys = (uint64_t*)p;
    if (dev_alloc(&p, (n + LIST_PAD) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_v1 = (uint32_t*)p;
    if (dev_alloc(&p, (n + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_o1 = (uint32_t*)p;
    if (dev_alloc(&p, (n + LIST_PAD) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_v2 = (uint32_t*)p;

    hc_status st;
    LaunchTimer t_radix, t_boundary;
    t_radix.on = t_boundary.on = (flags & HC_BUILD_TIME_KERNELS) != 0;
    {
        Tmp tmp(s);
        Ctl* d_ctl;
        if ((st = tmp.get(&d_ctl, 1)) != HC_OK) return bail(st);
        if (cudaMemsetAsync(d_ctl, 0, sizeof(Ctl), s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "memset"));
        if (n == 0) {
            if (cudaMemsetAsync(idx->d_o1, 0, 4, s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
            *out = idx;
            return HC_OK;
        }
        colmax_kernel<<<grid_for(n, 256, 4), 256, 0, s>>>((const uint2*)d_pairs, n, d_ctl);
        if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "colmax_kernel"));
        Ctl h;
        if ((st = check_ctl(d_ctl, s, &h)) != HC_OK) return bail(st);
        idx->max_first = ao ? h.maxv[1] : h.maxv[0];
        idx->max_second = ao ? h.maxv[0] : h.maxv[1];
        std::vector<DigitSpec> specs;
        for (uint32_t b = 0; b < bits_of(idx->max_second); b += 8) specs.push_back({0, b, 0, 1, 0, 1});
        for (uint32_t b = 0; b < bits_of(idx->max_first); b += 8) specs.push_back({0, 32 + b, 0, 1, 0, 1});
        if (specs.empty()) {
            pack_kernel<<<grid_for(n, 256, 4), 256, 0, s>>>((const uint2*)d_pairs, idx->d_keys, n, ao);
            if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "pack_kernel"));
        } else if ((st = radix_passes(d_pairs, true, ao, n, specs, idx->d_keys, tmp, d_ctl, s, &t_radix,
                                      (flags & HC_BUILD_TEST_STALL_SORT) != 0)) != HC_OK) {
            return bail(st);
        }
        if ((st = t_boundary.mark(s)) != HC_OK) return bail(st);
        if ((st = run_boundary(idx->d_keys, n, false, 0, 1, 0, 1, idx->d_v1, idx->d_o1, idx->d_v2, tmp, d_ctl, s,
                               (flags & HC_BUILD_TEST_STALL_SCAN) != 0)) != HC_OK)
            return bail(st);
        if ((st = t_boundary.mark(s)) != HC_OK) return bail(st);
        maxrun_kernel<<<grid_for(n, 256, 8), 256, 0, s>>>(idx->d_o1, n, d_ctl);
        if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "maxrun_kernel"));
        if ((st = check_ctl(d_ctl, s, &h)) != HC_OK) return bail(st);
        if (t_radix.on) {
            idx->ms_radix = t_radix.sum();
            idx->n_radix = t_radix.launches();
            idx->ms_boundary = t_boundary.sum();
        }
        if ((flags & HC_BUILD_CHECK_DUPLICATES) && h.dup)
            return bail(fail(HC_ERR_DUPLICATE, "build_index: the relation holds a repeated row"));
        idx->l1 = h.l1;
        idx->max_run = h.maxrun;
        if (flags & BUILD_NO_DIRECTORIES) {
            *out = idx;
            return HC_OK;
        }
        if (v1pos_eligible(n, idx->max_first)) {
            const uint64_t dn = (uint64_t)idx->max_first + 1;
            if (dev_alloc(&p, dn * 4, s) != HC_OK) return bail(HC_ERR_OOM);
            idx->d_v1pos = (uint32_t*)p;
            idx->v1pos_n = (uint32_t)dn;
            if (cudaMemsetAsync(idx->d_v1pos, 0xFF, dn * 4, s) != cudaSuccess)
                return bail(cuda_fail(cudaGetLastError(), "memset"));
            v1pos_kernel<<<grid_for(idx->l1, 256, 8), 256, 0, s>>>(idx->d_v1, idx->l1, nullptr, idx->d_v1pos,
                                                                    idx->v1pos_n);
            if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "v1pos_kernel"));
        }
        if ((st = build_level_directories(idx, s)) != HC_OK) return bail(st);
    }
    *out = idx;
    return HC_OK;
}

// Directories of a built index: V2 by the runs of O1, and V1 as one run
// when it has no position map.
hc_status build_level_directories(hc_index* idx, cudaStream_t s) {
    if (idx->max_run >= DIR_MIN)
        HC_TRY(build_directory(idx->d_v2, idx->n, idx->d_o1, idx->l1, nullptr, nullptr, s, &idx->d_g2));
    if (idx->d_v1pos == nullptr && idx->l1 >= DIR_MIN)
        HC_TRY(build_directory(idx->d_v1, idx->l1, nullptr, idx->l1, nullptr, nullptr, s, &idx->d_g1));
    return HC_OK;
}

// Levels of a unary relation whose values are already sorted and distinct:
// keys = value << 32, O1[i] = i (O1[n] = n), V2 = 0.
__global__ void unary_levels_kernel(const uint32_t* __restrict__ values, uint64_t n, uint64_t* __restrict__ keys,
                                    uint32_t* __restrict__ o1, uint32_t* __restrict__ v2) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
        o1[i] = (uint32_t)i;
        if (i < n) {
            keys[i] = (uint64_t)values[i] << 32;
            v2[i] = 0;
        }
    }
}

hc_status build_unary_impl(const uint32_t* d_values, uint64_t n, uint32_t max_value, cudaStream_t s,
                           hc_index** out) {
    if (!out) return fail(HC_ERR_ARG, "build_unary_index: out is NULL");
    *out = nullptr;
    if (n > 0 && !d_values) return fail(HC_ERR_ARG, "build_unary_index: d_values is NULL");
    if (n >= 0xFFFFFFFFull) return fail(HC_ERR_CAPACITY, "build_unary_index: n must be below 2^32 - 1");
    hc_index* idx = new hc_index();
    idx->n = n;
    idx->l1 = n;  // distinct values: one run per row
    idx->max_run = n ? 1 : 0;
    idx->attr_order = 0;
    idx->max_first = n ? max_value : 0;
    idx->max_second = 0;
    auto bail = [&](hc_status st) {
        index_release(idx, s);
        return st;
    };
    void* p;
    if (dev_alloc(&p, std::max<uint64_t>(n, 1) * 8, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_keys = (uint64_t*)p;
    if (dev_alloc(&p, (n + LIST_PAD) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_v1 = (uint32_t*)p;
    if (dev_alloc(&p, (n + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_o1 = (uint32_t*)p;
    if (dev_alloc(&p, (n + LIST_PAD) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    idx->d_v2 = (uint32_t*)p;
    if (n > 0 && cudaMemcpyAsync(idx->d_v1, d_values, n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "copy"));
    unary_levels_kernel<<<grid_for(n + 1, 256, 8), 256, 0, s>>>(d_values, n, idx->d_keys, idx->d_o1, idx->d_v2);
    if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "unary_levels_kernel"));
    if (v1pos_eligible(n, idx->max_first)) {
        const uint64_t dn = (uint64_t)idx->max_first + 1;
        if (dev_alloc(&p, dn * 4, s) != HC_OK) return bail(HC_ERR_OOM);
        idx->d_v1pos = (uint32_t*)p;
        idx->v1pos_n = (uint32_t)dn;
        if (cudaMemsetAsync(idx->d_v1pos, 0xFF, dn * 4, s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "memset"));
        v1pos_kernel<<<grid_for(n, 256, 8), 256, 0, s>>>(d_values, n, nullptr, idx->d_v1pos, idx->v1pos_n);
        if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "v1pos_kernel"));
    }
    hc_status st = build_level_directories(idx, s);
    if (st != HC_OK) return bail(st);
    *out = idx;
    return HC_OK;
}

void partitioned_release(hc_partitioned* p, cudaStream_t s) {
    if (!p) return;
    dev_free(p->d_keys, s);
    dev_free(p->d_bpref, s);
    dev_free(p->d_v1, s);
    dev_free(p->d_o1, s);
    dev_free(p->d_v2, s);
    dev_free(p->d_lvl1_start, s);
    dev_free(p->d_l1, s);
    dev_free(p->d_v1pos, s);
    dev_free(p->d_g1, s);
    dev_free(p->d_g2, s);
    delete p;
}

hc_status partition_impl(const hc_index* idx, uint32_t seed_a, uint32_t pa, uint32_t seed_b, uint32_t pb,
                         cudaStream_t s, hc_partitioned** out) {
    if (!out) return fail(HC_ERR_ARG, "partition: out is NULL");
    *out = nullptr;
    if (!idx) return fail(HC_ERR_ARG, "partition: index is NULL");
    if (idx->stats_only) return fail(HC_ERR_ARG, "partition: a statistics-only index has no data");
    if (pa == 0 || pb == 0 || (uint64_t)pa * pb > 65536ull)
        return fail(HC_ERR_ARG, "partition: shares must be >= 1 with product <= 65536");
    const uint64_t n = idx->n;
    const uint32_t np = pa * pb;
    hc_partitioned* part = new hc_partitioned();
    part->n = n;
    part->n_parts = np;
    part->pa = pa;
    part->pb = pb;
    part->seed_a = seed_a;
    part->seed_b = seed_b;
    part->stream = s;
    auto bail = [&](hc_status st) {
        partitioned_release(part, s);
        return st;
    };
    void* p;
    if (dev_alloc(&p, std::max<uint64_t>(n, 1) * 8, s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_keys = (uint64_t*)p;
    if (dev_alloc(&p, (uint64_t)(np + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_bpref = (uint32_t*)p;
    if (dev_alloc(&p, (n + LIST_PAD) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_v1 = (uint32_t*)p;
    if (dev_alloc(&p, (n + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_o1 = (uint32_t*)p;
    if (dev_alloc(&p, (n + LIST_PAD) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_v2 = (uint32_t*)p;
    if (dev_alloc(&p, (uint64_t)(np + 1) * 4, s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_lvl1_start = (uint32_t*)p;
    if (dev_alloc(&p, sizeof(Ctl), s) != HC_OK) return bail(HC_ERR_OOM);
    part->d_l1 = (uint32_t*)p;  // holds a Ctl; l1 is read from its field
    Ctl* d_ctl = (Ctl*)p;
    if (cudaMemsetAsync(d_ctl, 0, sizeof(Ctl), s) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));

    hc_status st;
    {
        Tmp tmp(s);
        if (n == 0) {
            if (cudaMemsetAsync(part->d_o1, 0, 4, s) != cudaSuccess ||
                cudaMemsetAsync(part->d_bpref, 0, (np + 1) * 4, s) != cudaSuccess ||
                cudaMemsetAsync(part->d_lvl1_start, 0, (np + 1) * 4, s) != cudaSuccess)
                return bail(cuda_fail(cudaGetLastError(), "memset"));
            part->l1_known = true;
            *out = part;
            return HC_OK;
        }
        if (np == 1) {
            if (cudaMemcpyAsync(part->d_keys, idx->d_keys, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return bail(cuda_fail(cudaGetLastError(), "copy"));
        } else {
            std::vector<DigitSpec> specs;
            for (uint32_t b = 0; b < bits_of(np - 1); b += 8) specs.push_back({1, b, seed_a, pa, seed_b, pb});
            if ((st = radix_passes(idx->d_keys, false, 0, n, specs, part->d_keys, tmp, d_ctl, s)) != HC_OK)
                return bail(st);
        }
        if ((st = run_boundary(part->d_keys, n, true, seed_a, pa, seed_b, pb, part->d_v1, part->d_o1, part->d_v2, tmp,
                               d_ctl, s)) != HC_OK)
            return bail(st);
        directory_kernel<<<grid_for(np + 1, 128, 2), 128, 0, s>>>(part->d_keys, n, seed_a, pa, seed_b, pb, part->d_o1,
                                                                  d_ctl, part->d_bpref, part->d_lvl1_start);
        if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "directory_kernel"));
        // partitions on the first attribute alone hold each value once: one
        // position map over the concatenated V1 serves every partition
        if (pb == 1 && v1pos_eligible(n, idx->max_first)) {
            const uint64_t dn = (uint64_t)idx->max_first + 1;
            if (dev_alloc(&p, dn * 4, s) != HC_OK) return bail(HC_ERR_OOM);
            part->d_v1pos = (uint32_t*)p;
            part->v1pos_n = (uint32_t)dn;
            if (cudaMemsetAsync(part->d_v1pos, 0xFF, dn * 4, s) != cudaSuccess)
                return bail(cuda_fail(cudaGetLastError(), "memset"));
            v1pos_kernel<<<grid_for(n, 256, 8), 256, 0, s>>>(part->d_v1, n, &d_ctl->l1, part->d_v1pos,
                                                              part->v1pos_n);
            if (cudaError_t le = launch_check()) return bail(cuda_fail(le, "v1pos_kernel"));
        }
        // bucket directories: V2 by the runs of O1 (l1 runs, a device-side
        // count), V1 by partitions when it has no position map
        if (idx->max_run >= DIR_MIN &&
            (st = build_directory(part->d_v2, n, part->d_o1, n, &d_ctl->l1, &d_ctl->err, s, &part->d_g2)) != HC_OK)
            return bail(st);
        if (part->d_v1pos == nullptr &&
            (st = build_directory(part->d_v1, n, part->d_lvl1_start, np, nullptr, &d_ctl->err, s, &part->d_g1)) != HC_OK)
            return bail(st);
    }
    *out = part;
    return HC_OK;
}

hc_status partitioned_sync(hc_partitioned* p) {
    if (p->l1_known) return HC_OK;
    Ctl h;
    HC_CUDA_TRY(cudaMemcpyAsync(&h, p->d_l1, sizeof(Ctl), cudaMemcpyDeviceToHost, p->stream));
    HC_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (h.err & DEV_ERR_TIMEOUT) return fail(HC_ERR_TIMEOUT, "a look-back wait in partitioning gave up");
    p->l1 = h.l1;
    p->l1_known = true;
    return HC_OK;
}

const uint32_t* partitioned_l1_ptr(const hc_partitioned* p) { return &((const Ctl*)p->d_l1)->l1; }
const uint32_t* partitioned_err_ptr(const hc_partitioned* p) { return &((const Ctl*)p->d_l1)->err; }

template <typename T>
hc_status exclusive_scan_impl(const T* d_in, uint64_t* d_out, uint64_t n_max, const uint32_t* d_n, uint32_t* d_err,
                              cudaStream_t s) {
    Tmp tmp(s);
    const uint64_t ntiles = std::max<uint64_t>(1, (n_max + SCAN_TILE - 1) / SCAN_TILE);
    if (ntiles > 0xFFFFFFFFull) return fail(HC_ERR_CAPACITY, "scan: too many tiles");
    uint64_t* status;
    uint32_t* ctr;
    HC_TRY(tmp.get(&status, ntiles));
    HC_TRY(tmp.get(&ctr, 1));
    HC_CUDA_TRY(cudaMemsetAsync(status, 0, ntiles * sizeof(uint64_t), s));
    HC_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), s));
    if ((((uintptr_t)d_in | (uintptr_t)d_out) & 15u) == 0)
        scan_kernel<T, true><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(d_in, d_out, n_max, d_n, status, ctr, d_err,
                                                                        wait_limit_ns());
    else
        scan_kernel<T, false><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(d_in, d_out, n_max, d_n, status, ctr, d_err,
                                                                         wait_limit_ns());
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}

hc_status exclusive_scan_u32_to_u64(const uint32_t* d_in, uint64_t* d_out, uint64_t n_max, const uint32_t* d_n,
                                    uint32_t* d_err, cudaStream_t s) {
    return exclusive_scan_impl<uint32_t>(d_in, d_out, n_max, d_n, d_err, s);
}
hc_status exclusive_scan_u64(const uint64_t* d_in, uint64_t* d_out, uint64_t n_max, const uint32_t* d_n,
                             uint32_t* d_err, cudaStream_t s) {
    return exclusive_scan_impl<uint64_t>(d_in, d_out, n_max, d_n, d_err, s);
}

}  // namespace hc

namespace hc {
namespace {
__global__ void noalloc_info_kernel(const Ctl* __restrict__ ctl, uint32_t* __restrict__ info) {
    info[0] = ctl->l1;
    info[1] = (ctl->err & DEV_ERR_TIMEOUT ? 1u : 0u) | (ctl->dup ? 2u : 0u);
}
}  // namespace
}  // namespace hc

// ---------------------------------------------------------------------------
// Allocation-free CoCo level build (hc_coco_levels_noalloc).
//
// Some callers cannot let this library allocate device memory: services
// whose device memory is entirely reserved up front by another allocator
// (a library-side cudaMalloc would fail or fragment that reservation), and
// request paths that forbid any allocation so that their latency never
// includes an allocator call.  For them this entry point runs the same
// run-boundary kernel as hc_build_index on keys the caller has already
// sorted, writing only into the caller's buffers.  The kernel's look-back
// scratch lives in the fixed array below, which every GPU that loads this
// library holds until the process exits.
namespace hc {
namespace {

constexpr uint32_t NOALLOC_MAX_TILES = 4096;  // 4096 tiles of 4096 rows
constexpr uint64_t NOALLOC_MAX_ROWS = (uint64_t)NOALLOC_MAX_TILES * SORT_TILE;  // 16,777,216 rows
// NOALLOC_MAX_TILES look-back words, then one control block (8 words).
constexpr uint32_t NOALLOC_WORDS = NOALLOC_MAX_TILES + 8;
static_assert(sizeof(Ctl) <= 8 * sizeof(uint64_t), "control block must fit the scratch tail");

static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];

// Device address of g_noalloc_scratch for each device, looked up once per
// device with that device current.  In host code the array's name is only a
// host-side stand-in, never a device address, so kernels always receive the
// looked-up pointer.
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

hc_status noalloc_scratch(uint64_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) return fail(HC_ERR_CAPACITY, "coco_levels_noalloc: device ordinal above 255");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = (uint64_t*)g_noalloc_addr[dev];
    return HC_OK;
}

}  // namespace
}  // namespace hc

extern "C" hc_status hc_coco_levels_noalloc(const uint64_t* d_sorted_keys, uint64_t n, uint32_t* d_v1,
                                            uint32_t* d_o1, uint32_t* d_v2, uint32_t* d_info, void* stream) {
    using namespace hc;
    if (n > NOALLOC_MAX_ROWS)
        return fail(HC_ERR_CAPACITY, "coco_levels_noalloc: n = " + std::to_string(n) + " rows exceeds the fixed " +
                                         "scratch limit of " + std::to_string(NOALLOC_MAX_ROWS) + " rows");
    if (!d_o1 || !d_info || (n > 0 && (!d_sorted_keys || !d_v1 || !d_v2)))
        return fail(HC_ERR_ARG, "coco_levels_noalloc: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* scratch = nullptr;
    HC_TRY(noalloc_scratch(&scratch));
    Ctl* ctl = (Ctl*)(scratch + NOALLOC_MAX_TILES);
    const uint64_t ntiles = n == 0 ? 0 : (n + SORT_TILE - 1) / SORT_TILE;
    // the scratch keeps the previous call's words: clear the status words
    // this call reads and the control block
    if (ntiles > 0) HC_CUDA_TRY(cudaMemsetAsync(scratch, 0, ntiles * sizeof(uint64_t), s));
    HC_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    if (n == 0) {
        HC_CUDA_TRY(cudaMemsetAsync(d_o1, 0, sizeof(uint32_t), s));
    } else {
        boundary_kernel<false><<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(d_sorted_keys, n, 0, 1, 0, 1, d_v1, d_o1,
                                                                          d_v2, scratch, &ctl->tile_counter[MAX_PASSES],
                                                                          ctl, wait_limit_ns(), 0u);
        HC_CUDA_TRY(launch_check());
    }
    // d_info[0] = l1, d_info[1] = flags: bit 0 a look-back wait gave up,
    // bit 1 two adjacent rows are equal
    noalloc_info_kernel<<<1, 1, 0, s>>>(ctl, d_info);
    HC_CUDA_TRY(launch_check());
    return HC_OK;
}
