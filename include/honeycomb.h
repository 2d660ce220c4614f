/*
 * honeycomb.h -- C ABI of the GB300 (sm_103a) HoneyComb join library.
 *
 * The library evaluates full conjunctive queries of binary atoms (Eq.
 * "full:cq" of Wu & Suciu, "HoneyComb: A Parallel Worst-Case Optimal Join on
 * Multicores") by Generic Join over CoCo indexes, with the variable domains
 * split into HyperCube shares.  Three calls follow the paper's architecture
 * (Sec. 3): hc_build_index (Preprocessor: sort + CoCo, Sec. 4),
 * hc_choose_shares (Optimizer: cost model and plan decision, Sec. 5.2-5.3),
 * hc_run_join (Preprocessor partitioning + Executor, Sec. 4-5).  Relations of
 * arity up to 3 (k-level CoCo, k-ary Generic Join, loop-order choice) are
 * declared in honeycomb_kary.h.
 *
 * Conventions for every entry point:
 *  - Device pointers ("d_" prefix) are CUDA device memory of the current
 *    device; host pointers are ordinary memory.  `stream` is a cudaStream_t
 *    passed as void* (NULL = the legacy default stream).  Work is enqueued on
 *    that stream; where a call must wait for the GPU (to size an allocation or
 *    to return a host value) it says so.
 *  - Relations are sets of uint32 pairs stored as n rows of two uint32 values
 *    (row-major, [n][2]).  Repeated rows are not allowed (Sec. 4 assumes a
 *    unique relation when it drops the last offset array).
 *  - Objects returned through an out-pointer (hc_index, hc_result) are owned
 *    by the library and released with their _free call; inputs stay owned by
 *    the caller and are never freed or modified.
 *  - Every call returns an hc_status; HC_OK is 0.  On failure no output
 *    object is returned and hc_last_error() describes the failure (a
 *    thread-local string).  No call throws or aborts.
 */
#ifndef HONEYCOMB_H
#define HONEYCOMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HC_OK = 0,
    HC_ERR_ARG = 1,        /* an argument violates the contract stated at the call    */
    HC_ERR_OOM = 2,        /* device or host allocation failed                         */
    HC_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed              */
    HC_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up (result is invalid)   */
    HC_ERR_CAPACITY = 5,   /* a size exceeds a fixed limit of the library              */
    HC_ERR_DUPLICATE = 6,  /* the relation holds a repeated row (checking mode only)   */
    HC_ERR_BUSY = 7        /* a serving queue or admission budget is full              */
} hc_status;

#define HC_MAX_VARS 8
#define HC_MAX_ATOMS 12

/* One atom R_j(X_var0, X_var1): column 0 of its relation holds the values
 * of variable var0, column 1 those of var1 (var0 != var1).  With var1 =
 * HC_UNARY the atom is unary, R_j(X_var0): the set of column-0 values of its
 * relation (an index with attr_order 0; column 1 is ignored).  Unary atoms
 * express a selection pushed into the query (Sec. 2), e.g. restricting a
 * variable to a vertex subset. */
#define HC_UNARY 0xFFu
typedef struct {
    uint8_t var0;
    uint8_t var1;
} hc_atom;

/* A full conjunctive query Q(X_0..X_{n_vars-1}) <- R_0(..) ^ ... (Eq.
 * "full:cq").  Every variable must occur in some atom.  order[i] is the
 * variable bound by loop i of Generic Join (Sec. 2); it must list each
 * variable once.  Predicates are pushed into the atoms by the caller, as
 * selections on their relations (Sec. 2). */
typedef struct {
    uint32_t n_vars;
    uint32_t n_atoms;
    hc_atom atoms[HC_MAX_ATOMS];
    uint8_t order[HC_MAX_VARS];
} hc_query;

typedef struct hc_index hc_index;
typedef struct hc_result hc_result;

/* ------------------------------------------------------------ build_index
 * CoCo index of one binary relation (Sec. 4, "Construction of CoCo"):
 * the rows sorted lexicographically in attribute order `attr_order` (0: by
 * column 0 then column 1; 1: by column 1 then column 0) by an LSD radix sort,
 * then one run-boundary scan producing
 *    V1[l1]   distinct first-attribute values, ascending          (uint32)
 *    O1[l1+1] start of each value's run in V2, O1[l1] = n          (uint32)
 *    V2[n]    second-attribute values, in sorted row order         (uint32)
 * (the last level's offsets are dropped because the relation is a set).
 *   d_pairs  device, [n][2] uint32, caller-owned, read only.
 *   n        number of rows; 0 < n < 2^32 - 1 (HC_ERR_CAPACITY above).
 *   out      receives the library-owned index (free with hc_index_free).
 * Waits for the GPU once (to read the column maxima that size the sort).
 * The rows must be distinct; with HC_BUILD_CHECK_DUPLICATES in `flags` a
 * repeated row returns HC_ERR_DUPLICATE instead of an index.  With
 * HC_BUILD_TIME_KERNELS the radix passes and the run-boundary scan are timed
 * with CUDA events on `stream` (see hc_index_view).
 * A bounded device-side wait (a look-back of the sort or of the scan) that
 * runs past hc_wait_limit_ns() returns HC_ERR_TIMEOUT and no index; the
 * kernels after it do nothing, so no device memory outside the call's own
 * buffers is touched and the context stays usable.  Two flags exist for
 * testing that path only: with HC_BUILD_TEST_STALL_SORT the first tile of
 * the first radix pass never publishes its look-back status (a relation
 * whose values need no radix pass is not affected), with
 * HC_BUILD_TEST_STALL_SCAN the first tile of the run-boundary scan never
 * does; the tiles after it wait for it until the limit and the call returns
 * HC_ERR_TIMEOUT (the relation must span more than one tile: 6,144 rows
 * for the sort, 4,096 for the scan). */
#define HC_BUILD_CHECK_DUPLICATES 1u
#define HC_BUILD_TIME_KERNELS 2u
#define HC_BUILD_TEST_STALL_SORT 0x100u
#define HC_BUILD_TEST_STALL_SCAN 0x200u
hc_status hc_build_index(const uint32_t* d_pairs, uint64_t n, uint32_t attr_order, uint32_t flags,
                         void* stream, hc_index** out);
hc_status hc_index_free(hc_index* index);

/* Index of a unary relation given as its values, strictly ascending, on the
 * device (d_values[n], caller-owned, read only): the index of the pairs
 * (value, 0) in attribute order 0 that hc_build_index would build, made
 * without sorting and without waiting for the GPU.  V1 = the values, O1[i]
 * = i (O1[n] = n), V2 = 0.  max_value must equal the largest value
 * (d_values[n-1]); it sizes the V1 position map and the optimizer's domain
 * estimate.  The order is not checked: unsorted or repeated values give
 * wrong join results.  Used for the selections a serving request pushes into
 * its query as unary atoms (Sec. 2).  0 <= n < 2^32 - 1. */
hc_status hc_build_unary_index(const uint32_t* d_values, uint64_t n, uint32_t max_value, void* stream,
                               hc_index** out);

/* Read-only view of an index's device arrays (valid until hc_index_free). */
typedef struct {
    uint64_t n;             /* rows                                            */
    uint64_t l1;            /* distinct first-attribute values                 */
    uint32_t attr_order;
    uint32_t max_first;     /* largest first-attribute value (0 if n == 0)     */
    uint32_t max_second;
    const uint32_t* d_v1;   /* [l1]                                            */
    const uint32_t* d_o1;   /* [l1+1]                                          */
    const uint32_t* d_v2;   /* [n]                                             */
    const uint64_t* d_keys; /* [n] sorted rows as (first << 32 | second)       */
    /* filled when built with HC_BUILD_TIME_KERNELS, else 0:                 */
    float ms_radix_passes;    /* device time of the radix-pass launches, summed  */
    uint32_t n_radix_passes;  /* radix-pass launches                             */
    float ms_boundary;        /* device time of the run-boundary scan            */
    uint64_t max_run;         /* rows of the most frequent first-attribute value */
    uint32_t v1pos_n;         /* entries of the V1 position map (0: none; a map  */
                              /* is built when the first attribute's values are  */
                              /* dense: max_first + 1 <= 4 n + 2^20, max_first < */
                              /* 0xFFFFFFFF), else V1 is searched                 */
} hc_index_view;
hc_status hc_index_get_view(const hc_index* index, hc_index_view* out);

/* A statistics-only index: no device arrays, only the sizes the optimizer
 * reads (n rows, l1 distinct first-attribute values, attribute order and the
 * largest first / second values) and, when known, max_run, the rows of the
 * most frequent first-attribute value (0 = unknown; else 1 <= max_run <=
 * n - l1 + 1).  Host only, needs no GPU.  Accepted by hc_choose_shares and
 * hc_join_footprint (which applies hc_run_join's list-length limit when
 * max_run is known); hc_run_join and hc_partition_index reject it with
 * HC_ERR_ARG.  Free with hc_index_free.  Requires l1 <= n and l1 >= 1 when
 * n >= 1. */
hc_status hc_index_from_stats(uint64_t n, uint64_t l1, uint32_t attr_order, uint32_t max_first,
                              uint32_t max_second, uint64_t max_run, hc_index** out);

/* --------------------------------------------------- coco_levels_noalloc
 * The CoCo levels V1, O1, V2 (as hc_build_index writes them) of rows that
 * the caller has already sorted, computed without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library allocate device memory -- services whose device
 * memory is all reserved up front by another allocator, and request paths
 * that must not call an allocator at all.
 *   d_sorted_keys  device, [n] rows as (first << 32 | second), ascending.
 *   n              rows; at most 16,777,216 (2^24), else HC_ERR_CAPACITY
 *                  before any device work.
 *   d_v1 [n], d_o1 [n + 1], d_v2 [n]   device outputs, caller-owned.
 *   d_info [2]     device output: d_info[0] = l1 (the number of V1
 *                  entries), d_info[1] = flags: bit 0 set when a bounded
 *                  look-back wait gave up (the outputs are then invalid),
 *                  bit 1 set when two adjacent rows are equal (not a set).
 * Enqueued on `stream` without waiting.  Calls no cudaMalloc, cudaFree or
 * other allocating routine; the kernel's scratch is one fixed array of
 * 32,832 bytes inside the library, held by every GPU that loads it until the
 * process exits.  The first call on a device looks up that array's device
 * address (once per device), so make it before any stream capture; the
 * address is kept for the life of the process, so calls must not cross a
 * cudaDeviceReset of that device.  All calls share the array and each call
 * clears what it reads: calls whose work overlaps on the GPU (other streams,
 * other host threads) race. */
hc_status hc_coco_levels_noalloc(const uint64_t* d_sorted_keys, uint64_t n, uint32_t* d_v1, uint32_t* d_o1,
                                 uint32_t* d_v2, uint32_t* d_info, void* stream);

/* ------------------------------------------------------- partition_index
 * HyperCube partitioning of one indexed relation (Sec. 4, partitioning
 * paragraphs and Example "partition"): a row (a, b) in the index's attribute
 * order has partition identifiers s_a = share(a; seed_a, pa) and
 * s_b = share(b; seed_b, pb), share(x; seed, P) = (fmix32(x ^ seed) * P) >> 32,
 * and partition id pid = s_a * pb + s_b (lexicographic order, as B^pref).
 * The result R~ holds every row exactly once (no replication), partitions
 * concatenated in pid order, each sorted by (a, b) (a stable scatter of the
 * sorted index), and one CoCo per partition:
 *    keys[n]        R~ as (a << 32 | b)                                 (uint64)
 *    bpref[np+1]    B^pref: start of partition p in R~; bpref[np] = n   (uint32)
 *    v1[l1], o1[l1+1], v2[n]  per-partition CoCo levels concatenated;
 *                   o1 entries are row positions in R~ (o1[l1] = n)    (uint32)
 *    lvl1_start[np+1]  first level-1 entry of partition p in v1        (uint32)
 * with np = pa * pb, 1 <= np <= 2^16.  Enqueued on `stream` without waiting.
 * The partitioned relation is library-owned (hc_partitioned_free). */
typedef struct hc_partitioned hc_partitioned;
hc_status hc_partition_index(const hc_index* index, uint32_t seed_a, uint32_t pa, uint32_t seed_b,
                             uint32_t pb, void* stream, hc_partitioned** out);
typedef struct {
    uint64_t n, l1, n_parts;
    uint32_t pa, pb;
    const uint64_t* d_keys;
    const uint32_t* d_bpref;
    const uint32_t* d_v1;
    const uint32_t* d_o1;
    const uint32_t* d_v2;
    const uint32_t* d_lvl1_start;
} hc_partitioned_view;
/* Waits for the partitioning's stream (l1 is read back), then fills `out`. */
hc_status hc_partitioned_get_view(hc_partitioned* p, hc_partitioned_view* out);
hc_status hc_partitioned_free(hc_partitioned* p);

/* ---------------------------------------------------------- choose_shares
 * Shares P_i for each variable (Sec. 5.2 cost model, Lemma "cost-ub" and
 * Eq. "total:cost"; Sec. 5.3 plan decision): among power-of-two share
 * vectors with product P, drop those whose replicated cost exceeds twice the
 * unpartitioned cost or that give some variable more shares than its domain
 * supports (|Dom(X_i)| < 3 P_i ln P_i), then take the one of least evenness
 * E = sum_i P_sigma(i) w(i), w(i) = max(1 - i/100, 3/4); ties go to the
 * lexicographically smallest vector.  Host only; reads only the indexes'
 * sizes.  idx[j] is the index bound to atom j.  P must be a power of two,
 * 1 <= P <= 2^16.  shares_out[v] for v < n_vars, 1 elsewhere. */
hc_status hc_choose_shares(const hc_query* q, const hc_index* const* idx, uint32_t P,
                           uint32_t shares_out[HC_MAX_VARS]);

/* Variable order and shares together (Sec. 5.3, "Plan Decision"): for every
 * order sigma of the query's variables (n_vars! of them; q->order is ignored)
 * the shares are chosen as by hc_choose_shares under that order, and the
 * order kept is the one whose replicated cost (Eq. "total:cost") at those
 * shares is least; ties go to the smaller unpartitioned cost, then to the
 * lexicographically smallest order.  Statistics are read from the indexes as
 * by hc_choose_shares and do not depend on their attribute order (a
 * statistics-only index serves).  order_out[0..n_vars) receives the loop
 * order (variable ids); a run with it needs, for atom j, an index whose
 * attr_order puts the atom's variables in that order.  shares_out as in
 * hc_choose_shares.  Host only; HC_ERR_ARG as hc_choose_shares, and for
 * n_vars > 8. */
hc_status hc_choose_plan(const hc_query* q, const hc_index* const* idx, uint32_t P, uint8_t order_out[HC_MAX_VARS],
                         uint32_t shares_out[HC_MAX_VARS]);

/* Estimated cost of a plan (Sec. 5.2): level_cost[i] is the bound of Lemma
 * "cost-ub" for loop i with all shares 1, and *replicated_cost is Eq.
 * "total:cost" for the given shares (per variable id).  dom_out[v] is the
 * domain size estimate of variable v used by the domain rule.  Host only;
 * the same estimates drive hc_choose_shares. */
hc_status hc_plan_cost(const hc_query* q, const hc_index* const* idx, const uint32_t shares[HC_MAX_VARS],
                       double level_cost[HC_MAX_VARS], double dom_out[HC_MAX_VARS], double* replicated_cost);

/* ------------------------------------------------------------- run_join */
#define HC_MODE_COUNT 0u
#define HC_MODE_MATERIALIZE 1u

#define HC_FLAG_CELL_COUNTS 1u /* also return the count of each HyperCube cell        */
#define HC_FLAG_STATS 2u       /* also return the intersection work counter           */
#define HC_FLAG_TIME_KERNELS 4u /* time the search kernel launches with device events  */
/* Per-cell profile (the skew study of Sec. 1, Examples 1-3, where each
 * HyperCube cell is a thread of work): for every cell, its work units (the
 * HC_FLAG_STATS counter restricted to the cell's bindings) and the SM clock
 * cycles the warps spent on its work items (clock64 spans, summed; the
 * analogue of a thread's time).  Implies HC_FLAG_STATS (so no query
 * rewriting); the first search pass records it. */
#define HC_FLAG_CELL_PROFILE 16u
/* Query rewriting (Sec. 5.1) is on by default for queries of 4+ variables
 * whose last loop has two or more lists fixed before the loop above it (the
 * 4-clique's R3[y] and R6[x] under order X,Y,Z,U): their intersection is
 * computed once per binding of loop n-3 (e.g. per y) and the last loop
 * intersects it with the remaining lists.  It needs lift_arena words of
 * device scratch per resident warp, and is off with HC_FLAG_STATS (the work
 * counter measures the unrewritten loops) or with: */
#define HC_FLAG_NO_LIFT 8u

typedef struct {
    uint32_t shares[HC_MAX_VARS]; /* P_v per variable id (>= 1); their product = cells  */
    uint32_t seeds[HC_MAX_VARS];  /* hash seed per variable id                          */
    uint32_t mode;                /* HC_MODE_COUNT or HC_MODE_MATERIALIZE               */
    uint32_t flags;               /* HC_FLAG_*                                          */
    uint32_t item_grain;          /* loop-2 candidates per work item (0: default)       */
    uint32_t block_threads;       /* threads per block of the search kernel, a multiple */
                                  /* of 32 up to 128 (0: default 128)                   */
    uint32_t merge_min;           /* last loop: two lists both at least this long ...   */
    uint32_t merge_ratio;         /* ... and within this length ratio are intersected    */
                                  /* by a warp block merge, others by binary search      */
                                  /* (0: defaults 32 and 4; 0xFFFFFFFF: never merge)     */
    uint32_t slice_grain;         /* 4+ loops: loop-3 candidates per work slice of a     */
                                  /* loop-2 binding (0: default 256; 0xFFFFFFFF: none)   */
    uint32_t lift_arena;          /* query rewriting: words of device scratch per warp   */
                                  /* for lifted intersections (0: default 16384; at most  */
                                  /* 2^26)                                                 */
    uint64_t out_capacity;        /* materialize: 0 runs a counting pass, then an        */
                                  /* emitting pass (tuples cell-major, in a fixed order); */
                                  /* > 0 runs one pass writing into an output pool of    */
                                  /* about this many tuples (order not fixed), and falls */
                                  /* back to the emitting pass if the pool overflows     */
    uint32_t dir_min;             /* a list search in a sorted run of at least this     */
                                  /* many values reads the run's bucket directory first */
                                  /* (Sec. 5 search; built with every index for runs of */
                                  /* 16 or more): 0 = 16; 0xFFFFFFFF = plain binary     */
                                  /* search everywhere                                   */
    uint32_t pair_min;            /* last loop of two lists, not merged: a binding whose */
                                  /* shorter list has at least this many values is      */
                                  /* searched by the whole warp, its values 32 at a time */
                                  /* (0: default 32; 0xFFFFFFFF: never, all bindings'    */
                                  /* values are spread over the lanes together)          */
} hc_join_params;

/* Generic Join of q over the indexes, one logical worker per HyperCube cell
 * (Sec. 5, Listing C of Fig. "algo-comp").  Limit: the search counts a
 * batch's candidates (up to 32 bindings' shortest lists) in 32 bits, so at
 * every loop after the first the shortest list must stay below 2^27 values;
 * the call returns HC_ERR_CAPACITY before any device work when the indexes
 * allow a longer one (a sub-list's bound is its index's max_run, a
 * top-level list's its l1).  R-MAT 23, 258 M rows, has at most about 10^6
 * rows per key.
 *   idx[j]   index bound to atom j; its attr_order must sort the atom's
 *            variables in loop order (Sec. 4: T(Z,X) under order X,Y,Z is
 *            sorted by X first), else HC_ERR_ARG.
 *   params   shares and hash seeds per variable; a variable value x goes to
 *            share s = (fmix32(x ^ seed) * P) >> 32 (MurmurHash3 finaliser).
 *            Atoms whose two variables both have one share are read in place;
 *            the others are partitioned per call (Sec. 4).
 *   out      library-owned result (hc_result_free).
 * Count mode enqueues everything and returns without waiting; the count is
 * read with hc_result_get (which waits).  Materialize mode waits for the
 * device to size its output (see out_capacity).  Output tuples hold n_vars
 * uint32 values in variable-id order; the result is a set (no repeats)
 * whatever the shares. */
hc_status hc_run_join(const hc_query* q, const hc_index* const* idx, const hc_join_params* params,
                      void* stream, hc_result** out);

/* Generic Join as hc_run_join in materialize mode, with the tuples delivered
 * to host memory (Sec. 6 measures a join end to end, from the relations to
 * all output tuples).  The search runs as up to 16 launches over consecutive
 * ranges of its work items; after each launch its part of the output pool is
 * compacted on the device and copied to h_tuples on a second stream while
 * the next launch runs, so the transfer overlaps the search.
 *   h_tuples   host, [capacity][n_vars] uint32, caller-owned; receives the
 *              tuples (variable-id order, order of rows not fixed).  Page-
 *              locked memory (cudaHostAlloc / cudaHostRegister) lets the
 *              copies overlap the search; pageable memory works, slower.
 *   capacity   rows h_tuples holds.
 *   count_out  receives |Q|.
 * params->mode and params->out_capacity are ignored (the device pool is sized
 * from capacity).  Waits for the stream before returning; h_tuples is
 * complete then.  If |Q| > capacity the call returns HC_ERR_CAPACITY with
 * *count_out = |Q| (the rows written are then incomplete): call again with a
 * buffer that large.  Other errors as hc_run_join. */
hc_status hc_run_join_to_host(const hc_query* q, const hc_index* const* idx, const hc_join_params* params,
                              uint32_t* h_tuples, uint64_t capacity, uint64_t* count_out, void* stream);

/* Device memory a count-mode hc_run_join with these arguments may allocate
 * at most (bytes), for admission control; host only, enqueues nothing.  The
 * arguments are checked as hc_run_join checks them. */
hc_status hc_join_footprint(const hc_query* q, const hc_index* const* idx, const hc_join_params* params,
                            uint64_t* bytes_out);

typedef struct {
    uint64_t count;             /* |Q|                                                */
    uint64_t n_tuples;          /* tuples in d_tuples (materialize), else 0           */
    const uint32_t* d_tuples;   /* [n_tuples][n_vars], library-owned, or NULL         */
    uint64_t n_cells;           /* product of the shares                              */
    const uint64_t* d_cell_counts; /* [n_cells] with HC_FLAG_CELL_COUNTS, else NULL   */
    uint64_t work;              /* with HC_FLAG_STATS: sum over loops and bindings of  */
                                /* (number of lists) * (shortest list length), else 0 */
    uint64_t n_items;           /* work items of the join kernel                      */
    float ms_join_kernel;       /* with HC_FLAG_TIME_KERNELS: device time of the search */
                                /* kernel launches (CUDA events on the join's stream)  */
    uint32_t n_join_launches;   /* search kernel launches of this join (1 or 2)         */
    const uint64_t* d_cell_profile; /* [n_cells][2] (work units, SM cycles) with           */
                                /* HC_FLAG_CELL_PROFILE, else NULL                      */
} hc_result_view;
/* Waits for the result's stream, then fills `out`. */
hc_status hc_result_get(hc_result* r, hc_result_view* out);
hc_status hc_result_free(hc_result* r);

/* ---------------------------------------------------------------- batches
 * Many count-mode joins in one persistent search launch (the paper's
 * scheduler runs its P logical workers by work stealing, Sec. 3
 * "Allocator"; here the work items of all queries form one space handed out
 * by one atomic counter, so warps move on to whichever query still has work).
 *   qs[n], prm[n]  the queries and their parameters (mode must be COUNT);
 *   idx_flat       the indexes of query 0's atoms, then query 1's, ...;
 *   n              1..65536 queries of 3 or 4 variables, in any mix of the
 *                  four built-in shapes (3 or 4 loops, with up to 2 or up to
 *                  4 lists and opened atoms per loop); a batch of three or
 *                  four shapes runs them in one launch that switches per
 *                  query (at the occupancy of the widest shape).
 * hc_batch_create plans every query, partitions atoms whose shares need it
 * and allocates the batch's device memory (waits for the GPU once).
 * hc_batch_launch enqueues the loop-1 passes of all queries and the one
 * search launch, without waiting.  hc_batch_capture records that work once
 * as a CUDA graph on `stream` (a created, non-default stream); later
 * hc_batch_launch calls replay the graph.  hc_batch_counts waits for the
 * last launch and writes counts[n].  The indexes must outlive the batch. */
typedef struct hc_batch hc_batch;
hc_status hc_batch_create(const hc_query* qs, const hc_index* const* idx_flat, const hc_join_params* prm, uint32_t n,
                          void* stream, hc_batch** out);
hc_status hc_batch_launch(hc_batch* b, void* stream);
hc_status hc_batch_capture(hc_batch* b, void* stream);
hc_status hc_batch_counts(hc_batch* b, uint64_t* counts);
hc_status hc_batch_free(hc_batch* b);

/* -------------------------------------------------------------- utilities */
const char* hc_status_str(hc_status s);
const char* hc_last_error(void);
/* Limit, in nanoseconds, of every bounded device-side wait (the decoupled
 * look-backs of the sort, the scans and the level builds) in kernels
 * launched after the call; process-wide, default 2,000,000,000 (2 s).  A wait
 * that runs past it makes its call return HC_ERR_TIMEOUT.  0 gives up at the
 * first status word that is not ready, which can fail a healthy build. */
hc_status hc_set_wait_limit_ns(uint64_t ns);
uint64_t hc_wait_limit_ns(void);
/* Library version and the compute capability it was built for (e.g. 103). */
uint32_t hc_version(void);
/* Kernels this library has launched in this process so far (host counter). */
uint64_t hc_kernel_launches(void);
uint32_t hc_target_sm(void);

#ifdef __cplusplus
}
#endif
#endif /* HONEYCOMB_H */
