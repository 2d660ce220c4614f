/*
 * honeycomb_kary.h -- relations of arity 1 to 3: the k-level CoCo index
 * (Sec. 4, "CoCo": one level (V_r, O_r) per attribute) and Generic Join over
 * it (Sec. 5), for hypergraph queries such as the paper's Loomis-Whitney
 * query LW and Clover-Triangle query CT (Table "Queries").
 *
 * The conventions of honeycomb.h hold: device pointers carry a "d_" prefix,
 * `stream` is a cudaStream_t passed as void*, library-owned objects are
 * released with their _free call, every call returns an hc_status and sets
 * hc_last_error() on failure.  Results are hc_result objects, read with
 * hc_result_get and released with hc_result_free.
 */
#ifndef HONEYCOMB_KARY_H
#define HONEYCOMB_KARY_H
#include "honeycomb.h"
#ifdef __cplusplus
extern "C" {
#endif

#define HC_KMAX_ARITY 3
#define HC_KMAX_VARS 6 /* variables of a k-ary query */

typedef struct hc_kindex hc_kindex;

/* ------------------------------------------------------------ build_kindex
 * k-level CoCo of one relation of arity k = 1..3 (Sec. 4): the rows are
 * sorted lexicographically with column level_cols[0] first, then
 * level_cols[1], ..., and for each level d
 *    V_d[l_d]      the value of level d of each distinct prefix of length
 *                  d+1, in sorted order                            (uint32)
 *    O_d[l_d + 1]  for d < k-1: start of each prefix's children in level
 *                  d+1, O_d[l_d] = l_{d+1}                          (uint32)
 * with l_{k-1} = n (the last level's offsets are dropped: a set).
 *   d_rows      device, [n][k] uint32 row-major, caller-owned, read only.
 *   n           rows, 0 <= n < 2^32 - 1 (HC_ERR_CAPACITY above).
 *   arity       k, 1..3.
 *   level_cols  host, [k]: the column stored at each level, a permutation
 *               of 0..k-1 (NULL: 0, 1, ..).
 *   flags       HC_BUILD_CHECK_DUPLICATES: a repeated row returns
 *               HC_ERR_DUPLICATE instead of an index; HC_BUILD_TIME_KERNELS:
 *               the sort and the level scan are timed (hc_kindex_view).
 * The rows are sorted as one 64-bit key per row when the levels' value bits
 * add up to at most 64 (packed), else one level at a time (stable by
 * position).  Waits for the GPU (column maxima, level sizes).  Rows must be
 * distinct; without the check flag repeated rows give wrong join results. */
hc_status hc_build_kindex(const uint32_t* d_rows, uint64_t n, uint32_t arity, const uint8_t* level_cols,
                          uint32_t flags, void* stream, hc_kindex** out);

/* ------------------------------------------------ build_kindex_partitioned
 * The same index for a relation partitioned for HyperCube shares (Sec. 4,
 * "Preprocessor", Example "partition"): column c of a row has the partition
 * identifier s_c = h_c(x_c) = (fmix32(x_c ^ seeds[c]) * shares[c]) >> 32
 * (fmix32: the MurmurHash3 32-bit finaliser), and the row's partition is
 *    p = (..(s_0 * shares[1] + s_1) * shares[2] + s_2..)
 * (column 0 most significant: partitions in the lexicographic order of their
 * identifiers).  The partitions are concatenated in order of p (R~), each
 * with its own k-level CoCo: V_d and O_d are the partitions' levels
 * concatenated, O_d pointing into the concatenated level d+1, and the view
 * gives each partition's first row (B^pref) and first level-0 entry.
 *   seeds, shares  host, [arity]: per column; shares[c] >= 1 with product
 *                  at most 65536 (HC_ERR_ARG otherwise, and when either is
 *                  NULL).  A product of 1 builds the unpartitioned index.
 * Other arguments and errors as hc_build_kindex.  A partitioned index keeps
 * a level-0 position map only when the deeper levels' columns have share 1
 * (each level-0 value then sits in one partition).  Waits for the GPU. */
hc_status hc_build_kindex_partitioned(const uint32_t* d_rows, uint64_t n, uint32_t arity, const uint8_t* level_cols,
                                      const uint32_t* seeds, const uint32_t* shares, uint32_t flags, void* stream,
                                      hc_kindex** out);
hc_status hc_kindex_free(hc_kindex* index);

typedef struct {
    uint64_t n;                   /* rows                                             */
    uint32_t arity;               /* k                                                */
    uint8_t level_cols[HC_KMAX_ARITY]; /* column of each level (unused entries 0)      */
    uint8_t packed;               /* 1: sorted as packed 64-bit keys                  */
    uint64_t len[HC_KMAX_ARITY];  /* l_d (0 for d >= k)                               */
    uint32_t max_value[HC_KMAX_ARITY]; /* largest value of level d                    */
    const uint32_t* d_v[HC_KMAX_ARITY]; /* V_d [l_d]                                  */
    const uint32_t* d_o[HC_KMAX_ARITY]; /* O_d [l_d + 1] for d < k-1, else NULL       */
    /* filled when built with HC_BUILD_TIME_KERNELS, else 0:                         */
    float ms_sort;                /* device time of the sort stage                    */
    float ms_levels;              /* device time of the level scan                    */
    uint32_t n_parts;             /* partitions (1: unpartitioned)                    */
    uint32_t shares[HC_KMAX_ARITY]; /* per column (1 when unpartitioned)              */
    uint32_t seeds[HC_KMAX_ARITY];  /* per column (0 when unpartitioned)              */
    /* n_parts > 1, else NULL; device, [n_parts + 1], entry n_parts closes the last: */
    const uint32_t* d_bpref;        /* B^pref: first row of each partition in R~ (n)  */
    const uint32_t* d_level0_start; /* first level-0 entry of each partition (l_0)    */
} hc_kindex_view;
hc_status hc_kindex_get_view(const hc_kindex* index, hc_kindex_view* out);

/* A statistics-only k-level index for planning: no device arrays, only the
 * sizes the optimizer reads (n rows, l_d per level with l_{k-1} = n, the
 * largest value of each level, the level order).  Host only, needs no GPU;
 * hc_run_kjoin rejects it with HC_ERR_ARG.  Requires 1 <= l_0 <= .. <= n
 * when n >= 1.  Free with hc_kindex_free. */
hc_status hc_kindex_from_stats(uint64_t n, uint32_t arity, const uint8_t* level_cols, const uint64_t* len,
                               const uint32_t* max_value, hc_kindex** out);

/* ---------------------------------------------------------------- run_kjoin
 * One atom R_j(X_var[0], .., X_var[arity-1]): column c of its relation
 * holds the values of variable var[c]; the variables of an atom are
 * distinct. */
typedef struct {
    uint8_t arity;
    uint8_t var[HC_KMAX_ARITY];
} hc_katom;

/* A full conjunctive query over atoms of arity 1..3 (Eq. "full:cq");
 * order[i] is the variable bound by loop i of Generic Join (Sec. 2). */
typedef struct {
    uint32_t n_vars;  /* 1..HC_KMAX_VARS */
    uint32_t n_atoms; /* 1..HC_MAX_ATOMS */
    hc_katom atoms[HC_MAX_ATOMS];
    uint8_t order[HC_MAX_VARS];
} hc_kquery;

typedef struct {
    uint32_t mode;          /* HC_MODE_COUNT or HC_MODE_MATERIALIZE                    */
    uint32_t flags;         /* HC_FLAG_STATS, HC_FLAG_TIME_KERNELS, HC_FLAG_CELL_COUNTS */
    uint32_t item_grain;    /* loop-1 candidates per work item (0: sized from the run)  */
    uint32_t block_threads; /* threads per block of the search kernel: 32, 64, 96 or   */
                            /* 128 (0: 128)                                             */
    uint32_t pair_min;      /* last loop: a binding with at least this many candidates  */
                            /* is searched by the whole warp, 128 candidates at a time  */
                            /* (0: 32; 0xFFFFFFFF: never)                               */
} hc_kjoin_params;

/* Generic Join of q over k-level indexes (Sec. 5) in every HyperCube cell
 * (Sec. 4-5).  The shares come from the indexes: an index built with
 * hc_build_kindex_partitioned partitions each variable of its atom, and
 * every atom holding a variable must partition it with the same share and
 * seed (share 1 everywhere for an unpartitioned variable; HC_ERR_ARG
 * otherwise).  Cells are numbered by the mixed radix of the variables'
 * coordinates, variable 0 most significant (at most 2^20 cells,
 * HC_ERR_CAPACITY), and cell (c_0, ..) intersects, in each atom, the
 * partition its variables' coordinates select; the cells' results are
 * disjoint and their union is Q.  Loop 0 runs as a flat pass over the
 * loop-0 candidates of all cells (in each cell, the shortest of its
 * lists); later loops run in a persistent kernel whose warps take work
 * items (ranges of loop-1 candidates) from an atomic counter and walk the
 * rest of the loops depth first, 32 candidates at a time, each searched in
 * the loop's other lists.
 *   idx[j]   index bound to atom j, of the atom's arity; its levels must
 *            hold the atom's variables in loop order (level d's variable is
 *            bound before level d+1's), else HC_ERR_ARG.
 *   Limits: at most 4 atoms hold any one variable, n_vars <= HC_KMAX_VARS,
 *   fewer than 2^32 - 1 loop-0 candidates over all cells (HC_ERR_CAPACITY).
 * Count mode enqueues everything and returns without waiting.
 * Materialize mode counts first, waits, then writes the tuples (n_vars
 * uint32 values in variable-id order, in no fixed order).  With
 * HC_FLAG_STATS the view's `work` is the sum over loops and bindings of
 * (number of lists) * (shortest list length), summed over the cells; with
 * HC_FLAG_CELL_COUNTS the view's d_cell_counts[n_cells] holds the count of
 * each cell.  n_items is 0. */
hc_status hc_run_kjoin(const hc_kquery* q, const hc_kindex* const* idx, const hc_kjoin_params* params,
                       void* stream, hc_result** out);

/* --------------------------------------------------------------- planning
 * Estimated cost of a k-ary query's loop order (Sec. 5.2, Lemma "cost-ub",
 * one cell): level_cost[i] for loop i of q->order, with a binding's list in
 * an atom estimated as D(bound columns + the loop's column) / D(bound
 * columns), D the number of distinct combinations of a column set (exact for
 * the prefixes of the index's level order and for all columns, else the
 * product of single-column counts bounded by the rows), and a k-way
 * intersection over a domain of dom values keeping prod(lengths) /
 * dom^(k-1), at most the shortest.  dom_out[v]: the domain estimate of
 * variable v (the least single-column count among its atoms).  For binary
 * atoms these are hc_plan_cost's level costs without query rewriting.  Host
 * only; statistics-only indexes serve; the indexes' level orders need not
 * match q->order.  The level sizes of a partitioned index count a prefix
 * once per partition that holds it, so estimates are best taken from the
 * unpartitioned indexes. */
hc_status hc_kplan_cost(const hc_kquery* q, const hc_kindex* const* idx, double level_cost[HC_MAX_VARS],
                        double dom_out[HC_MAX_VARS]);
/* Loop order of least estimated cost (the sum of hc_kplan_cost's level
 * costs) over all n_vars! orders; ties go to the lexicographically smallest
 * order (q->order is ignored).  order_out[0..n_vars) receives it (0xFF
 * after).  Host only. */
hc_status hc_choose_korder(const hc_kquery* q, const hc_kindex* const* idx, uint8_t order_out[HC_MAX_VARS]);

#ifdef __cplusplus
}
#endif
#endif /* HONEYCOMB_KARY_H */
