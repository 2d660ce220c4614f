/*
 * CPU oracle: Generic Join over relations of arity 1 to 3 (Sec. 2, "Generic
 * Join Algorithm"), for the k-ary queries of the paper's Table "Queries"
 * (Loomis-Whitney LW and Clover-Triangle CT over ternary relations).  TEST
 * INFRASTRUCTURE ONLY, like oracle.c; it shares no code with the CUDA library.
 *
 * The plain definition, computed slowly:
 *   - each atom's rows are sorted lexicographically with the atom's columns
 *     taken in loop order of their variables: the k-level sorted trie of
 *     Sec. 4 (CoCo) generalised from two levels, kept here as the sorted
 *     rows themselves;
 *   - every atom keeps the half-open range of its rows that agree with the
 *     values bound so far (the level restriction of Sec. 5);
 *   - loop i runs over the distinct values of X_i in the range of the atom
 *     holding X_i with the fewest rows in range, keeps a value when every
 *     other atom holding X_i has rows with it (found by binary search in its
 *     range), narrows every such atom's range to the value's rows and goes to
 *     loop i+1.  Each complete binding is one output tuple of Eq. "full:cq".
 *
 * With a work output, each loop also adds (number of lists) * (shortest list
 * length) for every binding it runs under, a list's length being the number
 * of distinct values of the variable's column in the atom's range: the work
 * measure of the library's statistics (the per-binding cost of Sec. 5.2
 * without its log factor).
 *
 * Counting can run on several threads: the rows of the first loop's
 * shortest list are cut into pieces at value boundaries, each thread runs
 * the loops over its piece (a value is searched in the other lists only
 * within its own piece's range of that list, so every binding of the first
 * loop belongs to exactly one thread), and the counts and work are summed.
 *
 * Errors are returned as non-zero codes.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK_MAXV 8
#define OK_MAXA 16

enum { OK_OK = 0, OK_EARG = 1, OK_ENOMEM = 2 };

typedef struct {
    uint32_t c[3]; /* columns in loop order of their variables; unused columns 0 */
} row3_t;

typedef struct {
    int k;      /* arity, 1..3 */
    uint64_t n; /* rows */
    row3_t *r;  /* sorted */
} katom_t;

typedef struct {
    int nv, na;
    int order[OK_MAXV];
    katom_t a[OK_MAXA];
    int nat[OK_MAXV];          /* atoms holding the variable of loop i */
    int at[OK_MAXV][OK_MAXA];  /* their indices */
    int dep[OK_MAXV][OK_MAXA]; /* the column of that variable in each */
    uint64_t lo[OK_MAXA], hi[OK_MAXA];
    uint32_t bind[OK_MAXV];
    uint64_t count;
    uint64_t work;
    int want_work;
    int skip_work0; /* the first loop's work is added once, outside the threads */
    uint32_t *out;
    uint64_t cap;
} kplan_t;

static int cmp_row3(const void *x, const void *y) {
    const row3_t *a = (const row3_t *)x, *b = (const row3_t *)y;
    for (int d = 0; d < 3; ++d) {
        if (a->c[d] != b->c[d]) return a->c[d] < b->c[d] ? -1 : 1;
    }
    return 0;
}

/* First row in [lo, hi) whose column d is >= v (rows in range agree on the
 * columns before d, so column d is sorted there). */
static uint64_t first_ge(const katom_t *a, uint64_t lo, uint64_t hi, int d, uint32_t v) {
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a->r[mid].c[d] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* First row in [lo, hi) whose column d is > v. */
static uint64_t first_gt(const katom_t *a, uint64_t lo, uint64_t hi, int d, uint32_t v) {
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a->r[mid].c[d] <= v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

static void emit(kplan_t *p) {
    if (p->out && p->count < p->cap) memcpy(p->out + p->count * (uint64_t)p->nv, p->bind, sizeof(uint32_t) * p->nv);
    p->count++;
}

/* Distinct values of column d in rows [lo, hi) (sorted there). */
static uint64_t distinct_in(const katom_t *a, uint64_t lo, uint64_t hi, int d) {
    uint64_t c = 0;
    for (uint64_t r = lo; r < hi; ++r)
        if (r == lo || a->r[r].c[d] != a->r[r - 1].c[d]) c++;
    return c;
}

static void loop_level(kplan_t *p, int i) {
    if (p->want_work && !(i == 0 && p->skip_work0)) {
        uint64_t shortest = UINT64_MAX;
        for (int q = 0; q < p->nat[i]; ++q) {
            const int j = p->at[i][q];
            const uint64_t len = distinct_in(&p->a[j], p->lo[j], p->hi[j], p->dep[i][q]);
            if (len < shortest) shortest = len;
        }
        p->work += (uint64_t)p->nat[i] * shortest;
    }
    /* the atom with the fewest rows in range supplies the candidates */
    int drv = -1;
    for (int q = 0; q < p->nat[i]; ++q) {
        int j = p->at[i][q];
        if (drv < 0 || p->hi[j] - p->lo[j] < p->hi[p->at[i][drv]] - p->lo[p->at[i][drv]]) drv = q;
    }
    const int jd = p->at[i][drv], dd = p->dep[i][drv];
    const katom_t *ad = &p->a[jd];
    uint64_t save_lo[OK_MAXA], save_hi[OK_MAXA];
    for (int q = 0; q < p->nat[i]; ++q) {
        save_lo[q] = p->lo[p->at[i][q]];
        save_hi[q] = p->hi[p->at[i][q]];
    }
    uint64_t r = save_lo[drv];
    while (r < save_hi[drv]) {
        const uint32_t v = ad->r[r].c[dd];
        const uint64_t r_end = first_gt(ad, r, save_hi[drv], dd, v);
        uint64_t nlo[OK_MAXA], nhi[OK_MAXA];
        int present = 1;
        for (int q = 0; q < p->nat[i] && present; ++q) {
            if (q == drv) {
                nlo[q] = r;
                nhi[q] = r_end;
                continue;
            }
            const katom_t *a = &p->a[p->at[i][q]];
            const int d = p->dep[i][q];
            nlo[q] = first_ge(a, save_lo[q], save_hi[q], d, v);
            nhi[q] = first_gt(a, nlo[q], save_hi[q], d, v);
            if (nlo[q] == nhi[q]) present = 0;
        }
        if (present) {
            for (int q = 0; q < p->nat[i]; ++q) {
                p->lo[p->at[i][q]] = nlo[q];
                p->hi[p->at[i][q]] = nhi[q];
            }
            p->bind[p->order[i]] = v;
            if (i == p->nv - 1)
                emit(p);
            else
                loop_level(p, i + 1);
        }
        r = r_end;
    }
    for (int q = 0; q < p->nat[i]; ++q) {
        p->lo[p->at[i][q]] = save_lo[q];
        p->hi[p->at[i][q]] = save_hi[q];
    }
}

static void *count_worker(void *arg) {
    loop_level((kplan_t *)arg, 0);
    return NULL;
}

/* Count with up to nthreads threads (see the top of the file). */
static int count_threaded(kplan_t *p, int nthreads) {
    if (nthreads > 64) nthreads = 64;
    /* the first loop's list with the fewest rows, and its column there */
    int q0 = 0;
    for (int q = 1; q < p->nat[0]; ++q)
        if (p->a[p->at[0][q]].n < p->a[p->at[0][q0]].n) q0 = q;
    const int j0 = p->at[0][q0], d0 = p->dep[0][q0];
    const katom_t *a0 = &p->a[j0];
    if (p->want_work) { /* the first loop's work, once, over the full lists */
        uint64_t shortest = UINT64_MAX;
        for (int q = 0; q < p->nat[0]; ++q) {
            const int j = p->at[0][q];
            const uint64_t len = distinct_in(&p->a[j], 0, p->a[j].n, p->dep[0][q]);
            if (len < shortest) shortest = len;
        }
        p->work += (uint64_t)p->nat[0] * shortest;
    }
    /* piece t: rows [cut[t], cut[t+1]) of atom j0, cut at value boundaries */
    uint64_t cut[65];
    cut[0] = 0;
    for (int t = 1; t < nthreads; ++t) {
        uint64_t r = a0->n * (uint64_t)t / (uint64_t)nthreads;
        if (r < cut[t - 1]) r = cut[t - 1];
        while (r > 0 && r < a0->n && a0->r[r].c[d0] == a0->r[r - 1].c[d0]) ++r;
        cut[t] = r;
    }
    cut[nthreads] = a0->n;
    kplan_t *w = (kplan_t *)calloc((size_t)nthreads, sizeof(kplan_t));
    pthread_t th[64];
    int live[64];
    if (!w) return OK_ENOMEM;
    for (int t = 0; t < nthreads; ++t) {
        w[t] = *p;
        w[t].count = 0;
        w[t].work = 0;
        w[t].skip_work0 = 1;
        w[t].lo[j0] = cut[t];
        w[t].hi[j0] = cut[t + 1];
        live[t] = pthread_create(&th[t], NULL, count_worker, &w[t]) == 0;
        if (!live[t]) count_worker(&w[t]);
    }
    for (int t = 0; t < nthreads; ++t) {
        if (live[t]) pthread_join(th[t], NULL);
        p->count += w[t].count;
        p->work += w[t].work;
    }
    free(w);
    return OK_OK;
}

/* Generic Join of a full conjunctive query over atoms of arity 1..3.
 *   nv, na         variables (<= 8) and atoms (<= 16)
 *   arity[j]       1, 2 or 3
 *   vars[3*j + c]  variable of column c of atom j (distinct within an atom)
 *   rows[j]        n[j] rows of arity[j] values, row-major (relations are sets)
 *   order          loop order (variable ids), or NULL for 0, 1, ...
 *   out, cap       optional: up to cap tuples of nv values (variable-id order)
 *   count_out      number of output tuples
 *   work_out       optional: the work measure described at the top
 *   nthreads       threads for counting (ignored when tuples are written) */
int oc_kgj(int nv, int na, const int *arity, const int *vars, const uint32_t *const *rows, const uint64_t *n,
           const int *order, uint32_t *out, uint64_t cap, uint64_t *count_out, uint64_t *work_out, int nthreads) {
    if (nv < 1 || nv > OK_MAXV || na < 1 || na > OK_MAXA || !arity || !vars || !rows || !n || !count_out)
        return OK_EARG;
    kplan_t *p = (kplan_t *)calloc(1, sizeof(kplan_t));
    if (!p) return OK_ENOMEM;
    int rc = OK_OK;
    int rank[OK_MAXV];
    p->nv = nv;
    p->na = na;
    int seen[OK_MAXV] = {0};
    for (int i = 0; i < nv; ++i) {
        const int v = order ? order[i] : i;
        if (v < 0 || v >= nv || seen[v]) {
            rc = OK_EARG;
            goto done;
        }
        seen[v] = 1;
        p->order[i] = v;
        rank[v] = i;
    }
    for (int j = 0; j < na; ++j) {
        const int k = arity[j];
        if (k < 1 || k > 3) {
            rc = OK_EARG;
            goto done;
        }
        /* columns ordered by the loop rank of their variables */
        int cols[3] = {0, 1, 2};
        for (int c = 0; c < k; ++c) {
            const int v = vars[3 * j + c];
            if (v < 0 || v >= nv) {
                rc = OK_EARG;
                goto done;
            }
            for (int c2 = 0; c2 < c; ++c2)
                if (vars[3 * j + c2] == v) {
                    rc = OK_EARG;
                    goto done;
                }
        }
        for (int x = 1; x < k; ++x)
            for (int y = x; y > 0 && rank[vars[3 * j + cols[y]]] < rank[vars[3 * j + cols[y - 1]]]; --y) {
                int t = cols[y];
                cols[y] = cols[y - 1];
                cols[y - 1] = t;
            }
        katom_t *a = &p->a[j];
        a->k = k;
        a->n = n[j];
        a->r = (row3_t *)calloc(n[j] ? n[j] : 1, sizeof(row3_t));
        if (!a->r) {
            rc = OK_ENOMEM;
            goto done;
        }
        for (uint64_t r = 0; r < n[j]; ++r)
            for (int d = 0; d < k; ++d) a->r[r].c[d] = rows[j][r * (uint64_t)k + cols[d]];
        qsort(a->r, n[j], sizeof(row3_t), cmp_row3);
        for (int d = 0; d < k; ++d) {
            const int i = rank[vars[3 * j + cols[d]]];
            p->at[i][p->nat[i]] = j;
            p->dep[i][p->nat[i]] = d;
            p->nat[i]++;
        }
        p->lo[j] = 0;
        p->hi[j] = n[j];
    }
    for (int i = 0; i < nv; ++i)
        if (p->nat[i] == 0) {
            rc = OK_EARG; /* a variable in no atom */
            goto done;
        }
    p->out = out;
    p->cap = out ? cap : 0;
    p->want_work = work_out != NULL;
    if (nthreads > 1 && !out) {
        rc = count_threaded(p, nthreads);
        if (rc != OK_OK) goto done;
    } else {
        loop_level(p, 0);
    }
    *count_out = p->count;
    if (work_out) *work_out = p->work;
done:
    for (int j = 0; j < na; ++j) free(p->a[j].r);
    free(p);
    return rc;
}
