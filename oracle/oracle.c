/*
 * CPU oracle for the HoneyComb hot path (Wu & Suciu, "HoneyComb: A Parallel
 * Worst-Case Optimal Join on Multicores").  TEST INFRASTRUCTURE ONLY: it is
 * called by the test-suite, by the smoke check and by the timed CPU baseline
 * of the benchmark, never by the product path.  It shares no code with the
 * CUDA library.
 *
 * Everything here is the plain definition, computed slowly:
 *   - oc_coco_build     : the CoCo trie of a binary relation (Sec. 4, the
 *                         "Construction of CoCo" paragraphs and Fig.
 *                         "cocoindex"): sort the relation lexicographically
 *                         in the chosen column order (a library qsort), then
 *                         one loop over the sorted rows emits a new level-1
 *                         entry whenever the first column changes.
 *   - oc_fmix32, oc_share : the per-variable hash h_i (x) mod P_i of the
 *                         HyperCube partitioning (Sec. 2 "HyperCube
 *                         Algorithm" footnote, Sec. 4).  The paper leaves the
 *                         hash open; h(x) = fmix32(x xor seed) (the MurmurHash3
 *                         finaliser, Appleby 2011) with share index
 *                         (h * P) >> 32 is the reading used throughout.
 *   - oc_partition      : the partitioned relation R~_j, its histogram B_j
 *                         and exclusive prefix B^pref_j in lexicographic order
 *                         of the partition identifiers (Sec. 4, the
 *                         partitioning paragraphs and Example "partition"),
 *                         and one CoCo per partition.
 *   - oc_gj_count / oc_gj_enumerate : Generic Join (Sec. 2 "Generic Join
 *                         Algorithm"): n nested loops in the chosen variable
 *                         order; loop i intersects the columns of every atom
 *                         holding X_i (the full top level of atoms whose first
 *                         attribute is X_i, the sub-array R[x] (Sec. 5, level
 *                         restriction, read as half open [O[idx], O[idx+1]))
 *                         of atoms whose first attribute is already bound),
 *                         by a plain k-way linear merge.  The result is the set
 *                         of all bindings satisfying every atom (Eq.
 *                         "full:cq"); count mode adds the size of the last
 *                         intersection.
 *   - the work counter  : sum over levels and bindings of |S| * min N, the
 *                         per-binding intersection cost of Sec. 5.2 ("Cost
 *                         Model") without its log factor, with N taken as the
 *                         lengths of the lists actually intersected.
 *
 * No blocking, fusion or reordering beyond those definitions.  Errors are
 * returned as non-zero codes.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_MAXV 8
#define OC_MAXA 16

enum { OC_OK = 0, OC_EARG = 1, OC_ENOMEM = 2, OC_ECAP = 3 };

/* ---------------------------------------------------------------- hashing */

uint32_t oc_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

uint32_t oc_share(uint32_t x, uint32_t seed, uint32_t p) {
    return (uint32_t)(((uint64_t)oc_fmix32(x ^ seed) * (uint64_t)p) >> 32);
}

/* ------------------------------------------------------------------- trie */

typedef struct {
    uint64_t n, l1;
    uint32_t *v1; /* [l1]   distinct first values, ascending          */
    uint64_t *o1; /* [l1+1] start of each value's run in v2; o1[l1]=n  */
    uint32_t *v2; /* [n]    second values                              */
} trie_t;

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Sorted keys (first << 32 | second) of a relation in column order `swap`. */
static uint64_t *sorted_keys(const uint32_t *pairs, uint64_t n, int swap) {
    uint64_t *k = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!k) return NULL;
    for (uint64_t t = 0; t < n; ++t) {
        uint32_t a = pairs[2 * t + (swap ? 1 : 0)], b = pairs[2 * t + (swap ? 0 : 1)];
        k[t] = ((uint64_t)a << 32) | b;
    }
    qsort(k, n, sizeof(uint64_t), cmp_u64);
    return k;
}

/* Levels of the trie from keys already sorted: one pass, a new level-1 entry
 * whenever the first column differs from the previous row. */
static int trie_from_sorted(const uint64_t *k, uint64_t n, trie_t *t) {
    t->n = n;
    t->v1 = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    t->o1 = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    t->v2 = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!t->v1 || !t->o1 || !t->v2) return OC_ENOMEM;
    uint64_t l = 0;
    for (uint64_t r = 0; r < n; ++r) {
        uint32_t a = (uint32_t)(k[r] >> 32);
        if (r == 0 || (uint32_t)(k[r - 1] >> 32) != a) {
            t->v1[l] = a;
            t->o1[l] = r;
            ++l;
        }
        t->v2[r] = (uint32_t)k[r];
    }
    t->o1[l] = n;
    t->l1 = l;
    return OC_OK;
}

static void trie_free(trie_t *t) {
    free(t->v1);
    free(t->o1);
    free(t->v2);
    memset(t, 0, sizeof(*t));
}

static int build_trie(const uint32_t *pairs, uint64_t n, int swap, trie_t *t) {
    memset(t, 0, sizeof(*t));
    uint64_t *k = sorted_keys(pairs, n, swap);
    if (!k) return OC_ENOMEM;
    int rc = trie_from_sorted(k, n, t);
    free(k);
    return rc;
}

/* Returns 1 when the relation holds a repeated pair (it must be a set). */
int oc_has_duplicates(const uint32_t *pairs, uint64_t n) {
    uint64_t *k = sorted_keys(pairs, n, 0);
    if (!k) return -1;
    int dup = 0;
    for (uint64_t t = 1; t < n && !dup; ++t) dup = k[t] == k[t - 1];
    free(k);
    return dup;
}

/* CoCo of a binary relation.  attr_order 0 keys (col0, col1), 1 keys
 * (col1, col0).  Caller buffers: v1[n], o1[n+1], v2[n]. */
int oc_coco_build(const uint32_t *pairs, uint64_t n, int attr_order, uint32_t *v1, uint64_t *o1,
                  uint32_t *v2, uint64_t *l1_out) {
    if ((attr_order != 0 && attr_order != 1) || (n && !pairs)) return OC_EARG;
    trie_t t;
    int rc = build_trie(pairs, n, attr_order, &t);
    if (rc) {
        trie_free(&t);
        return rc;
    }
    memcpy(v1, t.v1, t.l1 * sizeof(uint32_t));
    memcpy(o1, t.o1, (t.l1 + 1) * sizeof(uint64_t));
    memcpy(v2, t.v2, n * sizeof(uint32_t));
    *l1_out = t.l1;
    trie_free(&t);
    return OC_OK;
}

/* -------------------------------------------------------------- partition */

/* Partitioned relation.  Tuple (a, b) (in attr_order) has identifiers
 * s_a = share(a, seed_a, pa), s_b = share(b, seed_b, pb) and partition
 * pid = s_a * pb + s_b (lexicographic).  Outputs: rt[2n] the tuples of each
 * partition, partitions concatenated by pid and each sorted by (a, b);
 * hist[pa*pb] = B; pref[pa*pb+1] = exclusive prefix of B (pref[last] = n);
 * per-partition CoCo concatenated: v1[<=n], o1[<=n+1] (offsets into rt, i.e.
 * global), lvl1_start[pa*pb+1] (start of each partition's level 1 in v1). */
int oc_partition(const uint32_t *pairs, uint64_t n, int attr_order, uint32_t seed_a, uint32_t pa,
                 uint32_t seed_b, uint32_t pb, uint32_t *rt, uint64_t *hist, uint64_t *pref,
                 uint32_t *v1, uint64_t *o1, uint64_t *lvl1_start, uint64_t *l1_total) {
    if ((attr_order != 0 && attr_order != 1) || pa == 0 || pb == 0) return OC_EARG;
    uint64_t np = (uint64_t)pa * pb;
    uint64_t *k = sorted_keys(pairs, n, attr_order);
    if (!k) return OC_ENOMEM;
    memset(hist, 0, np * sizeof(uint64_t));
    for (uint64_t t = 0; t < n; ++t) {
        uint32_t a = (uint32_t)(k[t] >> 32), b = (uint32_t)k[t];
        hist[(uint64_t)oc_share(a, seed_a, pa) * pb + oc_share(b, seed_b, pb)]++;
    }
    pref[0] = 0;
    for (uint64_t p = 0; p < np; ++p) pref[p + 1] = pref[p] + hist[p];
    uint64_t *cur = (uint64_t *)malloc((np ? np : 1) * sizeof(uint64_t));
    if (!cur) {
        free(k);
        return OC_ENOMEM;
    }
    memcpy(cur, pref, np * sizeof(uint64_t));
    /* rows visited in sorted order, so each partition comes out sorted */
    for (uint64_t t = 0; t < n; ++t) {
        uint32_t a = (uint32_t)(k[t] >> 32), b = (uint32_t)k[t];
        uint64_t p = (uint64_t)oc_share(a, seed_a, pa) * pb + oc_share(b, seed_b, pb);
        uint64_t d = cur[p]++;
        rt[2 * d] = a;
        rt[2 * d + 1] = b;
    }
    free(cur);
    free(k);
    uint64_t l = 0;
    for (uint64_t p = 0; p < np; ++p) {
        lvl1_start[p] = l;
        for (uint64_t r = pref[p]; r < pref[p + 1]; ++r) {
            if (r == pref[p] || rt[2 * (r - 1)] != rt[2 * r]) {
                v1[l] = rt[2 * r];
                o1[l] = r;
                ++l;
            }
        }
    }
    lvl1_start[np] = l;
    o1[l] = n;
    *l1_total = l;
    return OC_OK;
}

/* ---------------------------------------------------------- generic join */

typedef struct {
    int nv, na;
    int order[OC_MAXV];             /* order[i] = variable bound by loop i      */
    int rank[OC_MAXV];              /* rank[v]  = loop that binds variable v    */
    int first[OC_MAXA], second[OC_MAXA];
    trie_t trie[OC_MAXA];
    int nsrc[OC_MAXV];
    int src_atom[OC_MAXV][OC_MAXA + 1];
    int src_top[OC_MAXV][OC_MAXA + 1]; /* 1: top level of the atom, 0: R[x]    */
    const uint32_t *filter;         /* optional sorted restriction of loop 1   */
    uint64_t nfilter;
} plan_t;

typedef struct {
    uint64_t lo[OC_MAXA], hi[OC_MAXA];
    uint32_t val[OC_MAXV];
    uint64_t count, work;
    int enumerate;
    uint32_t *out;
    uint64_t cap, nout;
    int overflow;
} state_t;

/* k-way linear merge of sorted lists; calls back with the positions of each
 * common value.  Returns the number of common values. */
typedef struct {
    const uint32_t *base[OC_MAXA + 1];
    uint64_t lo[OC_MAXA + 1], hi[OC_MAXA + 1];
    int k;
} lists_t;

static void plan_lists(const plan_t *p, int lvl, const state_t *s, lists_t *L) {
    L->k = 0;
    for (int q = 0; q < p->nsrc[lvl]; ++q) {
        int j = p->src_atom[lvl][q];
        if (p->src_top[lvl][q]) {
            L->base[L->k] = p->trie[j].v1;
            L->lo[L->k] = 0;
            L->hi[L->k] = p->trie[j].l1;
        } else {
            L->base[L->k] = p->trie[j].v2;
            L->lo[L->k] = s->lo[j];
            L->hi[L->k] = s->hi[j];
        }
        L->k++;
    }
    if (lvl == 0 && p->filter) {
        L->base[L->k] = p->filter;
        L->lo[L->k] = 0;
        L->hi[L->k] = p->nfilter;
        L->k++;
    }
}

static void emit(const plan_t *p, state_t *s) {
    if (s->nout >= s->cap) {
        s->overflow = 1;
        s->nout++;
        return;
    }
    for (int v = 0; v < p->nv; ++v) s->out[s->nout * (uint64_t)p->nv + v] = s->val[v];
    s->nout++;
}

static void gj_level(const plan_t *p, int lvl, state_t *s);

/* Intersect the lists of loop `lvl` and descend for every common value. */
static void gj_intersect_and_descend(const plan_t *p, int lvl, state_t *s, const lists_t *L) {
    uint64_t cur[OC_MAXA + 1];
    uint64_t minlen = UINT64_MAX;
    int nsrc = p->nsrc[lvl];
    for (int q = 0; q < L->k; ++q) {
        cur[q] = L->lo[q];
        uint64_t len = L->hi[q] - L->lo[q];
        if (q < nsrc && len < minlen) minlen = len;
    }
    s->work += (uint64_t)nsrc * (minlen == UINT64_MAX ? 0 : minlen);
    int last = lvl == p->nv - 1;
    for (;;) {
        int done = 0;
        uint32_t mx = 0;
        for (int q = 0; q < L->k; ++q) {
            if (cur[q] >= L->hi[q]) {
                done = 1;
                break;
            }
            if (L->base[q][cur[q]] > mx) mx = L->base[q][cur[q]];
        }
        if (done) break;
        int all_eq = 1;
        for (int q = 0; q < L->k; ++q) {
            while (cur[q] < L->hi[q] && L->base[q][cur[q]] < mx) cur[q]++;
            if (cur[q] >= L->hi[q]) {
                done = 1;
                break;
            }
            if (L->base[q][cur[q]] != mx) all_eq = 0;
        }
        if (done) break;
        if (!all_eq) continue;
        /* mx is common to every list: bind it */
        int var = p->order[lvl];
        s->val[var] = mx;
        if (last && !s->enumerate) {
            s->count++;
        } else {
            uint64_t save_lo[OC_MAXA], save_hi[OC_MAXA];
            for (int q = 0; q < nsrc; ++q) {
                if (!p->src_top[lvl][q]) continue;
                int j = p->src_atom[lvl][q];
                save_lo[j] = s->lo[j];
                save_hi[j] = s->hi[j];
                s->lo[j] = p->trie[j].o1[cur[q]];
                s->hi[j] = p->trie[j].o1[cur[q] + 1];
            }
            if (last) {
                s->count++;
                emit(p, s);
            } else {
                gj_level(p, lvl + 1, s);
            }
            for (int q = 0; q < nsrc; ++q) {
                if (!p->src_top[lvl][q]) continue;
                int j = p->src_atom[lvl][q];
                s->lo[j] = save_lo[j];
                s->hi[j] = save_hi[j];
            }
        }
        for (int q = 0; q < L->k; ++q) cur[q]++;
    }
}

static void gj_level(const plan_t *p, int lvl, state_t *s) {
    lists_t L;
    plan_lists(p, lvl, s, &L);
    gj_intersect_and_descend(p, lvl, s, &L);
}

/* atoms: na entries of (pairs pointer, n, var of column 0, var of column 1). */
static int plan_build(int nv, int na, const uint32_t *const *pairs, const uint64_t *n,
                      const int *var0, const int *var1, const int *order, const uint32_t *filter,
                      uint64_t nfilter, plan_t *p) {
    memset(p, 0, sizeof(*p));
    if (nv < 1 || nv > OC_MAXV || na < 1 || na > OC_MAXA) return OC_EARG;
    p->nv = nv;
    p->na = na;
    int seen[OC_MAXV] = {0};
    for (int i = 0; i < nv; ++i) {
        if (order[i] < 0 || order[i] >= nv || seen[order[i]]) return OC_EARG;
        seen[order[i]] = 1;
        p->order[i] = order[i];
        p->rank[order[i]] = i;
    }
    int covered[OC_MAXV] = {0};
    for (int j = 0; j < na; ++j) {
        /* var1 = -1: a unary atom R_j(X_var0) over column 0 of its relation */
        if (var0[j] < 0 || var0[j] >= nv || var1[j] < -1 || var1[j] >= nv || var0[j] == var1[j])
            return OC_EARG;
        covered[var0[j]] = 1;
        if (var1[j] >= 0) covered[var1[j]] = 1;
    }
    for (int v = 0; v < nv; ++v)
        if (!covered[v]) return OC_EARG; /* every variable occurs in some atom */
    for (int j = 0; j < na; ++j) {
        int swap = var1[j] >= 0 && p->rank[var1[j]] < p->rank[var0[j]];
        p->first[j] = swap ? var1[j] : var0[j];
        p->second[j] = var1[j] < 0 ? -1 : (swap ? var0[j] : var1[j]);
        int rc = build_trie(pairs[j], n[j], swap, &p->trie[j]);
        if (rc) return rc;
    }
    for (int i = 0; i < nv; ++i) {
        int v = p->order[i];
        for (int j = 0; j < na; ++j) {
            if (p->first[j] == v) {
                p->src_atom[i][p->nsrc[i]] = j;
                p->src_top[i][p->nsrc[i]] = 1;
                p->nsrc[i]++;
            } else if (p->second[j] == v) {
                p->src_atom[i][p->nsrc[i]] = j;
                p->src_top[i][p->nsrc[i]] = 0;
                p->nsrc[i]++;
            }
        }
    }
    p->filter = filter;
    p->nfilter = filter ? nfilter : 0;
    return OC_OK;
}

static void plan_free(plan_t *p) {
    for (int j = 0; j < p->na; ++j) trie_free(&p->trie[j]);
}

/* Loop-1 bindings are shared out over threads: thread t takes every T-th
 * common value of the loop-1 intersection and runs the inner loops on it. */
typedef struct {
    const plan_t *p;
    uint32_t *vals;
    uint64_t (*pos)[OC_MAXA + 1];
    uint64_t nvals;
    int t, nthreads;
    uint64_t count, work;
    uint64_t *per_top; /* optional per loop-1 value counts */
} worker_t;

static void *gj_worker(void *arg) {
    worker_t *w = (worker_t *)arg;
    const plan_t *p = w->p;
    state_t s;
    memset(&s, 0, sizeof(s));
    for (uint64_t i = (uint64_t)w->t; i < w->nvals; i += (uint64_t)w->nthreads) {
        uint64_t c0 = s.count;
        int var = p->order[0];
        s.val[var] = w->vals[i];
        for (int q = 0; q < p->nsrc[0]; ++q) {
            int j = p->src_atom[0][q]; /* loop 1 only has top-level sources */
            s.lo[j] = p->trie[j].o1[w->pos[i][q]];
            s.hi[j] = p->trie[j].o1[w->pos[i][q] + 1];
        }
        if (p->nv == 1)
            s.count++;
        else
            gj_level(p, 1, &s);
        if (w->per_top) w->per_top[i] = s.count - c0;
    }
    w->count = s.count;
    w->work = s.work;
    return NULL;
}

/* Loop-1 intersection with positions in every list. */
static int level1(const plan_t *p, uint32_t **vals_out, uint64_t (**pos_out)[OC_MAXA + 1],
                  uint64_t *n_out, uint64_t *work) {
    lists_t L;
    state_t dummy;
    memset(&dummy, 0, sizeof(dummy));
    plan_lists(p, 0, &dummy, &L);
    uint64_t cap = UINT64_MAX, minlen = UINT64_MAX;
    for (int q = 0; q < L.k; ++q) {
        uint64_t len = L.hi[q] - L.lo[q];
        if (len < cap) cap = len;
        if (q < p->nsrc[0] && len < minlen) minlen = len;
    }
    *work += (uint64_t)p->nsrc[0] * minlen;
    uint32_t *vals = (uint32_t *)malloc((cap ? cap : 1) * sizeof(uint32_t));
    uint64_t(*pos)[OC_MAXA + 1] = malloc((cap ? cap : 1) * sizeof(*pos));
    if (!vals || !pos) {
        free(vals);
        free(pos);
        return OC_ENOMEM;
    }
    uint64_t cur[OC_MAXA + 1], nv = 0;
    for (int q = 0; q < L.k; ++q) cur[q] = L.lo[q];
    for (;;) {
        int done = 0;
        uint32_t mx = 0;
        for (int q = 0; q < L.k; ++q) {
            if (cur[q] >= L.hi[q]) {
                done = 1;
                break;
            }
            if (L.base[q][cur[q]] > mx) mx = L.base[q][cur[q]];
        }
        if (done) break;
        int all_eq = 1;
        for (int q = 0; q < L.k; ++q) {
            while (cur[q] < L.hi[q] && L.base[q][cur[q]] < mx) cur[q]++;
            if (cur[q] >= L.hi[q]) {
                done = 1;
                break;
            }
            if (L.base[q][cur[q]] != mx) all_eq = 0;
        }
        if (done) break;
        if (all_eq) {
            vals[nv] = mx;
            for (int q = 0; q < L.k; ++q) pos[nv][q] = cur[q];
            nv++;
            for (int q = 0; q < L.k; ++q) cur[q]++;
        }
    }
    *vals_out = vals;
    *pos_out = pos;
    *n_out = nv;
    return OC_OK;
}

/* Count of the full conjunctive query.  Optional: filter (sorted values that
 * loop 1 is restricted to, i.e. a selection pushed into the loop-1 atoms),
 * per_top[] (count per loop-1 value, in ascending value order, sized by a
 * prior call that returns *n_top), work_out (the work counter). */
int oc_gj_count(int nv, int na, const uint32_t *const *pairs, const uint64_t *n, const int *var0,
                const int *var1, const int *order, const uint32_t *filter, uint64_t nfilter,
                int nthreads, uint64_t *count_out, uint64_t *work_out, uint64_t *per_top,
                uint64_t per_top_cap, uint64_t *n_top) {
    plan_t p;
    int rc = plan_build(nv, na, pairs, n, var0, var1, order, filter, nfilter, &p);
    if (rc) {
        plan_free(&p);
        return rc;
    }
    uint32_t *vals = NULL;
    uint64_t(*pos)[OC_MAXA + 1] = NULL;
    uint64_t nvals = 0, work = 0;
    rc = level1(&p, &vals, &pos, &nvals, &work);
    if (rc) {
        plan_free(&p);
        return rc;
    }
    if (n_top) *n_top = nvals;
    if (per_top && per_top_cap < nvals) per_top = NULL, rc = OC_ECAP;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    worker_t w[256];
    pthread_t th[256];
    int live[256];
    for (int t = 0; t < nthreads; ++t) {
        w[t] = (worker_t){&p, vals, pos, nvals, t, nthreads, 0, 0, per_top};
        live[t] = nthreads > 1 && pthread_create(&th[t], NULL, gj_worker, &w[t]) == 0;
        if (!live[t]) gj_worker(&w[t]);
    }
    uint64_t count = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (live[t]) pthread_join(th[t], NULL);
        count += w[t].count;
        work += w[t].work;
    }
    *count_out = count;
    if (work_out) *work_out = work;
    free(vals);
    free(pos);
    plan_free(&p);
    return rc;
}

/* All output tuples (single thread), each as nv values in variable-id order.
 * Writes at most `cap` tuples; *n_out is the full count (OC_ECAP if it did
 * not fit).  Tuples come in the loop order's lexicographic order. */
int oc_gj_enumerate(int nv, int na, const uint32_t *const *pairs, const uint64_t *n,
                    const int *var0, const int *var1, const int *order, const uint32_t *filter,
                    uint64_t nfilter, uint32_t *out, uint64_t cap, uint64_t *n_out) {
    plan_t p;
    int rc = plan_build(nv, na, pairs, n, var0, var1, order, filter, nfilter, &p);
    if (rc) {
        plan_free(&p);
        return rc;
    }
    state_t s;
    memset(&s, 0, sizeof(s));
    s.enumerate = 1;
    s.out = out;
    s.cap = cap;
    if (nv == 1) {
        lists_t L;
        plan_lists(&p, 0, &s, &L);
        gj_intersect_and_descend(&p, 0, &s, &L);
    } else {
        gj_level(&p, 0, &s);
    }
    *n_out = s.nout;
    plan_free(&p);
    return s.overflow ? OC_ECAP : OC_OK;
}

/* HyperCube cell of each output tuple: cell = mixed-radix number of the
 * per-variable shares (s_1, ..., s_n) in variable-id order, s_1 most
 * significant.  tuples[nt * nv] in variable-id order. */
int oc_tuple_cells(const uint32_t *tuples, uint64_t nt, int nv, const uint32_t *seeds,
                   const uint32_t *shares, uint32_t *cell_out) {
    if (nv < 1 || nv > OC_MAXV) return OC_EARG;
    for (int v = 0; v < nv; ++v)
        if (shares[v] == 0) return OC_EARG;
    for (uint64_t t = 0; t < nt; ++t) {
        uint64_t c = 0;
        for (int v = 0; v < nv; ++v)
            c = c * shares[v] + oc_share(tuples[t * (uint64_t)nv + v], seeds[v], shares[v]);
        cell_out[t] = (uint32_t)c;
    }
    return OC_OK;
}
