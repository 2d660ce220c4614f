// C ABI entry points, error reporting, device memory and the share optimizer.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <string>
#include <vector>

#include "hc_internal.cuh"

namespace hc {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_wait_ns{2000000000ull};  // bounded device waits: 2 s by default

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

hc_status fail(hc_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

hc_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HC_ERR_OOM : HC_ERR_CUDA;
}

// Stream-ordered allocations from the device's default memory pool.  The
// pool keeps freed memory for reuse instead of returning it to the driver.
hc_status dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    static thread_local int configured_device = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    if (configured_device != dev) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        configured_device = dev;
    }
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 1, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(HC_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                    cudaGetErrorString(e));
    }
    return HC_OK;
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    static thread_local int dev_cached = -1, sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != dev_cached) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        dev_cached = dev;
    }
    return sms;
}

hc_status result_get(hc_result* r, hc_result_view* v);

// ------------------------------------------------------------ share choice
// Cost of one loop order with all shares 1 (Sec. 5.2): for loop i the
// bound of Lemma "cost-ub",
//   C_i = |S(X_i)| * (sum min N) * log2(1 + sum max N / sum min N),
// with the sums over the bindings of the prefix query Q(X_1..X_{i-1}).  The
// number of those bindings is estimated level by level: a binding's lists at
// loop i have average lengths  |R_j.X_first| (a top level, distinct first
// values) or |R_j| / |R_j.X_first| (a sub-list R_j[x]), and a k-way
// intersection of lists of average lengths s_1..s_k over a domain of D values
// keeps about s_1 * ... * s_k / D^(k-1) values (independence), at most
// min s_q.  The per-binding averages give sum min N and sum max N (the
// paper's own ratio estimate, the example after Lemma "cost-ub").  The
// query rewriting run_join applies by default is part of the estimate.
struct AtomStat {
    double rows, col0_distinct, col1_distinct;
};

static void level_costs(const hc_query* q, const int* rank, const AtomStat* st, const double* dom, double* cost) {
    const int nv = (int)q->n_vars, na = (int)q->n_atoms;
    double bindings = 1.0;
    double before[HC_MAX_VARS];  // bindings of the prefix query ahead of loop i
    for (int i = 0; i < nv; ++i) {
        before[i] = bindings;
        int v = q->order[i];
        // query rewriting (Sec. 5.1), as run_join applies it: at the last loop
        // of a query of 4+ variables, two or more lists fixed before loop i-1
        // ("far") are intersected once per binding of loop i-2; the result
        // joins the last loop's lists, and its cost is charged to loop i-1
        // (Sec. 5.2: the lifted relations count at the earlier loop)
        const bool may_lift = i == nv - 1 && nv >= 4;
        double smin = INFINITY, smax = 0.0, prod = 1.0;
        double fmin = INFINITY, fmax = 0.0, fprod = 1.0;
        int k = 0, kf = 0;
        for (int j = 0; j < na; ++j) {
            int a = q->atoms[j].var0, b = q->atoms[j].var1;
            if (a != v && b != v) continue;
            const bool unary = b == (int)HC_UNARY;
            const int other = a == v ? b : a;
            const bool top = unary || rank[other] > i;  // v is the atom's first variable in loop order
            const int first = (unary || rank[a] < rank[b]) ? a : b;
            const double fd = first == a ? st[j].col0_distinct : st[j].col1_distinct;
            const double len = top ? fd : st[j].rows / std::max(1.0, fd);
            if (may_lift && (top || rank[other] <= i - 2)) {
                fmin = std::min(fmin, len);
                fmax = std::max(fmax, len);
                fprod *= len;
                ++kf;
                continue;
            }
            smin = std::min(smin, len);
            smax = std::max(smax, len);
            prod *= len;
            ++k;
        }
        if (kf == 1) {  // a single far list is not rewritten
            smin = std::min(smin, fmin);
            smax = std::max(smax, fmax);
            prod *= fprod;
            ++k;
        } else if (kf >= 2) {
            if (fmin > 0) cost[i - 1] += (double)kf * before[i - 1] * fmin * log2(1.0 + fmax / fmin);
            const double lifted = std::min(fprod / pow(std::max(1.0, dom[v]), (double)(kf - 1)), fmin);
            smin = std::min(smin, lifted);
            smax = std::max(smax, lifted);
            prod *= lifted;
            ++k;
        }
        if (k == 0 || !(smin > 0)) {
            cost[i] = 0.0;
            bindings = 0.0;
            continue;
        }
        double sum_min = bindings * smin, sum_max = bindings * smax;
        cost[i] = (double)k * sum_min * log2(1.0 + sum_max / sum_min);
        double keep = prod / pow(std::max(1.0, dom[v]), (double)(k - 1));
        bindings *= std::min(keep, smin);
    }
}

// Loop ranks, per-atom statistics, domain estimates and per-loop costs.
static hc_status plan_inputs(const hc_query* q, const hc_index* const* idx, int* rank, double* dom, double* cost) {
    if (!q || !idx) return fail(HC_ERR_ARG, "plan: NULL argument");
    const int nv = (int)q->n_vars, na = (int)q->n_atoms;
    if (nv < 1 || nv > HC_MAX_VARS || na < 1 || na > HC_MAX_ATOMS)
        return fail(HC_ERR_ARG, "plan: need 1..8 variables and 1..12 atoms");
    bool seen[HC_MAX_VARS] = {false};
    for (int i = 0; i < nv; ++i) {
        int v = q->order[i];
        if (v >= nv || seen[v]) return fail(HC_ERR_ARG, "plan: order must list every variable once");
        seen[v] = true;
        rank[v] = i;
    }
    AtomStat st[HC_MAX_ATOMS];
    for (int v = 0; v < nv; ++v) dom[v] = INFINITY;
    for (int j = 0; j < na; ++j) {
        if (!idx[j]) return fail(HC_ERR_ARG, "plan: missing index");
        int a = q->atoms[j].var0, b = q->atoms[j].var1;
        const bool unary = b == (int)HC_UNARY;
        if (a >= nv || (b >= nv && !unary) || a == b) return fail(HC_ERR_ARG, "plan: bad atom");
        const hc_index* ix = idx[j];
        // the index knows the distinct count of its own first attribute; the
        // other attribute's is bounded by its largest value + 1 and by the rows
        double d_first = (double)ix->l1;
        double d_second = std::min((double)ix->n, (double)ix->max_second + 1.0);
        double d_col0 = ix->attr_order == 0 ? d_first : d_second;  // column 0 holds var0
        double d_col1 = ix->attr_order == 0 ? d_second : d_first;
        st[j].rows = (double)ix->n;
        st[j].col0_distinct = d_col0;
        st[j].col1_distinct = d_col1;
        dom[a] = std::min(dom[a], d_col0);
        if (!unary) dom[b] = std::min(dom[b], d_col1);
    }
    for (int v = 0; v < nv; ++v)
        if (!(dom[v] < INFINITY)) return fail(HC_ERR_ARG, "plan: a variable occurs in no atom");
    level_costs(q, rank, st, dom, cost);
    return HC_OK;
}

// Eq. "total:cost": sum_i (prod_{k>i} P_sigma(k)) C_i, shares per variable id.
static double replicated(const hc_query* q, const double* cost, const uint32_t* shares) {
    const int nv = (int)q->n_vars;
    double rep = 0.0;
    for (int i = 0; i < nv; ++i) {
        double m = 1.0;
        for (int k = i + 1; k < nv; ++k) m *= (double)shares[q->order[k]];
        rep += m * cost[i];
    }
    return rep;
}

hc_status plan_cost_impl(const hc_query* q, const hc_index* const* idx, const uint32_t* shares, double* level_cost,
                         double* dom_out, double* rep_out) {
    int rank[HC_MAX_VARS];
    double dom[HC_MAX_VARS], cost[HC_MAX_VARS];
    HC_TRY(plan_inputs(q, idx, rank, dom, cost));
    if (!shares) return fail(HC_ERR_ARG, "plan_cost: NULL shares");
    for (int v = 0; v < HC_MAX_VARS; ++v) {
        if (level_cost) level_cost[v] = v < (int)q->n_vars ? cost[v] : 0.0;
        if (dom_out) dom_out[v] = v < (int)q->n_vars ? dom[v] : 0.0;
    }
    if (rep_out) *rep_out = replicated(q, cost, shares);
    return HC_OK;
}

hc_status choose_shares_impl(const hc_query* q, const hc_index* const* idx, uint32_t P, uint32_t* out) {
    if (!out) return fail(HC_ERR_ARG, "choose_shares: NULL argument");
    if (P == 0 || (P & (P - 1)) != 0 || P > 65536) return fail(HC_ERR_ARG, "choose_shares: P must be a power of two <= 2^16");
    int rank[HC_MAX_VARS];
    double dom[HC_MAX_VARS], cost[HC_MAX_VARS];
    HC_TRY(plan_inputs(q, idx, rank, dom, cost));
    const int nv = (int)q->n_vars;
    double base = 0.0;
    for (int i = 0; i < nv; ++i) base += cost[i];

    // enumerate exponent vectors (e_v = log2 P_v, per variable id) summing to log2(P)
    const int total = __builtin_ctz(P);
    std::vector<int> e(nv, 0), best, fallback;
    double best_even = INFINITY, fb_cost = INFINITY;
    auto lex_less = [](const std::vector<int>& x, const std::vector<int>& y) {
        return std::lexicographical_compare(x.begin(), x.end(), y.begin(), y.end());
    };
    auto consider = [&]() {
        uint32_t sh[HC_MAX_VARS];
        for (int v = 0; v < nv; ++v) sh[v] = 1u << e[v];
        const double rep = replicated(q, cost, sh);
        // |Dom(X_v)| >= 3 P_v ln P_v
        for (int v = 0; v < nv; ++v) {
            const double pv = (double)(1u << e[v]);
            if (pv > 1.0 && dom[v] < 3.0 * pv * log(pv)) return;
        }
        if (rep < fb_cost || (rep == fb_cost && lex_less(e, fallback))) {
            fb_cost = rep;
            fallback = e;
        }
        if (rep > 2.0 * base) return;
        double even = 0.0;  // E = sum_i P_sigma(i) w(i), w(i) = max(1 - i/100, 3/4), i from 1
        for (int i = 0; i < nv; ++i) even += (double)(1u << e[q->order[i]]) * std::max(1.0 - (i + 1) / 100.0, 0.75);
        if (best.empty() || even < best_even - 1e-9 || (fabs(even - best_even) <= 1e-9 && lex_less(e, best))) {
            best_even = even;
            best = e;
        }
    };
    // odometer over all compositions of `total` into nv parts
    std::function<void(int, int)> rec = [&](int v, int left) {
        if (v == nv - 1) {
            e[v] = left;
            consider();
            return;
        }
        for (int x = 0; x <= left; ++x) {
            e[v] = x;
            rec(v + 1, left - x);
        }
    };
    rec(0, total);
    for (int v = 0; v < HC_MAX_VARS; ++v) out[v] = 1;
    const std::vector<int>& pick = !best.empty() ? best : fallback;
    if (pick.empty()) {
        out[q->order[0]] = P;  // no vector meets the domain rule: all shares on loop 1
        return HC_OK;
    }
    for (int v = 0; v < nv; ++v) out[v] = 1u << pick[v];
    return HC_OK;
}

// Sec. 5.3 plan decision over all loop orders: the shares of each order as
// chosen above, the order of least replicated cost at its shares.
hc_status choose_plan_impl(const hc_query* q, const hc_index* const* idx, uint32_t P, uint8_t* order_out,
                           uint32_t* shares_out) {
    if (!q || !idx || !order_out || !shares_out) return fail(HC_ERR_ARG, "choose_plan: NULL argument");
    const int nv = (int)q->n_vars;
    if (nv < 1 || nv > HC_MAX_VARS) return fail(HC_ERR_ARG, "choose_plan: need 1..8 variables");
    hc_query w = *q;
    std::vector<uint8_t> perm(nv), best_perm;
    for (int i = 0; i < nv; ++i) perm[i] = (uint8_t)i;
    uint32_t best_sh[HC_MAX_VARS];
    double best_rep = 0.0, best_base = 0.0;
    auto less = [](double a, double b) { return a < b - 1e-9 * std::max(1.0, std::fabs(b)); };
    do {  // lexicographic order, so the first of equal plans is kept
        for (int i = 0; i < nv; ++i) w.order[i] = perm[i];
        uint32_t sh[HC_MAX_VARS];
        HC_TRY(choose_shares_impl(&w, idx, P, sh));
        int rank[HC_MAX_VARS];
        double dom[HC_MAX_VARS], cost[HC_MAX_VARS];
        HC_TRY(plan_inputs(&w, idx, rank, dom, cost));
        double base = 0.0;
        for (int i = 0; i < nv; ++i) base += cost[i];
        const double rep = replicated(&w, cost, sh);
        const bool better = best_perm.empty() || less(rep, best_rep) ||
                            (!less(best_rep, rep) && less(base, best_base));
        if (better) {
            best_perm = perm;
            best_rep = rep;
            best_base = base;
            std::copy(sh, sh + HC_MAX_VARS, best_sh);
        }
    } while (std::next_permutation(perm.begin(), perm.end()));
    for (int i = 0; i < HC_MAX_VARS; ++i) order_out[i] = i < nv ? best_perm[i] : (uint8_t)0xFF;
    std::copy(best_sh, best_sh + HC_MAX_VARS, shares_out);
    return HC_OK;
}

}  // namespace hc

// ------------------------------------------------------------------- C ABI
extern "C" {

hc_status hc_build_index(const uint32_t* d_pairs, uint64_t n, uint32_t attr_order, uint32_t flags, void* stream,
                         hc_index** out) {
    return hc::build_index_impl(d_pairs, n, attr_order, flags & ~hc::BUILD_NO_DIRECTORIES, (cudaStream_t)stream, out);
}

hc_status hc_build_unary_index(const uint32_t* d_values, uint64_t n, uint32_t max_value, void* stream,
                               hc_index** out) {
    return hc::build_unary_impl(d_values, n, max_value, (cudaStream_t)stream, out);
}

hc_status hc_index_from_stats(uint64_t n, uint64_t l1, uint32_t attr_order, uint32_t max_first, uint32_t max_second,
                              uint64_t max_run, hc_index** out) {
    if (!out) return hc::fail(HC_ERR_ARG, "index_from_stats: out is NULL");
    *out = nullptr;
    if (attr_order > 1 || l1 > n || (n > 0 && l1 == 0))
        return hc::fail(HC_ERR_ARG, "index_from_stats: need attr_order 0/1 and 1 <= l1 <= n");
    if (max_run > 0 && (n == 0 || max_run > n - l1 + 1))
        return hc::fail(HC_ERR_ARG, "index_from_stats: max_run must be 0 (unknown) or in [1, n - l1 + 1]");
    hc_index* ix = new hc_index();
    ix->n = n;
    ix->l1 = l1;
    ix->attr_order = attr_order;
    ix->max_first = max_first;
    ix->max_second = max_second;
    ix->max_run = max_run;  // 0: unknown (not checked against the search kernels' list limit)
    ix->stats_only = true;
    *out = ix;
    return HC_OK;
}

hc_status hc_index_free(hc_index* index) {
    if (!index) return HC_OK;
    hc::index_release(index, nullptr);
    return HC_OK;
}

hc_status hc_index_get_view(const hc_index* ix, hc_index_view* out) {
    if (!ix || !out) return hc::fail(HC_ERR_ARG, "index_get_view: NULL argument");
    out->n = ix->n;
    out->l1 = ix->l1;
    out->attr_order = ix->attr_order;
    out->max_first = ix->max_first;
    out->max_second = ix->max_second;
    out->d_v1 = ix->d_v1;
    out->d_o1 = ix->d_o1;
    out->d_v2 = ix->d_v2;
    out->d_keys = ix->d_keys;
    out->ms_radix_passes = ix->ms_radix;
    out->n_radix_passes = ix->n_radix;
    out->ms_boundary = ix->ms_boundary;
    out->max_run = ix->max_run;
    out->v1pos_n = ix->v1pos_n;
    return HC_OK;
}

hc_status hc_partition_index(const hc_index* index, uint32_t seed_a, uint32_t pa, uint32_t seed_b, uint32_t pb,
                             void* stream, hc_partitioned** out) {
    return hc::partition_impl(index, seed_a, pa, seed_b, pb, (cudaStream_t)stream, out);
}

hc_status hc_partitioned_get_view(hc_partitioned* p, hc_partitioned_view* out) {
    if (!p || !out) return hc::fail(HC_ERR_ARG, "partitioned_get_view: NULL argument");
    hc_status st = hc::partitioned_sync(p);
    if (st != HC_OK) return st;
    out->n = p->n;
    out->l1 = p->l1;
    out->n_parts = p->n_parts;
    out->pa = p->pa;
    out->pb = p->pb;
    out->d_keys = p->d_keys;
    out->d_bpref = p->d_bpref;
    out->d_v1 = p->d_v1;
    out->d_o1 = p->d_o1;
    out->d_v2 = p->d_v2;
    out->d_lvl1_start = p->d_lvl1_start;
    return HC_OK;
}

hc_status hc_partitioned_free(hc_partitioned* p) {
    if (!p) return HC_OK;
    hc::partitioned_release(p, p->stream);
    return HC_OK;
}

hc_status hc_choose_shares(const hc_query* q, const hc_index* const* idx, uint32_t P, uint32_t shares_out[HC_MAX_VARS]) {
    return hc::choose_shares_impl(q, idx, P, shares_out);
}

hc_status hc_choose_plan(const hc_query* q, const hc_index* const* idx, uint32_t P, uint8_t order_out[HC_MAX_VARS],
                         uint32_t shares_out[HC_MAX_VARS]) {
    return hc::choose_plan_impl(q, idx, P, order_out, shares_out);
}

hc_status hc_plan_cost(const hc_query* q, const hc_index* const* idx, const uint32_t shares[HC_MAX_VARS],
                       double level_cost[HC_MAX_VARS], double dom_out[HC_MAX_VARS], double* replicated_cost) {
    return hc::plan_cost_impl(q, idx, shares, level_cost, dom_out, replicated_cost);
}

hc_status hc_run_join(const hc_query* q, const hc_index* const* idx, const hc_join_params* params, void* stream,
                      hc_result** out) {
    return hc::run_join_impl(q, idx, params, (cudaStream_t)stream, out);
}

hc_status hc_result_get(hc_result* r, hc_result_view* out) { return hc::result_get(r, out); }

hc_status hc_run_join_to_host(const hc_query* q, const hc_index* const* idx, const hc_join_params* params,
                              uint32_t* h_tuples, uint64_t capacity, uint64_t* count_out, void* stream) {
    return hc::run_join_to_host_impl(q, idx, params, h_tuples, capacity, count_out, (cudaStream_t)stream);
}

hc_status hc_join_footprint(const hc_query* q, const hc_index* const* idx, const hc_join_params* params,
                            uint64_t* bytes_out) {
    return hc::join_footprint_impl(q, idx, params, bytes_out);
}

hc_status hc_batch_create(const hc_query* qs, const hc_index* const* idx_flat, const hc_join_params* prm, uint32_t n,
                          void* stream, hc_batch** out) {
    return hc::batch_create(qs, idx_flat, prm, n, (cudaStream_t)stream, out);
}
hc_status hc_batch_launch(hc_batch* b, void* stream) { return hc::batch_launch(b, (cudaStream_t)stream); }
hc_status hc_batch_capture(hc_batch* b, void* stream) { return hc::batch_capture(b, (cudaStream_t)stream); }
hc_status hc_batch_counts(hc_batch* b, uint64_t* counts) { return hc::batch_counts(b, counts); }
hc_status hc_batch_free(hc_batch* b) {
    hc::batch_release(b);
    return HC_OK;
}

hc_status hc_result_free(hc_result* r) {
    hc::result_release(r);
    return HC_OK;
}

const char* hc_status_str(hc_status s) {
    switch (s) {
        case HC_OK: return "ok";
        case HC_ERR_ARG: return "invalid argument";
        case HC_ERR_OOM: return "out of memory";
        case HC_ERR_CUDA: return "CUDA error";
        case HC_ERR_TIMEOUT: return "bounded device wait gave up";
        case HC_ERR_CAPACITY: return "size beyond a fixed limit";
        case HC_ERR_DUPLICATE: return "relation holds a repeated row";
        case HC_ERR_BUSY: return "queue or budget full";
    }
    return "unknown status";
}

const char* hc_last_error(void) { return hc::g_last_error.c_str(); }

uint32_t hc_version(void) { return 100; }

hc_status hc_set_wait_limit_ns(uint64_t ns) {
    hc::g_wait_ns.store(ns, std::memory_order_relaxed);
    return HC_OK;
}
uint64_t hc_wait_limit_ns(void) { return hc::g_wait_ns.load(std::memory_order_relaxed); }
uint64_t hc_kernel_launches(void) { return hc::g_launches.load(std::memory_order_relaxed); }
uint32_t hc_target_sm(void) { return 103; }

}  // extern "C"
