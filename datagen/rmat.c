/* R-MAT edge draws for the seeded input generators (inputs only: no join
 * arithmetic lives here).
 *
 * Edge e takes its level-l quadrant from a 32-bit draw
 *     w = half (l & 1) of mix64(key + (e * 32 + l / 2) * GOLDEN)
 * where mix64 is the SplitMix64 output function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) and key is
 * derived from the seed.  Quadrant (0,0), (0,1), (1,0), (1,1) is chosen when
 * w < t1, t1 <= w < t2, t2 <= w < t3, w >= t3.  Being counter based, the
 * result does not depend on the thread count or the platform.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct {
    uint32_t *src, *dst;
    uint64_t begin, end, key;
    int scale;
    uint32_t t1, t2, t3;
} job_t;

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    for (uint64_t e = j->begin; e < j->end; ++e) {
        uint32_t u = 0, v = 0;
        uint64_t word = 0;
        for (int l = 0; l < j->scale; ++l) {
            if ((l & 1) == 0) word = mix64(j->key + (e * 32u + (uint64_t)(l >> 1)) * GOLDEN);
            uint32_t w = (l & 1) ? (uint32_t)(word >> 32) : (uint32_t)word;
            uint32_t ub = w >= j->t2;
            uint32_t vb = (w >= j->t1 && w < j->t2) || (w >= j->t3);
            u = (u << 1) | ub;
            v = (v << 1) | vb;
        }
        j->src[e] = u;
        j->dst[e] = v;
    }
    return NULL;
}

int rmat_fill(uint32_t *src, uint32_t *dst, uint64_t m, int scale, uint64_t seed,
              uint32_t t1, uint32_t t2, uint32_t t3, int nthreads) {
    if (scale < 1 || scale > 31 || nthreads < 1) return 1;
    if (nthreads > 256) nthreads = 256;
    uint64_t key = mix64(seed + GOLDEN);
    pthread_t th[256];
    int live[256];
    job_t jobs[256];
    uint64_t per = (m + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t b = per * (uint64_t)t, e = b + per;
        if (b > m) b = m;
        if (e > m) e = m;
        jobs[t] = (job_t){src, dst, b, e, key, scale, t1, t2, t3};
        live[t] = pthread_create(&th[t], NULL, worker, &jobs[t]) == 0;
        if (!live[t]) worker(&jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        if (live[t]) pthread_join(th[t], NULL);
    return 0;
}
