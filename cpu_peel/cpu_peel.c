/*
 * Parallel CPU comparison for the benchmark (not the oracle, not the product
 * path): a level-synchronous peel (the Peel paradigm of Sec. III) over all
 * host cores with OpenMP. It reports what a multicore CPU does on the same
 * graphs; its results are checked against the oracle.
 *
 * Level k: every residual vertex whose residual degree is <= k is peeled at
 * k; peeling v decrements the residual degree of each residual neighbour u
 * with an atomic fetch-and-subtract, and the thread whose decrement takes u
 * from k + 1 to k peels u in the same level (the next wave). A decrement can
 * only undershoot k on a vertex already peeled at k, so the level ends by
 * writing k back to every vertex it peeled. Empty levels are skipped: k jumps
 * to the smallest residual degree.
 *
 * int64 offsets, int32 neighbour ids, n < 2^31. Returns 0, or -1 when memory
 * runs out.
 */
#include <limits.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

int cpu_peel_threads(void) { return omp_get_max_threads(); }

int cpu_peel_coreness(const int64_t *rp, const int32_t *ci, int64_t n, int32_t *core)
{
    const size_t cap = (size_t)(n > 0 ? n : 1);
    int32_t *res = malloc(sizeof(int32_t) * cap);      /* residual vertices */
    int32_t *res2 = malloc(sizeof(int32_t) * cap);
    int32_t *wave = malloc(sizeof(int32_t) * cap);     /* the current wave */
    int32_t *nextw = malloc(sizeof(int32_t) * cap);    /* the wave it appends */
    int32_t *peeled = malloc(sizeof(int32_t) * cap);   /* every vertex of the level */
    unsigned char *gone = calloc(cap, 1);
    if (!res || !res2 || !wave || !nextw || !peeled || !gone) {
        free(res); free(res2); free(wave); free(nextw); free(peeled); free(gone);
        return -1;
    }
    int64_t nres = 0;
    for (int64_t v = 0; v < n; ++v) {
        core[v] = (int32_t)(rp[v + 1] - rp[v]);
        if (core[v] > 0) res[nres++] = (int32_t)v;
        else gone[v] = 1;
    }
    int64_t k = 0;
    while (nres > 0) {
        int32_t mn = INT_MAX;
#pragma omp parallel for reduction(min : mn) schedule(static)
        for (int64_t i = 0; i < nres; ++i) {
            const int32_t c = core[res[i]];
            if (c < mn) mn = c;
        }
        if (mn > k) k = mn;
        /* first wave: the residual vertices at or below k */
        int64_t ncur = 0;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < nres; ++i) {
            const int32_t v = res[i];
            if (core[v] <= k) {
                gone[v] = 1;
                int64_t pos;
#pragma omp atomic capture
                pos = ncur++;
                wave[pos] = v;
            }
        }
        memcpy(peeled, wave, sizeof(int32_t) * (size_t)ncur);
        int64_t total = ncur;
        while (ncur > 0) {
            int64_t nn = 0;
#pragma omp parallel for schedule(dynamic, 64)
            for (int64_t i = 0; i < ncur; ++i) {
                const int32_t v = wave[i];
                for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                    const int32_t u = ci[e];
                    if (__atomic_load_n(&gone[u], __ATOMIC_RELAXED)) continue;
                    if (__atomic_load_n(&core[u], __ATOMIC_RELAXED) <= k) continue;
                    const int32_t old = __atomic_fetch_sub(&core[u], 1, __ATOMIC_RELAXED);
                    if (old == k + 1) {   /* this decrement took u to k: peel it now */
                        __atomic_store_n(&gone[u], 1, __ATOMIC_RELAXED);
                        int64_t pos;
#pragma omp atomic capture
                        pos = nn++;
                        nextw[pos] = u;
                    }
                }
            }
            memcpy(peeled + total, nextw, sizeof(int32_t) * (size_t)nn);
            total += nn;
            int32_t *t = wave;
            wave = nextw;
            nextw = t;
            ncur = nn;
        }
        /* undershoots are repaired: every vertex peeled in this level has coreness k */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < total; ++i) core[peeled[i]] = (int32_t)k;
        int64_t nk = 0;
        for (int64_t i = 0; i < nres; ++i)
            if (!gone[res[i]]) res2[nk++] = res[i];
        int32_t *t = res;
        res = res2;
        res2 = t;
        nres = nk;
    }
    free(res); free(res2); free(wave); free(nextw); free(peeled); free(gone);
    return 0;
}
