/*
 * CPU oracle for k-core decomposition -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. It shares no code, header or helper with the CUDA path.
 *
 * Problem (Sec. I): the k-core of G is the maximal subgraph in which every
 * vertex has degree >= k; core(v) is the largest k such that v lies in the
 * k-core; an isolated vertex has core 0.
 *
 * Contents
 *   oracle_bz            Batagelj-Zaversnik O(n + m) bucket peel (Sec. VI,
 *                        "In-Memory Setting"): vertices kept sorted by current
 *                        degree in `vert`, with `bin` (bucket starts) and
 *                        `pos` (index of each vertex in `vert`).
 *   oracle_bz_batched    the same, graph by graph, over a packed batch.
 *   oracle_hindex_jacobi Index2core paradigm (Alg. 2) run synchronously: every
 *                        round sets core[v] <- HINDEX(core[nbr(v)]) from the
 *                        previous round's values, until nothing changes.
 *   oracle_peelone       Alg. 4 (PeelOne) run sequentially, with the dynamic
 *                        frontier processed in waves; counts levels and waves.
 *   oracle_histocore     Alg. 6 (HistoCore) run sequentially round by round,
 *                        with an optional check of the histogram invariant.
 *   oracle_gpp           Alg. 3 (General Parallel Peel, the baseline of
 *                        Sec. V) run in its synchronous scan/scatter steps.
 *   oracle_nbrcore       NbrCore and CntCore (Alg. 5), the Index2core
 *   oracle_cntcore       baselines of Sec. IV-A and V, run synchronously.
 *   oracle_check         fixpoint and certificate checks of a coreness vector.
 *
 * Graphs are CSR: row_ptr (int64, n + 1 entries), col_idx (int32, row_ptr[n]
 * entries), simple and symmetric. Every function returns 0 on success and a
 * negative value when it cannot allocate its scratch memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DEG(rp, v) ((int32_t)((rp)[(v) + 1] - (rp)[(v)]))

/* ------------------------------------------------------------------------ */
/* Batagelj-Zaversnik                                                        */
/* ------------------------------------------------------------------------ */

int oracle_bz(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *deg)
{
    if (n <= 0) return 0;
    int32_t md = 0;
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = DEG(rp, v);
        if (deg[v] > md) md = deg[v];
    }
    int64_t *bin = (int64_t *)calloc((size_t)md + 1, sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *vert = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!bin || !pos || !vert) { free(bin); free(pos); free(vert); return -1; }

    /* counting sort by degree: bin[d] becomes the first index of bucket d */
    for (int64_t v = 0; v < n; ++v) bin[deg[v]]++;
    int64_t start = 0;
    for (int32_t d = 0; d <= md; ++d) {
        int64_t num = bin[d];
        bin[d] = start;
        start += num;
    }
    for (int64_t v = 0; v < n; ++v) {
        pos[v] = bin[deg[v]];
        vert[pos[v]] = (int32_t)v;
        bin[deg[v]]++;
    }
    for (int32_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
    bin[0] = 0;

    /* peel in order of current degree; a neighbour with a larger current
       degree moves to the front of its bucket and the bucket boundary moves
       past it, which drops its degree by one */
    for (int64_t i = 0; i < n; ++i) {
        int32_t v = vert[i];
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t u = ci[e];
            if (deg[u] > deg[v]) {
                int32_t du = deg[u];
                int64_t pu = pos[u];
                int64_t pw = bin[du];
                int32_t w = vert[pw];
                if (u != w) {
                    pos[u] = pw; vert[pu] = w;
                    pos[w] = pu; vert[pw] = u;
                }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    free(bin); free(pos); free(vert);
    return 0;
}

/* Packed batch: graph g has n_g = vtx_off[g+1] - vtx_off[g] vertices; its
   graph-local int32 row_ptr (n_g + 1 entries) starts at row_ptr + vtx_off[g] + g;
   its graph-local col_idx starts at col_idx + arc_off[g]. */
int oracle_bz_batched(int64_t G, const int64_t *vtx_off, const int64_t *arc_off,
                      const int32_t *row_ptr, const int32_t *col_idx, int32_t *core)
{
    int64_t maxn = 0;
    for (int64_t g = 0; g < G; ++g) {
        int64_t ng = vtx_off[g + 1] - vtx_off[g];
        if (ng > maxn) maxn = ng;
    }
    int64_t *rp = (int64_t *)malloc((size_t)(maxn + 1) * sizeof(int64_t));
    if (!rp) return -1;
    for (int64_t g = 0; g < G; ++g) {
        int64_t ng = vtx_off[g + 1] - vtx_off[g];
        const int32_t *lrp = row_ptr + vtx_off[g] + g;
        for (int64_t v = 0; v <= ng; ++v) rp[v] = lrp[v];
        int rc = oracle_bz(ng, rp, col_idx + arc_off[g], core + vtx_off[g]);
        if (rc) { free(rp); return rc; }
    }
    free(rp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* HINDEX (Alg. 2): the largest h such that at least h of the values are >= h.
   Values are clipped to `cap` (the h-index of d values never exceeds d).
   `cnt` must hold cap + 1 entries.                                          */
/* ------------------------------------------------------------------------ */
static int32_t hindex_of(const int64_t *rp, const int32_t *ci, const int32_t *val,
                         int64_t v, int32_t cap, int64_t *cnt)
{
    for (int32_t i = 0; i <= cap; ++i) cnt[i] = 0;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        int32_t x = val[ci[e]];
        cnt[x < cap ? x : cap]++;
    }
    int64_t s = 0;
    int32_t h = cap;
    for (; h > 0; --h) {
        s += cnt[h];
        if (s >= h) break;
    }
    return h;
}

int oracle_hindex_jacobi(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
                         int64_t *rounds_out)
{
    int64_t rounds = 0;
    if (n <= 0) { if (rounds_out) *rounds_out = 0; return 0; }
    int32_t md = 0;
    for (int64_t v = 0; v < n; ++v) {
        core[v] = DEG(rp, v);
        if (core[v] > md) md = core[v];
    }
    int32_t *nxt = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *cnt = (int64_t *)malloc(((size_t)md + 2) * sizeof(int64_t));
    if (!nxt || !cnt) { free(nxt); free(cnt); return -1; }
    for (;;) {
        int64_t changed = 0;
        for (int64_t v = 0; v < n; ++v) {
            int32_t h = hindex_of(rp, ci, core, v, DEG(rp, v), cnt);
            nxt[v] = h;
            changed += (h != core[v]);
        }
        if (!changed) break;
        ++rounds;
        memcpy(core, nxt, (size_t)n * sizeof(int32_t));
    }
    free(nxt); free(cnt);
    if (rounds_out) *rounds_out = rounds;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 4, PeelOne, sequential. core starts at the degree. Level k takes the
   residual vertices with core == k as its frontier; removing a frontier
   vertex lowers every residual neighbour with core > k by one, and a
   neighbour that reaches k joins the frontier of the same level (the dynamic
   frontier). Levels with no vertex are skipped (k jumps to the smallest
   residual value); the frontier of a level is processed in waves, wave w+1
   being the vertices that reached k during wave w.
   stats[0] = non-empty levels, stats[1] = largest k, stats[2] = waves,
   stats[3] = decrements applied, stats[4] = arcs scanned from frontiers.  */
/* ------------------------------------------------------------------------ */
int oracle_peelone(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
                   int64_t *stats)
{
    int64_t st[5] = {0, 0, 0, 0, 0};
    int32_t *res = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *q = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!res || !q) { free(res); free(q); return -1; }
    int64_t nres = 0;
    for (int64_t v = 0; v < n; ++v) {
        core[v] = DEG(rp, v);
        if (core[v] > 0) res[nres++] = (int32_t)v;
    }
    int64_t qtail = 0;
    int32_t k = 0;
    while (nres > 0) {
        /* scan: smallest residual value, then the frontier */
        int32_t kmin = INT32_MAX;
        for (int64_t i = 0; i < nres; ++i)
            if (core[res[i]] < kmin) kmin = core[res[i]];
        k = kmin;
        int64_t qhead = qtail, keep = 0;
        for (int64_t i = 0; i < nres; ++i) {
            int32_t v = res[i];
            if (core[v] == k) q[qtail++] = v;
            else res[keep++] = v;
        }
        nres = keep;
        st[0]++;
        /* scatter, wave by wave */
        while (qhead < qtail) {
            int64_t wave_end = qtail;
            st[2]++;
            for (; qhead < wave_end; ++qhead) {
                int32_t v = q[qhead];
                st[4] += DEG(rp, v);
                for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                    int32_t u = ci[e];
                    if (core[u] > k) {
                        core[u] -= 1;          /* never below k, since core[u] > k */
                        st[3]++;
                        if (core[u] == k) q[qtail++] = u;
                    }
                }
            }
        }
        /* drop the vertices that joined this level from the residual list */
        keep = 0;
        for (int64_t i = 0; i < nres; ++i)
            if (core[res[i]] > k) res[keep++] = res[i];
        nres = keep;
    }
    st[1] = k;
    free(res); free(q);
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 6, HistoCore, sequential and round-synchronous.
   histo[v][s] for s = 1..deg(v) is stored at histo[rp[v] + s - 1].
   InitHisto: histo[v][min(deg u, deg v)] += 1 for every arc (v, u).
   V_cnt: vertices whose count in slot core[v] is below core[v].
   SumHisto(v): sum the slots from core_old down to the first k with
     sum >= k; core[v] <- k, oldcore[v] <- core_old, histo[v][k] <- sum.
   UpdateHisto(v) for each neighbour u with core[u] > core[v]: remove v from
     slot min(oldcore[v], core[u]) and add it to slot core[v]; u joins the
     next V_cnt when oldcore[v] >= core[u] and that slot held exactly core[u].
   stats[0] = rounds, stats[1] = frontier vertices summed over rounds,
   stats[2] = slots read by SumHisto, stats[3] = arcs scanned by UpdateHisto,
   stats[4] = neighbour updates (pairs of histogram edits),
   stats[5] = invariant violations seen (0 when all checks pass).
   check = 1 verifies the histogram invariant and V_cnt after every round
   (O(m) per round; for small graphs).                                      */
/* ------------------------------------------------------------------------ */
static int64_t histo_invariant_violations(int64_t n, const int64_t *rp, const int32_t *ci,
                                          const int32_t *core, const int32_t *histo,
                                          const uint8_t *in_next, int64_t *cnt)
{
    int64_t bad = 0;
    for (int64_t v = 0; v < n; ++v) {
        int32_t d = DEG(rp, v), K = core[v];
        if (d == 0) { bad += (K != 0); continue; }
        if (K < 1 || K > d) { bad++; continue; }
        for (int32_t i = 0; i <= K; ++i) cnt[i] = 0;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t x = core[ci[e]];
            cnt[x < K ? x : K]++;
        }
        for (int32_t i = 1; i <= K; ++i) bad += (histo[rp[v] + i - 1] != cnt[i]);
        int below = histo[rp[v] + K - 1] < K;
        bad += (below != (int)in_next[v]);
    }
    return bad;
}

int oracle_histocore(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
                     int64_t *stats, int check)
{
    int64_t st[6] = {0, 0, 0, 0, 0, 0};
    int64_t A = n > 0 ? rp[n] : 0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *histo = (int32_t *)calloc((size_t)(A > 0 ? A : 1), sizeof(int32_t));
    int32_t *oldcore = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc(nn * sizeof(int32_t));
    uint8_t *mark = (uint8_t *)calloc(nn, 1);
    int32_t md = 0;
    for (int64_t v = 0; v < n; ++v) {
        core[v] = DEG(rp, v);
        if (core[v] > md) md = core[v];
    }
    int64_t *cnt = (int64_t *)malloc(((size_t)md + 2) * sizeof(int64_t));
    if (!histo || !oldcore || !cur || !nxt || !mark || !cnt) {
        free(histo); free(oldcore); free(cur); free(nxt); free(mark); free(cnt);
        return -1;
    }
    /* InitHisto */
    for (int64_t v = 0; v < n; ++v) {
        int32_t dv = core[v];
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t du = core[ci[e]];
            histo[rp[v] + (du < dv ? du : dv) - 1] += 1;
        }
    }
    int64_t ncur = 0;
    for (int64_t v = 0; v < n; ++v) {
        int32_t d = core[v];
        if (d >= 1 && histo[rp[v] + d - 1] < d) { cur[ncur++] = (int32_t)v; mark[v] = 1; }
    }
    if (check) st[5] += histo_invariant_violations(n, rp, ci, core, histo, mark, cnt);

    while (ncur > 0) {
        st[0]++;
        st[1] += ncur;
        for (int64_t i = 0; i < ncur; ++i) mark[cur[i]] = 0;
        /* SumHisto: every frontier vertex changes (Thm. 2) */
        for (int64_t i = 0; i < ncur; ++i) {
            int32_t v = cur[i];
            int32_t K = core[v], k = K;
            int64_t sum = 0;
            for (; k >= 1; --k) {
                sum += histo[rp[v] + k - 1];
                st[2]++;
                if (sum >= k) break;
            }
            if (k == K || k < 1) { st[5]++; continue; }
            core[v] = k;
            oldcore[v] = K;
            histo[rp[v] + k - 1] = (int32_t)sum;
        }
        /* UpdateHisto */
        int64_t nnext = 0;
        for (int64_t i = 0; i < ncur; ++i) {
            int32_t v = cur[i];
            int32_t x = oldcore[v], y = core[v];
            st[3] += DEG(rp, v);
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                int32_t u = ci[e];
                int32_t K = core[u];
                if (K > y) {
                    int32_t *slot = &histo[rp[u] + (x < K ? x : K) - 1];
                    int32_t old = *slot;
                    *slot = old - 1;
                    histo[rp[u] + y - 1] += 1;
                    st[4]++;
                    if (x >= K && old == K) {
                        if (mark[u]) st[5]++;           /* pushed twice */
                        mark[u] = 1;
                        nxt[nnext++] = u;
                    }
                }
            }
        }
        int32_t *t = cur; cur = nxt; nxt = t;
        ncur = nnext;
        if (check) st[5] += histo_invariant_violations(n, rp, ci, core, histo, mark, cnt);
    }
    free(histo); free(oldcore); free(cur); free(nxt); free(mark); free(cnt);
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3, General Parallel Peel, run sequentially in its synchronous form.
   deg[] (residual degree) and rem[] (removed flag) are separate arrays;
   core[] receives the level at which a vertex is removed. Each step scans
   every vertex for the frontier {v : !rem[v], deg[v] <= k}; an empty scan
   raises k by one; otherwise the frontier gets core = k and rem = 1, and the
   scatter lowers deg[u] of every non-removed neighbour u by one. Isolated
   vertices leave at k = 0.
   stats[0] = scatter steps (scans with a non-empty frontier),
   stats[1] = scans (including the empty ones that raise k),
   stats[2] = decrements, stats[3] = arcs scanned from frontiers,
   stats[4] = largest k that removed a vertex.                              */
/* ------------------------------------------------------------------------ */
int oracle_gpp(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
               int64_t *stats)
{
    int64_t st[5] = {0, 0, 0, 0, 0};
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *deg = (int32_t *)malloc(nn * sizeof(int32_t));
    uint8_t *rem = (uint8_t *)calloc(nn, 1);
    int32_t *front = (int32_t *)malloc(nn * sizeof(int32_t));
    if (!deg || !rem || !front) { free(deg); free(rem); free(front); return -1; }
    for (int64_t v = 0; v < n; ++v) deg[v] = DEG(rp, v);
    int64_t nres = n;
    int32_t k = 0;
    while (nres > 0) {
        st[1]++;
        int64_t nf = 0;
        for (int64_t v = 0; v < n; ++v)
            if (!rem[v] && deg[v] <= k) front[nf++] = (int32_t)v;
        if (nf == 0) { k++; continue; }
        for (int64_t i = 0; i < nf; ++i) {
            core[front[i]] = k;
            rem[front[i]] = 1;
        }
        nres -= nf;
        st[0]++;
        st[4] = k;
        for (int64_t i = 0; i < nf; ++i) {
            int32_t v = front[i];
            st[3] += DEG(rp, v);
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
                if (!rem[ci[e]]) { deg[ci[e]]--; st[2]++; }
        }
    }
    free(deg); free(rem); free(front);
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The Index2core variants of Sec. IV-A and the evaluation, run
   synchronously (every round reads the previous round's estimates).
   Estimates start at the degree. The active set starts as every vertex of
   degree >= 1.
   nbrcore (NbrCore): every active vertex recomputes HINDEX of its
     neighbours' estimates; the vertices whose estimate fell form C, and the
     next active set is the union of their neighbourhoods.
   cntcore (CntCore, Alg. 5): every active vertex counts cnt = the neighbours
     whose estimate is >= its own; the frontier is {cnt < estimate}, whose
     vertices recompute HINDEX (they all fall, by Thm. 2; a frontier vertex
     that keeps its estimate counts as a violation). The next active set is
     the union of the frontier's neighbourhoods.
   Both stop after a round in which no estimate changes (for CntCore, by
   Thm. 2, a round whose frontier is empty).
   stats[0] = rounds that changed an estimate, stats[1] = sum of active-set
   sizes over all rounds executed, stats[2] = sum of the changed (NbrCore)
   or frontier (CntCore) sizes, stats[3] = arcs scanned (HINDEX and cnt each
   read the whole adjacency), stats[4] = violations.                        */
/* ------------------------------------------------------------------------ */
static int index2core_sync(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
                           int64_t *stats, int use_cnt)
{
    int64_t st[5] = {0, 0, 0, 0, 0};
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t md = 0;
    for (int64_t v = 0; v < n; ++v) {
        core[v] = DEG(rp, v);
        if (core[v] > md) md = core[v];
    }
    int32_t *act = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *chg = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *newv = (int32_t *)malloc(nn * sizeof(int32_t));
    uint8_t *mark = (uint8_t *)calloc(nn, 1);
    int64_t *cnt = (int64_t *)malloc(((size_t)md + 2) * sizeof(int64_t));
    if (!act || !nxt || !chg || !newv || !mark || !cnt) {
        free(act); free(nxt); free(chg); free(newv); free(mark); free(cnt);
        return -1;
    }
    int64_t nact = 0;
    for (int64_t v = 0; v < n; ++v)
        if (DEG(rp, v) > 0) act[nact++] = (int32_t)v;
    while (nact > 0) {
        st[1] += nact;
        int64_t nchg = 0, nfront = 0;
        for (int64_t i = 0; i < nact; ++i) {
            int32_t v = act[i], d = DEG(rp, v);
            if (use_cnt) {
                int64_t c = 0;
                for (int64_t e = rp[v]; e < rp[v + 1]; ++e) c += (core[ci[e]] >= core[v]);
                st[3] += d;
                if (c >= core[v]) continue;   /* not in the frontier */
            }
            int32_t h = hindex_of(rp, ci, core, v, core[v] < d ? core[v] : d, cnt);
            st[3] += d;
            if (use_cnt) nfront++;
            if (h < core[v]) {
                chg[nchg] = v;
                newv[nchg++] = h;
            } else if (use_cnt) {
                st[4]++;   /* a frontier vertex that kept its estimate */
            }
        }
        st[2] += use_cnt ? nfront : nchg;
        if (nchg == 0) break;
        st[0]++;
        /* apply after every vertex of the round has read the old estimates */
        for (int64_t i = 0; i < nchg; ++i) core[chg[i]] = newv[i];
        int64_t nn2 = 0;
        for (int64_t i = 0; i < nchg; ++i) {
            int32_t v = chg[i];
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
                if (!mark[ci[e]]) { mark[ci[e]] = 1; nxt[nn2++] = ci[e]; }
        }
        for (int64_t i = 0; i < nn2; ++i) mark[nxt[i]] = 0;
        int32_t *t = act; act = nxt; nxt = t;
        nact = nn2;
    }
    free(act); free(nxt); free(chg); free(newv); free(mark); free(cnt);
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
}

int oracle_nbrcore(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
                   int64_t *stats)
{
    return index2core_sync(n, rp, ci, core, stats, 0);
}

int oracle_cntcore(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core,
                   int64_t *stats)
{
    return index2core_sync(n, rp, ci, core, stats, 1);
}

/* ------------------------------------------------------------------------ */
/* Checks of a coreness vector (necessary conditions, O(m)):
   out[0] = vertices with core < 0 or core > deg
   out[1] = vertices whose certificate fails: fewer than core[v] neighbours
            u with core[u] >= core[v] (a valid certificate for every v means
            core is a lower bound of the true coreness)
   out[2] = vertices where core[v] != HINDEX(core[nbr(v)]) (Alg. 2 fixpoint) */
/* ------------------------------------------------------------------------ */
int oracle_check(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *core,
                 int64_t *out)
{
    out[0] = out[1] = out[2] = 0;
    int32_t md = 0;
    for (int64_t v = 0; v < n; ++v) if (DEG(rp, v) > md) md = DEG(rp, v);
    int64_t *cnt = (int64_t *)malloc(((size_t)md + 2) * sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t v = 0; v < n; ++v) {
        int32_t d = DEG(rp, v), c = core[v];
        if (c < 0 || c > d) { out[0]++; continue; }
        int64_t ge = 0;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) ge += (core[ci[e]] >= c);
        if (ge < c) out[1]++;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
            if (core[ci[e]] < 0) { out[2]++; goto next; }   /* HINDEX needs values >= 0 */
        if (hindex_of(rp, ci, core, v, d, cnt) != c) out[2]++;
    next:;
    }
    free(cnt);
    return 0;
}
