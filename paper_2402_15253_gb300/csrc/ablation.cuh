// The baselines the paper compares its methods with (Sec. V), built on the
// same persistent-kernel runtime (grid barrier, degree-class expansion) so
// that a comparison isolates the algorithmic difference:
//
//   gpp::run  General Parallel Peel (Alg. 3): a residual-degree array deg[]
//             and a removed flag rem[] kept apart from core[]; each step scans
//             every vertex for {!rem, deg <= k}, an empty scan raises k by one,
//             and the scatter lowers deg[u] of every non-removed neighbour
//             (no dynamic frontier, no level skipping).
//   i2c::run  the Index2core baselines, synchronous rounds from estimates equal
//             to the degrees. NbrCore: every active vertex recomputes HINDEX
//             (Alg. 2) of its neighbours' estimates; CntCore (Alg. 5): an
//             active vertex first counts cnt = its neighbours with an estimate
//             >= its own, and only the frontier {cnt < estimate} (Thm. 2)
//             recomputes HINDEX. HINDEX is built the way Sec. IV-A describes,
//             with no histogram kept between rounds: Step I fills a histogram
//             row of the vertex from its whole adjacency, Step II sums it from
//             the estimate downwards (and clears it). The next active set is
//             the union of the neighbourhoods of the vertices that changed.
//
// Vertex lists are kept in two parts, as elsewhere: vertices of degree <=
// small_deg in a plain list, larger ones as (vertex, chunk) entries.
#pragma once

#include "pico_device.cuh"

namespace pico {

// Appends v (degree d) to a split vertex list, warp-cooperatively: every lane
// of the warp calls; lanes with `pred` append.
__device__ __forceinline__ void warp_append_vertex(bool pred, int v, long long d, int *sl,
                                                   unsigned *sc, unsigned scap, int2 *bl,
                                                   unsigned *bc, unsigned bcap, Ctrl *ctl,
                                                   const Tuning &tn)
{
    const bool small = pred && d <= tn.small_deg;
    const unsigned pos = warp_push(sc, small);
    if (small) {
        if (pos < scap) sl[pos] = v;
        else set_error(ctl, kErrNotConverged);
    }
    warp_push_chunks(pred && !small, v, d, bl, bc, bcap, ctl, tn.chunk);
}

namespace gpp {

// live counters of three consecutive scans (slot = scan index mod 3): a
// scan resets the next scan's slot, which nobody touches until then
enum : int { L_QS = 0 /* 0..2 */, L_QB = 3 /* 3..5 */, L_RES = 6 /* 6..8 */ };

template <typename Off>
struct Params {
    const Off *rp;
    const int *ci;
    long long n;
    int *core;                 // output: the level at which a vertex is removed
    int *deg;                  // residual degree
    unsigned char *rem;        // removed flag
    int *qs;                   // frontier: small vertices (n slots)
    int2 *qb;                  // frontier: chunks of large vertices
    unsigned qb_cap;
    Ctrl *ctl;
    Tuning tn;
};

// scatter: every non-removed neighbour loses one unit of residual degree
template <typename Off>
struct ScatterArc {
    static constexpr int kArcs = 4;
    const unsigned char *rem;
    int *deg;
    unsigned long long n_arcs = 0, n_atomics = 0;
    __device__ __forceinline__ bool item(int, int &, int &) { return true; }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&)[kArcs], const int (&)[kArcs])
    {
        unsigned char r[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) r[j] = valid[j] ? __ldcg(rem + u[j]) : (unsigned char)1;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            n_arcs += valid[j];
            if (!r[j]) {
                red_add(deg + u[j], -1);
                ++n_atomics;
            }
        }
    }
};

template <typename Off, typename Dom>
__device__ void run(const Params<Off> &p, Dom &dom, unsigned *s_tmp, unsigned long long *st,
                    unsigned long long &arcs, unsigned long long &atomics)
{
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const long long n = p.n;
    const long long first = (long long)dom.cta() * blockDim.x;

    for (long long v = first + threadIdx.x; v < n; v += nthreads) {
        p.deg[v] = (int)(p.rp[v + 1] - p.rp[v]);
        p.rem[v] = 0;
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];

    int k = 0;
    long long nres = n;
    unsigned slot = 0;
    const long long max_scans = n + p.rp[n] + 2;   // each scan removes a vertex or raises k
    for (long long scans = 1; nres > 0; ++scans) {
        if (scans > max_scans) {
            if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
            return;
        }
        if (dom.leader()) {
            const unsigned nx = (slot + 1) % 3;
            live[L_QS + nx] = 0;
            live[L_QB + nx] = 0;
            live[L_RES + nx] = 0;
        }
        // scan every vertex for the frontier {!rem, deg <= k}
        for (long long base = first; base < n; base += nthreads) {
            const long long v = base + threadIdx.x;
            bool front = false, keep = false;
            long long d = 0;
            if (v < n && !__ldcg(p.rem + v)) {
                if (ldcg(p.deg + v) <= k) {
                    front = true;
                    p.core[v] = k;
                    p.rem[v] = 1;
                    d = (long long)(p.rp[v + 1] - p.rp[v]);
                } else {
                    keep = true;
                }
            }
            const bool small = front && d <= p.tn.small_deg;
            unsigned pos, unused;
            block_push2(small, keep, &live[L_QS + slot], &live[L_RES + slot], pos, unused, s_tmp);
            if (small) p.qs[pos] = (int)v;   // at most n frontier vertices in a step
            warp_push_chunks(front && !small, (int)v, d, p.qb, &live[L_QB + slot], p.qb_cap, ctl,
                             p.tn.chunk);
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) {
            ++st[kStBarriers];
            ++st[kStScans];
        }
        const unsigned nqs = snap[L_QS + slot], nqb = snap[L_QB + slot];
        nres = (long long)snap[L_RES + slot];
        slot = (slot + 1) % 3;
        if (nqs + nqb == 0) {   // no vertex with deg <= k: next k
            ++k;
            continue;
        }
        if (threadIdx.x == 0) {
            ++st[kStSubrounds];
            if ((unsigned long long)k > st[kStKmax]) st[kStKmax] = (unsigned long long)k;
        }
        ScatterArc<Off> f{p.rem, p.deg};
        expand(p.rp, p.ci, p.qs, nqs, p.qb, nqb, gwarp, nwarps, f, p.tn,
               batch_width(nqs, nqb, nwarps));
        arcs += f.n_arcs;
        atomics += f.n_atomics;
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
    }
}

}  // namespace gpp

namespace i2c {

// live counters: active lists per round parity (small, chunks), frontier
// lists, changed lists, and vertex counts of the active, frontier and
// changed sets
enum : int {
    L_AS = 0, L_AB = 1, /* parity 1: 2, 3 */ L_FS = 4, L_FB = 5, L_CS = 6, L_CB = 7,
    L_NACT = 8 /* parity 1: 9 */, L_NFRONT = 10, L_NCHG = 11
};

template <typename Off>
struct Params {
    const Off *rp;
    const int *ci;
    long long n, m;
    int *core;                 // output
    int *est;                  // estimates (the previous round's during a round)
    int *newv;                 // new estimate of a changed vertex
    int *cnt;                  // CntCore: cnt of an active vertex (0 at rest)
    int *stamp;                // round + 1 in which a vertex was last made active
    int *hist;                 // histogram rows, shaped like col_idx (0 at rest)
    int *as[2], *fs, *cs;      // small parts of the active, frontier, changed lists
    int2 *ab[2], *fb, *cb;     // chunk parts
    unsigned cap;              // entries of each chunk list
    Ctrl *ctl;
    Tuning tn;
};

// CntCore: cnt[v] += |{arcs (v, u) : est[u] >= est[v]}|
template <typename Off>
struct CntArc {
    static constexpr int kArcs = 4;
    const int *est;
    int *cnt;
    unsigned long long n_arcs = 0, n_atomics = 0;
    __device__ __forceinline__ bool item(int v, int &a, int &)
    {
        a = ldcg(est + v);
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&vo)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&a)[kArcs], const int (&)[kArcs])
    {
        int e[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) e[j] = valid[j] ? ldcg(est + u[j]) : -1;
        // a chunk of one vertex (every lane's arcs belong to it): one add per warp
        const bool one = __all_sync(kFull, vo[0] == __shfl_sync(kFull, vo[0], 0) &&
                                               vo[kArcs - 1] == vo[0]);
        int mine = 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            n_arcs += valid[j];
            const bool ge = valid[j] && e[j] >= a[j];
            if (one) {
                mine += ge;
            } else if (ge) {
                red_add(cnt + vo[j], 1);
                ++n_atomics;
            }
        }
        if (one) {
            const int tot = __reduce_add_sync(kFull, mine);
            if ((threadIdx.x & 31) == 0 && tot) {
                red_add(cnt + vo[0], tot);
                ++n_atomics;
            }
        }
    }
};

// Step I of HINDEX: hist[v][min(est[u], est[v])] += 1 over v's adjacency
template <typename Off>
struct HistArc {
    static constexpr int kArcs = 4;
    const int *est;
    int *hist;
    unsigned long long n_arcs = 0, n_atomics = 0;
    __device__ __forceinline__ bool item(int v, int &a, int &)
    {
        a = ldcg(est + v);
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&rs)[kArcs],
                                         const int (&K)[kArcs], const int (&)[kArcs])
    {
        int e[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) e[j] = valid[j] ? ldcg(est + u[j]) : 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            n_arcs += valid[j];
            // slot min(e, K); a 0 would support no h >= 1
            const int s = e[j] < K[j] ? e[j] : K[j];
            if (valid[j] && s > 0) {
                ++n_atomics;
                red_add(hist + rs[j] + s - 1, 1);
            }
        }
    }
};

// Next active set: every neighbour of a changed vertex, once per round
template <typename Off>
struct ActArc {
    static constexpr int kArcs = 4;
    const Off *rp;
    int *stamp;
    int mark;                  // round + 1
    int *as;
    int2 *ab;
    unsigned *c_as, *c_ab, *c_nact;   // counters of the next round's lists
    unsigned n, cap;
    Ctrl *ctl;
    Tuning tn;
    __device__ __forceinline__ bool item(int, int &, int &) { return true; }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&)[kArcs], const int (&)[kArcs])
    {
        bool fresh[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            fresh[j] = valid[j] && ldcg(stamp + u[j]) != mark && atomicExch(stamp + u[j], mark) != mark;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            const long long d = fresh[j] ? (long long)(rp[u[j] + 1] - rp[u[j]]) : 0;
            warp_append_vertex(fresh[j], u[j], d, as, c_as, n, ab, c_ab, cap, ctl, tn);
            const unsigned c = __popc(__ballot_sync(kFull, fresh[j]));
            if ((threadIdx.x & 31) == 0 && c) atomicAdd(c_nact, c);
        }
    }
};

// Calls fn(v, lane-uniform) for every vertex of a split list: each entry of
// the small part, and the first chunk entry of each large vertex. Small
// vertices go one per thread (fn_thread), large ones one per warp (fn_warp).
template <typename FT, typename FW>
__device__ __forceinline__ void for_vertices(const int *sl, unsigned ns, const int2 *bl,
                                             unsigned nb, unsigned tid, unsigned nthreads,
                                             unsigned gwarp, unsigned nwarps, FT fn_thread,
                                             FW fn_warp)
{
    for (unsigned base = tid - (tid & 31); base < ns; base += nthreads) {
        const unsigned i = base + (tid & 31);
        fn_thread(i < ns, i < ns ? ldcg(sl + i) : 0);
    }
    for (unsigned i = gwarp; i < nb; i += nwarps) {
        const int2 e = __ldcg(bl + i);
        if (e.y == 0) fn_warp(e.x);
    }
}

// Step II by one thread: sums hist[v] from K down to the first k with sum >= k,
// clears the row; returns k
template <typename Off>
__device__ __forceinline__ int hindex_thread(const Params<Off> &p, int v, int K)
{
    int *row = p.hist + p.rp[v];
    int sum = 0, h = 0;
    for (int k = K; k >= 1; --k) {
        sum += ldcg(row + k - 1);
        if (h == 0 && sum >= k) h = k;
        row[k - 1] = 0;
    }
    return h;
}

// Step II by one warp (32 slots per step), then the warp clears the row
template <typename Off>
__device__ __forceinline__ int hindex_warp(const Params<Off> &p, int v, int K)
{
    const int lane = threadIdx.x & 31;
    int *row = p.hist + p.rp[v];
    int carry = 0, h = 0;
    for (int top = K; top >= 1 && h == 0; top -= 32) {
        const int slot = top - lane;
        int inc = slot >= 1 ? ldcg(row + slot - 1) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const unsigned b = __ballot_sync(kFull, slot >= 1 && carry + inc >= slot);
        if (b) h = __shfl_sync(kFull, slot, __ffs(b) - 1);
        carry = __shfl_sync(kFull, carry + inc, 31);
    }
    for (int s = lane; s < K; s += 32) row[s] = 0;
    return h;
}

template <typename Off, typename Dom, bool UseCnt>
__device__ void run(const Params<Off> &p, Dom &dom, unsigned *s_tmp, unsigned long long *st,
                    unsigned long long &arcs, unsigned long long &atomics)
{
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const long long n = p.n;
    const long long first = (long long)dom.cta() * blockDim.x;

    // estimates = degrees; the first active set is every non-isolated vertex
    for (long long base = first; base < n; base += nthreads) {
        const long long v = base + threadIdx.x;
        long long d = 0;
        if (v < n) {
            d = (long long)(p.rp[v + 1] - p.rp[v]);
            p.est[v] = (int)d;
            p.stamp[v] = 0;
            if (UseCnt) p.cnt[v] = 0;
        }
        warp_append_vertex(d > 0, (int)v, d, p.as[0], &live[L_AS], (unsigned)n, p.ab[0],
                           &live[L_AB], p.cap, ctl, p.tn);
        const unsigned c = __popc(__ballot_sync(kFull, d > 0));
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&live[L_NACT], c);
    }
    for (long long i = first + threadIdx.x; i < p.m; i += nthreads) p.hist[i] = 0;
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    const long long max_rounds = p.m + 2;
    for (long long r = 0;; ++r) {
        const int par = (int)(r & 1), np = 1 - par;
        const unsigned nas = snap[2 * par + L_AS], nab = snap[2 * par + L_AB];
        const unsigned nact = snap[L_NACT + par];
        if (nas + nab == 0) break;
        if (r >= max_rounds) {
            if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
            return;
        }
        if (threadIdx.x == 0) st[kStActive] += nact;
        if (dom.leader()) {   // lists filled later in this round
            live[2 * np + L_AS] = 0;
            live[2 * np + L_AB] = 0;
            live[L_NACT + np] = 0;
            live[L_FS] = 0;
            live[L_FB] = 0;
            live[L_CS] = 0;
            live[L_CB] = 0;
            live[L_NFRONT] = 0;
            live[L_NCHG] = 0;
        }
        const int *fs = p.as[par];
        const int2 *fb = p.ab[par];
        unsigned nfs = nas, nfb = nab;
        if (UseCnt) {
            {
                CntArc<Off> f{p.est, p.cnt};
                expand(p.rp, p.ci, p.as[par], nas, p.ab[par], nab, gwarp, nwarps, f, p.tn,
                       batch_width(nas, nab, nwarps));
                arcs += f.n_arcs;
                atomics += f.n_atomics;
            }
            if (!dom.sync()) return;
            if (threadIdx.x == 0) ++st[kStBarriers];
            // frontier {cnt < estimate}; cnt back to 0
            auto front_thread = [&](bool ok, int v) {
                bool in = false;
                long long d = 0;
                if (ok) {
                    const int c = ldcg(p.cnt + v);
                    p.cnt[v] = 0;
                    in = c < ldcg(p.est + v);
                    d = (long long)(p.rp[v + 1] - p.rp[v]);
                }
                warp_append_vertex(in, v, d, p.fs, &live[L_FS], (unsigned)n, p.fb, &live[L_FB],
                                   p.cap, ctl, p.tn);
                const unsigned c = __popc(__ballot_sync(kFull, in));
                if ((threadIdx.x & 31) == 0 && c) atomicAdd(&live[L_NFRONT], c);
            };
            auto front_warp = [&](int v) {
                const int c = ldcg(p.cnt + v);
                const bool in = c < ldcg(p.est + v);
                __syncwarp();
                if ((threadIdx.x & 31) == 0) p.cnt[v] = 0;
                const long long d = (long long)(p.rp[v + 1] - p.rp[v]);
                if ((threadIdx.x & 31) == 0 && in) atomicAdd(&live[L_NFRONT], 1u);
                warp_push_chunks((threadIdx.x & 31) == 0 && in, v, d, p.fb, &live[L_FB], p.cap,
                                 ctl, p.tn.chunk);
            };
            for_vertices(p.as[par], nas, p.ab[par], nab, tid, nthreads, gwarp, nwarps,
                         front_thread, front_warp);
            if (!dom.sync()) return;
            if (threadIdx.x == 0) {
                ++st[kStBarriers];
                st[kStFrontier] += snap[L_NFRONT];
            }
            fs = p.fs;
            fb = p.fb;
            nfs = snap[L_FS];
            nfb = snap[L_FB];
        }
        // Step I: histogram rows of the vertices that recompute HINDEX
        {
            HistArc<Off> f{p.est, p.hist};
            expand(p.rp, p.ci, fs, nfs, fb, nfb, gwarp, nwarps, f, p.tn,
                   batch_width(nfs, nfb, nwarps));
            arcs += f.n_arcs;
            atomics += f.n_atomics;
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        // Step II: HINDEX; the vertices whose estimate falls are listed
        {
            auto sum_thread = [&](bool ok, int v) {
                bool fell = false;
                long long d = 0;
                if (ok) {
                    const int K = ldcg(p.est + v);
                    const int h = hindex_thread(p, v, K);
                    if (h < K) {
                        fell = true;
                        p.newv[v] = h;
                        d = (long long)(p.rp[v + 1] - p.rp[v]);
                    }
                }
                warp_append_vertex(fell, v, d, p.cs, &live[L_CS], (unsigned)n, p.cb, &live[L_CB],
                                   p.cap, ctl, p.tn);
                const unsigned c = __popc(__ballot_sync(kFull, fell));
                if ((threadIdx.x & 31) == 0 && c) atomicAdd(&live[L_NCHG], c);
            };
            auto sum_warp = [&](int v) {
                const int K = ldcg(p.est + v);
                const int h = hindex_warp(p, v, K);
                const long long d = (long long)(p.rp[v + 1] - p.rp[v]);
                if ((threadIdx.x & 31) == 0 && h < K) {
                    p.newv[v] = h;
                    atomicAdd(&live[L_NCHG], 1u);
                }
                warp_push_chunks((threadIdx.x & 31) == 0 && h < K, v, d, p.cb, &live[L_CB], p.cap,
                                 ctl, p.tn.chunk);
            };
            for_vertices(fs, nfs, fb, nfb, tid, nthreads, gwarp, nwarps, sum_thread, sum_warp);
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        const unsigned ncs = snap[L_CS], ncb = snap[L_CB], nchg = snap[L_NCHG];
        if (nchg == 0) break;
        if (threadIdx.x == 0) {
            ++st[kStRounds];
            if (!UseCnt) st[kStFrontier] += nchg;
        }
        // apply the new estimates; the next active set is their neighbourhoods
        for_vertices(
            p.cs, ncs, p.cb, ncb, tid, nthreads, gwarp, nwarps,
            [&](bool ok, int v) {
                if (ok) p.est[v] = ldcg(p.newv + v);
            },
            [&](int v) {
                if ((threadIdx.x & 31) == 0) p.est[v] = ldcg(p.newv + v);
            });
        {
            ActArc<Off> f{p.rp,
                          p.stamp,
                          (int)(r + 1),
                          p.as[np],
                          p.ab[np],
                          &live[2 * np + L_AS],
                          &live[2 * np + L_AB],
                          &live[L_NACT + np],
                          (unsigned)n,
                          p.cap,
                          ctl,
                          p.tn};
            expand(p.rp, p.ci, p.cs, ncs, p.cb, ncb, gwarp, nwarps, f, p.tn,
                   batch_width(ncs, ncb, nwarps));
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
    }
    for (long long v = first + threadIdx.x; v < n; v += nthreads) p.core[v] = ldcg(p.est + v);
}

}  // namespace i2c
}  // namespace pico
