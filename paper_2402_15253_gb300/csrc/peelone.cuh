// PeelOne (Sec. III, Alg. 4) on one graph, for either synchronisation domain
// (the whole grid, or one CTA of the batched kernel).
//
// core[] doubles as the residual degree and the coreness (Sec. III-C, step 2:
// one array instead of deg[] + rem[]). Level k:
//   scan    the compacted list of residual vertices is filtered: core == k
//           -> frontier queue (Alg. 4 "scan"; Cor. 1 guarantees no residual
//           vertex is below k), core > k -> kept for the next level, smaller
//           values belong to vertices already peeled and are dropped. The
//           smallest kept value is recorded so that an empty level jumps
//           straight to the next non-empty one.
//   scatter for each frontier vertex v and neighbour u with core[u] > k,
//           core[u] is decremented atomically; the thread whose decrement
//           takes u from k + 1 to k appends u to the frontier of the same
//           level (the dynamic frontier of Sec. III-C, step 3). Each wave of
//           the frontier ends with a barrier of the domain; the level ends
//           when a wave appends nothing.
//   repair  the clamp of atomicSub_{>=k} (Sec. III-B) is realised as a guard
//           (core[u] > k, read before the atomic) plus an exact repair: a
//           racing decrement can only hit a vertex already queued at level k
//           (Thm. 1: its coreness is k), so after the level every vertex of
//           the level's queue is written back to k. Values seen in between
//           are only compared against k, where a dip below k and k itself
//           give the same answer.
// The guard read goes through L1 (most arcs of a skewed graph end at a few
// hubs). An L1 line can be older than L2 within a level, but the estimates of
// unqueued vertices only decrease, so an old value is never below the current
// one: it can only send a thread to an atomic that finds u already at k (an
// overshoot, handled as above), never skip a needed decrement. Vertices of
// earlier levels are at most k - 1 in every copy, and repaired values are
// compared only after the barrier that ends the level, whose acquire makes
// L1 loads observe them.
// Every vertex is queued exactly once over the whole run (only one thread can
// move it from k + 1 to k), so the queue is the peel order and needs n slots.
//
// Two other ways to keep a decrement from taking a vertex below k are built
// for comparison (the ablation of Sec. V, Fig. 4): kPeelCas is the paper's
// atomicSub_{>=k} as a compare-and-swap loop that never writes a value below
// k (no repair needed); kPeelAddBack is the atomicAdd method of Fig. 4a, where
// a thread whose decrement went below k adds the unit back at once. All three
// give the same levels, waves and results; `extra` counts the atomics beyond
// the successful decrements (overshoots repaired, failed compare-and-swaps,
// or overshoot-plus-add-back pairs).
#pragma once

#include "pico_device.cuh"

namespace pico {
namespace peel {

// live counters: queue tails, then kept-count and min slots of three scans
enum : int { L_QS = 0, L_QB = 1, L_KEPT = 2 /* 2..4 */, L_MIN = 5 /* 5..7 */ };

constexpr int kScanItems = 4;   // residual-list entries per thread per scan step

template <typename Off>
struct Params {
    const Off *rp;
    const int *ci;
    long long n;
    int *core;
    int *res0, *res1;     // residual lists (ping-pong), n slots each
    int *qs;              // queue of small vertices, n slots
    int2 *qb;             // queue of (vertex, chunk) entries of large vertices
    unsigned qb_cap;
    Ctrl *ctl;            // status word (errors)
    Tuning tn;
};

template <typename Off, int Mode = kPeelRepair>
struct Arc {
    static constexpr int kArcs = 4;
    const Off *rp;
    int *core;
    int *qs;
    int2 *qb;
    unsigned qb_cap;
    Ctrl *ctl;
    unsigned *live;
    int k;
    unsigned qs_cap;
    Tuning tn;
    unsigned long long n_arcs = 0, n_atomics = 0, n_extra = 0;

    __device__ __forceinline__ bool item(int, int &, int &) { return true; }

    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&)[kArcs], const int (&)[kArcs])
    {
        int c[kArcs], old[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) c[j] = valid[j] ? __ldca(core + u[j]) : 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            old[j] = 0;
            if (valid[j]) {
                ++n_arcs;
                if (c[j] > k) {
                    if (Mode == kPeelCas) {   // atomicSub_{>=k}: never below k
                        int cur = c[j];
                        for (;;) {
                            const int prev = atomicCAS(core + u[j], cur, cur - 1);
                            ++n_atomics;
                            if (prev == cur) {
                                old[j] = cur;
                                break;
                            }
                            ++n_extra;
                            if (prev <= k) {   // another thread took u to k
                                old[j] = prev;
                                break;
                            }
                            cur = prev;
                        }
                    } else {
                        old[j] = atomicSub(core + u[j], 1);
                        ++n_atomics;
                        if (old[j] <= k) {   // overshoot past k (a racing decrement)
                            if (Mode == kPeelAddBack) {
                                atomicAdd(core + u[j], 1);
                                ++n_atomics;
                                n_extra += 2;
                            } else {
                                ++n_extra;   // undone by the repair after the level
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            // the decrement that moved u from k + 1 to k appends it (once)
            const bool push = valid[j] && c[j] > k && old[j] == k + 1;
            long long d = 0;
            bool small = false, large = false;
            if (push) {
                d = (long long)(rp[u[j] + 1] - rp[u[j]]);
                small = d <= tn.small_deg;
                large = !small;
            }
            const unsigned pos = warp_push(&live[L_QS], small);
            if (small) {
                if (pos < qs_cap) qs[pos] = u[j];
                else set_error(ctl, kErrNotConverged);
            }
            warp_push_chunks(large, u[j], d, qb, &live[L_QB], qb_cap, ctl, tn.chunk);
        }
    }
};

template <typename Off>
__device__ __forceinline__ void repair(const Params<Off> &p, int k, unsigned s0, unsigned e0,
                                       unsigned s1, unsigned e1, unsigned tid, unsigned nthreads)
{
    for (unsigned i = s0 + tid; i < e0; i += nthreads) p.core[ldcg(p.qs + i)] = k;
    for (unsigned i = s1 + tid; i < e1; i += nthreads) p.core[__ldcg(&p.qb[i].x)] = k;
}

// PeelOne on one graph. Every thread of the domain calls it. st: per-CTA
// statistics in shared memory (thread 0 writes); s_tmp: >= 128 shared words.
template <typename Off, typename Dom, int Mode = kPeelRepair>
__device__ void run(const Params<Off> &p, Dom &dom, unsigned *s_tmp, unsigned long long *st,
                    PhaseClock &clk, unsigned long long &arcs, unsigned long long &atomics,
                    unsigned long long &extra)
{
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const long long n = p.n;
    const long long first = (long long)dom.cta() * blockDim.x;

    // init: core = degree; residual list = non-isolated vertices
    {
        unsigned mx = 0;
        for (long long base = first; base < n; base += nthreads) {
            const long long v = base + threadIdx.x;
            bool keep = false;
            if (v < n) {
                const int d = (int)(p.rp[v + 1] - p.rp[v]);
                p.core[v] = d;
                keep = d > 0;
                if (keep) mx = max(mx, (unsigned)(INT_MAX - d));
            }
            unsigned pos, unused;
            block_push2(keep, false, &live[L_KEPT], &live[L_KEPT], pos, unused, s_tmp);
            if (keep) p.res0[pos] = (int)v;
        }
        block_max_to(mx, &live[L_MIN], s_tmp);
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    if (Dom::kGrid) clk.end(st, kPhInit);

    unsigned nres = snap[L_KEPT];
    int k = INT_MAX - (int)snap[L_MIN];
    unsigned slot = 1;   // kept/min slot of the next scan (slot 0: init)
    int cur = 0;
    int prev_k = -1;
    unsigned r_s0 = 0, r_e0 = 0, r_s1 = 0, r_e1 = 0;
    unsigned qs_tail = 0, qb_tail = 0;
    long long scans = 0;
    const long long max_scans = 2 * n + 4;

    while (nres > 0) {
        if (++scans > max_scans) {
            if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
            return;
        }
        if (dom.leader()) {
            live[L_KEPT + (slot + 1) % 3] = 0;
            live[L_MIN + (slot + 1) % 3] = 0;
        }
        if (Mode == kPeelRepair && prev_k >= 0)
            repair(p, prev_k, r_s0, r_e0, r_s1, r_e1, tid, nthreads);
        prev_k = -1;

        // scan the residual list at level k (kScanItems vertices per thread)
        const int *rin = cur ? p.res1 : p.res0;
        int *rout = cur ? p.res0 : p.res1;
        unsigned mx = 0;
        const long long step = (long long)nthreads * kScanItems;
        for (long long base = first * kScanItems; base < nres; base += step) {
            int v[kScanItems], c[kScanItems];
            long long d[kScanItems];
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) {
                const long long i = base + threadIdx.x + (long long)j * blockDim.x;
                v[j] = i < nres ? ldcg(rin + i) : -1;
            }
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) c[j] = v[j] >= 0 ? ldcg(p.core + v[j]) : -1;
            unsigned nsmall = 0, nkeep = 0;
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) {
                d[j] = 0;
                if (c[j] == k) d[j] = (long long)(p.rp[v[j] + 1] - p.rp[v[j]]);
                nsmall += (c[j] == k && d[j] <= p.tn.small_deg);
                nkeep += (c[j] > k);
                if (c[j] > k) mx = max(mx, (unsigned)(INT_MAX - c[j]));
            }
            unsigned pq, pk;
            block_alloc2(nsmall, nkeep, &live[L_QS], &live[L_KEPT + slot], pq, pk, s_tmp);
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) {
                if (c[j] == k && d[j] <= p.tn.small_deg) {
                    if (pq < (unsigned)n) p.qs[pq] = v[j];
                    else set_error(ctl, kErrNotConverged);
                    ++pq;
                }
                if (c[j] > k) rout[pk++] = v[j];   // pk < nres <= n
            }
#pragma unroll
            for (int j = 0; j < kScanItems; ++j)
                warp_push_chunks(c[j] == k && d[j] > p.tn.small_deg, v[j], d[j], p.qb, &live[L_QB],
                                 p.qb_cap, ctl, p.tn.chunk);
        }
        block_max_to(mx, &live[L_MIN + slot], s_tmp);
        if (!dom.sync()) return;
        if (threadIdx.x == 0) {
            ++st[kStBarriers];
            ++st[kStScans];
            st[kStScanned] += nres;
        }
        if (Dom::kGrid) clk.end(st, kPhScan, nres);

        const unsigned qs0 = qs_tail, qb0 = qb_tail;
        unsigned e0 = snap[L_QS], e1 = snap[L_QB];
        nres = snap[L_KEPT + slot];
        const int kmin_kept = INT_MAX - (int)snap[L_MIN + slot];
        slot = (slot + 1) % 3;
        cur ^= 1;
        if (e0 == qs0 && e1 == qb0) {   // empty level: jump to the smallest kept value
            k = kmin_kept;
            continue;
        }
        if (threadIdx.x == 0) {
            ++st[kStLevels];
            if ((unsigned long long)k > st[kStKmax]) st[kStKmax] = (unsigned long long)k;
        }

        // scatter, wave by wave (dynamic frontier)
        unsigned s0 = qs0, s1 = qb0;
        while (s0 < e0 || s1 < e1) {
            const unsigned units = (e0 - s0 + 31) / 32 + (e1 - s1);
            Arc<Off, Mode> f{p.rp, p.core, p.qs, p.qb, p.qb_cap, ctl, live, k, (unsigned)n, p.tn};
            expand(p.rp, p.ci, p.qs + s0, e0 - s0, p.qb + s1, e1 - s1, gwarp, nwarps, f, p.tn,
                   batch_width(e0 - s0, e1 - s1, nwarps));
            arcs += f.n_arcs;
            atomics += f.n_atomics;
            extra += f.n_extra;
            if (!dom.sync()) return;
            if (threadIdx.x == 0) {
                ++st[kStBarriers];
                ++st[kStSubrounds];
            }
            if (Dom::kGrid)
                clk.end(st, units < 64 ? kPhWaveTiny : (units < nwarps ? kPhWaveMid : kPhWaveWide),
                        units);
            s0 = e0;
            s1 = e1;
            e0 = snap[L_QS];
            e1 = snap[L_QB];
        }
        qs_tail = e0;
        qb_tail = e1;
        prev_k = k;
        r_s0 = qs0;
        r_e0 = e0;
        r_s1 = qb0;
        r_e1 = e1;
        k = k + 1;
    }
    if (Mode == kPeelRepair && prev_k >= 0)
        repair(p, prev_k, r_s0, r_e0, r_s1, r_e1, tid, nthreads);
}

}  // namespace peel
}  // namespace pico
