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

#include <type_traits>

#include "pico_device.cuh"

namespace pico {
namespace peel {

// live counters: queue tails, then kept-count and min slots of three scans,
// then (asynchronous levels) the static frontier's small and chunk counts
enum : int {
    L_QS = 0, L_QB = 1, L_KEPT = 2 /* 2..4 */, L_MIN = 5 /* 5..7 */, L_FS = 8 /* 8..10 */,
    L_FB = 11 /* 11..13 */
};

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
    // asynchronous levels only (run_async)
    int *work = nullptr;  // residual degrees; `core` then receives each vertex's level
    int *fs = nullptr;    // the scan's frontier of small vertices, n slots
    int2 *fb = nullptr;   // the scan's frontier chunk entries, qb_cap slots
    Line *actl = nullptr; // AsyncLine lines, then one line per CTA (level-end flags)
};

// Lines of the asynchronous level control block (run_async).
enum : int { A_QS_HEAD = 0, A_QB_HEAD = 1, A_DONE = 2, A_FLAGS = 3 /* one per CTA */ };
constexpr int kMaxAsyncCtas = 2048;   // CTAs the control block has flag lines for

// Capacity of the list of (vertex, chunk) entries of large vertices, for
// every allowed tuning (chunk >= kMinChunk, small_deg >= kMinSmallDeg).
__host__ __device__ inline size_t chunk_list_capacity(long long m)
{
    return (size_t)(m / kMinChunk + m / (kMinSmallDeg + 1) + 2);
}

// Carves PeelOne's scratch (the control block, residual lists and queues;
// with `async` also the work array, the scan frontier lists and the
// asynchronous control lines) from c and sets n and the pointers of p.
template <typename Off, typename C>
inline void carve(Params<Off> &p, C &c, long long n, long long m, bool async)
{
    p.n = n;
    p.ctl = c.template take<Ctrl>(1);
    p.res0 = c.template take<int>(n);
    p.res1 = c.template take<int>(n);
    p.qs = c.template take<int>(n);
    p.qb_cap = (unsigned)chunk_list_capacity(m);
    p.qb = c.template take<int2>(p.qb_cap);
    if (async) {
        p.work = c.template take<int>(n);
        p.fs = c.template take<int>(n);
        p.fb = c.template take<int2>(p.qb_cap);
        p.actl = c.template take<Line>(A_FLAGS + kMaxAsyncCtas);
    } else {
        p.work = nullptr;
        p.fs = nullptr;
        p.fb = nullptr;
        p.actl = nullptr;
    }
}

template <typename Off, int Mode = kPeelRepair, bool kAsync = false>
struct Arc {
    static constexpr int kArcs = 4;
    const Off *rp;
    int *core;            // residual degrees (run_async: the work array)
    int *qs;
    int2 *qb;
    unsigned qb_cap;
    Ctrl *ctl;
    unsigned *live;
    int k;
    unsigned qs_cap;
    Tuning tn;
    int *out = nullptr;   // run_async: receives k for every vertex queued at level k
    int *loc = nullptr;   // run_async: this warp's 32 shared-memory slots for the small
    unsigned loc_n = 0;   // vertices it walks itself next (warp-uniform count)
    bool hub = false;     // run_async: this walk reads each neighbour before its
                          // decrement (warp-uniform; chunks of high-degree vertices)
    unsigned long long n_arcs = 0, n_atomics = 0, n_extra = 0;

    __device__ __forceinline__ bool item(int, int &, int &) { return true; }

    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&)[kArcs], const int (&)[kArcs])
    {
        int c[kArcs], old[kArcs];
        // Asynchronous levels with the repair clamp need no guard read: the
        // work array's values matter only while a vertex is unqueued, and a
        // decrement of a queued vertex returns at most k (no append). One
        // dependent round trip less per arc.
        // A hub's chunk still reads first: most of its arcs end at vertices
        // peeled earlier, and a load costs L2 less than an atomic.
        constexpr bool kGuard = !(kAsync && Mode == kPeelRepair);
        const bool guard = kGuard || hub;
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            c[j] = valid[j] ? (guard ? (kGuard ? __ldca(core + u[j]) : __ldcg(core + u[j])) : INT_MAX)
                            : 0;
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
        if (kAsync) {
            // the decrement that moved u from k + 1 to k appends it (once), to
            // this warp's local slots while they last, else to qs; its degree
            // class is decided when it is walked
            const unsigned lane = threadIdx.x & 31;
#pragma unroll
            for (int j = 0; j < kArcs; ++j) {
                const bool push = valid[j] && c[j] > k && old[j] == k + 1;
                if (push) out[u[j]] = k;
                const unsigned b = __ballot_sync(kFull, push);
                const unsigned rank = __popc(b & ((1u << lane) - 1u));
                const unsigned room = 32u - loc_n;
                const bool local = push && rank < room;
                if (local) loc[loc_n + rank] = u[j];
                loc_n += min(room, (unsigned)__popc(b));
                const bool listed = push && !local;
                const unsigned pos = warp_push(&live[L_QS], listed);
                if (listed) {
                    if (pos < qs_cap) st_relaxed(qs + pos, u[j]);
                    else set_error(ctl, kErrNotConverged);
                }
            }
            return;
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

// With int32 offsets a dynamic chunk entry holds its arc range [s, t), so
// that its walk needs no row bounds (one dependent load less per chunk);
// with int64 offsets it holds (vertex, chunk index), as the scan's entries
// do.
template <typename Off>
struct RangeEntries : std::integral_constant<bool, sizeof(Off) == 4> {};

// Whether the chunks of a vertex of degree d peeled at level k read each
// neighbour before decrementing it (see kPeelGuard).
__device__ __forceinline__ bool hub_guard(long long d, int k, int g)
{
    return g > 0 && d > (long long)g * k;
}

// Warp-cooperative append of the arc ranges of large vertices: every lane
// with `pred` owns a vertex whose row starts at rs and holds d arcs; the warp
// writes the ceil(d / chunk) ranges [a, b) of each such vertex in turn, as
// (a, b), or as (a, ~b) when `guard` is set (b >= 1, so ~b <= -2 never
// equals the empty slot's -1).
__device__ __forceinline__ void warp_push_ranges(bool pred, int rs, int d, bool guard, int2 *list,
                                                 unsigned *counter, unsigned cap, Ctrl *ctl,
                                                 int chunk)
{
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(kFull, pred);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int s0 = __shfl_sync(kFull, rs, src);
        const int dd = __shfl_sync(kFull, d, src);
        const bool gg = __shfl_sync(kFull, (int)guard, src) != 0;
        const unsigned nch = (unsigned)((dd + chunk - 1) / chunk);
        unsigned pos = 0;
        if (lane == 0) pos = atomicAdd(counter, nch);
        pos = __shfl_sync(kFull, pos, 0);
        if ((unsigned long long)pos + nch > cap) {
            if (lane == 0) set_error(ctl, kErrNotConverged);
            continue;
        }
        for (unsigned c = lane; c < nch; c += 32) {
            const int a = s0 + (int)c * chunk;
            const int b = dd - (int)c * chunk > chunk ? a + chunk : s0 + dd;
            st_relaxed(list + pos + c, make_int2(a, gg ? ~b : b));
        }
    }
}

// One warp walks the arcs [s, t) of col_idx (a range entry).
template <typename F>
__device__ __forceinline__ void walk_range(const int *__restrict__ ci, int s, int t, F &f)
{
    constexpr int U = F::kArcs;
    const int lane = threadIdx.x & 31;
    for (int e0 = s; e0 < t; e0 += 32 * U) {
        bool valid[U];
        int vo[U], u[U], ao[U], bo[U], rso[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int e = e0 + 32 * j + lane;
            valid[j] = e < t;
            u[j] = valid[j] ? __ldg(ci + e) : -1;
            vo[j] = -1;
            rso[j] = 0;
            ao[j] = 0;
            bo[j] = 0;
        }
        f.arcs(valid, vo, u, rso, ao, bo);
    }
}

// One warp walks chunk c of the adjacency of vertex v (a (vertex, chunk)
// entry), reading each neighbour first when v's degree calls for it.
template <typename Off, typename F>
__device__ __forceinline__ void walk_chunk_guarded(const Off *__restrict__ rp,
                                                   const int *__restrict__ ci, int v, int c, F &f,
                                                   const Tuning &tn)
{
    constexpr int U = F::kArcs;
    const int lane = threadIdx.x & 31;
    const Off rs = rp[v], re = rp[v + 1];
    const Off s = rs + (Off)c * tn.chunk;
    const Off t = (s + tn.chunk < re) ? s + tn.chunk : re;
    f.hub = hub_guard((long long)(re - rs), f.k, tn.peel_guard);
    for (Off e0 = s; e0 < t; e0 += 32 * U) {
        bool valid[U];
        int vo[U], u[U], ao[U], bo[U];
        Off rso[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const Off e = e0 + 32 * j + lane;
            valid[j] = e < t;
            u[j] = valid[j] ? __ldg(ci + e) : -1;
            vo[j] = v;
            rso[j] = rs;
            ao[j] = 0;
            bo[j] = 0;
        }
        f.arcs(valid, vo, u, rso, ao, bo);
    }
    f.hub = false;
}

// ---------------------------------------------------------------------------
// PeelOne with asynchronous levels (the whole grid, one graph)
// ---------------------------------------------------------------------------
// The wave structure above ends every wave of the dynamic frontier with a grid
// barrier. Here a level needs one barrier, after its scan; within the level,
// warps take the dynamic frontier as it is appended:
//   scan     as above, but the frontier goes to separate lists (fs: small
//            vertices, fb: chunk entries), and every frontier vertex gets its
//            final value out[v] = k at once. The residual degrees live in a
//            work array, so no repair pass is needed: its values matter only
//            while a vertex is unqueued (they are exact then: each queued
//            neighbour decrements it once), and a queued vertex's value is
//            only ever compared with k, where a dip below k and k answer
//            alike. For the same reason the repair mode needs no guard read
//            before a decrement: the decrement's return value decides.
//   barrier  its last arrival sets the ticket heads (below) and snapshots
//            the counters; the scan's frontier is then final.
//   static   the scan's frontier is walked like one wave (as expand() does).
//   hubs     a chunk of a vertex whose degree exceeds tn.peel_guard * k reads
//            each neighbour's residual degree before the decrement and skips
//            the atomic when it is <= k: such a vertex has about k neighbours
//            left, so most of its arcs end at vertices peeled earlier, and a
//            load costs L2 less than an atomic. Other walks issue the
//            decrement at once (no dependent round trip on a chain).
//   dynamic  the decrement that takes u from k + 1 to k writes out[u] = k and
//            appends u: to 32 local slots of its warp (shared memory) while
//            they last, else to the queue qs. A vertex's degree class is
//            decided when it is walked: one above small_deg is then listed as
//            chunk entries in qb (arc ranges with int32 offsets). Queue slots start as -1 (set at launch) and
//            are written once in the whole run. Every warp holds a ticket of
//            32 consecutive qs slots and one of one qb slot; each pass of its
//            loop walks what has arrived in them plus at most one batch of its
//            local slots (so that no listed entry waits behind a long local
//            chain), and takes the next ticket (one atomic on a head counter)
//            once one is used up. The first tickets of a level are dealt out
//            without atomics (consecutive tickets to different CTAs), so the
//            heads start past them.
//   end      the level is over when every listed entry (scan frontiers, qs and
//            qb tails) has been walked. A warp that finds nothing new adds
//            what it walked to its CTA's count (shared memory); the warp that
//            leaves its CTA with no busy warp adds that count to `done` and,
//            if `done` then equals the listed entries (read after its
//            acquire-release add, so no listing is missed), writes the level
//            into one flag line per CTA (release). Local entries are never
//            listed: a warp holding some has not yet added the listed entry
//            they descend from. Idle warps poll their tickets and their
//            CTA's flag, less and less often.
// A warp may still poll stale tickets when other warps start the next scan;
// the scan writes only fs/fb, and the next level's queue slots are written
// only after its barrier, which every warp must reach first. By Thm. 1 and
// Cor. 1 the order in which a level's vertices are processed does not change
// the result; each vertex is still queued exactly once (one decrement takes
// it from k + 1 to k, or the scan finds it at k), so the levels, the arcs
// walked and the successful decrements are the same as in the wave form.
template <typename Off, int Mode = kPeelRepair>
__device__ void run_async(const Params<Off> &p, GridDom &dom, unsigned *s_tmp,
                          unsigned long long *st, PhaseClock &clk, unsigned long long &arcs,
                          unsigned long long &atomics, unsigned long long &extra)
{
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const unsigned lane = threadIdx.x & 31;
    const long long n = p.n;
    const long long first = (long long)blockIdx.x * blockDim.x;
    unsigned *qs_head = p.actl[A_QS_HEAD].w;
    unsigned *qb_head = p.actl[A_QB_HEAD].w;
    unsigned long long *done = reinterpret_cast<unsigned long long *>(p.actl[A_DONE].w);
    int *my_flag = reinterpret_cast<int *>(p.actl[A_FLAGS + blockIdx.x].w);
    // ticket index of this warp: consecutive tickets go to different CTAs
    const unsigned tix = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    __shared__ int s_loc[kThreads / 32][32];   // local slots of each warp
    __shared__ unsigned s_busy;                // warps of this CTA that are not idle
    __shared__ unsigned long long s_acc;       // walked by idle warps, not yet in `done`

    // init: work = degree, isolated vertices get 0, residual list, queue
    // slots empty, control lines zero
    {
        unsigned mx = 0;
        for (long long base = first; base < n; base += nthreads) {
            const long long v = base + threadIdx.x;
            bool keep = false;
            if (v < n) {
                const int d = (int)(p.rp[v + 1] - p.rp[v]);
                p.work[v] = d;
                if (d == 0) p.core[v] = 0;
                p.qs[v] = -1;
                keep = d > 0;
                if (keep) mx = max(mx, (unsigned)(INT_MAX - d));
            }
            unsigned pos, unused;
            block_push2(keep, false, &live[L_KEPT], &live[L_KEPT], pos, unused, s_tmp);
            if (keep) p.res0[pos] = (int)v;
        }
        for (unsigned i = tid; i < p.qb_cap; i += nthreads) p.qb[i] = make_int2(-1, -1);
        if (threadIdx.x < 32) p.actl[A_FLAGS + blockIdx.x].w[threadIdx.x] = 0;
        if (blockIdx.x == 0 && threadIdx.x < 32 * A_FLAGS)
            p.actl[threadIdx.x >> 5].w[threadIdx.x & 31] = 0;
        block_max_to(mx, &live[L_MIN], s_tmp);
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    clk.end(st, kPhInit);

    unsigned nres = snap[L_KEPT];
    int k = INT_MAX - (int)snap[L_MIN];
    unsigned slot = 1;   // kept/min/frontier slot of the next scan (slot 0: init)
    int cur = 0;
    unsigned long long listed_static = 0;   // scan frontier entries of all levels so far
    long long scans = 0;
    const long long max_scans = 2 * n + 4;
    const unsigned long long limit_ns = dom.limit_ns;

    while (nres > 0) {
        if (++scans > max_scans) {
            if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
            return;
        }
        if (dom.leader()) {
            const unsigned nx = (slot + 1) % 3;
            live[L_KEPT + nx] = 0;
            live[L_MIN + nx] = 0;
            live[L_FS + nx] = 0;
            live[L_FB + nx] = 0;
        }

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
            for (int j = 0; j < kScanItems; ++j) c[j] = v[j] >= 0 ? ldcg(p.work + v[j]) : -1;
            unsigned nsmall = 0, nkeep = 0;
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) {
                d[j] = 0;
                if (c[j] == k) {
                    d[j] = (long long)(p.rp[v[j] + 1] - p.rp[v[j]]);
                    p.core[v[j]] = k;
                }
                nsmall += (c[j] == k && d[j] <= p.tn.small_deg);
                nkeep += (c[j] > k);
                if (c[j] > k) mx = max(mx, (unsigned)(INT_MAX - c[j]));
            }
            unsigned pf, pk;
            block_alloc2(nsmall, nkeep, &live[L_FS + slot], &live[L_KEPT + slot], pf, pk, s_tmp);
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) {
                if (c[j] == k && d[j] <= p.tn.small_deg) p.fs[pf++] = v[j];   // pf < nres <= n
                if (c[j] > k) rout[pk++] = v[j];                              // pk < nres <= n
            }
#pragma unroll
            for (int j = 0; j < kScanItems; ++j)
                warp_push_chunks(c[j] == k && d[j] > p.tn.small_deg, v[j], d[j], p.fb,
                                 &live[L_FB + slot], p.qb_cap, ctl, p.tn.chunk);
        }
        block_max_to(mx, &live[L_MIN + slot], s_tmp);
        // the last arrival deals out the level's first tickets by moving the
        // heads past them
        const bool ok = dom.sync_hook([&](const uint4 *t) {
            const unsigned *w = reinterpret_cast<const unsigned *>(t);
            __stcg(qs_head, w[L_QS] + 32u * nwarps);
            __stcg(qb_head, w[L_QB] + nwarps);
        });
        if (!ok) return;
        if (threadIdx.x == 0) {
            ++st[kStBarriers];
            ++st[kStScans];
            st[kStScanned] += nres;
        }
        clk.end(st, kPhScan, nres);

        const unsigned t0 = snap[L_QS], b0 = snap[L_QB];
        const unsigned nfs = snap[L_FS + slot], nfb = snap[L_FB + slot];
        nres = snap[L_KEPT + slot];
        const int kmin_kept = INT_MAX - (int)snap[L_MIN + slot];
        slot = (slot + 1) % 3;
        cur ^= 1;
        if (nfs == 0 && nfb == 0) {   // empty level: jump to the smallest kept value
            k = kmin_kept;
            continue;
        }
        if (threadIdx.x == 0) {
            ++st[kStLevels];
            if ((unsigned long long)k > st[kStKmax]) st[kStKmax] = (unsigned long long)k;
        }
        listed_static += nfs + nfb;

        if (threadIdx.x == 0) {
            s_busy = blockDim.x >> 5;
            s_acc = 0;
        }
        __syncthreads();

        Arc<Off, Mode, true> f{p.rp, p.work, p.qs, p.qb, p.qb_cap, ctl, live, k, (unsigned)n, p.tn};
        f.out = p.core;
        f.loc = s_loc[threadIdx.x >> 5];
        // walks one vertex per lane (v < 0: none); a vertex of degree above
        // small_deg is listed as chunk entries (qb) instead
        auto walk_vertices = [&](int v) {
            Off rs = 0;
            long long d = 0;
            if (v >= 0) {
                rs = p.rp[v];
                d = (long long)(p.rp[v + 1] - rs);
            }
            const bool large = d > p.tn.small_deg;
            if (RangeEntries<Off>::value)
                warp_push_ranges(large, (int)rs, (int)d, hub_guard(d, k, p.tn.peel_guard), p.qb,
                                 &live[L_QB], p.qb_cap, ctl, p.tn.chunk);
            else
                warp_push_chunks<true>(large, v, d, p.qb, &live[L_QB], p.qb_cap, ctl, p.tn.chunk);
            walk_batch(p.ci, large ? -1 : v, rs, large ? 0 : (int)d, f);
        };

        // static part: the scan's frontier, walked like one wave (batches of
        // small vertices, then (vertex, chunk) entries)
        const unsigned vb = batch_width(nfs, nfb, nwarps);
        unsigned long long walked = 0;   // listed entries walked, not yet added to `done`
        {
            const unsigned nbatch = (nfs + vb - 1u) / vb;
            for (unsigned unit = gwarp; unit < nbatch + nfb; unit += nwarps) {
                if (unit < nbatch) {
                    const unsigned idx = unit * vb + lane;
                    int v = -1;
                    if (lane < vb && idx < nfs) v = ldcg(p.fs + idx);
                    walk_small_batch(p.rp, p.ci, v, f, p.tn.small_deg);
                    walked += min(vb, nfs - unit * vb);
                } else {
                    const int2 ent = __ldcg(p.fb + (unit - nbatch));   // written by other CTAs
                    walk_chunk_guarded(p.rp, p.ci, ent.x, ent.y, f, p.tn);
                    walked += 1;
                }
            }
        }

        // dynamic part. Each pass walks what has arrived in this warp's
        // tickets and at most one batch of its local slots, so that listed
        // entries never wait behind a long local chain. An idle warp adds what
        // it walked to its CTA's count; the warp that leaves the CTA with no
        // busy warp adds the CTA's count to `done` (local entries were never
        // listed and are not counted). Idle warps poll less and less often.
        unsigned ts = t0 + 32u * tix;   // small ticket: qs slots ts .. ts + 31
        unsigned tmask = 0;             // its slots already walked (one bit per lane)
        unsigned tb = b0 + tix;         // chunk ticket: qb slot tb
        bool busy = true;               // counted in s_busy
        unsigned spins = 0;
        unsigned long long idle_since = 0;
        for (;;) {
            // probes (independent loads, one round trip): the first slot of
            // the small ticket not yet walked (slots are reserved in order, so
            // it is written first but for a moment), the chunk slot, the flag
            const unsigned first_open = __ffs(~tmask) - 1u;   // tmask != kFull here
            int probe = -1, fl = 0;
            int2 e = make_int2(-1, -1);
            if (lane == 0) {
                if (ts + first_open < (unsigned)n) probe = ld_relaxed(p.qs + ts + first_open);
                if (tb < p.qb_cap) e = ld_relaxed(p.qb + tb);
                fl = ld_relaxed(my_flag);
            }
            bool worked = false;
            if (f.loc_n) {   // one batch of local slots while the probes are in flight
                __syncwarp();   // the lanes' writes to the local slots are visible
                const int lv = lane < f.loc_n ? f.loc[lane] : -1;
                __syncwarp();   // every lane has read its slot before new writes
                f.loc_n = 0;
                walk_vertices(lv);
                worked = true;
            }
            probe = __shfl_sync(kFull, probe, 0);
            if (probe >= 0) {   // read the whole ticket
                const unsigned sl = ts + lane;
                int v = -1;
                if (!((tmask >> lane) & 1u) && sl < (unsigned)n) v = ld_relaxed(p.qs + sl);
                const unsigned got = __ballot_sync(kFull, v >= 0);
                if (got) {
                    if (!busy) {
                        if (lane == 0) atomicAdd(&s_busy, 1u);
                        busy = true;
                    }
                    walk_vertices(v);
                    tmask |= got;
                    walked += __popc(got);
                    worked = true;
                    if (tmask == kFull) {
                        unsigned nt = 0;
                        if (lane == 0) nt = atomicAdd(qs_head, 32u);
                        ts = __shfl_sync(kFull, nt, 0);
                        tmask = 0;
                    }
                }
            }
            e.x = __shfl_sync(kFull, e.x, 0);
            e.y = __shfl_sync(kFull, e.y, 0);
            if (e.x >= 0 && e.y != -1) {   // both words of the chunk entry written
                if (!busy) {
                    if (lane == 0) atomicAdd(&s_busy, 1u);
                    busy = true;
                }
                unsigned nt = 0;   // the next ticket, taken while this entry is walked
                if (lane == 0) nt = atomicAdd(qb_head, 1u);
                if constexpr (RangeEntries<Off>::value) {
                    f.hub = e.y < 0;
                    walk_range(p.ci, e.x, e.y < 0 ? ~e.y : e.y, f);
                    f.hub = false;
                } else {
                    walk_chunk_guarded(p.rp, p.ci, e.x, e.y, f, p.tn);
                }
                walked += 1;
                worked = true;
                tb = __shfl_sync(kFull, nt, 0);
            }
            if (worked || f.loc_n) {
                spins = 0;
                idle_since = 0;
                continue;
            }
            int fin = 0, over = 0;
            if (busy) {   // going idle
                __syncwarp();   // the warp's appends are ordered before lane 0's adds
                if (lane == 0) {
                    if (walked) atomicAdd(&s_acc, walked);
                    if (atomicSub(&s_busy, 1u) == 1u) {   // the CTA's last busy warp
                        const unsigned long long add = atomicExch(&s_acc, 0ull);
                        if (add) {
                            unsigned long long old;
                            asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                                         : "=l"(old)
                                         : "l"(done), "l"(add)
                                         : "memory");
                            const unsigned long long listed =
                                listed_static + (unsigned long long)ld_relaxed(&live[L_QS]) +
                                (unsigned long long)ld_relaxed(&live[L_QB]);
                            fin = old + add == listed;
                        }
                    }
                }
                walked = 0;
                busy = false;
            }
            if (lane == 0) {
                over = fl >= k;
                if (!over && !fin && (++spins & 15) == 0) {
                    const unsigned long long t = gtime();
                    if (idle_since == 0) idle_since = t;
                    if (status_of(ctl) != 0) over = 1;
                    else if (t - idle_since > limit_ns) {
                        set_error(ctl, kErrTimeout);
                        over = 1;
                    }
                }
            }
            fin = __shfl_sync(kFull, fin, 0);
            if (fin) {   // the level's last listed entry has been walked
                __threadfence();   // one fence, then plain strong stores: a release
                for (unsigned c = lane; c < gridDim.x; c += 32)
                    st_relaxed(reinterpret_cast<int *>(p.actl[A_FLAGS + c].w), k);
                break;
            }
            if (__shfl_sync(kFull, over, 0)) {
                if (lane == 0) (void)ld_acquire(my_flag);
                __syncwarp();
                break;
            }
            spins = __shfl_sync(kFull, spins, 0);
            __nanosleep(spins < 64 ? 32 : (spins < 512 ? 256 : 1024));
        }
        arcs += f.n_arcs;
        atomics += f.n_atomics;
        extra += f.n_extra;
        clk.end(st, kPhLevel, nfs + nfb);
        k = k + 1;
    }
}

}  // namespace peel
}  // namespace pico
