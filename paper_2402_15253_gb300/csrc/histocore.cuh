// HistoCore (Sec. IV-B, Alg. 6) on one graph, for either synchronisation domain
// (the whole grid, or one CTA of the batched kernel).
//
// histo[v][s] for s = 1..deg(v) lives at histo[row_ptr[v] + s - 1], so the
// histogram array has the shape of col_idx (m entries) and slot 0 is not
// stored. For s < core[v] the slot counts neighbours whose estimate is s; slot
// core[v] counts neighbours whose estimate is >= core[v] (the cnt of Thm. 2,
// stored in the histogram as Sec. IV-B describes); slots above core[v] are
// stale and never read.
//
//   InitHisto   histo[v][min(deg u, deg v)] += 1 over all arcs, then
//               V_cnt = {v : deg v >= 1, histo[v][deg v] < deg v}.
//   SumHisto    for v in V_cnt: sum the slots from core_old downwards until
//               the running sum reaches the slot index k; core[v] <- k,
//               mv[v] <- {core_old, k}, histo[v][k] <- sum (the new cnt).
//               By Thm. 2 every vertex of V_cnt changes.
//   UpdateHisto for changed v (x = core_old, y = core[v]) and neighbour u
//               with K = core[u] > y (types N1/N3 of Sec. IV-B): remove v
//               from slot min(x, K), add it to slot y; u joins the next V_cnt
//               when x >= K and slot K held exactly K before the decrement
//               (its cnt just fell below K). Slot K only decreases here, so u
//               is appended at most once per round.
// A grid barrier separates SumHisto from UpdateHisto (UpdateHisto reads the
// new estimates) and UpdateHisto from the next SumHisto (all edits of a
// round are in place before any vertex sums), which is the synchronous model
// of Alg. 6.
//
// UpdateHisto direction. Alg. 6 pushes: each changed vertex v edits the rows
// of its neighbours. On a large graph the rows edited in one round are spread
// over far more memory than L2 holds, and almost every edit then misses. The
// pull form issues the same edits from the other end: every vertex u whose
// estimate is above the smallest new estimate of the round walks its own
// adjacency and, for each neighbour w that changed in this round, applies
// w's edit to u's row. With a symmetric adjacency both forms apply the same
// multiset of edits (arc (v, u) pushed is arc (u, v) pulled), so the
// histograms, the next V_cnt (the same set of vertices whose slot K fell
// below K, see the deferred decision below) and the result are identical;
// only the order of the edits differs,
// and a warp pulling 32 consecutive rows edits one contiguous stretch of the
// histogram. Pulling scans the arcs of every row that an edit can reach
// instead of those of the changed vertices, so the auto mode pulls only in
// rounds whose changed vertices hold at least pull_pct % of the arcs of a
// graph with at least kPullMinArcs arcs. A vertex's {old, new} estimates are
// kept per round parity (mv[r & 1]) so that pulling rows can tell whether a
// neighbour changed in this round; SumHisto of round r clears the entries of
// round r-1's changed vertices in the other buffer (their lists are intact
// until UpdateHisto of round r appends to them). Pulling rows gather the
// record of every neighbour, so a packed copy (mvp: old << 16 | new in one
// word, half the bytes of mv) is what they read; estimates above 65534 store
// a sentinel that sends the reader to mv.
//
// Deferred V_cnt decision in pull rounds. Deciding the append at the edit
// needs the old value of slot K, so every edit of slot K is an atomic whose
// result the warp waits for before its next arcs. A pull round instead makes
// every edit a reduction, marks the rows whose slot K it decremented (cand),
// and after a barrier lists the marked u with histo[u][K] < K. The set is the
// same: after SumHisto every vertex has cnt >= K (unchanged vertices kept it,
// changed ones set it to a sum >= h), slot K only decreases in UpdateHisto,
// so its count ends below K exactly when one decrement took it from K to K-1.
//
// Neighbour gathers (the estimates in InitHisto and push rounds, the packed
// records in pull rounds) go through L1 (ld.global.ca): on skewed graphs most
// arcs end at a few hubs, whose records then hit in L1. These arrays are not
// written during the phases that gather them, and every grid barrier ends
// with an acquire at GPU scope, after which a weak load observes every write
// made before the barrier, so no line cached in an earlier phase is read.
//
// Load balance. V_cnt is kept as three lists by the estimate K that SumHisto
// will walk down from: K <= 32 one thread per vertex, K <= 2048 one warp per
// vertex (32 slots per step, warp suffix scan), larger K one CTA per vertex.
// UpdateHisto walks adjacency through expand() (batched small vertices,
// chunked large ones), so the changed vertices are listed again by degree.
#pragma once

#include "pico_device.cuh"

namespace pico {
namespace histo {

constexpr int kWarpK = 32;      // K above which a warp walks the histogram
constexpr int kBlockK = 2048;   // K above which a CTA walks the histogram

// live counters: V_cnt lists (T/W/B) per round parity, update lists, init
// chunks, INT_MAX - smallest new estimate of the round, and the arcs of the
// round's changed vertices (64-bit, two words, 8-byte aligned)
enum : int {
    L_T = 0, L_W = 1, L_B = 2, /* parity 1: 3..5 */ L_US = 6, L_UB = 7, L_IB = 8, L_YMIN = 9,
    L_VOL = 10 /* and 11 */
};

// Per-vertex record {estimate, histogram base (= row_ptr[v])}: UpdateHisto
// needs both for every neighbour it edits, and one 8-byte (16-byte with int64
// offsets) gather replaces two scattered 4-byte gathers from separate arrays.
template <typename Off> struct VRecOf { using type = int2; };
template <> struct VRecOf<long long> { using type = longlong2; };
template <typename Off> using VRec = typename VRecOf<Off>::type;

template <typename Off>
__device__ __forceinline__ VRec<Off> make_vrec(int est, Off base);
template <>
__device__ __forceinline__ int2 make_vrec<int>(int est, int base) { return make_int2(est, base); }
template <>
__device__ __forceinline__ longlong2 make_vrec<long long>(int est, long long base)
{
    return make_longlong2(est, base);
}

template <typename Off>
struct Params {
    const Off *rp;
    const int *ci;
    long long n, m;
    int *core;                    // output: coreness, written at the end
    VRec<Off> *vinfo;             // n records {estimate, histogram base}
    int2 *mv[2];                  // per round parity: {old, new} estimate of the vertices
                                  // changed in that round, {0, 0} for the others
    unsigned *mvp[2] = {nullptr, nullptr};   // the same records packed (kMvpWide: read mv),
                                             // 0 for the others; nullptr: pull rounds read mv
    int *histo;                   // m slots (zeroed by run() when zero_histo)
    int *tl[2], *wl[2], *bl[2];   // V_cnt lists by class, per parity (n slots each)
    int *us;                      // changed vertices of small degree
    int2 *ub;                     // chunks of changed vertices of large degree
    int2 *ib;                     // chunks of every vertex of large degree (InitHisto and
                                  // pull rounds; nullptr: InitHisto uses ub, never pull)
    unsigned ub_cap;              // entries of ub, and of ib
    Ctrl *ctl;                    // status word (errors)
    bool zero_histo;
    Tuning tn;
    // Start from min(init_est[v], deg v), at least 1, instead of the degrees
    // (core maintenance); nullptr: the degrees, as Alg. 6. From any start the rounds
    // end with cnt >= estimate everywhere, so the estimates are then a lower
    // bound of the coreness, and the coreness itself when the start is an
    // upper bound of it.
    const int *init_est = nullptr;
    // Marks of the rows whose cnt slot a pull round decremented (n bytes,
    // rounded up to 4; zero between rounds); nullptr: pull rounds decide the
    // append at the edit, as push rounds do.
    unsigned char *cand = nullptr;
};

// Packed {old, new} record: old << 16 | new when old <= 65534 (new < old);
// kMvpWide otherwise (never a packed value, since new < old).
constexpr unsigned kMvpWide = 0xffffffffu;
__device__ __forceinline__ unsigned pack_mv(int x, int y)
{
    return x <= 0xfffe ? ((unsigned)x << 16) | (unsigned)y : kMvpWide;
}

__device__ __forceinline__ int kclass(int K) { return K <= kWarpK ? 0 : (K <= kBlockK ? 1 : 2); }

template <typename Off>
struct InitArc {
    static constexpr int kArcs = 4;
    const VRec<Off> *vinfo;
    int *histo;
    unsigned long long n_arcs = 0;
    __device__ __forceinline__ bool item(int v, int &a, int &)
    {
        a = (int)__ldcg(vinfo + v).x;
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&rs)[kArcs],
                                         const int (&dv)[kArcs], const int (&)[kArcs])
    {
        int du[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) du[j] = valid[j] ? (int)__ldca(vinfo + u[j]).x : 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            if (valid[j]) {
                ++n_arcs;
                red_add(histo + rs[j] + (du[j] < dv[j] ? du[j] : dv[j]) - 1, 1);
            }
    }
};

// Appends the vertices whose cnt fell below their estimate to the next
// V_cnt, by the class of the estimate K (one aggregated append per class).
template <int U>
__device__ __forceinline__ void append_vcnt(const bool (&push)[U], const int (&vtx)[U],
                                            const int (&K)[U], unsigned *live, int *tl, int *wl,
                                            int *bl, unsigned cap, Ctrl *ctl)
{
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const int cls = kclass(K[j]);
        const unsigned p0 = warp_push(&live[L_T], push[j] && cls == 0);
        const unsigned p1 = warp_push(&live[L_W], push[j] && cls == 1);
        const unsigned p2 = warp_push(&live[L_B], push[j] && cls == 2);
        if (push[j]) {
            const unsigned pos = cls == 0 ? p0 : (cls == 1 ? p1 : p2);
            if (pos >= cap) set_error(ctl, kErrNotConverged);
            else if (cls == 0) tl[pos] = vtx[j];
            else if (cls == 1) wl[pos] = vtx[j];
            else bl[pos] = vtx[j];
        }
    }
}

// The edits of one arc between a changed vertex (estimate x -> y) and a vertex
// u with estimate K and histogram row ru (types N1 and N3 of Sec. IV-B: only
// when K > y). Returns true when u's cnt fell below K by this edit.
template <typename Off>
__device__ __forceinline__ bool edit_row(int *histo, Off ru, int K, int x, int y,
                                         unsigned long long &n_atomics)
{
    if (K <= y) return false;
    n_atomics += 2;
    red_add(histo + ru + y - 1, 1);
    if (x >= K)   // slot K holds cnt: its old value decides the append
        return atomicSub(histo + ru + K - 1, 1) == K;
    red_add(histo + ru + x - 1, -1);   // slot x < K: no append can follow
    return false;
}

// Push form of UpdateHisto: arcs of the changed vertices.
template <typename Off>
struct UpdateArc {
    static constexpr int kArcs = 4;
    const VRec<Off> *vinfo;
    const int2 *mv;        // {old, new} estimates of this round
    int *histo;
    int *tl, *wl, *bl;
    Ctrl *ctl;
    unsigned *live_base;   // counters of the domain
    int par;               // parity of the next round's lists
    unsigned cap;          // slots of each list (n)
    unsigned long long n_arcs = 0, n_atomics = 0;

    __device__ __forceinline__ bool item(int v, int &x, int &y)
    {
        const int2 r = __ldcg(mv + v);
        x = r.x;
        y = r.y;
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&x)[kArcs], const int (&y)[kArcs])
    {
        int K[kArcs];
        Off ru[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            VRec<Off> r = make_vrec<Off>(0, 0);
            if (valid[j]) r = __ldca(vinfo + u[j]);
            K[j] = (int)r.x;
            ru[j] = (Off)r.y;
        }
        bool push[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            push[j] = false;
            if (valid[j]) {
                ++n_arcs;
                push[j] = edit_row(histo, ru[j], K[j], x[j], y[j], n_atomics);
            }
        }
        append_vcnt(push, u, K, live_base + 3 * par, tl, wl, bl, cap, ctl);
    }
};

// Pull form of UpdateHisto: arcs of every vertex u whose estimate K is above
// the smallest new estimate of the round; the edit of arc (u, w) is the one
// w's push would make to u's row, when w changed in this round.
template <typename Off>
struct PullArc {
    static constexpr int kArcs = 4;
    const VRec<Off> *vinfo;
    const int2 *mv;        // {old, new} estimates of this round ({0, 0}: unchanged)
    int *histo;
    int *tl, *wl, *bl;
    Ctrl *ctl;
    unsigned *live_base;
    int par;
    unsigned cap;
    int ymin;              // no row with K <= ymin can be edited
    unsigned char *cand;   // row marks of the deferred V_cnt decision (nullptr: decide here)
    const unsigned *mvp;   // packed records of this round (nullptr: gather mv)
    unsigned long long n_arcs = 0, n_atomics = 0;

    __device__ __forceinline__ bool item(int u, int &K, int &)
    {
        K = (int)__ldcg(vinfo + u).x;
        return K > ymin;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&uu)[kArcs],
                                         const int (&w)[kArcs], const Off (&ru)[kArcs],
                                         const int (&K)[kArcs], const int (&)[kArcs])
    {
        int2 r[kArcs];
        if (mvp) {
            unsigned q[kArcs];
#pragma unroll
            for (int j = 0; j < kArcs; ++j) q[j] = valid[j] ? __ldca(mvp + w[j]) : 0u;
#pragma unroll
            for (int j = 0; j < kArcs; ++j)
                r[j] = q[j] == kMvpWide ? __ldcg(mv + w[j])
                                        : make_int2((int)(q[j] >> 16), (int)(q[j] & 0xffffu));
        } else {
#pragma unroll
            for (int j = 0; j < kArcs; ++j) r[j] = valid[j] ? __ldcg(mv + w[j]) : make_int2(0, 0);
        }
        if (cand) {   // reductions only; rows whose slot K fell are listed after the barrier
#pragma unroll
            for (int j = 0; j < kArcs; ++j) {
                if (!valid[j]) continue;
                ++n_arcs;
                const int x = r[j].x, y = r[j].y;
                if (x == 0 || K[j] <= y) continue;
                n_atomics += 2;
                red_add(histo + ru[j] + y - 1, 1);
                red_add(histo + ru[j] + (x < K[j] ? x : K[j]) - 1, -1);
                if (x >= K[j]) cand[uu[j]] = 1;
            }
            return;
        }
        bool push[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            push[j] = false;
            if (valid[j]) {
                ++n_arcs;
                if (r[j].x != 0) push[j] = edit_row(histo, ru[j], K[j], r[j].x, r[j].y, n_atomics);
            }
        }
        append_vcnt(push, uu, K, live_base + 3 * par, tl, wl, bl, cap, ctl);
    }
};

// Deferred V_cnt decision of a pull round (after its barrier): every marked
// row u with histo[u][K] < K joins V_cnt of parity np; the marks are cleared.
// Each thread takes 4 vertices (one 32-bit word of marks) per step; the up to
// 3 padding bytes past n are never set by an edit and only cleared here.
template <typename Off>
__device__ __forceinline__ void collect_vcnt(const Params<Off> &p, unsigned *live, int np,
                                             unsigned tid, unsigned nthreads)
{
    const unsigned lane = threadIdx.x & 31;
    const long long n = p.n, ngroups = (n + 3) >> 2;
    unsigned *const words = reinterpret_cast<unsigned *>(p.cand);
    for (long long base = (long long)(tid - lane); base < ngroups; base += nthreads) {
        const long long g = base + lane;
        const unsigned marks = g < ngroups ? __ldcg(words + g) : 0u;
        if (!__any_sync(kFull, marks != 0u)) continue;
        if (marks) words[g] = 0u;
        bool in[4];
        int vtx[4], K[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            vtx[j] = (int)(4 * g + j);
            in[j] = false;
            K[j] = 0;
            if (vtx[j] < n && ((marks >> (8 * j)) & 0xffu)) {   // the padding is never a row
                const VRec<Off> rec = __ldcg(p.vinfo + vtx[j]);
                K[j] = (int)rec.x;
                in[j] = ldcg(p.histo + (Off)rec.y + K[j] - 1) < K[j];
            }
        }
        append_vcnt(in, vtx, K, live + 3 * np, p.tl[np], p.wl[np], p.bl[np], (unsigned)n, p.ctl);
    }
}

// Per-thread totals of the vertices a thread changed in SumHisto.
struct RoundAcc {
    unsigned long long arcs = 0;   // their degrees
    int ymin = INT_MAX;            // their smallest new estimate
};

// Records the result of SumHisto for v (estimate K -> h) in round parity
// par. Returns the degree of v, or -1 when v did not change (impossible on a
// valid graph by Thm. 2).
template <typename Off>
__device__ __forceinline__ long long sum_apply(const Params<Off> &p, int par, int v, Off rs, int K,
                                               int h, int sum, RoundAcc &acc)
{
    if (h >= K || h < 1) {
        set_error(p.ctl, kErrBadGraph);
        return -1;
    }
    p.vinfo[v].x = h;
    p.mv[par][v] = make_int2(K, h);
    if (p.mvp[par]) p.mvp[par][v] = pack_mv(K, h);
    p.histo[rs + h - 1] = sum;
    const long long d = (long long)(p.rp[v + 1] - rs);
    acc.arcs += (unsigned long long)d;
    acc.ymin = h < acc.ymin ? h : acc.ymin;
    return d;
}

// Lists a changed vertex of small degree d for UpdateHisto; a larger one is
// listed by its chunks, which the caller's warp or CTA writes together.
template <typename Off>
__device__ __forceinline__ void list_small(const Params<Off> &p, unsigned *live, int v,
                                           long long d)
{
    if (d < 0 || d > p.tn.small_deg) return;
    const unsigned pos = atomicAdd(&live[L_US], 1u);
    if (pos < (unsigned)p.n) p.us[pos] = v;
    else set_error(p.ctl, kErrNotConverged);
}

// Slots each thread reads per step of a warp or CTA walk (consecutive,
// descending): a warp step covers 4 x 32 slots, a CTA step 8 x 512.
constexpr int kWalkSlots = 4;
constexpr int kBlockWalkSlots = 8;

// SumHisto by one CTA for a vertex with a large estimate.
template <typename Off>
__device__ void sum_block(const Params<Off> &p, int par, unsigned *live, int v, int *s,
                          unsigned long long &slots, RoundAcc &acc)
{
    const VRec<Off> rec = __ldcg(p.vinfo + v);
    const Off rs = (Off)rec.y;
    const int K = (int)rec.x;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int carry = 0;
    for (int top = K; top >= 1; top -= kBlockWalkSlots * (int)blockDim.x) {
        const int s0 = top - kBlockWalkSlots * (int)threadIdx.x;   // this thread: s0, s0 - 1, ...
        int r[kBlockWalkSlots], t = 0;
#pragma unroll
        for (int j = 0; j < kBlockWalkSlots; ++j) {
            const int slot = s0 - j;
            t += slot >= 1 ? ldcg(p.histo + rs + slot - 1) : 0;
            r[j] = t;
        }
        int inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, inc, o);
            if ((int)lane >= o) inc += y;
        }
        if (lane == 31) s[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int x = lane < nw ? s[lane] : 0;
            int wi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, wi, o);
                if ((int)lane >= o) wi += y;
            }
            if (lane < nw) s[32 + lane] = wi - x;
            if (lane == 0) s[64] = INT_MAX;
        }
        __syncthreads();
        const int before = carry + s[32 + warp] + inc - t;   // slots above s0
        int found = INT_MAX, frun = 0;
#pragma unroll
        for (int j = kBlockWalkSlots - 1; j >= 0; --j)
            if (s0 - j >= 1 && before + r[j] >= s0 - j) {
                found = kBlockWalkSlots * (int)threadIdx.x + j;
                frun = before + r[j];
            }
        if (found != INT_MAX) atomicMin(&s[64], found);
        __syncthreads();
        const int first = s[64];   // the highest slot that qualifies
        if (first != INT_MAX) {
            if (first == found) {
                const int slot = s0 - first % kBlockWalkSlots;
                slots += (unsigned long long)(K - slot + 1);
                const long long d = sum_apply(p, par, v, rs, K, slot, frun, acc);
                list_small(p, live, v, d);
                unsigned nch = 0, pos = 0;
                if (d > p.tn.small_deg) {   // the CTA writes the chunk entries
                    nch = (unsigned)((d + p.tn.chunk - 1) / p.tn.chunk);
                    pos = atomicAdd(&live[L_UB], nch);
                    if ((unsigned long long)pos + nch > p.ub_cap) {
                        set_error(p.ctl, kErrNotConverged);
                        nch = 0;
                    }
                }
                s[65] = (int)nch;
                s[66] = (int)pos;
            }
            __syncthreads();
            const unsigned nch = (unsigned)s[65], pos = (unsigned)s[66];
            for (unsigned c = threadIdx.x; c < nch; c += blockDim.x)
                p.ub[pos + c] = make_int2(v, (int)c);
            __syncthreads();
            return;
        }
        carry += s[32 + nw - 1] + s[nw - 1];   // total of this tile
        __syncthreads();
    }
    if (threadIdx.x == 0) set_error(p.ctl, kErrBadGraph);   // sum never reached k
}

// SumHisto by one warp for a vertex with a medium estimate.
template <typename Off>
__device__ __forceinline__ void sum_warp(const Params<Off> &p, int par, unsigned *live, int v,
                                         unsigned long long &slots, RoundAcc &acc)
{
    const int lane = threadIdx.x & 31;
    const VRec<Off> rec = __ldcg(p.vinfo + v);
    const Off rs = (Off)rec.y;
    const int K = (int)rec.x;
    int carry = 0;
    for (int top = K; top >= 1; top -= 32 * kWalkSlots) {
        const int s0 = top - kWalkSlots * lane;   // this lane: s0, s0 - 1, ...
        int r[kWalkSlots], t = 0;
#pragma unroll
        for (int j = 0; j < kWalkSlots; ++j) {
            const int slot = s0 - j;
            t += slot >= 1 ? ldcg(p.histo + rs + slot - 1) : 0;
            r[j] = t;
        }
        int inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const int before = carry + inc - t;   // slots above s0
        int found = kWalkSlots, frun = 0;
#pragma unroll
        for (int j = kWalkSlots - 1; j >= 0; --j)
            if (s0 - j >= 1 && before + r[j] >= s0 - j) {
                found = j;
                frun = before + r[j];
            }
        const unsigned b = __ballot_sync(kFull, found < kWalkSlots);
        if (b) {
            const int L = __ffs(b) - 1;   // the lowest lane holds the highest slots
            long long d = -1;
            if (lane == L) {
                const int slot = s0 - found;
                slots += (unsigned long long)(K - slot + 1);
                d = sum_apply(p, par, v, rs, K, slot, frun, acc);
                list_small(p, live, v, d);
            }
            warp_push_chunks(lane == L && d > p.tn.small_deg, v, d, p.ub, &live[L_UB], p.ub_cap,
                             p.ctl, p.tn.chunk);
            return;
        }
        carry += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) set_error(p.ctl, kErrBadGraph);
}

// SumHisto by one thread for a vertex with a small estimate; returns the
// vertex degree (or -1, see sum_apply).
template <typename Off>
__device__ __forceinline__ long long sum_thread(const Params<Off> &p, int par, int v,
                                                unsigned long long &slots, RoundAcc &acc)
{
    const VRec<Off> rec = __ldcg(p.vinfo + v);
    const Off rs = (Off)rec.y;
    const int K = (int)rec.x;
    int sum = 0, k = K;
    for (; k >= 1; --k) {
        sum += ldcg(p.histo + rs + k - 1);
        if (sum >= k) break;
    }
    slots += (unsigned long long)(K - k + 1);
    return sum_apply(p, par, v, rs, K, k, sum, acc);
}

// Whether UpdateHisto of this round pulls (see the direction note above);
// vol: arcs of the round's changed vertices. Uniform over the domain.
template <typename Off>
__device__ __forceinline__ bool pull_round(const Params<Off> &p, unsigned long long vol)
{
    if (p.ib == nullptr || p.tn.update_mode == kUpdatePush) return false;
    if (p.tn.update_mode == kUpdatePull) return true;
    return p.m >= kPullMinArcs &&
           vol * 100ull >= (unsigned long long)p.tn.pull_pct * (unsigned long long)p.m;
}

// Adds the warp's round totals to the domain's counters (lane 0 of each warp).
__device__ __forceinline__ void fold_round(const RoundAcc &acc, unsigned *live)
{
    unsigned long long a = acc.arcs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(kFull, a, o);
    const int ym = __reduce_min_sync(kFull, acc.ymin);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(reinterpret_cast<unsigned long long *>(&live[L_VOL]), a);
        if (ym != INT_MAX) atomicMax(&live[L_YMIN], (unsigned)(INT_MAX - ym));
    }
}

// HistoCore on one graph. Every thread of the domain calls it. st: per-CTA
// statistics in shared memory (thread 0 writes); s_tmp: >= 256 shared words.
// arcs counts InitHisto's arcs plus the arcs of every round's changed vertices
// (the arcs Alg. 6 scans, whatever the direction); pulled counts the arcs
// that pull rounds scanned.
template <typename Off, typename Dom>
__device__ void run(const Params<Off> &p0, Dom &dom, unsigned *s_tmp, unsigned long long *st,
                    PhaseClock &clk, unsigned long long &arcs, unsigned long long &atomics,
                    unsigned long long &slots, unsigned long long &pulled)
{
    const Params<Off> &p = p0;
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const long long n = p.n;
    const long long first = (long long)dom.cta() * blockDim.x;
    int2 *const ilist = p.ib ? p.ib : p.ub;   // chunks of every large vertex

    if (p.zero_histo) {
        for (long long i = first + threadIdx.x; i < p.m; i += nthreads) p.histo[i] = 0;
    }
    // core = degree; no vertex changed yet; chunk list of the large vertices
    for (long long base = first; base < n; base += nthreads) {
        const long long v = base + threadIdx.x;
        long long d = 0;
        if (v < n) {
            const Off r0 = p.rp[v];
            d = (long long)(p.rp[v + 1] - r0);
            int e0 = (int)d;
            if (p.init_est && d > 0) {   // a non-isolated vertex has coreness >= 1
                const int x = ldcg(p.init_est + v);
                e0 = x < 1 ? 1 : (x < e0 ? x : e0);
            }
            p.vinfo[v] = make_vrec<Off>(e0, r0);
            p.mv[0][v] = make_int2(0, 0);
            p.mv[1][v] = make_int2(0, 0);
            if (p.mvp[0]) {
                p.mvp[0][v] = 0u;
                p.mvp[1][v] = 0u;
            }
            if (p.cand) p.cand[v] = 0;
        }
        const unsigned nch =
            d > p.tn.small_deg ? (unsigned)((d + p.tn.chunk - 1) / p.tn.chunk) : 0u;
        const unsigned pos = block_alloc(nch, &live[L_IB], s_tmp);
        const bool fits = (unsigned long long)pos + nch <= p.ub_cap;
        if (nch && !fits) set_error(ctl, kErrNotConverged);
        warp_fill_chunks(fits ? nch : 0u, pos, (int)v, ilist);
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    if (Dom::kGrid) clk.end(st, kPhInit);
    const unsigned nib = snap[L_IB];

    // InitHisto
    {
        InitArc<Off> f{p.vinfo, p.histo};
        expand(p.rp, p.ci, (const int *)nullptr, (unsigned)n, ilist, nib, gwarp, nwarps, f, p.tn);
        arcs += f.n_arcs;
        atomics += f.n_arcs;
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    if (Dom::kGrid) clk.end(st, kPhInitHisto);

    // initial V_cnt (parity 0)
    for (long long base = first; base < n; base += nthreads) {
        const long long v = base + threadIdx.x;
        bool in[3] = {false, false, false};
        if (v < n) {
            const VRec<Off> rec = __ldcg(p.vinfo + v);
            const int d = (int)rec.x;
            if (d >= 1 && ldcg(p.histo + (Off)rec.y + d - 1) < d) in[kclass(d)] = true;
        }
        unsigned *const ctr[3] = {&live[L_T], &live[L_W], &live[L_B]};
        unsigned pos[3];
        block_pushN<3>(in, ctr, pos, s_tmp);
        if (in[0]) p.tl[0][pos[0]] = (int)v;
        if (in[1]) p.wl[0][pos[1]] = (int)v;
        if (in[2]) p.bl[0][pos[2]] = (int)v;
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    if (Dom::kGrid) clk.end(st, kPhInit);

    const long long max_rounds = p.m + 2;
    unsigned pt = 0, pw = 0, pb = 0;   // V_cnt sizes of the previous round
    for (long long r = 0;; ++r) {
        const int par = (int)(r & 1), np = 1 - par;
        const unsigned nt = snap[3 * par + L_T], nwl = snap[3 * par + L_W],
                       nb = snap[3 * par + L_B];
        if (nt + nwl + nb == 0) break;
        if (r >= max_rounds) {
            if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
            return;
        }
        if (threadIdx.x == 0) {
            ++st[kStRounds];
            st[kStFrontier] += nt + nwl + nb;
        }
        if (dom.leader()) {
            live[3 * np + L_T] = 0;
            live[3 * np + L_W] = 0;
            live[3 * np + L_B] = 0;
        }
        // the previous round's changed vertices are not changed in this one:
        // clear their entries of the other parity (read by nobody until the
        // next round's UpdateHisto; their lists are intact until this round's)
        for (long long i = first + threadIdx.x; i < (long long)pt + pw + pb; i += nthreads) {
            const unsigned k = (unsigned)i;
            const int v = k < pt ? ldcg(p.tl[np] + k)
                                 : (k < pt + pw ? ldcg(p.wl[np] + (k - pt))
                                                : ldcg(p.bl[np] + (k - pt - pw)));
            p.mv[np][v] = make_int2(0, 0);
            if (p.mvp[np]) p.mvp[np][v] = 0u;
        }
        // SumHisto: CTA items, then warp items, then thread items
        RoundAcc acc;
        for (unsigned i = dom.cta(); i < nb; i += dom.ncta())
            sum_block(p, par, live, ldcg(p.bl[par] + i), (int *)s_tmp, slots, acc);
        for (unsigned i = gwarp; i < nwl; i += nwarps)
            sum_warp(p, par, live, ldcg(p.wl[par] + i), slots, acc);
        for (long long base = first; base < nt; base += nthreads) {
            const long long i = base + threadIdx.x;
            int v = 0;
            long long d = -1;
            if (i < nt) {
                v = ldcg(p.tl[par] + i);
                d = sum_thread(p, par, v, slots, acc);
            }
            const bool small = d >= 0 && d <= p.tn.small_deg;
            unsigned pos, unused;
            block_push2(small, false, &live[L_US], &live[L_US], pos, unused, s_tmp);
            if (small) {
                if (pos < (unsigned)n) p.us[pos] = v;
                else set_error(ctl, kErrNotConverged);
            }
            warp_push_chunks(d > p.tn.small_deg, v, d, p.ub, &live[L_UB], p.ub_cap, ctl,
                             p.tn.chunk);
        }
        fold_round(acc, live);
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        if (Dom::kGrid) clk.end(st, kPhSumHisto, nt + nwl + nb);
        pt = nt;
        pw = nwl;
        pb = nb;

        // UpdateHisto over the changed vertices, pushed or pulled
        const unsigned nus = snap[L_US], nub = snap[L_UB];
        const unsigned long long vol =
            (unsigned long long)snap[L_VOL] | ((unsigned long long)snap[L_VOL + 1] << 32);
        const int ymin = INT_MAX - (int)snap[L_YMIN];
        if (dom.leader()) {
            live[L_US] = 0;
            live[L_UB] = 0;
            live[L_YMIN] = 0;
            live[L_VOL] = 0;
            live[L_VOL + 1] = 0;
        }
        const bool pull = pull_round(p, vol);
        if (pull) {
            PullArc<Off> f{p.vinfo, p.mv[par], p.histo, p.tl[np], p.wl[np], p.bl[np],
                           ctl,     live,      np,      (unsigned)n, ymin,    p.cand,
                           p.mvp[par]};
            expand(p.rp, p.ci, (const int *)nullptr, (unsigned)n, ilist, nib, gwarp, nwarps, f,
                   p.tn, batch_width((unsigned)n, nib, nwarps));
            arcs += acc.arcs;
            pulled += f.n_arcs;
            atomics += f.n_atomics;
            if (threadIdx.x == 0) ++st[kStPullRounds];
            if (p.cand) {   // all edits in place: list the rows whose cnt fell below K
                if (!dom.sync()) return;
                if (threadIdx.x == 0) ++st[kStBarriers];
                collect_vcnt(p, live, np, tid, nthreads);
            }
        } else {
            UpdateArc<Off> f{p.vinfo, p.mv[par], p.histo, p.tl[np], p.wl[np], p.bl[np],
                             ctl,     live,      np,      (unsigned)n};
            expand(p.rp, p.ci, p.us, nus, p.ub, nub, gwarp, nwarps, f, p.tn,
                   batch_width(nus, nub, nwarps));
            arcs += f.n_arcs;
            atomics += f.n_atomics;
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        if (Dom::kGrid) clk.end(st, pull ? kPhUpdatePull : kPhUpdateHisto, pull ? (unsigned)n : nus + nub);
    }
    // the estimates are the coreness now (no vertex has cnt < estimate)
    for (long long v = first + threadIdx.x; v < n; v += nthreads) p.core[v] = (int)__ldcg(p.vinfo + v).x;
}

}  // namespace histo
}  // namespace pico
