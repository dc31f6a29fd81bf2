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
//               oldcore[v] <- core_old, histo[v][k] <- sum (the new cnt).
//               By Thm. 2 every vertex of V_cnt changes.
//   UpdateHisto for changed v (x = oldcore[v], y = core[v]) and neighbour u
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

// live counters: V_cnt lists (T/W/B) per round parity, update lists, init chunks
enum : int { L_T = 0, L_W = 1, L_B = 2, /* parity 1: 3..5 */ L_US = 6, L_UB = 7, L_IB = 8 };

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
    int *oldcore;
    int *histo;                   // m slots (zeroed by run() when zero_histo)
    int *tl[2], *wl[2], *bl[2];   // V_cnt lists by class, per parity (n slots each)
    int *us;                      // changed vertices of small degree
    int2 *ub;                     // chunks of changed vertices of large degree
    unsigned ub_cap;
    Ctrl *ctl;                    // status word (errors)
    bool zero_histo;
    Tuning tn;
};

__device__ __forceinline__ int kclass(int K) { return K <= kWarpK ? 0 : (K <= kBlockK ? 1 : 2); }

template <typename Off>
struct InitArc {
    static constexpr int kArcs = 4;
    const VRec<Off> *vinfo;
    int *histo;
    unsigned long long n_arcs = 0;
    __device__ __forceinline__ void item(int v, int &a, int &) { a = (int)__ldcg(vinfo + v).x; }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&rs)[kArcs],
                                         const int (&dv)[kArcs], const int (&)[kArcs])
    {
        int du[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) du[j] = valid[j] ? (int)__ldcg(vinfo + u[j]).x : 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            if (valid[j]) {
                ++n_arcs;
                red_add(histo + rs[j] + (du[j] < dv[j] ? du[j] : dv[j]) - 1, 1);
            }
    }
};

template <typename Off>
struct UpdateArc {
    static constexpr int kArcs = 4;
    const VRec<Off> *vinfo;
    const int *oldcore;
    int *histo;
    int *tl, *wl, *bl;
    Ctrl *ctl;
    unsigned *live_base;   // counters of the domain
    int par;               // parity of the next round's lists
    unsigned cap;          // slots of each list (n)
    unsigned long long n_arcs = 0, n_atomics = 0;

    __device__ __forceinline__ void item(int v, int &x, int &y)
    {
        x = ldcg(oldcore + v);
        y = (int)__ldcg(vinfo + v).x;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const Off (&)[kArcs],
                                         const int (&x)[kArcs], const int (&y)[kArcs])
    {
        int K[kArcs], old[kArcs];
        Off ru[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            VRec<Off> r = make_vrec<Off>(0, 0);
            if (valid[j]) r = __ldcg(vinfo + u[j]);
            K[j] = (int)r.x;
            ru[j] = (Off)r.y;
        }
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            old[j] = 0;
            if (valid[j]) {
                ++n_arcs;
                if (K[j] > y[j]) {   // types N1 and N3: the change is visible to u
                    if (x[j] >= K[j]) {   // slot K holds cnt: its old value decides the append
                        old[j] = atomicSub(histo + ru[j] + K[j] - 1, 1);
                    } else {              // slot x < K: no append can follow
                        red_add(histo + ru[j] + x[j] - 1, -1);
                    }
                    red_add(histo + ru[j] + y[j] - 1, 1);
                    n_atomics += 2;
                }
            }
        }
        unsigned *live = live_base + 3 * par;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            const bool push = valid[j] && K[j] > y[j] && x[j] >= K[j] && old[j] == K[j];
            const int cls = kclass(K[j]);
            const unsigned p0 = warp_push(&live[L_T], push && cls == 0);
            const unsigned p1 = warp_push(&live[L_W], push && cls == 1);
            const unsigned p2 = warp_push(&live[L_B], push && cls == 2);
            if (push) {
                const unsigned pos = cls == 0 ? p0 : (cls == 1 ? p1 : p2);
                if (pos >= cap) set_error(ctl, kErrNotConverged);
                else if (cls == 0) tl[pos] = u[j];
                else if (cls == 1) wl[pos] = u[j];
                else bl[pos] = u[j];
            }
        }
    }
};

// Records the result of SumHisto for v. Returns the degree of v, or -1 when
// v did not change (impossible on a valid graph by Thm. 2).
template <typename Off>
__device__ __forceinline__ long long sum_apply(const Params<Off> &p, int v, Off rs, int K,
                                               int h, int sum)
{
    if (h >= K || h < 1) {
        set_error(p.ctl, kErrBadGraph);
        return -1;
    }
    p.vinfo[v].x = h;
    p.oldcore[v] = K;
    p.histo[rs + h - 1] = sum;
    return (long long)(p.rp[v + 1] - rs);
}

// Lists a changed vertex of degree d for UpdateHisto (single-thread path).
template <typename Off>
__device__ __forceinline__ void list_changed(const Params<Off> &p, unsigned *live, int v,
                                             long long d)
{
    if (d < 0) return;
    if (d <= p.tn.small_deg) {
        const unsigned pos = atomicAdd(&live[L_US], 1u);
        if (pos < (unsigned)p.n) p.us[pos] = v;
        else set_error(p.ctl, kErrNotConverged);
    } else if (!push_chunks(v, d, p.ub, &live[L_UB], p.ub_cap, p.tn.chunk)) {
        set_error(p.ctl, kErrNotConverged);
    }
}

template <typename Off>
__device__ __forceinline__ void sum_done(const Params<Off> &p, unsigned *live, int v, Off rs,
                                         int K, int h, int sum)
{
    list_changed(p, live, v, sum_apply(p, v, rs, K, h, sum));
}

// SumHisto by one CTA for a vertex with a large estimate.
template <typename Off>
__device__ void sum_block(const Params<Off> &p, unsigned *live, int v, int *s,
                          unsigned long long &slots)
{
    const VRec<Off> rec = __ldcg(p.vinfo + v);
    const Off rs = (Off)rec.y;
    const int K = (int)rec.x;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int carry = 0;
    for (int top = K; top >= 1; top -= (int)blockDim.x) {
        const int slot = top - (int)threadIdx.x;
        const int val = slot >= 1 ? ldcg(p.histo + rs + slot - 1) : 0;
        int inc = val;
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
        const int run = carry + s[32 + warp] + inc;
        if (slot >= 1 && run >= slot) atomicMin(&s[64], (int)threadIdx.x);
        __syncthreads();
        const int first = s[64];
        if (first != INT_MAX) {
            if ((int)threadIdx.x == first) {
                slots += (unsigned long long)(K - slot + 1);
                sum_done(p, live, v, rs, K, slot, run);
            }
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
__device__ __forceinline__ void sum_warp(const Params<Off> &p, unsigned *live, int v,
                                         unsigned long long &slots)
{
    const int lane = threadIdx.x & 31;
    const VRec<Off> rec = __ldcg(p.vinfo + v);
    const Off rs = (Off)rec.y;
    const int K = (int)rec.x;
    int carry = 0;
    for (int top = K; top >= 1; top -= 32) {
        const int slot = top - lane;
        const int val = slot >= 1 ? ldcg(p.histo + rs + slot - 1) : 0;
        int inc = val;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const int run = carry + inc;
        const unsigned b = __ballot_sync(kFull, slot >= 1 && run >= slot);
        if (b) {
            const int L = __ffs(b) - 1;
            if (lane == L) {
                slots += (unsigned long long)(K - slot + 1);
                sum_done(p, live, v, rs, K, slot, run);
            }
            return;
        }
        carry = __shfl_sync(kFull, run, 31);
    }
    if (lane == 0) set_error(p.ctl, kErrBadGraph);
}

// SumHisto by one thread for a vertex with a small estimate; returns the
// vertex degree (or -1, see sum_apply).
template <typename Off>
__device__ __forceinline__ long long sum_thread(const Params<Off> &p, int v,
                                                unsigned long long &slots)
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
    return sum_apply(p, v, rs, K, k, sum);
}

// HistoCore on one graph. Every thread of the domain calls it. st: per-CTA
// statistics in shared memory (thread 0 writes); s_tmp: >= 256 shared words.
template <typename Off, typename Dom>
__device__ void run(const Params<Off> &p0, Dom &dom, unsigned *s_tmp, unsigned long long *st,
                    PhaseClock &clk, unsigned long long &arcs, unsigned long long &atomics,
                    unsigned long long &slots)
{
    const Params<Off> &p = p0;
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const long long n = p.n;
    const long long first = (long long)dom.cta() * blockDim.x;

    if (p.zero_histo) {
        for (long long i = first + threadIdx.x; i < p.m; i += nthreads) p.histo[i] = 0;
    }
    // core = degree; chunk list of the large vertices for InitHisto
    for (long long base = first; base < n; base += nthreads) {
        const long long v = base + threadIdx.x;
        long long d = 0;
        if (v < n) {
            const Off r0 = p.rp[v];
            d = (long long)(p.rp[v + 1] - r0);
            p.vinfo[v] = make_vrec<Off>((int)d, r0);
        }
        const unsigned nch =
            d > p.tn.small_deg ? (unsigned)((d + p.tn.chunk - 1) / p.tn.chunk) : 0u;
        const unsigned pos = block_alloc(nch, &live[L_IB], s_tmp);
        if (nch && (unsigned long long)pos + nch <= p.ub_cap)
            for (unsigned c = 0; c < nch; ++c) p.ub[pos + c] = make_int2((int)v, (int)c);
        else if (nch)
            set_error(ctl, kErrNotConverged);
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    if (Dom::kGrid) clk.end(st, kPhInit);

    // InitHisto
    {
        InitArc<Off> f{p.vinfo, p.histo};
        expand(p.rp, p.ci, (const int *)nullptr, (unsigned)n, p.ub, snap[L_IB], gwarp, nwarps, f,
               p.tn);
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
    for (long long r = 0;; ++r) {
        const int par = (int)(r & 1);
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
            const int np = 1 - par;
            live[3 * np + L_T] = 0;
            live[3 * np + L_W] = 0;
            live[3 * np + L_B] = 0;
        }
        // SumHisto: CTA items, then warp items, then thread items
        for (unsigned i = dom.cta(); i < nb; i += dom.ncta())
            sum_block(p, live, ldcg(p.bl[par] + i), (int *)s_tmp, slots);
        for (unsigned i = gwarp; i < nwl; i += nwarps) sum_warp(p, live, ldcg(p.wl[par] + i), slots);
        for (long long base = first; base < nt; base += nthreads) {
            const long long i = base + threadIdx.x;
            int v = 0;
            long long d = -1;
            if (i < nt) {
                v = ldcg(p.tl[par] + i);
                d = sum_thread(p, v, slots);
            }
            const bool small = d >= 0 && d <= p.tn.small_deg;
            unsigned pos, unused;
            block_push2(small, false, &live[L_US], &live[L_US], pos, unused, s_tmp);
            if (small) {
                if (pos < (unsigned)n) p.us[pos] = v;
                else set_error(ctl, kErrNotConverged);
            }
            if (d > p.tn.small_deg) list_changed(p, live, v, d);
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        if (Dom::kGrid) clk.end(st, kPhSumHisto, nt + nwl + nb);

        // UpdateHisto over the changed vertices
        const unsigned nus = snap[L_US], nub = snap[L_UB];
        if (dom.leader()) {
            live[L_US] = 0;
            live[L_UB] = 0;
        }
        {
            const int np = 1 - par;
            UpdateArc<Off> f{p.vinfo, p.oldcore, p.histo, p.tl[np], p.wl[np], p.bl[np],
                             ctl,     live,      np,      (unsigned)n};
            expand(p.rp, p.ci, p.us, nus, p.ub, nub, gwarp, nwarps, f, p.tn,
                   batch_width(nus, nub, nwarps));
            arcs += f.n_arcs;
            atomics += f.n_atomics;
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        if (Dom::kGrid) clk.end(st, kPhUpdateHisto, nus + nub);
    }
    // the estimates are the coreness now (no vertex has cnt < estimate)
    for (long long v = first + threadIdx.x; v < n; v += nthreads) p.core[v] = (int)__ldcg(p.vinfo + v).x;
}

}  // namespace histo
}  // namespace pico
