// Device-side building blocks shared by the PeelOne and HistoCore kernels.
//
// * Ctrl: the per-call control block (grid barrier, status word, live
//   counters and their per-barrier snapshots, statistics).
// * grid_sync: a bounded grid-wide barrier for persistent cooperative
//   launches. The last CTA to arrive copies the live counters into a snapshot
//   before releasing the others, so every CTA sees the same counter values
//   after the barrier. A CTA that waits longer than the time limit records
//   PICO_ERR_TIMEOUT and returns false; every CTA returns false once any
//   error is recorded, so an error ends the launch instead of hanging it.
// * block_push2 / warp_push: aggregated appends to global lists (one atomic
//   per block or per warp instead of one per element).
// * expand: load-balanced traversal of the adjacency of a vertex list. Small
//   vertices (degree <= small_deg) are taken 32 at a time by a warp, which
//   walks their concatenated neighbour lists with all lanes; large vertices
//   are pre-split into chunks of `chunk` arcs, one chunk per warp.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace pico {

constexpr unsigned kFull = 0xffffffffu;
// Work assignment by degree class (tunable per device, see Tuning): a vertex
// of degree <= small_deg is "small" (batched 32 per warp unit); a larger one
// is split into chunks of `chunk` arcs, one chunk per warp unit. The scratch
// bounds assume small_deg >= kMinSmallDeg and chunk >= kMinChunk.
constexpr int kSmallDeg = 32;     // default small-degree threshold
constexpr int kChunk = 256;       // default chunk size
constexpr int kMinSmallDeg = 32, kMaxSmallDeg = 256;
constexpr int kMinChunk = 64, kMaxChunk = 4096;

// Direction of HistoCore's UpdateHisto: push from the changed vertices (the
// formulation of Alg. 6), pull into every vertex whose row an edit can reach,
// or choose per round (auto).
constexpr int kUpdateAuto = 0, kUpdatePush = 1, kUpdatePull = 2;
constexpr int kPullPct = 50;                  // auto: pull when the changed vertices
                                              // hold >= this % of the arcs ...
constexpr long long kPullMinArcs = 1ll << 22;  // ... of a graph with at least this many

// How PeelOne keeps a decrement from taking a vertex below the level k
// (peelone.cuh): guard + repair after the level, compare-and-swap loop, or
// add-back.
enum : int { kPeelRepair = 0, kPeelCas = 1, kPeelAddBack = 2 };

// PeelOne's asynchronous levels issue a decrement for every arc without
// reading the neighbour first. A vertex peeled at level k has about k
// neighbours left, so when its degree is well above k most of its arcs end at
// vertices peeled earlier. Chunks of a vertex with degree > kPeelGuard * k
// read the neighbour's residual degree first and skip the atomic when it is
// <= k (0: never).
constexpr int kPeelGuard = 4;

struct Tuning {
    int small_deg;
    int chunk;
    int cluster_log2;   // batched form: graphs with >= 2^cluster_log2 arcs use a cluster
    int update_mode = kUpdateAuto;
    int pull_pct = kPullPct;
    int peel_guard = kPeelGuard;   // PeelOne: guard the arcs of vertices of degree > peel_guard * k
};
constexpr int kClusterNever = 62;   // cluster_log2 value that disables clusters
constexpr int kClusterLog2 = 21;    // default
constexpr int kThreads = 512;     // threads per CTA of the persistent kernels
constexpr int kLiveWords = 32;

enum : int {
    kOk = 0,
    kErrNotConverged = -4,
    kErrTimeout = -5,
    kErrBadGraph = -6,
};

struct alignas(128) Line {
    unsigned w[32];
};

// Statistics slots (match pico_stats field order after `algo`).
enum StatIdx : int {
    kStLevels = 0, kStKmax, kStSubrounds, kStScans, kStRounds, kStFrontier,
    kStBarriers, kStArcs, kStAtomics, kStSlots, kStBlocks, kStScanned, kStPulled,
    kStPullRounds, kStExtra, kStActive,
    kStPhaseNs = 16,      // 16..23: device time per phase kind (CTA 0's view)
    kStPhaseCount = 24,   // 24..31: phases per kind
    kStCount = 32
};

// Phase kinds for the timing statistics.
enum PhaseKind : int {
    kPhInit = 0, kPhScan, kPhWaveTiny, kPhWaveMid, kPhWaveWide, kPhInitHisto, kPhSumHisto,
    kPhUpdateHisto,
    kPhUpdatePull,  // trace only: counted as kPhUpdateHisto in the statistics
    kPhLevel        // trace only: one asynchronous PeelOne level, counted as kPhWaveWide
};


struct Ctrl {
    Line bar;                 // w[0..1]: arrivals at grid barriers (64-bit, whole launch)
    Line gen;                 // w[0]: grid barriers completed
    Line stat;                // w[0] status, w[1] CTAs that finished
    Line live;                // counters updated with atomics
    Line snap[2];             // live counters as of the last barrier (by parity)
    unsigned long long stats[kStCount];
};

// Phase trace (opt-in): one entry per phase of the most recent call.
constexpr int kTraceCap = 8192;
struct TraceEntry {
    unsigned kind;            // PhaseKind
    unsigned units;           // work units of the phase (vertices or chunks)
    unsigned long long ns;    // device time of the phase
};

// Per-device record of the most recent call, read by pico_get_stats,
// pico_last_device_status and pico_get_trace.
struct LastResult {
    int status;               // sticky: first error since the last read
    int pad;
    long long algo;
    unsigned long long stats[kStCount];
    unsigned trace_len;
    unsigned trace_on;        // set by the host when PICO_TRACE is on
    TraceEntry trace[kTraceCap];
};

// ---------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-phase device time, kept by thread 0 of CTA 0 (the only writer); with
// a trace record, every phase is also appended to it.
struct PhaseClock {
    unsigned long long t_prev = 0;
    TraceEntry *trace = nullptr;
    unsigned *trace_len = nullptr;
    __device__ __forceinline__ void start()
    {
        if (blockIdx.x == 0 && threadIdx.x == 0) t_prev = gtime();
    }
    __device__ __forceinline__ void end(unsigned long long *st, int kind, unsigned units = 0)
    {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned long long t = gtime();
            const int sk =
                kind == kPhLevel ? kPhWaveWide : (kind > kPhUpdateHisto ? kPhUpdateHisto : kind);
            st[kStPhaseNs + sk] += t - t_prev;
            st[kStPhaseCount + sk] += 1;
            if (trace && *trace_len < (unsigned)kTraceCap) {
                trace[*trace_len] = TraceEntry{(unsigned)kind, units, t - t_prev};
                ++*trace_len;
            }
            t_prev = t;
        }
    }
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int2 ld_relaxed(const int2 *p)
{
    int2 v;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p)
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(int2 *p, int2 v)
{
    asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(v.x), "r"(v.y)
                 : "memory");
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Mutable device data written by other CTAs is read through L2 only.
__device__ __forceinline__ int ldcg(const int *p) { return __ldcg(p); }

__device__ __forceinline__ void set_error(Ctrl *c, int code)
{
    atomicCAS(reinterpret_cast<int *>(&c->stat.w[0]), 0, code);
}

__device__ __forceinline__ int status_of(Ctrl *c)
{
    return ld_relaxed(reinterpret_cast<const int *>(&c->stat.w[0]));
}

// ---------------------------------------------------------------------------
// grid barrier with counter snapshot
// ---------------------------------------------------------------------------
// s_snap: shared memory, kLiveWords + 1 words; after the call s_snap[i] holds
// the live counter i as of the barrier and s_snap[kLiveWords] the status.
// gen: barriers this CTA has completed in the launch (the same in every CTA).
// Thread 0 of each CTA takes part. Arrivals count up over the whole launch
// (a 64-bit counter, never reset), so barrier number gen is complete when
// (gen + 1) x gridDim.x CTAs have arrived. The arrival is one acquire-release
// atomic (it publishes the CTA's counter updates, ordered before it by the
// CTA barrier, and lets the last arrival see everyone's). The last arrival
// copies the live counters into the snapshot of the barrier's parity with
// vector loads and stores and releases the generation word; the others wait
// for that word with acquire loads (bounded: limit_ns and the status word)
// and read the snapshot. A snapshot of parity p is rewritten two barriers
// later, which every reader must reach first.
// grid_sync_hook is the same barrier with `hook(live)` run by the last arrival
// on the live counters it has loaded, before it publishes the snapshot and
// releases the others: the hook's stores (relaxed, global) are visible to
// every CTA after the barrier.
struct NoHook {
    __device__ __forceinline__ void operator()(const uint4 *) const {}
};

template <typename Hook>
__device__ __forceinline__ bool grid_sync_hook(Ctrl *c, unsigned *s_snap,
                                               unsigned long long limit_ns, unsigned gen,
                                               const Hook &hook)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned par = (gen + 1) & 1;
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x;
        unsigned long long old;
        asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], 1;"
                     : "=l"(old)
                     : "l"(reinterpret_cast<unsigned long long *>(c->bar.w))
                     : "memory");
        uint4 *snap = reinterpret_cast<uint4 *>(c->snap[par].w);
        if (old + 1 == target) {
            const uint4 *live = reinterpret_cast<const uint4 *>(c->live.w);
            uint4 t[kLiveWords / 4];
#pragma unroll
            for (int i = 0; i < kLiveWords / 4; ++i) t[i] = __ldcg(live + i);
            hook(t);
#pragma unroll
            for (int i = 0; i < kLiveWords / 4; ++i) __stcg(snap + i, t[i]);
            st_release(&c->gen.w[0], gen + 1);
        } else {
            const unsigned long long t0 = gtime();
            unsigned spins = 0;
            while (ld_acquire(&c->gen.w[0]) == gen) {
                if ((++spins & 63) == 0) {
                    if (status_of(c) != 0) break;
                    if (gtime() - t0 > limit_ns) {
                        set_error(c, kErrTimeout);
                        break;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kLiveWords / 4; ++i) {
            const uint4 t = __ldcg(snap + i);
            s_snap[4 * i] = t.x;
            s_snap[4 * i + 1] = t.y;
            s_snap[4 * i + 2] = t.z;
            s_snap[4 * i + 3] = t.w;
        }
        s_snap[kLiveWords] = (unsigned)status_of(c);
    }
    __syncthreads();
    return s_snap[kLiveWords] == 0;
}

static __device__ __noinline__ bool grid_sync(Ctrl *c, unsigned *s_snap,
                                              unsigned long long limit_ns, unsigned gen)
{
    return grid_sync_hook(c, s_snap, limit_ns, gen, NoHook{});
}

// Called once by every CTA at the end of a persistent kernel: folds the CTA's
// statistics into the call's control block; the last CTA publishes the
// status and statistics to the per-device LastResult.
__device__ __forceinline__ void finish_block(Ctrl *c, LastResult *last, int algo,
                                             const unsigned long long *local, int nlocal)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < nlocal; ++i)
            if (local[i]) atomicAdd(&c->stats[i], local[i]);
        __threadfence();
        unsigned done = atomicAdd(&c->stat.w[1], 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            int st = status_of(c);
            if (st != 0) atomicCAS(&last->status, 0, st);
            last->algo = algo;
            for (int i = 0; i < kStCount; ++i)
                last->stats[i] = atomicAdd(&c->stats[i], 0ull);
            last->stats[kStBlocks] = gridDim.x;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// aggregated appends
// ---------------------------------------------------------------------------
// Warp-aggregated append: all lanes of the warp call; lanes with `pred`
// receive consecutive slots of *counter.
__device__ __forceinline__ unsigned warp_push(unsigned *counter, bool pred)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned b = __ballot_sync(kFull, pred);
    unsigned base = 0;
    if (b) {
        const int leader = __ffs(b) - 1;
        if ((int)lane == leader) base = atomicAdd(counter, (unsigned)__popc(b));
        base = __shfl_sync(kFull, base, leader);
    }
    return base + __popc(b & ((1u << lane) - 1u));
}

// Block-aggregated append to two lists at once. Every thread of the CTA must
// call it (block-uniform control flow). s: shared scratch of >= 128 words.
__device__ __forceinline__ void block_push2(bool p0, bool p1, unsigned *c0, unsigned *c1,
                                            unsigned &pos0, unsigned &pos1, unsigned *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned b0 = __ballot_sync(kFull, p0), b1 = __ballot_sync(kFull, p1);
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) {
        s[warp] = __popc(b0);
        s[32 + warp] = __popc(b1);
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned x0 = lane < nw ? s[lane] : 0u, x1 = lane < nw ? s[32 + lane] : 0u;
        unsigned i0 = x0, i1 = x1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y0 = __shfl_up_sync(kFull, i0, o), y1 = __shfl_up_sync(kFull, i1, o);
            if ((int)lane >= o) {
                i0 += y0;
                i1 += y1;
            }
        }
        const unsigned t0 = __shfl_sync(kFull, i0, 31), t1 = __shfl_sync(kFull, i1, 31);
        unsigned base0 = 0, base1 = 0;
        if (lane == 0) {
            if (t0) base0 = atomicAdd(c0, t0);
            if (t1) base1 = atomicAdd(c1, t1);
        }
        base0 = __shfl_sync(kFull, base0, 0);
        base1 = __shfl_sync(kFull, base1, 0);
        if (lane < nw) {
            s[64 + lane] = base0 + i0 - x0;
            s[96 + lane] = base1 + i1 - x1;
        }
    }
    __syncthreads();
    pos0 = s[64 + warp] + __popc(b0 & lt);
    pos1 = s[96 + warp] + __popc(b1 & lt);
    __syncthreads();
}

// Block-wide minimum folded into *target with one atomicMin per CTA.
__device__ __forceinline__ void block_min_to(int v, int *target, int *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = __reduce_min_sync(kFull, v);
    if (lane == 0) s[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int x = lane < nw ? s[lane] : INT_MAX;
        x = __reduce_min_sync(kFull, x);
        if (lane == 0 && x != INT_MAX) atomicMin(target, x);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// load-balanced adjacency expansion
// ---------------------------------------------------------------------------
// Writes reserved chunk entries: every lane with nch > 0 owns entries
// pos .. pos + nch - 1 of vertex v (reserved by the caller). A lane writes a
// short list itself; the warp writes the longer ones (hubs) together.
__device__ __forceinline__ void warp_fill_chunks(unsigned nch, unsigned pos, int v, int2 *list)
{
    constexpr unsigned kOwn = 8;
    const int lane = threadIdx.x & 31;
    if (nch <= kOwn)
        for (unsigned c = 0; c < nch; ++c) list[pos + c] = make_int2(v, (int)c);
    unsigned m = __ballot_sync(kFull, nch > kOwn);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const unsigned nn = __shfl_sync(kFull, nch, src), pp = __shfl_sync(kFull, pos, src);
        const int vv = __shfl_sync(kFull, v, src);
        for (unsigned c = lane; c < nn; c += 32) list[pp + c] = make_int2(vv, (int)c);
    }
}

// Warp-cooperative append of the chunk entries of large vertices: every
// lane with `pred` owns vertex v of degree d; the whole warp writes the
// ceil(d / chunk) entries of each such vertex in turn.
template <bool kRelaxedStores = false>
__device__ __forceinline__ void warp_push_chunks(bool pred, int v, long long d, int2 *list,
                                                 unsigned *counter, unsigned cap, Ctrl *ctl,
                                                 int chunk)
{
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(kFull, pred);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int vv = __shfl_sync(kFull, v, src);
        const long long dd = __shfl_sync(kFull, d, src);
        const unsigned nch = (unsigned)((dd + chunk - 1) / chunk);
        unsigned pos = 0;
        if (lane == 0) pos = atomicAdd(counter, nch);
        pos = __shfl_sync(kFull, pos, 0);
        if ((unsigned long long)pos + nch > cap) {
            if (lane == 0) set_error(ctl, kErrNotConverged);
            continue;
        }
        for (unsigned c = lane; c < nch; c += 32) {
            if (kRelaxedStores) st_relaxed(list + pos + c, make_int2(vv, (int)c));
            else list[pos + c] = make_int2(vv, (int)c);
        }
    }
}

// Default number of arcs a lane issues per step of expand(): their loads and
// atomics are independent, so that many memory round trips per lane are in
// flight. A functor sets its own count as F::kArcs.
constexpr int kU = 4;

// Fire-and-forget atomic add (a reduction: no value comes back, so the warp
// does not wait for it).
__device__ __forceinline__ void red_add(int *p, int v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Functor interface used by expand() (U = F::kArcs):
//   bool item(int v, int &a, int &b)     per-vertex prologue (lane-local);
//                                        false skips the vertex's arcs
//   void arcs(const bool (&valid)[U], const int (&v)[U], const int (&u)[U],
//             const Off (&rs)[U], const int (&a)[U], const int (&b)[U])
//                                        called by ALL 32 lanes together with
//                                        U arcs (v -> u) per lane; rs = row_ptr[v]
// `small` lists small vertices (nullptr: the identity list 0..nsmall-1, where
// vertices with degree > tn.small_deg are skipped because their chunks are in
// `big`). `big` lists (vertex, chunk) pairs.
// Small vertices per warp unit for a phase with nsmall small vertices and
// nbig chunk units: 32 when there is enough work for every warp, otherwise
// fewer (a power of two) so that the phase's units spread over more warps and
// its longest unit, which bounds the phase, gets shorter.
__device__ __forceinline__ unsigned batch_width(unsigned nsmall, unsigned nbig, unsigned nwarps)
{
    if (nsmall == 0) return 32u;
    const unsigned free_warps = nwarps > nbig ? nwarps - nbig : 1u;
    unsigned vb = 32u;
    while (vb > 1u && (nsmall + vb - 1u) / vb < free_warps) vb >>= 1;
    return vb;
}

// One warp walks the concatenated adjacency of up to 32 small vertices, one
// per lane (v < 0: no vertex; a vertex of degree above max_deg is skipped,
// its arcs being listed as chunks elsewhere): a warp prefix sum of the
// degrees and a 5-step shuffle search give each arc's owner; every lane
// issues U arcs per step.
template <typename Off, typename F>
__device__ __forceinline__ void walk_batch(const int *__restrict__ ci, int v, Off rs, int d, F &f);

template <typename Off, typename F>
__device__ __forceinline__ void walk_small_batch(const Off *__restrict__ rp,
                                                 const int *__restrict__ ci, int v, F &f,
                                                 int max_deg)
{
    int d = 0;
    Off rs = 0;
    if (v >= 0) {
        rs = rp[v];
        const Off dd = rp[v + 1] - rs;
        if (dd <= max_deg) d = (int)dd;
    }
    walk_batch(ci, v, rs, d, f);
}

// The same walk with each lane's row start rs = row_ptr[v] and the number d
// of its arcs to walk given (d = 0: none).
template <typename Off, typename F>
__device__ __forceinline__ void walk_batch(const int *__restrict__ ci, int v, Off rs, int d, F &f)
{
    constexpr int U = F::kArcs;
    const int lane = threadIdx.x & 31;
    int a = 0, b = 0;
    if (d > 0 && !f.item(v, a, b)) d = 0;
    int incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - d;
    const int T = __shfl_sync(kFull, incl, 31);
    for (int base = 0; base < T; base += 32 * U) {
        bool valid[U];
        int vo[U], u[U], ao[U], bo[U];
        Off rso[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int fidx = base + 32 * j + lane;
            int o = 0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const int ex = __shfl_sync(kFull, excl, o + s);
                if (ex <= fidx) o += s;
            }
            vo[j] = __shfl_sync(kFull, v, o);
            rso[j] = __shfl_sync(kFull, rs, o);
            const int exo = __shfl_sync(kFull, excl, o);
            ao[j] = __shfl_sync(kFull, a, o);
            bo[j] = __shfl_sync(kFull, b, o);
            valid[j] = fidx < T;
            u[j] = valid[j] ? __ldg(ci + rso[j] + (fidx - exo)) : -1;
        }
        f.arcs(valid, vo, u, rso, ao, bo);
    }
}

// One warp walks chunk `c` (tn.chunk arcs) of the adjacency of vertex v.
template <typename Off, typename F>
__device__ __forceinline__ void walk_chunk(const Off *__restrict__ rp, const int *__restrict__ ci,
                                           int v, int c, F &f, const Tuning &tn)
{
    constexpr int U = F::kArcs;
    const int lane = threadIdx.x & 31;
    const Off rs = rp[v], re = rp[v + 1];
    const Off s = rs + (Off)c * tn.chunk;
    const Off t = (s + tn.chunk < re) ? s + tn.chunk : re;
    int a = 0, b = 0;
    if (!f.item(v, a, b)) return;
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
            ao[j] = a;
            bo[j] = b;
        }
        f.arcs(valid, vo, u, rso, ao, bo);
    }
}

template <typename Off, typename F>
__device__ __forceinline__ void expand(const Off *__restrict__ rp, const int *__restrict__ ci,
                                       const int *small, unsigned nsmall, const int2 *big,
                                       unsigned nbig, unsigned gwarp, unsigned nwarps, F &f,
                                       const Tuning &tn, unsigned vb = 32u)
{
    const int lane = threadIdx.x & 31;
    const unsigned nbatch = (nsmall + vb - 1u) / vb;
    const unsigned total = nbatch + nbig;
    for (unsigned unit = gwarp; unit < total; unit += nwarps) {
        if (unit < nbatch) {
            const unsigned idx = unit * vb + lane;
            int v = -1;
            if ((unsigned)lane < vb && idx < nsmall) v = small ? ldcg(small + idx) : (int)idx;
            walk_small_batch(rp, ci, v, f, tn.small_deg);
        } else {
            const int2 ent = __ldcg(big + (unit - nbatch));   // written by other CTAs
            walk_chunk(rp, ci, ent.x, ent.y, f, tn);
        }
    }
}

}  // namespace pico

namespace pico {

// Block-wide maximum folded into *target with one atomicMax per CTA.
__device__ __forceinline__ void block_max_to(unsigned v, unsigned *target, unsigned *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = __reduce_max_sync(kFull, v);
    if (lane == 0) s[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned x = lane < nw ? s[lane] : 0u;
        x = __reduce_max_sync(kFull, x);
        if (lane == 0 && x != 0u) atomicMax(target, x);
    }
    __syncthreads();
}

// Block-wide sum of a per-thread counter, added to *target by thread 0.
__device__ __forceinline__ void block_sum_to(unsigned long long v, unsigned long long *target,
                                             unsigned long long *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0) s[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (unsigned w = 0; w < nw; ++w) t += s[w];
        if (t) atomicAdd(target, t);
    }
    __syncthreads();
}

}  // namespace pico

namespace pico {

// Block-aggregated append to N lists at once (generalises block_push2).
// Every thread of the CTA must call it. s: shared scratch of >= 64 * N words.
template <int N>
__device__ __forceinline__ void block_pushN(const bool (&p)[N], unsigned *const (&ctr)[N],
                                            unsigned (&pos)[N], unsigned *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned b[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        b[j] = __ballot_sync(kFull, p[j]);
        if (lane == 0) s[32 * j + warp] = __popc(b[j]);
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const unsigned x = lane < nw ? s[32 * j + lane] : 0u;
            unsigned inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(kFull, inc, o);
                if ((int)lane >= o) inc += y;
            }
            const unsigned t = __shfl_sync(kFull, inc, 31);
            unsigned base = 0;
            if (lane == 0 && t) base = atomicAdd(ctr[j], t);
            base = __shfl_sync(kFull, base, 0);
            if (lane < nw) s[32 * (N + j) + lane] = base + inc - x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < N; ++j) pos[j] = s[32 * (N + j) + warp] + __popc(b[j] & lt);
    __syncthreads();
}

// Block-aggregated allocation of `cnt` consecutive slots per thread from
// *counter (one atomic per CTA). Returns this thread's first slot.
__device__ __forceinline__ unsigned block_alloc(unsigned cnt, unsigned *counter, unsigned *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(kFull, inc, o);
        if ((int)lane >= o) inc += y;
    }
    if (lane == 31) s[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned x = lane < nw ? s[lane] : 0u;
        unsigned wi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(kFull, wi, o);
            if ((int)lane >= o) wi += y;
        }
        const unsigned t = __shfl_sync(kFull, wi, 31);
        unsigned base = 0;
        if (lane == 0 && t) base = atomicAdd(counter, t);
        base = __shfl_sync(kFull, base, 0);
        if (lane < nw) s[32 + lane] = base + wi - x;
    }
    __syncthreads();
    const unsigned r = s[32 + warp] + inc - cnt;
    __syncthreads();
    return r;
}

}  // namespace pico

namespace pico {

// Block-aggregated allocation from two counters at once: each thread asks
// for n0 slots of *c0 and n1 slots of *c1 and receives its first slot of
// each. Every thread of the CTA must call it. s: shared scratch >= 128 words.
__device__ __forceinline__ void block_alloc2(unsigned n0, unsigned n1, unsigned *c0, unsigned *c1,
                                             unsigned &b0, unsigned &b1, unsigned *s)
{
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned i0 = n0, i1 = n1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y0 = __shfl_up_sync(kFull, i0, o), y1 = __shfl_up_sync(kFull, i1, o);
        if ((int)lane >= o) {
            i0 += y0;
            i1 += y1;
        }
    }
    if (lane == 31) {
        s[warp] = i0;
        s[32 + warp] = i1;
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned x0 = lane < nw ? s[lane] : 0u, x1 = lane < nw ? s[32 + lane] : 0u;
        unsigned w0 = x0, w1 = x1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y0 = __shfl_up_sync(kFull, w0, o), y1 = __shfl_up_sync(kFull, w1, o);
            if ((int)lane >= o) {
                w0 += y0;
                w1 += y1;
            }
        }
        const unsigned t0 = __shfl_sync(kFull, w0, 31), t1 = __shfl_sync(kFull, w1, 31);
        unsigned g0 = 0, g1 = 0;
        if (lane == 0) {
            if (t0) g0 = atomicAdd(c0, t0);
            if (t1) g1 = atomicAdd(c1, t1);
        }
        g0 = __shfl_sync(kFull, g0, 0);
        g1 = __shfl_sync(kFull, g1, 0);
        if (lane < nw) {
            s[64 + lane] = g0 + w0 - x0;
            s[96 + lane] = g1 + w1 - x1;
        }
    }
    __syncthreads();
    b0 = s[64 + warp] + i0 - n0;
    b1 = s[96 + warp] + i1 - n1;
    __syncthreads();
}

}  // namespace pico

namespace pico {

// ---------------------------------------------------------------------------
// synchronisation domains of the persistent kernels
// ---------------------------------------------------------------------------
// GridDom: the whole grid works on one graph; a phase ends with grid_sync and
//   the counters live in the global control block.
// CtaDom: one CTA works on one graph (the batched form); a phase ends with
//   __syncthreads and the counters live in shared memory. The global status
//   word is polled every 256 phases (loops are bounded regardless).
// Both give every thread the counters as of the end of the last phase in
// s_snap, and the loop geometry of the domain (thread rank, threads, CTAs).
struct GridDom {
    Ctrl *ctl;
    unsigned *s_snap;
    unsigned long long limit_ns;
    unsigned gen = 0;   // barriers passed (the same in every thread of the launch)
    static constexpr bool kGrid = true;
    __device__ __forceinline__ unsigned *live() const { return ctl->live.w; }
    __device__ __forceinline__ bool sync() { return grid_sync(ctl, s_snap, limit_ns, gen++); }
    template <typename Hook>
    __device__ __forceinline__ bool sync_hook(const Hook &h)
    {
        return grid_sync_hook(ctl, s_snap, limit_ns, gen++, h);
    }
    __device__ __forceinline__ unsigned tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ unsigned nthreads() const { return gridDim.x * blockDim.x; }
    __device__ __forceinline__ unsigned cta() const { return blockIdx.x; }
    __device__ __forceinline__ unsigned ncta() const { return gridDim.x; }
    __device__ __forceinline__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
};

struct CtaDom {
    Ctrl *ctl;
    unsigned *s_live;   // kLiveWords counters (shared memory)
    unsigned *s_snap;   // kLiveWords + 1 words (shared memory)
    unsigned nsync;
    static constexpr bool kGrid = false;
    // Zeroes the counters; every thread of the CTA calls it.
    __device__ __forceinline__ void reset()
    {
        __syncthreads();
        if (threadIdx.x < kLiveWords) s_live[threadIdx.x] = 0;
        if (threadIdx.x == 0) s_snap[kLiveWords] = 0;
        __syncthreads();
    }
    __device__ __forceinline__ unsigned *live() const { return s_live; }
    __device__ __forceinline__ bool sync()
    {
        __syncthreads();
        if (threadIdx.x < kLiveWords) s_snap[threadIdx.x] = s_live[threadIdx.x];
        if (threadIdx.x == 0 && (++nsync & 255u) == 0) s_snap[kLiveWords] = (unsigned)status_of(ctl);
        __syncthreads();
        return s_snap[kLiveWords] == 0;
    }
    __device__ __forceinline__ unsigned tid() const { return threadIdx.x; }
    __device__ __forceinline__ unsigned nthreads() const { return blockDim.x; }
    __device__ __forceinline__ unsigned cta() const { return 0; }
    __device__ __forceinline__ unsigned ncta() const { return 1; }
    __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
};

}  // namespace pico

#include <cooperative_groups.h>

namespace pico {

// ClusterDom: the CTAs of one thread-block cluster work on one graph (the
// batched form's large graphs). The counters live in the shared memory of
// the cluster's rank-0 CTA and are reached by every CTA through distributed
// shared memory; a phase ends with the hardware cluster barrier, after which
// each CTA copies the counters into its own snapshot and a second cluster
// barrier keeps them unchanged until every CTA has copied them. The global
// status is read by rank 0 alone into counter word kClusterStatusWord, so
// every CTA takes the same decision after the same barrier (a CTA leaving
// alone would leave the others waiting at the next cluster barrier).
constexpr int kClusterStatusWord = kLiveWords - 1;

struct ClusterDom {
    Ctrl *ctl;
    unsigned *s_live;   // this CTA's counter words (only rank 0's are used)
    unsigned *live0;    // rank 0's counter words (distributed shared memory)
    unsigned *s_snap;   // kLiveWords + 1 words, this CTA's shared memory
    unsigned rank, size;
    unsigned nsync;
    static constexpr bool kGrid = false;
    __device__ __forceinline__ void reset()
    {
        cooperative_groups::this_cluster().sync();
        if (rank == 0 && threadIdx.x < kLiveWords) s_live[threadIdx.x] = 0;
        cooperative_groups::this_cluster().sync();
    }
    __device__ __forceinline__ unsigned *live() const { return live0; }
    __device__ __forceinline__ bool sync()
    {
        if (rank == 0 && threadIdx.x == 0 && (++nsync & 255u) == 0)
            s_live[kClusterStatusWord] = (unsigned)status_of(ctl);
        cooperative_groups::this_cluster().sync();
        if (threadIdx.x < kLiveWords) s_snap[threadIdx.x] = live0[threadIdx.x];
        cooperative_groups::this_cluster().sync();
        return s_snap[kClusterStatusWord] == 0;
    }
    __device__ __forceinline__ unsigned tid() const { return rank * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ unsigned nthreads() const { return size * blockDim.x; }
    __device__ __forceinline__ unsigned cta() const { return rank; }
    __device__ __forceinline__ unsigned ncta() const { return size; }
    __device__ __forceinline__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
};

}  // namespace pico
