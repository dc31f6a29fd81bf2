// Batched form: the coreness of G independent graphs in one launch.
//
// Coreness is defined per connected component (Sec. I: the k-core is a
// maximal subgraph), so graphs packed side by side are solved independently.
// The kernel runs the same algorithm bodies as the single-graph kernels
// (peel::run, histo::run) in two phases over a schedule that lists graphs by
// decreasing arc count (power-of-two buckets):
//   large graphs (at least 2^cluster_log2 arcs, a tuning value; listed first): each
//     thread-block cluster of kClusterCtas CTAs takes one graph at a time
//     (ClusterDom: counters in the rank-0 CTA's shared memory, reached
//     through distributed shared memory; hardware cluster barriers);
//   the rest: every CTA takes one graph at a time (CtaDom: counters in its
//     own shared memory, __syncthreads).
// Tickets come from two global counters, so the largest graphs start first
// and the small ones fill in behind them.
//
// Scratch is sliced per graph: vertex-indexed arrays at vtx_off[g], the
// histogram at arc_off[g], and chunk lists at arc_off[g] / 16 + 2g with
// m_g / 16 + 2 entries (at least m_g / chunk + m_g / (small_deg + 1) + 2 for
// every allowed tuning: chunk >= 64 and small_deg >= 32).
#include "histocore.cuh"
#include "peelone.cuh"
#include "pico_launch.h"

namespace pico {
namespace {

constexpr int kBuckets = 64;
constexpr int kClusterCtas = 8;                 // CTAs per cluster (portable size)

// control words of the batched launch (in Ctrl::live)
enum : int { B_SMALL = 0, B_LARGE = 1, B_NLARGE = 2 };

struct BatchParams {
    const long long *vtx_off, *arc_off;
    int G;
    const int *rp, *ci;
    int *core;
    int *order;
    int *res0, *res1, *qs;                          // PeelOne
    int *histo, *lists[6], *us;                     // HistoCore
    int2 *vinfo, *mv[2], *ichunks;
    int2 *chunks;                                   // both
    Ctrl *ctl;
    Tuning tn;
};

__device__ __forceinline__ int size_bucket(long long m)
{
    return m <= 0 ? 0 : 64 - __clzll(m);
}

// Lists the graphs by decreasing arc-count bucket (one CTA) and records how
// many lead the list with at least 2^cluster_log2 arcs (bucket b holds arc
// counts in [2^(b-1), 2^b)).
__global__ void __launch_bounds__(1024)
    schedule_kernel(const long long *arc_off, int G, int *order, Ctrl *ctl, int cluster_log2)
{
    __shared__ unsigned cnt[kBuckets];
    __shared__ unsigned start[kBuckets];
    if (threadIdx.x < kBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += blockDim.x)
        atomicAdd(&cnt[size_bucket(arc_off[g + 1] - arc_off[g])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            start[b] = run;
            run += cnt[b];
            if (b == cluster_log2 + 1) ctl->live.w[B_NLARGE] = run;
        }
    }
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const unsigned pos = atomicAdd(&start[size_bucket(arc_off[g + 1] - arc_off[g])], 1u);
        order[pos] = g;
    }
}

// Solves graph g of the batch in domain `dom`.
template <int Algo, typename Dom>
__device__ __forceinline__ void solve_graph(const BatchParams &bp, int g, Dom &dom, unsigned *s_tmp,
                                            unsigned long long *st, PhaseClock &clk,
                                            unsigned long long &arcs, unsigned long long &atomics,
                                            unsigned long long &slots, unsigned long long &pulled)
{
    const long long v0 = bp.vtx_off[g], n = bp.vtx_off[g + 1] - v0;
    const long long a0 = bp.arc_off[g], m = bp.arc_off[g + 1] - a0;
    if (n <= 0) return;
    dom.reset();
    int2 *chunks = bp.chunks + (a0 / 16 + 2ll * g);
    const unsigned chunk_cap = (unsigned)(m / 16 + 2);
    if (Algo == 0) {
        peel::Params<int> p{bp.rp + v0 + g, bp.ci + a0,    n,      bp.core + v0,
                            bp.res0 + v0,   bp.res1 + v0,  bp.qs + v0, chunks,
                            chunk_cap,      bp.ctl,        bp.tn};
        unsigned long long extra = 0;
        peel::run(p, dom, s_tmp, st, clk, arcs, atomics, extra);
    } else {
        histo::Params<int> p;
        p.rp = bp.rp + v0 + g;
        p.ci = bp.ci + a0;
        p.n = n;
        p.m = m;
        p.core = bp.core + v0;
        p.vinfo = bp.vinfo + v0;
        p.mv[0] = bp.mv[0] + v0;
        p.mv[1] = bp.mv[1] + v0;
        p.histo = bp.histo + a0;
        p.tl[0] = bp.lists[0] + v0;
        p.wl[0] = bp.lists[1] + v0;
        p.bl[0] = bp.lists[2] + v0;
        p.tl[1] = bp.lists[3] + v0;
        p.wl[1] = bp.lists[4] + v0;
        p.bl[1] = bp.lists[5] + v0;
        p.us = bp.us + v0;
        p.ub = chunks;
        p.ib = bp.ichunks + (a0 / 16 + 2ll * g);
        p.ub_cap = chunk_cap;
        p.ctl = bp.ctl;
        p.zero_histo = true;
        p.tn = bp.tn;
        histo::run(p, dom, s_tmp, st, clk, arcs, atomics, slots, pulled);
    }
}

template <int Algo, int Threads>
__global__ void __launch_bounds__(Threads, 512 / Threads * 2)
    batched_kernel(BatchParams bp, LastResult *last)
{
    namespace cg = cooperative_groups;
    __shared__ __align__(16) unsigned s_live[kLiveWords];   // 64-bit counters need 8-byte alignment
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[256];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];
    __shared__ int s_ticket;
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned crank = cluster.block_rank(), csize = cluster.num_blocks();
    PhaseClock clk;
    unsigned long long arcs = 0, atomics = 0, slots = 0, pulled = 0;

    // phase 1: large graphs, one cluster per graph
    const int nlarge = (int)ld_relaxed(&bp.ctl->live.w[B_NLARGE]);
    {
        ClusterDom dom{bp.ctl, s_live, cluster.map_shared_rank(s_live, 0), s_snap, crank, csize,
                       0u};
        int *ticket0 = cluster.map_shared_rank(&s_ticket, 0);
        for (;;) {
            if (crank == 0 && threadIdx.x == 0) {
                const int t = (int)atomicAdd(&bp.ctl->live.w[B_LARGE], 1u);
                s_ticket = (t < nlarge && status_of(bp.ctl) == 0) ? t : -1;
            }
            cluster.sync();
            const int t = *ticket0;
            cluster.sync();
            if (t < 0) break;
            solve_graph<Algo>(bp, bp.order[t], dom, s_tmp, st, clk, arcs, atomics, slots, pulled);
        }
    }
    // phase 2: the other graphs, one CTA per graph
    {
        CtaDom dom{bp.ctl, s_live, s_snap, 0u};
        for (;;) {
            if (threadIdx.x == 0) s_ticket = nlarge + (int)atomicAdd(&bp.ctl->live.w[B_SMALL], 1u);
            __syncthreads();
            const int t = s_ticket;
            __syncthreads();
            if (t >= bp.G || status_of(bp.ctl) != 0) break;
            solve_graph<Algo>(bp, bp.order[t], dom, s_tmp, st, clk, arcs, atomics, slots, pulled);
            __syncthreads();
        }
    }
    block_sum_to(arcs, &bp.ctl->stats[kStArcs], s_red);
    block_sum_to(atomics, &bp.ctl->stats[kStAtomics], s_red);
    block_sum_to(slots, &bp.ctl->stats[kStSlots], s_red);
    block_sum_to(pulled, &bp.ctl->stats[kStPulled], s_red);
    if (threadIdx.x == 0) {
        atomicMax(&bp.ctl->stats[kStKmax], st[kStKmax]);
        st[kStKmax] = 0;
    }
    finish_block(bp.ctl, last, Algo, st, kStCount);
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace

size_t batched_ws_bytes(int G, long long total_n, long long total_m, int algo)
{
    Carver c(nullptr);
    c.take<Ctrl>(1);
    c.take<int>(G);
    const size_t nchunks = (size_t)(total_m / 16 + 2ll * G + 2);
    if (algo == 0) {
        for (int i = 0; i < 3; ++i) c.take<int>(total_n);
    } else {
        c.take<int2>(total_n);  // vinfo
        c.take<int2>(total_n);  // mv[0]
        c.take<int2>(total_n);  // mv[1]
        c.take<int>(total_m);   // histo
        for (int i = 0; i < 7; ++i) c.take<int>(total_n);
        c.take<int2>(nchunks);  // chunk lists of every large vertex
    }
    c.take<int2>(nchunks);
    return c.size();
}

int launch_batched(const int64_t *vtx_off, const int64_t *arc_off, int G, const int32_t *rp,
                   const int32_t *ci, long long total_n, long long total_m, int32_t *core,
                   int algo, void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg)
{
    Carver c(ws);
    BatchParams bp{};
    bp.vtx_off = reinterpret_cast<const long long *>(vtx_off);
    bp.arc_off = reinterpret_cast<const long long *>(arc_off);
    bp.G = G;
    bp.rp = rp;
    bp.ci = ci;
    bp.core = core;
    bp.ctl = c.take<Ctrl>(1);
    bp.order = c.take<int>(G);
    if (algo == 0) {
        bp.res0 = c.take<int>(total_n);
        bp.res1 = c.take<int>(total_n);
        bp.qs = c.take<int>(total_n);
    } else {
        bp.vinfo = c.take<int2>(total_n);
        bp.mv[0] = c.take<int2>(total_n);
        bp.mv[1] = c.take<int2>(total_n);
        bp.histo = c.take<int>(total_m);
        for (int i = 0; i < 6; ++i) bp.lists[i] = c.take<int>(total_n);
        bp.us = c.take<int>(total_n);
        bp.ichunks = c.take<int2>((size_t)(total_m / 16 + 2ll * G + 2));
    }
    bp.chunks = c.take<int2>((size_t)(total_m / 16 + 2ll * G + 2));
    bp.tn = cfg.tn;
    if (cudaMemsetAsync(bp.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;
    schedule_kernel<<<1, 1024, 0, stream>>>(bp.arc_off, G, bp.order, bp.ctl, cfg.tn.cluster_log2);
    if (cudaGetLastError() != cudaSuccess) return -3;

    const int threads = cfg.batched_threads == 256 ? 256 : 512;
    const int vi = (algo & 1) * 2 + (threads == 256 ? 1 : 0);
    static int occ[4][64] = {};
    int &o = occ[vi][cfg.device & 63];
    const void *fns[4] = {(const void *)batched_kernel<0, 512>, (const void *)batched_kernel<0, 256>,
                          (const void *)batched_kernel<1, 512>, (const void *)batched_kernel<1, 256>};
    const void *fn = fns[vi];
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = 0;
    lc.stream = stream;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (o == 0) {   // clusters that fit on the device at once
        lc.gridDim = dim3(kClusterCtas * cfg.sms);
        if (cudaOccupancyMaxActiveClusters(&o, fn, &lc) != cudaSuccess || o <= 0) return -3;
    }
    // persistent grid: every resident cluster, but no more clusters than graphs need
    const long long need = ((long long)G + kClusterCtas - 1) / kClusterCtas;
    const int clusters = need < o ? (int)need : o;
    lc.gridDim = dim3(kClusterCtas * clusters);
    void *args[] = {&bp, &last};
    if (cudaLaunchKernelExC(&lc, fn, args) != cudaSuccess) return -3;
    return 0;
}

}  // namespace pico
