// Method selection per graph (PICO_ALGO_AUTO): one persistent cooperative
// kernel that first measures the graph's largest degree, then runs PeelOne or
// HistoCore on it. The decision is made on the device (no host round trip, so
// the call stays asynchronous and capturable) and is uniform over the grid
// (every CTA reads the same snapshot after the barrier).
//
// The rule comes from timing both methods on GB300 over R-MAT (scale 14-24,
// edge factor 4-16), Chung-Lu (beta 2.1, planted K_3000), Erdos-Renyi and
// grid graphs. PeelOne's time is dominated by its level and wave barriers (a
// phase costs ~7 us on the whole grid), and the number of levels grows with
// the skew of the degree distribution. HistoCore needs far fewer rounds on
// skewed graphs, but its per-round work grows with the arcs. HistoCore was
// faster exactly on the skewed graphs (d_max >= 64 d_avg) that are small
// against their skew: m^2 <= 2^14 d_max n, i.e. m <= 2^14 d_max / d_avg.
// Results never depend on the choice; pico_get_stats reports the method used.
#include <algorithm>

#include "histocore.cuh"
#include "peelone.cuh"
#include "pico.h"
#include "pico_launch.h"

namespace pico {
namespace {

constexpr int kLiveDmax = 20;   // live word for the degree maximum (unused by both methods)
constexpr double kAutoSkew = 64.0;      // d_max / d_avg at least this ...
constexpr double kAutoScale = 16384.0;  // ... and m^2 <= this * d_max * n: HistoCore

__device__ __forceinline__ bool prefer_histocore(long long n, long long m, unsigned dmax)
{
    if (n <= 0 || m <= 0) return false;
    const double d = (double)dmax, nn = (double)n, mm = (double)m;
    return d * nn >= kAutoSkew * mm && mm * mm <= kAutoScale * d * nn;
}

template <typename Off>
__global__ void __launch_bounds__(kThreads, 2)
    hybrid_kernel(peel::Params<Off> pp, histo::Params<Off> hp, LastResult *last,
                  unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[256];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long arcs = 0, atomics = 0, slots = 0, pulled = 0, extra = 0;
    PhaseClock clk;
    if (blockIdx.x == 0 && threadIdx.x == 0 && last->trace_on) {
        last->trace_len = 0;
        clk.trace = last->trace;
        clk.trace_len = &last->trace_len;
    }
    clk.start();
    GridDom dom{pp.ctl, s_snap, limit_ns};
    unsigned *live = dom.live();
    const long long n = pp.n;
    unsigned mx = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned)(pp.rp[v + 1] - pp.rp[v]));
    block_max_to(mx, &live[kLiveDmax], s_tmp);
    bool use_histo = false;
    if (dom.sync()) {
        if (threadIdx.x == 0) ++st[kStBarriers];
        use_histo = prefer_histocore(n, hp.m, s_snap[kLiveDmax]);
        if (use_histo)
            histo::run(hp, dom, s_tmp, st, clk, arcs, atomics, slots, pulled);
        else if (pp.work)
            peel::run_async<Off, kPeelRepair>(pp, dom, s_tmp, st, clk, arcs, atomics, extra);
        else
            peel::run<Off, GridDom, kPeelRepair>(pp, dom, s_tmp, st, clk, arcs, atomics, extra);
    }
    block_sum_to(arcs, &pp.ctl->stats[kStArcs], s_red);
    block_sum_to(atomics, &pp.ctl->stats[kStAtomics], s_red);
    block_sum_to(slots, &pp.ctl->stats[kStSlots], s_red);
    block_sum_to(pulled, &pp.ctl->stats[kStPulled], s_red);
    block_sum_to(extra, &pp.ctl->stats[kStExtra], s_red);
    if (blockIdx.x != 0 && threadIdx.x < kStCount) st[threadIdx.x] = 0;
    finish_block(pp.ctl, last, use_histo ? PICO_ALGO_HISTOCORE : PICO_ALGO_PEELONE, st,
                 kStCount);
}

}  // namespace

size_t hybrid_ws_bytes(long long n, long long m)
{
    const size_t a = peelone_ws_bytes(n, m, true), b = histocore_ws_bytes(n, m);
    return a > b ? a : b;   // the two methods' scratch overlaps: only one runs
}

template <typename Off>
int launch_hybrid(const Off *rp, const int *ci, long long n, long long m, int *core, void *ws,
                  LastResult *last, cudaStream_t stream, const LaunchCfg &cfg)
{
    static int occ[64] = {};
    int &o = occ[cfg.device & 63];
    if (o == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hybrid_kernel<Off>, kThreads, 0) !=
                cudaSuccess ||
            o <= 0)
            return -3;
    }
    const int per_sm = o < cfg.max_blocks_per_sm ? o : cfg.max_blocks_per_sm;
    const int ctas = cfg.sms * per_sm;
    peel::Params<Off> pp;
    histo::Params<Off> hp;
    {
        Carver c(ws);
        peel::carve(pp, c, n, m, cfg.peel_async && ctas <= peel::kMaxAsyncCtas);
        pp.rp = rp;
        pp.ci = ci;
        pp.core = core;
        pp.tn = cfg.tn;
    }
    {
        Carver c(ws);   // same base: both control blocks are the same one
        hp.rp = rp;
        hp.ci = ci;
        hp.n = n;
        hp.m = m;
        hp.core = core;
        hp.ctl = c.take<Ctrl>(1);
        hp.vinfo = reinterpret_cast<histo::VRec<Off> *>(c.take<longlong2>(n));
        hp.mv[0] = c.take<int2>(n);
        hp.mv[1] = c.take<int2>(n);
        hp.mvp[0] = c.take<unsigned>(n);
        hp.mvp[1] = c.take<unsigned>(n);
        hp.histo = c.take<int>(m);
        for (int i = 0; i < 2; ++i) {
            hp.tl[i] = c.take<int>(n);
            hp.wl[i] = c.take<int>(n);
            hp.bl[i] = c.take<int>(n);
        }
        hp.us = c.take<int>(n);
        hp.ub_cap = (unsigned)chunk_capacity(m);
        hp.ub = c.take<int2>(hp.ub_cap);
        hp.ib = c.take<int2>(hp.ub_cap);
        hp.cand = c.take<unsigned char>((size_t)((n + 3) & ~3ll));
        hp.zero_histo = true;   // cleared in the kernel, only when HistoCore runs
        hp.tn = cfg.tn;
    }
    if (cudaMemsetAsync(pp.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&pp, &hp, &last, &limit};
    // PeelOne's residual degrees stay in L2 (when HistoCore runs, the window
    // covers part of its scratch instead, which is harmless)
    const size_t win = pp.work ? std::min<size_t>((size_t)n * sizeof(int), cfg.l2_window) : 0;
    if (launch_cooperative((const void *)hybrid_kernel<Off>, dim3(ctas), dim3(kThreads), args, 0,
                           stream, pp.work, win) != cudaSuccess)
        return -3;
    if (win > 0 && l2_release(pp.work, win, stream) != cudaSuccess) return -3;
    return 0;
}

template int launch_hybrid<int>(const int *, const int *, long long, long long, int *, void *,
                                LastResult *, cudaStream_t, const LaunchCfg &);
template int launch_hybrid<long long>(const long long *, const int *, long long, long long, int *,
                                      void *, LastResult *, cudaStream_t, const LaunchCfg &);

}  // namespace pico
