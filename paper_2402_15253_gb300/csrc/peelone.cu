// PeelOne (Sec. III, Alg. 4) on one graph as one persistent cooperative
// kernel: the algorithm body is peel::run (peelone.cuh) over the whole grid.
#include "peelone.cuh"
#include "pico.h"
#include "pico_launch.h"

namespace pico {
namespace {

template <typename Off, int Mode>
__global__ void __launch_bounds__(kThreads, 2)
    peelone_kernel(peel::Params<Off> p, LastResult *last, unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[128];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];   // statistics, written by thread 0
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long arcs = 0, atomics = 0, extra = 0;
    PhaseClock clk;
    if (blockIdx.x == 0 && threadIdx.x == 0 && last->trace_on) {
        last->trace_len = 0;
        clk.trace = last->trace;
        clk.trace_len = &last->trace_len;
    }
    clk.start();
    GridDom dom{p.ctl, s_snap, limit_ns};
    peel::run<Off, GridDom, Mode>(p, dom, s_tmp, st, clk, arcs, atomics, extra);
    block_sum_to(arcs, &p.ctl->stats[kStArcs], s_red);
    block_sum_to(atomics, &p.ctl->stats[kStAtomics], s_red);
    block_sum_to(extra, &p.ctl->stats[kStExtra], s_red);
    if (blockIdx.x != 0 && threadIdx.x < kStCount) st[threadIdx.x] = 0;
    finish_block(p.ctl, last,
                 Mode == kPeelRepair ? PICO_ALGO_PEELONE
                                     : (Mode == kPeelCas ? PICO_ALGO_PEEL_CAS : PICO_ALGO_PEEL_ADDBACK),
                 st, kStCount);
}

}  // namespace

size_t chunk_capacity(long long m)
{
    // enough for every allowed tuning (chunk >= kMinChunk, small_deg >= kMinSmallDeg)
    return (size_t)(m / kMinChunk + m / (kMinSmallDeg + 1) + 2);
}

size_t peelone_ws_bytes(long long n, long long m)
{
    Carver c(nullptr);
    c.take<Ctrl>(1);
    c.take<int>(n);
    c.take<int>(n);
    c.take<int>(n);
    c.take<int2>(chunk_capacity(m));
    return c.size();
}

template <typename Off>
int launch_peelone(const Off *rp, const int *ci, long long n, long long m, int *core, void *ws,
                   LastResult *last, cudaStream_t stream, const LaunchCfg &cfg, int mode)
{
    Carver c(ws);
    peel::Params<Off> p;
    p.rp = rp;
    p.ci = ci;
    p.n = n;
    p.core = core;
    p.ctl = c.take<Ctrl>(1);
    p.res0 = c.take<int>(n);
    p.res1 = c.take<int>(n);
    p.qs = c.take<int>(n);
    p.qb_cap = (unsigned)chunk_capacity(m);
    p.qb = c.take<int2>(p.qb_cap);
    p.tn = cfg.tn;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;

    if (mode < kPeelRepair || mode > kPeelAddBack) return -1;
    const void *fns[3] = {(const void *)peelone_kernel<Off, kPeelRepair>,
                          (const void *)peelone_kernel<Off, kPeelCas>,
                          (const void *)peelone_kernel<Off, kPeelAddBack>};
    static int occ[3][64] = {};
    int &o = occ[mode][cfg.device & 63];
    if (o == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fns[mode], kThreads, 0) !=
                cudaSuccess ||
            o <= 0)
            return -3;
    }
    const int per_sm = o < cfg.max_blocks_per_sm ? o : cfg.max_blocks_per_sm;
    dim3 grid(cfg.sms * per_sm), block(kThreads);
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&p, &last, &limit};
    if (cudaLaunchCooperativeKernel(fns[mode], grid, block, args, 0, stream) != cudaSuccess)
        return -3;
    return 0;
}

template int launch_peelone<int>(const int *, const int *, long long, long long, int *, void *,
                                 LastResult *, cudaStream_t, const LaunchCfg &, int);
template int launch_peelone<long long>(const long long *, const int *, long long, long long,
                                       int *, void *, LastResult *, cudaStream_t,
                                       const LaunchCfg &, int);

}  // namespace pico
