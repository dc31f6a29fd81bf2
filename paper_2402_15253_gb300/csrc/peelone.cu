// PeelOne (Sec. III, Alg. 4) on one graph as one persistent cooperative
// kernel: the algorithm body is peel::run_async (peelone.cuh) over the whole
// grid, or peel::run (a grid barrier per frontier wave) when asynchronous
// levels are switched off.
#include "peelone.cuh"
#include "pico.h"
#include "pico_launch.h"

namespace pico {
namespace {

template <typename Off, int Mode, bool kAsync>
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
    if (kAsync)
        peel::run_async<Off, Mode>(p, dom, s_tmp, st, clk, arcs, atomics, extra);
    else
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

size_t chunk_capacity(long long m) { return peel::chunk_list_capacity(m); }

size_t peelone_ws_bytes(long long n, long long m, bool async)
{
    Carver c(nullptr);
    peel::Params<int> p;
    peel::carve(p, c, n, m, async);
    return c.size();
}

template <typename Off>
int launch_peelone(const Off *rp, const int *ci, long long n, long long m, int *core, void *ws,
                   LastResult *last, cudaStream_t stream, const LaunchCfg &cfg, int mode)
{
    if (mode < kPeelRepair || mode > kPeelAddBack) return -1;
    const void *fns[2][3] = {{(const void *)peelone_kernel<Off, kPeelRepair, false>,
                              (const void *)peelone_kernel<Off, kPeelCas, false>,
                              (const void *)peelone_kernel<Off, kPeelAddBack, false>},
                             {(const void *)peelone_kernel<Off, kPeelRepair, true>,
                              (const void *)peelone_kernel<Off, kPeelCas, true>,
                              (const void *)peelone_kernel<Off, kPeelAddBack, true>}};
    static int occ[2][3][64] = {};
    bool async = cfg.peel_async;
    int &o = occ[async][mode][cfg.device & 63];
    if (o == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fns[async][mode], kThreads, 0) !=
                cudaSuccess ||
            o <= 0)
            return -3;
    }
    const int per_sm = o < cfg.max_blocks_per_sm ? o : cfg.max_blocks_per_sm;
    const int ctas = cfg.sms * per_sm;
    if (ctas > peel::kMaxAsyncCtas) async = false;   // the level-end flags have no room

    Carver c(ws);
    peel::Params<Off> p;
    peel::carve(p, c, n, m, async);
    p.rp = rp;
    p.ci = ci;
    p.core = core;
    p.tn = cfg.tn;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;

    dim3 grid(ctas), block(kThreads);
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&p, &last, &limit};
    if (launch_cooperative(fns[async][mode], grid, block, args, 0, stream) != cudaSuccess)
        return -3;
    return 0;
}

template int launch_peelone<int>(const int *, const int *, long long, long long, int *, void *,
                                 LastResult *, cudaStream_t, const LaunchCfg &, int);
template int launch_peelone<long long>(const long long *, const int *, long long, long long,
                                       int *, void *, LastResult *, cudaStream_t,
                                       const LaunchCfg &, int);

}  // namespace pico
