// PeelOne (Sec. III, Alg. 4) on one graph as one persistent cooperative
// kernel: the algorithm body is peel::run_async (peelone.cuh) over the whole
// grid, or peel::run (a grid barrier per frontier wave) when asynchronous
// levels are switched off.
#include <algorithm>

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

// Reads a range (16 bytes a thread per step); the values are not used.
__global__ void __launch_bounds__(256) touch_kernel(const int4 *p, size_t count, int *sink)
{
    int acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        const int4 v = __ldcg(p + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x7fffffff && sink) *sink = acc;   // keeps the loads
}

}  // namespace

cudaError_t l2_release(const void *p, size_t bytes, cudaStream_t stream)
{
    const size_t count = bytes / sizeof(int4);
    if (!p || count == 0) return cudaSuccess;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)std::min<size_t>((count + 255) / 256, 1024));
    lc.blockDim = dim3(256);
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = const_cast<void *>(p);
    attr[0].val.accessPolicyWindow.num_bytes = count * sizeof(int4);
    attr[0].val.accessPolicyWindow.hitRatio = 1.0f;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const int4 *q = static_cast<const int4 *>(p);
    int *sink = nullptr;
    void *args[] = {&q, (void *)&count, &sink};
    return cudaLaunchKernelExC(&lc, (const void *)touch_kernel, args);
}

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
    // the residual degrees (the target of every decrement) stay in L2
    const size_t win = async ? std::min<size_t>((size_t)n * sizeof(int), cfg.l2_window) : 0;
    if (launch_cooperative(fns[async][mode], grid, block, args, 0, stream, p.work, win) !=
        cudaSuccess)
        return -3;
    if (win > 0 && l2_release(p.work, win, stream) != cudaSuccess) return -3;
    return 0;
}

template int launch_peelone<int>(const int *, const int *, long long, long long, int *, void *,
                                 LastResult *, cudaStream_t, const LaunchCfg &, int);
template int launch_peelone<long long>(const long long *, const int *, long long, long long,
                                       int *, void *, LastResult *, cudaStream_t,
                                       const LaunchCfg &, int);

}  // namespace pico
