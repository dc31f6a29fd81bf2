// HistoCore (Sec. IV-B, Alg. 6) on one graph as one persistent cooperative
// kernel: the algorithm body is histo::run (histocore.cuh) over the whole grid.
#include "histocore.cuh"
#include "pico_launch.h"

namespace pico {
namespace {

template <typename Off>
__global__ void __launch_bounds__(kThreads, 2)
    histocore_kernel(histo::Params<Off> p, LastResult *last, unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[256];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];   // statistics, written by thread 0
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long arcs = 0, atomics = 0, slots = 0, pulled = 0;
    PhaseClock clk;
    if (blockIdx.x == 0 && threadIdx.x == 0 && last->trace_on) {
        last->trace_len = 0;
        clk.trace = last->trace;
        clk.trace_len = &last->trace_len;
    }
    clk.start();
    GridDom dom{p.ctl, s_snap, limit_ns};
    histo::run(p, dom, s_tmp, st, clk, arcs, atomics, slots, pulled);
    block_sum_to(arcs, &p.ctl->stats[kStArcs], s_red);
    block_sum_to(pulled, &p.ctl->stats[kStPulled], s_red);
    block_sum_to(atomics, &p.ctl->stats[kStAtomics], s_red);
    block_sum_to(slots, &p.ctl->stats[kStSlots], s_red);
    if (blockIdx.x != 0 && threadIdx.x < kStCount) st[threadIdx.x] = 0;
    finish_block(p.ctl, last, 1, st, kStCount);
}

}  // namespace

size_t histocore_ws_bytes(long long n, long long m)
{
    Carver c(nullptr);
    c.take<Ctrl>(1);
    c.take<longlong2>(n);  // vinfo (sized for int64 offsets)
    c.take<int2>(n);       // mv[0]
    c.take<int2>(n);       // mv[1]
    c.take<unsigned>(n);   // mvp[0]
    c.take<unsigned>(n);   // mvp[1]
    c.take<int>(m);        // histo
    for (int i = 0; i < 6; ++i) c.take<int>(n);
    c.take<int>(n);        // us
    c.take<int2>(chunk_capacity(m));   // ub
    c.take<int2>(chunk_capacity(m));   // ib
    c.take<unsigned char>((size_t)((n + 3) & ~3ll));   // cand
    return c.size();
}

template <typename Off>
int launch_histocore(const Off *rp, const int *ci, long long n, long long m, int *core,
                     void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg,
                     const int *init_est)
{
    Carver c(ws);
    histo::Params<Off> p;
    p.rp = rp;
    p.ci = ci;
    p.n = n;
    p.m = m;
    p.core = core;
    p.ctl = c.take<Ctrl>(1);
    p.vinfo = reinterpret_cast<histo::VRec<Off> *>(c.take<longlong2>(n));
    p.mv[0] = c.take<int2>(n);
    p.mv[1] = c.take<int2>(n);
    p.mvp[0] = c.take<unsigned>(n);
    p.mvp[1] = c.take<unsigned>(n);
    p.histo = c.take<int>(m);
    for (int i = 0; i < 2; ++i) {
        p.tl[i] = c.take<int>(n);
        p.wl[i] = c.take<int>(n);
        p.bl[i] = c.take<int>(n);
    }
    p.us = c.take<int>(n);
    p.ub_cap = (unsigned)chunk_capacity(m);
    p.ub = c.take<int2>(p.ub_cap);
    p.ib = c.take<int2>(p.ub_cap);
    p.cand = c.take<unsigned char>((size_t)((n + 3) & ~3ll));
    p.zero_histo = false;
    p.tn = cfg.tn;
    p.init_est = init_est;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;
    if (m > 0 && cudaMemsetAsync(p.histo, 0, (size_t)m * sizeof(int), stream) != cudaSuccess)
        return -3;

    static int occ[64] = {};
    int &o = occ[cfg.device & 63];
    if (o == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, histocore_kernel<Off>, kThreads,
                                                          0) != cudaSuccess ||
            o <= 0)
            return -3;
    }
    const int per_sm = o < cfg.max_blocks_per_sm ? o : cfg.max_blocks_per_sm;
    dim3 grid(cfg.sms * per_sm), block(kThreads);
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&p, &last, &limit};
    if (launch_cooperative((const void *)histocore_kernel<Off>, grid, block, args, 0,
                                    stream) != cudaSuccess)
        return -3;
    return 0;
}

template int launch_histocore<int>(const int *, const int *, long long, long long, int *, void *,
                                   LastResult *, cudaStream_t, const LaunchCfg &, const int *);
template int launch_histocore<long long>(const long long *, const int *, long long, long long,
                                         int *, void *, LastResult *, cudaStream_t,
                                         const LaunchCfg &, const int *);

}  // namespace pico
