// The comparison baselines of Sec. V (ablation.cuh) on one graph, each as one
// persistent cooperative kernel over the whole grid: GPP (Alg. 3), NbrCore and
// CntCore (Alg. 5).
#include "ablation.cuh"
#include "pico.h"
#include "pico_launch.h"

namespace pico {
namespace {

template <typename Off>
__global__ void __launch_bounds__(kThreads, 2)
    gpp_kernel(gpp::Params<Off> p, LastResult *last, unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[256];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long arcs = 0, atomics = 0;
    GridDom dom{p.ctl, s_snap, limit_ns};
    gpp::run(p, dom, s_tmp, st, arcs, atomics);
    block_sum_to(arcs, &p.ctl->stats[kStArcs], s_red);
    block_sum_to(atomics, &p.ctl->stats[kStAtomics], s_red);
    if (blockIdx.x != 0 && threadIdx.x < kStCount) st[threadIdx.x] = 0;
    finish_block(p.ctl, last, PICO_ALGO_GPP, st, kStCount);
}

template <typename Off, bool UseCnt>
__global__ void __launch_bounds__(kThreads, 2)
    i2c_kernel(i2c::Params<Off> p, LastResult *last, unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[256];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long arcs = 0, atomics = 0;
    GridDom dom{p.ctl, s_snap, limit_ns};
    i2c::run<Off, GridDom, UseCnt>(p, dom, s_tmp, st, arcs, atomics);
    block_sum_to(arcs, &p.ctl->stats[kStArcs], s_red);
    block_sum_to(atomics, &p.ctl->stats[kStAtomics], s_red);
    if (blockIdx.x != 0 && threadIdx.x < kStCount) st[threadIdx.x] = 0;
    finish_block(p.ctl, last, UseCnt ? PICO_ALGO_CNTCORE : PICO_ALGO_NBRCORE, st,
                 kStCount);
}

// Persistent grid of the kernel: every co-resident CTA, capped per SM.
int persistent_grid(const void *fn, const LaunchCfg &cfg, int *cache)
{
    int &o = cache[cfg.device & 63];
    if (o == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kThreads, 0) != cudaSuccess ||
            o <= 0)
            return -1;
    }
    return cfg.sms * (o < cfg.max_blocks_per_sm ? o : cfg.max_blocks_per_sm);
}

}  // namespace

size_t gpp_ws_bytes(long long n, long long m)
{
    Carver c(nullptr);
    c.take<Ctrl>(1);
    c.take<int>(n);             // deg
    c.take<unsigned char>(n);   // rem
    c.take<int>(n);             // qs
    c.take<int2>(chunk_capacity(m));
    return c.size();
}

size_t index2core_ws_bytes(long long n, long long m)
{
    Carver c(nullptr);
    c.take<Ctrl>(1);
    for (int i = 0; i < 4; ++i) c.take<int>(n);   // est, newv, cnt, stamp
    c.take<int>(m);                               // hist
    for (int i = 0; i < 4; ++i) c.take<int>(n);   // as[2], fs, cs
    for (int i = 0; i < 4; ++i) c.take<int2>(chunk_capacity(m));
    return c.size();
}

template <typename Off>
int launch_gpp(const Off *rp, const int *ci, long long n, long long m, int *core, void *ws,
               LastResult *last, cudaStream_t stream, const LaunchCfg &cfg)
{
    Carver c(ws);
    gpp::Params<Off> p;
    p.rp = rp;
    p.ci = ci;
    p.n = n;
    p.core = core;
    p.ctl = c.take<Ctrl>(1);
    p.deg = c.take<int>(n);
    p.rem = c.take<unsigned char>(n);
    p.qs = c.take<int>(n);
    p.qb_cap = (unsigned)chunk_capacity(m);
    p.qb = c.take<int2>(p.qb_cap);
    p.tn = cfg.tn;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;
    static int occ[64] = {};
    const int grid = persistent_grid((const void *)gpp_kernel<Off>, cfg, occ);
    if (grid <= 0) return -3;
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&p, &last, &limit};
    if (launch_cooperative((const void *)gpp_kernel<Off>, dim3(grid), dim3(kThreads),
                                    args, 0, stream) != cudaSuccess)
        return -3;
    return 0;
}

template <typename Off>
int launch_index2core(const Off *rp, const int *ci, long long n, long long m, int *core,
                      void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg,
                      bool use_cnt)
{
    Carver c(ws);
    i2c::Params<Off> p;
    p.rp = rp;
    p.ci = ci;
    p.n = n;
    p.m = m;
    p.core = core;
    p.ctl = c.take<Ctrl>(1);
    p.est = c.take<int>(n);
    p.newv = c.take<int>(n);
    p.cnt = c.take<int>(n);
    p.stamp = c.take<int>(n);
    p.hist = c.take<int>(m);
    p.as[0] = c.take<int>(n);
    p.as[1] = c.take<int>(n);
    p.fs = c.take<int>(n);
    p.cs = c.take<int>(n);
    p.cap = (unsigned)chunk_capacity(m);
    p.ab[0] = c.take<int2>(p.cap);
    p.ab[1] = c.take<int2>(p.cap);
    p.fb = c.take<int2>(p.cap);
    p.cb = c.take<int2>(p.cap);
    p.tn = cfg.tn;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) return -3;
    static int occ[2][64] = {};
    const void *fn = use_cnt ? (const void *)i2c_kernel<Off, true>
                             : (const void *)i2c_kernel<Off, false>;
    const int grid = persistent_grid(fn, cfg, occ[use_cnt ? 1 : 0]);
    if (grid <= 0) return -3;
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&p, &last, &limit};
    if (launch_cooperative(fn, dim3(grid), dim3(kThreads), args, 0, stream) !=
        cudaSuccess)
        return -3;
    return 0;
}

template int launch_gpp<int>(const int *, const int *, long long, long long, int *, void *,
                             LastResult *, cudaStream_t, const LaunchCfg &);
template int launch_gpp<long long>(const long long *, const int *, long long, long long, int *,
                                   void *, LastResult *, cudaStream_t, const LaunchCfg &);
template int launch_index2core<int>(const int *, const int *, long long, long long, int *,
                                    void *, LastResult *, cudaStream_t, const LaunchCfg &, bool);
template int launch_index2core<long long>(const long long *, const int *, long long, long long,
                                          int *, void *, LastResult *, cudaStream_t,
                                          const LaunchCfg &, bool);

}  // namespace pico
