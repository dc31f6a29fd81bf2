// Host-side interface between the C ABI (capi.cu) and the kernel translation
// units. Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pico_device.cuh"

namespace pico {

struct LastResult;

// Launch geometry and tuning of the persistent kernels for the current device.
struct LaunchCfg {
    int device;
    int sms;                       // streaming multiprocessors
    int max_blocks_per_sm;         // cap on co-resident CTAs per SM
    unsigned long long limit_ns;   // time limit of every device-side wait
    Tuning tn;                     // degree-class work assignment
    int batched_threads;           // threads per CTA of the batched kernel (256 or 512)
    bool peel_async = false;       // single-graph PeelOne: asynchronous levels (run_async)
};

// Launches a persistent kernel whose CTAs must all be resident at once (its
// grid barrier waits for every CTA): a cooperative launch, made through
// cudaLaunchKernelExC so that a stream capture can record it in a CUDA graph.
inline cudaError_t launch_cooperative(const void *fn, dim3 grid, dim3 block, void **args,
                                      size_t smem, cudaStream_t stream)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelExC(&lc, fn, args);
}

// Sub-buffer carving of a scratch allocation (256-byte aligned pieces).
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
    size_t size() const { return (off + 255) & ~size_t(255); }
};

// Capacity of the list of (vertex, chunk) entries of large vertices: every
// vertex of degree > kSmallDeg contributes ceil(deg / kChunk) entries.
size_t chunk_capacity(long long m);

// async: with the arrays of asynchronous levels (peel::run_async)
size_t peelone_ws_bytes(long long n, long long m, bool async = false);
size_t histocore_ws_bytes(long long n, long long m);

// mode: kPeelRepair (PeelOne), kPeelCas or kPeelAddBack (ablations)
template <typename Off>
int launch_peelone(const Off *rp, const int *ci, long long n, long long m, int *core,
                   void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg,
                   int mode = 0);

// init_est: start from these estimates (core maintenance; may alias core)
template <typename Off>
int launch_histocore(const Off *rp, const int *ci, long long n, long long m, int *core,
                     void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg,
                     const int *init_est = nullptr);

// the comparison baselines of Sec. V (ablation.cu)
size_t gpp_ws_bytes(long long n, long long m);
size_t index2core_ws_bytes(long long n, long long m);

template <typename Off>
int launch_gpp(const Off *rp, const int *ci, long long n, long long m, int *core, void *ws,
               LastResult *last, cudaStream_t stream, const LaunchCfg &cfg);

template <typename Off>
int launch_index2core(const Off *rp, const int *ci, long long n, long long m, int *core,
                      void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg,
                      bool use_cnt);

// core maintenance (dyn.cu)
namespace dyn {
size_t maint_ws_bytes(long long n, long long m);
}

// method selection per graph (hybrid.cu)
size_t hybrid_ws_bytes(long long n, long long m);

template <typename Off>
int launch_hybrid(const Off *rp, const int *ci, long long n, long long m, int *core, void *ws,
                  LastResult *last, cudaStream_t stream, const LaunchCfg &cfg);

size_t batched_ws_bytes(int G, long long total_n, long long total_m, int algo);

int launch_batched(const int64_t *vtx_off, const int64_t *arc_off, int G, const int32_t *rp,
                   const int32_t *ci, long long total_n, long long total_m, int32_t *core,
                   int algo, void *ws, LastResult *last, cudaStream_t stream, const LaunchCfg &cfg);

int selftest_wait_timeout(LastResult *last, int limit_ms, cudaStream_t stream, const LaunchCfg &cfg);

// The current device's launch configuration and per-device status record
// (capi.cu); returns a pico_status.
int current_device(LaunchCfg *cfg, LastResult **last);


}  // namespace pico
