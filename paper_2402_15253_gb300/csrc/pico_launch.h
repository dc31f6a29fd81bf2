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
    size_t l2_window = 0;          // largest L2 access-policy window to mark persisting (0: none)
    bool validate = false;         // single-graph calls validate their graph first (PICO_VALIDATE=1)
};

// Launches a persistent kernel whose CTAs must all be resident at once (its
// grid barrier waits for every CTA): a cooperative launch, made through
// cudaLaunchKernelExC so that a stream capture can record it in a CUDA graph.
// With win_bytes > 0, the launch also marks [win, win + win_bytes) as
// persisting in L2 (an access-policy window; the lines keep that status after
// the kernel until l2_release).
inline cudaError_t launch_cooperative(const void *fn, dim3 grid, dim3 block, void **args,
                                      size_t smem, cudaStream_t stream,
                                      const void *win = nullptr, size_t win_bytes = 0)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (win && win_bytes > 0) {
        attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[1].val.accessPolicyWindow.base_ptr = const_cast<void *>(win);
        attr[1].val.accessPolicyWindow.num_bytes = win_bytes;
        attr[1].val.accessPolicyWindow.hitRatio = 1.0f;
        attr[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        lc.numAttrs = 2;
    }
    return cudaLaunchKernelExC(&lc, fn, args);
}

// Returns the lines of [p, p + bytes) that a launch marked persisting to
// normal status (a read of the range under a window with the normal
// property), so that they stop taking L2 from later kernels. Stream-ordered.
cudaError_t l2_release(const void *p, size_t bytes, cudaStream_t stream);

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

// Input validation (validate.cu): ORs the PICO_DEFECT_* bits it finds into
// *flag (device memory, zeroed by the caller), stream-ordered.
template <typename Off>
int launch_validate(const Off *rp, const int *ci, long long n, long long m, unsigned *flag,
                    cudaStream_t stream, const LaunchCfg &cfg);

// The current device's launch configuration and per-device status record
// (capi.cu); returns a pico_status.
int current_device(LaunchCfg *cfg, LastResult **last);


}  // namespace pico
