// pico_coreness_noalloc: PeelOne for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc or any allocating routine while they
// run: code that executes inside a memory budget fixed up front (a service
// that reserved all device memory at start-up), a host thread that must not
// take the allocator's locks, or an embedding framework that owns every
// allocation. The regular entry points take their scratch from CUDA's
// stream-ordered allocator, so those callers get this variant instead: its
// scratch is one array compiled into the library (`g_noalloc_scratch`,
// kNoAllocScratchBytes bytes), which the CUDA runtime places in device memory
// when it loads this module on a device and keeps there until the process
// exits.
//
// The host cannot pass `g_noalloc_scratch` itself to a kernel: in host code
// that name refers to a host-side stand-in, not to device memory. The device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) by the first call made on the device, and cached.
//
// Every call on a device shares the one array, and the array keeps whatever
// the previous call left in it: each call clears the parts that must start at
// zero (the control block and the status record) on its stream before the
// kernel runs. Calls whose work overlaps on the GPU (concurrent streams, or
// host threads racing) would use the same array at once and must not happen.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "pico.h"
#include "pico_device.cuh"
#include "pico_launch.h"

namespace {

// Largest graph this entry point accepts (see include/pico.h).
constexpr long long kMaxN = PICO_NOALLOC_MAX_VERTICES;
constexpr long long kMaxM = PICO_NOALLOC_MAX_ARCS;
// Status record + PeelOne scratch for the limits above under every allowed
// tuning (17.9 MiB), rounded up.
constexpr size_t kNoAllocScratchBytes = size_t(19) << 20;
constexpr size_t kStatusBytes = 512;   // LastResult header, padded to 256-byte alignment
// The status record's header (status, statistics, trace switch) must fit in
// kStatusBytes; its trace array is never written by this entry point.
static_assert(offsetof(pico::LastResult, trace) <= kStatusBytes, "status record too large");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    pico::LaunchCfg cfg{};
};

constexpr int kMaxDevices = 64;
NoAllocDevice g_na[kMaxDevices];
std::mutex g_na_mu;

// One-time per-device set-up: checks the device and resolves the device
// address of the scratch array. Performs no allocation.
int noalloc_device(NoAllocDevice **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PICO_ERR_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lock(g_na_mu);
    NoAllocDevice &d = g_na[dev];
    if (!d.ready) {
        int major = 0, minor = 0, sms = 0, coop = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
            cudaGetLastError();
            return PICO_ERR_NO_DEVICE;
        }
        if (major != 10 || minor != 3 || !coop) return PICO_ERR_NO_DEVICE;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return PICO_ERR_CUDA;
        }
        if (kStatusBytes + pico::peelone_ws_bytes(kMaxN, kMaxM) > kNoAllocScratchBytes)
            return PICO_ERR_INVALID_ARG;   // the array is too small for the stated limits
        d.scratch = static_cast<unsigned char *>(p);
        d.cfg.device = dev;
        d.cfg.sms = sms;
        d.cfg.max_blocks_per_sm = 2;
        d.cfg.limit_ns = 4000ull * 1000000ull;
        d.cfg.tn = pico::Tuning{pico::kSmallDeg, pico::kChunk, pico::kClusterLog2};
        d.cfg.batched_threads = pico::kThreads;
        d.ready = true;
    }
    *out = &d;
    return PICO_OK;
}

}  // namespace

extern "C" int pico_coreness_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int64_t n,
                                     int64_t m, int32_t *out_core, int32_t *out_status,
                                     pico_stream_t stream)
{
    if (n < 0 || m < 0) return PICO_ERR_INVALID_ARG;
    if (n > kMaxN || m > kMaxM) return PICO_ERR_INVALID_ARG;   // beyond the scratch array
    if (n > 0 && (!row_ptr || !out_core || (m > 0 && !col_idx))) return PICO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocDevice *d = nullptr;
    int rc = noalloc_device(&d);
    if (rc != PICO_OK) return rc;
    pico::LastResult *status = reinterpret_cast<pico::LastResult *>(d->scratch);
    if (cudaMemsetAsync(status, 0, offsetof(pico::LastResult, trace), s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (n > 0 && m == 0 &&
        cudaMemsetAsync(out_core, 0, (size_t)n * sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (n > 0 && m > 0 &&
        pico::launch_peelone<int>(row_ptr, col_idx, n, m, out_core, d->scratch + kStatusBytes,
                                  status, s, d->cfg) != 0) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (out_status &&
        cudaMemcpyAsync(out_status, &status->status, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}
