// Self-test of the failure path of the persistent kernels' bounded waits.
//
// The kernel runs the grid barrier of the persistent kernels with one CTA
// that never arrives, so no CTA ever releases the others: their waits run
// out after the given limit, record PICO_ERR_TIMEOUT in the status word and
// return, and the launch ends. Nothing faults, traps or hangs; the context
// stays usable, which the host then checks by reading the status.
#include "pico.h"
#include "pico_device.cuh"
#include "pico_launch.h"

namespace pico {
namespace {

__global__ void __launch_bounds__(256) wait_timeout_kernel(Ctrl *ctl, LastResult *last,
                                                           unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned long long st[kStCount];
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    if (blockIdx.x != 0) grid_sync(ctl, s_snap, limit_ns, 0);   // CTA 0 never arrives
    finish_block(ctl, last, -1, st, kStCount);
}

}  // namespace

int selftest_wait_timeout(LastResult *last, int limit_ms, cudaStream_t stream, const LaunchCfg &cfg)
{
    Ctrl *ctl = nullptr;
    if (cudaMallocAsync(&ctl, sizeof(Ctrl), stream) != cudaSuccess) return -2;
    int rc = 0;
    if (cudaMemsetAsync(ctl, 0, sizeof(Ctrl), stream) != cudaSuccess) rc = -3;
    unsigned long long limit = (unsigned long long)limit_ms * 1000000ull;
    void *args[] = {&ctl, &last, &limit};
    if (rc == 0 && launch_cooperative((const void *)wait_timeout_kernel, dim3(cfg.sms),
                                               dim3(256), args, 0, stream) != cudaSuccess)
        rc = -3;
    cudaFreeAsync(ctl, stream);
    return rc;
}

}  // namespace pico
