// Input validation of a single-graph CSR: the paper's graphs are simple and
// undirected (Sec. II-A), and both methods rely on it (PeelOne decrements
// each neighbour once per arc, HistoCore's pulled rounds read an edit from
// the far end of each arc). Two launches on the caller's stream:
//   rows  row_ptr[0] == 0, row_ptr non-decreasing, row_ptr[n] == m;
//   arcs  (only when the rows passed, so that every row lies inside
//         col_idx) every neighbour id in [0, n), no self-loop, every row
//         strictly increasing (sorted, hence no duplicate), and every arc
//         (v, u) matched by (u, v), looked up by binary search in u's row.
// Each kernel ORs the defects it finds into one device word. Every load is
// bounds-checked first, so a malformed graph becomes a reported defect,
// never an out-of-range access.
#include "pico.h"
#include "pico_device.cuh"
#include "pico_launch.h"

namespace pico {
namespace {

template <typename Off>
__global__ void __launch_bounds__(256)
    validate_rows(const Off *rp, long long n, long long m, unsigned *flag)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        const long long a = (long long)rp[v];
        if (v == 0 && a != 0) bad = true;
        if (v == n && a != m) bad = true;
        if (v < n) {
            const long long b = (long long)rp[v + 1];
            if (a < 0 || b < a || b > m) bad = true;
        }
    }
    if (bad) atomicOr(flag, PICO_DEFECT_ROWS);
}

template <typename Off>
__global__ void __launch_bounds__(256)
    validate_arcs(const Off *rp, const int *ci, long long n, unsigned *flag)
{
    // the rows kernel ran before on this stream: its word is final here
    if (*reinterpret_cast<volatile unsigned *>(flag) & PICO_DEFECT_ROWS) return;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    // one warp per vertex, its lanes over the vertex's arcs
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const Off a = rp[v], b = rp[v + 1];
        for (Off e = a + lane; e < b; e += 32) {
            const int u = ci[e];
            if (u < 0 || (long long)u >= n) {
                bad |= PICO_DEFECT_IDS;
                continue;
            }
            if ((long long)u == v) bad |= PICO_DEFECT_LOOP;
            if (e + 1 < b && ci[e + 1] <= u) bad |= PICO_DEFECT_ORDER;
            // (v, u) needs (u, v): v in u's row (an unsorted row of u may
            // hide it; that row is reported as unsorted anyway)
            Off lo = rp[u];
            const Off end = rp[u + 1];
            Off hi = end;
            while (lo < hi) {
                const Off mid = lo + (hi - lo) / 2;
                if ((long long)ci[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= end || (long long)ci[lo] != v) bad |= PICO_DEFECT_ASYMMETRIC;
        }
    }
    bad = __reduce_or_sync(kFull, bad);
    if (bad && lane == 0) atomicOr(flag, bad);
}

}  // namespace

template <typename Off>
int launch_validate(const Off *rp, const int *ci, long long n, long long m, unsigned *flag,
                    cudaStream_t stream, const LaunchCfg &cfg)
{
    const unsigned blocks = (unsigned)(cfg.sms > 0 ? cfg.sms * 8 : 1024);
    validate_rows<Off><<<blocks, 256, 0, stream>>>(rp, n, m, flag);
    if (cudaGetLastError() != cudaSuccess) return -3;
    validate_arcs<Off><<<blocks, 256, 0, stream>>>(rp, ci, n, flag);
    if (cudaGetLastError() != cudaSuccess) return -3;
    return 0;
}

template int launch_validate<int>(const int *, const int *, long long, long long, unsigned *,
                                  cudaStream_t, const LaunchCfg &);
template int launch_validate<long long>(const long long *, const int *, long long, long long,
                                        unsigned *, cudaStream_t, const LaunchCfg &);

}  // namespace pico
