// The C ABI declared in include/pico.h: argument checks, per-device state,
// stream-ordered scratch allocation and dispatch to the persistent kernels.
#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "pico.h"
#include "pico_device.cuh"
#include "pico_launch.h"

static_assert(PICO_UPDATE_AUTO == pico::kUpdateAuto && PICO_UPDATE_PUSH == pico::kUpdatePush &&
                  PICO_UPDATE_PULL == pico::kUpdatePull,
              "update directions of the ABI and the kernels differ");

namespace {

struct DeviceState {
    bool init = false;
    pico::LaunchCfg cfg{};
    pico::LastResult *last = nullptr;   // device memory
};

constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

long long env_ll(const char *name, long long dflt)
{
    const char *s = std::getenv(name);
    if (!s || !*s) return dflt;
    char *end = nullptr;
    long long v = std::strtoll(s, &end, 10);
    return (end && *end == '\0' && v > 0) ? v : dflt;
}

// Per-device setup, done once per device by the first call on it (so the
// first call should not be inside a stream capture).
int device_state(DeviceState **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PICO_ERR_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.init) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return PICO_ERR_NO_DEVICE;
        }
        if (prop.major != 10 || prop.minor != 3 || !prop.cooperativeLaunch)
            return PICO_ERR_NO_DEVICE;
        d.cfg.device = dev;
        d.cfg.sms = prop.multiProcessorCount;
        d.cfg.max_blocks_per_sm = (int)env_ll("PICO_BLOCKS_PER_SM", 2);
        d.cfg.limit_ns = (unsigned long long)env_ll("PICO_WAIT_LIMIT_MS", 4000) * 1000000ull;
        d.cfg.tn = pico::Tuning{pico::kSmallDeg, pico::kChunk, pico::kClusterLog2};
        d.cfg.batched_threads = pico::kThreads;
        d.cfg.peel_async = env_ll("PICO_PEEL_WAVES", 0) == 0;
        d.cfg.validate = env_ll("PICO_VALIDATE", 0) == 1;
        // PICO_PEEL_GUARD=G: PeelOne reads a neighbour before decrementing it
        // in the chunks of vertices of degree > G * k (0: never)
        if (const char *g = std::getenv("PICO_PEEL_GUARD"); g && *g)
            d.cfg.tn.peel_guard = std::max(0, std::atoi(g));
        // With PICO_L2_PERSIST=1, the L2 set-aside for persisting lines (a
        // limit of this process's context) is raised to the device maximum,
        // and the PeelOne launches mark their residual degrees persisting and
        // return them to normal status when they end. Off by default: the
        // set-aside slows HistoCore in the same process more than it helps
        // PeelOne.
        d.cfg.l2_window = 0;
        if (env_ll("PICO_L2_PERSIST", 0) == 1) {
            int mx = 0, mw = 0;
            size_t cur = 0;
            if (cudaDeviceGetAttribute(&mx, cudaDevAttrMaxPersistingL2CacheSize, dev) ==
                    cudaSuccess &&
                cudaDeviceGetAttribute(&mw, cudaDevAttrMaxAccessPolicyWindowSize, dev) ==
                    cudaSuccess &&
                mx > 0 && mw > 0 && cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
                if (cur < (size_t)mx && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, mx) == cudaSuccess)
                    cur = mx;
                d.cfg.l2_window = std::min<size_t>(cur, (size_t)mw);
            }
            cudaGetLastError();
        }
        if (cudaMalloc(&d.last, sizeof(pico::LastResult)) != cudaSuccess) {
            cudaGetLastError();
            return PICO_ERR_OOM;
        }
        if (cudaMemset(d.last, 0, sizeof(pico::LastResult)) != cudaSuccess) {
            cudaGetLastError();
            return PICO_ERR_CUDA;
        }
        const unsigned trace_on = env_ll("PICO_TRACE", 0) > 0 ? 1u : 0u;
        if (cudaMemcpy(&d.last->trace_on, &trace_on, sizeof(unsigned), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            cudaGetLastError();
            return PICO_ERR_CUDA;
        }
        // Keep freed scratch in this process's pool for the next call.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
        d.init = true;
    }
    *out = &d;
    return PICO_OK;
}

// Launch configuration of a device, copied under the lock (pico_set_tuning
// may change it from another thread).
pico::LaunchCfg cfg_of(const DeviceState *d)
{
    std::lock_guard<std::mutex> lock(g_mu);
    return d->cfg;
}

// Host-side fault injection for tests: with PICO_FAULT_ALLOC=1 every
// scratch allocation of the compute entry points is reported as failed.
bool fault_alloc() { return env_ll("PICO_FAULT_ALLOC", 0) > 0; }

bool single_graph_algo(int algo) { return algo >= PICO_ALGO_PEELONE && algo <= PICO_ALGO_AUTO; }

size_t single_ws_bytes(long long n, long long m, int algo)
{
    switch (algo) {
    case PICO_ALGO_PEELONE:
    case PICO_ALGO_PEEL_CAS:
    case PICO_ALGO_PEEL_ADDBACK: return pico::peelone_ws_bytes(n, m, true);
    case PICO_ALGO_HISTOCORE: return pico::histocore_ws_bytes(n, m);
    case PICO_ALGO_GPP: return pico::gpp_ws_bytes(n, m);
    case PICO_ALGO_NBRCORE:
    case PICO_ALGO_CNTCORE: return pico::index2core_ws_bytes(n, m);
    case PICO_ALGO_AUTO: return pico::hybrid_ws_bytes(n, m);
    default: return 0;
    }
}

template <typename Off>
int launch_single(const Off *rp, const int32_t *ci, int64_t n, int64_t m, int32_t *out, int algo,
                  void *ws, pico::LastResult *last, cudaStream_t stream,
                  const pico::LaunchCfg &cfg)
{
    switch (algo) {
    case PICO_ALGO_PEELONE:
        return pico::launch_peelone<Off>(rp, ci, n, m, out, ws, last, stream, cfg,
                                         pico::kPeelRepair);
    case PICO_ALGO_PEEL_CAS:
        return pico::launch_peelone<Off>(rp, ci, n, m, out, ws, last, stream, cfg,
                                         pico::kPeelCas);
    case PICO_ALGO_PEEL_ADDBACK:
        return pico::launch_peelone<Off>(rp, ci, n, m, out, ws, last, stream, cfg,
                                         pico::kPeelAddBack);
    case PICO_ALGO_HISTOCORE:
        return pico::launch_histocore<Off>(rp, ci, n, m, out, ws, last, stream, cfg);
    case PICO_ALGO_GPP: return pico::launch_gpp<Off>(rp, ci, n, m, out, ws, last, stream, cfg);
    case PICO_ALGO_AUTO: return pico::launch_hybrid<Off>(rp, ci, n, m, out, ws, last, stream, cfg);
    case PICO_ALGO_NBRCORE:
    case PICO_ALGO_CNTCORE:
        return pico::launch_index2core<Off>(rp, ci, n, m, out, ws, last, stream, cfg,
                                            algo == PICO_ALGO_CNTCORE);
    default: return -1;
    }
}

// Validates one graph (see pico_validate_graph): two kernels, then the
// defect word is read back (the stream is synchronised).
template <typename Off>
int validate_impl(const Off *rp, const int32_t *ci, int64_t n, int64_t m, uint32_t *defects,
                  cudaStream_t stream)
{
    if (defects) *defects = 0;
    if (n < 0 || m < 0) return PICO_ERR_INVALID_ARG;
    if (n == 0) {
        if (m == 0) return PICO_OK;
        if (defects) *defects = PICO_DEFECT_ROWS;
        return PICO_ERR_BAD_GRAPH;
    }
    if (!rp || (m > 0 && !ci)) return PICO_ERR_INVALID_ARG;
    if (n >= INT32_MAX || (sizeof(Off) == 4 && m >= INT32_MAX)) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    unsigned *flag = nullptr;
    if (fault_alloc() || cudaMallocAsync(&flag, sizeof(unsigned), stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_OOM;
    }
    unsigned found = 0;
    bool ok = cudaMemsetAsync(flag, 0, sizeof(unsigned), stream) == cudaSuccess &&
              pico::launch_validate<Off>(rp, ci, n, m, flag, stream, cfg_of(d)) == 0 &&
              cudaMemcpyAsync(&found, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, stream) ==
                  cudaSuccess;
    cudaFreeAsync(flag, stream);
    ok = cudaStreamSynchronize(stream) == cudaSuccess && ok;
    if (!ok) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (defects) *defects = found;
    return found ? PICO_ERR_BAD_GRAPH : PICO_OK;
}

template <typename Off>
int coreness_impl(const Off *rp, const int32_t *ci, int64_t n, int64_t m, int32_t *out,
                  int algo, cudaStream_t stream)
{
    if (n < 0 || m < 0 || !single_graph_algo(algo)) return PICO_ERR_INVALID_ARG;
    if (n == 0) return PICO_OK;
    if (!rp || !out || (m > 0 && !ci)) return PICO_ERR_INVALID_ARG;
    if (n >= INT32_MAX) return PICO_ERR_INVALID_ARG;
    if (sizeof(Off) == 4 && m >= INT32_MAX) return PICO_ERR_INVALID_ARG;
    if (m >= (1ll << 36)) return PICO_ERR_INVALID_ARG;   // chunk lists use 32-bit indices
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    if (cfg_of(d).validate) {   // PICO_VALIDATE=1
        rc = validate_impl<Off>(rp, ci, n, m, nullptr, stream);
        if (rc != PICO_OK) return rc;
    }
    if (m == 0) {   // no arcs: every vertex is isolated
        if (cudaMemsetAsync(out, 0, (size_t)n * sizeof(int32_t), stream) != cudaSuccess) {
            cudaGetLastError();
            return PICO_ERR_CUDA;
        }
        return PICO_OK;
    }
    const size_t bytes = single_ws_bytes(n, m, algo);
    void *ws = nullptr;
    if (fault_alloc() || cudaMallocAsync(&ws, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_OOM;
    }
    rc = launch_single<Off>(rp, ci, n, m, out, algo, ws, d->last, stream, cfg_of(d));
    cudaFreeAsync(ws, stream);
    if (rc != 0) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

}  // namespace

namespace pico {
int current_device(LaunchCfg *cfg, LastResult **last)
{
    DeviceState *d = nullptr;
    const int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    *cfg = cfg_of(d);
    *last = d->last;
    return PICO_OK;
}
}  // namespace pico

extern "C" {

int pico_coreness(const int32_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                  int32_t *out_core, int algo, pico_stream_t stream)
{
    return coreness_impl<int>(row_ptr, col_idx, n, m, out_core, algo, (cudaStream_t)stream);
}

int pico_coreness_i64(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                      int32_t *out_core, int algo, pico_stream_t stream)
{
    return coreness_impl<long long>(reinterpret_cast<const long long *>(row_ptr), col_idx, n, m,
                                    out_core, algo, (cudaStream_t)stream);
}

int pico_validate_graph(const int32_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                        uint32_t *defects, pico_stream_t stream)
{
    return validate_impl<int>(row_ptr, col_idx, n, m, defects, (cudaStream_t)stream);
}

int pico_validate_graph_i64(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                            uint32_t *defects, pico_stream_t stream)
{
    return validate_impl<long long>(reinterpret_cast<const long long *>(row_ptr), col_idx, n, m,
                                    defects, (cudaStream_t)stream);
}

int pico_coreness_batched(const int64_t *vtx_off, const int64_t *arc_off, int32_t G,
                          const int32_t *row_ptr, const int32_t *col_idx,
                          int64_t total_vertices, int64_t total_arcs, int32_t *out_core,
                          int algo, pico_stream_t stream)
{
    if (algo == PICO_ALGO_AUTO) algo = PICO_ALGO_PEELONE;   // faster on every measured class
    if (G < 0 || total_vertices < 0 || total_arcs < 0 ||
        (algo != PICO_ALGO_PEELONE && algo != PICO_ALGO_HISTOCORE))
        return PICO_ERR_INVALID_ARG;
    if (G == 0 || total_vertices == 0) return PICO_OK;
    if (!vtx_off || !arc_off || !row_ptr || !out_core || (total_arcs > 0 && !col_idx))
        return PICO_ERR_INVALID_ARG;
    if (total_vertices >= (1ll << 40) || total_arcs >= (1ll << 40)) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = pico::batched_ws_bytes(G, total_vertices, total_arcs, algo);
    void *ws = nullptr;
    if (fault_alloc() || cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_OOM;
    }
    rc = pico::launch_batched(vtx_off, arc_off, G, row_ptr, col_idx, total_vertices, total_arcs,
                              out_core, algo, ws, d->last, s, cfg_of(d));
    cudaFreeAsync(ws, s);
    if (rc != 0) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

size_t pico_workspace_bytes_batched(int32_t G, int64_t total_vertices, int64_t total_arcs,
                                    int algo)
{
    if (G < 0 || total_vertices < 0 || total_arcs < 0) return 0;
    if (algo == PICO_ALGO_AUTO) algo = PICO_ALGO_PEELONE;
    if (algo != PICO_ALGO_PEELONE && algo != PICO_ALGO_HISTOCORE) return 0;
    return pico::batched_ws_bytes(G, total_vertices, total_arcs, algo);
}

size_t pico_workspace_bytes(int64_t n, int64_t m, int algo)
{
    if (n < 0 || m < 0) return 0;
    return single_ws_bytes(n, m, algo);
}

const char *pico_status_string(int status)
{
    switch (status) {
    case PICO_OK: return "ok";
    case PICO_ERR_INVALID_ARG: return "invalid argument";
    case PICO_ERR_OOM: return "out of device memory";
    case PICO_ERR_CUDA: return "CUDA runtime error";
    case PICO_ERR_NOT_CONVERGED: return "device loop exceeded its bound";
    case PICO_ERR_TIMEOUT: return "device-side wait timed out";
    case PICO_ERR_BAD_GRAPH: return "malformed graph";
    case PICO_ERR_NO_DEVICE: return "no usable sm_103 device";
    default: return "unknown status";
    }
}

int pico_last_device_status(pico_stream_t stream)
{
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    int st = 0;
    if (cudaMemcpy(&st, &d->last->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(&d->last->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return st;
}

int pico_get_stats(pico_stream_t stream, pico_stats *out)
{
    if (!out) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    pico::LastResult h;
    if (cudaMemcpy(&h, d->last, offsetof(pico::LastResult, trace_len), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    std::memset(out, 0, sizeof(*out));
    out->algo = h.algo;
    out->levels = (int64_t)h.stats[pico::kStLevels];
    out->kmax = (int64_t)h.stats[pico::kStKmax];
    out->subrounds = (int64_t)h.stats[pico::kStSubrounds];
    out->scans = (int64_t)h.stats[pico::kStScans];
    out->rounds = (int64_t)h.stats[pico::kStRounds];
    out->frontier = (int64_t)h.stats[pico::kStFrontier];
    out->barriers = (int64_t)h.stats[pico::kStBarriers];
    out->arcs = (int64_t)h.stats[pico::kStArcs];
    out->atomics = (int64_t)h.stats[pico::kStAtomics];
    out->slots = (int64_t)h.stats[pico::kStSlots];
    out->blocks = (int64_t)h.stats[pico::kStBlocks];
    out->scanned = (int64_t)h.stats[pico::kStScanned];
    out->pulled = (int64_t)h.stats[pico::kStPulled];
    out->pull_rounds = (int64_t)h.stats[pico::kStPullRounds];
    out->extra = (int64_t)h.stats[pico::kStExtra];
    out->active = (int64_t)h.stats[pico::kStActive];
    for (int i = 0; i < 8; ++i) {
        out->phase_ns[i] = (int64_t)h.stats[pico::kStPhaseNs + i];
        out->phase_count[i] = (int64_t)h.stats[pico::kStPhaseCount + i];
    }
    return PICO_OK;
}

int pico_get_trace(pico_stream_t stream, int64_t *out, int cap)
{
    if (cap < 0 || (cap > 0 && !out)) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    unsigned len = 0;
    if (cudaMemcpy(&len, &d->last->trace_len, sizeof(len), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    const int k = (int)(len < (unsigned)cap ? len : (unsigned)cap);
    if (k == 0) return 0;
    static thread_local pico::TraceEntry buf[pico::kTraceCap];
    if (cudaMemcpy(buf, d->last->trace, sizeof(pico::TraceEntry) * k, cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    for (int i = 0; i < k; ++i) {
        out[3 * i] = buf[i].kind;
        out[3 * i + 1] = buf[i].units;
        out[3 * i + 2] = (int64_t)buf[i].ns;
    }
    return k;
}

int pico_selftest_wait_timeout(int limit_ms, pico_stream_t stream)
{
    if (limit_ms < 1 || limit_ms > 10000) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    (void)pico_last_device_status(stream);   // start from a clean status
    rc = pico::selftest_wait_timeout(d->last, limit_ms, (cudaStream_t)stream, cfg_of(d));
    if (rc != 0) {
        cudaGetLastError();
        return rc == -2 ? PICO_ERR_OOM : PICO_ERR_CUDA;
    }
    return pico_last_device_status(stream);
}

int pico_set_tuning(int small_deg, int chunk, int batched_threads, int cluster_log2)
{
    if (small_deg < pico::kMinSmallDeg || small_deg > pico::kMaxSmallDeg ||
        chunk < pico::kMinChunk || chunk > pico::kMaxChunk ||
        (batched_threads != 256 && batched_threads != 512) || cluster_log2 < 10 ||
        cluster_log2 > pico::kClusterNever)
        return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    d->cfg.tn.small_deg = small_deg;
    d->cfg.tn.chunk = chunk;
    d->cfg.tn.cluster_log2 = cluster_log2;
    d->cfg.batched_threads = batched_threads;
    return PICO_OK;
}

int pico_get_tuning(int *small_deg, int *chunk, int *batched_threads, int *cluster_log2)
{
    if (!small_deg || !chunk || !batched_threads || !cluster_log2) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    *small_deg = d->cfg.tn.small_deg;
    *chunk = d->cfg.tn.chunk;
    *batched_threads = d->cfg.batched_threads;
    *cluster_log2 = d->cfg.tn.cluster_log2;
    return PICO_OK;
}

int pico_set_histo_update(int mode, int pull_pct)
{
    if (mode < PICO_UPDATE_AUTO || mode > PICO_UPDATE_PULL || pull_pct < 1 || pull_pct > 100)
        return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    d->cfg.tn.update_mode = mode;
    d->cfg.tn.pull_pct = pull_pct;
    return PICO_OK;
}

int pico_get_histo_update(int *mode, int *pull_pct)
{
    if (!mode || !pull_pct) return PICO_ERR_INVALID_ARG;
    DeviceState *d = nullptr;
    int rc = device_state(&d);
    if (rc != PICO_OK) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    *mode = d->cfg.tn.update_mode;
    *pull_pct = d->cfg.tn.pull_pct;
    return PICO_OK;
}

int pico_version(void) { return 100; }

}  // extern "C"
