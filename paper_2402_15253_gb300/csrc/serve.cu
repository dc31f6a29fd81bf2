// Request server: continuous batching of coreness requests on one GPU.
//
// Clients submit host CSR graphs (pinned memory, so copies are asynchronous)
// with an arrival time. An engine thread owns the device work:
//   admission  arrived requests are taken in arrival order while the device
//              bytes they need (packed CSR + result + the batched call's
//              scratch, as pico_workspace_bytes_batched counts it) fit in the
//              budget next to the requests already on the device;
//   batching   the admitted requests form one micro-batch, copied into a
//              packed multi-graph CSR and solved by one batched launch
//              (pico_coreness_batched) on a free stream; up to `streams`
//              micro-batches run at once, so requests that arrive while others
//              are on the GPU are admitted as slots and memory free up and
//              their work overlaps on the device;
//   completion each micro-batch ends with an event; when it has fired the
//              results are in the clients' buffers, the memory returns to the
//              budget and the requests are reported done with their
//              completion time and the micro-batch's device time (events
//              around its copies in, its launch and its copies out).
// With single_graph = 1 and max_batch = 1 the engine instead runs one
// request at a time with the single-graph entry point (the sequential plain
// path, kept as the baseline).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "pico.h"

namespace {

using Clock = std::chrono::steady_clock;

long long now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch())
        .count();
}

struct Request {
    long long ticket;
    const int32_t *rp;
    const int32_t *ci;
    long long n, m;
    int32_t *out;
    long long arrival_ns;
};

struct Batch {
    std::vector<Request> reqs;
    size_t bytes = 0;
    void *dev = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    int slot = -1;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct pico_server {
    pico_server_config cfg;
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::vector<long long *> h_offsets;   // pinned, per slot: vtx_off | arc_off
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;           // submitted, in arrival order
    std::vector<Batch> inflight;
    std::vector<long long> done_tickets, done_times, done_device;
    size_t inflight_bytes = 0;
    long long next_ticket = 0, submitted = 0, completed = 0;
    int error = PICO_OK;
    bool stop = false;
    std::thread engine;

    size_t batch_bytes(long long G, long long tn, long long tm) const
    {
        size_t b = align256(sizeof(long long) * 2 * (G + 1)) + align256(4 * (tn + G)) +
                   align256(4 * tm) + align256(4 * tn);
        if (cfg.single_graph)
            b += pico_workspace_bytes(tn, tm, cfg.algo);
        else
            b += pico_workspace_bytes_batched((int32_t)G, tn, tm, cfg.algo);
        return b;
    }

    // Launches one micro-batch on stream slot `slot`. Called by the engine only.
    int launch(Batch &b)
    {
        cudaStream_t s = streams[b.slot];
        if (cudaEventRecord(b.start, s) != cudaSuccess) return PICO_ERR_CUDA;
        long long G = (long long)b.reqs.size(), tn = 0, tm = 0;
        long long *h = h_offsets[b.slot];
        h[0] = 0;
        h[G + 1] = 0;
        for (long long i = 0; i < G; ++i) {
            tn += b.reqs[i].n;
            tm += b.reqs[i].m;
            h[i + 1] = tn;
            h[G + 2 + i] = tm;
        }
        const size_t off_b = align256(sizeof(long long) * 2 * (G + 1));
        const size_t rp_b = align256(4 * (tn + G)), ci_b = align256(4 * tm);
        if (cudaMallocAsync(&b.dev, off_b + rp_b + ci_b + align256(4 * tn), s) != cudaSuccess) {
            b.dev = nullptr;
            return PICO_ERR_OOM;
        }
        char *base = static_cast<char *>(b.dev);
        long long *d_off = reinterpret_cast<long long *>(base);
        int32_t *d_rp = reinterpret_cast<int32_t *>(base + off_b);
        int32_t *d_ci = reinterpret_cast<int32_t *>(base + off_b + rp_b);
        int32_t *d_out = reinterpret_cast<int32_t *>(base + off_b + rp_b + ci_b);
        if (cudaMemcpyAsync(d_off, h, sizeof(long long) * 2 * (G + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return PICO_ERR_CUDA;
        long long vo = 0, ao = 0;
        for (long long i = 0; i < G; ++i) {
            const Request &r = b.reqs[i];
            if (cudaMemcpyAsync(d_rp + vo + i, r.rp, 4 * (r.n + 1), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                (r.m > 0 && cudaMemcpyAsync(d_ci + ao, r.ci, 4 * r.m, cudaMemcpyHostToDevice, s) !=
                                cudaSuccess))
                return PICO_ERR_CUDA;
            vo += r.n;
            ao += r.m;
        }
        int rc;
        if (cfg.single_graph) {
            rc = PICO_OK;
            vo = 0;
            ao = 0;
            for (long long i = 0; i < G && rc == PICO_OK; ++i) {
                const Request &r = b.reqs[i];
                rc = pico_coreness(d_rp + vo + i, d_ci + ao, r.n, r.m, d_out + vo, cfg.algo,
                                   (pico_stream_t)s);
                vo += r.n;
                ao += r.m;
            }
        } else {
            rc = pico_coreness_batched(reinterpret_cast<const int64_t *>(d_off),
                                       reinterpret_cast<const int64_t *>(d_off + G + 1), (int32_t)G,
                                       d_rp, d_ci, tn, tm, d_out,
                                       cfg.algo, (pico_stream_t)s);
        }
        if (rc != PICO_OK) return rc;
        vo = 0;
        for (long long i = 0; i < G; ++i) {
            const Request &r = b.reqs[i];
            if (r.n > 0 && cudaMemcpyAsync(r.out, d_out + vo, 4 * r.n, cudaMemcpyDeviceToHost, s) !=
                               cudaSuccess)
                return PICO_ERR_CUDA;
            vo += r.n;
        }
        if (cudaEventRecord(b.done, s) != cudaSuccess) return PICO_ERR_CUDA;
        cudaFreeAsync(b.dev, s);
        b.dev = nullptr;
        return PICO_OK;
    }

    void run()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lock(mu);
        while (true) {
            // completions
            for (size_t i = 0; i < inflight.size();) {
                Batch &b = inflight[i];
                const cudaError_t q = cudaEventQuery(b.done);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                if (q != cudaSuccess && error == PICO_OK) error = PICO_ERR_CUDA;
                const long long t = now_ns();
                float dev_ms = -1.0f;
                if (q == cudaSuccess && cudaEventElapsedTime(&dev_ms, b.start, b.done) != cudaSuccess)
                    dev_ms = -1.0f;
                const long long dev_ns = dev_ms >= 0.0f ? (long long)(dev_ms * 1e6) : -1;
                for (const Request &r : b.reqs) {
                    done_tickets.push_back(r.ticket);
                    done_times.push_back(t);
                    done_device.push_back(dev_ns);
                }
                completed += (long long)b.reqs.size();
                inflight_bytes -= b.bytes;
                slot_busy[b.slot] = false;
                cudaEventDestroy(b.start);
                cudaEventDestroy(b.done);
                inflight[i] = std::move(inflight.back());
                inflight.pop_back();
            }
            cudaGetLastError();
            if (stop && pending.empty() && inflight.empty()) break;

            // admission and launch
            const long long t = now_ns();
            int slot = -1;
            for (int i = 0; i < (int)slot_busy.size(); ++i)
                if (!slot_busy[i]) {
                    slot = i;
                    break;
                }
            bool launched = false;
            if (slot >= 0 && !pending.empty() && pending.front().arrival_ns <= t) {
                Batch b;
                long long tn = 0, tm = 0;
                while (!pending.empty() && pending.front().arrival_ns <= t &&
                       (int)b.reqs.size() < cfg.max_batch) {
                    const Request &r = pending.front();
                    const size_t need = batch_bytes((long long)b.reqs.size() + 1, tn + r.n, tm + r.m);
                    if (inflight_bytes + need > cfg.hbm_budget_bytes) break;
                    tn += r.n;
                    tm += r.m;
                    b.bytes = need;
                    b.reqs.push_back(r);
                    pending.pop_front();
                }
                if (!b.reqs.empty()) {
                    b.slot = slot;
                    slot_busy[slot] = true;
                    inflight_bytes += b.bytes;
                    cudaEventCreate(&b.start);   // timed: the device time of the batch
                    cudaEventCreate(&b.done);
                    lock.unlock();
                    const int rc = launch(b);
                    lock.lock();
                    if (rc != PICO_OK) {
                        if (error == PICO_OK) error = rc;
                        cudaGetLastError();
                        if (b.dev) cudaFreeAsync(b.dev, streams[b.slot]);
                        b.dev = nullptr;
                        cudaEventRecord(b.done, streams[b.slot]);
                    }
                    inflight.push_back(std::move(b));
                    launched = true;
                }
            }
            if (!launched) {
                // sleep until the next arrival, a submission, or a short poll
                long long wait = 20000;   // ns between completion polls
                if (inflight.empty() && !pending.empty())
                    wait = std::max(0ll, pending.front().arrival_ns - now_ns());
                if (inflight.empty() && pending.empty()) wait = 10000000;
                cv.wait_for(lock, std::chrono::nanoseconds(std::min(wait, 10000000ll)));
            }
        }
    }
};

extern "C" {

int64_t pico_clock_ns(void) { return now_ns(); }

pico_server *pico_server_create(const pico_server_config *cfg)
{
    if (!cfg || cfg->streams < 1 || cfg->streams > 64 || cfg->max_batch < 1 ||
        (cfg->algo != PICO_ALGO_PEELONE && cfg->algo != PICO_ALGO_HISTOCORE &&
         cfg->algo != PICO_ALGO_AUTO))
        return nullptr;
    pico_server *s = new pico_server();
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return nullptr;
    }
    for (int i = 0; i < cfg->streams; ++i) {
        cudaStream_t st;
        long long *h = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc(&h, sizeof(long long) * 2 * (cfg->max_batch + 1), cudaHostAllocDefault) !=
                cudaSuccess) {
            cudaGetLastError();
            for (auto x : s->streams) cudaStreamDestroy(x);
            for (auto x : s->h_offsets) cudaFreeHost(x);
            delete s;
            return nullptr;
        }
        s->streams.push_back(st);
        s->h_offsets.push_back(h);
        s->slot_busy.push_back(false);
    }
    s->engine = std::thread([s] { s->run(); });
    return s;
}

int64_t pico_server_submit(pico_server *s, const int32_t *row_ptr, const int32_t *col_idx,
                           int64_t n, int64_t m, int32_t *out_core, int64_t arrival_ns)
{
    if (!s || n < 0 || m < 0 || n >= INT32_MAX || m >= INT32_MAX || !row_ptr ||
        (n > 0 && !out_core) || (m > 0 && !col_idx))
        return PICO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return PICO_ERR_INVALID_ARG;
    if (s->batch_bytes(1, n, m) > s->cfg.hbm_budget_bytes) return PICO_ERR_OOM;
    Request r{s->next_ticket++, row_ptr, col_idx, n, m, out_core, arrival_ns};
    // keep `pending` ordered by arrival time (submissions are usually in order)
    auto it = s->pending.end();
    while (it != s->pending.begin() && (it - 1)->arrival_ns > arrival_ns) --it;
    s->pending.insert(it, r);
    ++s->submitted;
    s->cv.notify_one();
    return r.ticket;
}

int pico_server_poll_device(pico_server *s, int64_t *tickets, int64_t *done_ns,
                            int64_t *device_ns, int cap)
{
    if (!s || cap < 0 || (cap > 0 && (!tickets || !done_ns))) return PICO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    const int k = (int)std::min<size_t>((size_t)cap, s->done_tickets.size());
    for (int i = 0; i < k; ++i) {
        tickets[i] = s->done_tickets[i];
        done_ns[i] = s->done_times[i];
        if (device_ns) device_ns[i] = s->done_device[i];
    }
    s->done_tickets.erase(s->done_tickets.begin(), s->done_tickets.begin() + k);
    s->done_times.erase(s->done_times.begin(), s->done_times.begin() + k);
    s->done_device.erase(s->done_device.begin(), s->done_device.begin() + k);
    return k;
}

int pico_server_poll(pico_server *s, int64_t *tickets, int64_t *done_ns, int cap)
{
    return pico_server_poll_device(s, tickets, done_ns, nullptr, cap);
}

int pico_server_drain(pico_server *s)
{
    if (!s) return PICO_ERR_INVALID_ARG;
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->completed == s->submitted) return s->error;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int pico_server_destroy(pico_server *s)
{
    if (!s) return PICO_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_one();
    }
    s->engine.join();
    const int err = s->error;
    for (auto x : s->streams) cudaStreamDestroy(x);
    for (auto x : s->h_offsets) cudaFreeHost(x);
    delete s;
    return err;
}

}  // extern "C"
