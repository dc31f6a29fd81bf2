// Partitioned HistoCore: the h-index iteration of Alg. 6 over a graph whose
// vertices are split into contiguous ranges, each range's rows (estimates,
// histograms, V_cnt) held by its own partition. Index2core suits this split
// (Sec. VI, distributed k-core; multi-GPU processing is named as future work
// in Sec. VII): a round needs from other partitions only the {old, new}
// estimates of the vertices that changed in it.
//
// One round, for every partition at once (the synchronous model of Alg. 6):
//   sum      SumHisto over the partition's own V_cnt: estimate K -> h, the
//            new cnt into slot h, and a record (v, K, h) of every change.
//   exchange every partition receives every partition's records of the
//            round (an all-gather; here the caller moves them) and the
//            smallest new estimate of the round.
//   apply    the records are scattered into a vertex-indexed {old, new}
//            array; every own row u with estimate K above the round's
//            smallest new estimate walks its arcs and, for each changed
//            neighbour w (x -> y) with K > y, moves w from slot min(x, K) to
//            slot y (types N1/N3 of Sec. IV-B, pulled: arc (w, u) pushed is
//            arc (u, w) pulled); rows whose slot K fell below K form the next
//            V_cnt (the deferred decision of the single-graph kernel: slot K
//            only falls during UpdateHisto, so it ends below K exactly when
//            one decrement took it from K to K - 1); the array is cleared.
// No kernel waits on another: each phase is an ordinary launch that ends,
// and the exchange sits between launches, so partitions can live on other
// devices (or processes) with the same calls. A partition reads only its own
// rows of the graph. The single-device driver (pico_coreness_partitioned),
// where every partition can read the whole graph, also pushes: in a round
// whose changed vertices hold few arcs, those vertices walk their own arcs
// and each partition applies the edits that fall on its rows (the same
// edits as pulled, reached from the other end of each arc).
//
// Rows are addressed by local index i (vertex lo + i); their adjacency is
// col_idx[row_ptr[lo + i] ..] with global neighbour ids; the histogram of a
// partition is laid out like its slice of col_idx.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pico.h"
#include "pico_device.cuh"
#include "pico_launch.h"

namespace pico {
namespace part {

// device counters of a partition
struct Counters {
    unsigned vcnt[2];      // V_cnt sizes by parity
    unsigned changed;      // records of the round
    unsigned nib;          // chunk entries of the large rows
    int ymax;              // INT_MAX - smallest new estimate of the round (atomicMax)
    int err;
    unsigned long long vol;   // arcs of the round's changed vertices
};

struct Arrays {
    const long long *rp;   // global row_ptr (n + 1)
    const int *ci;         // global col_idx
    long long lo, np;      // rows lo .. lo + np - 1
    long long *lrp;        // local row starts: lrp[i] = rp[lo + i] - rp[lo] (np + 1)
    const int *lci;        // ci + rp[lo]
    int *est;              // np estimates
    int *hist;             // local histogram (lrp[np] slots)
    int *vc[2];            // V_cnt by parity (local indices)
    int *rec;              // records of the round: 3 ints each (v, old, new), np slots
    int2 *mvg;             // n entries, {0, 0} but for the changed vertices of a round
    unsigned char *cand;   // row marks of the apply phase (np, padded to 4)
    int2 *ib;              // chunks of the rows with degree > small_deg
    unsigned ib_cap;
    Counters *cnt;
    Tuning tn;
};

constexpr int kBlock = 512;

__device__ __forceinline__ int gdeg(const long long *rp, int v) { return (int)(rp[v + 1] - rp[v]); }

__global__ void __launch_bounds__(kBlock) init_kernel(Arrays a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    __shared__ unsigned s_tmp[128];
    const long long base0 = a.rp[a.lo];
    for (long long b = (long long)blockIdx.x * blockDim.x; b <= a.np; b += stride) {
        const long long i = b + threadIdx.x;
        long long d = 0;
        if (i <= a.np) a.lrp[i] = a.rp[a.lo + i] - base0;
        if (i < a.np) {
            d = a.rp[a.lo + i + 1] - a.rp[a.lo + i];
            a.est[i] = (int)d;
            a.cand[i] = 0;
        }
        const unsigned nch =
            d > a.tn.small_deg ? (unsigned)((d + a.tn.chunk - 1) / a.tn.chunk) : 0u;
        const unsigned pos = block_alloc(nch, &a.cnt->nib, s_tmp);
        const bool fits = (unsigned long long)pos + nch <= a.ib_cap;
        if (nch && !fits) a.cnt->err = 1;
        warp_fill_chunks(fits ? nch : 0u, pos, (int)i, a.ib);
    }
}

// InitHisto: row i counts its neighbours by min(degree of the neighbour, own degree)
struct InitArc {
    static constexpr int kArcs = 4;
    const long long *rp;
    const int *est;
    int *hist;
    __device__ __forceinline__ bool item(int i, int &dv, int &)
    {
        dv = est[i];
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&w)[kArcs], const long long (&rs)[kArcs],
                                         const int (&dv)[kArcs], const int (&)[kArcs])
    {
        int dw[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) dw[j] = valid[j] ? gdeg(rp, w[j]) : 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            if (valid[j]) red_add(hist + rs[j] + (dw[j] < dv[j] ? dw[j] : dv[j]) - 1, 1);
    }
};

__global__ void __launch_bounds__(kBlock) inithisto_kernel(Arrays a)
{
    InitArc f{a.rp, a.est, a.hist};
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    expand(a.lrp, a.lci, (const int *)nullptr, (unsigned)a.np, a.ib, a.cnt->nib, gwarp, nwarps, f,
           a.tn);
}

// the initial V_cnt: rows with degree >= 1 whose cnt (slot deg) is below deg
__global__ void __launch_bounds__(kBlock) vcnt0_kernel(Arrays a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < a.np; b += stride) {
        const long long i = b + threadIdx.x;
        bool in = false;
        if (i < a.np) {
            const int d = a.est[i];
            in = d >= 1 && a.hist[a.lrp[i] + d - 1] < d;
        }
        const unsigned pos = warp_push(&a.cnt->vcnt[0], in);
        if (in) a.vc[0][pos] = (int)i;   // pos < np: each row once
    }
}

// SumHisto of row i (estimate K): the slots from K downwards until the running
// sum reaches the slot index; records the change. One thread walks K <= 32
// slots, one warp larger estimates (32 slots a step, suffix sums).
__device__ __forceinline__ void apply_sum(const Arrays &a, int i, int K, int h, int sum)
{
    a.est[i] = h;
    a.hist[a.lrp[i] + h - 1] = sum;
    const unsigned pos = atomicAdd(&a.cnt->changed, 1u);   // < np: each V_cnt row once
    a.rec[3 * pos] = (int)(a.lo + i);
    a.rec[3 * pos + 1] = K;
    a.rec[3 * pos + 2] = h;
    atomicMax(&a.cnt->ymax, INT_MAX - h);
    atomicAdd(&a.cnt->vol, (unsigned long long)(a.lrp[i + 1] - a.lrp[i]));
}

__global__ void __launch_bounds__(kBlock) sum_kernel(Arrays a, int par, unsigned nv)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned base = gwarp * 32; base < nv; base += nwarps * 32) {
        const unsigned idx = base + lane;
        int i = -1, K = 0;
        if (idx < nv) {
            i = a.vc[par][idx];
            K = a.est[i];
        }
        // small estimates: this lane alone
        if (i >= 0 && K <= 32) {
            const long long rs = a.lrp[i];
            int sum = 0, k = K;
            for (; k >= 1; --k) {
                sum += a.hist[rs + k - 1];
                if (sum >= k) break;
            }
            if (k >= 1 && k < K) apply_sum(a, i, K, k, sum);
            else a.cnt->err = 2;   // every V_cnt vertex changes (Thm. 2)
        }
        // larger estimates: the whole warp, one row after another
        unsigned big = __ballot_sync(kFull, i >= 0 && K > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int bi = __shfl_sync(kFull, i, src), bK = __shfl_sync(kFull, K, src);
            const long long rs = a.lrp[bi];
            int carry = 0, found_k = 0, found_sum = 0;
            for (int top = bK; top >= 1 && !found_k; top -= 32) {
                const int slot = top - (int)lane;   // lane 0 holds the highest slot
                const int x = slot >= 1 ? a.hist[rs + slot - 1] : 0;
                int inc = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, inc, o);
                    if ((int)lane >= o) inc += y;
                }
                const int run = carry + inc;   // sum of the slots from bK down to `slot`
                const unsigned hit = __ballot_sync(kFull, slot >= 1 && run >= slot);
                if (hit) {
                    const int L = __ffs(hit) - 1;   // the highest qualifying slot
                    found_k = __shfl_sync(kFull, slot, L);
                    found_sum = __shfl_sync(kFull, run, L);
                }
                carry += __shfl_sync(kFull, inc, 31);
            }
            if (lane == 0) {
                if (found_k >= 1 && found_k < bK) apply_sum(a, bi, bK, found_k, found_sum);
                else a.cnt->err = 2;
            }
        }
    }
}

// records of the round (all partitions) -> {old, new} by vertex; clear == true
// writes {0, 0} back
__global__ void __launch_bounds__(kBlock) scatter_kernel(int2 *mvg, long long n, const int *rec,
                                                         long long count, bool clear, int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += stride) {
        const int v = rec[3 * r];
        if (v < 0 || v >= n) {
            *err = 3;
            continue;
        }
        mvg[v] = clear ? make_int2(0, 0) : make_int2(rec[3 * r + 1], rec[3 * r + 2]);
    }
}

// UpdateHisto pulled into the own rows whose estimate exceeds the round's
// smallest new estimate
struct PullArc {
    static constexpr int kArcs = 4;
    const int *est;
    const int2 *mvg;
    int *hist;
    unsigned char *cand;
    int ymin;
    __device__ __forceinline__ bool item(int i, int &K, int &)
    {
        K = est[i];
        return K > ymin;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&ii)[kArcs],
                                         const int (&w)[kArcs], const long long (&rs)[kArcs],
                                         const int (&K)[kArcs], const int (&)[kArcs])
    {
        int2 r[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) r[j] = valid[j] ? __ldg(mvg + w[j]) : make_int2(0, 0);
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            const int x = r[j].x, y = r[j].y;
            if (!valid[j] || x == 0 || K[j] <= y) continue;
            red_add(hist + rs[j] + y - 1, 1);
            red_add(hist + rs[j] + (x < K[j] ? x : K[j]) - 1, -1);
            if (x >= K[j]) cand[ii[j]] = 1;
        }
    }
};

__global__ void __launch_bounds__(kBlock) pull_kernel(Arrays a, int ymin)
{
    PullArc f{a.est, a.mvg, a.hist, a.cand, ymin};
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    expand(a.lrp, a.lci, (const int *)nullptr, (unsigned)a.np, a.ib, a.cnt->nib, gwarp, nwarps, f,
           a.tn);
}

// marked rows whose cnt fell below their estimate form the next V_cnt
__global__ void __launch_bounds__(kBlock) collect_kernel(Arrays a, int np_par)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < a.np; b += stride) {
        const long long i = b + threadIdx.x;
        bool in = false;
        if (i < a.np && a.cand[i]) {
            a.cand[i] = 0;
            const int K = a.est[i];
            in = a.hist[a.lrp[i] + K - 1] < K;
        }
        const unsigned pos = warp_push(&a.cnt->vcnt[np_par], in);
        if (in) a.vc[np_par][pos] = (int)i;
    }
}

// Push form of UpdateHisto for the single-device driver, where every
// partition can read the whole CSR: the round's changed vertices (listed
// once for all partitions: small ones, chunks of large ones) walk their own
// arcs, and each partition applies the edits that fall on its rows. It
// applies the same multiset of edits as the pull form (arc (w, u) pushed is
// arc (u, w) pulled) and marks the same rows; it scans the changed vertices'
// arcs once per partition instead of every arc of the partition's rows.
struct PushLists {
    int *small;        // changed vertices of degree <= small_deg
    int2 *big;         // (vertex, chunk) entries of the larger ones
    unsigned *count;   // [0] small, [1] big
    unsigned small_cap, big_cap;
    int *err;
};

__global__ void __launch_bounds__(kBlock) push_lists_kernel(const long long *rp, long long n,
                                                            const int *rec, long long count,
                                                            PushLists l, Tuning tn)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < count; b += stride) {
        const long long r = b + threadIdx.x;
        int w = -1;
        long long d = 0;
        if (r < count) {
            w = rec[3 * r];
            if (w >= 0 && w < n) d = rp[w + 1] - rp[w];
            else w = -1;
        }
        const bool small = w >= 0 && d > 0 && d <= tn.small_deg;
        const unsigned pos = warp_push(&l.count[0], small);
        if (small) {
            if (pos < l.small_cap) l.small[pos] = w;
            else *l.err = 1;
        }
        const unsigned lane = threadIdx.x & 31;
        unsigned m = __ballot_sync(kFull, w >= 0 && d > tn.small_deg);
        while (m) {   // the warp writes each large vertex's chunk entries
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const int vv = __shfl_sync(kFull, w, src);
            const long long dd = __shfl_sync(kFull, d, src);
            const unsigned nch = (unsigned)((dd + tn.chunk - 1) / tn.chunk);
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&l.count[1], nch);
            base = __shfl_sync(kFull, base, 0);
            if ((unsigned long long)base + nch > l.big_cap) {
                if (lane == 0) *l.err = 1;
                continue;
            }
            for (unsigned c = lane; c < nch; c += 32) l.big[base + c] = make_int2(vv, (int)c);
        }
    }
}

struct PushArc {
    static constexpr int kArcs = 4;
    const int2 *mvg;
    const int *est;
    const long long *lrp;
    int *hist;
    unsigned char *cand;
    long long lo, np;
    __device__ __forceinline__ bool item(int w, int &x, int &y)
    {
        const int2 r = mvg[w];
        x = r.x;
        y = r.y;
        return x != 0;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const long long (&)[kArcs],
                                         const int (&x)[kArcs], const int (&y)[kArcs])
    {
        long long i[kArcs];
        int K[kArcs];
        long long rs[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            i[j] = (long long)u[j] - lo;
            const bool mine = valid[j] && i[j] >= 0 && i[j] < np;
            K[j] = mine ? est[i[j]] : 0;
            rs[j] = mine ? lrp[i[j]] : 0;
        }
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            if (K[j] <= y[j]) continue;   // not this partition's row, or no edit (K <= y)
            red_add(hist + rs[j] + y[j] - 1, 1);
            red_add(hist + rs[j] + (x[j] < K[j] ? x[j] : K[j]) - 1, -1);
            if (x[j] >= K[j]) cand[i[j]] = 1;
        }
    }
};

__global__ void __launch_bounds__(kBlock) push_kernel(Arrays a, PushLists l)
{
    PushArc f{a.mvg, a.est, a.lrp, a.hist, a.cand, a.lo, a.np};
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned ns = l.count[0] < l.small_cap ? l.count[0] : l.small_cap;
    const unsigned nb = l.count[1] < l.big_cap ? l.count[1] : l.big_cap;
    expand(a.rp, a.ci, l.small, ns, l.big, nb, gwarp, nwarps, f, a.tn);
}

}  // namespace part
}  // namespace pico

struct pico_part {
    int device;
    long long n, lo, hi, m_local;
    pico::part::Arrays a;
    void *mem;                 // from the stream-ordered pool, released on `stream`
    cudaStream_t stream;
    int par;                   // parity of the current V_cnt
    unsigned long long vcnt;   // its size
    long long changed;         // records of the last sum
    int ymin;                  // smallest new estimate of the last sum
    unsigned long long vol;    // arcs of the vertices of those records
    int grid;
};

namespace {

// Synchronises the stream and copies the partition's counters to *c; the
// status of what the partition's kernels found.
int sync_read(pico_part *p, cudaStream_t s, pico::part::Counters *c)
{
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(c, p->a.cnt, sizeof *c, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (c->err == 1) return PICO_ERR_NOT_CONVERGED;
    if (c->err) return PICO_ERR_BAD_GRAPH;
    return PICO_OK;
}

}  // namespace

extern "C" {

pico_part *pico_part_create(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t lo,
                            int64_t hi, pico_stream_t stream)
{
    if (!row_ptr || n < 1 || lo < 0 || hi > n || lo >= hi || n >= INT32_MAX) return nullptr;
    pico::LaunchCfg cfg;
    pico::LastResult *last = nullptr;
    if (pico::current_device(&cfg, &last) != PICO_OK) return nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    long long b[2] = {0, 0};
    if (cudaMemcpy(&b[0], row_ptr + lo, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&b[1], row_ptr + hi, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const long long np = hi - lo, ml = b[1] - b[0];
    if (ml < 0 || (ml > 0 && !col_idx)) return nullptr;
    pico_part *p = new pico_part();
    p->device = cfg.device;
    p->n = n;
    p->lo = lo;
    p->hi = hi;
    p->m_local = ml;
    const size_t ib_cap = pico::chunk_capacity(ml);
    pico::Carver c0(nullptr);
    c0.take<pico::part::Counters>(1);
    c0.take<unsigned char>((size_t)((np + 3) & ~3ll));   // cand
    const size_t zero_bytes = c0.size();
    c0.take<long long>(np + 1);
    c0.take<int>(np);
    c0.take<int>(ml > 0 ? ml : 1);
    c0.take<int>(np);
    c0.take<int>(np);
    c0.take<int>(3 * np);
    c0.take<int2>(n);
    c0.take<int2>(ib_cap);
    p->stream = s;
    if (cudaMallocAsync(&p->mem, c0.size(), s) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return nullptr;
    }
    pico::Carver c(p->mem);
    pico::part::Arrays &a = p->a;
    a.cnt = c.take<pico::part::Counters>(1);
    a.cand = c.take<unsigned char>((size_t)((np + 3) & ~3ll));
    a.lrp = c.take<long long>(np + 1);
    a.est = c.take<int>(np);
    a.hist = c.take<int>(ml > 0 ? ml : 1);
    a.vc[0] = c.take<int>(np);
    a.vc[1] = c.take<int>(np);
    a.rec = c.take<int>(3 * np);
    a.mvg = c.take<int2>(n);
    a.ib = c.take<int2>(ib_cap);
    a.ib_cap = (unsigned)ib_cap;
    a.rp = reinterpret_cast<const long long *>(row_ptr);
    a.ci = col_idx;
    a.lo = lo;
    a.np = np;
    a.lci = col_idx ? col_idx + b[0] : nullptr;
    a.tn = cfg.tn;
    p->grid = cfg.sms * 4;
    p->par = 0;
    bool ok = cudaMemsetAsync(p->mem, 0, zero_bytes, s) == cudaSuccess &&
              cudaMemsetAsync(a.hist, 0, (size_t)(ml > 0 ? ml : 1) * sizeof(int), s) == cudaSuccess &&
              cudaMemsetAsync(a.mvg, 0, (size_t)n * sizeof(int2), s) == cudaSuccess;
    if (ok) {
        pico::part::init_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(a);
        if (ml > 0) pico::part::inithisto_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(a);
        pico::part::vcnt0_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(a);
        ok = cudaGetLastError() == cudaSuccess;
    }
    pico::part::Counters cn{};
    ok = ok && sync_read(p, s, &cn) == PICO_OK;
    if (!ok) {
        cudaGetLastError();
        cudaFreeAsync(p->mem, s);
        delete p;
        return nullptr;
    }
    p->vcnt = cn.vcnt[0];
    return p;
}

int pico_part_sum(pico_part *p, int64_t *n_changed, int32_t *ymin, pico_stream_t stream)
{
    if (!p || !n_changed || !ymin) return PICO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int par = p->par;
    // counters of this round: records and their smallest estimate
    pico::part::Counters *cd = p->a.cnt;
    if (cudaMemsetAsync(&cd->changed, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(&cd->ymax, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(&cd->vol, 0, sizeof(unsigned long long), s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (p->vcnt > 0) {
        pico::part::sum_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(p->a, par, (unsigned)p->vcnt);
        if (cudaGetLastError() != cudaSuccess) return PICO_ERR_CUDA;
    }
    pico::part::Counters c{};
    const int rc = sync_read(p, s, &c);
    if (rc != PICO_OK) return rc;
    if (c.changed != p->vcnt) return PICO_ERR_BAD_GRAPH;   // Thm. 2: every V_cnt vertex changes
    p->changed = c.changed;
    p->ymin = c.changed ? INT_MAX - c.ymax : INT_MAX;
    p->vol = c.vol;
    *n_changed = p->changed;
    *ymin = p->ymin;
    return PICO_OK;
}

const int32_t *pico_part_records(pico_part *p) { return p ? p->a.rec : nullptr; }

int pico_part_copy_records(pico_part *p, int32_t *dst, pico_stream_t stream)
{
    if (!p || (p->changed > 0 && !dst)) return PICO_ERR_INVALID_ARG;
    if (p->changed > 0 &&
        cudaMemcpyAsync(dst, p->a.rec, (size_t)3 * p->changed * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

}  // extern "C"

namespace {
// UpdateHisto of one partition for the round's records: pulled into its
// rows, or (push != nullptr, single device only) pushed from the listed
// changed vertices.
int apply_impl(pico_part *p, const int32_t *records, int64_t count, int32_t ymin,
               int64_t *next_vcnt, pico_stream_t stream, const pico::part::PushLists *push)
{
    if (!p || count < 0 || (count > 0 && !records) || !next_vcnt) return PICO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int np_par = 1 - p->par;
    pico::part::Counters *cd = p->a.cnt;
    if (cudaMemsetAsync(&cd->vcnt[np_par], 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (count > 0) {
        const int g = (int)std::min<long long>(p->grid, (count + pico::part::kBlock - 1) / pico::part::kBlock);
        pico::part::scatter_kernel<<<g, pico::part::kBlock, 0, s>>>(p->a.mvg, p->n, records, count,
                                                                    false, &cd->err);
        if (p->m_local > 0 && push)
            pico::part::push_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(p->a, *push);
        else if (p->m_local > 0)
            pico::part::pull_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(p->a, ymin);
        pico::part::collect_kernel<<<p->grid, pico::part::kBlock, 0, s>>>(p->a, np_par);
        pico::part::scatter_kernel<<<g, pico::part::kBlock, 0, s>>>(p->a.mvg, p->n, records, count,
                                                                    true, &cd->err);
        if (cudaGetLastError() != cudaSuccess) return PICO_ERR_CUDA;
    }
    pico::part::Counters c{};
    const int rc = sync_read(p, s, &c);
    if (rc != PICO_OK) return rc;
    p->par = np_par;
    p->vcnt = c.vcnt[np_par];
    *next_vcnt = (int64_t)p->vcnt;
    return PICO_OK;
}

}  // namespace

extern "C" {

int pico_part_apply(pico_part *p, const int32_t *records, int64_t count, int32_t ymin,
                    int64_t *next_vcnt, pico_stream_t stream)
{
    return apply_impl(p, records, count, ymin, next_vcnt, stream, nullptr);
}

int pico_part_coreness(pico_part *p, int32_t *out_core, pico_stream_t stream)
{
    if (!p || !out_core) return PICO_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(out_core, p->a.est, (size_t)(p->hi - p->lo) * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

void pico_part_destroy(pico_part *p)
{
    if (!p) return;
    cudaFreeAsync(p->mem, p->stream);
    cudaGetLastError();
    delete p;
}

int pico_coreness_partitioned(const int64_t *row_ptr, const int32_t *col_idx, int64_t n,
                              int64_t m, int32_t *out_core, int32_t parts, int64_t *rounds,
                              pico_stream_t stream)
{
    if (n < 0 || m < 0 || parts < 1 || parts > 1024) return PICO_ERR_INVALID_ARG;
    if (n == 0) {
        if (rounds) *rounds = 0;
        return PICO_OK;
    }
    if (!row_ptr || !out_core || (m > 0 && !col_idx) || n >= INT32_MAX) return PICO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int P = (int)std::min<long long>(parts, n);
    std::vector<pico_part *> ps(P, nullptr);
    int rc = PICO_OK;
    for (int q = 0; q < P && rc == PICO_OK; ++q) {
        ps[q] = pico_part_create(row_ptr, col_idx, n, n * q / P, n * (q + 1) / P, stream);
        if (!ps[q]) rc = PICO_ERR_OOM;
    }
    int *all = nullptr;   // every partition's records of a round, in partition order
    if (rc == PICO_OK && cudaMallocAsync(&all, (size_t)3 * n * sizeof(int) + 16, s) != cudaSuccess) {
        cudaGetLastError();
        rc = PICO_ERR_OOM;
    }
    // lists of a pushed round's changed vertices, shared by the partitions
    pico::part::PushLists pl{};
    void *plmem = nullptr;
    pico::LaunchCfg cfg;
    pico::LastResult *last = nullptr;
    if (rc == PICO_OK) rc = pico::current_device(&cfg, &last);
    if (rc == PICO_OK) {
        pico::Carver c(nullptr);
        c.take<unsigned>(4);
        c.take<int>(n);
        c.take<int2>(pico::chunk_capacity(m));
        if (cudaMallocAsync(&plmem, c.size(), s) != cudaSuccess) {
            cudaGetLastError();
            rc = PICO_ERR_OOM;
        } else {
            pico::Carver d(plmem);
            pl.count = d.take<unsigned>(4);
            pl.err = reinterpret_cast<int *>(pl.count + 2);
            pl.small = d.take<int>(n);
            pl.small_cap = (unsigned)n;
            pl.big = d.take<int2>(pico::chunk_capacity(m));
            pl.big_cap = (unsigned)pico::chunk_capacity(m);
        }
    }
    long long r = 0;
    while (rc == PICO_OK) {
        long long total = 0;
        unsigned long long vol = 0;
        int ymin = INT_MAX;
        for (int q = 0; q < P && rc == PICO_OK; ++q) {   // SumHisto in every partition
            int64_t c = 0;
            int32_t y = 0;
            rc = pico_part_sum(ps[q], &c, &y, stream);
            if (rc != PICO_OK) break;
            // the exchange: this partition's records join the round's list
            if (c > 0 && cudaMemcpyAsync(all + 3 * total, pico_part_records(ps[q]),
                                         (size_t)3 * c * sizeof(int), cudaMemcpyDeviceToDevice,
                                         s) != cudaSuccess) {
                cudaGetLastError();
                rc = PICO_ERR_CUDA;
            }
            total += c;
            vol += ps[q]->vol;
            ymin = std::min(ymin, (int)y);
        }
        if (rc != PICO_OK || total == 0) break;
        ++r;
        if (r > m + 2) {
            rc = PICO_ERR_NOT_CONVERGED;
            break;
        }
        // Push when every partition scanning the changed vertices' arcs costs
        // less than half of pulling every arc (the measured crossover of the
        // single-graph kernel is near half the arcs).
        const bool push = (unsigned long long)P * vol * 2 < (unsigned long long)m;
        if (push) {
            if (cudaMemsetAsync(pl.count, 0, 4 * sizeof(unsigned), s) != cudaSuccess) {
                cudaGetLastError();
                rc = PICO_ERR_CUDA;
                break;
            }
            const int g = (int)std::min<long long>(cfg.sms * 4, (total + pico::part::kBlock - 1) /
                                                                    pico::part::kBlock);
            pico::part::push_lists_kernel<<<g, pico::part::kBlock, 0, s>>>(
                reinterpret_cast<const long long *>(row_ptr), n, all, total, pl, cfg.tn);
            if (cudaGetLastError() != cudaSuccess) {
                rc = PICO_ERR_CUDA;
                break;
            }
        }
        for (int q = 0; q < P && rc == PICO_OK; ++q) {   // UpdateHisto in every partition
            int64_t next = 0;
            rc = apply_impl(ps[q], all, total, ymin, &next, stream, push ? &pl : nullptr);
        }
        if (rc == PICO_OK && push) {
            int perr = 0;
            if (cudaMemcpy(&perr, pl.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                rc = PICO_ERR_CUDA;
            } else if (perr) {
                rc = PICO_ERR_NOT_CONVERGED;
            }
        }
    }
    for (int q = 0; q < P && rc == PICO_OK; ++q)
        rc = pico_part_coreness(ps[q], out_core + n * q / P, stream);
    if (rc == PICO_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        rc = PICO_ERR_CUDA;
    }
    if (all) cudaFreeAsync(all, s);
    if (plmem) cudaFreeAsync(plmem, s);
    cudaGetLastError();
    for (pico_part *p : ps) pico_part_destroy(p);
    if (rounds) *rounds = r;
    return rc;
}

}  // extern "C"
