// Core maintenance: the coreness of a graph kept up to date under batches of
// edge insertions and deletions, without recomputing it from the degrees.
// The paper lists core maintenance among the uses of Index2core (Sec. I,
// related work in Sec. VI); this is the path built on this library's kernels.
//
// A batch is applied in three steps, all on the device:
//   1. The CSR is rebuilt: new degrees, an exclusive scan for the offsets,
//      the surviving arcs copied row by row (a deleted arc is found in a hash
//      set of the batch's deleted arcs), the inserted arcs appended.
//   2. Deletions: coreness can only fall. The old coreness (capped at the new
//      degree, at least 1) is an upper bound, so HistoCore's rounds (Alg. 6)
//      started from it instead of the degrees end at the new coreness: they
//      stop with cnt >= estimate everywhere, which bounds the estimates by the
//      coreness, and never go below it. Only the vertices whose cnt fell
//      below their estimate, and those their changes reach, do any work.
//      With insertions in the batch the start is not an upper bound, but the
//      result is still a lower bound of the new coreness.
//   3. Insertions: coreness can only rise; the value after step 2 is a lower
//      bound. A pass tries to raise vertices by one: the candidates are the
//      vertices w with at least core(w) + 1 neighbours of core >= core(w)
//      (that count, cd, is kept between batches); the pass works on its
//      region, the candidates connected to a seed through candidates of equal
//      core (seeds: the inserted edges' endpoints, then the vertices the
//      previous pass raised and their neighbours; see run() for why no other
//      vertex can rise). Each region vertex counts its support (neighbours of
//      higher core, or of equal core that are candidates) and those whose
//      support falls below core(w) + 1 are peeled, which lowers their
//      equal-core candidate neighbours' support, wave by wave as in PeelOne's
//      dynamic frontier. The survivors of level K together with the vertices
//      of core > K have minimum degree K + 1, so they lie in the (K + 1)-core
//      and rise by one. Passes repeat until one raises nothing. Then no vertex
//      is below its coreness: for the smallest k with a vertex below k in the
//      true k-core X, those vertices all have core k - 1, are candidates, and
//      keep a support of at least k from X through every peel, so they rise
//      once their component is in a region, which it is.
#include <algorithm>
#include <cstring>

#include "ablation.cuh"
#include "pico.h"
#include "pico_launch.h"

namespace pico {
namespace dyn {

// ---------------------------------------------------------------------------
// arc hash sets (open addressing, linear probing; 0 marks an empty slot)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long arc_key(int u, int v)
{
    return ((unsigned long long)(unsigned)u << 32 | (unsigned)v) + 1ull;
}

// slot of a key: the 64-bit finaliser of MurmurHash3 (Appleby), then the mask
__device__ __forceinline__ unsigned hash_slot(unsigned long long k, unsigned mask)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (unsigned)k & mask;
}

// false if the key was already present (or the table is full)
__device__ __forceinline__ bool set_insert(unsigned long long *tab, unsigned mask,
                                           unsigned long long k)
{
    unsigned s = hash_slot(k, mask);
    for (unsigned probe = 0; probe <= mask; ++probe, s = (s + 1) & mask) {
        const unsigned long long prev = atomicCAS(tab + s, 0ull, k);
        if (prev == 0ull) return true;
        if (prev == k) return false;
    }
    return false;
}

__device__ __forceinline__ bool set_has(const unsigned long long *tab, unsigned mask,
                                        unsigned long long k)
{
    unsigned s = hash_slot(k, mask);
    for (unsigned probe = 0; probe <= mask; ++probe, s = (s + 1) & mask) {
        const unsigned long long x = __ldcg(tab + s);
        if (x == k) return true;
        if (x == 0ull) return false;
    }
    return false;
}

// batch errors (first one wins)
enum : int { kBadId = 1, kDupInBatch = 2, kMissingArc = 3, kExistingArc = 4, kNegDegree = 5 };

__device__ __forceinline__ void fail(int *err, int code) { atomicCAS(err, 0, code); }

// ---------------------------------------------------------------------------
// step 1: CSR rebuild
// ---------------------------------------------------------------------------
// Per-vertex insert/delete counts, touched flags and the two arc sets.
__global__ void count_kernel(const int *ins, long long n_ins, const int *del, long long n_del,
                             long long n, int *ins_cnt, int *del_cnt, unsigned char *touched,
                             unsigned long long *instab, unsigned insmask,
                             unsigned long long *deltab, unsigned delmask, int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ins + n_del;
         i += stride) {
        const bool is_ins = i < n_ins;
        const int *e = is_ins ? ins + 2 * i : del + 2 * (i - n_ins);
        const int u = e[0], v = e[1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) {
            fail(err, kBadId);
            continue;
        }
        unsigned long long *tab = is_ins ? instab : deltab;
        const unsigned mask = is_ins ? insmask : delmask;
        if (!set_insert(tab, mask, arc_key(u, v)) || !set_insert(tab, mask, arc_key(v, u))) {
            fail(err, kDupInBatch);
            continue;
        }
        int *cnt = is_ins ? ins_cnt : del_cnt;
        atomicAdd(cnt + u, 1);
        atomicAdd(cnt + v, 1);
        const unsigned char bit = is_ins ? 1 : 2;
        atomicOr(reinterpret_cast<unsigned *>(touched + (u & ~3)), (unsigned)bit << (8 * (u & 3)));
        atomicOr(reinterpret_cast<unsigned *>(touched + (v & ~3)), (unsigned)bit << (8 * (v & 3)));
    }
}

// new degree of every vertex (into new_rp[v + 1], scanned in place afterwards)
__global__ void degree_kernel(const long long *rp, long long n, const int *ins_cnt,
                              const int *del_cnt, long long *new_rp, int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const long long d = rp[v + 1] - rp[v] + ins_cnt[v] - del_cnt[v];
        if (d < 0) fail(err, kNegDegree);
        new_rp[v + 1] = d < 0 ? 0 : d;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) new_rp[0] = 0;
}

// In-place inclusive scan of a[1..n] by one persistent cooperative grid: each
// CTA sums its contiguous range, CTA sums are scanned after a grid barrier,
// then each CTA scans its range on top of its offset.
__global__ void __launch_bounds__(kThreads) scan_kernel(long long *a, long long n, Ctrl *ctl,
                                                         long long *cta_sum,
                                                         unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ long long s_w[kThreads / 32];
    __shared__ long long s_carry;
    GridDom dom{ctl, s_snap, limit_ns};
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = 1 + (long long)blockIdx.x * per;
    const long long hi = lo + per < n + 1 ? lo + per : n + 1;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long mine = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) mine += a[i];
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFull, mine, o);
    if (lane == 0) s_w[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (unsigned w = 0; w < nw; ++w) t += s_w[w];
        cta_sum[blockIdx.x] = t;
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) {
        long long off = 0;
        for (unsigned b = 0; b < blockIdx.x; ++b) off += __ldcg(cta_sum + b);
        s_carry = off;
    }
    __syncthreads();
    for (long long base = lo; base < hi; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        long long x = i < hi ? a[i] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = lane < nw ? s_w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(kFull, w, o);
                if ((int)lane >= o) w += y;
            }
            if (lane < nw) s_w[lane] = w;
        }
        __syncthreads();
        const long long before = (warp ? s_w[warp - 1] : 0) + s_carry;
        if (i < hi) a[i] = x + before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_w[nw - 1];
        __syncthreads();
    }
}

// set_has for a table that no thread writes during the kernel (built by an
// earlier launch): the probes may go through the read-only cache.
__device__ __forceinline__ bool set_has_ro(const unsigned long long *tab, unsigned mask,
                                           unsigned long long k)
{
    unsigned s = hash_slot(k, mask);
    for (unsigned probe = 0; probe <= mask; ++probe, s = (s + 1) & mask) {
        const unsigned long long x = __ldg(tab + s);
        if (x == k) return true;
        if (x == 0ull) return false;
    }
    return false;
}

// Copies one old row's surviving arcs: every lane of the warp calls with the
// same u; arcs [e0, e1) of the old row. 1024 arcs at a time: the lanes first
// decide which arcs survive (one bit per step), then reserve the survivors'
// positions with one atomic on the row's cursor, then write them in order.
__device__ __forceinline__ void copy_piece(int u, long long e0, long long e1, const int *ci,
                                           const long long *new_rp, int *new_ci, int *cursor,
                                           unsigned char tflag, const unsigned long long *instab,
                                           unsigned insmask, const unsigned long long *deltab,
                                           unsigned delmask, int *err)
{
    const unsigned lane = threadIdx.x & 31;
    const long long r0 = new_rp[u], r1 = new_rp[u + 1];
    for (long long s0 = e0; s0 < e1; s0 += 1024) {
        const long long s1 = s0 + 1024 < e1 ? s0 + 1024 : e1;
        unsigned keepbits = 0;
        int cnt = 0;
#pragma unroll 4
        for (int st = 0; st < 32; ++st) {
            const long long i = s0 + 32 * st + lane;
            if (i < s1) {
                const int v = ci[i];
                bool keep = true;
                if ((tflag & 2) && set_has_ro(deltab, delmask, arc_key(u, v))) keep = false;
                if ((tflag & 1) && set_has_ro(instab, insmask, arc_key(u, v)))
                    fail(err, kExistingArc);
                if (keep) {
                    keepbits |= 1u << st;
                    ++cnt;
                }
            }
        }
        const int tot = __reduce_add_sync(kFull, cnt);
        int base = 0;
        if (lane == 0 && tot) base = atomicAdd(cursor + u, tot);
        base = __shfl_sync(kFull, base, 0);
        int off = 0;
        for (int st = 0; st < 32; ++st) {
            const bool keep = (keepbits >> st) & 1u;
            const unsigned b = __ballot_sync(kFull, keep);
            if (keep) {
                const long long pos = r0 + base + off + __popc(b & ((1u << lane) - 1u));
                if (pos < r1) new_ci[pos] = ci[s0 + 32 * st + lane];
                else fail(err, kMissingArc);
            }
            off += __popc(b);
        }
    }
}

constexpr long long kPiece = 4096;   // arcs of a row that one warp copies at a time

// tp[v + 1] = 1 for a row the batch touches (scanned afterwards: then tp[v + 1]
// counts the touched rows up to v)
__global__ void flag_kernel(const unsigned char *touched, long long n, long long *tp)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        tp[v + 1] = touched[v] ? 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) tp[0] = 0;
}

// The touched rows in increasing order (T), their old arc ranges and the
// shift of the untouched rows that follow each of them; the touched rows
// longer than kPiece are also listed in big.
__global__ void segments_kernel(const unsigned char *touched, long long n, const long long *tp,
                                const long long *rp, const long long *new_rp, int *T,
                                long long *seg_start, long long *seg_end, long long *shift,
                                int *big, int *nbig)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!touched[v]) continue;
        const long long i = tp[v + 1] - 1;
        T[i] = (int)v;
        seg_start[i] = rp[v];
        seg_end[i] = rp[v + 1];
        shift[i] = new_rp[v + 1] - rp[v + 1];
        if (rp[v + 1] - rp[v] > kPiece) big[atomicAdd(nbig, 1)] = (int)v;
    }
}

// The arcs of the untouched rows keep their order and move by the shift of
// the touched row before them (0 before the first): one coalesced pass over
// the old arcs. Each warp copies one contiguous range, 1024 arcs per step: one
// binary search finds the touched row before the range, later steps advance
// from it, and a step that holds no touched arc copies with a single shift.
__global__ void __launch_bounds__(512) bulk_copy_kernel(const int *ci, long long m_old,
                                                        int *new_ci, const long long *seg_start,
                                                        const long long *seg_end,
                                                        const long long *shift, const long long *ntp)
{
    const unsigned lane = threadIdx.x & 31;
    const long long nT = *ntp;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long span = ((m_old + nwarps - 1) / nwarps + 31) & ~31ll;
    const long long a0 = gw * span, a1 = a0 + span < m_old ? a0 + span : m_old;
    if (a0 >= a1) return;
    long long i = -1;   // last touched row starting at or before the step's first arc
    if (lane == 0) {
        long long lo = 0, hi = nT;   // first index with seg_start > a0
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (seg_start[mid] <= a0) lo = mid + 1;
            else hi = mid;
        }
        i = lo - 1;
    }
    i = __shfl_sync(kFull, i, 0);
    for (long long c0 = a0; c0 < a1; c0 += 1024) {
        const long long c1 = c0 + 1024 < a1 ? c0 + 1024 : a1;
        while (i + 1 < nT && seg_start[i + 1] <= c0) ++i;   // the same in every lane
        const long long se = i >= 0 ? seg_end[i] : -1;
        const long long ns = i + 1 < nT ? seg_start[i + 1] : LLONG_MAX;
        if (c0 >= se && c1 <= ns) {   // no touched arc in the step
            const long long sh = i >= 0 ? shift[i] : 0;
            // all loads of a batch of 8 before its stores (the arrays may
            // alias as far as the compiler knows): 8 loads in flight a lane
            for (long long e0 = c0 + lane; e0 < c1; e0 += 8 * 32) {
                int x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const long long e = e0 + 32 * j;
                    x[j] = e < c1 ? __ldcs(ci + e) : 0;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const long long e = e0 + 32 * j;
                    if (e < c1) __stcs(new_ci + e + sh, x[j]);
                }
            }
            continue;
        }
        long long t = i;
        for (long long e = c0 + lane; e < c1; e += 32) {
            while (t + 1 < nT && seg_start[t + 1] <= e) ++t;
            if (t >= 0 && e < seg_end[t]) continue;   // a touched row: copied elsewhere
            new_ci[e + (t >= 0 ? shift[t] : 0)] = ci[e];
        }
    }
}

// Touched rows: the surviving arcs, checked against the batch's arc sets.
// Rows of at most kPiece arcs one warp each; longer ones (big) piece by
// piece, every warp taking pieces (w, w + nwarps, ...).
__global__ void __launch_bounds__(512) touched_copy_kernel(
    const long long *rp, const int *ci, const int *T, const long long *ntp, const long long *new_rp,
    int *new_ci, int *cursor, const unsigned char *touched, const int *big, const int *nbig,
    const unsigned long long *instab, unsigned insmask, const unsigned long long *deltab,
    unsigned delmask, int *err)
{
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nT = *ntp;
    for (long long j = gw; j < nT; j += nwarps) {
        const int u = T[j];
        const long long e0 = rp[u], e1 = rp[u + 1];
        if (e1 - e0 <= kPiece)
            copy_piece(u, e0, e1, ci, new_rp, new_ci, cursor, touched[u], instab, insmask, deltab,
                       delmask, err);
    }
    const int nb = *nbig;
    long long k = gw;   // global piece index over the big rows, in list order
    for (int j = 0; j < nb; ++j) {
        const int u = big[j];
        const long long e0 = rp[u], e1 = rp[u + 1];
        const long long pieces = (e1 - e0 + kPiece - 1) / kPiece;
        for (; k < pieces; k += nwarps) {
            const long long s = e0 + k * kPiece;
            copy_piece(u, s, s + kPiece < e1 ? s + kPiece : e1, ci, new_rp, new_ci, cursor,
                       touched[u], instab, insmask, deltab, delmask, err);
        }
        k -= pieces;
    }
}

// inserted arcs appended after the copies
__global__ void insert_kernel(const int *ins, long long n_ins, const long long *new_rp,
                              int *new_ci, int *cursor, int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n_ins;
         i += stride) {
        const int u = ins[i], v = ins[i ^ 1];
        const long long pos = new_rp[u] + atomicAdd(cursor + u, 1);
        if (pos < new_rp[u + 1]) new_ci[pos] = v;
        else fail(err, kMissingArc);
    }
}

// every touched row filled exactly (a deleted edge that was not in the graph
// leaves a gap; untouched rows are copied whole)
__global__ void check_kernel(const int *T, const long long *ntp, const long long *new_rp,
                             const int *cursor, int *err)
{
    const long long nT = *ntp;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nT; j += stride) {
        const int v = T[j];
        if ((long long)cursor[v] != new_rp[v + 1] - new_rp[v]) fail(err, kMissingArc);
    }
}

// ---------------------------------------------------------------------------
// step 3: insertion passes
// ---------------------------------------------------------------------------
namespace maint {

enum : int {
    L_ALLB = 0, L_CS = 1, L_CB = 2, L_QS = 3, L_QB = 4, L_NC = 5, L_RAISED = 6, L_RS = 7, L_RB = 8
};

struct Params {
    const long long *rp;
    const int *ci;
    long long n, m;
    int *core;             // in: a lower bound of the coreness; out: the coreness
    int *cd;               // neighbours of core >= own (exact for the final cores on return)
    int *sup;              // support of a candidate
    unsigned char *flag;   // 1 candidate, 3 peeled candidate, 4 just raised, 0 otherwise
    int2 *allb;            // chunks of every large vertex
    int *cs, *qs, *rs;     // candidates, peel queue, raised vertices (small vertices)
    int2 *cb, *qb, *rb;    // their chunks
    unsigned cap;
    Ctrl *ctl;
    Tuning tn;
    int max_passes;
    const int *ins;         // the batch's inserted edges (pairs): the first pass's seeds
    long long n_ins;
    int *reg;               // 1 while in the current pass's region (0 at rest)
    int max_depth;          // region levels before falling back to every candidate
    bool cd_valid;          // cd holds the counts of the graph without the inserted
                            // edges (which are added here) instead of being counted
    bool count_only;        // count cd over all arcs and stop
};

// Lists x in the current pass's region when pred holds and x is a candidate
// not listed yet. Called by all 32 lanes together.
__device__ __forceinline__ void visit(bool pred, int x, const long long *rp,
                                      const unsigned char *flag, int *reg, int *cs, int2 *cb,
                                      unsigned *live, unsigned n, unsigned cap, Ctrl *ctl,
                                      const Tuning &tn)
{
    bool fresh = false;
    long long d = 0;
    if (pred && __ldcg(flag + x) == 1) fresh = atomicCAS(reg + x, 0, 1) == 0;
    if (fresh) d = rp[x + 1] - rp[x];
    warp_append_vertex(fresh, x, d, cs, &live[L_CS], n, cb, &live[L_CB], cap, ctl, tn);
    const unsigned c = __popc(__ballot_sync(kFull, fresh));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&live[L_NC], c);
}

// region growth: the candidate neighbours of a listed vertex at its own core
// (same_core), or every candidate neighbour of a vertex raised in the previous
// pass (the seeds of a later pass)
struct GrowArc {
    static constexpr int kArcs = 4;
    const long long *rp;
    const int *core;
    const unsigned char *flag;
    int *sup;              // support, counted on the way (same_core), as SupArc does
    int *reg;
    int *cs;
    int2 *cb;
    unsigned *live;
    unsigned n, cap;
    Ctrl *ctl;
    Tuning tn;
    bool same_core;
    unsigned long long n_arcs = 0;
    __device__ __forceinline__ bool item(int v, int &a, int &)
    {
        a = ldcg(core + v);
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&vo)[kArcs],
                                         const int (&u)[kArcs], const long long (&)[kArcs],
                                         const int (&a)[kArcs], const int (&)[kArcs])
    {
        bool take[kArcs], s[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            take[j] = false;
            s[j] = false;
            if (valid[j]) {
                const bool fc = __ldcg(flag + u[j]) == 1;
                if (same_core) {
                    const int cu = ldcg(core + u[j]);
                    take[j] = fc && cu == a[j];
                    s[j] = cu > a[j] || take[j];
                } else {
                    take[j] = fc;
                }
            }
            n_arcs += valid[j];
        }
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            visit(take[j], u[j], rp, flag, reg, cs, cb, live, n, cap, ctl, tn);
        if (!same_core) return;
        const bool one = __all_sync(kFull, vo[0] == __shfl_sync(kFull, vo[0], 0) &&
                                               vo[kArcs - 1] == vo[0]);
        int mine = 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            if (one) mine += s[j];
            else if (s[j]) red_add(sup + vo[j], 1);
        }
        if (one) {
            const int tot = __reduce_add_sync(kFull, mine);
            if ((threadIdx.x & 31) == 0 && tot) red_add(sup + vo[0], tot);
        }
    }
};

// support: neighbours of higher core, or of equal core that are candidates
struct SupArc {
    static constexpr int kArcs = 4;
    const int *core;
    const unsigned char *flag;
    int *sup;
    unsigned long long n_arcs = 0;
    __device__ __forceinline__ bool item(int v, int &a, int &)
    {
        a = ldcg(core + v);
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&vo)[kArcs],
                                         const int (&u)[kArcs], const long long (&)[kArcs],
                                         const int (&a)[kArcs], const int (&)[kArcs])
    {
        bool s[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            s[j] = false;
            if (valid[j]) {
                const int cu = ldcg(core + u[j]);
                s[j] = cu > a[j] || (cu == a[j] && (__ldcg(flag + u[j]) & 1));
            }
        }
        const bool one = __all_sync(kFull, vo[0] == __shfl_sync(kFull, vo[0], 0) &&
                                               vo[kArcs - 1] == vo[0]);
        int mine = 0;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            n_arcs += valid[j];
            if (one) mine += s[j];
            else if (s[j]) red_add(sup + vo[j], 1);
        }
        if (one) {
            const int tot = __reduce_add_sync(kFull, mine);
            if ((threadIdx.x & 31) == 0 && tot) red_add(sup + vo[0], tot);
        }
    }
};

// after a pass: a raised vertex v recounts cd over its row with the new
// values, and adds itself to the cd of its neighbours that were not raised and
// sit at its new value (it now counts for them)
struct RaiseArc {
    static constexpr int kArcs = 4;
    const int *core;
    const unsigned char *flag;
    int *cd;
    unsigned long long n_arcs = 0;
    __device__ __forceinline__ bool item(int v, int &a, int &)
    {
        a = ldcg(core + v);
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&vo)[kArcs],
                                         const int (&u)[kArcs], const long long (&)[kArcs],
                                         const int (&a)[kArcs], const int (&)[kArcs])
    {
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            if (!valid[j]) continue;
            ++n_arcs;
            const int cu = ldcg(core + u[j]);
            if (cu >= a[j]) red_add(cd + vo[j], 1);
            if (cu == a[j] && __ldcg(flag + u[j]) != 4) red_add(cd + u[j], 1);
        }
    }
};

// peel: a peeled candidate w lowers the support of its equal-core candidates
struct PeelArc {
    static constexpr int kArcs = 4;
    const long long *rp;
    int *core;
    int *sup;
    unsigned char *flag;
    int *qs;
    int2 *qb;
    unsigned *c_qs, *c_qb;
    unsigned n, cap;
    Ctrl *ctl;
    Tuning tn;
    unsigned long long n_arcs = 0, n_atomics = 0;
    __device__ __forceinline__ bool item(int w, int &a, int &)
    {
        a = ldcg(core + w);
        return true;
    }
    __device__ __forceinline__ void arcs(const bool (&valid)[kArcs], const int (&)[kArcs],
                                         const int (&u)[kArcs], const long long (&)[kArcs],
                                         const int (&a)[kArcs], const int (&)[kArcs])
    {
        bool hit[kArcs];
#pragma unroll
        for (int j = 0; j < kArcs; ++j)
            hit[j] = valid[j] && ldcg(core + u[j]) == a[j] && __ldcg(flag + u[j]) == 1;
#pragma unroll
        for (int j = 0; j < kArcs; ++j) {
            n_arcs += valid[j];
            bool push = false;
            if (hit[j]) {
                ++n_atomics;
                push = atomicSub(sup + u[j], 1) == a[j] + 1;   // support fell below a + 1
                if (push) flag[u[j]] = 3;
            }
            const long long d = push ? rp[u[j] + 1] - rp[u[j]] : 0;
            warp_append_vertex(push, u[j], d, qs, c_qs, n, qb, c_qb, cap, ctl, tn);
        }
    }
};

__device__ void run(const Params &p, GridDom &dom, unsigned *s_tmp, unsigned long long *st,
                    unsigned long long &arcs, unsigned long long &atomics)
{
    Ctrl *ctl = p.ctl;
    unsigned *live = dom.live();
    const unsigned *snap = dom.s_snap;
    const unsigned tid = dom.tid(), nthreads = dom.nthreads();
    const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
    const long long n = p.n;
    const long long first = (long long)dom.cta() * blockDim.x;

    for (long long base = first; base < n; base += nthreads) {
        const long long v = base + threadIdx.x;
        long long d = 0;
        if (v < n) {
            d = p.rp[v + 1] - p.rp[v];
            if (!p.cd_valid) p.cd[v] = 0;
            p.flag[v] = 0;
            p.reg[v] = 0;
        }
        const unsigned nch =
            d > p.tn.small_deg ? (unsigned)((d + p.tn.chunk - 1) / p.tn.chunk) : 0u;
        const unsigned pos = block_alloc(nch, &live[L_ALLB], s_tmp);
        const bool fits = (unsigned long long)pos + nch <= p.cap;
        if (nch && !fits) set_error(ctl, kErrNotConverged);
        warp_fill_chunks(fits ? nch : 0u, pos, (int)v, p.allb);
    }
    if (p.cd_valid) {   // the inserted arcs join the counts
        for (long long i = tid; i < p.n_ins; i += nthreads) {
            const int a = ldcg(p.ins + 2 * i), b = ldcg(p.ins + 2 * i + 1);
            const int ca = ldcg(p.core + a), cb = ldcg(p.core + b);
            if (cb >= ca) red_add(p.cd + a, 1);
            if (ca >= cb) red_add(p.cd + b, 1);
        }
    }
    if (!dom.sync()) return;
    if (threadIdx.x == 0) ++st[kStBarriers];
    const unsigned nallb = snap[L_ALLB];
    unsigned prs = 0, prb = 0;   // vertices raised in the previous pass (rs, rb)
    auto visit_p = [&](bool pred, int x) {
        visit(pred, x, p.rp, p.flag, p.reg, p.cs, p.cb, live, (unsigned)n, p.cap, ctl, p.tn);
    };

    for (int pass = 0; pass < p.max_passes; ++pass) {
        if (dom.leader()) {
            for (int w = L_CS; w <= L_RB; ++w) live[w] = 0;
        }
        // A (first pass): cd = neighbours of core >= own, for every vertex;
        // later passes keep it up to date from the raised vertices (G)
        if (pass == 0 && !p.cd_valid) {
            i2c::CntArc<long long> f{p.core, p.cd};
            expand(p.rp, p.ci, (const int *)nullptr, (unsigned)n, p.allb, nallb, gwarp, nwarps, f,
                   p.tn);
            arcs += f.n_arcs;
            atomics += f.n_atomics;
            if (!dom.sync()) return;
            if (threadIdx.x == 0) ++st[kStBarriers];
            if (p.count_only) return;
        }
        // B: candidates (flag 1)
        for (long long base = first; base < n; base += nthreads) {
            const long long v = base + threadIdx.x;
            if (v < n) {
                const int c = ldcg(p.core + v);
                const long long d = p.rp[v + 1] - p.rp[v];
                p.sup[v] = 0;
                p.flag[v] = d >= c + 1 && ldcg(p.cd + v) >= c + 1 ? 1 : 0;
            }
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        // Region of the pass: the candidates connected to a seed through
        // candidates of equal core, listed in cs / cb. Seeds: in the first
        // pass the endpoints of the inserted edges (of an edge between
        // different cores only the lower end, which is the only one whose
        // count at its own core it raises); later, the vertices raised in the
        // previous pass and their neighbours. Every component T of survivors
        // at core c holds a seed:
        //  - later passes: without one, T and its neighbours had the same
        //    cores and T the same support in the previous pass, whose region
        //    (by induction) held T's component, so T would have risen then;
        //  - first pass: without one, T's support comes from edges that were
        //    in the graph before the batch, towards T and vertices of core
        //    >= c + 1, which were already in the old (c+1)-core (deletions
        //    only lower cores). So T lay in the old (c+1)-core. With
        //    insertions alone the cores are the old coreness, a contradiction.
        //    After deletions in the same batch, the cores are what HistoCore
        //    reached from min(old core, degree): the greatest estimates below
        //    that start that no count contradicts, and raising T to c + 1
        //    stays below the start and contradicts no count, another
        //    contradiction.
        if (pass == 0) {
            for (long long base = (long long)(tid - (tid & 31)); base < p.n_ins; base += nthreads) {
                const long long i = base + (tid & 31);
                const bool ok = i < p.n_ins;
                const int a = ok ? ldcg(p.ins + 2 * i) : 0, b = ok ? ldcg(p.ins + 2 * i + 1) : 0;
                const int ca = ok ? ldcg(p.core + a) : 0, cb = ok ? ldcg(p.core + b) : 0;
                visit_p(ok && cb >= ca, a);
                visit_p(ok && ca >= cb, b);
            }
        } else {
            i2c::for_vertices(
                p.rs, prs, p.rb, prb, tid, nthreads, gwarp, nwarps,
                [&](bool ok, int v) { visit_p(ok, v); },
                [&](int v) { visit_p((threadIdx.x & 31) == 0, v); });
            GrowArc f{p.rp, p.core, p.flag, p.sup, p.reg, p.cs, p.cb, live, (unsigned)n, p.cap,
                      ctl,  p.tn,   false};
            expand(p.rp, p.ci, p.rs, prs, p.rb, prb, gwarp, nwarps, f, p.tn,
                   batch_width(prs, prb, nwarps));
            arcs += f.n_arcs;
        }
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        // The search scans the arcs of every vertex it lists once and counts
        // its support on the way; x0 / x1 end the prefix of cs / cb so scanned.
        unsigned x0 = 0, x1 = 0;
        {
            unsigned g0 = 0, g1 = 0, h0 = snap[L_CS], h1 = snap[L_CB];
            int depth = 0;
            while (g0 < h0 || g1 < h1) {
                if (++depth > p.max_depth) {   // a long chain: take every candidate
                    for (long long base = first; base < n; base += nthreads) {
                        const long long v = base + threadIdx.x;
                        visit_p(v < n, (int)v);
                    }
                    if (!dom.sync()) return;
                    if (threadIdx.x == 0) ++st[kStBarriers];
                    break;
                }
                GrowArc f{p.rp, p.core, p.flag, p.sup, p.reg, p.cs, p.cb, live, (unsigned)n, p.cap,
                          ctl,  p.tn,   true};
                expand(p.rp, p.ci, p.cs + g0, h0 - g0, p.cb + g1, h1 - g1, gwarp, nwarps, f,
                       p.tn, batch_width(h0 - g0, h1 - g1, nwarps));
                arcs += f.n_arcs;
                if (!dom.sync()) return;
                if (threadIdx.x == 0) ++st[kStBarriers];
                g0 = h0;
                g1 = h1;
                h0 = snap[L_CS];
                h1 = snap[L_CB];
            }
            x0 = g0;
            x1 = g1;
        }
        if (threadIdx.x == 0) st[kStActive] += snap[L_NC];
        if (snap[L_NC] == 0) break;   // no seeded component: nothing can rise
        const unsigned ncs = snap[L_CS], ncb = snap[L_CB];
        // C: support of the listed vertices the search did not scan
        if (x0 < ncs || x1 < ncb) {
            SupArc f{p.core, p.flag, p.sup};
            expand(p.rp, p.ci, p.cs + x0, ncs - x0, p.cb + x1, ncb - x1, gwarp, nwarps, f, p.tn,
                   batch_width(ncs - x0, ncb - x1, nwarps));
            arcs += f.n_arcs;
            if (!dom.sync()) return;
            if (threadIdx.x == 0) ++st[kStBarriers];
        }
        // D: the candidates without enough support start the peel
        i2c::for_vertices(
            p.cs, ncs, p.cb, ncb, tid, nthreads, gwarp, nwarps,
            [&](bool ok, int v) {
                bool out = false;
                long long d = 0;
                if (ok && ldcg(p.sup + v) < ldcg(p.core + v) + 1) {
                    out = true;
                    p.flag[v] = 3;
                    d = p.rp[v + 1] - p.rp[v];
                }
                warp_append_vertex(out, v, d, p.qs, &live[L_QS], (unsigned)n, p.qb, &live[L_QB],
                                   p.cap, ctl, p.tn);
            },
            [&](int v) {
                const bool out = ldcg(p.sup + v) < ldcg(p.core + v) + 1;   // the same in every lane
                if ((threadIdx.x & 31) == 0 && out) p.flag[v] = 3;
                warp_push_chunks((threadIdx.x & 31) == 0 && out, v, p.rp[v + 1] - p.rp[v], p.qb,
                                 &live[L_QB], p.cap, ctl, p.tn.chunk);
            });
        if (!dom.sync()) return;
        if (threadIdx.x == 0) ++st[kStBarriers];
        // E: peel wave by wave
        unsigned s0 = 0, s1 = 0, e0 = snap[L_QS], e1 = snap[L_QB];
        long long waves = 0;
        while (s0 < e0 || s1 < e1) {
            if (++waves > n + 2) {
                if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
                return;
            }
            PeelArc f{p.rp,         p.core,       p.sup,       p.flag, p.qs, p.qb,
                      &live[L_QS],  &live[L_QB],  (unsigned)n, p.cap,  ctl,  p.tn};
            expand(p.rp, p.ci, p.qs + s0, e0 - s0, p.qb + s1, e1 - s1, gwarp, nwarps, f, p.tn,
                   batch_width(e0 - s0, e1 - s1, nwarps));
            arcs += f.n_arcs;
            atomics += f.n_atomics;
            if (!dom.sync()) return;
            if (threadIdx.x == 0) {
                ++st[kStBarriers];
                ++st[kStSubrounds];
            }
            s0 = e0;
            s1 = e1;
            e0 = snap[L_QS];
            e1 = snap[L_QB];
        }
        // F: the survivors rise by one (flag 4, listed); other flags back to 0
        i2c::for_vertices(
            p.cs, ncs, p.cb, ncb, tid, nthreads, gwarp, nwarps,
            [&](bool ok, int v) {
                bool up = false;
                long long d = 0;
                if (ok) {
                    up = __ldcg(p.flag + v) == 1;
                    if (up) {
                        p.core[v] = ldcg(p.core + v) + 1;
                        p.cd[v] = 0;
                        d = p.rp[v + 1] - p.rp[v];
                    }
                    p.flag[v] = up ? 4 : 0;
                    p.reg[v] = 0;
                }
                warp_append_vertex(up, v, d, p.rs, &live[L_RS], (unsigned)n, p.rb, &live[L_RB],
                                   p.cap, ctl, p.tn);
                const unsigned c = __popc(__ballot_sync(kFull, up));
                if ((threadIdx.x & 31) == 0 && c) atomicAdd(&live[L_RAISED], c);
            },
            [&](int v) {
                bool up = false;
                if ((threadIdx.x & 31) == 0) {
                    up = __ldcg(p.flag + v) == 1;
                    if (up) {
                        p.core[v] = ldcg(p.core + v) + 1;
                        p.cd[v] = 0;
                        atomicAdd(&live[L_RAISED], 1u);
                    }
                    p.flag[v] = up ? 4 : 0;
                    p.reg[v] = 0;
                }
                warp_push_chunks(up, v, p.rp[v + 1] - p.rp[v], p.rb, &live[L_RB], p.cap, ctl,
                                 p.tn.chunk);
            });
        if (!dom.sync()) return;
        if (threadIdx.x == 0) {
            ++st[kStBarriers];
            st[kStFrontier] += snap[L_RAISED];
            if (snap[L_RAISED]) ++st[kStRounds];
        }
        if (snap[L_RAISED] == 0) break;
        if (pass + 1 == p.max_passes) {
            if (threadIdx.x == 0) set_error(ctl, kErrNotConverged);
            return;
        }
        // G: cd brought up to date around the raised vertices, flags back to 0
        {
            const unsigned nrs = snap[L_RS], nrb = snap[L_RB];
            prs = nrs;
            prb = nrb;
            RaiseArc f{p.core, p.flag, p.cd};
            expand(p.rp, p.ci, p.rs, nrs, p.rb, nrb, gwarp, nwarps, f, p.tn,
                   batch_width(nrs, nrb, nwarps));
            arcs += f.n_arcs;
            if (!dom.sync()) return;
            if (threadIdx.x == 0) ++st[kStBarriers];
            i2c::for_vertices(
                p.rs, nrs, p.rb, nrb, tid, nthreads, gwarp, nwarps,
                [&](bool ok, int v) {
                    if (ok) p.flag[v] = 0;
                },
                [&](int v) {
                    if ((threadIdx.x & 31) == 0) p.flag[v] = 0;
                });
            if (!dom.sync()) return;
            if (threadIdx.x == 0) ++st[kStBarriers];
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2)
    maint_kernel(Params p, LastResult *last, unsigned long long limit_ns)
{
    __shared__ unsigned s_snap[kLiveWords + 1];
    __shared__ unsigned s_tmp[256];
    __shared__ unsigned long long s_red[32];
    __shared__ unsigned long long st[kStCount];
    if (threadIdx.x < kStCount) st[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long arcs = 0, atomics = 0;
    GridDom dom{p.ctl, s_snap, limit_ns};
    run(p, dom, s_tmp, st, arcs, atomics);
    block_sum_to(arcs, &p.ctl->stats[kStArcs], s_red);
    block_sum_to(atomics, &p.ctl->stats[kStAtomics], s_red);
    if (blockIdx.x != 0 && threadIdx.x < kStCount) st[threadIdx.x] = 0;
    finish_block(p.ctl, last, PICO_STATS_MAINTENANCE, st, kStCount);
}

}  // namespace maint

size_t maint_ws_bytes(long long n, long long m)
{
    Carver c(nullptr);
    c.take<Ctrl>(1);
    c.take<int>(n);             // sup
    c.take<unsigned char>(n);   // flag
    c.take<int>(n);             // cs
    c.take<int>(n);             // qs
    c.take<int>(n);             // rs
    c.take<int>(n);             // reg
    for (int i = 0; i < 4; ++i) c.take<int2>(chunk_capacity(m));
    return c.size();
}

}  // namespace dyn
}  // namespace pico

// ---------------------------------------------------------------------------
// the state and the C ABI
// ---------------------------------------------------------------------------
struct pico_dyn {
    int device;
    long long n, m, cap;
    long long *rp[2];
    int *ci[2];
    int cur;
    int *core;
    int *cd;         // per vertex: neighbours of core >= own (insertion passes)
    bool cd_valid;   // cd matches the current graph and coreness
    // Cost model of the recomputation fallback: device time of the last full
    // computation, and the size and device time of the last batch that ran
    // each maintenance step (deletions, insertions; size 0: none yet).
    double full_ms = 0, del_ms = 0, ins_ms = 0, mix_ms = 0;
    long long del_k = 0, ins_k = 0, mix_k = 0;   // mix: both steps of a batch with both kinds
    double cd_ms = 0;   // one count of cd over all arcs (insertion passes after deletions)
    // device time of the last update's CSR rebuild and of its coreness step
    double last_rebuild_ms = -1, last_coreness_ms = -1;
    // scratch of the coreness steps (deletions, insertion passes, a recomputation),
    // sized for the arc capacity and kept for the state's lifetime
    void *ws2 = nullptr;
    size_t ws2_bytes = 0;
    // scratch of the CSR rebuild (grown to the largest batch seen)
    void *ws1 = nullptr;
    size_t ws1_bytes = 0;
    int policy = PICO_DYN_AUTO;
    int last_kind = PICO_DYN_MAINTAINED;
};

namespace {

unsigned pow2_at_least(long long x)
{
    unsigned p = 1024;
    while ((long long)p < x && p < (1u << 31)) p <<= 1;
    return p;
}

// Device time between two events recorded around work on one stream (the
// stream is synchronised); negative when the events failed.
struct EventTimer {
    cudaEvent_t e[2] = {nullptr, nullptr};
    EventTimer()
    {
        if (cudaEventCreate(&e[0]) != cudaSuccess || cudaEventCreate(&e[1]) != cudaSuccess)
            cudaGetLastError();
    }
    ~EventTimer()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
    void start(cudaStream_t s) { if (e[0]) cudaEventRecord(e[0], s); }
    void stop(cudaStream_t s) { if (e[1]) cudaEventRecord(e[1], s); }
    double ms()
    {
        float t = -1.0f;
        if (!e[0] || !e[1] || cudaEventSynchronize(e[1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, e[0], e[1]) != cudaSuccess) {
            cudaGetLastError();
            return -1.0;
        }
        return t;
    }
};

int sync_status(cudaStream_t s)
{
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

}  // namespace

extern "C" {

namespace {

// Carves the insertion passes' scratch from ws (maint_ws_bytes) and launches
// them on the state's current graph, or only the count of cd (count_only).
bool launch_maint(pico_dyn *d, const long long *rp, const int *ci, long long m, const int32_t *ins,
                  long long n_ins, bool cd_valid, bool count_only, void *ws,
                  cudaStream_t s, const pico::LaunchCfg &cfg, pico::LastResult *last)
{
    const long long n = d->n;
    pico::dyn::maint::Params p{};
    pico::Carver cw(ws);
    p.rp = rp;
    p.ci = ci;
    p.n = n;
    p.m = m;
    p.core = d->core;
    p.cd = d->cd;
    p.ctl = cw.take<pico::Ctrl>(1);
    p.sup = cw.take<int>(n);
    p.flag = cw.take<unsigned char>(n);
    p.cs = cw.take<int>(n);
    p.qs = cw.take<int>(n);
    p.rs = cw.take<int>(n);
    p.reg = cw.take<int>(n);
    p.cap = (unsigned)pico::chunk_capacity(m);
    p.allb = cw.take<int2>(p.cap);
    p.cb = cw.take<int2>(p.cap);
    p.qb = cw.take<int2>(p.cap);
    p.rb = cw.take<int2>(p.cap);
    p.tn = cfg.tn;
    p.max_passes = (int)std::min<long long>(n_ins + 1, 1ll << 30);
    p.ins = ins;
    p.n_ins = n_ins;
    p.max_depth = 128;
    p.cd_valid = cd_valid;
    p.count_only = count_only;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(pico::Ctrl), s) != cudaSuccess) return false;
    static int occ[64] = {};
    int &o = occ[cfg.device & 63];
    if (o == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, pico::dyn::maint::maint_kernel,
                                                       pico::kThreads, 0) != cudaSuccess ||
         o <= 0))
        return false;
    const int per_sm = o < cfg.max_blocks_per_sm ? o : cfg.max_blocks_per_sm;
    unsigned long long limit = cfg.limit_ns;
    void *args[] = {&p, &last, &limit};
    return pico::launch_cooperative((const void *)pico::dyn::maint::maint_kernel,
                                       dim3(cfg.sms * per_sm), dim3(pico::kThreads), args, 0, s) ==
           cudaSuccess;
}

}  // namespace

pico_dyn *pico_dyn_create(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                          int64_t capacity_arcs, pico_stream_t stream)
{
    if (n < 1 || m < 0 || capacity_arcs < m || !row_ptr || (m > 0 && !col_idx)) return nullptr;
    if (n >= INT32_MAX || capacity_arcs >= (1ll << 36)) return nullptr;
    pico::LaunchCfg cfg;
    pico::LastResult *last = nullptr;
    if (pico::current_device(&cfg, &last) != PICO_OK) return nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    pico_dyn *d = new pico_dyn();
    d->device = cfg.device;
    d->n = n;
    d->m = m;
    d->cap = capacity_arcs;
    d->cur = 0;
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) {
        ok = cudaMalloc(&d->rp[i], (size_t)(n + 1) * sizeof(long long)) == cudaSuccess &&
             cudaMalloc(&d->ci[i], (size_t)(capacity_arcs > 0 ? capacity_arcs : 1) * sizeof(int)) ==
                 cudaSuccess;
    }
    ok = ok && cudaMalloc(&d->core, (size_t)n * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&d->cd, (size_t)n * sizeof(int)) == cudaSuccess;
    d->ws2_bytes = std::max({pico::histocore_ws_bytes(n, capacity_arcs),
                             pico::dyn::maint_ws_bytes(n, capacity_arcs),
                             pico::hybrid_ws_bytes(n, capacity_arcs)});
    ok = ok && cudaMalloc(&d->ws2, d->ws2_bytes) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d->rp[0], row_ptr, (size_t)(n + 1) * sizeof(long long),
                               cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    ok = ok && (m == 0 || cudaMemcpyAsync(d->ci[0], col_idx, (size_t)m * sizeof(int),
                                          cudaMemcpyDeviceToDevice, s) == cudaSuccess);
    // the first coreness runs PICO_ALGO_AUTO on the state's scratch, as a
    // recomputation does, twice: the second run's time, the cost model's
    // reference, holds no allocation and no first launch of the kernel
    EventTimer full;
    for (int rep = 0; rep < 2 && ok; ++rep) {
        full.start(s);
        if (m > 0)
            ok = pico::launch_hybrid<long long>(d->rp[0], d->ci[0], n, m, d->core, d->ws2, last,
                                                s, cfg) == 0;
        else
            ok = cudaMemsetAsync(d->core, 0, (size_t)n * sizeof(int), s) == cudaSuccess;
        full.stop(s);
    }
    // cd for the first insertion batch: one count over all arcs
    EventTimer count;
    count.start(s);
    ok = ok && launch_maint(d, d->rp[0], d->ci[0], m, nullptr, 0, false, true, d->ws2, s, cfg,
                            last);
    count.stop(s);
    ok = ok && sync_status(s) == PICO_OK && pico_last_device_status(stream) == PICO_OK;
    if (!ok) {
        cudaGetLastError();
        pico_dyn_destroy(d);
        return nullptr;
    }
    d->cd_valid = true;
    d->full_ms = full.ms();
    d->cd_ms = std::max(0.0, count.ms());
    return d;
}

int pico_dyn_update(pico_dyn *d, const int32_t *ins, int64_t n_ins, const int32_t *del,
                    int64_t n_del, pico_stream_t stream)
{
    if (!d || n_ins < 0 || n_del < 0 || (n_ins > 0 && !ins) || (n_del > 0 && !del))
        return PICO_ERR_INVALID_ARG;
    const long long n = d->n, m_old = d->m, m_new = d->m + 2 * n_ins - 2 * n_del;
    if (m_new < 0 || m_new > d->cap || n_ins + n_del > (1ll << 28)) return PICO_ERR_INVALID_ARG;
    if (n_ins == 0 && n_del == 0) return PICO_OK;
    pico::LaunchCfg cfg;
    pico::LastResult *last = nullptr;
    int rc = pico::current_device(&cfg, &last);
    if (rc != PICO_OK) return rc;
    if (cfg.device != d->device) return PICO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long long *rp = d->rp[d->cur];
    const int *ci = d->ci[d->cur];
    long long *nrp = d->rp[1 - d->cur];
    int *nci = d->ci[1 - d->cur];
    const unsigned insmask = pow2_at_least(4 * n_ins + 1) - 1, delmask = pow2_at_least(4 * n_del + 1) - 1;
    // scratch: counts, cursors, flags, touched-row lists, hash sets, scans
    const long long nt_cap = std::min<long long>(n, 2 * (n_ins + n_del));
    using pico::Carver;
    Carver c0(nullptr);
    c0.take<int>(n);                     // ins_cnt
    c0.take<int>(n);                     // del_cnt
    c0.take<int>(n);                     // cursor
    c0.take<unsigned char>(n + 4);       // touched
    c0.take<int>(4);                     // nbig, err
    c0.take<unsigned long long>(insmask + 1ull);
    c0.take<unsigned long long>(delmask + 1ull);
    c0.take<long long>(4096);            // scan sums
    c0.take<pico::Ctrl>(1);
    c0.take<pico::Ctrl>(1);
    const size_t zero_bytes = c0.size();
    c0.take<long long>(n + 1);           // touched-row scan
    c0.take<int>(nt_cap);                // touched rows in order
    c0.take<int>(nt_cap);                // the long ones
    for (int i = 0; i < 3; ++i) c0.take<long long>(nt_cap);   // their arc ranges, shifts
    const size_t pre_bytes = c0.size();
    if (pre_bytes > d->ws1_bytes) {   // grow the rebuild's scratch (kept for later batches)
        if (d->ws1) {
            cudaStreamSynchronize(s);
            cudaFree(d->ws1);
        }
        d->ws1 = nullptr;
        d->ws1_bytes = 0;
        if (cudaMalloc(&d->ws1, pre_bytes) != cudaSuccess) {
            cudaGetLastError();
            d->ws1 = nullptr;
            return PICO_ERR_OOM;
        }
        d->ws1_bytes = pre_bytes;
    }
    void *ws = d->ws1;
    Carver c(ws);
    int *ins_cnt = c.take<int>(n), *del_cnt = c.take<int>(n), *cursor = c.take<int>(n);
    unsigned char *touched = c.take<unsigned char>(n + 4);
    int *flags = c.take<int>(4);
    unsigned long long *instab = c.take<unsigned long long>(insmask + 1ull);
    unsigned long long *deltab = c.take<unsigned long long>(delmask + 1ull);
    long long *sums = c.take<long long>(4096);
    pico::Ctrl *sctl = c.take<pico::Ctrl>(1), *sctl2 = c.take<pico::Ctrl>(1);
    long long *tp = c.take<long long>(n + 1);
    int *T = c.take<int>(nt_cap), *big = c.take<int>(nt_cap);
    long long *seg_start = c.take<long long>(nt_cap), *seg_end = c.take<long long>(nt_cap);
    long long *shift = c.take<long long>(nt_cap);
    void *ws2 = d->ws2;
    int *nbig = flags, *err = flags + 1;
    const int G = cfg.sms * 4;
    auto scan = [&](long long *arr, pico::Ctrl *ctl) {   // in-place scan of arr[1..n]
        long long *a = arr;
        long long nn = n;
        unsigned long long limit = cfg.limit_ns;
        void *args[] = {&a, &nn, &ctl, &sums, &limit};
        return pico::launch_cooperative((const void *)pico::dyn::scan_kernel, dim3(cfg.sms),
                                           dim3(pico::kThreads), args, 0, s) == cudaSuccess;
    };
    EventTimer trebuild;
    trebuild.start(s);
    bool ok = cudaMemsetAsync(ws, 0, zero_bytes, s) == cudaSuccess;
    if (ok) {
        pico::dyn::count_kernel<<<G, 256, 0, s>>>(ins, n_ins, del, n_del, n, ins_cnt, del_cnt,
                                                 touched, instab, insmask, deltab, delmask, err);
        pico::dyn::degree_kernel<<<G, 256, 0, s>>>(rp, n, ins_cnt, del_cnt, nrp, err);
        pico::dyn::flag_kernel<<<G, 256, 0, s>>>(touched, n, tp);
        ok = cudaGetLastError() == cudaSuccess && scan(nrp, sctl) && scan(tp, sctl2);
    }
    if (ok) {
        pico::dyn::segments_kernel<<<G, 256, 0, s>>>(touched, n, tp, rp, nrp, T, seg_start,
                                                    seg_end, shift, big, nbig);
        pico::dyn::bulk_copy_kernel<<<cfg.sms * 2, 512, 0, s>>>(ci, m_old, nci, seg_start, seg_end,
                                                               shift, tp + n);
        pico::dyn::touched_copy_kernel<<<cfg.sms * 2, 512, 0, s>>>(
            rp, ci, T, tp + n, nrp, nci, cursor, touched, big, nbig, instab, insmask, deltab,
            delmask, err);
        if (n_ins > 0)
            pico::dyn::insert_kernel<<<G, 256, 0, s>>>(ins, n_ins, nrp, nci, cursor, err);
        pico::dyn::check_kernel<<<G, 256, 0, s>>>(T, tp + n, nrp, cursor, err);
        ok = cudaGetLastError() == cudaSuccess;
    }
    trebuild.stop(s);
    int herr = 0;
    ok = ok && sync_status(s) == PICO_OK &&
         cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    long long m_chk = -1;
    ok = ok && cudaMemcpy(&m_chk, nrp + n, sizeof(long long), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok || herr != 0 || m_chk != m_new) {
        cudaGetLastError();
        return !ok ? PICO_ERR_CUDA : PICO_ERR_BAD_GRAPH;   // the state is unchanged
    }
    // the graph is consistent: switch to it and bring the coreness up to date
    d->last_rebuild_ms = trebuild.ms();
    d->last_coreness_ms = -1;
    d->cur = 1 - d->cur;
    d->m = m_new;
    const bool cd_was_valid = d->cd_valid;
    d->cd_valid = false;   // until insertion passes leave it exact
    // Maintain, or recompute from scratch when the batch's predicted
    // maintenance time exceeds the last full computation's. A step's time
    // is predicted from the last batch that ran it, scaled by the edge
    // counts, only when the sizes are within a factor of two (a step's cost
    // is not linear over a wider range); otherwise the batch is maintained
    // and measured. Insertion passes that must first recount cd (after
    // deletions, or when cd is stale) add one count over all arcs, timed
    // when the state was created. A batch with both kinds is predicted from
    // the last such batch when one of a similar size ran; otherwise from the
    // two steps' separate costs times kMixedPenalty, because insertion passes
    // that follow deletions search wider regions than the same insertions
    // into an unchanged graph (on R-MAT scale 24 with 10,000 edges of each
    // kind, 1.75 G arcs against 1.37 G, and 15 % more time than the sum).
    constexpr double kMixedPenalty = 1.25;
    const bool cd_recount = n_ins > 0 && !(cd_was_valid && n_del == 0);
    bool recompute = d->policy == PICO_DYN_RECOMPUTE;
    if (d->policy == PICO_DYN_AUTO && d->full_ms > 0) {
        auto near = [](long long k, long long k0) { return k0 > 0 && 2 * k >= k0 && k <= 2 * k0; };
        const bool mixed = n_del > 0 && n_ins > 0;
        bool known = (n_del == 0 || near(n_del, d->del_k)) && (n_ins == 0 || near(n_ins, d->ins_k));
        double pred = (n_del ? d->del_ms * (double)n_del / (double)std::max(1ll, d->del_k) : 0.0) +
                      (n_ins ? d->ins_ms * (double)n_ins / (double)std::max(1ll, d->ins_k) : 0.0) +
                      (cd_recount ? d->cd_ms : 0.0);
        if (mixed && near(n_del + n_ins, d->mix_k)) {
            known = true;
            pred = d->mix_ms * (double)(n_del + n_ins) / (double)d->mix_k;
        } else if (mixed) {
            pred *= kMixedPenalty;
        }
        recompute = known && pred > d->full_ms;
    }
    if (recompute) {
        EventTimer full;
        full.start(s);
        if (m_new > 0)   // PICO_ALGO_AUTO on the state's scratch
            rc = pico::launch_hybrid<long long>(nrp, nci, n, m_new, d->core, ws2, last, s, cfg) == 0
                     ? PICO_OK
                     : PICO_ERR_CUDA;
        else
            rc = cudaMemsetAsync(d->core, 0, (size_t)n * sizeof(int), s) == cudaSuccess
                     ? PICO_OK
                     : PICO_ERR_CUDA;
        full.stop(s);
        if (rc != PICO_OK) {
            cudaGetLastError();
            return rc;
        }
        if (sync_status(s) != PICO_OK) return PICO_ERR_CUDA;
        const double t = full.ms();
        if (t > 0) d->full_ms = t;
        d->last_coreness_ms = t;
        d->last_kind = PICO_DYN_RECOMPUTED;
        return pico_last_device_status(stream);   // cd stays invalid: the next insertion
    }                                             // batch recounts it
    EventTimer tdel, tins;
    tdel.start(s);
    if (n_del > 0 && m_new > 0) {
        rc = pico::launch_histocore<long long>(nrp, nci, n, m_new, d->core, ws2, last, s, cfg,
                                               d->core);
        if (rc != 0 || cudaGetLastError() != cudaSuccess) ok = false;
    } else if (n_del > 0) {
        ok = cudaMemsetAsync(d->core, 0, (size_t)n * sizeof(int), s) == cudaSuccess;
    }
    tdel.stop(s);
    tins.start(s);
    if (ok && n_ins > 0)
        ok = launch_maint(d, nrp, nci, m_new, ins, n_ins, cd_was_valid && n_del == 0, false, ws2,
                          s, cfg, last);
    tins.stop(s);
    if (!ok) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    if (sync_status(s) != PICO_OK) return PICO_ERR_CUDA;
    const int st = pico_last_device_status(stream);
    d->last_coreness_ms = tdel.ms() + tins.ms();
    d->cd_valid = st == PICO_OK && n_ins > 0;
    d->last_kind = PICO_DYN_MAINTAINED;
    if (st == PICO_OK) {
        const double a = tdel.ms(), b = tins.ms();
        if (n_del > 0 && a > 0) {
            d->del_ms = a;
            d->del_k = n_del;
        }
        if (n_ins > 0 && b > 0) {   // the passes alone, without the recount of cd
            d->ins_ms = std::max(0.1 * b, b - (cd_recount ? d->cd_ms : 0.0));
            d->ins_k = n_ins;
        }
        if (n_del > 0 && n_ins > 0 && a > 0 && b > 0) {
            d->mix_ms = a + b;
            d->mix_k = n_del + n_ins;
        }
    }
    return st;
}

int pico_dyn_set_policy(pico_dyn *d, int policy)
{
    if (!d || policy < PICO_DYN_AUTO || policy > PICO_DYN_RECOMPUTE) return PICO_ERR_INVALID_ARG;
    d->policy = policy;
    return PICO_OK;
}

int pico_dyn_last_update_kind(pico_dyn *d)
{
    if (!d) return PICO_ERR_INVALID_ARG;
    return d->last_kind;
}

int pico_dyn_last_update_times(pico_dyn *d, double *rebuild_ms, double *coreness_ms)
{
    if (!d || !rebuild_ms || !coreness_ms) return PICO_ERR_INVALID_ARG;
    *rebuild_ms = d->last_rebuild_ms;
    *coreness_ms = d->last_coreness_ms;
    return PICO_OK;
}

int pico_dyn_coreness(pico_dyn *d, int32_t *out_core, pico_stream_t stream)
{
    if (!d || !out_core) return PICO_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(out_core, d->core, (size_t)d->n * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

int pico_dyn_graph(pico_dyn *d, const int64_t **row_ptr, const int32_t **col_idx, int64_t *n,
                   int64_t *m)
{
    if (!d || !row_ptr || !col_idx || !n || !m) return PICO_ERR_INVALID_ARG;
    *row_ptr = reinterpret_cast<const int64_t *>(d->rp[d->cur]);
    *col_idx = d->ci[d->cur];
    *n = d->n;
    *m = d->m;
    return PICO_OK;
}

int pico_dyn_copy_graph(pico_dyn *d, int64_t *row_ptr, int32_t *col_idx, pico_stream_t stream)
{
    if (!d || !row_ptr || (d->m > 0 && !col_idx)) return PICO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(row_ptr, d->rp[d->cur], (size_t)(d->n + 1) * sizeof(int64_t),
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        (d->m > 0 && cudaMemcpyAsync(col_idx, d->ci[d->cur], (size_t)d->m * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, s) != cudaSuccess)) {
        cudaGetLastError();
        return PICO_ERR_CUDA;
    }
    return PICO_OK;
}

void pico_dyn_destroy(pico_dyn *d)
{
    if (!d) return;
    for (int i = 0; i < 2; ++i) {
        if (d->rp[i]) cudaFree(d->rp[i]);
        if (d->ci[i]) cudaFree(d->ci[i]);
    }
    if (d->core) cudaFree(d->core);
    if (d->cd) cudaFree(d->cd);
    if (d->ws2) cudaFree(d->ws2);
    if (d->ws1) cudaFree(d->ws1);
    cudaGetLastError();
    delete d;
}

}  // extern "C"
