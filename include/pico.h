/*
 * pico.h -- C ABI of the GB300 (sm_103a) k-core decomposition library.
 *
 * The library computes the coreness of every vertex of a simple undirected
 * graph: core(v) is the largest k such that v belongs to the k-core, the
 * maximal subgraph whose minimum degree is at least k; an isolated vertex has
 * core 0 (Sec. I of "PICO: Accelerating All k-Core Paradigms on GPU").
 * Two methods compute it and return identical vectors:
 *   PICO_ALGO_PEELONE    PeelOne (Sec. III, Alg. 4): level-synchronous peel
 *                        with the clamped decrement of Sec. III-B ("assertion")
 *                        and the dynamic frontier of Sec. III-C.
 *   PICO_ALGO_HISTOCORE  HistoCore (Sec. IV-B, Alg. 6): h-index iteration
 *                        over per-vertex neighbour histograms, restricted to
 *                        the vertices whose count fell below their estimate
 *                        (Thm. 2).
 *
 * Graph layout (CSR, device memory, read only):
 *   row_ptr  n + 1 offsets; row_ptr[0] == 0, non-decreasing;
 *            row_ptr[n] == m == the number of ARCS (twice the undirected
 *            edges: every edge {u, v} appears as u->v and v->u).
 *   col_idx  m int32 neighbour ids in [0, n). The graph must be symmetric,
 *            without self-loops or duplicate arcs. Neighbour order is free.
 *   out_core n int32 results, written in full (device memory, caller-owned).
 *
 * Asynchrony: every compute call is enqueued on `stream` (NULL = the legacy
 * default stream) and returns before the work is done. The return value
 * reports argument and launch errors only. Failures seen on the device (a
 * bounded wait that ran out, a malformed graph detected in flight) are
 * recorded in a per-device status word: read it with pico_last_device_status
 * after the call, which also synchronises the stream.
 *
 * Memory: scratch space comes from CUDA's stream-ordered allocator
 * (cudaMallocAsync on `stream`) and is released on the same stream when the
 * call's work ends; pico_workspace_bytes reports its size. Inputs are never
 * written. Concurrent calls on different streams are independent, except
 * that the per-device status word and statistics are shared (last writer wins).
 *
 * Requirements: a GPU of compute capability 10.3 (GB300); n < 2^31; for the
 * int32-offset entry points m < 2^31. Thread safety: calls may come from any
 * host thread; the CUDA device current on the calling thread is used.
 */
#ifndef PICO_H
#define PICO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *pico_stream_t;

typedef enum {
    PICO_ALGO_PEELONE = 0,   /* Alg. 4, Sec. III-C */
    PICO_ALGO_HISTOCORE = 1, /* Alg. 6, Sec. IV-B */
    /* The baselines of the paper's evaluation (Sec. V), for comparisons on the
       same runtime; single-graph entry points only (pico_coreness and
       pico_coreness_i64; the batched form and the server take methods 0 and
       1). They return the same coreness. */
    PICO_ALGO_GPP = 2,          /* General Parallel Peel, Alg. 3: separate residual
                                   degree and removed flag, no dynamic frontier */
    PICO_ALGO_PEEL_CAS = 3,     /* PeelOne with atomicSub_{>=k} as a compare-and-swap
                                   loop, as Sec. III-B states it */
    PICO_ALGO_PEEL_ADDBACK = 4, /* PeelOne with the atomicAdd method of Fig. 4a: an
                                   overshooting decrement is added back at once */
    PICO_ALGO_NBRCORE = 5,      /* NbrCore: neighbours of changed vertices recompute
                                   HINDEX (Alg. 2) from scratch */
    PICO_ALGO_CNTCORE = 6,      /* CntCore, Alg. 5: only the vertices with cnt below
                                   their estimate (Thm. 2) recompute HINDEX */
    /* Either method, chosen per graph (no counterpart in the paper, which
       leaves the choice open). Single-graph calls decide on the device from
       n, m and the largest degree: HistoCore when the degrees are skewed
       (d_max >= 64 m/n) and m^2 <= 2^14 d_max n, PeelOne otherwise (a rule
       fitted to GB300 timings of both methods). The batched form and the
       server run PeelOne for every graph, which was faster than HistoCore on
       every measured graph class in one-CTA and one-cluster domains.
       pico_get_stats reports the method that ran. */
    PICO_ALGO_AUTO = 7
} pico_algo;

typedef enum {
    PICO_OK = 0,
    PICO_ERR_INVALID_ARG = -1,   /* null pointer, negative size, unknown algo */
    PICO_ERR_OOM = -2,           /* scratch allocation failed */
    PICO_ERR_CUDA = -3,          /* a CUDA runtime call failed (launch, copy) */
    PICO_ERR_NOT_CONVERGED = -4, /* a device loop exceeded its proven bound */
    PICO_ERR_TIMEOUT = -5,       /* a device-side wait exceeded its time limit */
    PICO_ERR_BAD_GRAPH = -6,     /* validation found a malformed CSR */
    PICO_ERR_NO_DEVICE = -7      /* no usable sm_103 device is current */
} pico_status;

/*
 * Coreness of one graph with int32 offsets (m < 2^31).
 * n: vertices (>= 0); m: arcs (must equal row_ptr[n]); algo: a pico_algo.
 * n == 0 is a no-op. Returns PICO_OK or a negative pico_status.
 */
int pico_coreness(const int32_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                  int32_t *out_core, int algo, pico_stream_t stream);

/* The same with int64 offsets (row_ptr has n + 1 int64 entries). */
int pico_coreness_i64(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                      int32_t *out_core, int algo, pico_stream_t stream);

/*
 * Input validation (no counterpart in the paper, which takes simple
 * undirected graphs as given, Sec. II-A). Checks on the device that
 * (row_ptr, col_idx) is a graph the compute entry points are specified for,
 * and reports what it found as PICO_DEFECT_* bits:
 *   ROWS       row_ptr[0] != 0, row_ptr decreasing somewhere, or
 *              row_ptr[n] != m (the arcs are then not examined);
 *   IDS        a neighbour id outside [0, n);
 *   LOOP       a self-loop (v, v);
 *   ORDER      a row not strictly increasing: unsorted, or a duplicate arc;
 *   ASYMMETRIC an arc (v, u) without its reverse (u, v).
 * Validation requires sorted rows; the compute entry points themselves do
 * not (an unsorted but otherwise valid graph is reported as ORDER).
 * Every access is bounds-checked, so any input of the stated sizes is safe
 * to validate. defects: optional host pointer receiving the OR of the bits
 * (0 for a valid graph). The call synchronises `stream`. Returns PICO_OK,
 * PICO_ERR_BAD_GRAPH when a defect was found, PICO_ERR_INVALID_ARG for
 * negative sizes or null pointers, PICO_ERR_OOM or PICO_ERR_CUDA. n == 0 is
 * valid iff m == 0 and reads nothing.
 * With PICO_VALIDATE=1 in the environment (read when a device is first
 * used), pico_coreness and pico_coreness_i64 validate their graph first and
 * return PICO_ERR_BAD_GRAPH without computing when a defect is found; they
 * then synchronise their stream and cannot be captured in a CUDA graph.
 */
#define PICO_DEFECT_ROWS 1u
#define PICO_DEFECT_IDS 2u
#define PICO_DEFECT_LOOP 4u
#define PICO_DEFECT_ORDER 8u
#define PICO_DEFECT_ASYMMETRIC 16u
int pico_validate_graph(const int32_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                        uint32_t *defects, pico_stream_t stream);
int pico_validate_graph_i64(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                            uint32_t *defects, pico_stream_t stream);

/*
 * Coreness of G independent graphs packed back to back, in one launch.
 * Coreness is defined per graph (Sec. I), so the result equals G separate
 * calls; each graph must satisfy the single-graph contract and may be empty.
 *   vtx_off, arc_off: device int64 prefix offsets, G + 1 entries each
 *     (vtx_off[0] == arc_off[0] == 0); graph g owns vertices
 *     [vtx_off[g], vtx_off[g+1]) and arcs [arc_off[g], arc_off[g+1]).
 *   row_ptr: device int32, graph-local offsets (relative to arc_off[g]);
 *     graph g's n_g + 1 entries start at row_ptr[vtx_off[g] + g], so the
 *     array holds vtx_off[G] + G entries.
 *   col_idx: device int32, graph-local vertex ids, arc_off[G] entries.
 *   total_vertices, total_arcs: must equal vtx_off[G] and arc_off[G] (the
 *     host cannot read device memory without synchronising).
 *   out_core: device int32, vtx_off[G] entries, each graph's coreness.
 * One CTA solves one graph at a time, largest graphs first; a graph needs
 * fewer than 2^31 arcs. G == 0 is a no-op.
 */
int pico_coreness_batched(const int64_t *vtx_off, const int64_t *arc_off, int32_t G,
                          const int32_t *row_ptr, const int32_t *col_idx,
                          int64_t total_vertices, int64_t total_arcs, int32_t *out_core,
                          int algo, pico_stream_t stream);

/* Scratch bytes a batched call with these totals allocates. */
size_t pico_workspace_bytes_batched(int32_t G, int64_t total_vertices, int64_t total_arcs,
                                    int algo);

/*
 * PeelOne for callers that cannot allocate device memory. The paper has no
 * counterpart: this entry point exists for host code that must not call
 * cudaMalloc or any other allocating routine while it runs, for example a
 * service that reserved its whole device-memory budget at start-up, or an
 * embedding framework that owns every allocation. It computes what
 * pico_coreness(..., PICO_ALGO_PEELONE, ...) computes, allocates nothing, and
 * takes its scratch from one array compiled into the library: 19 MiB of
 * device memory that every GPU on which the library is loaded holds until
 * the process exits.
 *
 * Limits: n <= PICO_NOALLOC_MAX_VERTICES and m <= PICO_NOALLOC_MAX_ARCS;
 * larger graphs are rejected with PICO_ERR_INVALID_ARG before any GPU work.
 * out_status: optional device int32 (NULL to skip) that receives the
 * device-side status of this call (PICO_OK, or e.g. PICO_ERR_TIMEOUT) on
 * `stream`; these calls do not update pico_last_device_status or
 * pico_get_stats.
 * The first call on a device looks up the array's device address (no
 * allocation) and should come before any stream capture. All calls on a
 * device share the array; each call clears what must start at zero, but
 * calls whose GPU work overlaps (different streams, or threads racing) use
 * the same memory at once and race: issue them one after another.
 */
#define PICO_NOALLOC_MAX_VERTICES (1 << 20)
#define PICO_NOALLOC_MAX_ARCS (1 << 24)
int pico_coreness_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                          int32_t *out_core, int32_t *out_status, pico_stream_t stream);

/*
 * Request server: continuous batching of coreness requests on the current
 * device (the serving form; the paper has no counterpart). An engine thread
 * admits arrived requests in arrival order while their device bytes (packed
 * CSR, results and the batched call's scratch) fit in hbm_budget_bytes next
 * to the requests already on the device, packs them into one micro-batch and
 * solves it with one pico_coreness_batched launch on a free stream; up to
 * `streams` micro-batches run at once, so requests that arrive while others
 * run are admitted as slots and memory free up and overlap on the device.
 * With single_graph = 1 each request is solved by its own pico_coreness call
 * (with max_batch = 1 and streams = 1: the sequential plain path).
 */
typedef struct pico_server pico_server;

typedef struct {
    size_t hbm_budget_bytes; /* device bytes the admitted requests may hold */
    int algo;                /* PICO_ALGO_PEELONE, _HISTOCORE or _AUTO for every request */
    int streams;             /* micro-batches in flight at once (1..64) */
    int max_batch;           /* requests per micro-batch (>= 1) */
    int single_graph;        /* 1: one single-graph call per request */
} pico_server_config;

/* Creates a server on the current device; NULL on invalid config or failure. */
pico_server *pico_server_create(const pico_server_config *cfg);

/*
 * Submits one graph: host CSR (int32 row_ptr with n + 1 entries, int32
 * col_idx with m entries) and a host buffer of n int32 for the result. The
 * buffers must stay valid until the request completes and should be pinned
 * (page-locked) so that copies overlap. arrival_ns (pico_clock_ns's clock):
 * the request is not admitted before that time, so a recorded arrival
 * process can be replayed. Returns the ticket (>= 0) or a negative status
 * (PICO_ERR_OOM: the graph alone exceeds the budget).
 */
int64_t pico_server_submit(pico_server *server, const int32_t *row_ptr, const int32_t *col_idx,
                           int64_t n, int64_t m, int32_t *out_core, int64_t arrival_ns);

/* Moves up to cap completed tickets and their completion times
   (pico_clock_ns) into the arrays; returns how many, or a negative status. */
int pico_server_poll(pico_server *server, int64_t *tickets, int64_t *done_ns, int cap);

/* The same, and into device_ns (NULL to skip) the device time of the
   micro-batch that served each request: CUDA events around its copies to
   the device, its launch and the copies of its results back (-1 when the
   micro-batch failed). The host-side wait before admission is not in it. */
int pico_server_poll_device(pico_server *server, int64_t *tickets, int64_t *done_ns,
                            int64_t *device_ns, int cap);

/* Blocks until every submitted request has completed; returns the first
   error seen by the engine (PICO_OK if none). */
int pico_server_drain(pico_server *server);

/* Stops the engine after the submitted requests complete and frees the server. */
int pico_server_destroy(pico_server *server);

/* Monotonic clock of the server, in nanoseconds. */
int64_t pico_clock_ns(void);

/* Scratch bytes a single-graph call with these sizes allocates (admission
   accounting). Returns 0 for invalid arguments. */
size_t pico_workspace_bytes(int64_t n, int64_t m, int algo);

/* Static text for a pico_status value (never NULL). */
const char *pico_status_string(int status);

/*
 * Synchronises `stream`, then returns and clears the current device's sticky
 * device-side status: PICO_OK, or the first error recorded by any call since
 * the last read. Returns PICO_ERR_CUDA if the synchronisation itself fails.
 */
int pico_last_device_status(pico_stream_t stream);

/* Counters of the most recent call on the current device (after a
   synchronisation of its stream). Fields a method does not use stay 0. */
typedef struct {
    int64_t algo;        /* pico_algo of the call */
    int64_t levels;      /* PeelOne: non-empty levels executed */
    int64_t kmax;        /* PeelOne: largest level (the maximum coreness) */
    int64_t subrounds;   /* PeelOne: frontier waves over all levels */
    int64_t scans;       /* PeelOne: residual scans (levels + empty probes) */
    int64_t rounds;      /* HistoCore: SumHisto/UpdateHisto rounds */
    int64_t frontier;    /* HistoCore: sum over rounds of |V_cnt| */
    int64_t barriers;    /* grid-wide barriers executed */
    int64_t arcs;        /* PeelOne: adjacency entries read by the expansion phases;
                            HistoCore: arcs of InitHisto plus, per round, the arcs of the
                            changed vertices (what Alg. 6 scans, in either direction) */
    int64_t atomics;     /* atomic read-modify-writes on core[] or histo[] */
    int64_t slots;       /* HistoCore: histogram slots read by SumHisto */
    int64_t blocks;      /* CTAs of the persistent launch */
    int64_t scanned;     /* PeelOne: residual-list entries read, summed over scans */
    int64_t pulled;      /* HistoCore: arcs scanned by pull rounds of UpdateHisto */
    int64_t pull_rounds; /* HistoCore: rounds whose UpdateHisto pulled */
    int64_t extra;       /* PeelOne and its variants: atomics beyond the successful
                            decrements (overshoots; failed compare-and-swaps) */
    int64_t active;      /* NbrCore, CntCore: sum over rounds of the active-set size */
    /* Device time (ns) and count per phase kind, measured by CTA 0 from one
       grid barrier to the next: [0] init, [1] PeelOne residual scan,
       [2..4] PeelOne frontier waves with < 64 work units / fewer units than
       warps / more, [5] InitHisto, [6] SumHisto, [7] UpdateHisto. */
    int64_t phase_ns[8];
    int64_t phase_count[8];
} pico_stats;

int pico_get_stats(pico_stream_t stream, pico_stats *out);

/*
 * Phase trace of the most recent single-graph call on the current device,
 * recorded only when the environment variable PICO_TRACE=1 was set when the
 * device was first used (it costs one store per phase). Synchronises
 * `stream`, then writes up to cap entries of three int64 each: phase kind (as
 * in pico_stats.phase_ns), work units of the phase (vertices or chunks), and
 * its device time in ns. Returns the number of entries or a negative status.
 */
int pico_get_trace(pico_stream_t stream, int64_t *out, int cap);

/*
 * Self-test of device-side failure detection (no counterpart in the paper).
 * Runs the grid barrier of the persistent kernels with one CTA that never
 * arrives, so the other CTAs' bounded waits run out after limit_ms (1..10000)
 * milliseconds; nothing faults or hangs. Synchronises `stream` and returns
 * the device status the launch recorded: PICO_ERR_TIMEOUT when the failure
 * path works. Clears the sticky status before and after.
 * Environment: PICO_WAIT_LIMIT_MS sets the wait limit of the compute kernels
 * (default 4000, read once per device); PICO_FAULT_ALLOC=1 makes every
 * scratch allocation of the compute entry points fail with PICO_ERR_OOM
 * (host-side fault injection for tests).
 */
int pico_selftest_wait_timeout(int limit_ms, pico_stream_t stream);

/*
 * Degree-class work assignment of the current device's kernels (set by the
 * autotuner, paper_2402_15253_gb300/autotune.py): vertices of degree at most
 * small_deg (32..256) are batched 32 per warp; larger ones are split into
 * chunks of `chunk` arcs (64..4096), one per warp; batched_threads (256 or
 * 512) is the CTA size of the batched kernel, where a graph with at least
 * 2^cluster_log2 arcs (10..62; 62 disables clusters) is solved by a cluster of
 * 8 CTAs and every other graph by one CTA. Applies to later calls on the
 * device; defaults 32, 256, 512, 21. Results never depend on these values,
 * only the speed does.
 */
int pico_set_tuning(int small_deg, int chunk, int batched_threads, int cluster_log2);
int pico_get_tuning(int *small_deg, int *chunk, int *batched_threads, int *cluster_log2);

/*
 * Core maintenance (no counterpart in the paper, which lists it among the
 * uses of the Index2core paradigm): a graph and its coreness kept on the
 * device and brought up to date after each batch of edge insertions and
 * deletions, without recomputation from the degrees.
 *
 * pico_dyn_create copies the CSR (row_ptr int64, n + 1 entries; col_idx m
 * arcs; device memory, read only) into the state, which holds room for
 * capacity_arcs arcs (>= m), computes its coreness and synchronises `stream`.
 * Returns NULL for invalid arguments (n < 1, capacity below m) or failure.
 *
 * pico_dyn_update applies one batch of undirected edges: ins and del are
 * device arrays of n_ins and n_del pairs (u, v) (int32, 2 entries per edge).
 * Every deleted edge must be in the graph and every inserted edge must not;
 * no self-loops, no edge twice in a batch. Deletions are applied first. The
 * call synchronises `stream` and returns PICO_OK, PICO_ERR_BAD_GRAPH for a
 * batch that breaks these rules (the state is then unchanged),
 * PICO_ERR_INVALID_ARG (bad sizes, too little capacity) or a device status.
 * After an update with insertions, pico_get_stats describes the insertion
 * passes (algo PICO_STATS_MAINTENANCE: rounds = passes that raised a vertex,
 * frontier = vertices raised, active = vertices of the passes' regions, the
 * candidates connected to the inserted edges or to the last raised vertices);
 * otherwise the HistoCore rounds of the deletions (algo PICO_ALGO_HISTOCORE).
 *
 * pico_dyn_coreness copies the current coreness (n int32) to device memory;
 * pico_dyn_graph exposes the current CSR (device pointers owned by the state,
 * valid until the next update) and pico_dyn_copy_graph copies it out.
 */
#define PICO_STATS_MAINTENANCE 100
typedef struct pico_dyn pico_dyn;
pico_dyn *pico_dyn_create(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t m,
                          int64_t capacity_arcs, pico_stream_t stream);
int pico_dyn_update(pico_dyn *d, const int32_t *ins, int64_t n_ins, const int32_t *del,
                    int64_t n_del, pico_stream_t stream);
int pico_dyn_coreness(pico_dyn *d, int32_t *out_core, pico_stream_t stream);
int pico_dyn_graph(pico_dyn *d, const int64_t **row_ptr, const int32_t **col_idx, int64_t *n,
                   int64_t *m);
/* Copies the current CSR into caller buffers (device memory: n + 1 int64 and
   m int32, sizes from pico_dyn_graph), enqueued on `stream`. */
int pico_dyn_copy_graph(pico_dyn *d, int64_t *row_ptr, int32_t *col_idx, pico_stream_t stream);
void pico_dyn_destroy(pico_dyn *d);

/*
 * Recomputation fallback of pico_dyn_update (no counterpart in the paper).
 * Under PICO_DYN_AUTO (the default) an update recomputes the coreness from
 * scratch (PICO_ALGO_AUTO on the updated graph) instead of maintaining it
 * when the batch's predicted maintenance time exceeds the last full
 * computation's. The prediction scales the device time (measured with
 * events) that the deletion step and the insertion passes took in the last
 * batches that ran them by the ratio of edge counts, and is made only when
 * those batches were within a factor of two of this one in size (otherwise
 * the batch is maintained, and measured); insertion passes that follow
 * deletions add one count of neighbour estimates over all arcs, timed when
 * the state was created. A batch with both deletions and insertions is
 * predicted from the last such batch of a similar size, or else from the two
 * steps' separate times with a 25 % surcharge (its insertion passes search
 * wider regions after the deletions). PICO_DYN_MAINTAIN always
 * maintains, PICO_DYN_RECOMPUTE always recomputes. The result is the same
 * coreness either way. pico_dyn_last_update_kind reports what the last update
 * did (PICO_DYN_MAINTAINED or PICO_DYN_RECOMPUTED; after a recomputation
 * pico_get_stats describes the recomputing call).
 */
#define PICO_DYN_AUTO 0
#define PICO_DYN_MAINTAIN 1
#define PICO_DYN_RECOMPUTE 2
#define PICO_DYN_MAINTAINED 0
#define PICO_DYN_RECOMPUTED 1
int pico_dyn_set_policy(pico_dyn *d, int policy);
int pico_dyn_last_update_kind(pico_dyn *d);

/*
 * Device time (CUDA events, milliseconds) of the last successful
 * pico_dyn_update, split into the CSR rebuild (counts, scans, copies, the
 * batch's arcs) and the coreness step (deletions plus insertion passes, or
 * the recomputation). Both are -1 before the first update; the update has
 * synchronised the stream, so reading them waits for nothing. Returns
 * PICO_ERR_INVALID_ARG on a null argument. (No counterpart in the paper.)
 */
int pico_dyn_last_update_times(pico_dyn *d, double *rebuild_ms, double *coreness_ms);

/*
 * Partitioned HistoCore: Alg. 6 over a graph whose vertices are split into
 * contiguous ranges, each held by one partition (Index2core's fit to a
 * distributed setting, Sec. VI; multi-GPU processing is future work in Sec.
 * VII). A round runs SumHisto in every partition, then every partition
 * receives every partition's change records of the round and pulls the
 * UpdateHisto edits into its own rows; the rounds, the histograms and the
 * result equal those of the single-graph HistoCore. Partitions only meet in
 * the exchange, which the caller performs between calls, so they can live on
 * different devices or processes (the exchange is then an all-gather).
 *
 * pico_part_create sets up the partition of rows [lo, hi) of a graph given by
 * row_ptr (int64, n + 1 entries) and col_idx (device memory, read only; only
 * the partition's rows of col_idx are read), runs InitHisto and lists its
 * initial V_cnt; it synchronises `stream` and returns NULL on invalid
 * arguments (0 <= lo < hi <= n required) or failure. The partition owns its
 * device memory (estimates, histograms, lists, and an n-entry {old, new}
 * array), taken from the stream-ordered allocator on `stream`;
 * pico_part_destroy releases it on that same stream, which must still exist.
 *
 * pico_part_sum runs SumHisto over the partition's V_cnt and reports the
 * number of records of the round (*n_changed; 0 when its V_cnt was empty)
 * and their smallest new estimate (*ymin, INT32_MAX when none). The records
 * are 3 int32 each, (vertex, old estimate, new estimate), at
 * pico_part_records(p) (device memory, valid until the next pico_part_sum);
 * pico_part_copy_records enqueues their copy to dst (device memory, room for
 * 3 * n_changed int32) on `stream`.
 *
 * pico_part_apply takes the round's records of ALL partitions (device
 * memory, 3 * count int32, any order) and the smallest new estimate over all
 * of them, applies the UpdateHisto edits to the partition's rows and lists
 * its next V_cnt (*next_vcnt vertices). The computation is over when a round
 * has no records in any partition. Both calls synchronise `stream` and return
 * PICO_OK, PICO_ERR_INVALID_ARG, PICO_ERR_BAD_GRAPH (a record or a sum that
 * an invalid graph produces) or PICO_ERR_CUDA.
 *
 * pico_part_coreness copies the partition's estimates (hi - lo int32, device
 * memory) to out_core; after the last round they are the coreness.
 *
 * pico_coreness_partitioned runs the whole computation on the current device
 * with `parts` partitions of equal vertex ranges, moving the records between
 * them itself; *rounds (if not NULL) receives the number of rounds. Since
 * every partition can read the whole graph there, a round whose changed
 * vertices hold less than half the arcs divided by the partitions is pushed
 * (the changed vertices walk their arcs; each partition applies the edits on
 * its rows) instead of pulled; the result and the rounds are the same. It
 * synchronises `stream`. row_ptr is int64 (n + 1), col_idx has m entries.
 */
typedef struct pico_part pico_part;
pico_part *pico_part_create(const int64_t *row_ptr, const int32_t *col_idx, int64_t n, int64_t lo,
                            int64_t hi, pico_stream_t stream);
int pico_part_sum(pico_part *p, int64_t *n_changed, int32_t *ymin, pico_stream_t stream);
const int32_t *pico_part_records(pico_part *p);
int pico_part_copy_records(pico_part *p, int32_t *dst, pico_stream_t stream);
int pico_part_apply(pico_part *p, const int32_t *records, int64_t count, int32_t ymin,
                    int64_t *next_vcnt, pico_stream_t stream);
int pico_part_coreness(pico_part *p, int32_t *out_core, pico_stream_t stream);
void pico_part_destroy(pico_part *p);
int pico_coreness_partitioned(const int64_t *row_ptr, const int32_t *col_idx, int64_t n,
                              int64_t m, int32_t *out_core, int32_t parts, int64_t *rounds,
                              pico_stream_t stream);

/* Direction of HistoCore's UpdateHisto (Sec. IV-B, Alg. 6). */
#define PICO_UPDATE_AUTO 0   /* per round: pull when the round's changed vertices hold at
                                least pull_pct % of the arcs of a graph with >= 2^22 arcs */
#define PICO_UPDATE_PUSH 1   /* always push from the changed vertices (the paper's form) */
#define PICO_UPDATE_PULL 2   /* always pull (every round, every graph size) */

/*
 * Sets the UpdateHisto direction of later HistoCore calls on the current
 * device (no counterpart in the paper, which pushes). Pushing, each changed
 * vertex edits the histogram rows of its neighbours; pulling, every vertex
 * whose estimate an edit can reach walks its own adjacency and applies the
 * edits of its changed neighbours to its own row. Both apply the same edits
 * and give the same results and rounds; pulling scans more arcs but edits
 * one row at a time, which keeps the edits in L2 when the rows a round
 * touches exceed it. mode: PICO_UPDATE_*; pull_pct: 1..100, the auto-mode
 * threshold (default 50). Returns PICO_ERR_INVALID_ARG for other values.
 */
int pico_set_histo_update(int mode, int pull_pct);
int pico_get_histo_update(int *mode, int *pull_pct);

/* Library version, as major * 10000 + minor * 100 + patch. */
int pico_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PICO_H */
