/*
 * kcore.h -- C ABI of the GB300 k-core decomposition library.
 *
 * The library computes the coreness of every vertex of an undirected graph
 * (Def. 1, Sec. II: core(v) is the largest k such that v belongs to the
 * k-core, the inclusion-maximal vertex set inducing minimum degree >= k).
 * It does so with the local iteration of Alg. 1 (Montresor et al.) as adapted
 * to shared memory in Sec. IV (FastK): every estimate starts at the vertex's
 * degree and is repeatedly lowered to the capped h-index of its neighbours'
 * estimates; a vertex is re-evaluated only when a neighbour's new estimate
 * falls below its own (selective sending, Sec. III-B).  Estimates never
 * increase (the monotonicity the paper cites for dropping messages, Sec.
 * III-B), which makes in-place asynchronous updates sound; the fixed point
 * reached from the degrees is the coreness (Sec. III, convergence argument).
 * All work runs in sm_103a CUDA kernels; there is no CPU fallback.
 *
 * Conventions
 *   - Vertex ids are int32 in [0, n), n < 2^31; degrees must be < 2^30.
 *   - Return values are kcore_status: KCORE_OK (0), KCORE_PENDING (1) or a
 *     negative error.  No C++ exception crosses this boundary.  After an
 *     error, kcore_last_error() returns a message for the calling thread.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is ordered on that stream.
 *   - Pointers are host pointers unless a flag says device.  The caller keeps
 *     ownership of every array it passes; handles are owned by the library and
 *     released with the matching destroy call.
 *   - Functions taking a handle are not thread-safe on the same handle.
 */
#ifndef KCORE_H
#define KCORE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t kcore_status;

#define KCORE_OK                 0
#define KCORE_PENDING            1   /* kcore_poll: result not ready yet            */
#define KCORE_ERR_INVALID       -1   /* bad argument or malformed graph              */
#define KCORE_ERR_OOM           -2   /* device or host allocation failed             */
#define KCORE_ERR_CUDA          -3   /* a CUDA runtime call failed                   */
#define KCORE_ERR_NOT_CONVERGED -4   /* sweep cap reached with vertices still active */
#define KCORE_ERR_TIMEOUT       -5   /* a bounded device wait or a poll timed out    */
#define KCORE_ERR_AGAIN         -6   /* admission refused: queue full / over budget  */
#define KCORE_ERR_CANCELLED     -7   /* request was cancelled                        */

/* ---- flags -------------------------------------------------------------- */
#define KCORE_IN_DEVICE   (1u << 0)  /* input arrays are device pointers                 */
#define KCORE_IN_CLEAN    (1u << 1)  /* input CSR is already symmetric, loop-free,
                                        sorted ascending per row, without repeats     */
#define KCORE_OUT_DEVICE  (1u << 2)  /* coreness_out is a device pointer                 */
#define KCORE_SYNC_MODE   (1u << 3)  /* synchronous rounds (Alg. 3): every round reads a
                                        snapshot of the estimates; deterministic per
                                        round.  Default: in-place asynchronous sweeps */
#define KCORE_REFINED     (1u << 4)  /* synchronous mode: refined activation (Sec. IV,
                                        Further Optimizations): u re-activates v only
                                        if new_u < est(v) <= old_u.  Asynchronous
                                        mode uses it by default (see KCORE_SIMPLE)    */
#define KCORE_ASYNC       (1u << 5)  /* kcore_run returns once the work is enqueued;
                                        kcore_wait() reports the status               */
#define KCORE_GRAPH       (1u << 6)  /* kcore_run: capture the run (initialisation, the
                                        persistent sweep launch, output) into a CUDA
                                        graph on first use and replay it afterwards;
                                        needs KCORE_OUT_DEVICE.  Re-captured when the
                                        output pointer, mode flags or options change  */
#define KCORE_SIMPLE      (1u << 7)  /* asynchronous mode: the simple activation rule
                                        of Sec. III-B (v re-activated whenever
                                        new_u < est(v)).  Without it, asynchronous
                                        sweeps use the refined rule, kept exact under
                                        in-place updates: while v may still be
                                        evaluating in the same sweep, the simple rule
                                        applies to it; once v is done, its final
                                        estimate decides new_u < est(v) <= old_u.
                                        Both give the coreness; they differ in the
                                        work done                                      */

/* ---- options ------------------------------------------------------------ */
/*
 * Tuning knobs of the sweep engine.  Fill with kcore_default_options() and
 * override fields; 0 in a field means "library default".  The degree tiers
 * split the frontier by degree d: d <= t_lo is evaluated by one thread with a
 * register histogram, t_lo < d <= t_hi by one warp (estimates in registers up
 * to degree 128, staged in shared memory above), d > t_hi by one CTA with
 * shared-memory counters.
 */
typedef struct kcore_options {
    uint32_t struct_size;   /* sizeof(kcore_options)                                */
    int32_t  t_lo;          /* thread-tier degree bound, 1..16 (default 16)          */
    int32_t  t_hi;          /* warp-tier degree bound, t_lo..2048 (default 2048)     */
    int32_t  block;         /* threads per CTA of the sweep kernel, 64..512, x32     */
    int32_t  low_chunk;     /* thread tier: vertices per lane per work grab (1..8)   */
    int32_t  med_chunk;     /* warp tier: vertices per warp per work grab (1..64)    */
    int32_t  tail_max;      /* frontier size at or below which one CTA continues,
                               if it holds no vertex above t_hi and at most 16
                               above t_lo (default 1024; negative disables)      */
    int32_t  ctas_per_sm;   /* persistent CTAs per SM (0 = occupancy maximum)        */
    int32_t  max_ctas;      /* cap on the persistent grid (0 = no cap)               */
    int64_t  max_sweeps;    /* sweep cap (0 = 2m + n + 1, a hard bound: every
                               productive sweep lowers the sum of estimates)       */
    double   timeout_s;     /* budget of every bounded device wait (default 20 s)   */
    int32_t  build_sort;    /* cleaning of raw edge samples (kcore_create_coo and
                               batches): 1 = radix sorts of the samples'
                               canonical (min, max) keys and of the distinct
                               edges' transposes;
                               -1 = rows counted, filled and sorted one by one;
                               0 (default) = the sort when the input has at least
                               2^18 samples, 2*samples >= 8n, and rows of more
                               than 32 entries hold half of the entries or more
                               (estimated from every 16th run of 256 samples).
                               The cleaned graph is the same either way.          */
    int32_t  relabel;       /* vertex numbering of a graph built from edge samples
                               (kcore_create_coo): 1 = renumbered by descending
                               degree, 2 = by ascending degree, -1 = the input's
                               numbering, 0 (default) = descending degree when
                               the sample-based cleaner is chosen automatically
                               for hub-dominated inputs (see build_sort), else
                               the input's.  Renumbering packs the estimates of
                               high-degree vertices into few cache lines and
                               lists them together in every row; the cleaner
                               renumbers while it sorts (it takes the sorted
                               build).  Internal: coreness, warm starts and
                               kcore_copy_csr use the caller's ids (the copy of
                               a renumbered graph is rebuilt on the device, at
                               about the cost of a create).  Fixed at creation:
                               kcore_set_options does not change it.  Ignored by
                               kcore_create and by batches.                      */
} kcore_options;

/* Fill `opt` with the defaults. */
void kcore_default_options(kcore_options* opt);

/* ---- single graph ------------------------------------------------------- */
typedef struct kcore_graph kcore_graph;   /* opaque, library-owned */

/*
 * kcore_create -- build a device graph from a CSR.
 *   n             number of vertices (0 <= n < 2^31).
 *   row_ptr       n+1 offsets, int32 or int64 per `row_ptr_bytes` (4 or 8);
 *                 row_ptr[0] == 0, non-decreasing.  Row u lists the neighbours
 *                 col_idx[row_ptr[u] .. row_ptr[u+1]).
 *   col_idx       row_ptr[n] int32 vertex ids in [0, n).
 *   flags         KCORE_IN_DEVICE (inputs are device pointers),
 *                 KCORE_IN_CLEAN (skip cleaning; rows are checked to be strictly
 *                 increasing and loop-free, symmetry is the caller's promise).
 *   opt           NULL for defaults; copied.
 * Without KCORE_IN_CLEAN the input may be directed, repeated or contain
 * self-loops: the graph is cleaned on the device (Sec. IV-A: treated as
 * undirected, self-loops removed; Sec. III-B: rows kept as sorted vectors):
 * both directions of every pair, loops dropped, rows sorted, repeats removed.
 * The cleaned CSR keeps the input's row_ptr width.  The call returns after the
 * graph is built (it synchronises `cuda_stream`); the caller may free its
 * arrays on return.  Errors: ERR_INVALID (n, width, offsets or ids out of
 * range), ERR_OOM, ERR_CUDA.  *out is NULL on error.
 */
kcore_status kcore_create(int64_t n, const void* row_ptr, int32_t row_ptr_bytes,
                          const int32_t* col_idx, uint32_t flags,
                          const kcore_options* opt, void* cuda_stream, kcore_graph** out);

/*
 * kcore_create_coo -- build a device graph from raw edge samples.
 *   n             number of vertices; nnz samples src[i] -> dst[i] (int32, in
 *                 [0, n)), host or device per KCORE_IN_DEVICE.
 *   row_ptr_bytes width of the cleaned CSR's row_ptr: 4 (needs 2m < 2^31) or 8.
 * Every sample is an undirected edge; loops and repeats are removed as in
 * kcore_create.  Other arguments, ownership and errors as kcore_create.
 */
kcore_status kcore_create_coo(int64_t n, int64_t nnz, const int32_t* src, const int32_t* dst,
                              int32_t row_ptr_bytes, uint32_t flags, const kcore_options* opt,
                              void* cuda_stream, kcore_graph** out);

/*
 * kcore_run -- compute the coreness of every vertex.
 *   coreness_out  n int32 values, caller-owned; a host pointer, or a device
 *                 pointer with KCORE_OUT_DEVICE.
 *   flags         KCORE_OUT_DEVICE, KCORE_SYNC_MODE, KCORE_REFINED, KCORE_SIMPLE,
 *                 KCORE_ASYNC, KCORE_GRAPH.
 * Each run starts from est = degree (Alg. 1 initialisation) and iterates on the
 * device until no vertex is active; one persistent kernel runs every sweep.
 * Without KCORE_ASYNC the call waits for the result and returns its status;
 * with it, the call returns KCORE_OK once the work is enqueued on
 * `cuda_stream` and kcore_wait() returns the run's status.
 * Errors: ERR_INVALID (NULL arguments), ERR_NOT_CONVERGED (sweep cap hit; coreness_out then holds the current
 * estimates, an upper bound of the coreness), ERR_TIMEOUT (a bounded device
 * wait gave up), ERR_CUDA.
 */
kcore_status kcore_run(kcore_graph* g, int32_t* coreness_out, uint32_t flags, void* cuda_stream);

/*
 * kcore_set_options -- replace the graph's options (NULL = defaults).  A change
 * of t_lo/t_hi re-splits the vertices into tiers on `cuda_stream` (synchronous).
 * Errors: ERR_INVALID, ERR_CUDA.
 */
kcore_status kcore_set_options(kcore_graph* g, const kcore_options* opt, void* cuda_stream);

/* Wait for the last kcore_run on `g` and return its status. */
kcore_status kcore_wait(kcore_graph* g);

/* Sizes of the cleaned graph: vertices, directed CSR entries (2m), row_ptr width. */
kcore_status kcore_graph_info(const kcore_graph* g, int64_t* n, int64_t* nnz,
                              int32_t* row_ptr_bytes);

/*
 * kcore_copy_csr -- copy the cleaned CSR out (row_ptr in the graph's width,
 * n+1 entries; col_idx nnz entries), to host buffers, or device buffers with
 * KCORE_OUT_DEVICE.  Synchronous.
 */
kcore_status kcore_copy_csr(const kcore_graph* g, void* row_ptr_out, int32_t* col_idx_out,
                            uint32_t flags);

/*
 * Statistics of the last run (synchronises with it).  Per-sweep counts follow
 * Fig. 5 (activated vertices per iteration); bytes_algorithmic is what the
 * method must move for the vertices it evaluated: per evaluated vertex u,
 * 2 row_ptr entries + est[u], then one col_idx entry and one estimate gather
 * per adjacency entry read (entries_read: deg(u), or fewer when the
 * no-change test of a high-degree vertex found est[u] supporters early),
 * plus 4 bytes per update, plus the initialisation and output of the run
 * (estimates from the degrees, three frontier bitmaps, coreness written out:
 * 16 bytes per vertex and 12 bytes per 32 vertices).
 */
typedef struct kcore_run_stats {
    int64_t n, nnz;             /* graph size (nnz = 2m)                              */
    int64_t sweeps;             /* sweeps executed                                     */
    int64_t tail_sweeps;        /* of which run by a single CTA                         */
    int64_t evaluated;          /* sum over sweeps of the frontier size                */
    int64_t edges_scanned;      /* sum over sweeps of the frontier's degrees           */
    int64_t updates;            /* estimate decreases written                          */
    int64_t pushes;             /* vertices added to a next frontier                   */
    int64_t bytes_algorithmic;  /* see above                                           */
    int32_t status;             /* status of the run                                   */
    int32_t grid;               /* persistent CTAs launched                            */
    int32_t block;              /* threads per CTA                                     */
    int32_t row_ptr_bytes;
    float   ms_create;          /* kcore_create device time (cleaning)                 */
    float   ms_sweep;           /* sweep kernel device time                            */
    float   ms_run;             /* whole kcore_run device time (init..output)          */
    int64_t entries_read;       /* adjacency entries read to evaluate (<= edges_scanned) */
    int64_t decrease;           /* sum over updates of (old - new) estimate              */
} kcore_run_stats;

kcore_status kcore_stats(kcore_graph* g, kcore_run_stats* out);

/*
 * Per-sweep trace of the last run: frontier size, frontier degree sum,
 * updates, and the sweep's start time in ns after the first sweep's start
 * (device globaltimer), for sweeps [0, min(cap, recorded)); *count gets the
 * number written.  Any output pointer may be NULL.
 */
kcore_status kcore_sweep_trace(kcore_graph* g, int64_t* frontier, int64_t* degsum,
                               int64_t* updates, int64_t* start_ns, int64_t cap, int64_t* count);

/*
 * Further per-sweep columns of the same trace: adjacency entries read to
 * evaluate the frontier (below its degree sum where the no-change test stopped
 * early) and the sum of the estimate decreases made in the sweep.  Estimates
 * start at the degree and never go below the coreness, so after sweep s
 *   sum_v |est_v - core_v| = sum_v deg_v - sum_{s' <= s} decrease[s'] - sum_v core_v,
 * the convergence error of Fig. 4, without copying estimates out.
 * Same conventions as kcore_sweep_trace.
 */
kcore_status kcore_sweep_detail(kcore_graph* g, int64_t* entries_read, int64_t* decrease,
                                int64_t cap, int64_t* count);

/*
 * Per-tier columns of the same trace: for sweep s, frontier[3 s + q] is the
 * number of vertices of degree tier q (0: degree <= t_lo, one thread each;
 * 1: <= t_hi, one warp each; 2: above, one CTA each) in the sweep's frontier
 * and degsum[3 s + q] their degree sum.  Arrays hold 3 * cap values; either may
 * be NULL.  Same conventions as kcore_sweep_trace.
 */
kcore_status kcore_sweep_tiers(kcore_graph* g, int64_t* frontier, int64_t* degsum, int64_t cap,
                               int64_t* count);

/*
 * kcore_run_from -- the iteration started from caller-given upper bounds
 * instead of the degrees: dynamic core maintenance (Sec. VI names it as future
 * work; this is its local-iteration form).  The fixed point reached from any
 * pointwise upper bound of the coreness is the coreness (the operator is
 * monotone and the coreness is its largest fixed point, Sec. III), so:
 *   - after deleting edges (coreness can only drop): create the new graph and
 *     pass the old coreness as `start` with the deleted edges' endpoints as
 *     the frontier;
 *   - after inserting b edges (each raises a coreness by at most 1): pass
 *     old coreness + b as `start` and frontier = NULL (every vertex active).
 *   start       n int32, start[v] >= core(v) required (not checked: a start
 *               below the coreness gives a wrong result); values above the
 *               degree are lowered to it, and such a vertex and its neighbours
 *               join the frontier; negative values count as 0.
 *   frontier    nfrontier vertex ids active at the start (repeats allowed), or
 *               NULL for every vertex.  A vertex left out must satisfy
 *               start[v] <= h-index of its neighbours' starts (true for the
 *               old coreness where the neighbourhood did not change).  An id
 *               out of [0, n) gives KCORE_ERR_INVALID.
 *   flags       KCORE_IN_DEVICE (start and frontier are device pointers, read
 *               on cuda_stream), KCORE_OUT_DEVICE, KCORE_SYNC_MODE,
 *               KCORE_REFINED, KCORE_SIMPLE, KCORE_ASYNC as in kcore_run;
 *               KCORE_GRAPH is refused (ERR_INVALID).
 * Statistics and traces of the run are read as for kcore_run.
 */
kcore_status kcore_run_from(kcore_graph* g, const int32_t* start, const int32_t* frontier,
                            int64_t nfrontier, int32_t* coreness_out, uint32_t flags,
                            void* cuda_stream);

/* Release a graph (waits for its outstanding work).  NULL is ignored. */
void kcore_destroy(kcore_graph* g);

/*
 * kcore_run_noalloc -- coreness of a clean device CSR without allocating any
 * memory.  (The paper has no counterpart: this serves callers, not the method.)
 *
 * For callers that cannot allocate device memory while they call us: a
 * serving process that reserved the whole device for its own pool up front,
 * a real-time loop that must not stall on the allocator's implicit
 * synchronisation, code running inside another allocator's callback.  The
 * working memory is one fixed array compiled into the library, sized for
 * KCORE_NOALLOC_MAX_N vertices (about 19 MB); the estimates live in
 * coreness_out.  No call allocates: no cudaMalloc, cudaFree or allocating
 * library call.
 *
 * Where the array comes from: the CUDA runtime loads the library's device
 * code lazily by default (CUDA_MODULE_LOADING=LAZY since CUDA 12.2), so the
 * array, and the kernels this entry point launches, are loaded on a device
 * the first time they are used there, and stay until the process exits.  A
 * call with n = 0 does only that loading (the pointers may then be NULL):
 * make it once per device, with that device current, before reserving the
 * rest of the device memory; later calls then allocate nothing at all.  If
 * the device has no room left for them, that first call returns ERR_OOM.
 *
 *   n             0 <= n <= KCORE_NOALLOC_MAX_N; larger n gives ERR_INVALID.
 *   row_ptr       DEVICE pointer, n+1 offsets, int32 or int64 per
 *                 row_ptr_bytes (4 or 8), of a clean CSR: symmetric, rows
 *                 strictly increasing, no self-loops (the KCORE_IN_CLEAN form).
 *   col_idx       DEVICE pointer, row_ptr[n] int32 vertex ids.
 *   coreness_out  DEVICE pointer, n int32, caller-owned; it also holds the
 *                 estimates while the call runs.
 * The call is synchronous: it reads row_ptr[n] back and waits for the run
 * on `cuda_stream` before it returns, so it must not be called while that
 * stream is being captured into a CUDA graph.  Returns the run's status:
 * ERR_INVALID for offsets or entries that are not a clean CSR (ids outside
 * [0, n), a self-loop, a row not strictly increasing: checked on the device
 * before the first sweep), otherwise as kcore_run.
 * Every call shares the one array and finds the previous call's contents in
 * it; each call clears what must start at zero.  Calls that overlap on the GPU
 * (on two streams, or from two threads) race on the array: serialise them.
 */
#define KCORE_NOALLOC_MAX_N (1 << 19)
kcore_status kcore_run_noalloc(int64_t n, const void* row_ptr, int32_t row_ptr_bytes,
                               const int32_t* col_idx, int32_t* coreness_out, void* cuda_stream);

/* ---- batching and serving ------------------------------------------------ */
/*
 * A batch engine packs many graphs into one device arena and runs them
 * together in persistent sweep launches (continuous batching): graphs that
 * arrive while others are running are admitted, within the memory budget and
 * slot limit, at the next sweep-chunk boundary; finished graphs leave and free
 * their space.  The coreness is unique, so each graph's result is the same
 * alone or in any mix.
 */
typedef struct kcore_batch kcore_batch;   /* opaque, library-owned */

typedef struct kcore_serve_options {
    uint32_t struct_size;     /* sizeof(kcore_serve_options)                          */
    int64_t  mem_budget;      /* device bytes for the arena (0 = 4 GiB)               */
    int32_t  max_slots;       /* graphs resident at once (0 = 4096)                   */
    int32_t  max_queue;       /* queued, not yet admitted requests (0 = 1 << 20)      */
    int32_t  chunk_sweeps;    /* sweeps per persistent launch (0 = 16)               */
    int32_t  start_thread;    /* 1 = run the serving loop in a library thread;
                                 0 = caller drives it with kcore_batch_step           */
    kcore_options sweep;      /* sweep engine knobs (struct_size 0 = defaults)        */
    int64_t  host_staging;    /* page-locked host bytes holding queued graphs' samples
                                 and finished graphs' results, so that uploads and
                                 result copies run asynchronously (0 = 1 GiB; < 0 =
                                 none).  A graph that finds no room uses pageable
                                 memory; results are the same either way.          */
} kcore_serve_options;

void kcore_default_serve_options(kcore_serve_options* opt);

/* Create an engine; its CUDA stream is private.  Errors: ERR_INVALID, ERR_OOM, ERR_CUDA. */
kcore_status kcore_batch_create(const kcore_serve_options* opt, kcore_batch** out);

/*
 * Queue one graph (raw CSR as in kcore_create, HOST arrays only, copied before
 * return) and get a ticket.  Errors: ERR_INVALID; ERR_AGAIN when the queue is
 * full or the graph can never fit the budget.
 */
kcore_status kcore_submit(kcore_batch* b, int64_t n, const void* row_ptr, int32_t row_ptr_bytes,
                          const int32_t* col_idx, uint32_t flags, uint64_t* ticket);

/* Same, from raw edge samples (host arrays). */
kcore_status kcore_submit_coo(kcore_batch* b, int64_t n, int64_t nnz, const int32_t* src,
                              const int32_t* dst, uint32_t flags, uint64_t* ticket);

/*
 * Wait up to timeout_us (0 = do not wait, < 0 = forever) for a ticket.  On
 * KCORE_OK, n int32 coreness values are copied to the host buffer
 * coreness_out (may be NULL to discard) and the ticket is released.  Returns
 * KCORE_PENDING if not finished in time, ERR_CANCELLED, ERR_INVALID (unknown
 * ticket), or the request's own error.
 */
kcore_status kcore_poll(kcore_batch* b, uint64_t ticket, int32_t* coreness_out, int64_t timeout_us);

/*
 * Timing and placement of one request, for latency measurement and for
 * checking that the engine overlaps work (continuous batching).  Times are
 * seconds of the monotonic clock (CLOCK_MONOTONIC; the clock of
 * std::chrono::steady_clock and of Python's time.perf_counter on Linux).
 * Launch numbers count the engine's persistent sweep launches from 0: the
 * request took part in launches [admit_launch, retire_launch).
 */
typedef struct kcore_ticket_info {
    double  submit_s;        /* kcore_submit* accepted it (after copying)         */
    double  admit_s;         /* placed into the arena                            */
    double  done_s;          /* result ready (retired, cancelled or failed)      */
    int64_t admit_launch;    /* first persistent launch it took part in          */
    int64_t retire_launch;   /* launches run when it was retired                 */
    int64_t resident_at_admit;  /* other graphs resident when it was placed      */
} kcore_ticket_info;

/*
 * kcore_poll with the request's timing and placement: as kcore_poll, and on
 * any return other than KCORE_PENDING (the ticket is then released), *info
 * (may be NULL) gets the request's kcore_ticket_info.
 */
kcore_status kcore_poll_info(kcore_batch* b, uint64_t ticket, int32_t* coreness_out,
                             int64_t timeout_us, kcore_ticket_info* info);

/* Cancel a queued or running request; its slot is freed at the next chunk. */
kcore_status kcore_cancel(kcore_batch* b, uint64_t ticket);

/*
 * Drive the engine once (admit, one chunk of sweeps, retire) when it was
 * created with start_thread = 0.  *active gets the number of graphs resident
 * or queued afterwards.  An admission that fails before its graphs are placed
 * (device memory, upload, cleaning) fails only those graphs (their tickets
 * report the error; their memory is given back) and the step goes on with the
 * resident graphs; an error of the sweep launch or of placement fails every
 * resident graph and is returned here.
 */
kcore_status kcore_batch_step(kcore_batch* b, int64_t* active);

typedef struct kcore_batch_stats {
    int64_t submitted, completed, cancelled, failed;
    int64_t queued, resident;        /* right now                                      */
    int64_t launches, sweeps;        /* persistent launches and sweeps run             */
    int64_t arena_bytes, arena_used_peak;
    double  latency_p50_ms, latency_p99_ms;   /* submit -> result ready, completed ones */
    double  busy_s;                  /* wall time the engine spent with work resident  */
    double  admit_s, sweep_s, retire_s;  /* busy_s split by phase: admission (union
                                            build, cleaning, placement), sweep
                                            launches, retirement (result copies) */
    int64_t admissions;              /* admission batches placed into the arena        */
    int64_t admitted_while_busy;     /* graphs placed while other graphs were resident
                                        and unfinished (continuous batching)           */
} kcore_batch_stats;

kcore_status kcore_batch_stats_get(kcore_batch* b, kcore_batch_stats* out);

/* Stop the engine (cancels what is left) and release it.  NULL is ignored. */
void kcore_batch_destroy(kcore_batch* b);

/* ---- misc ----------------------------------------------------------------- */
/* Message of the last error on the calling thread ("" if none). */
const char* kcore_last_error(void);

/* Library version string. */
const char* kcore_version(void);

/* Number of CUDA kernels this library has launched in this process. */
int64_t kcore_kernel_launches(void);

/*
 * Device memory freed by the library stays cached in its per-device memory
 * pool for reuse by later graphs; this returns the cached blocks to the driver.
 */
void kcore_release_cached_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* KCORE_H */
