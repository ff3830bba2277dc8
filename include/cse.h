/*
 * cse.h -- C ABI of the GB300 library for parallel heuristic common
 * subexpression elimination (CSE) on ternary linear forms.
 *
 * Method: "Parallel Heuristic Exploration for Additive Complexity Reduction
 * in Fast Matrix Multiplication" (A. I. Perminov, arXiv 2512.13365).
 *   - an expression set E is a ternary matrix: one row per expression e_i,
 *     one column per variable x_j, entries alpha_ij in {-1, 0, 1}
 *     (Section 3.2.1); a fast-matmul scheme (m,n,p:r) gives three such sets,
 *     E_U = U (r x mn), E_V = V (r x np) and E_W = W^T (mp x r) (Section 3.2);
 *   - A_naive(E) = sum_i (nnz_i - 1); Cost(E) = n_f + A_naive(E_final)
 *     (Section 3.2.1);
 *   - each of n_processes independent processes per matrix repeats
 *     Algorithm 1: count canonical signed pairs (x_i + s x_j, i < j), select a
 *     pair with c > 1 by its strategy (g, ga, wr, gr, gi, mix, gp; Sections
 *     2.2 and 3.4), introduce x_k = x_i + s x_j and rewrite every row
 *     containing the pair;
 *   - processes share their best substitution prefixes (Section 3.5.2).
 *
 * All arithmetic is exact integer and every random draw is a Philox4x32-10
 * value keyed by (seed, process, step, matrix, purpose), so a search's
 * result is a pure function of (matrices, strategy mix, n_processes, seed,
 * step_budget and the options that change results): it does not depend on
 * launch configuration or on other searches running at the same time.
 *
 * Conventions
 *   - Matrices are int8, row-major, rows = expressions, cols = variables.
 *   - Variables are 0-based; fresh variable t (0-based) is x_{cols + t}.
 *   - A substitution entry is packed as  i | j << 10 | (s < 0) << 20  with
 *     i < j: it defines x_{cols+t} = x_i + s * x_j.
 *   - Every function returns CSE_OK (0) or an error code; on error
 *     cse_last_error() returns a message for the calling thread.
 *   - Handles are owned by the library until the matching *_free call.
 *     Functions copy their host inputs; output buffers belong to the caller.
 *   - There is no CPU fallback: without a CUDA device, calls that need one
 *     return CSE_ECUDA.
 */
#ifndef CSE_GB300_H
#define CSE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CSE_OK = 0,
    CSE_EINVAL = 1,   /* invalid argument (non-ternary entry, zero row, sizes) */
    CSE_ENOMEM = 2,   /* host or device allocation failed                      */
    CSE_ECUDA = 3,    /* CUDA runtime error (including: no device)             */
    CSE_ETIMEOUT = 4, /* a bounded wait expired                                */
    CSE_EBUSY = 5,    /* server admission refused (no room), non-blocking      */
    CSE_ESTATE = 6,   /* internal consistency check failed on the device       */
    CSE_ECANCELED = 7 /* the request was cancelled (cse_server_cancel)         */
};

/* Limits of this implementation. */
#define CSE_MAX_ROWS 256   /* rows (expressions) per matrix                    */
#define CSE_MAX_COLS 512   /* column capacity: original plus fresh variables   */
#define CSE_MAX_MATS 16    /* matrices per scheme                              */

typedef struct cse_scheme cse_scheme;
typedef struct cse_result cse_result;
typedef struct cse_server cse_server;

/* Integer strategy weights (Section 3.5.1): the paper's gi 8, ga 4, gr 2,
 * wr 1, mix 0.1, gp 0.01 become 800, 400, 200, 100, 10 and 1 here.  w_g is
 * Greedy (the paper gives it weight 0 apart from process 0's first run).
 * w_gp is Greedy-Potential (Section 2.2): every candidate is scored by a trial
 * substitution, (c - 1) 2^16 + a N with N the number of pairs that then occur
 * at least twice and a the run's alpha in units of 2^-16.  A run draws its
 * strategy from the weights in the order gi, ga, gr, wr, mix, g, gp.  At least
 * one weight must be nonzero; the sum must fit in 32 bits. */
typedef struct {
    uint32_t w_gi, w_ga, w_gr, w_wr, w_mix, w_g, w_gp;
} cse_strategy_mix;

/* Option flags. */
#define CSE_FLAG_GRAPH 1u  /* capture the whole launch sequence in one CUDA graph
                              and launch it once; the round kernels of different
                              matrix classes become parallel graph branches */
#define CSE_FLAG_TRACE 2u  /* record each process's trajectory hash (see
                              cse_proc_record); costs a few per cent */
#define CSE_FLAG_GI_SHARED_COINS 4u  /* changes results: Greedy-Intersections
                              draws one coin per candidate per step, seen by
                              every candidate it intersects, instead of one
                              coin per (scored, intersecting) pair; the paper
                              (Section 3.4.2) fixes only each coin's 1/2
                              marginal.  Scoring then costs O(m + columns) per
                              step through per-variable sums. */
#define CSE_FLAG_PERSISTENT 16u  /* cse_search_batch: the whole batch (every
                              round and sharing boundary of every search) as
                              one persistent cooperative kernel, with a grid
                              barrier between the steps and the boundaries;
                              with CSE_FLAG_GRAPH that one launch is captured
                              in a CUDA graph.  For the step clock, without
                              shared coins, every matrix at most 64 rows and
                              on the shared-memory engine (else CSE_EINVAL).
                              A barrier gives up after max_spin polls
                              (0 = 2^26, about 7 s) and the search reports
                              CSE_ETIMEOUT; results are those of the
                              searches run alone */
#define CSE_FLAG_WARP_ENGINE 8u  /* large matrices (those whose process state
                              does not fit a warp's shared-memory slice) run
                              on the one-warp-per-process engine only: the
                              default; the flag overrides CSE_FLAG_CTA_ENGINE */
#define CSE_FLAG_CTA_ENGINE 64u  /* large matrices run one process per CTA with
                              its arrays in shared memory for run starts and
                              for lists of at least cta_min_list candidates
                              at a round start, the rest on the
                              one-warp-per-process engine; results are
                              identical (on the (6,6,6:153) search the warp
                              engine alone is faster, hence the default) */
#define CSE_FLAG_WIDE_WORDS 32u  /* every matrix runs on the kernel of the next
                              power-of-two words per column (3 -> 4, 5..7 -> 8;
                              the extra row bits are zero), where its process
                              slice still fits the same memory path;
                              results, op counts included, are identical.
                              Without the flag a width cse_autotune chose for
                              the matrix's class applies */

/* Search options.  Fields that change results: share_interval,
 * share_permille, col_cap, patience_rounds and the flag
 * CSE_FLAG_GI_SHARED_COINS.  The rest only change how the work is launched.
 *
 * share_interval >= 1 selects the step clock: every process makes one step
 * per global step, and sharing happens every share_interval steps.
 * share_interval = 0 selects iteration mode, the paper's own schedule
 * (Sections 3.5.2 and 4): in each iteration every process performs one whole
 * run, from its start until no pair repeats (or the columns are used up);
 * sharing happens between iterations; step_budget is then the maximum number
 * of iterations, and the search stops earlier once the sum over the matrices
 * of the best Cost has not decreased for patience_rounds consecutive
 * iterations (the paper: 10; 0 = never early).  The draws of the steps of
 * iteration i use the step numbers i * col_cap, i * col_cap + 1, ... */
typedef struct {
    uint32_t share_interval;  /* steps between sharing boundaries; 0 =
                                 iteration mode                               */
    uint32_t share_permille;  /* share probability at a run start, 0..1000
                                 (paper default 40%: 400)                     */
    uint32_t col_cap;         /* column capacity, cols < col_cap <= 512       */
    uint32_t patience_rounds; /* iteration mode: iterations without
                                 improvement that end the search; must be 0
                                 with the step clock                          */
    uint64_t max_spin;        /* CSE_FLAG_PERSISTENT: polls of a grid barrier
                                 before it gives up (0 = 2^26)               */
    uint32_t procs_per_cta;   /* processes (warps) per CTA; 0 = automatic    */
    uint32_t flags;           /* CSE_FLAG_* bits; other bits must be 0       */
    uint32_t cta_list_cap;    /* launch parameter of large matrices: the
                                 candidate capacity of the process-per-CTA
                                 engine's shared-memory list, 0 = automatic
                                 (at most 6144); a process whose list
                                 outgrows it finishes that round on the
                                 one-warp-per-process engine.  Never changes
                                 results.                                     */
    uint32_t cta_min_list;    /* launch parameter of large matrices: a process
                                 whose run is under way with fewer candidates
                                 than this at a round start runs that round
                                 on the one-warp-per-process engine (one warp
                                 serves a short list better than a CTA);
                                 0 = automatic (2048).  Never changes
                                 results.                                     */
} cse_opts;

/* Default options: share_interval 32, share_permille 400, col_cap 128. */
void cse_opts_default(cse_opts* opts);

/* Loads n_mats expression sets.  mats[k] points to rows[k] x cols[k] int8
 * entries (row-major) in host memory; every entry must be -1, 0 or 1 and
 * every row must have at least one nonzero (A_naive counts nnz - 1 per row,
 * Section 3.2.1).  1 <= rows <= 256, 1 <= cols < 512, n_mats <= 16.  The data
 * is copied to the device (synchronously) and packed there into column
 * bitsets.  A matrix with more than 32767 initial repeated signed pairs
 * (candidates) is refused with CSE_EINVAL after the packing: the candidate
 * lists hold at most that many.  On success *out owns the device copy. */
int cse_scheme_load(const int8_t* const* mats, const int32_t* rows, const int32_t* cols,
                    int32_t n_mats, cse_scheme** out);

/* Loads a scheme (m,n,p:r) from its coefficient tensors (Section 3.1):
 * U is r x (m*n), V is r x (n*p), W is r x (m*p), each row-major with the
 * matrix entries in row-major order.  The three sets are E_U = U, E_V = V and
 * E_W = W^T (Section 3.2).  The Brent equations are not checked here (see
 * cse_brent_check): the synthetic stand-ins of real schemes do not satisfy
 * them, and the elimination does not need them. */
int cse_scheme_load_uvw(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U,
                        const int8_t* V, const int8_t* W, cse_scheme** out);

/* Checks the Brent equations of a scheme (m,n,p:r) (Section 3.1) on the
 * device: for every entry a_ij, b_j'k, c_i'k' the sum over the r products of
 * u_ij v_j'k w_i'k' must be 1 when j = j', i = i', k = k' and 0 otherwise.
 * U, V, W are host arrays in the layout of cse_scheme_load_uvw (any int8
 * values).  *violations = the number of index triples whose sum is wrong (0
 * for a valid scheme).  m n, n p, m p <= 4096, r <= 65536.  Synchronous; it
 * allocates and frees its own device buffers. */
int cse_brent_check(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                    const int8_t* W, int64_t* violations);

/* The generator behind every random draw of a search: Philox4x32-10 (Salmon,
 * Moraes, Dror and Shaw, SC'11), keyed by the search seed and counted by
 * (process, step, matrix and purpose, extra).  The paper leaves the source
 * of its random choices open (Sections 3.4-3.5); this entry point exposes the
 * device implementation for verification and for reproducing draws.
 * out[4q .. 4q+3] = Philox4x32-10(counter = counters[4q .. 4q+3],
 * key = (seed & 0xFFFFFFFF, seed >> 32)) for 0 <= q < n.  counters and out
 * are caller-owned host arrays of 4 n uint32; 0 <= n <= 2^24 (n = 0 touches
 * neither array nor the device).  Synchronous; it allocates and frees its
 * own device buffers.  Errors: CSE_EINVAL (n out of range, NULL array with
 * n > 0), CSE_ECUDA. */
int cse_philox(uint64_t seed, const uint32_t* counters, int64_t n, uint32_t* out);

/* Shape of a loaded matrix. */
int cse_scheme_shape(const cse_scheme* s, int32_t mat, int32_t* rows, int32_t* cols);

/* Runs the search: n_processes processes per matrix, step_budget steps each
 * (one step = at most one substitution, Algorithm 1), sharing every
 * opts->share_interval steps (Section 3.5.2).  The work is enqueued on
 * cuda_stream (a cudaStream_t, or NULL for the legacy default stream) and the
 * call returns without waiting; *out owns the device state and results.
 * n_processes <= 2^20, 0 <= step_budget < 2^31.  In iteration mode
 * (share_interval = 0) the call returns only when the search has finished:
 * the host reads the convergence state every 4 iterations, so the length of
 * the launch sequence depends on the data; step_budget (the maximum number
 * of iterations) times col_cap must stay below 2^31.  CSE_FLAG_GRAPH is
 * rejected in that mode. */
int cse_search(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_processes,
               uint64_t seed, int64_t step_budget, const cse_opts* opts, void* cuda_stream,
               cse_result** out);

/* Runs n_searches independent searches in one launch sequence (one CUDA
 * graph with CSE_FLAG_GRAPH): search i is scheme schemes[i] with mixes[i],
 * n_processes[i], seeds[i] and step_budgets[i]; all share *opts.  Every round
 * runs all searches' processes together, one kernel per class of matrices
 * with equal words per column.  Each search keeps its own step clock and
 * sharing snapshot, so outs[i] is identical to what cse_search returns for
 * search i alone (Sections 3.5.1-3.5.2 apply per search).  The schemes must
 * stay loaded until the results are fetched.  outs[i] are freed one by one
 * with cse_result_free; the device memory is released with the last one. */
int cse_search_batch(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                     const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                     const cse_opts* opts, void* cuda_stream, cse_result** outs);

/* One class of matrices as the tuner saw it. */
typedef struct {
    int32_t words_per_column;  /* W = ceil(rows / 32)                          */
    int32_t hbm_path;          /* 1: the process arrays live in HBM            */
    int32_t candidate_bound;   /* bucket (power of two) of the candidate bound */
    int32_t procs_per_cta;     /* chosen processes (warps) per CTA             */
    float trial_ms[4];         /* round-kernel time with 1..4 per CTA          */
    int32_t kernel_words;      /* chosen kernel words per column: W, or the
                                  next power of two when that was faster   */
    float trial_ms_wide[4];    /* the round kernels of the matrices that share
                                  the wider kernel, 1..4 per CTA (-1: W is a
                                  power of two, no wider trial)             */
} cse_tune_entry;

/* Launch autotuner.  Runs the given searches (as in cse_search_batch) for
 * min(step_budget, trial_steps) steps with 1, 2, 3 and 4 processes per CTA,
 * times every class of matrices (equal words per column and memory path)
 * with CUDA events, and caches the fastest choice per class in this process;
 * later searches with opts->procs_per_cta == 0 use it.  Classes whose words
 * per column are not a power of two are also timed on the kernel of the next
 * power of two (as CSE_FLAG_WIDE_WORDS does), and the wider kernel is cached
 * for the class when its round kernels take less time than those of every
 * class it would absorb; later searches (without the flag) use that width.
 * Launch parameters never change results.  Writes up to max_entries entries
 * and the number of classes into *n_entries.  Synchronous. */
int cse_autotune(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                 const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                 const cse_opts* opts, int32_t trial_steps, void* cuda_stream, cse_tune_entry* entries,
                 int32_t max_entries, int32_t* n_entries);

/* Sharing-interval tuner.  The interval changes the search (Section 3.5.2
 * shares between whole iterations, from the second on; here every
 * share_interval steps), so this is an explicit choice: each candidate
 * interval is run on
 * the given searches for min(step_budget, trial_steps) steps and the one with
 * the lowest total additions (sum over searches and matrices) is returned;
 * ties keep the earlier candidate.  Synchronous. */
int cse_tune_interval(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                      const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                      const cse_opts* opts, const uint32_t* candidates, int32_t n_candidates,
                      int32_t trial_steps, void* cuda_stream, uint32_t* best_interval, int64_t* best_total);

/* Waits for the search and copies the best substitution list of matrix mat:
 * up to cap_entries packed entries into subst (may be NULL), its length into
 * *n_subst, its Cost into *additions, and the sum of the best Cost over all
 * matrices into *total_additions (any pointer may be NULL).  The best list
 * is the lowest (Cost, process index) over all processes. */
int cse_result_fetch(const cse_result* r, int32_t mat, int32_t* subst, int32_t cap_entries,
                     int32_t* n_subst, int64_t* additions, int64_t* total_additions);

/* Per-process record of a finished search (for checking and analysis). */
typedef struct {
    int64_t best_cost;  /* Cost of the process's best substitution list      */
    int32_t best_len;   /* its length                                        */
    int32_t runs;       /* runs started (Algorithm 1 executions)             */
    uint64_t best_hash; /* FNV-1a over the 32-bit entries of the best list   */
    uint64_t traj_hash; /* FNV-1a over the trajectory: (t, 0xA0000000 |
                           strategy << 12 | replayed) at each run start and
                           (t, entry) at each substitution step; recorded
                           only with CSE_FLAG_TRACE, else the FNV offset
                           basis 0xCBF29CE484222325                          */
    int64_t ops;        /* algorithmic integer operations (see the counters
                           of cse_result_counters)                           */
    int64_t substeps;   /* steps that made a substitution                    */
    int32_t best_strategy; /* strategy of the run that produced the best
                              record, in the weight order gi 0, ga 1, gr 2,
                              wr 3, mix 4, g 5, gp 6; -1 if no run improved
                              on the input (per-strategy win counts)         */
    int32_t pad;
    int64_t method_ops; /* the method's own op count (cse_result_method_ops) */
} cse_proc_record;

/* Waits for the search and writes n_processes records of matrix mat. */
int cse_result_procs(const cse_result* r, int32_t mat, cse_proc_record* out);

/* The best-Cost curve of matrix mat: costs[r] = the lowest best record over
 * all processes after round r (step clock: after min((r + 1) share_interval,
 * step_budget) steps; iteration mode: after iteration r).  *n_points = the
 * rounds run, at most 4096 (later rounds are not recorded); up to max_points
 * are written. */
int cse_result_curve(const cse_result* r, int32_t mat, int32_t* costs, int32_t max_points, int32_t* n_points);

/* Waits for the search and reports, summed over all matrices and processes:
 * *process_steps = n_mats * n_processes * step_budget with the step clock,
 * the steps the runs actually made in iteration mode, *substeps = steps
 * that made a substitution, *alg_ops = algorithmic integer operations.
 * An algorithmic op count is defined per step from the method's quantities:
 * 10 W for a rewrite plus 5 W per pair count that can change (candidates
 * holding x_i or x_j, and x_k against every live column), W = ceil(rows/32);
 * 2 m for a g/ga/wr/gr selection over m candidates; for gi, per candidate p
 * 3 |I_p| + 8 plus 40 per 128-bit Philox block its coins use, I_p being the
 * candidates sharing a variable with p. */
int cse_result_counters(const cse_result* r, int64_t* process_steps, int64_t* substeps,
                        int64_t* alg_ops);

/* Waits for the search and reports *method_ops, summed over all matrices and
 * processes: the integer work the method itself must do, independent of how
 * the kernels do it (the roofline's numerator).  Per step: a rewrite
 * (Algorithm 1, substitution; Section 3.2.1) costs 6 per 64-bit word of a
 * column (ceil(rows / 64) words of +rows and -rows, read and written) plus,
 * for the pair counts it changes, the number of nonzeros of every rewritten
 * row before the rewrite; every selection scans the m candidates (m);
 * Greedy-Intersections (Section 3.4.2) adds 2 per intersect term (one coin
 * bit and one conditional add), or with shared coins 4 per candidate;
 * Greedy-Potential adds per candidate one trial rewrite (6 per 64-bit word
 * plus the nonzeros of the candidate's rows).  Replayed prefix substitutions
 * (Section 3.5.2) count as rewrites. */
int cse_result_method_ops(const cse_result* r, int64_t* method_ops);

/* Waits for the search and reports how its large-matrix process-rounds ran:
 * *cta_rounds on the process-per-CTA engine, *warp_rounds on the
 * one-warp-per-process HBM engine (process-rounds handed back by the CTA
 * engine included).  Both 0 for searches without large matrices. */
int cse_result_engine_rounds(const cse_result* r, int64_t* cta_rounds, int64_t* warp_rounds);

/* Device time of the search's kernels in milliseconds, from CUDA events
 * recorded around the round kernels on the search's stream: *round_ms sums
 * the step-engine launches, *total_ms spans the whole search. */
int cse_result_timing(const cse_result* r, float* round_ms, float* total_ms, int32_t* n_rounds);

/* Iteration mode only (share_interval = 0): waits for the search and reports
 * the iterations it ran, whether it stopped by the patience rule before its
 * maximum, and the final sum over the matrices of the best Cost. */
int cse_result_iterations(const cse_result* r, int32_t* iterations, int32_t* converged, int64_t* best_total);

/* Component-wise (hybrid) minimum over several results of the same scheme
 * (Section 5, component-wise analysis: the best U, V and W parts may come
 * from different runs).  Waits for every result; best_result[k] (n_mats
 * entries) = the index of the result with the lowest Cost for matrix k, the
 * first one on ties; *total_additions = the sum of those Costs.  The results
 * must have the same number and shapes of matrices. */
int cse_result_hybrid(const cse_result* const* results, int32_t n_results, int32_t* best_result,
                      int64_t* total_additions);

/* Kernel launches of the search's launch sequence (shared by all searches of
 * a batch) and the number of searches that shared it. */
int cse_result_launches(const cse_result* r, int32_t* kernels, int32_t* searches_in_launch);

/* ---- Checkpoint / resume ------------------------------------------------
 * The paper's tool keeps no checkpoints; these make long searches
 * restartable.  Every draw is keyed by (seed, process, step), so a search of
 * B1 + B2 steps that is checkpointed after B1 and resumed for B2 more gives
 * exactly the results (and per-process records) of one search of B1 + B2
 * steps.
 *
 * cse_checkpoint_size: bytes of the checkpoint of r (a header, then r's
 * device state byte for byte).
 * cse_checkpoint_save: waits for r and writes its checkpoint to host_buf
 * (bytes >= the size).  With the step clock the step budget must be a
 * multiple of share_interval (a sharing boundary); in iteration mode any
 * finished search qualifies.
 * cse_search_resume: starts a search from a checkpoint of a search of the
 * scheme s (same matrix shapes) that runs more_steps further steps
 * (iterations in iteration mode).  The strategy mix, seed, process count and
 * the options that change results come from the checkpoint; of launch_opts
 * (may be NULL) only procs_per_cta is used.  Like cse_search otherwise. */
int cse_checkpoint_size(const cse_result* r, size_t* bytes);
int cse_checkpoint_save(const cse_result* r, void* host_buf, size_t bytes);
int cse_search_resume(const cse_scheme* s, const void* checkpoint, size_t bytes, int64_t more_steps,
                      const cse_opts* launch_opts, void* cuda_stream, cse_result** out);

void cse_result_free(cse_result* r);
void cse_scheme_free(cse_scheme* s);

/* ---- Serving (continuous batching) ----------------------------------------
 * A server owns a worker thread and a CUDA stream on the current device.
 * Requests (a scheme and its search parameters) queue in FIFO order.  At
 * every round boundary the worker admits queued requests while (a) the
 * device memory of all active searches, and of finished ones whose results
 * have not been waited for (a result holds its search's device memory until
 * cse_result_free), stays within hbm_budget_bytes (0 = 85% of the device
 * memory free when the server is created), (b) the active searches'
 * processes (all matrices) stay within
 * max_active_processes (0 = 64 waves of one process per resident warp,
 * 64 x 32 x SMs) and (c) the shared-memory footprint of their process pools
 * (each process of a matrix on the shared-memory path holds one slice) stays
 * within as many waves of the GPU's shared memory as the process cap has
 * waves (waves x SMs x per-SM capacity); a request that exceeds a limit
 * alone runs alone.  A larger cap raises throughput at some cost in
 * time-to-result.  Then it
 * runs one round (one kernel per class of matrices over every active search,
 * then the share kernel).  Admitted searches run concurrently with those
 * already on the device and leave as soon as their step budget is done.  Each
 * search keeps its own step clock, so a request's result is exactly what
 * cse_search returns for it alone.  Of opts->flags only CSE_FLAG_TRACE is
 * used.  The server runs the step clock: share_interval = 0 is rejected. */
int cse_server_create(const cse_opts* opts, uint64_t hbm_budget_bytes, int64_t max_active_processes,
                      cse_server** out);

/* Queues a request; the scheme must stay loaded until its result is taken.
 * Returns CSE_EINVAL for invalid parameters (checked here), CSE_EBUSY when
 * 65536 requests are already waiting for admission.  *ticket identifies it. */
int cse_server_submit(cse_server* s, const cse_scheme* scheme, const cse_strategy_mix* mix, int32_t n_processes,
                      uint64_t seed, int64_t step_budget, uint64_t* ticket);

/* Waits up to timeout_us microseconds (negative: no limit) for a request;
 * CSE_ETIMEOUT if it is not done, else hands over its result (free it with
 * cse_result_free; cse_result_timing reports the time from submission to
 * completion).  Each ticket can be taken once. */
/* Cancels a request: a queued request leaves the queue at once; a running one
 * leaves the device at the next round boundary (its memory is released
 * there).  cse_server_wait on its ticket then returns CSE_ECANCELED.  Returns
 * CSE_EINVAL for an unknown ticket or a request that has already finished. */
int cse_server_cancel(cse_server* server, uint64_t ticket);

int cse_server_wait(cse_server* s, uint64_t ticket, int64_t timeout_us, cse_result** out);

/* Time-to-result percentiles (ms) over completed requests, process-steps
 * per second from the first submission to the last completion, and the
 * number of completed requests. */
int cse_server_stats(cse_server* s, double* p50_ms, double* p99_ms, double* steps_per_s, int32_t* completed);

/* The most searches that ran together in one round, and the rounds run so
 * far (either pointer may be NULL).  With a budget that no two requests fit
 * in together, the peak is 1. */
int cse_server_peak(cse_server* s, int32_t* max_active_searches, int32_t* rounds);

/* Stops the worker (requests not yet finished are dropped) and frees the
 * server.  No other call on it may be in progress. */
void cse_server_free(cse_server* s);


/* ---- Random-flip mode (Section 3.5.3) -------------------------------------
 * Writes n_variants variants of the scheme (m,n,p:r) for flip iteration
 * `iteration` into out_U/out_V/out_W (host, n_variants x r x (m n), (n p),
 * (m p), variant after variant, in the layout of cse_scheme_load_uvw):
 * variant 0 is the input, variant v >= 1 the input after a random number
 * F in [1, max_flips] of ternary flips of the flip graph the paper cites
 * (terms l != m whose factor X agrees up to a sign sigma get Y_l += sigma Y_m
 * and Z_m -= Z_l, Y and Z the other factors, only if both stay ternary and
 * nonzero; at most 32 F attempts, each drawn from Philox keyed by seed with
 * counter (v, iteration, 5 << 20, attempt + 1)).  Flips keep the scheme's
 * tensor, hence every Brent equation; flips[v] = the flips applied and
 * brent_violations[v] (optional) = the variant's violated Brent equations,
 * counted on the device (0 for a valid input).  The variants are generated
 * on the device, one warp each.  Limits as cse_brent_check; n_variants <=
 * 4096.  Searching the variants (one search each, e.g. with
 * cse_search_batch) and keeping the best is the caller's loop. */
int cse_flip_variants(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                      const int8_t* W, int32_t n_variants, uint64_t seed, int32_t iteration, int32_t max_flips,
                      int8_t* out_U, int8_t* out_V, int8_t* out_W, int32_t* flips, int64_t* brent_violations);

/* ---- One search split across ranks (Section 3.5: processes interact only
 * at the sharing boundaries) -----------------------------------------------
 * A shard runs processes [proc_begin, proc_begin + proc_count) of a search of
 * n_processes processes per matrix; its draws are keyed by the global process
 * index, so the union of the shards of a search is that search, bit for bit,
 * provided every sharing boundary is completed with the minima of all
 * shards.  Each rank (one GPU each) loops:
 *   cse_shard_round(h, keys, &left)     runs this round's steps; keys[k] =
 *                                       this shard's (best Cost << 32 |
 *                                       global process) minimum of matrix k
 *   (the caller takes the minimum of keys over the ranks, and the owner of
 *    each minimum fetches that process's best list with cse_shard_best_list
 *    and sends it to the others)
 *   cse_shard_share(h, min_keys, lists, lens)  completes the boundary
 * until left is 0.  The exchange is the caller's (for example an allreduce of
 * the keys and of the lists); the library stays on one GPU.  Only the step
 * clock (share_interval >= 1) is supported, without CSE_FLAG_GRAPH.  After the
 * last boundary, cse_result_fetch gives the search's result (the same on
 * every rank) and cse_result_procs / _counters / _method_ops this shard's
 * processes (proc_count records). */
int cse_search_shard(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_processes, int32_t proc_begin,
                     int32_t proc_count, uint64_t seed, int64_t step_budget, const cse_opts* opts, void* cuda_stream,
                     cse_result** out);
/* Enqueues the next round's step kernels and waits for them; writes n_mats
 * keys (host) and *rounds_left, the rounds left including this one (0: the
 * search is finished, nothing ran).  CSE_EINVAL if the previous round's
 * boundary is not completed. */
int cse_shard_round(cse_result* shard, uint64_t* round_keys, int32_t* rounds_left);
/* The best list of the process named by round_key (this shard's) in matrix
 * mat: *len <= col_cap entries into list (host).  CSE_EINVAL if another shard
 * holds that process. */
int cse_shard_best_list(const cse_result* shard, int32_t mat, uint64_t round_key, int32_t* list, int32_t* len);
/* Completes the round's sharing boundary (Section 3.5.2) with keys[n_mats],
 * the minima over all shards; for a matrix whose winner is another shard's,
 * lists[k * col_cap ..] and lens[k] hold its best list (host; may be NULL if
 * every winner is this shard's).  Waits for the share kernel. */
int cse_shard_share(cse_result* shard, const uint64_t* keys, const int32_t* lists, const int32_t* lens);

/* Integer-pipe microbenchmark: the measured peaks behind the roofline of the
 * step engine (integer bitset work, not a dense contraction).  Every resident
 * thread of a one-wave grid (up to 32 warps per SM) runs 8 independent chains
 * of one instruction mix for `iters` iterations:
 *   kind 0  3-input XOR (LOP3) + add (IADD3)      2 lane-ops per step
 *   kind 1  AND + popcount + add                   3 lane-ops per step
 *   kind 2  32-bit multiply-add (IMAD)             1 lane-op per step
 *   kind 3  32-bit multiply-high (IMAD.HI)         1 lane-op per step
 *   kind 4  3-input XOR (LOP3) alone               1 lane-op per step
 *   kind 5  3-input add (IADD3) alone              1 lane-op per step
 * Writes *ops_per_clk_per_sm (lane-ops per SM clock, from clock64() spans of
 * every block: independent of the clock frequency), *lane_ops_per_s (from
 * CUDA events) and *seconds (the launch's event time).  Allocates and frees a
 * small device buffer and synchronises the stream; CSE_EINVAL for a kind outside
 * 0..5 or iters outside [1, 2^40], CSE_ECUDA without a device. */
int cse_int_peak(int32_t kind, int64_t iters, void* cuda_stream, double* ops_per_clk_per_sm,
                 double* lane_ops_per_s, double* seconds);

/* ---- A search that allocates no device memory ------------------------------
 * The paper has no counterpart: this is an integration aid.  Some callers may
 * not allocate device memory when they run a search -- a host that has handed
 * the whole device to another framework's memory pool, a latency-critical
 * loop where an allocation can stall on device-wide synchronisation, a plugin
 * that only receives device pointers.  cse_search_static runs the same search
 * as cse_search with every byte of scratch (process states, best lists,
 * sharing snapshots, launch parameters) taken from one file-scope device
 * array of CSE_STATIC_SCRATCH_BYTES that every GPU loading this library keeps
 * until the process exits; it calls no allocation routine.
 *   - The scheme must already be loaded (cse_scheme_load allocates; do that
 *     during set-up).
 *   - d_lists: device buffer of n_mats * col_cap int32; matrix k's best list
 *     (packed entries) is written at d_lists + k * col_cap.
 *   - d_meta: device buffer of n_mats * 2 int32; (Cost, length) of matrix k
 *     at d_meta + 2k.  The values equal cse_result_fetch's for cse_search.
 *   - A search needing more scratch than CSE_STATIC_SCRATCH_BYTES is refused
 *     with CSE_ENOMEM before anything runs (the message gives the size).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *     that first call before any stream capture.  A device reset
 *     (cudaDeviceReset) makes the kept address stale: do not call this entry
 *     point again in a process that has reset the device.
 *   - Options as for cse_search, except that share_interval must be >= 1,
 *     patience_rounds 0, and CSE_FLAG_GRAPH is refused (CSE_EINVAL).
 *   - The call enqueues on cuda_stream and waits for the search to finish.
 *   - All calls share the one array and each re-initialises what it reads;
 *     calls that overlap on the GPU (for example from two host threads) race
 *     and corrupt each other. */
#define CSE_STATIC_SCRATCH_BYTES (32u << 20)
int cse_search_static(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_processes, uint64_t seed,
                      int64_t step_budget, const cse_opts* opts, void* cuda_stream, int32_t* d_lists,
                      int32_t* d_meta);

/* Message of the last error on the calling thread ("" if none). */
const char* cse_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
