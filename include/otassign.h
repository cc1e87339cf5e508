/*
 * otassign.h -- C ABI of libotassign.so, an exact GPU solver for the
 * assignment problem on dense integer cost matrices (sm_103a).
 *
 * The problem (paper "A Study of Performance of Optimal Transport",
 * Sec. 1, Eq. 1, with supplies r and demands c all ones): given an n x m cost
 * matrix C (n <= m), find an injective map sigma: [n] -> [m] that minimises
 * sum_i C[i][sigma(i)].  Two exact algorithms are offered:
 *
 *   OT_KM   Kuhn-Munkres (Hungarian) in shortest-augmenting-path form, one
 *           root row at a time in index order (Sec. 2.3 "Variations of the
 *           Hungarian algorithm", Sec. 4.1 "KM and variants").  With the
 *           tie-breaks below its assignment and duals are deterministic and
 *           identical to the CPU reference implementation.
 *   OT_BKM  batched KM (Sec. 2.3 "Batched KM"): augmenting paths are routed
 *           in batches along tight edges from all free rows at once and the
 *           duals are adjusted across the cut between reached and unreached
 *           vertices, as KM adjusts them.  Exact mode (scaling factor 1):
 *           its optimal cost equals OT_KM's; assignment and duals may differ
 *           among optimal ones but always form a valid certificate.
 *
 * Results.  row_to_col[i] = sigma(i); cost = sum_i C[i][sigma(i)] (int64);
 * duals u[n], v[m] (int64) with u_i + v_j <= C[i][j] for all (i, j),
 * equality on matched pairs, v_j <= 0, v_j = 0 on unmatched columns and
 * sum(u) + sum(v) = cost, which proves optimality by LP duality.
 *
 * Tie-breaks (the paper is silent): rows are rooted in index order (OT_KM),
 * the minimum slack selects the lowest column index, a slack entry changes
 * only on a strictly smaller value (OT_KM) or a smaller (value, row) pair
 * (OT_BKM).
 *
 * Memory.  Every pointer argument may be a device pointer or a host pointer;
 * the library asks the CUDA runtime which one it is.  Host inputs are copied
 * to device staging owned by the context and host outputs are written back
 * before the call returns.  With device pointers the call is asynchronous on
 * `stream` (a cudaStream_t) unless stated otherwise.  NULL (like the legacy
 * and per-thread default-stream handles) means the caller's default stream:
 * the library then works on a stream of its own that is ordered after the
 * work already queued on the default stream and before the work queued
 * there after the call.  Consecutive calls on one context are ordered among
 * themselves whatever streams they name.  The caller keeps ownership of all buffers and the
 * library keeps no caller pointer after the call returns.  The cost matrix is
 * row-major int32 with leading dimension ldc (elements, ldc >= m).
 *
 * Errors.  Every call returns OT_OK (0) or a negative OT_ERR_* code and
 * never throws or aborts; ot_last_error_string() gives detail.  Device code
 * never traps: device-side failures are reported in a status word.
 */
#ifndef OTASSIGN_H
#define OTASSIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OT_OK 0
#define OT_PENDING 1             /* ot_assign_poll: not finished yet */
#define OT_ERR_ARG (-1)          /* null pointer, n < 0, n > m, ldc < m, bad algo */
#define OT_ERR_OOM (-2)          /* device or host allocation failed */
#define OT_ERR_BUDGET (-3)       /* serving: request can never fit the HBM budget */
#define OT_ERR_TIMEOUT (-4)      /* a bounded device wait expired */
#define OT_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define OT_ERR_OVERFLOW (-6)     /* |C| too large for exact int64 duals */
#define OT_ERR_UNSUPPORTED (-7)  /* size or option the library does not support */
#define OT_ERR_TICKET (-8)       /* unknown or already collected ticket */

#define OT_KM 0
#define OT_BKM 1
#define OT_AUTO 2   /* per size bucket, whichever of OT_KM / OT_BKM the tuned table
                       names (built-in: KM for m <= 256, batched KM above); both are
                       exact, the optimal assignment and duals returned depend on it */
#define OT_AUCTION 3  /* the auction algorithm with epsilon-scaling (Sec. 2.3.3 "The
                       auction algorithm", Sec. 4.1 "Auction"), exact for integer costs:
                       costs shifted to start at 0 and scaled by m + 1, n < m padded with
                       zero-cost dummy rows, parallel (Jacobi) bidding rounds, the
                       highest bid (lowest row on ties) wins, eps_0 = max(1, R'/8) for
                       the scaled range R', eps /= 4 per stage down to 1.  Returns the
                       assignment and cost; u and v (when given) receive zeros.  Counters:
                       steps = bidding rounds, rows_scanned = bids, phases = eps stages,
                       cost_bytes = 4*m per bid of a real row, init_bytes = 4*n*m (the
                       range pass).  ot_assign_solve / _stats / _batched only, m <= 4096
                       (OT_ERR_UNSUPPORTED above). */

/* Per-solve counters, written by ot_assign_solve_stats. */
typedef struct ot_stats {
  int64_t steps;          /* dependent tree-growing steps (one argmin each) */
  int64_t rows_scanned;   /* cost rows evaluated (each over the columns outside T) */
  int64_t cost_bytes;     /* 4 x reduced costs evaluated: the algorithmic bytes */
  int64_t phases;         /* KM: rows rooted; BKM: dual-adjust/augment phases */
  int64_t augmentations;  /* augmenting paths applied */
  int64_t init_bytes;     /* BKM row-reduction pass bytes (4*n*m), else 0 */
  int64_t reserved[2];    /* [1]: bytes of cost elements actually loaded by the
                             scans (2 per element when rows were packed to
                             16 bits, else equal to cost_bytes) */
} ot_stats;

/* Context configuration.  A zero-filled struct (with device = -1) gives the
 * defaults; cfg = NULL in ot_ctx_create does the same. */
typedef struct ot_config {
  int32_t device;            /* CUDA device ordinal; -1 = current device */
  int64_t hbm_budget_bytes;  /* serving arena = admission budget; 0 = 4 GiB */
  int32_t max_inflight;      /* serving: max requests resident at once; 0 = 4096 */
  int32_t wave_streams;      /* serving: streams used for overlapping waves; 0 = 4 */
  const char* tune_file;     /* autotuner table (JSON-lines); NULL = built-in */
  uint32_t flags;            /* OT_CFG_* bits; 0 = defaults */
  int32_t max_group_ctas;    /* upper bound on the CTAs of one batched group-engine
                                launch; 0 = as many as fit on the device at once */
  int64_t step_limit;        /* dependent tree-growing steps one instance may take in
                                the warp/CTA group engine before its status becomes
                                OT_ERR_TIMEOUT (its results are then undefined; the
                                other instances are unaffected); 0 = only the built-in
                                guards.  For failure-detection tests. */
} ot_config;

/* ot_config.flags */
#define OT_CFG_NO_ROW_PACKING 1u  /* batched launches keep 32-bit cost rows (no 16-bit
                                     packing pass, 64-bit solver arithmetic) */
#define OT_CFG_DENSE_WIDE 2u      /* batched-KM instances too wide for one CTA run on the
                                     dense cluster engine (every tree row scanned in full)
                                     instead of the sparse-list engine; same results */

typedef struct ot_ctx ot_ctx;

/* Create / destroy a context (device buffers, streams, serving thread).
 * cfg may be NULL.  Destroy waits for outstanding work. */
int ot_ctx_create(ot_ctx** out, const ot_config* cfg);
void ot_ctx_destroy(ot_ctx* ctx);
const char* ot_last_error_string(const ot_ctx* ctx);

/* Solve one instance.  C[n*ldc], row_to_col[n], cost[1], u[n], v[m].
 * u and v may be NULL if the duals are not wanted.  n == 0 gives cost 0. */
int ot_assign_solve(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                    int32_t algo, int32_t* row_to_col, int64_t* cost, int64_t* u,
                    int64_t* v, void* stream);

/* As ot_assign_solve, then synchronises and fills *stats (host pointer). */
int ot_assign_solve_stats(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n,
                          int32_t m, int32_t algo, int32_t* row_to_col, int64_t* cost,
                          int64_t* u, int64_t* v, ot_stats* stats, void* stream);

/* Batched KM with a single scaling factor s >= 1, the paper's approximate
 * variant (Sec. 2.3 "Batched KM": costs rounded to small integers by one
 * factor; Table 3 runs it as a 1.1-approximation).  The assignment problem
 * is solved exactly on the scaled costs floor(C[i][j] / s) and the result's
 * cost under the original C is returned in *cost.  Writing
 * c = s*floor(c/s) + r with 0 <= r <= s-1 gives
 * OPT <= *cost <= OPT + n*(s-1); *bound (may be NULL) receives n*(s-1).
 * s = 1 is the exact solver.  Synchronous.  C, row_to_col, cost and bound
 * may be host or device pointers. */
int ot_assign_solve_scaled(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                           int32_t scale, int32_t* row_to_col, int64_t* cost, int64_t* bound,
                           void* stream);

/* Optimal transport with integer supplies and demands (Sec. 1, Eq. 1:
 * min <C, X> subject to X 1 = r, X^T 1 = c with nonnegative integer r, c),
 * solved exactly by vertex replication: row i is copied supply[i] times and
 * column j demand[j] times (copies in index order, so that OT_KM returns a
 * deterministic flow), the R x M assignment problem (R = sum(supply) <=
 * M = sum(demand)) is solved with `algo`, and flow[i*m + j] counts the
 * matched copies of (i, j).  With equal totals this is Eq. 1; with
 * R < M every column receives at most demand[j].  *cost = <C, X>.  Only
 * small totals are practical: OT_ERR_UNSUPPORTED if M > 65536 or
 * R*M > 2^30.  supply and demand are host arrays; C, flow (n*m int32) and
 * cost may be host or device pointers.  Synchronous. */
int ot_transport_solve(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                       const int32_t* supply, const int32_t* demand, int32_t algo, int64_t* cost,
                       int32_t* flow, void* stream);

/* Entropic optimal transport by log-domain Sinkhorn (Sec. 2.2 "Matrix
 * Scaling", Sec. 2.2.1 "Sinkhorn"; configuration of Sec. 4.1 "Sinkhorn"):
 * min <X, C> - h(X)/eta over X 1 = r, X^T 1 = c, solved as
 * X_ij = exp(f_i + g_j - eta C_ij).  Starting from f = g = 0, each
 * iteration scales every row (f_i = log r_i - LSE_j(g_j - eta C_ij)) and
 * then every column (g_j = log c_j - LSE_i(f_i - eta C_ij)).  The first
 * iterate whose residue sum_i |r_i - (X 1)_i| is at most eps_rel * sum(r)
 * is returned (the paper uses eps_rel = 1e-3 and no rounding; the column
 * sums are exact after the column scaling); with eps_rel <= 0, or when
 * max_iter iterations do not reach it, iterate max_iter is returned.
 *   C: device pointer, n x m int32 (ldc >= m); r (n), c (m): host arrays of
 *   positive supplies and demands with equal totals, or NULL for r = 1 and
 *   c = n/m.  f (n), g (m): float32 outputs (host or device, may be NULL);
 *   *cost = <C, X> (double), *residue, *iterations: host pointers
 *   (residue and iterations may be NULL).
 * Arithmetic is float32 for the exponent arguments, exponentials and sums
 * and double for the residue and cost accumulators.  Each iteration reads
 * C twice (a row pass and a column pass).  Synchronous.  OT_ERR_ARG for
 * n, m < 1, eta <= 0, max_iter < 1, non-positive or unbalanced marginals,
 * or a host C. */
int ot_sinkhorn_solve(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                      const double* r, const double* c, double eta, double eps_rel,
                      int32_t max_iter, float* f, float* g, double* cost, double* residue,
                      int32_t* iterations, void* stream);

/* Log-domain Sinkhorn on k independent instances (the iteration and
 * stopping rule of ot_sinkhorn_solve, unit marginals r = 1, c = n/m), one
 * CTA per instance.  All pointers are device pointers: C[t] (n[t] x m[t]
 * int32, ldc[t] >= m[t]), f[t] (n[t] floats), g[t] (m[t] floats), and the
 * arrays cost[k], residue[k] (double) and iterations[k] (int32).
 * Asynchronous on `stream`.  1 <= n[t], m[t] <= 4096 (OT_ERR_UNSUPPORTED
 * above); OT_ERR_ARG for eta <= 0 or max_iter < 1. */
int ot_sinkhorn_solve_batched(ot_ctx* ctx, int32_t k, const int32_t* const* C, const int64_t* ldc,
                              const int32_t* n, const int32_t* m, double eta, double eps_rel,
                              int32_t max_iter, float* const* f, float* const* g, double* cost,
                              double* residue, int32_t* iterations, void* stream);

/* Synchronise the context's stream and return the counters of the most
 * recent ot_assign_solve / ot_assign_solve_batched call on device pointers,
 * summed over its instances; reserved[0] receives the number of kernel
 * launches that call made.  *total is a host pointer. */
int ot_last_call_stats(ot_ctx* ctx, ot_stats* total);

/* One kernel launch of the most recent ot_assign_solve / _stats / _batched
 * call: the instances of one size bucket solved by one engine shape. */
typedef struct ot_launch_info {
  int32_t algo;                  /* OT_KM, OT_BKM or OT_AUCTION */
  int32_t threads_per_instance;  /* group shape (auction: threads per CTA) */
  int32_t cols_per_thread;       /* group shape (auction: 0) */
  int32_t instances;
  float ms;                      /* device time of the kernel (CUDA events around it), -1 if unknown */
  int32_t reserved;
  int64_t read_bytes;            /* cost bytes its scans loaded (as ot_stats.reserved[1]) */
  int64_t init_bytes;            /* row-reduction / range-pass bytes */
} ot_launch_info;

/* Synchronises, then describes the group- and auction-engine launches of
 * the most recent solve call (instances handed to the cluster engine are
 * not listed, nor are the launches of a large host-pointer batch staged in
 * chunks): *count receives their number, out[0 .. min(count, max)-1] their
 * descriptions. */
int ot_last_call_launches(ot_ctx* ctx, ot_launch_info* out, int32_t max, int32_t* count);

/* Solve k independent instances in one launch set (multi-instance
 * batching).  The array arguments are HOST arrays of length k; their
 * elements (C[t], row_to_col[t], u[t], v[t]) are device pointers, or all host
 * pointers.  cost[k] and status[k] follow the same rule as the element
 * pointers (device or host).  Instances are bucketed by size onto
 * warp-, CTA- or cluster-sized solver groups chosen by the autotuner table.
 * status[t] = 0 on success or a negative OT_ERR_* code for that instance.
 * Each instance's result is identical to solving it alone. */
int ot_assign_solve_batched(ot_ctx* ctx, int32_t k, const int32_t* const* C,
                            const int64_t* ldc, const int32_t* n, const int32_t* m,
                            int32_t algo, int32_t* const* row_to_col, int64_t* cost,
                            int64_t* const* u, int64_t* const* v, int32_t* status,
                            void* stream);

/* Serving (continuous batching).  submit copies C (host or device pointer)
 * into the context's device arena when the request is admitted under the HBM
 * budget; requests that arrive while others run are launched in overlapping
 * waves.  The caller's C may be reused as soon as submit returns.  *ticket
 * identifies the request.  OT_ERR_BUDGET if the request alone exceeds the
 * budget. */
int ot_assign_submit(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                     int32_t algo, uint64_t* ticket);

/* Poll a ticket: OT_PENDING while running; OT_OK once finished, after
 * copying the results into row_to_col[n], cost[1], u[n], v[m] (host or
 * device pointers; u, v may be NULL); the ticket is then retired.  A
 * negative code reports a failed request (also retiring it). */
int ot_assign_poll(ot_ctx* ctx, uint64_t ticket, int32_t* row_to_col, int64_t* cost,
                   int64_t* u, int64_t* v);

/* Completion query: the tickets of requests whose solve has ended (with a
 * result or an error) and that no earlier call returned, at most `max` of
 * them, into tickets[0 .. *count - 1] (host array).  Each is then collected
 * with ot_assign_poll, which does not answer OT_PENDING for it.  Requests
 * still waiting or running, and collected or cancelled ones, are not
 * returned.  A client that collects through this call does work in
 * proportion to the completions, not to the requests in flight. */
int ot_assign_completed(ot_ctx* ctx, uint64_t* tickets, int32_t max, int32_t* count);

/* Cancel a submitted request: its result is discarded and its ticket
 * retired (a later poll or cancel returns OT_ERR_TICKET).  A request still
 * waiting for admission, or admitted but not yet launched, is dropped at
 * once; a running one keeps its arena block until its solver has finished
 * (the GPU work is not interrupted), then the block is returned to the
 * budget.  OT_ERR_TICKET for an unknown, collected or cancelled ticket. */
int ot_assign_cancel(ot_ctx* ctx, uint64_t ticket);

/* Wait until every submitted request has finished (not collected). */
int ot_assign_drain(ot_ctx* ctx);

/* Serving counters (host pointer, 8 entries): submitted, admitted,
 * completed, waves launched, max concurrent waves observed, bytes resident,
 * budget bytes, requests refused. */
int ot_serving_counters(ot_ctx* ctx, int64_t* out8);

/* Autotuner: for every size bucket present in the given instances (device
 * pointers, as in ot_assign_solve_batched), time each compiled group shape
 * `repeats` times on exactly those instances and keep the fastest shape for
 * that bucket and algorithm in the context's table (also appended to
 * cfg->tune_file when one was given); with algo = OT_AUTO both algorithms
 * are timed and the faster becomes the bucket's OT_AUTO choice.  Results are
 * written to scratch and discarded.  Synchronises the device first (the
 * instances may still be in flight on any stream).  Returns OT_OK or an
 * error code. */
int ot_autotune(ot_ctx* ctx, int32_t k, const int32_t* const* C, const int64_t* ldc,
                const int32_t* n, const int32_t* m, int32_t algo, int32_t repeats);

/* Current table entry: shape (threads per instance, columns per thread)
 * used for instances with m in the bucket that contains `m`. */
int ot_tune_lookup(ot_ctx* ctx, int32_t algo, int32_t m, int32_t* threads_per_instance,
                   int32_t* cols_per_thread);

/* Force the table entry for the bucket containing m (tests, experiments).
 * threads_per_instance = cols_per_thread = 0 routes the bucket to the
 * cluster engine that otherwise takes instances with m > 4096 (lookup
 * reports 0, 0 for it).  With algo = OT_AUTO, threads_per_instance names the
 * algorithm (OT_KM or OT_BKM) that OT_AUTO uses for the bucket.  OT_ERR_UNSUPPORTED if the shape is not compiled in
 * or cannot hold the bucket's widest instance. */
int ot_tune_set(ot_ctx* ctx, int32_t algo, int32_t m, int32_t threads_per_instance,
                int32_t cols_per_thread);

/* Batched solve that allocates nothing on the device.  There is no
 * counterpart in the paper: this is a packaging of ot_assign_solve_batched
 * for callers that cannot call cudaMalloc -- for example code that runs
 * while another component owns the whole device memory budget (an inference
 * server's fixed arena, a framework allocator that must see every byte), or
 * code on a path where an allocation's implicit synchronisation or failure
 * is not acceptable.  It needs no context.
 *
 * The launch metadata (descriptors, launch order, work counters) goes to one
 * static device array of fixed size that the library's module carries, held
 * by every GPU that loads the library until the process exits.  Hence:
 *   - at most OT_NOALLOC_MAX_INSTANCES instances per call (else
 *     OT_ERR_UNSUPPORTED), each with m <= 4096 (else OT_ERR_UNSUPPORTED);
 *   - every pointer (C[t], row_to_col[t], u[t] and v[t] when given, cost[k],
 *     status[k] when given) must be device memory of the current device
 *     (else OT_ERR_ARG, before anything is launched): host data would need
 *     staging memory;
 *   - all calls share the array, so calls whose work overlaps on the GPU
 *     (different streams or threads) race: serialise them;
 *   - the first call on a device looks up the array's device address and may
 *     load the module; make that first call before any stream capture;
 *   - the metadata is uploaded from host bookkeeping that the next call
 *     overwrites, so a call on a stream that is being captured returns
 *     OT_ERR_UNSUPPORTED.
 * An instance with n == 0 gets cost 0, status 0 and (when v[t] is given)
 * v = 0.  OT_AUTO resolves with the built-in table.  Results are identical to
 * ot_assign_solve_batched's with a context that has the built-in table.
 * Asynchronous on `stream` (NULL = the legacy default stream); per-instance
 * device status codes go to status[k] when it is non-NULL. */
#define OT_NOALLOC_MAX_INSTANCES 1024
int ot_assign_solve_batched_noalloc(int32_t k, const int32_t* const* C, const int64_t* ldc,
                                    const int32_t* n, const int32_t* m, int32_t algo,
                                    int32_t* const* row_to_col, int64_t* cost,
                                    int64_t* const* u, int64_t* const* v, int32_t* status,
                                    void* stream);

/* Library version string, e.g. "otassign 0.1 sm_103a". */
const char* ot_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OTASSIGN_H */
