/*
 * ustat.h -- C ABI of the GB300 (sm_103a) engine for exact higher-order
 * U-statistics whose kernel factors over a graph (arXiv 2508.12627).
 *
 * What is computed (paper, Section 3.3, Algorithm 4 "Ustats"):
 *   U_sum = sum over ordered distinct m-tuples of
 *           prod_{edges (a,b,f)} F_f(x_a, x_b) * prod_{unary (v,g)} g(x_v)
 *         = sum over partitions pi of [m] of mu_pi * V_pi,
 *   mu_pi = (-1)^(m-|pi|) prod_{C in pi} (|C|-1)!      (Lemma "Decomposition of
 *           U-Statistic into V-Statistics", Section 3.3),
 *   V_pi  = the restricted V-statistic (Definition "Restricted V-Statistic"): the
 *           same product summed over tuples that are equal within each block of pi,
 *           evaluated as Einsum(T, A_pi) on the induced notation (Algorithm 3) by
 *           summing out one index at a time along an elimination order (Section
 *           3.2, Proposition "complexity_einsum").
 *   U_mean = U_sum / (n (n-1) ... (n-m+1)).
 *
 * Conventions
 *   - Vertices are 0-based.  Partitions are indexed in the lexicographic order of
 *     their restricted growth strings (rgs[0] = 0, rgs[i] <= 1 + max(rgs[0..i-1])),
 *     the order ustat_plan_info() reports.
 *   - Device pointers are plain CUDA device addresses on the current device.
 *     The caller owns X, every factor buffer, the workspace and the outputs.
 *     The library owns plans (host memory) and never allocates device memory.
 *   - Every function returns USTAT_OK (0) or a negative USTAT_ERR_* code; on error
 *     no output is written.  ustat_strerror() names a code.
 *   - Evaluation enqueues work on the given CUDA stream and returns without
 *     synchronising (ustat_eval_host and ustat_status synchronise the stream).
 */
#ifndef USTAT_H
#define USTAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define USTAT_OK                   0
#define USTAT_ERR_INVALID_ARG     -1  /* null pointer, bad graph, bad size or factor */
#define USTAT_ERR_N_LT_M          -2  /* n < m: the paper's U-statistic needs m <= n (Section 2.1) */
#define USTAT_ERR_TW_TOO_LARGE    -3  /* no elimination order with steps the engine executes */
#define USTAT_ERR_WORKSPACE       -4  /* workspace null, too small or misaligned */
#define USTAT_ERR_NONFINITE       -5  /* an input value is NaN or infinite (ustat_status) */
#define USTAT_ERR_CUDA            -6  /* a CUDA call failed (see ustat_last_cuda_error) */
#define USTAT_ERR_DEVICE_TIMEOUT  -7  /* a bounded device wait ran out */
#define USTAT_ERR_UNSUPPORTED     -8  /* m > 7, arity > 2, or a mode not built */

/* ---- factor kinds (per factor id) ---- */
#define USTAT_RBF       0  /* F(x,y) = exp(-||x-y||^2 / param); unit diagonal        */
#define USTAT_LINEAR    1  /* F(x,y) = (x . y) / param                                 */
#define USTAT_TANH_DOT  2  /* f(x) = tanh(x . w), w = data (device, d doubles); unary  */
#define USTAT_MATRIX    3  /* F given as data: device n x n float64, row-major          */
#define USTAT_VECTOR    4  /* f given as data: device n float64; unary                   */
/* Pairwise factors built on the device from the caller's data (the paper's
 * tensorization, Section 3.1, Algorithm 1, of its application kernels):        */
#define USTAT_DIST      5  /* F(i,j) = ||y_i - y_j||, data = Y (device n x param float64,
                              row-major): the distance matrices of dCov, Section 4.3  */
#define USTAT_LOWRANK   6  /* F(i,j) = sum_k P(i,k) Q(j,k), data = [P | Q] (device n x
                              2 param float64, row-major): the HOIF factors g and f of
                              Section 4.1 from their n x param dictionary terms        */
#define USTAT_COMPLEMENT 7 /* F = 1 - A, data = A (device n x n float64, row-major):
                              the non-edge factor of the motif kernels, Section 4.2   */
#define USTAT_GRAM      8  /* F(i,j) = sum_k P(i,k) P(j,k), data = P (device n x param
                              float64, row-major): the symmetric HOIF factor g of
                              Section 4.1; declared symmetric, so that the planner
                              reads it untransposed and skips mirror product tiles  */

/* ---- precision modes of the contractions ---- */
#define USTAT_FP64    0  /* all arithmetic in float64 (CUDA cores)                          */
#define USTAT_FP32    1  /* float32 factors and GEMMs (CUDA cores), float64 reductions       */
#define USTAT_TF32    2  /* GEMMs on tcgen05 kind::tf32, FP32 accumulation                   */
#define USTAT_BF16X3  3  /* GEMMs on tcgen05 kind::f16 with three bf16 fixed-point slices per
                            operand, exact integer accumulation of the leading slice product */
#define USTAT_BF16X4  4  /* as BF16X3 with four slices (8 more bits per operand row), for
                            factors whose rows span a wide dynamic range; matrices stored
                            and the GEMM epilogues evaluated in float64 */
#define USTAT_BF16X5  5  /* as BF16X4 with five slices (16 more bits than BF16X3): heavy-
                            tailed data whose sums are dominated by few terms */

/* ---- planners (choice of elimination order per partition) ---- */
#define USTAT_PLAN_EXHAUSTIVE  0  /* minimum modelled cost over all orders (<= 8 blocks) */
#define USTAT_PLAN_MINFILL     1  /* greedy minimum fill-in, ties by degree then label */

/*
 * The kernel graph: the multiplicative decomposition h = prod_k h_k(x[A_k]) of
 * the paper's Section 3.1 with signature tuples of length 2 (edges) and 1
 * (unary factors).  edge k is the ordered pair (edge_src[k], edge_dst[k]) with
 * factor id edge_factor[k]; its value is F(x_src, x_dst).  factor_kind[f] is
 * the USTAT_* kind of factor id f (pairwise kinds on edges, unary kinds on
 * unary entries).  Repeated pairs are separate factors (multiplied).
 */
typedef struct {
    int m;                     /* order of the U-statistic, 1 <= m <= 7          */
    int n_edges;
    const int *edge_src, *edge_dst, *edge_factor;
    int n_unary;
    const int *unary_vertex, *unary_factor;
    int n_factors;
    const int *factor_kind;
} ustat_graph;

typedef struct {
    int precision;   /* USTAT_FP64 / FP32 / TF32 / BF16X3 / BF16X4                   */
    int sparsify;    /* 1: zero-diagonal tensors T~ and only partitions in Pi_m^A
                        (Lemma "sparsification_trick", equation "quotient_set");
                        V_pi of skipped partitions is reported as 0                   */
    int planner;     /* USTAT_PLAN_*                                                  */
    int cse;         /* 1: share identical contractions across partitions             */
} ustat_options;

/* Factor values: param as in the kind's formula; data as described per kind. */
typedef struct {
    int kind;
    double param;
    const void *data;
} ustat_factor;

typedef struct ustat_plan ustat_plan_t;

/*
 * Build a plan (host only, no CUDA call): partitions, Moebius coefficients, the
 * quotient factor multigraph of each partition (Definition "Quotient Graph";
 * Algorithm 3), an elimination order per partition, and the lowered program of
 * device operations.  *out receives a plan owned by the library; free it with
 * ustat_plan_destroy().
 */
int ustat_plan(const ustat_graph *graph, const ustat_options *opts, ustat_plan_t **out);
void ustat_plan_destroy(ustat_plan_t *plan);

/*
 * A shard of the partition sum (U = sum over partitions of mu_pi V_pi, Lemma
 * "Decomposition of U-Statistic into V-Statistics", Section 3.3): the plan of rank `shard` of `n_shards`, which
 * evaluates its own partitions and reports V_pi = 0 for the others, so that the
 * element-wise sum over all shards of U_out and V_out (a sum of 2 + Bell(m)
 * float64 values, the one exchange step) gives the full result.
 *   Partitions that share a contraction under opts->cse stay on one shard; the
 *   groups go, costliest first, to the least loaded shard, each costed by the
 *   program that evaluates it alone at sample size n (algorithmic flops, at
 *   least one n^2 pass per operation).  The assignment is a function of the
 *   arguments only, so every rank computes the same one.
 *   owner : [Bell(m)] or NULL; receives each partition's shard, -1 for a
 *           partition that no shard evaluates (skipped by sparsification)
 *   *out  : a plan owned by the library, used like ustat_plan()'s; a shard with
 *           no partition gives U = 0 and V = 0
 * Errors as ustat_plan(); USTAT_ERR_INVALID_ARG if shard is not in [0, n_shards)
 * or n < 1.  Host only, no CUDA call.
 */
int ustat_plan_shard(const ustat_graph *graph, const ustat_options *opts, int shard, int n_shards,
                     int64_t n, int *owner, ustat_plan_t **out);

/*
 * Plan serialisation, for caching plans between processes (planning an order-7
 * graph searches thousands of orders per partition).  ustat_plan_serialize writes
 * the plan into buf (host memory, buf_len bytes; buf may be NULL to query the
 * size) and sets *needed to the bytes it takes.  ustat_plan_deserialize builds a
 * library-owned plan from such bytes; it checks the format, the sizes of the
 * records (a plan written by a build with other record layouts is refused) and
 * that every reference inside the plan is in range.  Errors:
 * USTAT_ERR_INVALID_ARG (NULL plan or out, buf_len too small, bytes that are not
 * a plan of this build).  Host only.
 */
int ustat_plan_serialize(const ustat_plan_t *plan, void *buf, size_t buf_len, size_t *needed);
int ustat_plan_deserialize(const void *buf, size_t len, ustat_plan_t **out);

/*
 * Plan report.  Any output pointer may be NULL.
 *   n_parts : number of partitions (Bell(m))
 *   mu      : [n_parts] Moebius coefficients mu_pi
 *   tw      : [n_parts] treewidth of the quotient graph G/pi (exact); -1 if skipped
 *   rgs     : [n_parts * m] restricted growth strings
 *   evaluated: [n_parts] 1 if V_pi is computed, 0 if skipped by sparsification or
 *             left to another shard (ustat_plan_shard)
 *   n_ops   : number of device operations in the lowered program
 *   n_gemm  : number of n^3 contractions (stored + fused) in the program
 *   n_gemm3 : number of n^4 contractions
 */
int ustat_plan_info(const ustat_plan_t *plan, int *n_parts, int *mu, int *tw, int *rgs,
                    int *evaluated, int *n_ops, int *n_gemm, int *n_gemm3);

/*
 * Text listing of the lowered program, one operation per line
 * ("<index> <op> out=<slot> ..."), NUL-terminated and truncated to buf_len.
 * *needed (may be NULL) receives the full length including the NUL.
 */
int ustat_plan_describe(const ustat_plan_t *plan, char *buf, size_t buf_len, size_t *needed);

/*
 * Algorithmic flop count for sample size n (the paper's cost model, Appendix D,
 * Lemma "complexity_one_index": eliminating an index with s neighbours costs
 * 2 n^(s+1)): flops_plan counts the lowered program (after sharing), flops_naive
 * counts every partition's own elimination without sharing.
 */
int ustat_plan_flops(const ustat_plan_t *plan, int64_t n, double *flops_plan, double *flops_naive);

/* Device workspace bytes needed by ustat_eval for sample size n, dimension d. */
int ustat_workspace_bytes(const ustat_plan_t *plan, int64_t n, int d, size_t *bytes);

/*
 * Evaluate U and every V_pi for one sample.
 *   X       : device, n x d row-major, x_dtype 0 = float64, 1 = float32
 *   factors : host array [n_factors] (the graph's factor ids), data pointers device
 *   ws      : device workspace of at least ustat_workspace_bytes() bytes, 256-byte
 *             aligned; its contents on entry are ignored
 *   stream  : cudaStream_t (NULL = legacy default stream)
 *   U_out   : device float64 [2] = {U_sum, U_mean}
 *   V_out   : device float64 [n_parts] (V_pi in partition order) or NULL
 * Errors: INVALID_ARG, N_LT_M (n < m), WORKSPACE, UNSUPPORTED, CUDA.
 */
int ustat_eval(ustat_plan_t *plan, const void *X, int x_dtype, int64_t n, int d,
               const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes,
               void *stream, double *U_out, double *V_out);
/*
 * Row shard of one evaluation over n_ranks ranks (one GPU each): U = sum_pi mu_pi
 * V_pi is built from scalars that are sums over index tuples (Section 3.3, Lemma
 * "Decomposition of U-Statistic into V-Statistics"; each V_pi is an Einsum over
 * the restricted index set, Definition "Restricted V-Statistic"), so the index
 * ranges of the heavy steps can be divided among ranks and the partial scalars
 * summed.  ustat_eval_rows runs the plan on this rank: the n^3 products that feed
 * only reductions are computed on the rank's contiguous range of their output
 * tiles, the treewidth-3 steps (split modes) on its range of the eliminated
 * index's values, everything else whole (X is replicated: the factor matrices
 * are built on every rank).  It writes the plan's scalars, float64 on the device,
 * scal_out[ustat_scalar_count()], such that the sum over ranks of scal_out is the
 * unsharded evaluation's scalars (scalars every rank computes whole are 0 except on
 * rank 0).  The caller sums the ranks' arrays (one all-reduce of that many
 * doubles) and calls ustat_combine, which forms U_out[2] and V_out[n_parts] (may
 * be NULL) on the device, as ustat_eval would.  n_ranks = 1 gives the whole
 * evaluation's scalars.  Workspace as for ustat_eval.  Errors as ustat_eval, and
 * USTAT_ERR_UNSUPPORTED for a plan whose steps read one of its scalars.
 */
int ustat_scalar_count(const ustat_plan_t *plan, int *count);
int ustat_eval_rows(ustat_plan_t *plan, int rank, int n_ranks, const void *X, int x_dtype, int64_t n, int d,
                    const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes, void *stream,
                    double *scal_out);
int ustat_combine(const ustat_plan_t *plan, const double *scal, int64_t n, void *stream, double *U_out,
                  double *V_out);

/* Treewidth-3 steps in the split modes run their GEMMs on a second stream that
 * each host thread creates (with two events) at its first such evaluation on a
 * device: on a new thread, make that first call before any stream capture. */

/*
 * Device status of the last evaluation that used workspace ws on stream: waits for
 * the stream, reads the workspace's error word (its first 4 bytes) and sets
 * *device_status to
 *   USTAT_OK,
 *   USTAT_ERR_DEVICE_TIMEOUT when a bounded device wait (an mbarrier wait of the
 *     tensor-core GEMM) gave up, or else
 *   USTAT_ERR_NONFINITE when an input value read by the evaluation (X, MATRIX or
 *     VECTOR data, the TANH_DOT weights through x . w) is NaN or infinite: the
 *     paper's U-statistic is a finite sum of finite terms (Section 2.1,
 *     Definition "U-Statistic"), which such an input has not.
 * In both error cases that evaluation's U and V are NaN.  Host call; blocks until
 * the stream's work is done.  Errors: USTAT_ERR_INVALID_ARG for a NULL ws or
 * device_status, USTAT_ERR_CUDA.
 */
int ustat_status(const void *ws, void *stream, int *device_status);

/*
 * Memory-lean evaluation.  The tensorization step stores each pairwise factor as an
 * n x n matrix and the products read it (the O(K n^2) space of Section 3.3's remark
 * on space complexity and of the appendix "A Discussion on the Space Complexity").
 * ustat_eval_lean stores no n x n object: the factor's rows are rebuilt from X in
 * panels of panel_rows rows, and every product runs panel pair by panel pair on
 * them, so the workspace is O(panel_rows x n) (a time-space trade: the factor rows
 * of the column panels are rebuilt once per row panel).  Same results as ustat_eval
 * (the same digits and per-entry accumulation; the reductions summed in another
 * order).  Supported: bf16x3 plans whose n^2 objects are RBF factors (d <= 256)
 * read only by s = 2 products that store nothing (for instance the triangle and the
 * 4-cycle; USTAT_ERR_UNSUPPORTED otherwise).
 *   panel_rows : a positive multiple of 128 (capped at n rounded up to 128)
 *   ws         : device, ustat_lean_workspace_bytes() bytes, 256-byte aligned
 * Other arguments, outputs, status word and errors as ustat_eval.
 */
int ustat_lean_workspace_bytes(const ustat_plan_t *plan, int64_t n, int d, int64_t panel_rows, size_t *bytes);
int ustat_eval_lean(ustat_plan_t *plan, const void *X, int x_dtype, int64_t n, int d,
                    const ustat_factor *factors, int n_factors, int64_t panel_rows, void *ws, size_t ws_bytes,
                    void *stream, double *U_out, double *V_out);

/*
 * The n x n matrix of one device-built factor, for a caller that evaluates several
 * U-statistics over the same factor (the distance matrices of Section 4.3's
 * distance-covariance example enter four U-statistics each): build it once here
 * and pass it to those evaluations as a USTAT_MATRIX factor.  Same definition and
 * arithmetic as the factor inside ustat_eval (the tensorization step of
 * Section 3.2: the factor tensor formed from the sample):
 *   kind  : USTAT_DIST (F(i,j) = ||y_i - y_j||, float64 coordinate differences),
 *           USTAT_LOWRANK (F(i,j) = sum_k P(i,k) Q(j,k), float64 products),
 *           USTAT_GRAM (F(i,j) = sum_k P(i,k) P(j,k)) or USTAT_COMPLEMENT
 *           (F = 1 - A); param and data as in ustat_factor
 *           (device float64, row-major)
 *   F     : device float64 n x n, row-major, every entry written (the diagonal too)
 *   ws    : device, at least 256 bytes, 256-byte aligned: its first word is reset
 *           and then collects the device status (non-finite data: NONFINITE),
 *           read by ustat_status(ws, stream, ...)
 * Asynchronous on stream; the caller owns every buffer.  Errors: INVALID_ARG
 * (another kind, a NULL pointer, ws not 256-byte aligned, n < 1, for DIST /
 * LOWRANK / GRAM a param that is not an integer in [1, 4096]), UNSUPPORTED (n > 2^20),
 * CUDA.
 */
int ustat_factor_matrix(int kind, double param, const double *data, int64_t n, double *F, void *ws,
                        void *stream);

/*
 * Test hook of the bounded device waits, off by default; not for production use.
 * Every later tensor-core GEMM launched by this process gives up a wait after
 * limit_cycles SM cycles (0 restores the default of about 4e9 cycles, two
 * seconds) and, with stall_producer != 0, issues no TMA copy at all, so that its
 * first wait runs out with nothing in flight: the evaluation then reports
 * USTAT_ERR_DEVICE_TIMEOUT through ustat_status and NaN results, and a later
 * evaluation with the hook off, on the same workspace, is correct again.  The
 * setting is process-wide (not per thread); set it with no evaluation in flight.
 * Errors: USTAT_ERR_INVALID_ARG for a negative limit.
 */
int ustat_debug_set_wait(long long limit_cycles, int stall_producer);

/*
 * Same computation with host inputs and outputs: X_host (n x d, x_dtype) is
 * copied into the workspace, factor data stay device pointers, and U_host[2] /
 * V_host[n_parts] (may be NULL) receive the results.  The workspace must hold
 * ustat_workspace_bytes() + ustat_host_staging_bytes().  Synchronises the stream.
 */
int ustat_host_staging_bytes(const ustat_plan_t *plan, int64_t n, int d, size_t *bytes);
int ustat_eval_host(ustat_plan_t *plan, const void *X_host, int x_dtype, int64_t n, int d,
                    const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes,
                    void *stream, double *U_host, double *V_host);

/*
 * Many independent samples, one plan, one after another on `stream`: sample i
 * has n[i] rows at X[i] (device, row-major, x_dtype), dimension d; results at
 * U_out[2*i], V_out[i*n_parts].  One workspace region sized for max(n) is
 * reused by every sample (ustat_batch_workspace_bytes).  Factor data are
 * shared by all samples.  The concurrent, graph-captured form is the
 * ustat_batched_* object below.
 */
int ustat_eval_batch(ustat_plan_t *plan, const void *const *X, int x_dtype, const int64_t *n,
                     int count, int d, const ustat_factor *factors, int n_factors, void *ws,
                     size_t ws_bytes, void *stream, double *U_out, double *V_out);
int ustat_batch_workspace_bytes(const ustat_plan_t *plan, const int64_t *n, int count, int d,
                                size_t *bytes);

/*
 * Batched evaluation object: one plan over `count` independent samples of
 * uneven size n[i] (dimension d), evaluated concurrently.  The paper treats one
 * sample at a time; batching is this engine's.
 *
 * Schedule.  Samples are spread over `lanes` CUDA streams (lanes <= max_lanes)
 * by longest-processing-time first on the plan's flop count at n[i]; each lane
 * runs its samples in order in its own workspace region, so small samples of
 * one lane overlap large samples of another.  The lanes fork from and join
 * back into the caller's stream with events.
 *
 * Graph.  ustat_batched_capture records one whole batched evaluation (every
 * sample, every partition, every lane) into a CUDA graph bound to the given X,
 * factor and output pointers; ustat_batched_replay launches that graph on a
 * stream (one host call per batch).  Capture needs a stream other than the
 * legacy default stream and per-operation profiling off.
 *
 * Autotuning.  ustat_batched_autotune times the batch (eagerly, synchronising
 * `stream`) for each lane count in {1, 2, 4, ...} <= max_lanes and for each
 * tensor-core GEMM tile variant per size class, keeps the fastest, stores the
 * GEMM choices in the plan (used by every later evaluation with that plan) and
 * returns the chosen lane count and time.  Re-capture after autotuning.
 *
 * Ownership and errors.  The object keeps a pointer to `plan` (which must
 * outlive it), its own copy of n[], its streams, events and graph.  The caller
 * owns X, factors, the workspace (ustat_batched_workspace_bytes, for
 * max_lanes lanes, 256-byte aligned) and U_out[2*count], V_out[count*n_parts].
 * Factor kinds with per-sample data (MATRIX, VECTOR) are rejected
 * (USTAT_ERR_UNSUPPORTED); n[i] < m gives USTAT_ERR_N_LT_M.  Streams are
 * created on the device current at the first run.
 */
/*
 * Kernel variant of a plan for one size class (0: n <= 1024, 1: <= 2048, 2: <= 3072,
 * 3: larger; -1: all): bits 0-1 pick the tensor-core GEMM's tile raster group (8,
 * 4, 16 or 2 tile rows), bits 2-3 its tile shape (0: 128 x 128 with 128-byte
 * k-blocks; 1: 128 x 64, bf16x3 only; 2: 128 x 128 with 64-byte k-blocks and a
 * deeper pipeline), bit 5 the RBF kernel-matrix build in the float32-storage
 * modes (0: squared distances from the Gram matrix X X^T on the tensor cores;
 * 1: direct differences on the CUDA cores), bit 4 the latter's tile (0: 128 x 128
 * with 256 threads; 1: 64 x 64 with 128 threads), bit 6 the treewidth-3 GEMMs of
 * BF16X4 (0: two double-buffered accumulator sets and a float32 epilogue; 1: the
 * four-accumulator layout of the float64-storage modes), bit 7 turns off the diagonal
 * correction of the split-mode products (faster where diagonals do not dominate,
 * less accurate where they do; the autotuner never sets it).  Results agree to the mode's
 * tolerance across variants (summation orders differ).  The autotuner below
 * sets these itself.
 */
int ustat_plan_set_variant(ustat_plan_t *plan, int size_class, int variant);

typedef struct ustat_batched ustat_batched_t;
int ustat_batched_create(ustat_plan_t *plan, const int64_t *n, int count, int d, int max_lanes,
                         ustat_batched_t **out);
void ustat_batched_destroy(ustat_batched_t *b);
int ustat_batched_workspace_bytes(const ustat_batched_t *b, size_t *bytes);
/* lanes in use; lane_of[i] (may be NULL) receives sample i's lane */
int ustat_batched_info(const ustat_batched_t *b, int *lanes, int *lane_of);
int ustat_batched_set_lanes(ustat_batched_t *b, int lanes);
/*
 * Grouped form (bf16x3 plans; grouped = 1 on, 0 back to the lane form): every
 * sample gets its own workspace region (ustat_batched_workspace_bytes grows to
 * the sum of the samples' workspaces plus the group images), the plan runs step
 * by step over all samples, and each s = 2 product step is ONE persistent
 * tensor-core launch over the tiles of all samples' products (largest samples
 * first), each sample's reductions added to its own scalars; the other steps run
 * per sample on the lanes.  The group images (per sample: tensor maps and product
 * arguments, in the workspace) are written by the first run or capture on a
 * workspace, and again when the workspace or a variant changes: that call copies
 * them from the host and synchronises the stream, before any capture.  Drops a
 * captured graph.  Same results as the lane form up to the order of the
 * reductions' float64 additions.  Errors: UNSUPPORTED for other precisions.
 */
int ustat_batched_set_grouped(ustat_batched_t *b, int grouped);
int ustat_batched_run(ustat_batched_t *b, const void *const *X, int x_dtype, const ustat_factor *factors,
                      int n_factors, void *ws, size_t ws_bytes, void *stream, double *U_out, double *V_out);
int ustat_batched_capture(ustat_batched_t *b, const void *const *X, int x_dtype,
                          const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes,
                          void *stream, double *U_out, double *V_out);
int ustat_batched_replay(ustat_batched_t *b, void *stream);
int ustat_batched_autotune(ustat_batched_t *b, const void *const *X, int x_dtype,
                           const ustat_factor *factors, int n_factors, void *ws, size_t ws_bytes,
                           void *stream, double *U_out, double *V_out, int *lanes_out, double *ms_out);

/*
 * Learned elimination-order ranker.  The paper picks each Einsum's summation
 * order with opt_einsum's greedy or dp search (Section 3.2; Appendix F compares
 * the two).  This engine's exhaustive and min-fill planners are the fallback and
 * the reference; the ranker is a small MLP cost model, trained on measured
 * times that the planner's own candidates produce, that picks per partition the
 * candidate of least predicted time.
 *
 * Candidates.  ustat_order_candidates lists the distinct feasible elimination
 * sequences of partition `part` (restricted-growth-string index; -1 = the
 * finest partition, i.e. the kernel graph's own contraction) with
 * USTAT_RANK_FEATURES float features each (log2 n and its square; counts of the
 * step kinds the sequence lowers to in isolation, of its symmetric n^3
 * products, of all its steps and of its stored n x n intermediates; the
 * Hadamard terms read; log2 of its flop count, of its n^3 and n^4 parts; the
 * quotient's size).  Writes
 * min(*count, max_cand) rows: orders[i*m ..] (block ids, -1 padded) and
 * features[i*USTAT_RANK_FEATURES ..].  Host only.
 *
 * ustat_plan_contraction: a plan that evaluates only the finest partition's
 * V-statistic (the other V_pi are reported as 0 and U is not the U-statistic)
 * along `order` (m vertex ids; NULL = the planner's choice); the timing target
 * of the ranker's training data.  Host only.
 *
 * MLP.  F = features inputs, two hidden ReLU layers of `hidden` units, one
 * output; float32 parameters in one device array of ustat_mlp_param_count
 * entries [W1 (hidden x F, row-major), b1, W2 (hidden x hidden), b2, w3, b3].
 * ustat_mlp_forward: y[r] for the rows of X (rows x F, device).
 * ustat_mlp_loss_grad: *loss = mean_r (y[r] - target[r])^2 and grad = its
 * gradient w.r.t. the parameters (both device, overwritten); needs
 * ustat_mlp_workspace_bytes of 256-byte aligned device workspace.
 * ustat_mlp_adam: one Adam step (Kingma and Ba) at step number `step` >= 1,
 * updating params, m and v in place.  F <= 32 and hidden <= 64.
 *
 * ustat_plan_learned: plan the U-statistic with, for every partition, the
 * candidate of least predicted time under `params` (hidden units `hidden`,
 * F = USTAT_RANK_FEATURES) at sample size n.  The features go through `ws`
 * (ustat_rank_workspace_bytes, device) and the forward kernel runs on `stream`,
 * which the call synchronises.  The rest of the planning (sharing, fusion) is
 * as for ustat_plan.
 */
#define USTAT_RANK_FEATURES 20
int ustat_order_candidates(const ustat_graph *graph, const ustat_options *opts, int64_t n, int part,
                           int max_cand, int *count, int *orders, float *features);
int ustat_plan_contraction(const ustat_graph *graph, const ustat_options *opts, const int *order,
                           ustat_plan_t **out);
/* the features of one given order of partition `part` (order: its block ids,
 * -1 padded to m); and the order a plan chose for every partition
 * (orders[n_parts*m], -1 padded; -1 rows for partitions not evaluated) */
int ustat_order_features(const ustat_graph *graph, const ustat_options *opts, int64_t n, int part,
                         const int *order, float *features);
int ustat_plan_orders(const ustat_plan_t *plan, int *orders);
int ustat_mlp_param_count(int features, int hidden);
int ustat_mlp_workspace_bytes(int features, int hidden, int rows, size_t *bytes);
int ustat_mlp_forward(const float *params, int features, int hidden, const float *X, int rows, float *y,
                      void *stream);
int ustat_mlp_loss_grad(const float *params, int features, int hidden, const float *X, const float *target,
                        int rows, void *ws, size_t ws_bytes, float *grad, float *loss, void *stream);
int ustat_mlp_adam(float *params, const float *grad, float *m, float *v, int count, float lr, float beta1,
                   float beta2, float eps, int step, void *stream);
int ustat_rank_workspace_bytes(const ustat_graph *graph, const ustat_options *opts, size_t *bytes);
int ustat_plan_learned(const ustat_graph *graph, const ustat_options *opts, int64_t n, const float *params,
                       int hidden, void *ws, size_t ws_bytes, void *stream, ustat_plan_t **out);

/*
 * Evaluation that allocates nothing: for callers that must not call cudaMalloc
 * (or any allocating routine) at evaluation time.  Examples are a service that
 * reserves all its device memory at start-up and forbids allocation afterwards;
 * a plug-in running inside a framework whose caching allocator owns the device
 * memory, so that a cudaMalloc behind its back can fail or fragment the pool;
 * and code on a latency-critical path, where an allocation may stall or
 * synchronise the device.
 *
 * Instead of a caller-supplied workspace, this call uses one scratch array of
 * USTAT_NOALLOC_MAX_BYTES that the library defines in device memory.  A GPU
 * holds that array from the moment the driver loads the library's device code
 * there (at the latest during the first call on that device) until the process
 * exits.  The caller still passes X, the factors and the outputs (as for
 * ustat_eval).
 *   - Returns USTAT_ERR_WORKSPACE (and writes nothing) when the workspace this
 *     evaluation needs, ustat_workspace_bytes(plan, n, d), exceeds
 *     USTAT_NOALLOC_MAX_BYTES.
 *   - The first call on a device is its set-up: it looks up the array's device
 *     address for that device (the device must be current), which may load the
 *     library's device code; make that first call before any stream capture.
 *   - All calls share the one array, which keeps the previous call's contents;
 *     the call clears what must start at zero itself.  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on the
 *     array: order them on one stream or synchronise between them.
 * The paper has no counterpart: this is a deployment variant of ustat_eval.
 */
#define USTAT_NOALLOC_MAX_BYTES (64u * 1024u * 1024u)
int ustat_eval_noalloc(ustat_plan_t *plan, const void *X, int x_dtype, int64_t n, int d,
                       const ustat_factor *factors, int n_factors, void *stream, double *U_out,
                       double *V_out);

/*
 * ustat_status for ustat_eval_noalloc, whose callers never see the scratch
 * array's device address: waits for `stream` and reads the error word of the
 * current device's array (the status of the last no-allocation evaluation on
 * this device).  USTAT_OK when no such evaluation has run on this device yet.
 * Errors: USTAT_ERR_INVALID_ARG (NULL device_status), USTAT_ERR_CUDA.
 */
int ustat_noalloc_status(void *stream, int *device_status);

/*
 * Per-operation timing for measurement.  While enabled (per host thread), every
 * device operation launched by ustat_eval on that thread is bracketed by a pair
 * of CUDA events on the evaluation stream.  ustat_profile_collect() waits for
 * the recorded events, adds their durations per operation kind into
 * ms[kind] and the kernel launches they made into launches[kind] (one per
 * operation, two per batch of a treewidth-3 step; arrays of ustat_profile_kinds()
 * entries, may be NULL), names the kinds through ustat_profile_kind_name(), and
 * resets the record.  Events are created once and reused; no device memory is
 * allocated.
 */
int ustat_profile_enable(int enable);
int ustat_profile_kinds(void);
const char *ustat_profile_kind_name(int kind);
int ustat_profile_collect(double *ms, int *launches);

/* The last CUDA error string seen by the library in this thread ("" if none). */
const char *ustat_last_cuda_error(void);
const char *ustat_strerror(int code);
/* Library version string. */
const char *ustat_version(void);

#ifdef __cplusplus
}
#endif
#endif /* USTAT_H */
