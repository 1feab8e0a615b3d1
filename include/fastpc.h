/*
 * fastpc.h -- C-ABI of the GB300 (sm_103a) PC-stable skeleton search of
 * "A Fast PC Algorithm with Reversed-order Pruning and A Parallelization
 * Strategy" (arXiv 2109.04626).
 *
 * Conventions shared by every entry point
 *  - Every call returns a pc_status; PC_OK is 0.  On failure the handle keeps a
 *    message readable with pc_last_error().  No C++ exception crosses the ABI.
 *  - The caller owns every buffer it passes in or out; the library owns its
 *    handle, the correlation matrices, the work queues, the sepset store and
 *    every other workspace (allocated with cudaMalloc on the current device at
 *    pc_create/pc_corr and released by pc_destroy).
 *  - Pointers documented "host or device" are classified with
 *    cudaPointerGetAttributes; host buffers are copied through pinned staging.
 *  - All GPU work is issued on the handle's stream (pc_set_stream; default the
 *    legacy default stream).  pc_corr is stream-ordered and returns without
 *    synchronising; pc_skeleton and pc_ci_batch synchronise before returning.
 *  - Matrices are row-major.  Node ids are 0..p-1.
 *  - Device-side failures (a guard queue that overflows, a bounded wait that
 *    expires) set a device status word that the next synchronising call turns
 *    into a pc_status.
 */
#ifndef FASTPC_H
#define FASTPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pc_handle pc_handle;   /* opaque, library-owned */

typedef enum {
    PC_OK = 0,
    PC_ERR_ARG = 1,      /* bad argument (null pointer, size out of range, bad key) */
    PC_ERR_CUDA = 2,     /* a CUDA runtime call failed                              */
    PC_ERR_OOM = 3,      /* device allocation failed                                */
    PC_ERR_STATE = 4,    /* call out of order (e.g. pc_skeleton before pc_corr)     */
    PC_ERR_DOF = 5,      /* n - l - 3 <= 0: the Fisher-z test is undefined          */
    PC_ERR_BUDGET = 6,   /* a stage would exceed the test budget (option "budget")  */
    PC_ERR_TIMEOUT = 7,  /* a device-side bounded wait expired                      */
    PC_ERR_INTERNAL = 8  /* a device-side consistency check failed                  */
} pc_status;

enum { PC_F32 = 0, PC_F64 = 1 };

/* Counters of one pc_skeleton call. */
typedef struct {
    uint64_t tests_executed;    /* CI tests the GPU evaluated (speculative ones included)     */
    uint64_t tests_canonical;   /* tests the sequential canonical order needs (oracle count)  */
    uint64_t tests_redecided;   /* tests re-decided in FP64 (guard or band)                   */
    uint64_t band_hits;         /* FP32 |z - q| inside the band                               */
    uint64_t guard_hits;        /* FP32 pivot ratio below the guard                           */
    uint64_t degenerate;        /* tests decided by the degeneracy rule                       */
    uint64_t complement_tests;  /* tests evaluated from a neighbourhood precision matrix     */
    uint64_t edges_removed;     /* unordered pairs removed                                    */
    uint64_t edges_kept;        /* unordered pairs in the returned skeleton                   */
    double max_abs_dz;          /* max |z_fp32 - z_fp64| over re-decided tests                */
    double t_skeleton_ms;       /* device time of the skeleton search (CUDA events)           */
    double flops;               /* arithmetic of the search, counted in the kernels (2/FMA)   */
    double flops_class[6];      /* the same split by kernel class (see pc_timing)             */
    int32_t levels_run;         /* stages visited                                             */
    int32_t stage_a_ran;        /* 1 if the l = p-2 stage ran in closed form                  */
    int32_t first_level;        /* first enumerated stage                                     */
    int32_t queue_overflows;    /* stages whose FP64 re-decision queue overflowed (each was re-run
                                   by the warp-per-test kernel; the queue grows for later runs) */
    uint64_t prec_builds;       /* neighbourhood precision blocks built (reversed order)      */
    uint64_t prec_downdates;    /* block downdates applied after deletions                    */
} pc_stats;

/* pc_create -- a handle for data of n samples over p variables, significance
 * level alpha (0 < alpha < 1) and conditioning-set cap max_level (< 0: none).
 * Sec. 2.2.2 (Fisher-z threshold Phi^{-1}(1-alpha/2)), Algorithm 1/2 inputs.
 * Requires 4 <= n <= 2^21 and 2 <= p <= 4096.  Allocates the handle's workspaces. */
pc_status pc_create(int64_t n, int32_t p, double alpha, int32_t max_level, pc_handle **out);

/* pc_destroy -- frees the handle and every library-owned allocation. */
void pc_destroy(pc_handle *h);

/* pc_set_opt / pc_get_opt -- named options (numeric values):
 *   "order"       0 = conventional (Algorithm 1, l ascending), 1 = reversed
 *                 (Algorithm 2, l descending; default)
 *   "stage_a"     1 = run the l = p-2 stage in closed form when n-p-1 > 0 (default)
 *   "precision"   0 = FP64 everywhere; 1 = FP32 SIMT correlation GEMM + FP32 tests
 *                 with FP64 re-decision; 2 = split-precision BF16x3 tensor-core
 *                 correlation GEMM + FP32 tests with FP64 re-decision (default)
 *   "band"        FP64 re-decision band on |z - q| (default 1e-3)
 *   "guard"       pivot-ratio guard: FP32 tests whose smallest Cholesky pivot is
 *                 below it are re-decided in FP64 (default 1e-3)
 *   "complement"  1 = evaluate high stages from maintained neighbourhood precision
 *                 matrices (default), 0 = direct tests only
 *   "budget"      maximum tests one stage may schedule (default 2e10)
 *   "timing"      1 = record per-kernel-class CUDA-event times (pc_timing); the
 *                 stage loop is then driven from the host, one launch per kernel
 *   "graph"       1 = run the stage loop as one CUDA graph whose conditional
 *                 WHILE node is driven by the device (default); 0 = host loop
 *   "stage_conds" 1 = inside that graph, conditional nodes skip the kernels a
 *                 stage has no work for (default); 0 = every kernel every stage
 *   "small_stage_kernel" 1 = stages l <= 12 of the FP32 modes run on the
 *                 rank-major one-thread-per-chunk kernel with bordered tests
 *                 (default); 0 = every stage on the one-warp-per-test kernel
 *   "learned"     1 = enumerate the conditioning sets of every ordered pair in
 *                 the order proposed by the scoring network (needs parameters:
 *                 pc_mlp_set_params or pc_mlp_train); 0 = lexicographic (default)
 *   "learned_rows" capacity of the per-stage score buffer in rows (default 2^24);
 *                 a stage with more candidate rows runs in lexicographic order
 *   "learned_min_tests" a stage is scored only if it schedules at least this
 *                 many tests (default 1e6); smaller stages run all their tests
 *                 in one wave, where the enumeration order saves nothing
 *   "learned_min_ratio" ... and at least this many tests per score row (one
 *                 row per candidate of a pair; default 8): at l = 1 a pair has
 *                 as many sets as candidates and scoring costs as much as testing
 *   "learned_max_level" ... and its l is at most this (default 8): a pair of a
 *                 larger stage has few candidates left, and scoring them saved
 *                 no time in the p = 1000 measurements
 * Launch shape of the test kernels (set by pc_autotune; results never depend on it):
 *   "lane_chunk"  consecutive sets of one pair per thread in the kernel of the
 *                 stages l <= 12 (1..256, default 8)
 *   "lane_rounds" chunks of every pair run rank-major (chunk r of all pairs
 *                 before chunk r+1) before the rest runs pair by pair (0..4096,
 *                 default 32)
 *   "lane_blocks" CTAs of 256 threads per SM of that kernel (1..32, default 8)
 *   "direct_warps" at most this many warps per CTA of the warp-per-test kernel
 *                 (1, 2, 4 or 8; default 8)
 *   "path_pool"   1 = search the path-restricted pools adj(G,i,j) n path(G,i,j)
 *                 of Algorithms 1 and 2 (Sec. 2.1 notation): the neighbours of
 *                 i or j, other than i and j, that lie on some simple i-j path of
 *                 the stage's frozen graph; one pool per unordered pair, searched
 *                 once, sets in lexicographic order of the ascending pool (side
 *                 0), FP64 tests, PC-stable, a host-driven stage loop; the
 *                 schedule runs on the largest pool.  0 = the neighbour sets
 *                 adj(u)\{v} of both endpoints (default).  Not with "learned" or
 *                 a batched handle.
 *   "pair_warp"   1 = at stages 1 and 2, the ordered pairs of nodes of degree
 *                 above "pair_warp_dmin" (default 32) run one warp per pair, the
 *                 32 lanes on 32 consecutive sets of the pair (default); 0 = off
 *   "node_dmax"   the other small-stage nodes of degree <= node_dmax (0..128,
 *                 default 128) run on the staged kernel, which holds
 *                 corr[adj(u), adj(u)] in shared memory; the rest read corr
 *                 from L2 (0 = staged kernel off)
 *   "stage_loop"  1 = problems of p <= 128 (not batched) run the stage loop in
 *                 one cooperative kernel, a grid-wide barrier where the captured
 *                 loop has a kernel boundary (tests, commit, degrees, next stage,
 *                 and in the reversed order the precision blocks); it runs the
 *                 complement tests and the direct tests of stages with at most
 *                 12 conditioning members and at most 16 tests per warp of its
 *                 grid, a warp each; from the first stage it does not take
 *                 (larger direct stages, or a stage the proposal may score) on,
 *                 the captured loop (default; skipped on a device without
 *                 cooperative launches).  0 = the captured loop throughout.
 *                 The results are the same either way.
 *   "comp_fp32"   1 = complement tests (reversed order) in FP32 first from the
 *                 FP64 precision blocks, decided there when a first-order
 *                 error bound with validity checks shows the FP64 decision is
 *                 the same and the statistic lies at least "band" from q, else
 *                 in FP64 (default; counted in tests_redecided, band_hits,
 *                 guard_hits); 0 = FP64 only.  Not used with "precision" 0.
 * Unknown keys return PC_ERR_ARG. */
pc_status pc_set_opt(pc_handle *h, const char *key, double val);
pc_status pc_get_opt(pc_handle *h, const char *key, double *val);

/* pc_set_stream -- cudaStream_t on which all later work is issued. */
pc_status pc_set_stream(pc_handle *h, void *stream);

/* pc_corr -- standardises the columns of X (FP64 mean and population sd) and
 * forms corr = Xs^T Xs / n with unit diagonal (Sec. 4, the matrix corr).
 * X: n x p row-major with row stride ld >= p elements, dtype PC_F32 or PC_F64,
 * host or device, caller-owned, read only.  Stream-ordered; X must stay valid
 * until the stream reaches the call. */
pc_status pc_corr(pc_handle *h, const void *X, int32_t dtype, int64_t ld);

/* pc_corr_get -- copies the correlation matrix (p x p row-major) into C32
 * and/or C64 (either may be NULL; host or device).  Synchronises. */
pc_status pc_corr_get(pc_handle *h, float *C32, double *C64);

/* pc_skeleton -- Phase I of Algorithm 2 (reversed order) or Algorithm 1
 * (conventional), PC-stable: the adjacency is frozen at the start of each
 * stage and deletions are applied at its end.  For every adjacent ordered pair
 * (u,v) and every S subset of adj(u)\{v} with |S| = l, in lexicographic order
 * (side 0: u = min(u,v) first), it tests u _||_ v | S with
 * sqrt(n-l-3)|atanh r_uv.S| <= Phi^{-1}(1-alpha/2) (Eq. 1, Sec. 2.2.2), r from
 * the Schur complement of Sec. 4.  Writes the skeleton into adj_out (p x p,
 * 0/1, symmetric, host or device; may be NULL) and the counters into stats
 * (host; may be NULL).  Sepsets stay in the handle (pc_sepsets_*).
 * Requires a prior pc_corr.  Synchronises. */
pc_status pc_skeleton(pc_handle *h, uint8_t *adj_out, pc_stats *stats);

/* pc_skeleton_many -- the skeleton searches of `count` independent problems
 * (each handle after its own pc_corr) run concurrently: every search is first
 * enqueued on its handle's stream (give each handle its own stream with
 * pc_set_stream; handles on one stream run one after the other), then each is
 * completed.  adj_out[i] (host or device, may be NULL; adj_out may be NULL),
 * stats[i] and status[i] (host, may be NULL) receive the per-problem results.
 * Returns the first failing status (each failure stays in its handle). */
pc_status pc_skeleton_many(pc_handle **hs, int32_t count, uint8_t **adj_out, pc_stats *stats,
                           pc_status *status);

/* pc_autotune -- chooses the launch shape of the test kernels for this
 * handle's problem (the data given to the last pc_corr): a coordinate search
 * over lane_chunk {4,8,16,32}, lane_rounds {4,16,64,256}, lane_blocks {4,8,16}
 * and direct_warps {2,4,8} -- and, for a handle that enumerates in the
 * proposal order ("learned" 1 with parameters), learned_max_level
 * {0 (no stage scored), 2, 4, 8}: the cost gate that keeps the scoring off
 * the stages where it costs more than the tests it saves -- each candidate
 * timed as the mean of `reps` (1..100) complete skeleton searches (CUDA events
 * on the handle's stream) after one warm run.  The handle keeps the fastest
 * shape; out (host, may be NULL) receives it with the times.  The shape
 * changes no skeleton (the proposal order changes only which separating set
 * is found first), so the handle holds a valid skeleton afterwards (as after
 * pc_skeleton).  Requires a prior pc_corr.  Not in the paper: a launch-shape
 * search for this GPU.  Errors of any run are returned as pc_skeleton returns
 * them. */
typedef struct {
    int32_t lane_chunk, lane_rounds, lane_blocks, direct_warps;
    double ms_default;  /* mean skeleton time with the shape before the search */
    double ms_best;     /* mean skeleton time with the chosen shape             */
    int32_t runs;       /* skeleton searches executed                           */
    int32_t learned_max_level;   /* the chosen option (searched only for a proposal-order handle) */
} pc_tune_result;
pc_status pc_autotune(pc_handle *h, int32_t reps, pc_tune_result *out);

/* pc_create_batch -- one handle over k independent problems (instance i: n[i]
 * samples of p[i] variables; 4 <= n[i] <= 2^21, 2 <= p[i] <= 4096, sum p[i] <=
 * 16384), all at the same alpha and max_level.  Instance i owns the global
 * node ids [off_i, off_i + p[i]), off_i = p[0] + ... + p[i-1]; its adjacency
 * starts as the complete graph on its own nodes, so every test stays inside
 * one instance and uses that instance's n in sqrt(n-l-3) (Eq. 1).  Each stage
 * of pc_skeleton is then one launch sequence over the tests of all instances;
 * the skeleton restricted to instance i equals that of a pc_create handle on
 * instance i alone.  Conventional order only (Algorithm 1; "order" 1 is
 * rejected).  Not in the paper: the paper runs one problem at a time.  Give the
 * data with pc_corr_block (pc_corr returns PC_ERR_STATE); pc_skeleton,
 * pc_sepsets_*, pc_ci_batch, pc_autotune and the pc_mlp_* calls then work in
 * global node ids (adj_out is sum p x sum p, block diagonal; the statistics
 * are totals).  pc_ci_batch rejects a test whose nodes span instances
 * (PC_ERR_ARG) and checks n-l-3 > 0 against the smallest n. */
pc_status pc_create_batch(int32_t k, const int64_t *n, const int32_t *p, double alpha, int32_t max_level,
                          pc_handle **out);

/* pc_corr_block -- pc_corr for instance i (0 <= i < k) of a batched handle: X
 * is n[i] x p[i] row-major with row stride ld >= p[i], PC_F32 or PC_F64, host
 * or device, caller-owned, read only.  Fills the diagonal block of corr of
 * instance i.  pc_skeleton needs every instance given at least once.
 * PC_ERR_STATE on a handle from pc_create, PC_ERR_ARG on a bad index. */
pc_status pc_corr_block(pc_handle *h, int32_t i, const void *X, int32_t dtype, int64_t ld);

/* pc_corr_blocks -- pc_corr_block for every instance of a batched handle in one
 * call: X[i], dtype[i], ld[i] (host arrays of k entries) as pc_corr_block's
 * arguments for instance i.  The instances' standardisation and correlation
 * GEMMs are independent (disjoint planes, disjoint diagonal blocks of corr),
 * so they run concurrently on up to 8 internal streams of the handle, each with
 * its own staging and split-K workspaces, forked from and joined back into the
 * handle's stream: the call is ordered on that stream like one pc_corr_block
 * per instance, and gives the same results.  With "precision" 0 (FP64 Gram,
 * one shared workspace) the instances run one after the other on the handle's
 * stream.  Timing class "corr" covers the whole fork and join; "corr_gemm" is
 * not recorded.  PC_ERR_STATE on a handle from pc_create, PC_ERR_ARG (nothing
 * issued) on a null array or a bad entry.  Not in the paper: it runs one
 * problem at a time. */
pc_status pc_corr_blocks(pc_handle *h, const void *const *X, const int32_t *dtype, const int64_t *ld);

/* pc_batch_layout -- the number of instances (1 for a pc_create handle) into
 * *k and, if offsets is not NULL, their first node ids plus the total
 * (k + 1 entries, host). */
pc_status pc_batch_layout(pc_handle *h, int32_t *k, int32_t *offsets);

/* pc_sepsets_count -- number of removed pairs of the last pc_skeleton and the
 * total length of their explicit sepsets (stage l = p-2 sets V\{u,v} are not
 * stored explicitly: their offset is -1). */
pc_status pc_sepsets_count(pc_handle *h, int64_t *n_removed, int64_t *pool_len);

/* pc_sepsets_get -- host buffers: pairs[2*k] = (a, b) with a < b, level[k],
 * side[k] (0: S from adj(a)\{b}, 1: from adj(b)\{a}), rank[k] (lexicographic
 * rank of S within its side), off[k] (offset into pool or -1) and pool
 * (the explicit sets, ascending node ids).  Any pointer may be NULL. */
pc_status pc_sepsets_get(pc_handle *h, int32_t *pairs, int32_t *level, int32_t *side,
                         int64_t *rank, int64_t *off, int32_t *pool);

/* pc_orient -- Phase II of Algorithm 1 (which Algorithm 2 shares, Sec. 3.3) on
 * the last pc_skeleton result and its separation sets: every unshielded triple
 * i - k - j with k not in S(i,j) becomes i -> k <- j, then rules R1-R4 are
 * applied until none orients an edge.  Order-free: all colliders are marked at
 * once and each rule round reads the marks of the round before; an edge marked
 * from both ends is bidirected.  R4 is taken with X_k and X_j non-adjacent.
 * codes_out: p x p int8, row-major, host or device, caller-owned; for the
 * ordered pair (a, b): 0 no edge, 1 a - b, 2 a -> b, 3 a <- b, 4 a <-> b (a
 * batched handle: the block-diagonal p x p matrix of all instances).
 * rounds_out (host, may be NULL): rule rounds that oriented an edge.
 * PC_ERR_STATE before pc_skeleton, PC_ERR_ARG for a NULL codes_out.  Runs on
 * the handle's stream; synchronises once per rule round. */
pc_status pc_orient(pc_handle *h, int8_t *codes_out, int32_t *rounds_out);

/* pc_ci_batch -- b raw CI tests on the current correlation matrix (the index
 * matrix B of Sec. 4 / Algorithm 3): test k is (ij[2k], ij[2k+1] | S[k*l .. k*l+l-1]).
 * Outputs r_out[k] (partial correlation), z_out[k] (sqrt(n-l-3)|atanh r|),
 * indep_out[k] (1 = independent).  Device pointers (caller-owned); any output
 * may be NULL.  Returns PC_ERR_DOF if n-l-3 <= 0, PC_ERR_ARG for ids out of
 * range or u == v.  Tests whose FP32 value is unreliable (pivot guard, |z-q|
 * band) are recomputed in FP64 from FP64 correlations.  Synchronises. */
pc_status pc_ci_batch(pc_handle *h, const int32_t *ij, const int32_t *S, int32_t l, int64_t b,
                      double *r_out, uint8_t *indep_out, float *z_out);

/* pc_last_stats -- counters of the last pc_skeleton or pc_ci_batch call (host). */
pc_status pc_last_stats(pc_handle *h, pc_stats *out);

/* pc_threshold -- q = Phi^{-1}(1 - alpha/2) as used by the handle. */
double pc_threshold(const pc_handle *h);

/* pc_fisher_threshold -- q = Phi^{-1}(1 - alpha/2) (host only, no GPU needed):
 * the two-sided normal quantile of the Fisher-z rule (Sec. 2.2.2).  Newton
 * iterations on log(erfc(x/sqrt 2)/2) = log(alpha/2).  NaN unless 0<alpha<1. */
double pc_fisher_threshold(double alpha);

/* pc_kernel_launches -- number of CUDA kernels this library has launched in
 * this process (all handles). */
int64_t pc_kernel_launches(void);

/* pc_timing -- with option "timing" = 1, the handle brackets its launches
 * with CUDA events on its stream, grouped by kernel class: 0 correlation,
 * 1 closed-form stage l=p-2, 2 neighbourhood precision builds and downdates,
 * 3 direct CI tests, 4 complement CI tests, 5 stage bookkeeping (neighbour
 * lists, counts, scans, commit), 6 proposal scoring, ordering and the FP64
 * re-test of the sepsets found in the proposal order, 7 the correlation GEMM
 * kernels alone (the tensor-core product and its split-K reduce, or the SIMT
 * Gram kernel; a part of class 0), 8 the stage loop in one kernel (option
 * "stage_loop": every class of work of the stages it runs).  Writes per-class
 * device milliseconds and launch-group counts accumulated since the last reset
 * (reset != 0 clears them afterwards).  ms and count have 9 entries; either may
 * be NULL. */
pc_status pc_timing(pc_handle *h, double *ms, int64_t *count, int32_t reset);

/* pc_corr_noalloc -- the correlation matrix without any allocation, for
 * callers that cannot call cudaMalloc: applications whose device memory is
 * reserved up front by their own pool or budget, and latency-critical loops
 * in which a cudaMalloc would synchronise the device.  The paper has no
 * counterpart; it computes what pc_corr computes in FP64 (corr = Xs^T Xs / n
 * of the FP64-standardised columns, unit diagonal), with no handle.
 *   X      device pointer, n x p row-major, row stride ld >= p, dtype PC_F32 or
 *          PC_F64 (caller-owned, read only)
 *   C_out  device pointer, p x p row-major FP64, row stride ldc >= p
 *          (caller-owned, fully written)
 *   stream cudaStream_t to issue on (NULL: legacy default stream); returns
 *          without synchronising
 * Its scratch (column means and 1/sd) is a file-scope __device__ array sized
 * for p <= 4096 (64 KiB on every GPU that loads the library, held until the
 * process exits); p > 4096, n < 2, host pointers or a bad dtype/stride return
 * PC_ERR_ARG before anything is launched; so do X or C_out on a device other
 * than the current one (make the buffers' device current before the call).  It calls no cudaMalloc, cudaFree
 * or other allocating routine.  The first call on each device looks up the
 * array's device address with that device current (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  All calls share
 * the one array: calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.  Each call
 * overwrites the statistics it uses, so nothing needs clearing between calls. */
pc_status pc_corr_noalloc(const void *X, int32_t dtype, int64_t n, int32_t p, int64_t ld,
                          double *C_out, int64_t ldc, void *stream);

/* ---- conditioning-set proposal network (no counterpart in the paper; it only
 * changes the order in which Algorithm 1/2 enumerate the sets of an edge, so
 * the skeleton is unchanged; every proposed sepset is re-verified in FP64).
 * A member score s(u,v,k) for candidate k of the ordered pair (u,v):
 *   h1 = relu(W1 x + b1) (16->128), h2 = relu(W2 h1 + b2) (128->128),
 *   s = w3 . h2 + b3; training loss mean BCE(sigmoid(s), y).
 * Parameters: one FP32 vector W1 (128x16 row-major), b1, W2 (128x128), b2, w3,
 * b3 -- pc_mlp_nparam() values.  Forward on the tensor cores in BF16 with FP32
 * accumulation.  Backward (option "mlp_backward" 1, default): the products
 * dL/dh1 = dL/da2 W2, dW2 = (dL/da2)^T h1 and dW1 = (dL/da1)^T x on the tensor
 * cores with BF16 operands (the back-propagated signals rounded to BF16) and
 * FP32 accumulation; db1, db2 sum those BF16 signals; dw3, db3 and the loss in
 * FP32; "mlp_backward" 0: the whole backward in FP32 on the CUDA cores.  Adam
 * updates FP32 master parameters. */
int32_t pc_mlp_nparam(void);
/* theta: host or device, pc_mlp_nparam() floats; resets the Adam state. */
pc_status pc_mlp_set_params(pc_handle *h, const float *theta, int64_t count);
pc_status pc_mlp_get_params(pc_handle *h, float *theta, int64_t count);
/* Features (16 floats per row, device) of R candidate rows given as device
 * quadruples (u, v, k, l | d << 16): candidate k of the ordered pair (u, v) at
 * stage l with candidate-set size d = |adj(u)\{v}|.  Needs pc_corr. */
pc_status pc_mlp_features(pc_handle *h, const int32_t *quads, int64_t R, float *feats);
/* Scores of R feature rows (device in, device out). */
pc_status pc_mlp_forward(pc_handle *h, const float *feats, int64_t R, float *scores);
/* Full-batch gradient of the mean BCE loss at the current parameters
 * (grad_out: host or device, pc_mlp_nparam() floats; loss may be NULL). */
pc_status pc_mlp_grad(pc_handle *h, const float *feats, const float *labels, int64_t R, float *grad_out,
                      double *loss);
/* Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) over contiguous mini-batches of
 * the given rows (device), `epochs` passes; final_loss = mean loss of the last
 * pass (may be NULL).  The caller shuffles the rows. */
pc_status pc_mlp_train(pc_handle *h, const float *feats, const float *labels, int64_t R, int32_t epochs,
                       int64_t batch, double lr, double *final_loss);

const char *pc_last_error(const pc_handle *h);
const char *pc_status_string(pc_status s);

#ifdef __cplusplus
}
#endif
#endif /* FASTPC_H */
