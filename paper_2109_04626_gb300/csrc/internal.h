// internal.h -- device-state layouts and launch wrappers shared by the
// translation units of libfastpc (not part of the public C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cuda_bf16.h>

namespace fpc {

constexpr unsigned long long KEY_NONE = ~0ull;
constexpr double DEGEN = 1e-12;        // degeneracy floor on conditional variances
constexpr int MAXP = 4096;             // largest p a handle accepts
constexpr int MAXP_BATCH = 32768;      // largest total p of a batched handle
constexpr int KC_MAX = 8;              // largest dropped-set size of the complement path
constexpr int PREC_MAX = 168;          // largest neighbourhood (|adj(u)|+1) kept as a precision block

// Device counters (one per handle), reset per pc_skeleton call.
struct DevCounters {
    unsigned long long tests_executed;
    unsigned long long tests_canonical;
    unsigned long long redecided;
    unsigned long long band_hits;
    unsigned long long guard_hits;
    unsigned long long degenerate;
    unsigned long long complement_tests;
    unsigned long long edges_removed;
    unsigned long long pool_len;       // sepset pool fill
    unsigned long long flops;          // FP32 direct-test arithmetic (2 per FMA)
    unsigned long long flops64_direct; // FP64 direct tests (re-decisions or FP64 mode)
    unsigned long long flops_comp;     // complement tests (FP64)
    unsigned long long flops_prec;     // neighbourhood precision builds and downdates (FP64)
    unsigned long long flops_stagea;   // closed-form stage l = p-2 (FP64)
    unsigned int max_dz_bits;          // float bits of max |z32 - z64|
    int status;                        // device-side error (pc_status value)
    int queue_overflows;               // stages whose FP64 re-decision queue overflowed
    unsigned long long prec_downdates; // neighbourhood blocks downdated
    unsigned long long prec_builds;    // neighbourhood blocks built
};

// Per-stage scalars: the stage index lives on the device so that the whole
// stage loop can run without host round trips (CUDA graph, conditional WHILE).
struct LevelInfo {
    int l;                              // stage being run
    int lstar;                          // max |adj(u)\{v}| over adjacent ordered pairs
    long long n_opairs;                 // adjacent ordered pairs
    unsigned long long total_direct;    // tests scheduled on the direct path
    unsigned long long total_comp;      // tests scheduled on the complement path
    unsigned long long edges;           // sum of degrees (2 x unordered edges)
    int n_build;                        // neighbourhood precision blocks to build
    int saturated;                      // a test count saturated 2^64
    int done;                           // the stage schedule has finished
    int halt;                           // stop the device loop (need_host | error | overflow)
    int need_host;                      // this stage needs a direct launch sized by the host
    int error;                          // pc_status of a device-detected error
    int pool_overflow;                  // the sepset pool was too small
    int levels_run;                     // stages visited (the closed-form l = p-2 included)
    int first_level;                    // first enumerated stage (-1: none)
    int stage_a_ran;                    // the closed-form stage l = p-2 ran
    int body_runs;                      // executions of the stage body (kernel accounting)
    int lane_rounds;                    // rank-major rounds of the small-stage kernel
    int lane_overflow;                  // the FP64 re-decision queue overflowed this stage
    int kernels_run;                    // kernels the captured stage loop executed
    unsigned deg_ticket;                // CTAs of the stage's degrees kernel done (last one runs the tail)
    unsigned long long node_next;       // next work item of the staged small-stage kernel
    unsigned long long pair_next;       // next ordered pair of the warp-per-pair kernel
};

// Conditional nodes of the captured stage body: the head kernel picks one branch
// of a switch over the stage's test kernels (stage_branch below); the tail
// kernel decides the precision-block updates.
struct StageConds {
    cudaGraphConditionalHandle tests, prec;
    int use;                            // 1 inside the captured stage body
    int has_comp, has_score, has_prec;  // which kernels the body has
};
constexpr int LANE_LMAX = 12;           // stages the lane-per-test kernel runs (FP32 modes)
// Staged small-stage kernel: a node whose frozen degree is at most NODE_DMAX has
// the block corr[adj(u), adj(u)] staged in shared memory by the CTA that runs
// its pairs; larger neighbourhoods stay on the kernel that reads corr from L2.
constexpr int NODE_DMAX = 128;
constexpr int NODE_THREADS = 256;
constexpr unsigned long long NODE_ITEM_CHUNKS = 512;    // chunks per work item (two per thread)
constexpr int NODE_ROUNDS_MAX = (int)NODE_ITEM_CHUNKS / 2 + 1;   // rank rounds an item spans (degree >= 2)
// Stages 1 <= l <= PAIRWARP_LMAX: the pairs of nodes of degree above
// pair_warp_dmin (default PAIRWARP_DMIN) run one warp per ordered pair, the
// lanes on consecutive sets of the pair.
constexpr int PAIRWARP_LMAX = 2;
constexpr int PAIRWARP_DMIN = 32;
constexpr int LANE_RANGES = 6;          // small-stage kernel instantiations: l 0-2, 3-4, 5-6, 7-8, 9-10, 11-12

// Branches of the stage's switch node.  kind: 0 .. LANE_RANGES-1 a small-stage
// kernel range, STAGE_KIND_DIRECT the warp-per-test kernel, STAGE_KIND_NONE
// neither; comp: the complement kernel as well; score: the proposal's scoring
// kernels first.  Only combinations with work have a branch, in four blocks:
// (comp 0, score 0) kinds but NONE, (comp 1, score 0) every kind, then with
// scoring (kinds but NONE) comp 0 and comp 1; blocks a handle cannot use
// (no complement or no proposal) are left out.  One switch node replaces a
// chain of four conditional nodes, each of which sat on the stage's critical path.
constexpr int STAGE_KIND_DIRECT = LANE_RANGES, STAGE_KIND_NONE = LANE_RANGES + 1;
__host__ __device__ inline int stage_branches(int has_comp, int has_score)
{
    const int k0 = LANE_RANGES + 1, k1 = LANE_RANGES + 2;
    return k0 + (has_comp ? k1 : 0) + (has_score ? k0 * (has_comp ? 2 : 1) : 0);
}
// Branch index of (kind, comp, score); stage_branches(...) when nothing runs.
__host__ __device__ inline int stage_branch(int kind, int comp, int score, int has_comp, int has_score)
{
    const int k0 = LANE_RANGES + 1, k1 = LANE_RANGES + 2;
    comp = comp && has_comp;
    score = score && has_score && kind != STAGE_KIND_NONE;
    if (kind == STAGE_KIND_NONE && !comp) return stage_branches(has_comp, has_score);
    if (!score) return comp ? k0 + kind : kind;
    return k0 + (has_comp ? k1 : 0) + (comp ? k0 : 0) + kind;
}
// kernels of a stage outside conditional nodes: head, commit, degrees + tail (one kernel)
constexpr int STAGE_FIXED_KERNELS = 3;
// the stage loop in one cooperative kernel (reversed order, complement-only stages)
constexpr int LOOP_THREADS = 256;
constexpr int LOOP_PMAX = 128;          // largest p it runs (its shared memory holds a p+1 block)
constexpr int LOOP_MMAX = 14;           // direct tests it runs: l + 2 <= LOOP_MMAX
constexpr unsigned long long LOOP_DIRECT_ROUNDS = 16;   // ... and at most this many per warp of its grid

// Everything the stage kernels need, by value.
struct GraphDev {
    int p;
    int W;                      // 32-bit words per adjacency row
    uint32_t *adj;              // p x W bitset
    int *deg;                   // p
    int *dchg;                  // p: neighbours the last degree pass found deleted (old - new degree)
    int *nbr;                   // p x p, ascending neighbour ids of the frozen graph
    long long *ooff;            // p+1, exclusive scan of deg (ordered-pair offsets)
    int *opu;                   // per ordered pair: its node u (stages of the small-stage kernel)
    unsigned long long *tn_off; // p+1: first direct test of each node (exclusive scan)
    unsigned long long *cn_off; // p+1: first complement test of each node
    unsigned long long *rn_off; // p+1: first remainder test of each node (small-stage kernel)
    unsigned long long *ia_off; // p+1: staged small-stage kernel, first items: one per staged node
    unsigned long long *it_off; // p+1: staged small-stage kernel, the nodes' further items
    unsigned long long *wo_off; // p+1: warp-per-pair kernel, first ordered pair of each of its nodes
    unsigned long long *best;   // p x p, best (side<<62 | rank) per unordered pair (a<b at a*p+b)
    const unsigned long long *binom;   // ldb x ldb saturating binomials
    int ldb;                    // p+1 (batched problems: largest instance p + 1)
    // batched problems (one handle over independent instances, block-diagonal):
    // the node range [blk_lo[u], blk_hi[u]) of u's instance; null for one problem
    const int *blk_lo, *blk_hi;
    const long long *nvec;      // batched problems: samples of each node's instance
    // batched problems: per-pair arrays (best, sep_*, prec_pos, c64 flags) and the
    // correlation matrices hold only the diagonal blocks, packed; pair (a, c) of one
    // instance is at prow[a] + c and the neighbour list of a at nrow[a].  Null for
    // one problem: a * p + c (a * ldc + c for the correlation matrices).
    const long long *prow, *nrow;
    unsigned char *scored;      // learned order: per stage, 1 if its sets ran in the proposed order
    int *sep_level;             // p x p (a<b at a*p+b), -1 none
    int *sep_side;
    long long *sep_rank;
    long long *sep_off;
    int *pool;                  // explicit sepsets
    long long pool_cap;
    // neighbourhood precision blocks (reversed order, complement path)
    double *prec;               // p x PREC_MAX x PREC_MAX
    int *prec_m;                // p: block size (0 = invalid)
    int *prec_mem;              // p x PREC_MAX: member node ids (ascending, u included)
    short *prec_pos;            // p x p: slot of node w in block u, -1 = absent/dead
    int *prec_need;             // p: build request flags
    // learned proposal (optional): per node, the first score row of its
    // candidates (pair j, position x) and, per row, the candidate at each place
    // of the proposal order as its index into nbr[u]
    unsigned long long *row_off;   // p+1 (nullptr: plain lexicographic order)
    const short *perm;
    long long rows_cap;
    LevelInfo *info;
    DevCounters *ctr;
};

struct TestParams {
    long long n;        // samples
    const long long *nvec;  // batched problems: samples of each node's instance (null: n)
    const long long *prow;  // batched problems: packed row bases of the correlation blocks
    double q;           // threshold Phi^{-1}(1-alpha/2)
    float qf;
    const double *rq_tab;   // stage l -> tanh(q / sqrt(n - l - 3)) (one problem's n), formed on the host
    double band;        // |z - q| band for FP64 re-decision
    double guard;       // pivot guard
    float eps_c;        // bound on |C32 - corr| (FP32 GEMM or cast: 2^-23; BF16x3 tensor cores: 1e-6)
    float dr_max;       // largest FP32 error bound on r trusted without FP64: 5e-6 where r is
                        // returned (raw tests); no limit where only the decision is (skeleton)
    // launch shape (autotuned; results do not depend on them)
    int lane_chunk;     // consecutive sets of one pair per thread in the small-stage kernel
    int lane_rounds;    // rank-major chunk rounds before the pair-major remainder
    int lane_blocks;    // CTAs of 256 threads per SM of the small-stage kernel
    int direct_warps;   // at most this many warps per CTA of the warp-per-test kernel
    int lane_stages;    // 1: stages l <= LANE_LMAX on the small-stage kernel (FP32 modes);
                        // 0: every stage on the warp-per-test kernel
    int node_dmax;      // stages 1 <= l <= LANE_LMAX: nodes of degree <= node_dmax run on the
                        // staged kernel (corr block in shared memory); 0: none
    int pair_warp;      // stages 1 <= l <= PAIRWARP_LMAX: the pairs of nodes of degree above
                        // pair_warp_dmin one warp per pair (0: off)
    int pair_warp_dmin;
    int precision;      // 0 fp64, 1/2 fp32 tests with FP64 re-decision
    int comp_fp32;      // complement tests in FP32 first, FP64 where the bound does not decide
    int reversed;
    int complement;
    // lazily filled FP64 correlations: entry (a,b) of C64 is valid once
    // c64_valid[a*p+b] is set; a missing entry is the warp's dot product of
    // the FP64 standardised columns a and b divided by n
    int lazy;
    int p;
    double learned_min;  // a stage is scored only if it schedules at least this many tests
    double learned_ratio;  // ... and at least this many tests per score row
    int learned_lmax;      // ... and its l is at most this
    const double *xs64;
    long long ldk;
    unsigned char *c64_valid;   // 0 missing, 1 valid, 2 claimed by c64_collect (allocated in whole words)
    int2 *c64_list;             // pairs (a < b) claimed for c64_fill
    unsigned long long *c64_list_len;
    unsigned long long c64_list_cap;
    unsigned char *pair_seen;   // per tested pair: its first queued test of the stage claimed (whole words)
    unsigned long long pair_seen_bytes;
};

// counts kernel launches (defined in fastpc_api.cu); inside a stream capture the
// count is remembered per captured body instead
void note_launch();

// ---- correlation (corr.cu)
cudaError_t launch_col_stats(const void *X, int dtype, long long n, int p, long long ld,
                             double *mean, double *rsd, cudaStream_t s);
cudaError_t launch_col_stats_split(const void *X, int dtype, long long n, int p, long long ld,
                                   double *mean, double *rsd, double *ws, cudaStream_t s);
size_t col_stats_ws_bytes(long long n, int p);
// stats_ws: the workspace launch_col_stats_split filled for the same X (FP32
// input reads the float splits of mean and 1/sd from it)
cudaError_t launch_standardize(const void *X, int dtype, long long n, int p, long long ld,
                               const double *mean, const double *rsd, const double *stats_ws, double *Xs64,
                               float *Xs32, uint16_t *Xhi, uint16_t *Xlo, long long ldk,
                               cudaStream_t s);
cudaError_t launch_syrk_f64(const double *Xs, long long n, long long ldk, int p, double *C64,
                            int ldc, double *ws, size_t ws_bytes, cudaStream_t s);
size_t syrk_f64_ws_bytes(long long n, int p);
cudaError_t launch_syrk_f32(const float *Xs, long long n, long long ldk, int p, float *C32,
                            int ldc, cudaStream_t s);
cudaError_t launch_c64_lazy_init(double *C64, int ldc, unsigned char *valid, int p, cudaStream_t s);
cudaError_t launch_cast_c(const double *C64, float *C32, int p, int ldc, cudaStream_t s);
cudaError_t launch_c64_lazy_init_block(double *C64, int ldc, unsigned char *valid, int P, int o, int pb,
                                       cudaStream_t s);
cudaError_t launch_cast_block(const double *C64, float *C32, int ldc, int o, int pb, cudaStream_t s);
bool tc_gemm_available();
cudaError_t launch_corr_bf16x3(const uint16_t *Xhi, const uint16_t *Xlo, long long n, long long ldk,
                               int p, float *C32, int ldc, float *ws, size_t ws_bytes, int *err,
                               cudaStream_t s);
size_t corr_bf16x3_ws_bytes(long long n, int p);

// ---- stage l = p-2 (stage_a.cu)
cudaError_t launch_inverse_spd(double *A, int m, int lda, double *work, int *singular,
                               cudaStream_t s);
cudaError_t launch_stage_a_decide(const double *P, int p, int ldp, const int *singular,
                                  GraphDev g, TestParams tp, cudaStream_t s);

// ---- stage kernels (level.cu); they read the stage index from info->l and
// return at once when info->done or info->halt is set
constexpr int LG_DIRECT = 24;          // direct-path stages a captured stage loop can run
constexpr int DIRECT_MMAX = 160;       // largest (l+2) matrix one warp holds in shared memory
cudaError_t launch_init_adj(GraphDev g, cudaStream_t s);
cudaError_t launch_level_degrees(GraphDev g, cudaStream_t s);
cudaError_t launch_tail(GraphDev g, TestParams tp, int cap, int mode, const int *stagea_singular,
                        int stagea_launched, cudaGraphConditionalHandle hc, int use_cond, StageConds sc,
                        cudaStream_t s);
cudaError_t launch_head(GraphDev g, TestParams tp, double budget, int mmax_direct, StageConds sc, cudaStream_t s);
cudaError_t launch_ci_direct(GraphDev g, TestParams tp, int mmax, const float *C32,
                             const double *C64, int ldc, cudaStream_t s);
cudaError_t launch_ci_complement(GraphDev g, TestParams tp, cudaStream_t s);
// range: one instantiation (0 .. LANE_RANGES-1) or -1 for all; prop: the
// variant for handles with a proposal network
cudaError_t launch_expand_adj(GraphDev g, uint8_t *out, cudaStream_t s);
// ---- path-restricted candidate pools (level.cu)
cudaError_t launch_pp_components(GraphDev g, int *comp, cudaStream_t s);
cudaError_t launch_pp_search(GraphDev g, TestParams tp, const double *C64, int ldc, const int *comp, int l,
                             int mode, int *maxpool, double budget, cudaStream_t s);
cudaError_t launch_pp_commit(GraphDev g, cudaStream_t s);
cudaError_t launch_ci_lane(GraphDev g, TestParams tp, const float *C32, const double *C64, int ldc,
                           unsigned long long *queue, unsigned long long qcap, unsigned long long *qlen,
                           int range, bool prop, cudaStream_t s);
int lane_range_of(int l);
cudaError_t launch_prec_update(GraphDev g, TestParams tp, const double *C64, int ldc, cudaStream_t s);
// ---- orientation, Algorithm 1 Phase II (orient.cu): arrowhead bitsets ah/at (p x W)
cudaError_t launch_orient_colliders(GraphDev g, uint32_t *ah, uint32_t *at, cudaStream_t s);
cudaError_t launch_orient_round(GraphDev g, const uint32_t *ah, const uint32_t *at, uint32_t *ah2, uint32_t *at2,
                                int *changed, cudaStream_t s);
cudaError_t launch_orient_codes(GraphDev g, const uint32_t *ah, const uint32_t *at, int8_t *out, cudaStream_t s);
// degrees of the frozen graph, then (last CTA) the stage tail of mode 0 in the same kernel
cudaError_t launch_degrees_tail(GraphDev g, TestParams tp, int cap, cudaGraphConditionalHandle hc, int use_cond,
                                StageConds sc, cudaStream_t s);
// the first stage's precision blocks seeded from the closed-form stage's inverse P
// (the downdate that follows drops the non-neighbours)
cudaError_t launch_prec_seed(GraphDev g, const double *P, int ldp, cudaStream_t s);
// the reversed order's stages of a problem of p <= LOOP_PMAX nodes in one
// cooperative kernel, from the stage the tail scheduled; returns at the first stage
// with direct tests of more than LOOP_MMAX - 2 members or that the proposal may
// score (cudaErrorCooperativeLaunchTooLarge when it cannot be
// resident).  pre: it first applies the first stage's block builds and downdates.
cudaError_t launch_stage_loop(GraphDev g, TestParams tp, const float *C32, const double *C64, int ldc,
                              double budget, int cap, int pre, cudaStream_t s);
cudaError_t launch_commit(GraphDev g, long long n_opairs_cap, int l_fixed, int explicit_sets,
                          cudaStream_t s);
size_t scan_ws_bytes(long long n);

// ---- proposal network (mlp.cu)
int mlp_nparam();
size_t mlp_pack_bytes();
cudaError_t launch_mlp_pack(const float *theta, uint8_t *wpack, cudaStream_t s);
cudaError_t launch_mlp_forward_feats(const float *feats, long long R, const uint8_t *wpack, const float *theta,
                                     float *scores, __nv_bfloat16 *h1, float *h2, int *err, GraphDev g,
                                     cudaStream_t s);
cudaError_t launch_mlp_score_stage(GraphDev g, const unsigned long long *row_off, long long rows_cap,
                                   const float *C32, int ldc, float sqn_over_q, float inv_q, const uint8_t *wpack,
                                   const float *theta, float *scores, short *perm, int *err, cudaStream_t s);
cudaError_t launch_mlp_backward_tc(const float *feats, const float *labels, const float *scores,
                                   const __nv_bfloat16 *h1, const float *h2, long long R, float inv_b,
                                   const float *theta, const uint8_t *wpack, float *grad, double *loss, int *err,
                                   cudaStream_t s);
cudaError_t launch_mlp_backward(const float *feats, const float *labels, const float *scores,
                                const __nv_bfloat16 *h1, const float *h2, long long R, float inv_b,
                                const float *theta, float *grad, double *loss, cudaStream_t s);
cudaError_t launch_adam(float *theta, const float *grad, float *m, float *v, float lr, int step, cudaStream_t s);
cudaError_t launch_mlp_features(const int *quads, long long R, const float *C32, int ldc, const long long *prow,
                                int p, long long n, const long long *nvec, double q, float *feats, int *err,
                                cudaStream_t s);
cudaError_t launch_reverify(GraphDev g, TestParams tp, const float *C32, const double *C64, int ldc, int lmax,
                            cudaStream_t s);

// ---- raw test batches (level.cu)
cudaError_t launch_ci_list(const int *ij, const int *S, int l, long long b, const float *C32,
                           const double *C64, int ldc, int p, TestParams tp, double *r_out,
                           uint8_t *indep_out, float *z_out, DevCounters *ctr, const int *blk_lo,
                           const int *blk_hi, cudaStream_t s);

}  // namespace fpc
