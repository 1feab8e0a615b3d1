// fastpc_api.cu -- the C-ABI of include/fastpc.h: handle, options, the
// correlation step and the host side of the stage loop (Algorithm 1 / 2).
#include "internal.h"
#include "../../include/fastpc.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using fpc::DevCounters;
using fpc::GraphDev;
using fpc::LevelInfo;
using fpc::TestParams;
typedef unsigned long long ull;

static std::atomic<long long> g_launches{0};
namespace fpc {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}

constexpr int NCLS = 9;   // class 7 (the correlation GEMM kernels) lies inside class 0
struct TimedPair {
    int cls;
    cudaEvent_t a, b;
};

// A stream and the workspaces of one correlation step (statistics partials,
// host-input staging, the tensor-core GEMM's split-K partials).
struct CorrLane {
    cudaStream_t s = nullptr;
    void *Xstage = nullptr;
    size_t Xstage_bytes = 0;
    double *stats_ws = nullptr;
    size_t stats_ws_bytes = 0;
    float *tc_ws = nullptr;
    size_t tc_ws_bytes = 0;
};

struct pc_handle {
    long long n = 0;
    int p = 0;
    double alpha = 0.01;
    int max_level = -1;
    double q = 0.0;
    // options
    int order = 1, stage_a = 1, precision = 2, complement = 1;
    double band = 1e-3, guard = 1e-3;
    double budget = 2.0e10;
    // batched problems (pc_create_batch): instance i owns nodes [boff[i], boff[i+1])
    // and the diagonal block of corr there; nblk = 0 for one problem
    int nblk = 0;
    std::vector<int> boff;
    std::vector<long long> pbase;        // first packed element of each instance's blocks
    size_t pair_elems = 0;               // entries of a per-pair array (p*p, or sum p_i^2)
    size_t c_elems = 0;                  // entries of a correlation matrix (p*ldc, or sum p_i^2)
    std::vector<long long> bn;
    std::vector<char> bdone;
    long long n_min = 0;
    // launch shape of the test kernels (pc_autotune)
    int lane_chunk = 8, lane_rounds = 32, lane_blocks = 8, direct_warps = 8;
    int node_dmax = fpc::NODE_DMAX;   // staged small-stage kernel: largest node degree (0: off)
    int comp_fp32 = 1;                // complement tests in FP32 first (FP32 modes)
    int stage_loop = 1;               // reversed order, p <= LOOP_PMAX: complement-only stages in one kernel
    int coop = -1;                    // device supports cooperative launches (-1: not asked yet)
    int pair_warp = 1;                // stages 1-2: warp-per-pair kernel for the larger nodes
    int pair_warp_dmin = fpc::PAIRWARP_DMIN;
    // path-restricted pools (option "path_pool"): component labels of the graph
    // without each node, the largest pool
    int path_pool = 0;
    // pc_corr_blocks: side streams with their own workspaces for the instances'
    // correlation steps (their planes and blocks are disjoint)
    std::vector<CorrLane> lanes;
    std::vector<cudaEvent_t> lane_ev;
    uint8_t *adj_stage = nullptr;     // the expanded skeleton for host outputs
    size_t adj_stage_bytes = 0;
    int *pp_comp = nullptr, *pp_max = nullptr;
    int stage_conds = 1;                 // conditional nodes in the captured stage body
    int lane_stages = 1;                 // small stages on the rank-major small-stage kernel
    cudaStream_t stream = 0;
    std::string err;
    // correlation
    long long ldk = 0;       // padded n (K-major planes)
    int ldc = 0;             // padded p
    double *mean = nullptr, *rsd = nullptr;
    double *Xs64 = nullptr;
    float *Xs32 = nullptr;
    uint16_t *Xhi = nullptr, *Xlo = nullptr;
    double *C64 = nullptr, *Pbuf = nullptr, *work = nullptr;
    float *C32 = nullptr, *tc_ws = nullptr;
    size_t tc_ws_bytes = 0;
    int *tc_err = nullptr;
    int *singular = nullptr;
    void *Xstage = nullptr;
    size_t Xstage_bytes = 0;
    bool have_corr = false;
    bool used_tc = false;
    // graph state
    GraphDev g{};
    ull *binom = nullptr;
    double *rq_tab = nullptr;         // per stage l: tanh(q / sqrt(n - l - 3)), the |r| threshold
    long long opair_cap = 0;
    LevelInfo *info_h = nullptr;     // pinned mirror
    DevCounters *ctr_h = nullptr;    // pinned mirror
    ull *sepcnt_h = nullptr;
    // orientation (Phase II): arrowhead bitsets, two rounds' worth, and a flag
    uint32_t *or_mk = nullptr;
    int *or_changed = nullptr;
    int8_t *or_codes = nullptr;
    bool have_skel = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    pc_stats last{};
    std::vector<void *> allocs;
    // captured stage loop (CUDA graph with a conditional WHILE node)
    int use_graph = 1;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t br_stream = nullptr;      // captures the bodies of conditional nodes
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphConditionalHandle hcond = 0;
    std::vector<double> graph_key;
    long long body_kernels = 0;      // kernel nodes in the captured stage body (all branches)
    double *syrk_ws = nullptr, *stats_ws = nullptr;
    unsigned char *c64_valid = nullptr;
    int2 *c64_list = nullptr;                  // FP64 entries claimed for the parallel fill
    unsigned long long *c64_list_len = nullptr;
    unsigned char *pair_seen = nullptr;        // per tested pair: first queued test claimed
    size_t pair_seen_bytes = 0;
    unsigned long long *rq = nullptr, *rq_len = nullptr;   // FP64 re-decision queue of the lane kernel
    unsigned long long rq_cap = 0;
    bool c64_full = false;             // C64 fully computed (else lazily, per entry)
    size_t stats_ws_bytes = 0;
    size_t syrk_ws_bytes = 0;
    // proposal network
    int learned = 0;
    float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    uint8_t *wpack = nullptr;
    int *mlp_err = nullptr;
    double *mlp_loss = nullptr;
    bool have_params = false;
    int adam_step = 0;
    unsigned long long *row_off = nullptr;
    short *perm = nullptr;
    float *stage_scores = nullptr;
    unsigned char *scored = nullptr;   // per stage: 1 if it ran in the proposed order
    long long rows_cap = 0;
    double learned_min = 1.0e6;
    double learned_ratio = 8.0;
    int learned_lmax = 8;
    int mlp_bwd_tc = 1;    // backward products on the tensor cores (BF16 operands); 0: FP32 CUDA cores
    // per-kernel-class timing
    int timing = 0;
    std::vector<TimedPair> pending;
    std::vector<cudaEvent_t> evpool;
    double cls_ms[NCLS] = {};
    long long cls_n[NCLS] = {};
};

// Brackets the launches of one kernel class with events on the handle's stream.
struct Timed {
    pc_handle *h;
    int cls;
    cudaEvent_t a = nullptr, b = nullptr;
    static cudaEvent_t get(pc_handle *h)
    {
        if (!h->evpool.empty()) {
            cudaEvent_t e = h->evpool.back();
            h->evpool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    Timed(pc_handle *h_, int c) : h(h_), cls(c)
    {
        if (!h->timing || cls < 0) return;
        a = get(h);
        b = get(h);
        cudaEventRecord(a, h->stream);
    }
    ~Timed()
    {
        if (!h->timing || cls < 0) return;
        cudaEventRecord(b, h->stream);
        h->pending.push_back({cls, a, b});
    }
};

// ---------------------------------------------------------------- helpers
static const char *kStatusNames[] = {"PC_OK",          "PC_ERR_ARG",    "PC_ERR_CUDA",
                                     "PC_ERR_OOM",     "PC_ERR_STATE",  "PC_ERR_DOF",
                                     "PC_ERR_BUDGET",  "PC_ERR_TIMEOUT", "PC_ERR_INTERNAL"};

static pc_status fail(pc_handle *h, pc_status s, const std::string &msg)
{
    if (h) h->err = msg;
    return s;
}

static pc_status cuda_fail(pc_handle *h, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA, m);
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);     \
    } while (0)

template <typename T>
static cudaError_t dalloc(pc_handle *h, T **p, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    *p = (T *)q;
    return cudaSuccess;
}

static void dfree(pc_handle *h, void *p)
{
    if (!p) return;
    auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
    if (it != h->allocs.end()) h->allocs.erase(it);
    cudaFree(p);
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Upper-tail normal quantile x with Q(x) = 0.5 erfc(x/sqrt 2) = a (0 < a < 1):
// Newton iterations on log Q(x) - log a, started from the tail asymptote.
static double upper_quantile(double a)
{
    if (a > 0.5) return -upper_quantile(1.0 - a);
    if (a == 0.5) return 0.0;
    double x = std::sqrt(-2.0 * std::log(a));
    for (int it = 0; it < 200; ++it) {
        double Q = 0.5 * std::erfc(x / std::sqrt(2.0));
        double phi = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
        double step = (std::log(Q) - std::log(a)) * Q / phi;   // g / g', g' = -phi/Q
        x += step;
        if (std::fabs(step) <= 1e-16 * std::max(1.0, std::fabs(x))) break;
    }
    return x;
}

static constexpr unsigned long long C64_LIST_CAP = 1ull << 20;   // pairs (8 MB)

static TestParams make_tp(const pc_handle *h)
{
    TestParams tp;
    tp.n = h->n;
    tp.nvec = h->g.nvec;
    tp.prow = h->g.prow;
    tp.q = h->q;
    tp.qf = (float)h->q;
    tp.rq_tab = h->rq_tab;
    tp.band = h->band;
    tp.guard = h->guard;
    tp.eps_c = h->used_tc ? 1.0e-6f : 1.2e-7f;
    tp.dr_max = 1.0f;            // skeleton: only the decision is returned (no bound on r itself)
    tp.lane_chunk = h->lane_chunk;
    tp.lane_rounds = h->lane_rounds;
    tp.lane_blocks = h->lane_blocks;
    tp.node_dmax = h->node_dmax;
    tp.comp_fp32 = h->comp_fp32 && h->precision != 0;
    tp.pair_warp = h->pair_warp;
    tp.pair_warp_dmin = h->pair_warp_dmin;
    tp.direct_warps = h->direct_warps;
    tp.lane_stages = h->lane_stages;
    tp.precision = h->precision;
    tp.reversed = h->order == 1;
    tp.complement = h->complement;
    tp.lazy = h->c64_full ? 0 : 1;
    tp.learned_min = h->learned_min;
    tp.learned_ratio = h->learned_ratio;
    tp.learned_lmax = h->learned_lmax;
    tp.p = h->p;
    tp.xs64 = h->Xs64;
    tp.ldk = h->ldk;
    tp.c64_valid = h->c64_valid;
    tp.c64_list = h->c64_list;
    tp.c64_list_len = h->c64_list_len;
    tp.c64_list_cap = h->c64_list ? C64_LIST_CAP : 0;
    tp.pair_seen = h->pair_seen;
    tp.pair_seen_bytes = h->pair_seen_bytes;
    return tp;
}

// ---------------------------------------------------------------- create / destroy
// pmax: largest problem size (binomial table), batch: block-diagonal batch
// layout (no precision blocks, conventional order only)
static pc_status create_impl(int64_t n, int32_t p, double alpha, int32_t max_level, int32_t pmax,
                             long long pool_cap, bool batch, size_t packed, pc_handle **out)
{
    pc_handle *h = new pc_handle();
    h->n = n;
    h->p = p;
    h->alpha = alpha;
    h->max_level = max_level;
    h->q = upper_quantile(alpha / 2.0);
    h->ldk = (n + 63) / 64 * 64;
    h->ldc = (p + 3) / 4 * 4;
    const int W = (p + 31) / 32;
    GraphDev &g = h->g;
    g.p = p;
    g.W = W;
    // per-pair arrays and correlation matrices: p x p (p x ldc), or the packed
    // diagonal blocks of a batch
    const size_t pp = batch ? packed : (size_t)p * p;
    h->pair_elems = pp;
    h->c_elems = batch ? packed : (size_t)p * h->ldc;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t ee) { if (e == cudaSuccess) e = ee; };
    A(dalloc(h, &g.adj, (size_t)p * W * sizeof(uint32_t)));
    A(dalloc(h, &g.deg, (size_t)p * sizeof(int)));
    A(dalloc(h, &g.dchg, (size_t)p * sizeof(int)));
    A(dalloc(h, &g.nbr, pp * sizeof(int)));
    A(dalloc(h, &g.ooff, (size_t)(p + 1) * sizeof(long long)));
    A(dalloc(h, &g.opu, (size_t)p * pmax * sizeof(int)));   // ordered pairs <= p * (largest p)
    h->opair_cap = (long long)p * (p - 1);
    A(dalloc(h, &g.tn_off, (size_t)(p + 2) * sizeof(ull)));
    A(dalloc(h, &g.cn_off, (size_t)(p + 2) * sizeof(ull)));
    A(dalloc(h, &g.rn_off, (size_t)(p + 2) * sizeof(ull)));
    A(dalloc(h, &g.ia_off, (size_t)(p + 2) * sizeof(ull)));
    A(dalloc(h, &g.it_off, (size_t)(p + 2) * sizeof(ull)));
    A(dalloc(h, &g.wo_off, (size_t)(p + 2) * sizeof(ull)));
    A(dalloc(h, &g.best, pp * sizeof(ull)));
    A(dalloc(h, &h->binom, (size_t)(pmax + 1) * (pmax + 1) * sizeof(ull)));
    A(dalloc(h, &h->rq_tab, (size_t)(pmax + 1) * sizeof(double)));
    A(dalloc(h, &g.sep_level, pp * sizeof(int)));
    A(dalloc(h, &g.sep_side, pp * sizeof(int)));
    A(dalloc(h, &g.sep_rank, pp * sizeof(long long)));
    A(dalloc(h, &g.sep_off, pp * sizeof(long long)));
    g.pool_cap = pool_cap;
    A(dalloc(h, &g.pool, (size_t)g.pool_cap * sizeof(int)));
    // neighbourhood precision blocks serve the reversed order only
    A(dalloc(h, &g.prec, batch ? sizeof(double) : (size_t)p * fpc::PREC_MAX * fpc::PREC_MAX * sizeof(double)));
    A(dalloc(h, &g.prec_m, (size_t)p * sizeof(int)));
    A(dalloc(h, &g.prec_mem, (size_t)p * fpc::PREC_MAX * sizeof(int)));
    A(dalloc(h, &g.prec_pos, pp * sizeof(short)));
    A(dalloc(h, &g.prec_need, (size_t)p * sizeof(int)));
    A(dalloc(h, &g.info, sizeof(LevelInfo)));
    A(dalloc(h, &g.ctr, sizeof(DevCounters)));
    A(dalloc(h, &h->mean, (size_t)p * sizeof(double)));
    A(dalloc(h, &h->rsd, (size_t)p * sizeof(double)));
    A(dalloc(h, &h->C64, h->c_elems * sizeof(double)));
    A(dalloc(h, &h->C32, h->c_elems * sizeof(float)));
    A(dalloc(h, &h->singular, sizeof(int)));
    A(dalloc(h, &h->tc_err, sizeof(int)));
    A(dalloc(h, &h->mlp_err, sizeof(int)));
    h->rq_cap = 1ull << 24;
    A(dalloc(h, &h->rq, (size_t)h->rq_cap * sizeof(ull)));
    A(dalloc(h, &h->rq_len, sizeof(ull)));
    A(dalloc(h, &h->mlp_loss, sizeof(double)));
    A(dalloc(h, &h->theta, (size_t)fpc::mlp_nparam() * sizeof(float)));
    A(dalloc(h, &h->adam_m, (size_t)fpc::mlp_nparam() * sizeof(float)));
    A(dalloc(h, &h->adam_v, (size_t)fpc::mlp_nparam() * sizeof(float)));
    A(dalloc(h, &h->grad, (size_t)fpc::mlp_nparam() * sizeof(float)));
    A(dalloc(h, &h->wpack, fpc::mlp_pack_bytes()));
    A(dalloc(h, &h->work, (size_t)(2 * p + 16) * sizeof(double)));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->info_h, sizeof(LevelInfo));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->ctr_h, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->br_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
    if (e != cudaSuccess) {
        pc_status st = e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
        pc_destroy(h);
        return st;
    }
    g.binom = h->binom;
    g.ldb = pmax + 1;
    // saturating Pascal triangle
    const int lb = pmax + 1;
    std::vector<ull> B((size_t)lb * lb, 0ull);
    for (int a = 0; a <= pmax; ++a) {
        B[(size_t)a * lb] = 1;
        for (int b = 1; b <= a; ++b) {
            ull x = B[(size_t)(a - 1) * lb + b - 1];
            ull y = b <= a - 1 ? B[(size_t)(a - 1) * lb + b] : 0ull;
            ull s = x + y;
            B[(size_t)a * lb + b] = (s < x || x == fpc::KEY_NONE || y == fpc::KEY_NONE) ? fpc::KEY_NONE : s;
        }
    }
    e = cudaMemcpy(h->binom, B.data(), B.size() * sizeof(ull), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pc_destroy(h);
        return PC_ERR_CUDA;
    }
    // the stage thresholds, formed once here (an FP64 tanh in every thread of a
    // stage's kernel costs microseconds on this GPU's FP64 pipe); stages past n - 4
    // have no tests
    std::vector<double> rq(pmax + 1, 0.0);
    for (int l = 0; l <= pmax; ++l)
        if (n - l - 3 > 0) rq[l] = std::tanh(h->q / std::sqrt((double)(n - l - 3)));
    e = cudaMemcpy(h->rq_tab, rq.data(), rq.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pc_destroy(h);
        return PC_ERR_CUDA;
    }
    *out = h;
    return PC_OK;
}

extern "C" pc_status pc_create(int64_t n, int32_t p, double alpha, int32_t max_level,
                               pc_handle **out)
{
    if (!out) return PC_ERR_ARG;
    *out = nullptr;
    if (n < 4 || n > (1ll << 21) || p < 2 || p > fpc::MAXP || !(alpha > 0.0 && alpha < 1.0))
        return PC_ERR_ARG;
    return create_impl(n, p, alpha, max_level, p, std::max<long long>(1 << 20, 16ll * p * p), false, 0, out);
}

// One handle over k independent problems laid out block-diagonally: instance i
// owns the nodes [off_i, off_i + p_i) (off_i = p_0 + ... + p_{i-1}).  Its
// adjacency starts as the complete graph on its own nodes only, so no test ever
// mixes instances, and each node's Fisher-z statistic uses its instance's n.
extern "C" pc_status pc_create_batch(int32_t k, const int64_t *n, const int32_t *p, double alpha,
                                     int32_t max_level, pc_handle **out)
{
    if (!out) return PC_ERR_ARG;
    *out = nullptr;
    if (k < 1 || k > fpc::MAXP_BATCH / 2 || !n || !p || !(alpha > 0.0 && alpha < 1.0)) return PC_ERR_ARG;
    long long ptot = 0, nmax = 0, nmin = 1ll << 40, pool = 0;
    int pmax = 0;
    for (int i = 0; i < k; ++i) {
        if (n[i] < 4 || n[i] > (1ll << 21) || p[i] < 2 || p[i] > fpc::MAXP) return PC_ERR_ARG;
        ptot += p[i];
        nmax = std::max<long long>(nmax, n[i]);
        nmin = std::min<long long>(nmin, n[i]);
        pmax = std::max(pmax, (int)p[i]);
        pool += 16ll * p[i] * p[i];
    }
    if (ptot > fpc::MAXP_BATCH) return PC_ERR_ARG;
    size_t packed = 0;
    for (int i = 0; i < k; ++i) packed += (size_t)p[i] * p[i];
    pc_handle *h = nullptr;
    if (pc_status r = create_impl(nmax, (int32_t)ptot, alpha, max_level, pmax, std::max<long long>(1 << 20, pool),
                                  true, packed, &h))
        return r;
    h->nblk = k;
    h->order = 0;
    h->n_min = nmin;
    h->boff.assign(k + 1, 0);
    h->bn.assign(n, n + k);
    h->bdone.assign(k, 0);
    h->pbase.assign(k + 1, 0);
    for (int i = 0; i < k; ++i) {
        h->boff[i + 1] = h->boff[i] + p[i];
        h->pbase[i + 1] = h->pbase[i] + (long long)p[i] * p[i];
    }
    std::vector<int> lo((size_t)ptot), hi((size_t)ptot);
    std::vector<long long> nv((size_t)ptot), prow((size_t)ptot), nrow((size_t)ptot);
    for (int i = 0; i < k; ++i)
        for (int u = h->boff[i]; u < h->boff[i + 1]; ++u) {
            lo[u] = h->boff[i];
            hi[u] = h->boff[i + 1];
            nv[u] = n[i];
            nrow[u] = h->pbase[i] + (long long)(u - h->boff[i]) * p[i];   // row u of block i
            prow[u] = nrow[u] - h->boff[i];                                // + global column id
        }
    int *dlo = nullptr, *dhi = nullptr;
    long long *dn = nullptr, *dprow = nullptr, *dnrow = nullptr;
    cudaError_t e = dalloc(h, &dlo, lo.size() * sizeof(int));
    if (e == cudaSuccess) e = dalloc(h, &dhi, hi.size() * sizeof(int));
    if (e == cudaSuccess) e = dalloc(h, &dn, nv.size() * sizeof(long long));
    if (e == cudaSuccess) e = dalloc(h, &dprow, prow.size() * sizeof(long long));
    if (e == cudaSuccess) e = dalloc(h, &dnrow, nrow.size() * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemcpy(dlo, lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dhi, hi.data(), hi.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dn, nv.data(), nv.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dprow, prow.data(), prow.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dnrow, nrow.data(), nrow.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pc_status st = e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
        pc_destroy(h);
        return st;
    }
    h->g.blk_lo = dlo;
    h->g.blk_hi = dhi;
    h->g.nvec = dn;
    h->g.prow = dprow;
    h->g.nrow = dnrow;
    *out = h;
    return PC_OK;
}

extern "C" pc_status pc_batch_layout(pc_handle *h, int32_t *k, int32_t *offsets)
{
    if (!h || !k) return PC_ERR_ARG;
    if (!h->nblk) {
        *k = 1;
        if (offsets) {
            offsets[0] = 0;
            offsets[1] = h->p;
        }
        return PC_OK;
    }
    *k = h->nblk;
    if (offsets)
        for (int i = 0; i <= h->nblk; ++i) offsets[i] = h->boff[i];
    return PC_OK;
}

extern "C" void pc_destroy(pc_handle *h)
{
    if (!h) return;
    for (auto &cl : h->lanes)
        if (cl.s) cudaStreamSynchronize(cl.s);
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->info_h) cudaFreeHost(h->info_h);
    if (h->ctr_h) cudaFreeHost(h->ctr_h);
    if (h->sepcnt_h) cudaFreeHost(h->sepcnt_h);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (auto &t : h->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : h->evpool) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (auto &cl : h->lanes)
        if (cl.s) cudaStreamDestroy(cl.s);
    for (auto e : h->lane_ev) cudaEventDestroy(e);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->br_stream) cudaStreamDestroy(h->br_stream);
    delete h;
}

// ---------------------------------------------------------------- options
extern "C" pc_status pc_set_opt(pc_handle *h, const char *key, double val)
{
    if (!h || !key) return PC_ERR_ARG;
    std::string k(key);
    if (k == "order") {
        if (val != 0 && val != 1) return fail(h, PC_ERR_ARG, "order must be 0 or 1");
        if (val == 1 && h->nblk) return fail(h, PC_ERR_ARG, "batched problems run the conventional order");
        h->order = (int)val;
    } else if (k == "stage_a") h->stage_a = val != 0;
    else if (k == "precision") {
        if (val != 0 && val != 1 && val != 2) return fail(h, PC_ERR_ARG, "precision must be 0, 1 or 2");
        h->precision = (int)val;
        h->have_corr = false;
        std::fill(h->bdone.begin(), h->bdone.end(), 0);   // batched: every instance again
    } else if (k == "band") {
        if (!(val >= 0)) return fail(h, PC_ERR_ARG, "band must be >= 0");
        h->band = val;
    } else if (k == "guard") {
        if (!(val >= 0)) return fail(h, PC_ERR_ARG, "guard must be >= 0");
        h->guard = val;
    } else if (k == "complement") h->complement = val != 0;
    else if (k == "timing") h->timing = val != 0;
    else if (k == "graph") h->use_graph = val != 0;
    else if (k == "learned") {
        if (val != 0 && !h->have_params) return fail(h, PC_ERR_STATE, "learned order needs parameters (pc_mlp_set_params or pc_mlp_train)");
        h->learned = val != 0;
    } else if (k == "learned_min_tests") {
        if (!(val >= 0)) return fail(h, PC_ERR_ARG, "learned_min_tests must be >= 0");
        h->learned_min = val;
    } else if (k == "learned_min_ratio") {
        if (!(val >= 0)) return fail(h, PC_ERR_ARG, "learned_min_ratio must be >= 0");
        h->learned_ratio = val;
    } else if (k == "learned_max_level") {
        if (!(val >= 0) || val > 1e6) return fail(h, PC_ERR_ARG, "learned_max_level must be in [0, 1e6]");
        h->learned_lmax = (int)val;
    } else if (k == "learned_rows") {
        if (!(val >= 0)) return fail(h, PC_ERR_ARG, "learned_rows must be >= 0");
        h->rows_cap = (long long)val;
    }
    else if (k == "budget") {
        if (!(val > 0)) return fail(h, PC_ERR_ARG, "budget must be > 0");
        h->budget = val;
    } else if (k == "stage_conds") {
        h->stage_conds = val != 0;
    } else if (k == "small_stage_kernel") {
        h->lane_stages = val != 0;

    } else if (k == "lane_chunk") {
        if (!(val >= 1 && val <= 256)) return fail(h, PC_ERR_ARG, "lane_chunk must be in [1, 256]");
        h->lane_chunk = (int)val;
    } else if (k == "lane_rounds") {
        if (!(val >= 0 && val <= 4096)) return fail(h, PC_ERR_ARG, "lane_rounds must be in [0, 4096]");
        h->lane_rounds = (int)val;
    } else if (k == "lane_blocks") {
        if (!(val >= 1 && val <= 32)) return fail(h, PC_ERR_ARG, "lane_blocks must be in [1, 32]");
        h->lane_blocks = (int)val;
    } else if (k == "mlp_backward") {
        if (!(val == 0 || val == 1)) return fail(h, PC_ERR_ARG, "mlp_backward must be 0 or 1");
        h->mlp_bwd_tc = (int)val;
    } else if (k == "path_pool") {
        if (!(val == 0 || val == 1)) return fail(h, PC_ERR_ARG, "path_pool must be 0 or 1");
        if (val == 1 && h->nblk) return fail(h, PC_ERR_ARG, "path_pool: a batched handle is not supported");
        h->path_pool = (int)val;
    } else if (k == "pair_warp") {
        if (!(val == 0 || val == 1)) return fail(h, PC_ERR_ARG, "pair_warp must be 0 or 1");
        h->pair_warp = (int)val;
    } else if (k == "pair_warp_dmin") {
        if (!(val >= 0 && val <= 16384)) return fail(h, PC_ERR_ARG, "pair_warp_dmin must be in [0, 16384]");
        h->pair_warp_dmin = (int)val;
    } else if (k == "node_dmax") {
        if (!(val >= 0 && val <= fpc::NODE_DMAX))
            return fail(h, PC_ERR_ARG, "node_dmax must be in [0, " + std::to_string(fpc::NODE_DMAX) + "]");
        h->node_dmax = (int)val;
    } else if (k == "stage_loop") {
        if (!(val == 0 || val == 1)) return fail(h, PC_ERR_ARG, "stage_loop must be 0 or 1");
        h->stage_loop = (int)val;
    } else if (k == "comp_fp32") {
        if (!(val == 0 || val == 1)) return fail(h, PC_ERR_ARG, "comp_fp32 must be 0 or 1");
        h->comp_fp32 = (int)val;
    } else if (k == "direct_warps") {
        if (val != 1 && val != 2 && val != 4 && val != 8) return fail(h, PC_ERR_ARG, "direct_warps must be 1, 2, 4 or 8");
        h->direct_warps = (int)val;
    } else return fail(h, PC_ERR_ARG, "unknown option: " + k);
    return PC_OK;
}

extern "C" pc_status pc_get_opt(pc_handle *h, const char *key, double *val)
{
    if (!h || !key || !val) return PC_ERR_ARG;
    std::string k(key);
    if (k == "order") *val = h->order;
    else if (k == "stage_a") *val = h->stage_a;
    else if (k == "precision") *val = h->precision;
    else if (k == "band") *val = h->band;
    else if (k == "guard") *val = h->guard;
    else if (k == "complement") *val = h->complement;
    else if (k == "timing") *val = h->timing;
    else if (k == "graph") *val = h->use_graph;
    else if (k == "learned") *val = h->learned;
    else if (k == "learned_rows") *val = (double)h->rows_cap;
    else if (k == "learned_min_tests") *val = h->learned_min;
    else if (k == "learned_min_ratio") *val = h->learned_ratio;
    else if (k == "learned_max_level") *val = h->learned_lmax;
    else if (k == "budget") *val = h->budget;
    else if (k == "stage_conds") *val = h->stage_conds;
    else if (k == "small_stage_kernel") *val = h->lane_stages;
    else if (k == "lane_chunk") *val = h->lane_chunk;
    else if (k == "lane_rounds") *val = h->lane_rounds;
    else if (k == "lane_blocks") *val = h->lane_blocks;
    else if (k == "node_dmax") *val = h->node_dmax;
    else if (k == "comp_fp32") *val = h->comp_fp32;
    else if (k == "stage_loop") *val = h->stage_loop;
    else if (k == "pair_warp") *val = h->pair_warp;
    else if (k == "path_pool") *val = h->path_pool;
    else if (k == "mlp_backward") *val = h->mlp_bwd_tc;
    else if (k == "pair_warp_dmin") *val = h->pair_warp_dmin;
    else if (k == "direct_warps") *val = h->direct_warps;
    else if (k == "tensor_core_gemm") *val = h->used_tc ? 1.0 : 0.0;
    else return fail(h, PC_ERR_ARG, "unknown option: " + k);
    return PC_OK;
}

extern "C" pc_status pc_set_stream(pc_handle *h, void *stream)
{
    if (!h) return PC_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return PC_OK;
}

extern "C" double pc_threshold(const pc_handle *h) { return h ? h->q : NAN; }

extern "C" double pc_fisher_threshold(double alpha)
{
    if (!(alpha > 0.0 && alpha < 1.0)) return NAN;
    return upper_quantile(alpha / 2.0);
}

extern "C" int64_t pc_kernel_launches(void) { return g_launches.load(); }

extern "C" pc_status pc_timing(pc_handle *h, double *ms, int64_t *count, int32_t reset)
{
    if (!h) return PC_ERR_ARG;
    if (!h->pending.empty()) {
        CK(cudaStreamSynchronize(h->stream));
        for (auto &t : h->pending) {
            float x = 0.f;
            CK(cudaEventElapsedTime(&x, t.a, t.b));
            h->cls_ms[t.cls] += x;
            h->cls_n[t.cls] += 1;
            h->evpool.push_back(t.a);
            h->evpool.push_back(t.b);
        }
        h->pending.clear();
    }
    for (int c = 0; c < NCLS; ++c) {
        if (ms) ms[c] = h->cls_ms[c];
        if (count) count[c] = h->cls_n[c];
        if (reset) {
            h->cls_ms[c] = 0;
            h->cls_n[c] = 0;
        }
    }
    return PC_OK;
}

extern "C" const char *pc_last_error(const pc_handle *h) { return h ? h->err.c_str() : "null handle"; }

extern "C" const char *pc_status_string(pc_status s)
{
    int i = (int)s;
    return (i >= 0 && i <= 8) ? kStatusNames[i] : "PC_UNKNOWN";
}

// ---------------------------------------------------------------- correlation
// the full FP64 correlation matrix (split-K Gram of the FP64 planes)
// FP64 Gram block of the planes' rows [o, o+p) into C64 (one problem: at row and
// column o with ldc; a batch instance: its packed block, leading dimension p)
static pc_status syrk64_block(pc_handle *h, int o, long long n, int p, int blk)
{
    double *out = blk < 0 ? h->C64 + (size_t)o * h->ldc + o : h->C64 + h->pbase[blk];
    const int ld = blk < 0 ? h->ldc : p;
    const size_t wsb = fpc::syrk_f64_ws_bytes(n, p);
    if (wsb > h->syrk_ws_bytes) {
        dfree(h, h->syrk_ws);
        h->syrk_ws = nullptr;
        CK(dalloc(h, &h->syrk_ws, wsb));
        h->syrk_ws_bytes = wsb;
    }
    CK(fpc::launch_syrk_f64(h->Xs64 + (size_t)o * h->ldk, n, h->ldk, p, out, ld, h->syrk_ws, h->syrk_ws_bytes,
                            h->stream));
    return PC_OK;
}

static pc_status materialize_c64(pc_handle *h)
{
    if (h->c64_full) return PC_OK;
    if (h->nblk) {
        // batched problems: each diagonal block from its own samples
        for (int i = 0; i < h->nblk; ++i)
            if (pc_status r = syrk64_block(h, h->boff[i], h->bn[i], h->boff[i + 1] - h->boff[i], i)) return r;
    } else {
        if (pc_status r = syrk64_block(h, 0, h->n, h->p, -1)) return r;
    }
    h->c64_full = true;
    return PC_OK;
}

// a bounded wait inside the tensor-core GEMM expired (device-side error word)
static pc_status check_tc(pc_handle *h)
{
    if (!h->used_tc) return PC_OK;
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (e) return fail(h, (pc_status)e, "tensor-core correlation GEMM: a bounded wait expired");
    return PC_OK;
}

// The pair list of the FP64 entries formed in parallel before a small stage's FP64
// pass (entries beyond it are formed on demand by the pass itself).
static pc_status alloc_c64_list(pc_handle *h)
{
    if (h->c64_list) return PC_OK;
    CK(dalloc(h, &h->c64_list, C64_LIST_CAP * sizeof(int2)));
    CK(dalloc(h, &h->c64_list_len, sizeof(unsigned long long)));
    h->pair_seen_bytes = (h->pair_elems + 7) / 4 * 4;    // whole words: claimed by CAS
    CK(dalloc(h, &h->pair_seen, h->pair_seen_bytes));
    return PC_OK;
}

// Standardisation and correlation GEMM of one problem, or of instance blk of a
// batched handle (its columns are rows [o, o+p) of the planes, its block of
// corr the diagonal block there).
// lane: run on a side stream with its own workspaces (pc_corr_blocks, which has
// allocated the handle's planes and flags and cleared the GEMM's error flag first)
static pc_status corr_impl(pc_handle *h, const void *X, int32_t dtype, int64_t ld, int blk, CorrLane *lane = nullptr)
{
    cudaStream_t s = lane ? lane->s : h->stream;
    void *&Xstage = lane ? lane->Xstage : h->Xstage;
    size_t &Xstage_bytes = lane ? lane->Xstage_bytes : h->Xstage_bytes;
    double *&stats_ws = lane ? lane->stats_ws : h->stats_ws;
    size_t &stats_ws_bytes = lane ? lane->stats_ws_bytes : h->stats_ws_bytes;
    float *&tc_ws = lane ? lane->tc_ws : h->tc_ws;
    size_t &tc_ws_bytes = lane ? lane->tc_ws_bytes : h->tc_ws_bytes;
    const int o = blk < 0 ? 0 : h->boff[blk];
    const int p = blk < 0 ? h->p : h->boff[blk + 1] - o;
    const long long n = blk < 0 ? h->n : h->bn[blk];
    if (!X || (dtype != PC_F32 && dtype != PC_F64) || ld < p)
        return fail(h, PC_ERR_ARG, "pc_corr: bad X, dtype or ld");
    const size_t esz = dtype == PC_F64 ? 8 : 4;
    const void *Xd = X;
    if (!is_device_ptr(X)) {
        size_t bytes = (size_t)n * ld * esz;
        if (bytes > Xstage_bytes) {
            dfree(h, Xstage);
            Xstage = nullptr;
            Xstage_bytes = 0;
            CK(dalloc(h, &Xstage, bytes));
            Xstage_bytes = bytes;
        }
        CK(cudaMemcpyAsync(Xstage, X, bytes, cudaMemcpyHostToDevice, s));
        Xd = Xstage;
    }
    const size_t plane = (size_t)h->p * h->ldk;
    if (!h->Xs64) {
        CK(dalloc(h, &h->Xs64, plane * sizeof(double)));
        CK(dalloc(h, &h->Xs32, plane * sizeof(float)));
        CK(dalloc(h, &h->Xhi, plane * sizeof(uint16_t)));
        CK(dalloc(h, &h->Xlo, plane * sizeof(uint16_t)));
        CK(cudaMemsetAsync(h->Xs64, 0, plane * sizeof(double), s));
        CK(cudaMemsetAsync(h->Xs32, 0, plane * sizeof(float), s));
        CK(cudaMemsetAsync(h->Xhi, 0, plane * sizeof(uint16_t), s));
        CK(cudaMemsetAsync(h->Xlo, 0, plane * sizeof(uint16_t), s));
    }
    Timed tm(h, lane ? -1 : 0);
    const size_t sws = fpc::col_stats_ws_bytes(n, p);
    if (sws > stats_ws_bytes) {
        dfree(h, stats_ws);
        stats_ws = nullptr;
        CK(dalloc(h, &stats_ws, sws));
        stats_ws_bytes = sws;
    }
    const size_t po = (size_t)o * h->ldk;                  // first plane row of this problem
    CK(fpc::launch_col_stats_split(Xd, dtype, n, p, ld, h->mean + o, h->rsd + o, stats_ws, s));
    const bool want_bf16 = h->precision == 2 && fpc::tc_gemm_available();
    CK(fpc::launch_standardize(Xd, dtype, n, p, ld, h->mean + o, h->rsd + o, stats_ws, h->Xs64 + po,
                               h->precision == 1 ? h->Xs32 + po : nullptr,
                               want_bf16 ? h->Xhi + po : nullptr, want_bf16 ? h->Xlo + po : nullptr, h->ldk,
                               s));
    // FP64 correlations: all of them when a stage needs whole blocks (reversed
    // order: closed-form stage, precision blocks) or the tests run in FP64;
    // otherwise per entry on demand when a test is re-decided in FP64
    h->c64_full = false;
    if (blk >= 0) {
        if (h->precision == 0) {
            if (pc_status r = syrk64_block(h, o, n, p, blk)) return r;
        } else {
            if (!h->c64_valid) {
                // whole 32-bit words: the claims of c64_collect CAS the word of a flag
                CK(dalloc(h, &h->c64_valid, (h->pair_elems + 7) / 4 * 4));
                CK(cudaMemsetAsync(h->c64_valid, 0, (h->pair_elems + 7) / 4 * 4, s));
                if (pc_status r = alloc_c64_list(h)) return r;
            }
            CK(fpc::launch_c64_lazy_init_block(h->C64 + h->pbase[blk], p, h->c64_valid + h->pbase[blk], p, 0, p,
                                               s));
        }
    } else if (h->precision == 0 || h->order == 1) {
        if (pc_status r = materialize_c64(h)) return r;
    } else {
        if (!h->c64_valid) {
            CK(dalloc(h, &h->c64_valid, ((size_t)p * p + 7) / 4 * 4));
            CK(cudaMemsetAsync(h->c64_valid, 0, ((size_t)p * p + 7) / 4 * 4, s));
            if (pc_status r = alloc_c64_list(h)) return r;
        }
        CK(fpc::launch_c64_lazy_init(h->C64, h->ldc, h->c64_valid, p, s));
    }
    // this problem's correlation block and its leading dimension
    float *C32b = blk < 0 ? h->C32 : h->C32 + h->pbase[blk];
    const int ldb = blk < 0 ? h->ldc : p;
    bool tc = false;
    if (h->precision == 0) {
        if (blk >= 0) CK(fpc::launch_cast_block(h->C64 + h->pbase[blk], h->C32 + h->pbase[blk], p, 0, p, s));
        else CK(fpc::launch_cast_c(h->C64, h->C32, p, h->ldc, s));
    } else if (h->precision == 1 || !want_bf16) {
        if (h->precision == 2) {
            // tensor-core path not available on this device: FP32 operands on the CUDA cores
            CK(fpc::launch_standardize(Xd, dtype, n, p, ld, h->mean + o, h->rsd + o, stats_ws, nullptr, h->Xs32 + po,
                                       nullptr, nullptr, h->ldk, s));
        }
        Timed tg(h, lane ? -1 : 7);
        CK(fpc::launch_syrk_f32(h->Xs32 + po, n, h->ldk, p, C32b, ldb, s));
    } else {
        const size_t need = fpc::corr_bf16x3_ws_bytes(n, p);
        if (need > tc_ws_bytes) {
            dfree(h, tc_ws);
            tc_ws = nullptr;
            CK(dalloc(h, &tc_ws, need));
            tc_ws_bytes = need;
        }
        if (blk <= 0 && !lane) CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
        Timed tg(h, lane ? -1 : 7);
        CK(fpc::launch_corr_bf16x3(h->Xhi + po, h->Xlo + po, n, h->ldk, p, C32b, ldb, tc_ws, tc_ws_bytes,
                                   h->tc_err, s));
        tc = true;
    }
    if (blk < 0) {
        h->used_tc = tc;
        if (!h->Pbuf) CK(dalloc(h, &h->Pbuf, (size_t)p * h->ldc * sizeof(double)));
        h->have_corr = true;
    } else {
        // every instance runs the same GEMM path (one precision per handle)
        h->used_tc = tc;
        h->bdone[blk] = 1;
        bool all = true;
        for (char d : h->bdone) all = all && d;
        h->have_corr = all;
        // FP64 tests read whole blocks: every block was formed in full above
        h->c64_full = all && h->precision == 0;
    }
    h->have_skel = false;
    return PC_OK;
}

extern "C" pc_status pc_corr(pc_handle *h, const void *X, int32_t dtype, int64_t ld)
{
    if (!h) return PC_ERR_ARG;
    if (h->nblk) return fail(h, PC_ERR_STATE, "batched handle: give each instance with pc_corr_block");
    return corr_impl(h, X, dtype, ld, -1);
}

extern "C" pc_status pc_corr_block(pc_handle *h, int32_t i, const void *X, int32_t dtype, int64_t ld)
{
    if (!h) return PC_ERR_ARG;
    if (!h->nblk) return fail(h, PC_ERR_STATE, "pc_corr_block needs a batched handle (pc_create_batch)");
    if (i < 0 || i >= h->nblk) return fail(h, PC_ERR_ARG, "pc_corr_block: instance index out of range");
    return corr_impl(h, X, dtype, ld, i);
}

extern "C" pc_status pc_corr_blocks(pc_handle *h, const void *const *X, const int32_t *dtype, const int64_t *ld)
{
    if (!h) return PC_ERR_ARG;
    if (!h->nblk) return fail(h, PC_ERR_STATE, "pc_corr_blocks needs a batched handle (pc_create_batch)");
    if (!X || !dtype || !ld) return fail(h, PC_ERR_ARG, "pc_corr_blocks: null array");
    const int k = h->nblk;
    for (int i = 0; i < k; ++i)
        if (!X[i] || (dtype[i] != PC_F32 && dtype[i] != PC_F64) || ld[i] < h->boff[i + 1] - h->boff[i])
            return fail(h, PC_ERR_ARG, "pc_corr_blocks: bad X, dtype or ld of instance " + std::to_string(i));
    if (h->precision == 0) {
        // the FP64 Gram shares one split-K workspace: one instance after the other
        for (int i = 0; i < k; ++i)
            if (pc_status r = corr_impl(h, X[i], dtype[i], ld[i], i)) return r;
        return PC_OK;
    }
    cudaStream_t s = h->stream;
    Timed tm(h, 0);
    // what the instances share, on the handle's stream before the fork: the
    // standardised planes, the FP64-validity flags, the GEMM's error flag
    const size_t plane = (size_t)h->p * h->ldk;
    if (!h->Xs64) {
        CK(dalloc(h, &h->Xs64, plane * sizeof(double)));
        CK(dalloc(h, &h->Xs32, plane * sizeof(float)));
        CK(dalloc(h, &h->Xhi, plane * sizeof(uint16_t)));
        CK(dalloc(h, &h->Xlo, plane * sizeof(uint16_t)));
        CK(cudaMemsetAsync(h->Xs64, 0, plane * sizeof(double), s));
        CK(cudaMemsetAsync(h->Xs32, 0, plane * sizeof(float), s));
        CK(cudaMemsetAsync(h->Xhi, 0, plane * sizeof(uint16_t), s));
        CK(cudaMemsetAsync(h->Xlo, 0, plane * sizeof(uint16_t), s));
    }
    if (!h->c64_valid) {
        CK(dalloc(h, &h->c64_valid, (h->pair_elems + 7) / 4 * 4));
        CK(cudaMemsetAsync(h->c64_valid, 0, (h->pair_elems + 7) / 4 * 4, s));
        if (pc_status r = alloc_c64_list(h)) return r;
    }
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
    const int nl = std::min(k, 8);
    while ((int)h->lanes.size() < nl) {
        CorrLane cl;
        CK(cudaStreamCreateWithFlags(&cl.s, cudaStreamNonBlocking));
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h->lanes.push_back(cl);
        h->lane_ev.push_back(ev);
    }
    if (h->lane_ev.size() < (size_t)nl + 1) {
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h->lane_ev.push_back(ev);
    }
    cudaEvent_t fork = h->lane_ev[nl];
    CK(cudaEventRecord(fork, s));
    for (int j = 0; j < nl; ++j) CK(cudaStreamWaitEvent(h->lanes[j].s, fork, 0));
    // the larger instances first, spread over the lanes
    std::vector<int> order(k);
    for (int i = 0; i < k; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)h->bn[a] * (h->boff[a + 1] - h->boff[a]) > (double)h->bn[b] * (h->boff[b + 1] - h->boff[b]);
    });
    for (int t = 0; t < k; ++t) {
        const int i = order[t];
        if (pc_status r = corr_impl(h, X[i], dtype[i], ld[i], i, &h->lanes[t % nl])) return r;
    }
    for (int j = 0; j < nl; ++j) {
        CK(cudaEventRecord(h->lane_ev[j], h->lanes[j].s));
        CK(cudaStreamWaitEvent(s, h->lane_ev[j], 0));
    }
    return PC_OK;
}

extern "C" pc_status pc_corr_get(pc_handle *h, float *C32, double *C64)
{
    if (!h) return PC_ERR_ARG;
    if (!h->have_corr) return fail(h, PC_ERR_STATE, "pc_corr_get before pc_corr");
    cudaStream_t s = h->stream;
    const int p = h->p;
    if (C64 && !h->c64_full) {
        Timed tm(h, 0);
        if (pc_status r = materialize_c64(h)) return r;
    }
    if (h->nblk) {
        // batched problems: the dense p x p matrix, zero off the diagonal blocks
        auto unpack = [&](void *dst, const void *src, size_t esz) -> cudaError_t {
            if (is_device_ptr(dst)) {
                cudaError_t e = cudaMemsetAsync(dst, 0, (size_t)p * p * esz, s);
                if (e != cudaSuccess) return e;
            } else {
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return e;
                std::memset(dst, 0, (size_t)p * p * esz);
            }
            for (int i = 0; i < h->nblk; ++i) {
                const int o = h->boff[i], pb = h->boff[i + 1] - o;
                cudaError_t e = cudaMemcpy2DAsync((char *)dst + ((size_t)o * p + o) * esz, (size_t)p * esz,
                                                  (const char *)src + (size_t)h->pbase[i] * esz, (size_t)pb * esz,
                                                  (size_t)pb * esz, pb, cudaMemcpyDefault, s);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        };
        if (C32) CK(unpack(C32, h->C32, sizeof(float)));
        if (C64) CK(unpack(C64, h->C64, sizeof(double)));
    } else {
        if (C32)
            CK(cudaMemcpy2DAsync(C32, p * sizeof(float), h->C32, h->ldc * sizeof(float),
                                 p * sizeof(float), p, cudaMemcpyDefault, s));
        if (C64)
            CK(cudaMemcpy2DAsync(C64, p * sizeof(double), h->C64, h->ldc * sizeof(double),
                                 p * sizeof(double), p, cudaMemcpyDefault, s));
    }
    CK(cudaStreamSynchronize(s));
    return check_tc(h);
}

// ---------------------------------------------------------------- skeleton
static pc_status read_info(pc_handle *h)
{
    CK(cudaMemcpyAsync(h->info_h, h->g.info, sizeof(LevelInfo), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PC_OK;
}

static int level_cap(const pc_handle *h)
{
    int cap = h->p - 2;
    if (h->max_level >= 0 && h->max_level < cap) cap = h->max_level;
    if (h->n - 4 < cap) cap = (int)(h->n - 4);
    return cap;
}

// One stage of the loop (every kernel reads l from the device): counts, scan
// and gate, the CI tests, the PC-stable commit, the next frozen graph, the
// next l and the loop condition, then the precision blocks of the next stage.
// Adds a conditional node (IF or SWITCH on handle hc) after the current capture
// dependencies of s and captures fn(i, stream) into its i-th body on the
// handle's branch stream.
template <class F>
static pc_status cond_node(pc_handle *h, cudaStream_t s, cudaGraphConditionalHandle hc,
                           cudaGraphConditionalNodeType type, unsigned size, F fn)
{
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = type;
    cp.conditional.size = size;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &cp));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    for (unsigned i = 0; i < size; ++i) {
        CK(cudaStreamBeginCaptureToGraph(h->br_stream, cp.conditional.phGraph_out[i], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
        pc_status st = fn((int)i, h->br_stream);
        cudaGraph_t out = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->br_stream, &out);
        if (st != PC_OK) return st;
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture (conditional body)");
    }
    return PC_OK;
}

// One stage of the loop (Algorithm 1 / 2 body).  use_cond: being captured into
// the WHILE body; the kernels without work in a stage then sit behind
// conditional nodes that the head and tail kernels set.  Otherwise (host loop)
// every kernel is launched and returns at once when it has nothing to do.
static pc_status enqueue_level(pc_handle *h, cudaStream_t s, int mmax, bool use_cond, bool timed)
{
    GraphDev &g = h->g;
    TestParams tp = make_tp(h);
    const bool use_prec = h->order == 1 && h->complement;
    auto T = [&](int cls) { return Timed(h, timed ? cls : -1); };
    fpc::StageConds sc = {};
    const bool conds = use_cond && h->stage_conds;
    if (conds) {
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, nullptr, nullptr, nullptr));
        sc.use = 1;
        sc.has_comp = use_prec;
        sc.has_score = h->learned && h->learned_lmax >= 1;
        sc.has_prec = use_prec;
        CK(cudaGraphConditionalHandleCreate(&sc.tests, cg, (unsigned)fpc::stage_branches(sc.has_comp, sc.has_score),
                                            0));
        if (sc.has_prec) CK(cudaGraphConditionalHandleCreate(&sc.prec, cg, 0, 0));
    }
    {
        auto t = T(5);
        CK(fpc::launch_head(g, tp, h->budget, mmax, sc, s));
    }
    const float sqn_over_q = (float)(std::sqrt((double)h->n) / h->q);
    auto score = [&](int, cudaStream_t st) -> pc_status {
        CK(fpc::launch_mlp_score_stage(g, h->row_off, h->rows_cap, h->C32, h->ldc, sqn_over_q,
                                       (float)(1.0 / h->q), h->wpack, h->theta, h->stage_scores, h->perm,
                                       h->mlp_err, st));
        return PC_OK;
    };
    // small stages: one lane-kernel range, the FP64 pass over its queue, and the
    // warp-per-test kernel that re-runs the stage if that queue overflowed
    auto lane = [&](int range, cudaStream_t st) -> pc_status {
        // the proposal-order variants only where a stage can be scored (the scoring
        // gate at 0 leaves every stage in the plain order)
        CK(fpc::launch_ci_lane(g, tp, h->C32, h->C64, h->ldc, h->rq, h->rq_cap, h->rq_len, range,
                               h->learned && h->learned_lmax >= 1, st));
        CK(fpc::launch_ci_direct(g, tp, fpc::LANE_LMAX + 2, h->C32, h->C64, h->ldc, st));
        return PC_OK;
    };
    auto direct = [&](int, cudaStream_t st) -> pc_status {
        CK(fpc::launch_ci_direct(g, tp, mmax, h->C32, h->C64, h->ldc, st));
        return PC_OK;
    };
    auto comp = [&](int, cudaStream_t st) -> pc_status {
        CK(fpc::launch_ci_complement(g, tp, st));
        return PC_OK;
    };
    auto prec = [&](int, cudaStream_t st) -> pc_status {
        CK(fpc::launch_prec_update(g, tp, h->C64, h->ldc, st));
        return PC_OK;
    };
    if (conds) {
        // one switch node: branch i runs [scoring,] the test kernel of its kind [, complement]
        auto branch = [&](int i, cudaStream_t st) -> pc_status {
            for (int sco = 0; sco <= sc.has_score; ++sco)
                for (int cmp = 0; cmp <= sc.has_comp; ++cmp)
                    for (int kind = 0; kind <= fpc::STAGE_KIND_NONE; ++kind) {
                        if ((kind == fpc::STAGE_KIND_NONE && (!cmp || sco)) ||
                            fpc::stage_branch(kind, cmp, sco, sc.has_comp, sc.has_score) != i)
                            continue;
                        if (sco)
                            if (pc_status r = score(0, st)) return r;
                        if (kind < fpc::LANE_RANGES) {
                            if (pc_status r = lane(kind, st)) return r;
                        } else if (kind == fpc::STAGE_KIND_DIRECT) {
                            if (pc_status r = direct(0, st)) return r;
                        }
                        if (cmp)
                            if (pc_status r = comp(0, st)) return r;
                        return PC_OK;
                    }
            return fail(h, PC_ERR_INTERNAL, "stage switch branch without a combination");
        };
        if (pc_status r = cond_node(h, s, sc.tests, cudaGraphCondTypeSwitch,
                                    (unsigned)fpc::stage_branches(sc.has_comp, sc.has_score), branch))
            return r;
    } else {
        if (h->learned && h->learned_lmax >= 1) {
            auto t = T(6);
            if (pc_status r = score(0, s)) return r;
        }
        {
            auto t = T(3);
            if (use_cond) {
                // captured without conditional nodes: every kernel, each returns at once
                // when the stage is not its own
                if (h->precision != 0 && h->lane_stages)
                    if (pc_status r = lane(-1, s)) return r;
                if (pc_status r = direct(0, s)) return r;
            } else {
                const int l = h->info_h->l;
                if (h->lane_stages && h->precision != 0 && l >= 0 && l <= fpc::LANE_LMAX) {
                    if (pc_status r = lane(fpc::lane_range_of(l), s)) return r;
                } else {
                    if (pc_status r = direct(0, s)) return r;
                }
            }
        }
        if (use_prec) {
            auto t = T(4);
            if (pc_status r = comp(0, s)) return r;
        }
    }
    {
        auto t = T(5);
        CK(fpc::launch_commit(g, h->opair_cap, -1, 1, s));
        CK(fpc::launch_degrees_tail(g, tp, level_cap(h), h->hcond, use_cond ? 1 : 0, sc, s));
    }
    if (use_prec) {
        if (conds) {
            if (pc_status r = cond_node(h, s, sc.prec, cudaGraphCondTypeIf, 1, prec)) return r;
        } else {
            auto t = T(2);
            if (pc_status r = prec(0, s)) return r;
        }
    }
    return PC_OK;
}

static std::vector<double> graph_key(const pc_handle *h)
{
    return {(double)h->order, (double)h->complement, (double)h->precision, h->band, h->guard,
            (double)h->used_tc, (double)h->c64_full, (double)h->learned, (double)(uintptr_t)h->perm, (double)h->rows_cap, h->learned_min, h->learned_ratio, (double)(uintptr_t)h->rq,
            h->budget, (double)level_cap(h), (double)(uintptr_t)h->g.pool, (double)h->g.pool_cap,
            (double)(uintptr_t)h->C32, (double)(uintptr_t)h->C64, (double)h->lane_chunk,
            (double)h->lane_rounds, (double)h->lane_blocks, (double)h->direct_warps, (double)h->stage_conds,
            (double)h->node_dmax, (double)h->pair_warp, (double)h->pair_warp_dmin, (double)h->learned_lmax,
            (double)h->comp_fp32,
            (double)h->lane_stages};
}

static void drop_graph(pc_handle *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->graph_key.clear();
}

// Capture the stage body once into the body of a conditional WHILE node.
static pc_status ensure_graph(pc_handle *h)
{
    std::vector<double> key = graph_key(h);
    if (h->gexec && key == h->graph_key) return PC_OK;
    drop_graph(h);
    CK(cudaGraphCreate(&h->graph, 0));
    CK(cudaGraphConditionalHandleCreate(&h->hcond, h->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h->hcond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    const long long l0 = g_launches.load();
    pc_status st = enqueue_level(h, h->cap_stream, fpc::LG_DIRECT + 2, true, false);
    h->body_kernels = g_launches.load() - l0;
    g_launches.fetch_sub(h->body_kernels);         // counted when the body executes
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &out);
    if (st != PC_OK) {
        drop_graph(h);
        return st;
    }
    if (e != cudaSuccess) {
        drop_graph(h);
        return cuda_fail(h, e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&h->gexec, h->graph, 0);
    if (e != cudaSuccess) {
        drop_graph(h);
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    h->graph_key = key;
    return PC_OK;
}

static pc_status clear_halt(pc_handle *h)
{
    // need_host and halt are adjacent ints after 'done'
    CK(cudaMemsetAsync(&h->g.info->halt, 0, sizeof(int), h->stream));
    CK(cudaMemsetAsync(&h->g.info->need_host, 0, sizeof(int), h->stream));
    return PC_OK;
}

static pc_status skeleton_enqueue(pc_handle *h)
{
    if (h->order == 1 && !h->c64_full) {
        Timed tm(h, 0);
        if (pc_status r = materialize_c64(h)) return r;
    }
    GraphDev &g = h->g;
    cudaStream_t s = h->stream;
    const int p = h->p;
    const long long n = h->n;
    const size_t pp = h->pair_elems;
    TestParams tp = make_tp(h);
    const bool timed = h->timing != 0;
    const bool graph = h->use_graph && !timed;
    if (h->learned) {
        if (!h->row_off) {
            if (h->rows_cap <= 0) h->rows_cap = 1ll << 24;
            CK(dalloc(h, &h->row_off, (size_t)(p + 2) * sizeof(ull)));
            CK(dalloc(h, &h->perm, (size_t)h->rows_cap * sizeof(short)));
            CK(dalloc(h, &h->stage_scores, (size_t)h->rows_cap * sizeof(float)));
            CK(dalloc(h, &h->scored, (size_t)p));
        }
        g.row_off = h->row_off;
        g.perm = h->perm;
        g.rows_cap = h->rows_cap;
        g.scored = h->scored;
        CK(cudaMemsetAsync(h->mlp_err, 0, sizeof(int), s));
        CK(cudaMemsetAsync(h->scored, 0, (size_t)p, s));
    } else {
        g.row_off = nullptr;
        g.perm = nullptr;
        g.rows_cap = 0;
        g.scored = nullptr;
    }
    if (graph) {
        if (pc_status r = ensure_graph(h)) return r;
    }

    // complete graph, empty sepset store
    CK(fpc::launch_init_adj(g, s));
    CK(cudaMemsetAsync(g.best, 0xff, pp * sizeof(ull), s));
    CK(cudaMemsetAsync(g.sep_level, 0xff, pp * sizeof(int), s));
    CK(cudaMemsetAsync(g.sep_off, 0xff, pp * sizeof(long long), s));
    CK(cudaMemsetAsync(g.prec_m, 0, (size_t)p * sizeof(int), s));
    CK(cudaMemsetAsync(g.prec_pos, 0xff, pp * sizeof(short), s));
    CK(cudaMemsetAsync(g.prec_need, 0, (size_t)p * sizeof(int), s));
    CK(cudaMemsetAsync(g.ctr, 0, sizeof(DevCounters), s));
    CK(cudaMemsetAsync(g.info, 0, sizeof(LevelInfo), s));
    CK(cudaMemsetAsync(&g.info->lstar, 0xff, sizeof(int), s));
    CK(cudaMemsetAsync(h->singular, 0, sizeof(int), s));
    CK(cudaEventRecord(h->ev0, s));

    int stage_a_launched = 0;
    {
        Timed t(h, 5);
        CK(fpc::launch_level_degrees(g, s));
        CK(fpc::launch_tail(g, tp, level_cap(h), 2, h->singular, 0, h->hcond, 0, fpc::StageConds{}, s));
    }
    if (h->order == 1 && h->stage_a && n - p - 1 > 0) {
        stage_a_launched = 1;
        {
            Timed t(h, 1);
            CK(cudaMemcpyAsync(h->Pbuf, h->C64, (size_t)p * h->ldc * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
            CK(fpc::launch_inverse_spd(h->Pbuf, p, h->ldc, h->work, h->singular, s));
            CK(fpc::launch_stage_a_decide(h->Pbuf, p, h->ldc, h->singular, g, tp, s));
        }
        {
            Timed t(h, 5);
            CK(fpc::launch_commit(g, h->opair_cap, p - 2, 0, s));
            CK(fpc::launch_level_degrees(g, s));
        }
    }
    {
        Timed t(h, 5);
        CK(fpc::launch_tail(g, tp, level_cap(h), 1, h->singular, stage_a_launched, h->hcond, 0, fpc::StageConds{},
                            s));
    }
    // the stage loop in one kernel for small problems (the reversed order's precision
    // blocks, when it has them, included)
    bool loop = h->stage_loop && p <= fpc::LOOP_PMAX && !h->nblk;
    if (loop && h->coop < 0) {
        int dev = 0, v = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev));
        h->coop = v;
    }
    loop = loop && h->coop;
    if (h->order == 1 && h->complement) {
        Timed t(h, 2);
        // after the closed-form stage: blocks from its inverse, then one downdate each
        // (in the stage loop kernel when it runs)
        if (stage_a_launched && p <= fpc::PREC_MAX) CK(fpc::launch_prec_seed(g, h->Pbuf, h->ldc, s));
        if (!loop) CK(fpc::launch_prec_update(g, tp, h->C64, h->ldc, s));
    }
    if (loop) {
        // the first blocks and the stages in one cooperative kernel; the captured loop (or
        // the host loop) goes on from the first stage the kernel does not take
        const bool blocks = h->order == 1 && h->complement;
        Timed t(h, 8);
        cudaError_t e = fpc::launch_stage_loop(g, tp, h->C32, h->C64, h->ldc, h->budget, level_cap(h),
                                               blocks ? 1 : 0, s);
        if (e == cudaErrorCooperativeLaunchTooLarge) {
            cudaGetLastError();                        // not resident: the captured loop runs it all
            if (blocks) CK(fpc::launch_prec_update(g, tp, h->C64, h->ldc, s));
        } else {
            CK(e);
        }
    }

    if (graph) CK(cudaGraphLaunch(h->gexec, s));
    return PC_OK;
}

static pc_status skeleton_complete(pc_handle *h, pc_stats *st, bool *overflow)
{
    GraphDev &g = h->g;
    cudaStream_t s = h->stream;
    const int p = h->p;
    TestParams tp = make_tp(h);
    std::memset(st, 0, sizeof(*st));
    *overflow = false;
    const bool timed = h->timing != 0;
    const bool graph = h->use_graph && !timed;
    // the stage loop
    for (int guard_iter = 0; guard_iter < 4 * p + 16; ++guard_iter) {
        if (graph) {
            if (guard_iter > 0) CK(cudaGraphLaunch(h->gexec, s));
            if (pc_status r = read_info(h)) return r;
        } else {
            if (pc_status r = read_info(h)) return r;
            if (h->info_h->done || h->info_h->halt) {
                // fall through to the checks below
            } else {
                int mmax = std::max(fpc::LG_DIRECT + 2, h->info_h->l + 2);
                if (mmax > fpc::DIRECT_MMAX) {
                    // the gate halts the stage if it really has direct tests that large
                    mmax = fpc::DIRECT_MMAX;
                }
                if (pc_status r = enqueue_level(h, s, mmax, false, timed)) return r;
                continue;
            }
        }
        const LevelInfo &I = *h->info_h;
        if (I.pool_overflow) {
            *overflow = true;
            return PC_OK;
        }
        if (I.error) {
            return fail(h, (pc_status)I.error,
                        "stage l=" + std::to_string(I.l) + " schedules " +
                            (I.saturated ? std::string(">2^64") :
                                           std::to_string((double)I.total_direct + (double)I.total_comp)) +
                            " tests, above the budget");
        }
        if (I.done) break;
        if (I.need_host) {
            // a direct-path stage too large for the captured layout: run it here, up to
            // the largest matrix one warp can hold in shared memory
            if (I.l + 2 > fpc::DIRECT_MMAX)
                return fail(h, PC_ERR_BUDGET,
                            "stage l=" + std::to_string(I.l) + " needs direct tests of size " +
                                std::to_string(I.l + 2) + " (largest supported " +
                                std::to_string(fpc::DIRECT_MMAX) + "); use the conventional order");
            if (pc_status r = clear_halt(h)) return r;
            if (pc_status r = enqueue_level(h, s, I.l + 2, false, timed)) return r;
        }
    }
    CK(cudaEventRecord(h->ev1, s));
    if (h->learned && h->learned_lmax >= 1) {
        // largest stage run: the first one in the reversed order, the last one conventionally
        Timed tm(h, h->timing ? 6 : -1);
        const int lmax = h->order == 1 ? h->info_h->first_level : h->info_h->l - 1;
        CK(fpc::launch_reverify(g, tp, h->C32, h->C64, h->ldc, lmax, s));
    }
    if (pc_status r = read_info(h)) return r;
    if (!h->info_h->done) return fail(h, PC_ERR_INTERNAL, "stage loop did not finish");
    CK(cudaMemcpyAsync(h->ctr_h, g.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const DevCounters &c = *h->ctr_h;
    const LevelInfo &I = *h->info_h;
    // the captured body counts the kernels its conditional nodes actually ran
    if (graph && h->stage_conds) g_launches.fetch_add((long long)I.kernels_run);
    else if (graph) g_launches.fetch_add((long long)I.body_runs * h->body_kernels);
    if (c.status)
        return fail(h, (pc_status)c.status,
                    h->learned ? "device-side error during the skeleton search (or a proposed sepset failed the FP64 re-verification)"
                               : "device-side error during the skeleton search");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    st->tests_executed = c.tests_executed;
    st->tests_canonical = c.tests_canonical;
    st->tests_redecided = c.redecided;
    st->band_hits = c.band_hits;
    st->guard_hits = c.guard_hits;
    st->degenerate = c.degenerate;
    st->complement_tests = c.complement_tests;
    st->edges_removed = c.edges_removed;
    st->edges_kept = I.edges / 2;
    unsigned int bits = c.max_dz_bits;
    float mdz;
    std::memcpy(&mdz, &bits, sizeof(mdz));
    st->max_abs_dz = mdz;
    st->t_skeleton_ms = ms;
    st->stage_a_ran = I.stage_a_ran;
    st->levels_run = I.levels_run;
    st->first_level = I.first_level;
    st->queue_overflows = c.queue_overflows;
    st->prec_builds = c.prec_builds;
    st->prec_downdates = c.prec_downdates;
    st->flops_class[1] = (double)c.flops_stagea + (I.stage_a_ran ? (double)p * p * p : 0.0);
    st->flops_class[2] = (double)c.flops_prec;
    st->flops_class[3] = (double)c.flops + (double)c.flops64_direct;
    st->flops_class[4] = (double)c.flops_comp;
    st->flops = st->flops_class[1] + st->flops_class[2] + st->flops_class[3] + st->flops_class[4];
    return PC_OK;
}

static pc_status skeleton_once(pc_handle *h, pc_stats *st, bool *overflow)
{
    if (pc_status r = skeleton_enqueue(h)) return r;
    return skeleton_complete(h, st, overflow);
}

static pc_status skeleton_run(pc_handle *h, pc_stats *st)
{
    for (int attempt = 0; attempt < 6; ++attempt) {
        bool overflow = false;
        if (pc_status r = skeleton_once(h, st, &overflow)) return r;
        if (!overflow) {
            // an overflowing FP64 re-decision queue made a stage re-run all its
            // tests on the warp-per-test kernel (correct, slow): a larger queue
            // for the later runs of this handle, up to 2^28 entries (2 GiB)
            if (st->queue_overflows > 0 && h->rq_cap < (1ull << 28)) {
                ull *nq = nullptr;
                const ull cap = h->rq_cap * 4;
                if (dalloc(h, &nq, (size_t)cap * sizeof(ull)) == cudaSuccess) {
                    dfree(h, h->rq);
                    h->rq = nq;
                    h->rq_cap = cap;
                }
            }
            return PC_OK;
        }
        // the sepset pool was too small: enlarge it and run again (deterministic)
        int *np = nullptr;
        long long cap = h->g.pool_cap * 4;
        CK(dalloc(h, &np, (size_t)cap * sizeof(int)));
        dfree(h, h->g.pool);
        h->g.pool = np;
        h->g.pool_cap = cap;
    }
    return fail(h, PC_ERR_INTERNAL, "sepset pool could not be sized");
}

static pc_status copy_adj(pc_handle *h, uint8_t *adj_out);

// Coordinate search over the launch shape of the test kernels: each knob in
// turn takes the candidate with the least mean skeleton time (CUDA events on
// the handle's stream, `reps` runs after one warm run); the others stay at
// their current best.  The skeleton and sepsets do not depend on the shape
// (frozen adjacency per stage, smallest key wins), so every run is a valid
// search and the handle keeps the fastest shape.
extern "C" pc_status pc_autotune(pc_handle *h, int32_t reps, pc_tune_result *out)
{
    if (!h || reps < 1 || reps > 100) return PC_ERR_ARG;
    if (!h->have_corr) return fail(h, PC_ERR_STATE, "pc_autotune before pc_corr");
    if (pc_status r = check_tc(h)) return r;
    static const int chunks[] = {4, 8, 16, 32};
    static const int rounds[] = {4, 16, 64, 256};
    static const int blocks[] = {4, 8, 16};
    static const int warps[] = {2, 4, 8};
    // the cost gate of the proposal order: the largest scored stage (0: none,
    // stage 0 has no sets to order), searched only when the handle enumerates in
    // the proposed order
    static const int lmaxs[] = {0, 2, 4, 8};
    struct Knob {
        int *field;
        const int *cand;
        int nc;
    } knobs[] = {{&h->lane_chunk, chunks, 4}, {&h->lane_rounds, rounds, 4}, {&h->lane_blocks, blocks, 3},
                 {&h->direct_warps, warps, 3}, {&h->learned_lmax, lmaxs, 4}};
    const int nknobs = (h->learned && h->have_params) ? 5 : 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    pc_status rs = PC_OK;
    int runs = 0;
    auto measure = [&](double *ms) -> pc_status {
        pc_stats st;
        if (pc_status r = skeleton_run(h, &st)) return r;            // warm run (graph capture)
        double tot = 0.0;
        for (int i = 0; i < reps; ++i) {
            CK(cudaEventRecord(e0, h->stream));
            if (pc_status r = skeleton_run(h, &st)) return r;
            CK(cudaEventRecord(e1, h->stream));
            CK(cudaEventSynchronize(e1));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e0, e1));
            tot += t;
        }
        runs += reps + 1;
        h->last = st;
        *ms = tot / reps;
        return PC_OK;
    };
    double best = 0.0;
    rs = measure(&best);
    const double first = best;
    for (int k = 0; k < nknobs && rs == PC_OK; ++k) {
        const int keep = *knobs[k].field;
        int pick = keep;
        for (int c = 0; c < knobs[k].nc && rs == PC_OK; ++c) {
            if (knobs[k].cand[c] == keep) continue;
            *knobs[k].field = knobs[k].cand[c];
            double t = 0.0;
            rs = measure(&t);
            if (rs == PC_OK && t < best) {
                best = t;
                pick = knobs[k].cand[c];
            }
        }
        *knobs[k].field = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != PC_OK) return rs;
    h->have_skel = true;
    if (out) {
        out->lane_chunk = h->lane_chunk;
        out->lane_rounds = h->lane_rounds;
        out->lane_blocks = h->lane_blocks;
        out->direct_warps = h->direct_warps;
        out->learned_max_level = h->learned_lmax;
        out->ms_default = first;
        out->ms_best = best;
        out->runs = runs;
    }
    return PC_OK;
}

// The search over the path-restricted pools adj(G,i,j) n path(G,i,j) of
// Algorithms 1 and 2 (Sec. 2.1 notation, option "path_pool"): PC-stable, one
// pool per unordered pair searched once (side 0), FP64 tests, driven from the
// host stage by stage.  Schedule as for the neighbour sets: Algorithm 1 runs
// l = 0, 1, ... while some pair's pool has at least l members; Algorithm 2 runs
// the closed-form stage l = p-2, then l = min(cap, p-3, largest pool) and
// l <- min(l-1, largest pool) down to 0.  The pools and the largest pool come
// from the graph as it is at the start of the stage.
static pc_status skeleton_pathpool_once(pc_handle *h, pc_stats *st, bool *overflow)
{
    GraphDev &g = h->g;
    cudaStream_t s = h->stream;
    const int p = h->p;
    const long long n = h->n;
    const size_t pp = h->pair_elems;
    *overflow = false;
    if (h->learned) return fail(h, PC_ERR_ARG, "path_pool: the proposal order does not apply to pair pools");
    if (!h->c64_full) {
        if (pc_status r = materialize_c64(h)) return r;
    }
    if (!h->pp_comp) {
        CK(dalloc(h, &h->pp_comp, (size_t)p * p * sizeof(int)));
        CK(dalloc(h, &h->pp_max, sizeof(int)));
    }
    TestParams tp = make_tp(h);
    tp.lazy = 0;                                         // the full FP64 matrix
    std::memset(st, 0, sizeof(*st));
    CK(cudaEventRecord(h->ev0, s));
    CK(fpc::launch_init_adj(g, s));
    CK(cudaMemsetAsync(g.best, 0xff, pp * sizeof(ull), s));
    CK(cudaMemsetAsync(g.sep_level, 0xff, pp * sizeof(int), s));
    CK(cudaMemsetAsync(g.sep_off, 0xff, pp * sizeof(long long), s));
    CK(cudaMemsetAsync(g.ctr, 0, sizeof(DevCounters), s));
    CK(cudaMemsetAsync(g.info, 0, sizeof(LevelInfo), s));
    CK(cudaMemsetAsync(h->singular, 0, sizeof(int), s));
    const int cap = level_cap(h);
    int levels = 0, first = -1, stage_a_ran = 0;
    auto largest_pool = [&](int *out) -> pc_status {
        CK(fpc::launch_pp_components(g, h->pp_comp, s));
        CK(cudaMemsetAsync(h->pp_max, 0xff, sizeof(int), s));
        CK(fpc::launch_pp_search(g, tp, h->C64, h->ldc, h->pp_comp, 0, 0, h->pp_max, h->budget, s));
        CK(cudaMemcpyAsync(out, h->pp_max, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return PC_OK;
    };
    auto stage = [&](int l) -> pc_status {
        if (l + 2 > fpc::DIRECT_MMAX) return fail(h, PC_ERR_BUDGET, "path_pool: a stage beyond l = 158");
        int status = 0;
        CK(cudaMemcpyAsync(&status, &g.ctr->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (status) return fail(h, (pc_status)status, "path_pool: a stage would exceed the test budget");
        CK(cudaMemsetAsync(&g.info->total_direct, 0, sizeof(unsigned long long), s));   // scheduled tests
        CK(fpc::launch_pp_search(g, tp, h->C64, h->ldc, h->pp_comp, l, 1, h->pp_max, h->budget, s));
        CK(fpc::launch_pp_commit(g, s));
        ++levels;
        if (first < 0) first = l;
        return PC_OK;
    };
    int mp = -1;
    if (h->order == 0) {
        for (int l = 0; l <= cap; ++l) {
            if (pc_status r = largest_pool(&mp)) return r;
            if (mp < l) break;
            if (pc_status r = stage(l)) return r;
        }
    } else {
        if (h->stage_a && n - p - 1 > 0) {
            // the closed-form stage l = p-2 on the complete graph (its only set is V\{u,v})
            CK(fpc::launch_level_degrees(g, s));
            CK(fpc::launch_tail(g, tp, cap, 2, h->singular, 0, h->hcond, 0, fpc::StageConds{}, s));
            CK(cudaMemcpyAsync(h->Pbuf, h->C64, (size_t)p * h->ldc * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CK(fpc::launch_inverse_spd(h->Pbuf, p, h->ldc, h->work, h->singular, s));
            CK(fpc::launch_stage_a_decide(h->Pbuf, p, h->ldc, h->singular, g, tp, s));
            CK(fpc::launch_commit(g, h->opair_cap, p - 2, 0, s));
            int sing = 0;
            CK(cudaMemcpyAsync(&sing, h->singular, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            stage_a_ran = sing ? 0 : 1;
            levels += stage_a_ran;
        }
        int l = cap;
        if (stage_a_ran && l > p - 3) l = p - 3;
        if (pc_status r = largest_pool(&mp)) return r;
        if (mp < l) l = mp;
        while (l >= 0) {
            if (pc_status r = stage(l)) return r;
            if (pc_status r = largest_pool(&mp)) return r;
            l = std::min(l - 1, mp);
        }
    }
    CK(cudaEventRecord(h->ev1, s));
    DevCounters c;
    CK(cudaMemcpyAsync(&c, g.ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
    if (pc_status r = read_info(h)) return r;
    if (h->info_h->pool_overflow) {
        *overflow = true;
        return PC_OK;
    }
    if (c.status) return fail(h, (pc_status)c.status, "device-side error in the path-pool search");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    st->tests_executed = c.tests_executed;
    st->tests_canonical = c.tests_canonical;
    st->degenerate = c.degenerate;
    st->tests_redecided = 0;
    st->edges_removed = c.edges_removed;
    st->edges_kept = (uint64_t)p * (p - 1) / 2 - c.edges_removed;
    st->levels_run = levels;
    st->first_level = first;
    st->stage_a_ran = stage_a_ran;
    st->t_skeleton_ms = ms;
    return PC_OK;
}

static pc_status skeleton_pathpool(pc_handle *h, pc_stats *st)
{
    for (int attempt = 0; attempt < 6; ++attempt) {
        bool overflow = false;
        if (pc_status r = skeleton_pathpool_once(h, st, &overflow)) return r;
        if (!overflow) return PC_OK;
        // the sepset pool was too small: enlarge it and run again (deterministic)
        int *np = nullptr;
        const long long cap = h->g.pool_cap * 4;
        CK(dalloc(h, &np, (size_t)cap * sizeof(int)));
        dfree(h, h->g.pool);
        h->g.pool = np;
        h->g.pool_cap = cap;
    }
    return fail(h, PC_ERR_INTERNAL, "sepset pool could not be sized");
}

extern "C" pc_status pc_skeleton(pc_handle *h, uint8_t *adj_out, pc_stats *stats)
{
    if (!h) return PC_ERR_ARG;
    if (!h->have_corr) return fail(h, PC_ERR_STATE, "pc_skeleton before pc_corr");
    if (pc_status r = check_tc(h)) return r;
    pc_stats st;
    pc_status r = h->path_pool ? skeleton_pathpool(h, &st) : skeleton_run(h, &st);
    if (r != PC_OK) return r;
    h->last = st;
    h->have_skel = true;
    if (stats) *stats = st;
    if (adj_out) return copy_adj(h, adj_out);
    return PC_OK;
}

// The skeleton as a p x p 0/1 matrix: expanded from the bitset on the device, into
// adj_out directly when it is device memory, else through a device staging buffer.
static pc_status copy_adj(pc_handle *h, uint8_t *adj_out)
{
    const size_t bytes = (size_t)h->p * h->p;
    cudaStream_t s = h->stream;
    if (is_device_ptr(adj_out)) {
        CK(fpc::launch_expand_adj(h->g, adj_out, s));
    } else {
        if (h->adj_stage_bytes < bytes) {
            dfree(h, h->adj_stage);
            h->adj_stage = nullptr;
            CK(dalloc(h, &h->adj_stage, bytes));
            h->adj_stage_bytes = bytes;
        }
        CK(fpc::launch_expand_adj(h->g, h->adj_stage, s));
        CK(cudaMemcpyAsync(adj_out, h->adj_stage, bytes, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return PC_OK;
}

extern "C" pc_status pc_skeleton_many(pc_handle **hs, int32_t count, uint8_t **adj_out, pc_stats *stats,
                                      pc_status *status)
{
    if (!hs || count < 0) return PC_ERR_ARG;
    std::vector<pc_status> st((size_t)count, PC_OK);
    // phase 1: every search is enqueued on its handle's stream (no host wait)
    for (int i = 0; i < count; ++i) {
        pc_handle *h = hs[i];
        if (!h) {
            st[i] = PC_ERR_ARG;
            continue;
        }
        if (!h->have_corr) {
            st[i] = fail(h, PC_ERR_STATE, "pc_skeleton_many: handle without pc_corr");
            continue;
        }
        st[i] = check_tc(h);
        if (st[i] == PC_OK) st[i] = skeleton_enqueue(h);
    }
    // phase 2: each search completes on its own stream
    pc_status first = PC_OK;
    for (int i = 0; i < count; ++i) {
        pc_handle *h = hs[i];
        pc_stats one;
        std::memset(&one, 0, sizeof(one));
        if (st[i] == PC_OK) {
            bool overflow = false;
            st[i] = skeleton_complete(h, &one, &overflow);
            if (st[i] == PC_OK && overflow) st[i] = skeleton_run(h, &one);   // larger pool, serial rerun
        }
        if (st[i] == PC_OK) {
            h->last = one;
            h->have_skel = true;
            if (adj_out && adj_out[i]) st[i] = copy_adj(h, adj_out[i]);
        }
        if (stats) stats[i] = one;
        if (status) status[i] = st[i];
        if (st[i] != PC_OK && first == PC_OK) first = st[i];
    }
    return first;
}

// every pair a < b of the handle's problem(s) in ascending (a, b) with its
// index in the per-pair arrays
template <class F>
static void for_pairs(const pc_handle *h, F fn)
{
    if (!h->nblk) {
        const int p = h->p;
        for (int a = 0; a < p; ++a)
            for (int b = a + 1; b < p; ++b) fn(a, b, (size_t)a * p + b);
        return;
    }
    for (int i = 0; i < h->nblk; ++i) {
        const int o = h->boff[i], pb = h->boff[i + 1] - o;
        for (int a = o; a < o + pb; ++a)
            for (int b = a + 1; b < o + pb; ++b)
                fn(a, b, (size_t)h->pbase[i] + (size_t)(a - o) * pb + (b - o));
    }
}

extern "C" pc_status pc_sepsets_count(pc_handle *h, int64_t *n_removed, int64_t *pool_len)
{
    if (!h) return PC_ERR_ARG;
    if (!h->have_skel) return fail(h, PC_ERR_STATE, "no skeleton yet");
    std::vector<int> lv(h->pair_elems);
    CK(cudaMemcpy(lv.data(), h->g.sep_level, lv.size() * sizeof(int), cudaMemcpyDeviceToHost));
    long long cnt = 0;
    for_pairs(h, [&](int, int, size_t e) { cnt += lv[e] >= 0; });
    if (n_removed) *n_removed = cnt;
    if (pool_len) {
        ull pl = 0;
        CK(cudaMemcpy(&pl, &h->g.ctr->pool_len, sizeof(ull), cudaMemcpyDeviceToHost));
        *pool_len = (int64_t)pl;
    }
    return PC_OK;
}

extern "C" pc_status pc_sepsets_get(pc_handle *h, int32_t *pairs, int32_t *level, int32_t *side,
                                    int64_t *rank, int64_t *off, int32_t *pool)
{
    if (!h) return PC_ERR_ARG;
    if (!h->have_skel) return fail(h, PC_ERR_STATE, "no skeleton yet");
    const size_t pp = h->pair_elems;
    std::vector<int> lv(pp), sd(pp);
    std::vector<long long> rk(pp), of(pp);
    CK(cudaMemcpy(lv.data(), h->g.sep_level, pp * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(sd.data(), h->g.sep_side, pp * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rk.data(), h->g.sep_rank, pp * sizeof(long long), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(of.data(), h->g.sep_off, pp * sizeof(long long), cudaMemcpyDeviceToHost));
    long long k = 0;
    for_pairs(h, [&](int a, int b, size_t e) {
        if (lv[e] < 0) return;
        if (pairs) { pairs[2 * k] = a; pairs[2 * k + 1] = b; }
        if (level) level[k] = lv[e];
        if (side) side[k] = sd[e];
        if (rank) rank[k] = rk[e];
        if (off) off[k] = of[e];
        ++k;
    });
    if (pool) {
        ull pl = 0;
        CK(cudaMemcpy(&pl, &h->g.ctr->pool_len, sizeof(ull), cudaMemcpyDeviceToHost));
        if (pl) CK(cudaMemcpy(pool, h->g.pool, (size_t)pl * sizeof(int), cudaMemcpyDeviceToHost));
    }
    return PC_OK;
}

// ---------------------------------------------------------------- orientation
// Algorithm 1, Phase II on the last skeleton and its separation sets: colliders,
// then rounds of R1-R4 until one orients nothing (order-free reading).
extern "C" pc_status pc_orient(pc_handle *h, int8_t *codes_out, int32_t *rounds_out)
{
    if (!h) return PC_ERR_ARG;
    if (!h->have_skel) return fail(h, PC_ERR_STATE, "pc_orient before pc_skeleton");
    if (!codes_out) return fail(h, PC_ERR_ARG, "pc_orient: codes_out is null");
    cudaStream_t s = h->stream;
    const size_t words = (size_t)h->p * h->g.W;
    if (!h->or_mk) {
        CK(dalloc(h, &h->or_mk, 4 * words * sizeof(uint32_t)));
        CK(dalloc(h, &h->or_changed, sizeof(int)));
    }
    uint32_t *ah = h->or_mk, *at = ah + words, *ah2 = at + words, *at2 = ah2 + words;
    CK(fpc::launch_orient_colliders(h->g, ah, at, s));
    // each round that changes something adds a mark; there are at most 32 W p marks
    const long long max_rounds = (long long)words * 32 + 1;
    int32_t rounds = 0;
    for (;;) {
        CK(fpc::launch_orient_round(h->g, ah, at, ah2, at2, h->or_changed, s));
        int changed = 0;
        CK(cudaMemcpyAsync(&changed, h->or_changed, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::swap(ah, ah2);
        std::swap(at, at2);
        if (!changed) break;
        if (++rounds > max_rounds) return fail(h, PC_ERR_INTERNAL, "pc_orient: rules did not settle");
    }
    const size_t pp = (size_t)h->p * h->p;
    int8_t *dst = codes_out;
    if (!is_device_ptr(codes_out)) {
        if (!h->or_codes) CK(dalloc(h, &h->or_codes, pp));
        dst = h->or_codes;
    }
    CK(fpc::launch_orient_codes(h->g, ah, at, dst, s));
    if (dst != codes_out) CK(cudaMemcpyAsync(codes_out, dst, pp, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (rounds_out) *rounds_out = rounds;
    return PC_OK;
}

// ---------------------------------------------------------------- raw tests
extern "C" pc_status pc_ci_batch(pc_handle *h, const int32_t *ij, const int32_t *S, int32_t l,
                                 int64_t b, double *r_out, uint8_t *indep_out, float *z_out)
{
    if (!h) return PC_ERR_ARG;
    if (!h->have_corr) return fail(h, PC_ERR_STATE, "pc_ci_batch before pc_corr");
    if (l < 0 || l > h->p - 2 || l > 126 || b < 0 || !ij || (l > 0 && !S))
        return fail(h, PC_ERR_ARG, "pc_ci_batch: bad l, b or pointers");
    // batched problems: the smallest instance bounds l for every test
    if ((h->nblk ? h->n_min : h->n) - l - 3 <= 0) return fail(h, PC_ERR_DOF, "n - l - 3 <= 0");
    if (b == 0) return PC_OK;
    cudaStream_t s = h->stream;
    TestParams tp = make_tp(h);
    tp.dr_max = 5e-6f;                                   // r itself is returned
    CK(cudaMemsetAsync(h->g.ctr, 0, sizeof(DevCounters), s));
    CK(fpc::launch_ci_list(ij, S, l, b, h->C32, h->C64, h->ldc, h->p, tp, r_out, indep_out, z_out,
                           h->g.ctr, h->g.blk_lo, h->g.blk_hi, s));
    CK(cudaMemcpyAsync(h->ctr_h, h->g.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->ctr_h->status)
        return fail(h, (pc_status)h->ctr_h->status,
                    "pc_ci_batch: node id out of range, u == v, or nodes of different instances");
    std::memset(&h->last, 0, sizeof(h->last));
    h->last.tests_executed = h->ctr_h->tests_executed;
    h->last.tests_redecided = h->ctr_h->redecided;
    h->last.band_hits = h->ctr_h->band_hits;
    h->last.guard_hits = h->ctr_h->guard_hits;
    h->last.degenerate = h->ctr_h->degenerate;
    return PC_OK;
}

extern "C" pc_status pc_last_stats(pc_handle *h, pc_stats *out)
{
    if (!h || !out) return PC_ERR_ARG;
    *out = h->last;
    return PC_OK;
}

// ---------------------------------------------------------------- proposal network
extern "C" int32_t pc_mlp_nparam(void) { return fpc::mlp_nparam(); }

extern "C" pc_status pc_mlp_set_params(pc_handle *h, const float *theta, int64_t count)
{
    if (!h || !theta || count != fpc::mlp_nparam()) return PC_ERR_ARG;
    cudaStream_t s = h->stream;
    const size_t bytes = (size_t)count * sizeof(float);
    CK(cudaMemcpyAsync(h->theta, theta, bytes, cudaMemcpyDefault, s));
    CK(cudaMemsetAsync(h->adam_m, 0, bytes, s));
    CK(cudaMemsetAsync(h->adam_v, 0, bytes, s));
    CK(fpc::launch_mlp_pack(h->theta, h->wpack, s));
    CK(cudaStreamSynchronize(s));
    h->have_params = true;
    h->adam_step = 0;
    return PC_OK;
}

extern "C" pc_status pc_mlp_get_params(pc_handle *h, float *theta, int64_t count)
{
    if (!h || !theta || count != fpc::mlp_nparam()) return PC_ERR_ARG;
    if (!h->have_params) return fail(h, PC_ERR_STATE, "no parameters set");
    CK(cudaMemcpyAsync(theta, h->theta, (size_t)count * sizeof(float), cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PC_OK;
}

extern "C" pc_status pc_mlp_features(pc_handle *h, const int32_t *quads, int64_t R, float *feats)
{
    if (!h || (R > 0 && (!quads || !feats)) || R < 0) return PC_ERR_ARG;
    if (!h->have_corr) return fail(h, PC_ERR_STATE, "pc_mlp_features before pc_corr");
    if (R == 0) return PC_OK;
    CK(cudaMemsetAsync(h->mlp_err, 0, sizeof(int), h->stream));
    CK(fpc::launch_mlp_features(quads, R, h->C32, h->ldc, h->g.prow, h->p, h->n, h->g.nvec, h->q, feats,
                                h->mlp_err, h->stream));
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->mlp_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (e) return fail(h, PC_ERR_ARG, "pc_mlp_features: node id out of range or repeated in a quadruple");
    return PC_OK;
}

// forward (and, with h1/h2, the activations a backward pass needs)
static pc_status mlp_forward(pc_handle *h, const float *feats, long long R, float *scores, __nv_bfloat16 *h1,
                             float *h2)
{
    CK(cudaMemsetAsync(h->mlp_err, 0, sizeof(int), h->stream));
    CK(fpc::launch_mlp_forward_feats(feats, R, h->wpack, h->theta, scores, h1, h2, h->mlp_err, h->g, h->stream));
    return PC_OK;
}

static pc_status mlp_check_err(pc_handle *h)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->mlp_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (e) return fail(h, (pc_status)e, "proposal network: a bounded wait in the tensor-core forward pass expired");
    return PC_OK;
}

extern "C" pc_status pc_mlp_forward(pc_handle *h, const float *feats, int64_t R, float *scores)
{
    if (!h || R < 0 || (R > 0 && (!feats || !scores))) return PC_ERR_ARG;
    if (!h->have_params) return fail(h, PC_ERR_STATE, "no parameters set");
    if (R == 0) return PC_OK;
    if (pc_status r = mlp_forward(h, feats, R, scores, nullptr, nullptr)) return r;
    return mlp_check_err(h);
}

struct MlpWork {
    float *scores = nullptr, *h2 = nullptr;
    __nv_bfloat16 *h1 = nullptr;
};

static pc_status mlp_work(pc_handle *h, long long rows, MlpWork &w)
{
    CK(dalloc(h, &w.scores, (size_t)rows * sizeof(float)));
    CK(dalloc(h, &w.h2, (size_t)rows * 128 * sizeof(float)));
    CK(dalloc(h, &w.h1, (size_t)rows * 128 * sizeof(__nv_bfloat16)));
    return PC_OK;
}

static void mlp_work_free(pc_handle *h, MlpWork &w)
{
    dfree(h, w.scores);
    dfree(h, w.h2);
    dfree(h, w.h1);
}

extern "C" pc_status pc_mlp_grad(pc_handle *h, const float *feats, const float *labels, int64_t R, float *grad_out,
                                 double *loss)
{
    if (!h || R <= 0 || !feats || !labels) return PC_ERR_ARG;
    if (!h->have_params) return fail(h, PC_ERR_STATE, "no parameters set");
    MlpWork w;
    pc_status st = mlp_work(h, R, w);
    if (st == PC_OK) st = mlp_forward(h, feats, R, w.scores, w.h1, w.h2);
    if (st == PC_OK) {
        cudaError_t e = cudaMemsetAsync(h->mlp_loss, 0, sizeof(double), h->stream);
        if (e == cudaSuccess)
            e = h->mlp_bwd_tc
                    ? fpc::launch_mlp_backward_tc(feats, labels, w.scores, w.h1, w.h2, R, 1.0f / (float)R, h->theta,
                                                  h->wpack, h->grad, h->mlp_loss, h->mlp_err, h->stream)
                    : fpc::launch_mlp_backward(feats, labels, w.scores, w.h1, w.h2, R, 1.0f / (float)R, h->theta,
                                               h->grad, h->mlp_loss, h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "pc_mlp_grad");
    }
    if (st == PC_OK) st = mlp_check_err(h);
    if (st == PC_OK && grad_out) {
        cudaError_t e = cudaMemcpy(grad_out, h->grad, (size_t)fpc::mlp_nparam() * sizeof(float), cudaMemcpyDefault);
        if (e != cudaSuccess) st = cuda_fail(h, e, "pc_mlp_grad copy");
    }
    if (st == PC_OK && loss) {
        double ls = 0;
        cudaError_t e = cudaMemcpy(&ls, h->mlp_loss, sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(h, e, "pc_mlp_grad loss");
        *loss = ls / (double)R;
    }
    cudaStreamSynchronize(h->stream);
    mlp_work_free(h, w);
    return st;
}

extern "C" pc_status pc_mlp_train(pc_handle *h, const float *feats, const float *labels, int64_t R, int32_t epochs,
                                  int64_t batch, double lr, double *final_loss)
{
    if (!h || R <= 0 || !feats || !labels || epochs < 1 || batch < 1 || !(lr > 0)) return PC_ERR_ARG;
    if (!h->have_params) return fail(h, PC_ERR_STATE, "no parameters set");
    const long long B = std::min<long long>(batch, R);
    MlpWork w;
    pc_status st = mlp_work(h, B, w);
    cudaStream_t s = h->stream;
    double last = 0.0;
    for (int ep = 0; ep < epochs && st == PC_OK; ++ep) {
        cudaError_t e = cudaMemsetAsync(h->mlp_loss, 0, sizeof(double), s);
        for (long long b0 = 0; b0 < R && e == cudaSuccess && st == PC_OK; b0 += B) {
            const long long nb = std::min<long long>(B, R - b0);
            st = mlp_forward(h, feats + b0 * 16, nb, w.scores, w.h1, w.h2);
            if (st != PC_OK) break;
            e = h->mlp_bwd_tc
                    ? fpc::launch_mlp_backward_tc(feats + b0 * 16, labels + b0, w.scores, w.h1, w.h2, nb,
                                                  1.0f / (float)nb, h->theta, h->wpack, h->grad, h->mlp_loss,
                                                  h->mlp_err, s)
                    : fpc::launch_mlp_backward(feats + b0 * 16, labels + b0, w.scores, w.h1, w.h2, nb,
                                               1.0f / (float)nb, h->theta, h->grad, h->mlp_loss, s);
            if (e == cudaSuccess) e = fpc::launch_adam(h->theta, h->grad, h->adam_m, h->adam_v, (float)lr, ++h->adam_step, s);
            if (e == cudaSuccess) e = fpc::launch_mlp_pack(h->theta, h->wpack, s);
        }
        if (e != cudaSuccess && st == PC_OK) st = cuda_fail(h, e, "pc_mlp_train");
        if (st == PC_OK) {
            double ls = 0;
            e = cudaMemcpyAsync(&ls, h->mlp_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(h, e, "pc_mlp_train loss");
            last = ls / (double)R;
        }
    }
    if (st == PC_OK) st = mlp_check_err(h);
    cudaStreamSynchronize(s);
    mlp_work_free(h, w);
    if (final_loss) *final_loss = last;
    return st;
}
