// level.cu -- one PC-stable stage of the skeleton search (the stage body of
// Algorithm 1 / Algorithm 2) on the GPU.
//
//  degrees      frozen neighbour lists (ascending) from the adjacency bitset
//  counts+scan  C(d, l) tests per adjacent ordered pair (u,v), d = |adj(u)\{v}|,
//               split between the direct path and the complement path
//  ci_direct    one warp per test: gather corr[S u {u,v}] into shared memory,
//               Cholesky of the S block, the trailing 2x2 is the Schur complement
//               H = H0 - H1 H2^{-1} H1^T of Sec. 4, rho = h12/sqrt(h11 h22),
//               Fisher z (Eq. 1); FP32 with an FP64 re-decision when the pivot
//               guard or the |z - q| band says FP32 cannot be trusted
//  ci_complement  high stages of the reversed order: with P = corr[F,F]^{-1},
//               F = adj(u) u {u}, and R = F \ (S u {u,v}) (|R| = d - l small),
//               the {u,v} block of corr[T,T]^{-1} (T = S u {u,v}) is
//               P_TT - P_TR P_RR^{-1} P_RT, one k x k solve per test
//  commit       delete the recorded edges (PC-stable, end of stage), expand the
//               first separating set of each removed pair, count the tests of
//               the sequential canonical order
#include "internal.h"
#include "device_util.cuh"
#include <algorithm>
#include <cooperative_groups.h>

namespace fpc {

namespace cg = cooperative_groups;

typedef unsigned long long ull;

__device__ __forceinline__ ull sat_add(ull a, ull b)
{
    ull c = a + b;
    return c < a ? KEY_NONE : c;
}


// small-stage kernel instantiation that runs stage l (l <= LANE_LMAX)
__host__ __device__ __forceinline__ int lane_range_of_dev(int l)
{
    return l <= 2 ? 0 : (l <= 4 ? 1 : (l <= 6 ? 2 : (l <= 8 ? 3 : (l <= 10 ? 4 : 5))));
}
int lane_range_of(int l) { return lane_range_of_dev(l); }

// samples behind the tests of node u (batched problems: its instance's n)
__device__ __forceinline__ long long n_of(const TestParams &tp, int u)
{
    return tp.nvec ? __ldg(tp.nvec + u) : tp.n;
}

// node u has tests at stage l only while n_u - l - 3 > 0 (one problem: the
// stage cap n - 4 already ensures it; batched problems differ in n)
__device__ __forceinline__ bool dof_ok(const TestParams &tp, int u, int l)
{
    return !tp.nvec || n_of(tp, u) - l - 3 > 0;
}

// the stage loop has finished or has been halted: nothing to do
__device__ __forceinline__ bool stopped(const LevelInfo *I) { return I->done || I->halt; }

// ---------------------------------------------------------------- frozen graph
// The complete graph (Algorithm 1/2 input): every bit v != u of row u set.
__global__ void init_adj_kernel(GraphDev g)
{
    const long long tot = (long long)g.p * g.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(i / g.W), w = (int)(i % g.W);
        uint32_t bits = 0xffffffffu;
        const int lo = w * 32;
        if (lo + 32 > g.p) bits = g.p - lo >= 32 ? 0xffffffffu : ((1u << (g.p - lo)) - 1u);
        if (u >= lo && u < lo + 32) bits &= ~(1u << (u - lo));
        if (g.blk_lo) {
            // batched problems: only nodes of u's own instance are adjacent
            const int b0 = g.blk_lo[u] - lo, b1 = g.blk_hi[u] - lo;
            const uint32_t keep_lo = b0 <= 0 ? 0xffffffffu : (b0 >= 32 ? 0u : ~((1u << b0) - 1u));
            const uint32_t keep_hi = b1 >= 32 ? 0xffffffffu : (b1 <= 0 ? 0u : ((1u << b1) - 1u));
            bits &= keep_lo & keep_hi;
        }
        g.adj[i] = bits;
    }
}

// Degrees and ascending neighbour lists of the current graph, one warp per node.
// Frozen neighbour list (ascending) and degree of node u from its adjacency row, by
// the calling warp.  l2: read the row through L2 (words other CTAs of the running
// kernel cleared with atomics).
__device__ __forceinline__ void node_degree(const GraphDev &g, int u, int lane, bool l2)
{
    const int old = lane == 0 ? (l2 ? __ldcg(g.deg + u) : g.deg[u]) : 0;
    const uint32_t *row = g.adj + (long long)u * g.W;
    int base = 0;
    for (int w0 = 0; w0 < g.W; w0 += 32) {
        const int w = w0 + lane;
        uint32_t bits = (w < g.W) ? (l2 ? __ldcg(row + w) : row[w]) : 0u;
        const int c = __popc(bits);
        int incl = c;
        for (int off = 1; off < 32; off <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        int pos = base + incl - c;
        while (bits) {
            int t = __ffs(bits) - 1;
            g.nbr[nidx(g, u) + pos++] = w * 32 + t;
            bits &= bits - 1;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        g.deg[u] = base;
        g.dchg[u] = old - base;
    }
}

__global__ void degrees_kernel(GraphDev g)
{
    const int lane = threadIdx.x & 31;
    const int u = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (u >= g.p || stopped(g.info)) return;
    node_degree(g, u, lane, false);
}

__device__ void tail_body(GraphDev g, TestParams tp, int cap, int mode, const int *stagea_singular,
                          int stagea_launched, cudaGraphConditionalHandle hc, int use_cond, StageConds sc,
                          bool fused);

// The degrees of a stage's frozen graph, then the stage tail (mode 0) in the last
// CTA to finish: the CTAs publish their degrees, take a ticket, and the last one
// resets the ticket and runs tail_body on the complete degree array.
__global__ void __launch_bounds__(256) degrees_tail_kernel(GraphDev g, TestParams tp, int cap,
                                                           cudaGraphConditionalHandle hc, int use_cond, StageConds sc)
{
    const int lane = threadIdx.x & 31;
    const int u = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (u < g.p && !stopped(g.info)) node_degree(g, u, lane, false);
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&g.info->deg_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) g.info->deg_ticket = 0u;     // every CTA has taken its ticket
    tail_body(g, tp, cap, 0, nullptr, 0, hc, use_cond, sc, true);
}

// Stages 1 and 2: the pairs of a node of degree above pair_warp_dmin run one
// warp per pair.
__device__ __forceinline__ bool pair_warped(const TestParams &tp, int l, int dg)
{
    return tp.pair_warp && l >= 1 && l <= PAIRWARP_LMAX && dg > tp.pair_warp_dmin;
}

// The small-stage tests of a node of degree dg at stage l >= 1 run on the staged
// kernel when its neighbourhood block fits the shared-memory layout (and the
// node is not one of the warp-per-pair kernel).
__device__ __forceinline__ bool node_staged(const TestParams &tp, int l, int dg)
{
    return l >= 1 && dg <= tp.node_dmax && !pair_warped(tp, l, dg);
}

// Chunk of the staged kernel for a node with T sets per pair and dg pairs: the
// lane chunk, smaller when the node has too few tests to give every thread of
// a CTA one chunk.
__device__ __forceinline__ ull node_chunk(const TestParams &tp, ull T, int dg)
{
    const ull fair = T * (ull)dg / NODE_THREADS;       // T * dg < 2^64: T <= C(127, 12), dg <= 128
    return fair < (ull)tp.lane_chunk ? (fair > 0 ? fair : 1ull) : (ull)tp.lane_chunk;
}

__device__ __forceinline__ bool comp_eligible(int d, int l, const TestParams &tp)
{
    const int k = d - l;
    return tp.reversed && tp.complement && d >= l && k <= KC_MAX && k < l && d + 2 <= PREC_MAX;
}

// One CTA after the degrees: ordered-pair offsets, L* = max |adj(u)\{v}|, edge
// count; then (mode 1) the first stage or (mode 0) the next stage, the loop
// condition, and the precision-block requests of that stage.  Mode 2 only
// scans (the complete graph before the closed-form stage).
//   Algorithm 1: l = 0, 1, ... while some pair has |adj(u)\{v}| >= l and l <= cap.
//   Algorithm 2: l = min(cap, L*) (below p-2 once the closed-form stage ran),
//                then l <- min(l-1, L*) while l >= 0.
// The tail of a stage (any block size that is a multiple of 32, up to 1024): the
// scan of the degrees into ordered-pair offsets, L*, the next stage and the loop
// condition, and the precision-block requests.  fused: run by the last CTA of the
// degrees kernel (which counts itself), whose other CTAs wrote deg: read through L2.
__device__ void tail_body(GraphDev g, TestParams tp, int cap, int mode, const int *stagea_singular,
                          int stagea_launched, cudaGraphConditionalHandle hc, int use_cond, StageConds sc,
                          bool fused)
{
    LevelInfo *I = g.info;
    __shared__ long long part[1024];
    __shared__ int smax[1024];
    __shared__ int sh_l, sh_go, sh_need, sh_removed;
    const int p = g.p, t = threadIdx.x;
    if (mode == 0 && t == 0) I->body_runs++;
    const int self = fused ? 0 : 1;                       // this kernel, when it is a launch of its own
    if (stopped(I)) {
        if (use_cond && t == 0) cudaGraphSetConditional(hc, 0u);
        if (sc.use && sc.has_prec && t == 0) cudaGraphSetConditional(sc.prec, 0u);
        if (sc.use && t == 0) I->kernels_run += self;
        return;
    }
    if (t == 0) sh_need = 0;
    const int nth = blockDim.x;                          // 32..1024, a multiple of 32
    const int per = (p + nth - 1) / nth;
    const int s0 = min(p, t * per), s1 = min(p, s0 + per);
    long long sum = 0;
    int mx = 0;
    for (int i = s0; i < s1; ++i) {
        const int dg = __ldcg(g.deg + i);
        sum += dg;
        mx = max(mx, dg);
    }
    part[t] = sum;
    smax[t] = mx;
    __syncthreads();
    for (int off = 1; off < nth; off <<= 1) {
        long long v = (t >= off) ? part[t - off] : 0;
        int m2 = (t >= off) ? smax[t - off] : 0;
        __syncthreads();
        part[t] += v;
        smax[t] = max(smax[t], m2);
        __syncthreads();
    }
    long long run = part[t] - sum;
    for (int i0 = s0; i0 < s1; i0 += 8) {              // batches of independent loads, then the stores
        int dv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) dv[k] = i0 + k < s1 ? __ldcg(g.deg + i0 + k) : 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (i0 + k < s1) {
                g.ooff[i0 + k] = run;
                run += dv[k];
            }
    }
    if (t == 0) {
        const long long tot = part[nth - 1];
        const int lstar = smax[nth - 1] - 1;              // -1 when no edge is left
        g.ooff[p] = tot;
        I->n_opairs = tot;
        sh_removed = I->edges != (unsigned long long)tot;   // the commit deleted edges
        I->edges = (unsigned long long)tot;
        I->lstar = lstar;
        if (mode == 1) {
            const int ran = stagea_launched && !*stagea_singular;
            I->stage_a_ran = ran;
            I->levels_run = ran;
            int l;
            bool go;
            if (tp.reversed) {
                l = cap;
                if (ran && l > p - 3) l = p - 3;
                if (lstar < l) l = lstar;
                go = l >= 0;
            } else {
                l = 0;
                go = cap >= 0 && lstar >= 0;
            }
            I->l = l;
            I->first_level = go ? l : -1;
            I->done = !go;
        } else if (mode == 0) {
            I->levels_run++;
            const int l = I->l;
            int nl;
            bool go;
            if (tp.reversed) {
                nl = min(l - 1, lstar);
                go = nl >= 0;
            } else {
                nl = l + 1;
                go = nl <= cap && lstar >= nl;
            }
            I->l = nl;
            I->done = !go;
        }
        sh_l = I->l;
        sh_go = !I->done;
    }
    __syncthreads();
    if (mode != 2 && sh_go && tp.reversed && tp.complement) {
        // precision blocks: all nodes that fit at the first stage, then the nodes
        // that have become small enough for the complement path at this stage
        for (int u = t; u < p; u += blockDim.x) {
            const int dg = __ldcg(g.deg + u);
            bool need;
            const int pmu = g.prec_m[u];
            if (mode == 1) need = dg >= 2 && dg + 1 <= PREC_MAX && pmu == 0;
            else need = dg > 0 && comp_eligible(dg - 1, sh_l, tp) && (pmu == 0 || pmu == -2);
            g.prec_need[u] = need;
            if (need) sh_need = 1;
        }
    }
    __syncthreads();
    if (use_cond && t == 0) cudaGraphSetConditional(hc, sh_go ? 1u : 0u);
    if (sc.use && sc.has_prec && t == 0) {
        // precision blocks change when a node asks for one or blocks lost members
        const int run = sh_go && (sh_need || sh_removed);
        cudaGraphSetConditional(sc.prec, run ? 1u : 0u);
        I->kernels_run += self + (run ? 1 : 0);          // the tail itself, the precision update
    } else if (sc.use && t == 0) {
        I->kernels_run += self;
    }
}

__global__ void __launch_bounds__(1024) tail_kernel(GraphDev g, TestParams tp, int cap, int mode,
                                                    const int *stagea_singular, int stagea_launched,
                                                    cudaGraphConditionalHandle hc, int use_cond, StageConds sc)
{
    tail_body(g, tp, cap, mode, stagea_singular, stagea_launched, hc, use_cond, sc, false);
}

__device__ __forceinline__ ull sat_mul(ull a, ull b)
{
    if (a == 0 || b == 0) return 0;
    if (a == KEY_NONE || b == KEY_NONE || a > KEY_NONE / b) return KEY_NONE;
    return a * b;
}

// The stage body's switch node (captured loop): which small-stage kernel range
// runs, or the warp-per-test kernel, and whether the complement and scoring
// kernels do.
__device__ __forceinline__ void set_stage_conds(const StageConds &sc, LevelInfo *I, int lane, int direct, int comp,
                                                int score, int lane_kernels)
{
    const int kind = lane < LANE_RANGES ? lane : (direct ? STAGE_KIND_DIRECT : STAGE_KIND_NONE);
    comp = comp && sc.has_comp;
    score = score && sc.has_score && kind != STAGE_KIND_NONE;
    cudaGraphSetConditional(sc.tests, (unsigned)stage_branch(kind, comp, score, sc.has_comp, sc.has_score));
    // head, commit, degrees + tail, the lane branch (kernel, [FP64 entries: collect, fill,]
    // FP64 pass, overflow pass) and the rest (the tail counts the precision update)
    I->kernels_run += STAGE_FIXED_KERNELS + (lane < LANE_RANGES ? lane_kernels : 0) + (kind == STAGE_KIND_DIRECT) +
                      comp + 2 * score;
}

// Exclusive saturating scan of NV values per thread over a block of up to 1024
// threads (warp shuffles, then one warp over the warp totals): ex[] receives the
// thread's exclusive prefixes, tot[] the block totals.  sh: 32*NV scratch.
template <int NV>
__device__ __forceinline__ void block_scan_sat(const ull (&v)[NV], ull (&ex)[NV], ull (&tot)[NV], ull *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    ull inc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        inc[k] = v[k];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const ull y = __shfl_up_sync(0xffffffffu, inc[k], off);
            if (lane >= off) inc[k] = sat_add(inc[k], y);
        }
        if (lane == 31) sh[k * 32 + w] = inc[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            ull x = lane < nw ? sh[k * 32 + lane] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const ull y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x = sat_add(x, y);
            }
            sh[k * 32 + lane] = x;                        // inclusive over warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const ull wex = __shfl_up_sync(0xffffffffu, inc[k], 1);
        const ull base = w ? sh[k * 32 + w - 1] : 0ull;
        ex[k] = sat_add(base, lane ? wex : 0ull);
        tot[k] = sh[k * 32 + nw - 1];
    }
    __syncthreads();                                      // sh reusable
}

// Work of stage l per node u: every ordered pair (u, v) has C(d, l) tests,
// d = |adj(u)| - 1, all on the direct path or all on the complement path.
// One CTA scans the per-node totals into tn_off / cn_off and gates the stage:
// budget and saturation (PC_ERR_BUDGET), or direct tests at an l larger than
// the direct kernel's shared-memory layout (the host runs that stage).  In the
// stages of the small-stage kernel it also lays out its rank-major rounds.
constexpr int HEAD_PER_MAX = MAXP_BATCH / 1024;           // nodes per thread at most
__device__ __noinline__ void head_body(const GraphDev &g, const TestParams &tp, double budget, int mmax_direct,
                                          const StageConds &conds)
{
    LevelInfo *I = g.info;
    if (stopped(I)) {
        if (conds.use && threadIdx.x == 0) set_stage_conds(conds, I, LANE_RANGES, 0, 0, 0, 0);
        return;
    }
    __shared__ ull sh[6 * 32];                           // scratch of block_scan_sat<6>
    const int p = g.p, l = I->l, t = threadIdx.x;
    const int per = (p + (int)blockDim.x - 1) / (int)blockDim.x;   // <= HEAD_PER_MAX
    const int s0 = min(p, t * per), s1 = min(p, s0 + per);
    // tests per pair of each of this thread's nodes; 0 for complement-path nodes' direct count
    ull Tn[HEAD_PER_MAX];
    bool cm[HEAD_PER_MAX];
    // each node's staged work items and degree, formed once (64-bit divisions)
    ull Ik[HEAD_PER_MAX];
    int Dg[HEAD_PER_MAX];
    // proposal rows: a direct-path node whose pairs have at least two sets to order
    // gets deg*(deg-1) score rows (pair j, candidate position x); the complement path
    // (dropped sets of at most KC_MAX members, reverse-lexicographic) keeps the plain order
    auto prows = [&](int dg, ull T) -> ull {
        return (g.row_off && l >= 1 && l <= tp.learned_lmax && T >= 2) ? (ull)dg * (ull)(dg - 1) : 0ull;
    };
    const bool small = tp.lane_stages && tp.precision != 0 && l <= LANE_LMAX;
    // staged kernel work items of a node: consecutive ranges of NODE_ITEM_CHUNKS
    // chunks of its rank-major chunk space (chunk r of every pair before r+1)
    auto items = [&](int dg, ull T) -> ull {
        if (!small || !T || !node_staged(tp, l, dg)) return 0ull;
        const ull ch = node_chunk(tp, T, dg);
        const ull nc = sat_mul((T + ch - 1) / ch, (ull)dg);
        return nc == KEY_NONE ? KEY_NONE : (nc + NODE_ITEM_CHUNKS - 1) / NODE_ITEM_CHUNKS;
    };
    // warp-per-pair kernel: the pairs of the larger direct nodes of stages 1-2
    auto warp_mode = [&](int dg, ull T) -> bool { return small && T && pair_warped(tp, l, dg); };
    // direct, complement, proposal rows, staged nodes (their first items), the
    // staged nodes' further items, warp-per-pair ordered pairs
    ull v[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull}, mxT = 0;
    bool sat = false;
    for (int u = s0; u < s1; ++u) {
        const int dg = g.deg[u], d = dg - 1;
        const ull T = (dg > 0 && d >= l && dof_ok(tp, u, l)) ? g.binom[(long long)d * g.ldb + l] : 0ull;
        const ull tot = sat_mul(T, (ull)dg);
        sat |= tot == KEY_NONE;
        const bool comp = T && comp_eligible(d, l, tp) && g.prec_m[u] > 0;
        Tn[u - s0] = T;
        cm[u - s0] = comp;
        Dg[u - s0] = dg;
        const ull k = comp ? 0ull : items(dg, T);
        Ik[u - s0] = k;
        if (comp) v[1] = sat_add(v[1], tot);
        else {
            v[0] = sat_add(v[0], tot);
            if (!k && !warp_mode(dg, T)) mxT = T > mxT ? T : mxT;   // the lane kernel's pairs only
            v[2] = sat_add(v[2], prows(dg, T));           // complement-path pairs keep the plain order
            v[3] += k ? 1ull : 0ull;
            v[4] = sat_add(v[4], k ? k - 1 : 0ull);
            v[5] += warp_mode(dg, T) ? (ull)dg : 0ull;
        }
    }
    const int ssat = __syncthreads_or(sat);
    ull ex[6], tot[6];
    block_scan_sat<6>(v, ex, tot, sh);
    // else: plain order this stage (too many rows, or too few tests for the order to matter)
    // score rows are one per candidate; the order pays off only when a pair has
    // many more sets than candidates (l >= 2 and large neighbourhoods)
    const double tests_all = (double)tot[0] + (double)tot[1];
    const bool rows_fit = tot[2] <= (ull)g.rows_cap && tests_all >= tp.learned_min &&
                          tests_all >= tp.learned_ratio * (double)tot[2];
    const ull rows_total = tot[2];
    if (t == 0 && g.scored) g.scored[l] = rows_fit && rows_total > 0;
    {
        ull rd = ex[0], rc = ex[1], rr = ex[2], ra = ex[3], ri = ex[4], rw = ex[5];
        for (int u = s0; u < s1; ++u) {
            const int dg = Dg[u - s0];
            const ull T = Tn[u - s0], tt = sat_mul(T, (ull)dg);
            g.tn_off[u] = rd;
            g.cn_off[u] = rc;
            g.ia_off[u] = ra;
            g.it_off[u] = ri;
            g.wo_off[u] = rw;
            if (g.row_off) g.row_off[u] = rows_fit ? rr : 0ull;
            if (cm[u - s0]) rc = sat_add(rc, tt);
            else {
                rd = sat_add(rd, tt);
                rr = sat_add(rr, prows(dg, T));
                const ull k = Ik[u - s0];
                ra += k ? 1ull : 0ull;
                ri = sat_add(ri, k ? k - 1 : 0ull);
                rw += (!cm[u - s0] && warp_mode(dg, T)) ? (ull)dg : 0ull;
            }
        }
    }
    // owner node of every ordered pair (the small-stage kernel's work items; the commit):
    // a warp takes 32 consecutive nodes, each lane loading one node's offset and degree
    // (one round of loads instead of one per node), then writes the nodes' runs in turn
    // with consecutive entries per lane group (coalesced stores)
    for (int u0 = (t >> 5) * 32; u0 < p; u0 += (int)blockDim.x) {
        const int ul = u0 + (t & 31);
        const long long bl = ul < p ? g.ooff[ul] : 0;
        const int dl = ul < p ? g.deg[ul] : 0;
        const int nk = min(32, p - u0);
        for (int k = 0; k < nk; ++k) {
            const long long b = __shfl_sync(0xffffffffu, bl, k);
            const int dg = __shfl_sync(0xffffffffu, dl, k);
            for (int jj = t & 31; jj < dg; jj += 32) g.opu[b + jj] = u0 + k;
        }
    }
    int rounds = 0;
    if (small && tot[0] > 0) {
        // rank-major rounds of the lane kernel: at most tp.lane_rounds chunks of
        // every direct pair, the rest in the pair-major remainder space rn_off
        for (int off = 16; off > 0; off >>= 1) {
            const ull y = __shfl_xor_sync(0xffffffffu, mxT, off);
            mxT = y > mxT ? y : mxT;
        }
        if ((t & 31) == 0) sh[t >> 5] = mxT;
        __syncthreads();
        ull maxT = 0;
        for (int i = 0; i < 32; ++i) maxT = sh[i] > maxT && i < ((int)blockDim.x >> 5) ? sh[i] : maxT;
        __syncthreads();
        const ull chunk = (ull)tp.lane_chunk;
        rounds = (int)(maxT == 0 ? 0 : min((ull)tp.lane_rounds, (maxT + chunk - 1) / chunk));
        const ull skip = (ull)rounds * chunk;
        ull v2[1] = {0ull};
        for (int u = s0; u < s1; ++u) {
            const ull T = Tn[u - s0];
            const int dg = Dg[u - s0];
            if (!cm[u - s0] && T > skip && !Ik[u - s0] && !warp_mode(dg, T))
                v2[0] = sat_add(v2[0], sat_mul(T - skip, (ull)dg));
        }
        ull ex2[1], tot2[1];
        block_scan_sat<1>(v2, ex2, tot2, sh);
        ull rr2 = ex2[0];
        for (int u = s0; u < s1; ++u) {
            const ull T = Tn[u - s0];
            const int dg = Dg[u - s0];
            g.rn_off[u] = rr2;
            if (!cm[u - s0] && T > skip && !Ik[u - s0] && !warp_mode(dg, T))
                rr2 = sat_add(rr2, sat_mul(T - skip, (ull)dg));
        }
        if (t == 0) g.rn_off[p] = tot2[0];
    }
    __syncthreads();
    if (t == 0) {
        I->lane_rounds = rounds;
        I->lane_overflow = 0;
        I->node_next = 0;
        I->pair_next = 0;
        g.wo_off[p] = tot[5];
        const ull td = tot[0], tc = tot[1];
        g.tn_off[p] = td;
        g.cn_off[p] = tc;
        g.ia_off[p] = tot[3];
        g.it_off[p] = tot[4];
        if (tot[4] == KEY_NONE) {                       // staged items saturated: treat as over budget
            I->error = 6;
            I->halt = 1;
        }
        if (g.row_off) g.row_off[p] = rows_fit ? rows_total : 0ull;
        I->total_direct = td;
        I->total_comp = tc;
        I->saturated = ssat || td == KEY_NONE || tc == KEY_NONE;
        if (I->saturated || (double)td + (double)tc > budget) {
            I->error = 6;                                // PC_ERR_BUDGET
            I->halt = 1;
        } else if (td > 0 && l + 2 > mmax_direct) {
            I->need_host = 1;
            I->halt = 1;
        }
        if (conds.use) {
            const bool run = !I->halt;
            set_stage_conds(conds, I, run && small && td > 0 ? lane_range_of_dev(l) : LANE_RANGES,
                            run && td > 0 && !small, run && tc > 0,
                            run && g.row_off && rows_fit && rows_total > 0,
                            (tp.lazy && tp.c64_list && tp.pair_seen ? 5 : 3) + (tp.node_dmax > 0 ? 1 : 0) +
                                (tp.pair_warp && l <= PAIRWARP_LMAX ? 1 : 0));
        }
    }
}

__global__ void __launch_bounds__(1024) head_kernel(GraphDev g, TestParams tp, double budget,
                                                    int mmax_direct, StageConds conds)
{
    head_body(g, tp, budget, mmax_direct, conds);
}

// test index t of the stage -> (u, j, rank): node by the per-node offsets,
// then j = (t - off[u]) / C(d,l) and rank = (t - off[u]) mod C(d,l)
__device__ __forceinline__ void locate_test(const GraphDev &g, const ull *noff, int l, ull t, int &u,
                                            int &j, int &d, ull &rank)
{
    const int p = g.p;
    u = (int)(upper_bound_dev(noff, (long long)p + 1, t) - 1);
    d = g.deg[u] - 1;
    const ull T = g.binom[(long long)d * g.ldb + l];
    const ull w = t - noff[u];
    const ull jj = w / T;
    j = (int)jj;
    rank = w - jj * T;
}

size_t scan_ws_bytes(long long n) { return 64 + 0 * n; }

// ---------------------------------------------------------------- warp test
// Cholesky of the leading l x l block of the (l+2) x (l+2) lower triangle M
// (row stride ms; order S..., u, v).  Lanes own rows.  After l steps the
// trailing 2x2 holds H = H0 - H1 H2^{-1} H1^T (Sec. 4).  pmin is the smallest
// of the l pivots (conditional variances of S_k given S_1..S_{k-1}), h11, h22.
// bad: a pivot, h11 or h22 <= DEGEN (the FP64 degeneracy rule) or not finite.
template <typename T>
__device__ __forceinline__ void warp_chol_test(T *M, int m, int ms, int l, T &r, T &pmin, bool &bad)
{
    const int lane = threadIdx.x & 31;
    pmin = (T)1e30;
    bad = false;
    for (int k = 0; k < l; ++k) {
        const T piv = M[k * ms + k];
        pmin = piv < pmin ? piv : pmin;
        if (!(piv > (T)DEGEN)) {
            bad = true;
            break;
        }
        const T rl = (T)1 / sqrt(piv);
        for (int i = k + 1 + lane; i < m; i += 32) M[i * ms + k] *= rl;
        __syncwarp();
        for (int i = k + 1 + lane; i < m; i += 32) {
            const T lik = M[i * ms + k];
            for (int c = k + 1; c <= i; ++c) M[i * ms + c] -= lik * M[c * ms + k];
        }
        __syncwarp();
    }
    if (bad) {
        r = (T)0;
        return;
    }
    const T h11 = M[l * ms + l], h22 = M[(l + 1) * ms + l + 1], h12 = M[(l + 1) * ms + l];
    pmin = h11 < pmin ? h11 : pmin;
    pmin = h22 < pmin ? h22 : pmin;
    if (!(h11 > (T)DEGEN) || !(h22 > (T)DEGEN)) {
        bad = true;
        r = (T)0;
        return;
    }
    r = h12 / sqrt(h11 * h22);
}

struct WarpAcc {
    ull tests, red, band, guard, degen, fl32, fl64;
    float maxdz;
};

// per-thread counters of the small-stage kernel (32-bit: a thread runs far fewer
// than 2^32 tests of one stage); its FP32 flops are tests x F(L), formed at the end
struct LaneAcc {
    unsigned tests, band, guard;
};

__device__ __forceinline__ ull flops_direct(int l)
{
    ull L = (ull)l;
    return (L * L * L) / 3 + 2 * L * L + 6 * L + 10;
}

// Fills the FP64 correlations the lower triangle of corr[nd, nd] needs (lazy
// mode): every missing entry is computed once by a whole warp -- lane t sums
// samples t, t+32, ... in order, a fixed butterfly adds the lanes -- and
// published with a fence before its flag, so racing warps write equal values.
__device__ __noinline__ void ensure_c64(const int *nd, int m, const TestParams &tp, double *C64, int ldc)
{
    const int lane = threadIdx.x & 31;
    const int ne = m * (m + 1) / 2;
    volatile unsigned char *valid = tp.c64_valid;
    for (int e0 = 0; e0 < ne; e0 += 32) {
        const int e = e0 + lane;
        bool miss = false;
        int a = 0, b = 0;
        if (e < ne) {
            int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
            while (i * (i + 1) / 2 > e) --i;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            const int c = e - i * (i + 1) / 2;
            a = nd[i];
            b = nd[c];
            miss = a != b && valid[cidx(tp.prow, tp.p, a, b)] != 1;
        }
        unsigned bal = __ballot_sync(0xffffffffu, miss);
        while (bal) {
            const int src = __ffs(bal) - 1;
            const int aa = __shfl_sync(0xffffffffu, a, src), bb = __shfl_sync(0xffffffffu, b, src);
            const double *xa = tp.xs64 + (long long)aa * tp.ldk, *xb = tp.xs64 + (long long)bb * tp.ldk;
            const long long na = n_of(tp, aa);
            // rows start 512-byte aligned (ldk is a multiple of 64): 16-byte loads,
            // four independent FMA chains per lane
            const double2 *xa2 = (const double2 *)xa, *xb2 = (const double2 *)xb;
            const long long nh = na >> 1;
            double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
            long long t = lane;
            for (; t + 32 < nh; t += 64) {
                const double2 a0 = __ldg(xa2 + t), b0 = __ldg(xb2 + t);
                const double2 a1 = __ldg(xa2 + t + 32), b1 = __ldg(xb2 + t + 32);
                acc0 = fma(a0.x, b0.x, acc0);
                acc1 = fma(a0.y, b0.y, acc1);
                acc2 = fma(a1.x, b1.x, acc2);
                acc3 = fma(a1.y, b1.y, acc3);
            }
            if (t < nh) {
                const double2 a0 = __ldg(xa2 + t), b0 = __ldg(xb2 + t);
                acc0 = fma(a0.x, b0.x, acc0);
                acc1 = fma(a0.y, b0.y, acc1);
            }
            if ((na & 1) && lane == 0) acc0 = fma(xa[na - 1], xb[na - 1], acc0);
            double acc = (acc0 + acc1) + (acc2 + acc3);
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                const double v = acc / (double)na;
                C64[cidx(tp.prow, ldc, aa, bb)] = v;
                C64[cidx(tp.prow, ldc, bb, aa)] = v;
                __threadfence();
                valid[cidx(tp.prow, tp.p, aa, bb)] = 1;
                valid[cidx(tp.prow, tp.p, bb, aa)] = 1;
            }
            bal &= bal - 1;
        }
        __syncwarp();
    }
    __threadfence_block();
    __syncwarp();
}

// ---------------------------------------------------------------- FP32 trust rule
// The FP32 trailing block (h11, h12, h22) of a test is the exact Schur
// complement of corr + E, where E holds the correlation step's entry errors
// (|E_ij| <= eps_c) and the backward error of the FP32 factorisation (every
// row of the Cholesky factor of a correlation matrix has unit norm, so each
// entry of that backward error is below a few m eps32; 4 m eps32 is taken).
// With b_u = corr_SS^{-1} corr_Su and b_v the regression coefficients of u
// and v on S, to first order in eps = eps_c + 4 m eps32
//   |dh12| <= eps A_u A_v,  |dh11| <= eps A_u^2,  |dh22| <= eps A_v^2,
//   A_u = 1 + |b_u|_1,  A_v = 1 + |b_v|_1,
// hence |dr| <= eps (A_u A_v / sqrt(h11 h22) + |r|/2 (A_u^2/h11 + A_v^2/h22)).
// The expansion is used only while eps A_u^2/h11, eps A_v^2/h22 and
// m eps |corr_SS^{-1}| (kap) stay below 0.05, and the bound is doubled to
// cover the higher-order terms and the rounding of the final ratio.  A test
// is trusted when |r| clears the threshold r_q = tanh(q / sqrt(n-l-3)) by
// more than that bound (then the FP64 decision of Eq. 1 is the same) and the
// statistic lies at least `band` from q; otherwise it is re-decided in FP64.
// Returns 0 trusted, 1 band (re-decide), 2 guard (re-decide); dr_out: the bound.
constexpr float EPS32 = 5.96e-8f;

__device__ __forceinline__ int fp32_trust(const TestParams &tp, int m, float sqf, float rq, float a, float h11,
                                          float h22, float ih, float Au, float Av, float kap, float &dr_out)
{
    const float eps = tp.eps_c + (4.0f * (float)m) * EPS32;
    const float i11 = __frcp_rn(h11), i22 = __frcp_rn(h22);
    const float qu = eps * Au * Au * i11, qv = eps * Av * Av * i22;
    dr_out = INFINITY;
    if (fmaxf(fmaxf(qu, qv), kap) > 0.05f) return 2;
    const float dr = 2.0f * eps * (Au * Av * ih + 0.5f * a * (Au * Au * i11 + Av * Av * i22)) + 8.0f * EPS32;
    dr_out = dr;
    if (dr > tp.dr_max) return 2;
    // |z - q| >= sqf |a - rq| / (1 - min(a, rq)^2) (mean-value theorem on atanh)
    const float gap = fabsf(a - rq), mn = fminf(a, rq);
    if (gap <= dr || sqf * gap < (float)tp.band * (1.0f - mn * mn)) return 1;
    return 0;
}

// l1 norms of the regression coefficients b_u = corr_SS^{-1} corr_Su and b_v
// from the factor warp_chol_test left in M (column k below the diagonal holds
// L_ik, the diagonal the pivots L_kk^2, rows l and l+1 hold L^{-1} corr_Su and
// L^{-1} corr_Sv): back substitution L^T b = y by the warp, column by column.
// Overwrites the first l entries of rows l and l+1.
__device__ __forceinline__ void warp_beta_l1(float *M, int ms, int l, float &bu, float &bv)
{
    const int lane = threadIdx.x & 31;
    float *yu = M + (long long)l * ms, *yv = M + (long long)(l + 1) * ms;
    float su = 0.f, sv = 0.f;
    for (int k = l - 1; k >= 0; --k) {
        __syncwarp();
        const float rl = rsqrtf(M[k * ms + k]);
        const float b_u = yu[k] * rl, b_v = yv[k] * rl;
        su += fabsf(b_u);
        sv += fabsf(b_v);
        for (int j = lane; j < k; j += 32) {
            const float lkj = M[k * ms + j];
            yu[j] -= lkj * b_u;
            yv[j] -= lkj * b_v;
        }
    }
    __syncwarp();
    bu = su;
    bv = sv;
}

// One CI test for node ids nd[0..m) (S..., u, v) by the calling warp.
// Returns independent; writes r and z (of the path that decided).
template <bool F64>
__device__ __forceinline__ bool warp_test(const int *nd, int m, int l, const float *C32,
                                          const double *C64, int ldc, const TestParams &tp,
                                          double sq, float sqf, void *Mbuf, int ms, WarpAcc &acc,
                                          double &r_out, float &z_out)
{
    const int lane = threadIdx.x & 31;
    bool need64 = F64, indep = false;
    float zf = 0.f, rf = 0.f;
    bool f32ok = false;
    if (!F64) {
        float *M = (float *)Mbuf;
        for (int i = 0; i < m; ++i)
            for (int c = lane; c <= i; c += 32) M[i * ms + c] = C32[cidx(tp.prow, ldc, nd[i], nd[c])];
        __syncwarp();
        float pmin;
        bool bad;
        warp_chol_test<float>(M, m, ms, l, rf, pmin, bad);
        __syncwarp();
        acc.fl32 += flops_direct(l);
        if (bad || pmin < (float)tp.guard) {
            need64 = true;
            ++acc.guard;
        } else {
            const float h11 = M[l * ms + l], h22 = M[(l + 1) * ms + l + 1];
            float bu, bv, dr;
            warp_beta_l1(M, ms, l, bu, bv);
            const float ih = rsqrtf(h11 * h22);
            const float a = fabsf(rf);
            const float rq = tanhf(tp.qf / sqf);
            // kap is not formed here (it would need corr_SS^{-1}); the pivot guard
            // and the two first-order ratios bound the expansion instead
            const int t = fp32_trust(tp, m, sqf, rq, a, h11, h22, ih, 1.0f + bu, 1.0f + bv, 0.0f, dr);
            zf = a < 1.0f ? sqf * atanhf(a) : INFINITY;
            if (t == 2) {
                need64 = true;
                ++acc.guard;
            } else if (t == 1) {
                need64 = true;
                ++acc.band;
            } else {
                indep = a <= rq;
                f32ok = true;
            }
        }
    }
    double r = rf;
    float z = zf;
    if (need64) {
        double *M = (double *)Mbuf;
        if (tp.lazy) ensure_c64(nd, m, tp, (double *)C64, ldc);
        for (int i = 0; i < m; ++i)
            for (int c = lane; c <= i; c += 32) {
                const long long o = cidx(tp.prow, ldc, nd[i], nd[c]);
                M[i * ms + c] = tp.lazy ? ((volatile const double *)C64)[o] : C64[o];
            }
        __syncwarp();
        double pmin;
        bool bad;
        warp_chol_test<double>(M, m, ms, l, r, pmin, bad);
        __syncwarp();
        acc.fl64 += flops_direct(l);
        if (bad) {
            indep = true;
            r = 0.0;
            z = 0.f;
            ++acc.degen;
        } else {
            double z64 = fabs(r) < 1.0 ? sq * fabs(atanh(r)) : INFINITY;
            indep = z64 <= tp.q;
            if (!F64 && isfinite(zf) && zf > 0.f) acc.maxdz = fmaxf(acc.maxdz, (float)fabs(zf - z64));
            z = (float)z64;
        }
        if (!F64) ++acc.red;
    }
    (void)f32ok;
    r_out = r;
    z_out = z;
    return indep;
}

__device__ __forceinline__ void flush_acc(const WarpAcc &acc, DevCounters *ctr)
{
    if (acc.tests) atomicAdd(&ctr->tests_executed, acc.tests);
    if (acc.red) atomicAdd(&ctr->redecided, acc.red);
    if (acc.band) atomicAdd(&ctr->band_hits, acc.band);
    if (acc.guard) atomicAdd(&ctr->guard_hits, acc.guard);
    if (acc.degen) atomicAdd(&ctr->degenerate, acc.degen);
    if (acc.fl32) atomicAdd(&ctr->flops, acc.fl32);
    if (acc.fl64) atomicAdd(&ctr->flops64_direct, acc.fl64);
    if (acc.maxdz > 0.f) atomic_max_float_pos(&ctr->max_dz_bits, acc.maxdz);
}

// Candidate position x of the ordered pair (u, j) (d candidates) -> node id:
// position x of adj(u)\{v} in ascending order (v sits at index j of nbr[u]), or
// the x-th candidate of the proposal order when the stage has one (perm holds
// the candidates' indices into nbr[u] in that order).
__device__ __forceinline__ int cand_node(const GraphDev &g, bool prop, int u, int j, int d, int x)
{
    if (prop) {
        const ull b = g.row_off[u];
        if (g.row_off[u + 1] > b) return g.nbr[nidx(g, u) + g.perm[b + (ull)j * d + x]];
    }
    return g.nbr[nidx(g, u) + x + (x >= j)];
}

// Did the head order stage l's candidates by the proposal?  Read once per kernel:
// the plain-order stages of a learned search then touch no proposal table.
__device__ __forceinline__ bool stage_prop(const GraphDev &g, int l)
{
    return g.row_off && g.scored && l >= 0 && g.scored[l];
}

__device__ __forceinline__ void sort_small(int *a, int n)
{
    for (int i = 1; i < n; ++i) {
        const int x = a[i];
        int k = i - 1;
        while (k >= 0 && a[k] > x) {
            a[k + 1] = a[k];
            --k;
        }
        a[k + 1] = x;
    }
}

// ---------------------------------------------------------------- direct path (skeleton)
template <bool F64>
__global__ void __launch_bounds__(256) ci_direct_kernel(GraphDev g, TestParams tp, int mmax,
                                                        const float *C32, const double *C64,
                                                        int ldc, int ms, int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (stopped(g.info)) return;
    const int l = g.info->l;
    const bool prop = stage_prop(g, l);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = l + 2;
    if (m > mmax) return;
    if (!F64 && tp.lane_stages && l <= LANE_LMAX && !g.info->lane_overflow) return;  // small stages: ci_lane_kernel
    unsigned char *mine = smem_raw + (size_t)wib * per_warp_bytes;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)mmax * ms * sizeof(double));
    int *pos = nd + mmax;
    const ull total = g.info->total_direct;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const double sq = sqrt((double)(tp.n - l - 3));
    const float sqf = (float)sq;
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    for (ull t = gw; t < total; t += nw) {
        int u, j, d;
        ull rank;
        locate_test(g, g.tn_off, l, t, u, j, d, rank);
        const int v = g.nbr[nidx(g, u) + j];
        const int side = u > v;
        const int a = min(u, v), b = max(u, v);
        const ull key = ((ull)side << 62) | rank;
        ull *bp = g.best + pidx(g, a, b);
        if (*(volatile ull *)bp < key) continue;   // an earlier set already separates
        if (lane == 0) {
            unrank_lex(rank, d, l, g.binom, g.ldb, pos);
            for (int i = 0; i < l; ++i) nd[i] = cand_node(g, prop, u, j, d, pos[i]);
            if (prop) sort_small(nd, l);        // the set is tested in ascending-id order
            nd[l] = u;
            nd[l + 1] = v;
        }
        __syncwarp();
        double r;
        float z;
        ++acc.tests;
        const double squ = tp.nvec ? sqrt((double)(n_of(tp, u) - l - 3)) : sq;
        bool ind = warp_test<F64>(nd, m, l, C32, C64, ldc, tp, squ, tp.nvec ? (float)squ : sqf, Mbuf, ms, acc,
                                  r, z);
        if (ind && lane == 0) atomicMin(bp, key);
        __syncwarp();
    }
    if (lane == 0) flush_acc(acc, g.ctr);
}


// bytes of one warp's buffer in the stage loop's direct tests: the FP64 matrix of
// LOOP_MMAX x (LOOP_MMAX + 1) and the member and position lists
__host__ __device__ constexpr size_t loop_direct_bytes()
{
    return ((size_t)LOOP_MMAX * (LOOP_MMAX + 1) * sizeof(double) + 2 * LOOP_MMAX * sizeof(int) + 15) / 16 * 16;
}

// The stage loop's direct tests of a small stage (l + 2 <= LOOP_MMAX): one warp per
// test as ci_direct_kernel, located by the CTA's own plan (doff: per-node offsets in
// shared memory, doff[p] = their total); mine: the warp's buffer of loop_direct_bytes.
template <bool F64>
__device__ __noinline__ void loop_direct_body(const GraphDev &g, const TestParams &tp, int l, const ull *doff,
                                              const float *C32, const double *C64, int ldc, unsigned char *mine)
{
    const int lane = threadIdx.x & 31;
    const int m = l + 2, ms = LOOP_MMAX + 1;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)LOOP_MMAX * ms * sizeof(double));
    int *pos = nd + LOOP_MMAX;
    const ull total = doff[g.p];
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const double sq = sqrt((double)(tp.n - l - 3));
    const float sqf = (float)sq;
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    for (ull t = gw; t < total; t += nw) {
        int u, j, d;
        ull rank;
        locate_test(g, doff, l, t, u, j, d, rank);
        const int v = g.nbr[nidx(g, u) + j];
        const int side = u > v;
        const ull key = ((ull)side << 62) | rank;
        ull *bp = g.best + pidx(g, min(u, v), max(u, v));
        if (*(volatile ull *)bp < key) continue;   // an earlier set already separates
        if (lane == 0) {
            unrank_lex(rank, d, l, g.binom, g.ldb, pos);
            for (int i = 0; i < l; ++i) nd[i] = g.nbr[nidx(g, u) + pos[i] + (pos[i] >= j)];
            nd[l] = u;
            nd[l + 1] = v;
        }
        __syncwarp();
        double r;
        float z;
        ++acc.tests;
        const bool ind = warp_test<F64>(nd, m, l, C32, C64, ldc, tp, sq, sqf, Mbuf, ms, acc, r, z);
        if (ind && lane == 0) atomicMin(bp, key);
        __syncwarp();
    }
    if (lane == 0) flush_acc(acc, g.ctr);
}

// ---------------------------------------------------------------- direct path, small stages
// One thread per chunk of tp.lane_chunk consecutive sets of one ordered pair
// (l <= LANE_LMAX): one unranking, then lexicographic successors; the
// (l+2)x(l+2) lower triangle (order S..., u, v) lives in registers and is
// factored with compile-time indices.  A chunk stops at the first set its pair
// already beats.  Tests the FP32 trust rule cannot trust go to a queue that a
// warp-per-test FP64 pass drains before the commit; when the queue is full the
// direct kernel re-runs the stage.

// Decision of one FP32 test of the small-stage kernel from the trailing 2x2
// (h11, h12, h22) and the smallest pivot: true = independent (the caller
// records the key and stops); a test the FP32 trust rule cannot trust goes
// to the FP64 queue.
// x: pivot of the border member given the prefix (1 without a prefix), bsu/bsv:
// |its regression coefficients| c_u/x, c_v/x; gs bounds the l1 norm of the
// regression coefficients of the border member on the prefix, so that
// A_u = A0u + bsu (1 + gs), A0u = 1 + |b_u(P)|_1, bounds 1 + |b_u(S)|_1 (and
// likewise for v).  With F = |Lp^{-1}|_F^2 >= |corr_PP^{-1}|_2, (F + 1)/x
// bounds |corr_SS^{-1}|_2; kapP = m eps (F + 1).
template <int L>
__device__ __forceinline__ bool lane_decide(const TestParams &tp, float sqf, float rq, float h11, float h12,
                                            float h22, float pmin, bool bad, float x, float bsu, float bsv,
                                            float gs, float kapP, float A0u, float A0v, ull flat, ull *queue,
                                            ull qcap, ull *qlen, LaneAcc &acc)
{
    constexpr int M = L + 2;
    pmin = fminf(pmin, fminf(h11, h22));
    bad |= !(h11 > 1e-12f) || !(h22 > 1e-12f);
    ++acc.tests;
    bool queue_it = false, ind = false;
    if (bad || pmin < (float)tp.guard) {
        queue_it = true;
        ++acc.guard;
    } else {
        const float ih = rsqrtf(h11 * h22);
        const float a = fabsf(h12 * ih);
        const float Au = fmaf(bsu, 1.0f + gs, A0u), Av = fmaf(bsv, 1.0f + gs, A0v);
        const float kap = kapP * __frcp_rn(x);
        float dr;
        const int t = fp32_trust(tp, M, sqf, rq, a, h11, h22, ih, Au, Av, kap, dr);
        if (t == 2) {
            queue_it = true;
            ++acc.guard;
        } else if (t == 1) {
            queue_it = true;
            ++acc.band;
        } else {
            ind = a <= rq;                              // |r| >= 1: z infinite, dependent
        }
    }
    if (queue_it) {
        const ull slot = atomicAdd(qlen, 1ull);
        if (slot < qcap) queue[slot] = flat;
    }
    return ind;
}

// Where the small-stage tests read corr.  A member is named by its index into
// the frozen neighbour list nbr[u]; a handle is what row() and get() take.
//   GlobalSrc: rows of the FP32 matrix in L2 (handles are node ids);
//   StagedSrc: the block corr[adj(u), adj(u)] and the row corr[u, adj(u)] that
//              a CTA staged in shared memory (handles are neighbour indices).
// corr is exactly symmetric (the GEMMs mirror one triangle), so corr(s, u) is
// read as corr(u, s) from u's row: the same value either way.
struct GlobalSrc {
    const float *C;
    const long long *prow;
    int ldc;
    const int *nb;
    const float *Cu, *Cv;      // rows of u and v
    int v;
    __device__ __forceinline__ int handle(int idx) const { return nb[idx]; }
    __device__ __forceinline__ const float *row(int h) const { return C + cidx(prow, ldc, h, 0); }
    __device__ __forceinline__ float get(const float *r, int h) const { return __ldg(r + h); }
    __device__ __forceinline__ float cu(int h) const { return __ldg(Cu + h); }
    __device__ __forceinline__ float cv(int h) const { return __ldg(Cv + h); }
    __device__ __forceinline__ float cuv() const { return __ldg(Cu + v); }
};

struct StagedSrc {
    const float *B;            // deg x deg, row stride ld: corr[nbr[u][a], nbr[u][b]]
    const float *cus;          // deg: corr[u, nbr[u][a]]
    int ld;
    int j;                     // v = nbr[u][j]
    __device__ __forceinline__ int handle(int idx) const { return idx; }
    __device__ __forceinline__ const float *row(int h) const { return B + h * ld; }
    __device__ __forceinline__ float get(const float *r, int h) const { return r[h]; }
    __device__ __forceinline__ float cu(int h) const { return cus[h]; }
    __device__ __forceinline__ float cv(int h) const { return B[j * ld + h]; }
    __device__ __forceinline__ float cuv() const { return cus[j]; }
};

// lexicographic successor of pos (L of d); returns the first position that changed
template <int L>
__device__ __forceinline__ int lex_next(int *pos, int d)
{
    int i = L - 1;
    while (i >= 0 && pos[i] == d - L + i) --i;
    if (i >= 0) {
        ++pos[i];
        for (int k2 = i + 1; k2 < L; ++k2) pos[k2] = pos[k2 - 1] + 1;
    }
    return i;
}

// lexicographic successor of pos (l of d positions, l known at run time)
__device__ __forceinline__ void lex_next_dyn(int *pos, int l, int d)
{
    int i = l - 1;
    while (i >= 0 && pos[i] == d - l + i) --i;
    if (i >= 0) {
        ++pos[i];
        for (int k2 = i + 1; k2 < l; ++k2) pos[k2] = pos[k2 - 1] + 1;
    }
}

// Lexicographic order over the candidate list (ascending ids, or the proposal's
// permutation of it): consecutive sets share their first L-1 members (all but
// one step in d-L+1).  The Cholesky factor of that prefix P, the rows of u and
// v eliminated by it (lu, lv) and the Schur block of (u, v) given P are kept in
// registers; each test borders them with the last member s: one row of corr
// (L+1 loads; corr_ss = 1), a forward substitution against P, then
//   x = 1 - |l_s|^2,  c_u = corr_us - lu.l_s,  c_v = corr_vs - lv.l_s,
//   H = H_P - [c_u c_v]^T [c_u c_v] / x
// -- the same Cholesky of the S block (Sec. 4) in bordered form, O(L^2) work.
// sqf = sqrt(n - L - 3) and rq = tanh(q / sqf), the stage's |r| threshold, come
// from the caller; pos0: the positions of the set at `rank` when the caller has
// unranked it (nullptr: unranked here).  CHECK: re-read the pair's key every
// fourth test (the callers that run one test per call check it themselves).
// Returns true when a test of the range separated (its key is recorded).
template <int L, bool PROP, class Src, bool CHECK = true, class PosT = short>
__device__ __forceinline__ bool lane_tests_lex(const GraphDev &g, const TestParams &tp, const Src &src, int u,
                                               int v, int j, int d, ull T, ull rank, ull rank_end, ull *queue,
                                               ull qcap, ull *qlen, LaneAcc &acc, float sqf, float rq,
                                               const PosT *pos0 = nullptr)
{
    constexpr int K = L > 0 ? L - 1 : 0;                 // prefix length
    constexpr int KA = K > 0 ? K : 1;
    // proposal order: position x of the enumeration is neighbour index perm[x]
    const short *pr = nullptr;
    if (PROP && stage_prop(g, L) && g.row_off[u + 1] > g.row_off[u]) pr = g.perm + g.row_off[u] + (ull)j * d;
    auto member = [&](int x) -> int { return src.handle((PROP && pr) ? (int)pr[x] : x + (x >= j)); };
    const int side = u > v;
    ull *bp = g.best + pidx(g, min(u, v), max(u, v));
    const ull tbase = g.tn_off[u] + (ull)j * T;
    const float cuv = src.cuv();
    int pos[L > 0 ? L : 1];
    if (pos0) {
#pragma unroll
        for (int i = 0; i < L; ++i) pos[i] = pos0[i];
    } else {
        unrank_lex(rank, d, L, g.binom, g.ldb, pos);
    }
    int sp[KA];
    float Lp[KA * (KA + 1) / 2], rd[KA], lu[KA], lv[KA];
    float huu = 1.f, hvv = 1.f, huv = cuv, ppmin = 1e30f;
    // prefix terms of the trust rule: 1 + |b_u(P)|_1, 1 + |b_v(P)|_1, sqrt(K |Lp^{-1}|_F^2)
    // and m eps (|Lp^{-1}|_F^2 + 1)
    const float kap_c = (float)(L + 2) * (tp.eps_c + (4.0f * (float)(L + 2)) * EPS32);
    float A0u = 1.f, A0v = 1.f, sKF = 0.f, kapP = kap_c;
    bool pbad = false, fresh = true;
    int since = 0;
    for (; rank < rank_end; ++rank) {
        const ull key = ((ull)side << 62) | rank;
        // an earlier set of this pair already separates: checked every fourth test
        // (the read goes to L2; at most three tests are wasted)
        if (CHECK && since == 0 && *(volatile ull *)bp < key) return false;
        since = (since + 1) & 3;
        if (K > 0 && fresh) {
            // factor the prefix and eliminate the rows of u and v by it
            ppmin = 1e30f;
            pbad = false;
#pragma unroll
            for (int i = 0; i < K; ++i) sp[i] = member(pos[i]);
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const float *Ci = src.row(sp[i]);
                float dd = 1.f;
#pragma unroll
                for (int c = 0; c < i; ++c) {
                    float t = src.get(Ci, sp[c]);
#pragma unroll
                    for (int c2 = 0; c2 < c; ++c2) t -= Lp[i * (i + 1) / 2 + c2] * Lp[c * (c + 1) / 2 + c2];
                    t *= rd[c];
                    Lp[i * (i + 1) / 2 + c] = t;
                    dd -= t * t;
                }
                ppmin = fminf(ppmin, dd);
                pbad |= !(dd > 1e-12f);
                const float rl = rsqrtf(fmaxf(dd, 1e-30f));
                Lp[i * (i + 1) / 2 + i] = dd * rl;
                rd[i] = rl;
                float tu = src.cu(sp[i]), tv = src.cv(sp[i]);
#pragma unroll
                for (int c = 0; c < i; ++c) {
                    tu -= lu[c] * Lp[i * (i + 1) / 2 + c];
                    tv -= lv[c] * Lp[i * (i + 1) / 2 + c];
                }
                lu[i] = tu * rl;
                lv[i] = tv * rl;
            }
            huu = 1.f;
            hvv = 1.f;
            huv = cuv;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                huu -= lu[i] * lu[i];
                hvv -= lv[i] * lv[i];
                huv -= lu[i] * lv[i];
            }
            // for the trust rule: F = |Lp^{-1}|_F^2 (columns of Lp^{-1} by forward
            // substitution) and the l1 norms of the prefix regression coefficients
            // b_u(P) = Lp^{-T} lu, b_v(P) = Lp^{-T} lv (back substitution)
            float Fp = 0.f;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                float zc[KA];
                zc[c] = rd[c];
                Fp = fmaf(zc[c], zc[c], Fp);
#pragma unroll
                for (int k2 = c + 1; k2 < K; ++k2) {
                    float t = 0.f;
#pragma unroll
                    for (int j2 = c; j2 < k2; ++j2) t = fmaf(Lp[k2 * (k2 + 1) / 2 + j2], zc[j2], t);
                    zc[k2] = -t * rd[k2];
                    Fp = fmaf(zc[k2], zc[k2], Fp);
                }
            }
            sKF = sqrtf((float)K * Fp);
            float BuP = 0.f, BvP = 0.f;
            {
                float bu_[KA], bv_[KA];
#pragma unroll
                for (int k2 = K - 1; k2 >= 0; --k2) {
                    float tu = lu[k2], tv = lv[k2];
#pragma unroll
                    for (int j2 = k2 + 1; j2 < K; ++j2) {
                        tu -= Lp[j2 * (j2 + 1) / 2 + k2] * bu_[j2];
                        tv -= Lp[j2 * (j2 + 1) / 2 + k2] * bv_[j2];
                    }
                    bu_[k2] = tu * rd[k2];
                    bv_[k2] = tv * rd[k2];
                    BuP += fabsf(bu_[k2]);
                    BvP += fabsf(bv_[k2]);
                }
            }
            A0u = 1.0f + BuP;
            A0v = 1.0f + BvP;
            kapP = kap_c * (Fp + 1.0f);
            fresh = false;
        }
        float h11 = huu, h22 = hvv, h12 = huv, pmin = ppmin;
        float xs = 1.f, bsu = 0.f, bsv = 0.f, gs = 0.f;
        bool bad = pbad;
        if (L > 0) {
            const int s = member(pos[L - 1]);
            const float *Cs = src.row(s);
            float ls[KA];
            float x = 1.f;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                float t = src.get(Cs, sp[i]);
#pragma unroll
                for (int c = 0; c < i; ++c) t -= ls[c] * Lp[i * (i + 1) / 2 + c];
                t *= rd[i];
                ls[i] = t;
                x -= t * t;
            }
            float cu = src.cu(s), cv = src.cv(s);
#pragma unroll
            for (int i = 0; i < K; ++i) {
                cu -= lu[i] * ls[i];
                cv -= lv[i] * ls[i];
            }
            pmin = fminf(pmin, x);
            bad |= !(x > 1e-12f);
            const float rx = __frcp_rn(fmaxf(x, 1e-30f));
            h11 -= cu * cu * rx;
            h22 -= cv * cv * rx;
            h12 -= cu * cv * rx;
            xs = fmaxf(x, 1e-30f);
            bsu = fabsf(cu * rx);
            bsv = fabsf(cv * rx);
            gs = K > 0 ? sKF * sqrtf(fmaxf(1.0f - x, 0.0f)) : 0.f;
        }
        if (lane_decide<L>(tp, sqf, rq, h11, h12, h22, pmin, bad, xs, bsu, bsv, gs, kapP, A0u, A0v, tbase + rank,
                           queue, qcap, qlen, acc)) {
            atomicMin(bp, key);
            return true;
        }
        if (rank + 1 < rank_end && lex_next<L>(pos, d) < L - 1) fresh = true;
    }
    return false;
}

// one chunk of a pair (PROP: the kernel variant of handles with a proposal
// network, whose scored stages enumerate over the permuted candidate list)
template <int L, bool PROP>
__device__ __forceinline__ void lane_chunk(const GraphDev &g, const TestParams &tp, const float *C32, int ldc,
                                           int u, int j, int d, ull T, ull rank, ull rank_end, ull *queue,
                                           ull qcap, ull *qlen, LaneAcc &acc)
{
    const int *nb = g.nbr + nidx(g, u);
    const int v = nb[j];
    const GlobalSrc src{C32, tp.prow, ldc, nb, C32 + cidx(tp.prow, ldc, u, 0), C32 + cidx(tp.prow, ldc, v, 0), v};
    const float sqf = sqrtf((float)(n_of(tp, u) - L - 3));
    lane_tests_lex<L, PROP>(g, tp, src, u, v, j, d, T, rank, rank_end, queue, qcap, qlen, acc, sqf,
                            tanhf(tp.qf / sqf));
}

// Phase A, rank-major: item g = (round r, ordered pair o), r = g / NP -- a wave
// covers rank chunk r of every direct pair, so a pair whose first chunks
// separate skips the rest.  Phase B: the ranks beyond rounds * lane_chunk of
// the pairs that have them, pair-major (per-node offsets rn_off).
template <int L, bool PROP>
__device__ __forceinline__ void lane_dispatch(const GraphDev &g, const TestParams &tp, const float *C32, int ldc,
                                              ull *queue, ull qcap, ull *qlen)
{
    LaneAcc acc = {0u, 0u, 0u};
    const int p = g.p;
    const long long NP = g.info->n_opairs;
    const int rounds = g.info->lane_rounds;
    const ull chunk = (ull)tp.lane_chunk;
    const long long G = (long long)gridDim.x * blockDim.x;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (NP > 0 && rounds > 0) {
        // item (r, o) = (gi / NP, gi % NP) stepped by G without dividing: one
        // division for the start and for the stride
        long long r = tid / NP, o = tid - r * NP;
        const long long Gq = G / NP, Gr = G - Gq * NP;
        for (; r < rounds; r += Gq, o += Gr) {
            if (o >= NP) {
                o -= NP;
                ++r;
                if (r >= rounds) break;
            }
            const int u = g.opu[o];                     // owner of ordered pair o
            if (g.tn_off[u + 1] == g.tn_off[u]) continue;   // not a direct node this stage
            if (g.ia_off[u + 1] != g.ia_off[u]) continue;   // its pairs run on the staged kernel
            if (g.wo_off[u + 1] != g.wo_off[u]) continue;   // ... or on the warp-per-pair kernel
            const int d = g.deg[u] - 1;
            const ull T = g.binom[(long long)d * g.ldb + L];
            const ull r0 = (ull)r * chunk;
            if (r0 >= T) continue;
            const ull r1 = r0 + chunk < T ? r0 + chunk : T;
            lane_chunk<L, PROP>(g, tp, C32, ldc, u, (int)(o - g.ooff[u]), d, T, r0, r1, queue, qcap, qlen, acc);
        }
    }
    const ull nb = g.rn_off[p];
    const ull skip = (ull)rounds * chunk;
    const ull nbc = (nb + chunk - 1) / chunk;
    for (ull c = (ull)tid; c < nbc; c += (ull)G) {
        // chunk c of the remainder space; it may cross pairs
        ull t = c * chunk;
        const ull tend = t + chunk < nb ? t + chunk : nb;
        while (t < tend) {
            const int u = (int)(upper_bound_dev(g.rn_off, (long long)p + 1, t) - 1);
            const int d = g.deg[u] - 1;
            const ull T = g.binom[(long long)d * g.ldb + L];
            const ull per = T - skip;                     // remainder ranks per pair of u
            const ull w = t - g.rn_off[u];
            const int j = (w >> 32) == 0 && (per >> 32) == 0 ? (int)((unsigned)w / (unsigned)per) : (int)(w / per);
            const ull rr = w - (ull)j * per;
            const ull take = per - rr < tend - t ? per - rr : tend - t;
            lane_chunk<L, PROP>(g, tp, C32, ldc, u, j, d, T, skip + rr, skip + rr + take, queue, qcap, qlen, acc);
            t += take;
        }
    }
    ull tests = acc.tests, band = acc.band, guard = acc.guard;
    for (int off = 16; off > 0; off >>= 1) {
        tests += __shfl_xor_sync(0xffffffffu, tests, off);
        band += __shfl_xor_sync(0xffffffffu, band, off);
        guard += __shfl_xor_sync(0xffffffffu, guard, off);
    }
    if ((threadIdx.x & 31) == 0) {
        WarpAcc w = {tests, 0, band, guard, 0, tests * flops_direct(L), 0, 0.f};
        flush_acc(w, g.ctr);
    }
}

template <int L, int HI, bool PROP>
__device__ __forceinline__ void lane_switch(int l, const GraphDev &g, const TestParams &tp, const float *C32, int ldc,
                                            ull *queue, ull qcap, ull *qlen)
{
    if constexpr (L <= HI) {
        if (l == L) lane_dispatch<L, PROP>(g, tp, C32, ldc, queue, qcap, qlen);
        else lane_switch<L + 1, HI, PROP>(l, g, tp, C32, ldc, queue, qcap, qlen);
    }
}

// Stages LO <= l <= HI (one instantiation per range keeps the register count of
// small l low: the launch sequence runs every range, all but one return at once).
template <int LO, int HI, bool PROP>
__global__ void __launch_bounds__(256, HI <= 2 ? 4 : (HI <= 4 ? 3 : (HI <= 8 ? 2 : 1)))
    ci_lane_kernel(GraphDev g, TestParams tp, const float *C32, int ldc,
                                                      ull *queue, ull qcap, ull *qlen)
{
    if (stopped(g.info)) return;
    const int l = g.info->l;
    const ull total = g.info->total_direct;
    if (tp.precision == 0 || l < LO || l > HI || total == 0) return;
    lane_switch<LO, HI, PROP>(l, g, tp, C32, ldc, queue, qcap, qlen);
}

// ---------------------------------------------------------------- staged small stages
// Every ordered pair (u, v) of a node u has the same candidate count d and the
// same C(d, l) sets, and every set it tests lies in adj(u): the block
// corr[adj(u), adj(u)] and the row corr[u, adj(u)] hold every entry the
// node's tests read.  The node's chunks are ordered rank-major (chunk r of
// every pair before chunk r+1) and cut into work items of NODE_ITEM_CHUNKS
// chunks; a CTA takes items from the per-stage counter, stages the node's block
// in shared memory (once for consecutive items of one node), and its threads
// run the item's chunks by the bordered tests of lane_tests_lex reading the
// staged block.  The arithmetic, the keys and the FP64 queue are those of the
// lane kernel, so the results are the same.
template <int L, bool PROP>
__device__ __forceinline__ void node_dispatch(const GraphDev &g, const TestParams &tp, const float *C32, int ldc,
                                              ull *queue, ull qcap, ull *qlen)
{
    extern __shared__ __align__(16) float node_smem[];
    __shared__ ull item_s;
    constexpr int LP = L > 0 ? L : 1;
    float *cus = node_smem;                              // NODE_DMAX floats
    short *pos_s = (short *)(node_smem + NODE_DMAX);     // NODE_ROUNDS_MAX x L start positions
    float *B = node_smem + NODE_DMAX + (NODE_ROUNDS_MAX * LP + 1) / 2;   // deg x deg
    LaneAcc acc = {0u, 0u, 0u};
    const int p = g.p;
    const ull na = g.ia_off[p], nitems = na + g.it_off[p];
    int staged = -1;                                     // node whose block is in shared memory
    for (;;) {
        __syncthreads();                                 // the last item's tests are done with the block
        if (threadIdx.x == 0) item_s = atomicAdd(&g.info->node_next, 1ull);
        __syncthreads();
        const ull it = item_s;
        if (it >= nitems) break;
        // the first item of every staged node comes first, then the further
        // items node by node: early chunks of all pairs run before late ones
        int u;
        ull loc;
        if (it < na) {
            u = (int)(upper_bound_dev(g.ia_off, (long long)p + 1, it) - 1);
            loc = 0;
        } else {
            u = (int)(upper_bound_dev(g.it_off, (long long)p + 1, it - na) - 1);
            loc = 1 + (it - na - g.it_off[u]);
        }
        const int dg = g.deg[u], d = dg - 1;
        const ull T = g.binom[(long long)d * g.ldb + L];
        const ull chunk = node_chunk(tp, T, dg);
        const ull nc = (T + chunk - 1) / chunk * (ull)dg;
        const ull c0 = loc * NODE_ITEM_CHUNKS;
        const ull c1 = c0 + NODE_ITEM_CHUNKS < nc ? c0 + NODE_ITEM_CHUNKS : nc;
        const int *nb = g.nbr + nidx(g, u);
        if (u != staged) {
            for (int e = threadIdx.x; e < dg * dg; e += blockDim.x) {
                const int a = e / dg, b = e - a * dg;
                B[e] = C32[cidx(tp.prow, ldc, nb[a], nb[b])];
            }
            for (int e = threadIdx.x; e < dg; e += blockDim.x) cus[e] = C32[cidx(tp.prow, ldc, u, nb[e])];
            staged = u;
        }
        // the item's chunks span the rank rounds r0 .. r1 (a round: chunk r of every
        // pair); every pair of the node has the same d, so each round's first set is
        // unranked once for the CTA
        const ull rb = c0 / (unsigned)dg, re = (c1 - 1) / (unsigned)dg;
        for (int q = threadIdx.x; q <= (int)(re - rb); q += blockDim.x) {
            int pq[LP];
            unrank_lex((rb + q) * chunk, d, L, g.binom, g.ldb, pq);
#pragma unroll
            for (int i = 0; i < L; ++i) pos_s[q * LP + i] = (short)pq[i];
        }
        __syncthreads();
        const float sqf = sqrtf((float)(n_of(tp, u) - L - 3)), rq = tanhf(tp.qf / sqf);
        for (ull c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const ull r = c / (unsigned)dg;
            const int j = (int)(c - r * (unsigned)dg);
            const ull r0 = r * chunk, r1 = r0 + chunk < T ? r0 + chunk : T;
            const StagedSrc src{B, cus, dg, j};
            lane_tests_lex<L, PROP>(g, tp, src, u, nb[j], j, d, T, r0, r1, queue, qcap, qlen, acc, sqf, rq,
                                    pos_s + (r - rb) * LP);
        }
    }
    ull tests = acc.tests, band = acc.band, guard = acc.guard;
    for (int off = 16; off > 0; off >>= 1) {
        tests += __shfl_xor_sync(0xffffffffu, tests, off);
        band += __shfl_xor_sync(0xffffffffu, band, off);
        guard += __shfl_xor_sync(0xffffffffu, guard, off);
    }
    if ((threadIdx.x & 31) == 0) {
        WarpAcc w = {tests, 0, band, guard, 0, tests * flops_direct(L), 0, 0.f};
        flush_acc(w, g.ctr);
    }
}

template <int L, int HI, bool PROP>
__device__ __forceinline__ void node_switch(int l, const GraphDev &g, const TestParams &tp, const float *C32, int ldc,
                                            ull *queue, ull qcap, ull *qlen)
{
    if constexpr (L <= HI) {
        if (l == L) node_dispatch<L, PROP>(g, tp, C32, ldc, queue, qcap, qlen);
        else node_switch<L + 1, HI, PROP>(l, g, tp, C32, ldc, queue, qcap, qlen);
    }
}

// Stages max(LO, 1) <= l <= HI, the nodes of the staged layout (it_off); the
// other nodes of those stages run on ci_lane_kernel.
template <int LO, int HI, bool PROP>
__global__ void __launch_bounds__(NODE_THREADS, HI <= 2 ? 3 : (HI <= 4 ? 3 : (HI <= 8 ? 2 : 1)))
    ci_node_kernel(GraphDev g, TestParams tp, const float *C32, int ldc, ull *queue, ull qcap, ull *qlen)
{
    if (stopped(g.info)) return;
    const int l = g.info->l;
    if (tp.precision == 0 || l < LO || l > HI || l < 1 || g.ia_off[g.p] == 0) return;
    node_switch<(LO > 1 ? LO : 1), HI, PROP>(l, g, tp, C32, ldc, queue, qcap, qlen);
}

// ---------------------------------------------------------------- one warp per pair (stages 1-2)
// At stages 1 and 2 the nodes too large for the staged layout have hundreds of
// neighbours.  A warp takes one of their ordered pairs (u, v) from the stage
// counter and walks its sets in lexicographic order, 32 at a time: lane i tests
// the set of rank base + i (the bordered test of lane_tests_lex, one set), so
// the rows corr[u, .], corr[v, .] and the prefix member's row are the same for
// the whole warp and the index arithmetic is shared.  The pair stops at the
// first block in which a test separates (keys by atomicMin: the lowest rank
// wins), or when the pair's key shows an earlier separation.
// Advance the lexicographic position (q0 < q1 < d) by k sets; positions past the
// last set stop at q0 = d - 1.
__device__ __forceinline__ void lex2_advance(int &q0, int &q1, int k, int d)
{
    q1 += k;
    while (q1 >= d && q0 < d - 1) {
        ++q0;
        q1 = q1 - d + q0 + 1;
    }
}

template <int L, bool PROP>
__device__ __forceinline__ void pairwarp_dispatch(const GraphDev &g, const TestParams &tp, const float *C32, int ldc,
                                                  ull *queue, ull qcap, ull *qlen)
{
    static_assert(L == 1 || L == 2, "the warp-per-pair kernel runs stages 1 and 2");
    const int lane = threadIdx.x & 31;
    LaneAcc acc = {0u, 0u, 0u};
    const int p = g.p;
    const ull npairs = g.wo_off[p];
    for (;;) {
        ull o = 0;
        if (lane == 0) o = atomicAdd(&g.info->pair_next, 1ull);
        o = __shfl_sync(0xffffffffu, o, 0);
        if (o >= npairs) break;
        const int u = (int)(upper_bound_dev(g.wo_off, (long long)p + 1, o) - 1);
        const int j = (int)(o - g.wo_off[u]);
        const int d = g.deg[u] - 1;
        const ull T = g.binom[(long long)d * g.ldb + L];
        const int *nb = g.nbr + nidx(g, u);
        const int v = nb[j];
        const GlobalSrc src{C32, tp.prow, ldc, nb, C32 + cidx(tp.prow, ldc, u, 0), C32 + cidx(tp.prow, ldc, v, 0),
                            v};
        const float sqf = sqrtf((float)(n_of(tp, u) - L - 3)), rq = tanhf(tp.qf / sqf);
        const ull *bp = g.best + pidx(g, min(u, v), max(u, v));
        const ull side = (ull)(u > v) << 62;
        int b0 = 0, b1 = 1;                               // positions of the block's first set (L = 2)
        for (ull base = 0; base < T; base += 32) {
            if (*(volatile const ull *)bp < (side | base)) break;   // an earlier set separates
            const ull rank = base + (ull)lane;
            int pos[L];
            if (L == 1) {
                pos[0] = (int)rank;
            } else {
                int q0 = b0, q1 = b1;
                lex2_advance(q0, q1, lane, d);
                pos[0] = q0;
                pos[L - 1] = q1;
            }
            bool found = false;
            if (rank < T)
                found = lane_tests_lex<L, PROP, GlobalSrc, false, int>(g, tp, src, u, v, j, d, T, rank, rank + 1,
                                                                       queue, qcap, qlen, acc, sqf, rq, pos);
            if (__any_sync(0xffffffffu, found)) break;
            if (L == 2) lex2_advance(b0, b1, 32, d);
        }
    }
    ull tests = acc.tests, band = acc.band, guard = acc.guard;
    for (int off = 16; off > 0; off >>= 1) {
        tests += __shfl_xor_sync(0xffffffffu, tests, off);
        band += __shfl_xor_sync(0xffffffffu, band, off);
        guard += __shfl_xor_sync(0xffffffffu, guard, off);
    }
    if (lane == 0) {
        WarpAcc w = {tests, 0, band, guard, 0, tests * flops_direct(L), 0, 0.f};
        flush_acc(w, g.ctr);
    }
}

template <bool PROP>
__global__ void __launch_bounds__(256, 4) ci_pairwarp_kernel(GraphDev g, TestParams tp, const float *C32, int ldc,
                                                             ull *queue, ull qcap, ull *qlen)
{
    if (stopped(g.info)) return;
    const int l = g.info->l;
    if (tp.precision == 0 || l < 1 || l > PAIRWARP_LMAX || g.wo_off[g.p] == 0) return;
    if (l == 1) pairwarp_dispatch<1, PROP>(g, tp, C32, ldc, queue, qcap, qlen);
    else pairwarp_dispatch<2, PROP>(g, tp, C32, ldc, queue, qcap, qlen);
}

// FP64 pass over the queued tests of the lane kernel (one warp per test).
__global__ void __launch_bounds__(256) ci_redecide_kernel(GraphDev g, TestParams tp, const double *C64, int ldc,
                                                          const ull *queue, const ull *qlen, ull qcap, int ms,
                                                          int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (stopped(g.info)) return;
    const int l = g.info->l;
    if (tp.precision == 0 || l > LANE_LMAX) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = l + 2;
    unsigned char *mine = smem_raw + (size_t)wib * per_warp_bytes;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)(LANE_LMAX + 2) * ms * sizeof(double));
    int *pos = nd + LANE_LMAX + 2;
    const ull nq = *qlen < qcap ? *qlen : qcap;
    // A full queue dropped tests: the direct kernel that follows then re-runs the
    // whole stage (FP32 first, FP64 inline), so no test goes undecided.  Keys
    // already set here are keys of independent tests, hence still valid minima.
    if (*qlen > qcap && blockIdx.x == 0 && threadIdx.x == 0) {
        g.info->lane_overflow = 1;
        atomicAdd(&g.ctr->queue_overflows, 1);
    }
    const bool prop = stage_prop(g, l);
    const double sq = sqrt((double)(tp.n - l - 3));
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    for (ull qi = (blockIdx.x * (ull)blockDim.x + threadIdx.x) >> 5; qi < nq;
         qi += ((ull)gridDim.x * blockDim.x) >> 5) {
        const ull t = queue[qi];
        int u, j, d;
        ull rank;
        locate_test(g, g.tn_off, l, t, u, j, d, rank);
        const int v = g.nbr[nidx(g, u) + j];
        const int side = u > v;
        const ull key = ((ull)side << 62) | rank;
        ull *bp = g.best + pidx(g, min(u, v), max(u, v));
        if (*(volatile ull *)bp < key) continue;
        if (lane == 0) {
            unrank_lex(rank, d, l, g.binom, g.ldb, pos);
            for (int i = 0; i < l; ++i) nd[i] = cand_node(g, prop, u, j, d, pos[i]);
            if (prop) sort_small(nd, l);
            nd[l] = u;
            nd[l + 1] = v;
        }
        __syncwarp();
        double r;
        float z;
        const double squ = tp.nvec ? sqrt((double)(n_of(tp, u) - l - 3)) : sq;
        const bool ind = warp_test<true>(nd, m, l, nullptr, C64, ldc, tp, squ, (float)squ, Mbuf, ms, acc, r, z);
        ++acc.red;
        if (ind && lane == 0) atomicMin(bp, key);
        __syncwarp();
    }
    acc.fl32 = 0;
    if (lane == 0) {
        if (acc.red) atomicAdd(&g.ctr->redecided, acc.red);
        if (acc.degen) atomicAdd(&g.ctr->degenerate, acc.degen);
        if (acc.fl64) atomicAdd(&g.ctr->flops64_direct, acc.fl64);
    }
}

// ---------------------------------------------------------------- FP64 entries of the queued tests
// The FP64 pass of a small stage needs, per queued test, the FP64 correlations of
// its l + 2 nodes.  Formed one by one by the warp that runs the test, each missing
// entry is a length-n dot product of FP64 standardised columns streamed from HBM,
// and a test's entries follow one another.  Instead, every missing entry is first
// claimed once (byte 0 -> 2 of its validity flag, by a CAS on the containing word)
// and listed; a whole CTA per listed entry then forms it; the FP64 pass finds them
// all present.
__device__ __forceinline__ bool claim_byte(unsigned char *flags, long long e)
{
    unsigned int *w = reinterpret_cast<unsigned int *>(reinterpret_cast<uintptr_t>(flags + e) & ~(uintptr_t)3);
    const int sh = (int)(reinterpret_cast<uintptr_t>(flags + e) & 3) * 8;
    unsigned int old = *(volatile unsigned int *)w;
    for (int it = 0; it < 64; ++it) {                    // bounded: a contended entry is formed on demand
        if ((old >> sh) & 0xffu) return false;          // valid, or claimed by another test
        const unsigned int prev = atomicCAS(w, old, old | (2u << sh));
        if (prev == old) return true;
        old = prev;
    }
    return false;
}

__device__ __forceinline__ void release_byte(unsigned char *flags, long long e)
{
    unsigned int *w = reinterpret_cast<unsigned int *>(reinterpret_cast<uintptr_t>(flags + e) & ~(uintptr_t)3);
    const int sh = (int)(reinterpret_cast<uintptr_t>(flags + e) & 3) * 8;
    atomicAnd(w, ~(0xffu << sh));
}

// One warp per queued test: its node set (as the FP64 pass builds it), then each
// missing pair (a < b) of it is claimed and listed -- for the first queued test of
// each tested pair only: a later one runs only if that test does not separate the
// pair, and then forms its entries on demand (dense problems queue many tests per
// pair, most of which an earlier set decides).
__global__ void __launch_bounds__(256) c64_collect_kernel(GraphDev g, TestParams tp, const ull *queue,
                                                          const ull *qlen, ull qcap)
{
    __shared__ int nds[8][LANE_LMAX + 2], poss[8][LANE_LMAX + 2];
    if (stopped(g.info)) return;
    const int l = g.info->l;
    if (tp.precision == 0 || l > LANE_LMAX || !tp.lazy || !tp.c64_list || !tp.pair_seen) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *nd = nds[wib], *pos = poss[wib];
    const ull nq = *qlen < qcap ? *qlen : qcap;
    const bool prop = stage_prop(g, l);
    const int m = l + 2;
    for (ull qi = (blockIdx.x * (ull)blockDim.x + threadIdx.x) >> 5; qi < nq;
         qi += ((ull)gridDim.x * blockDim.x) >> 5) {
        const ull t = queue[qi];
        int u, j, d;
        ull rank;
        locate_test(g, g.tn_off, l, t, u, j, d, rank);
        const int v = g.nbr[nidx(g, u) + j];
        const ull key = ((ull)(u > v) << 62) | rank;
        const long long ep = pidx(g, min(u, v), max(u, v));
        if (*(volatile ull *)(g.best + ep) < key) continue;   // no FP64 test follows
        int first = 0;
        if (lane == 0) first = claim_byte(tp.pair_seen, ep);
        if (!__shfl_sync(0xffffffffu, first, 0)) continue;    // not the pair's first queued test
        if (lane == 0) {
            unrank_lex(rank, d, l, g.binom, g.ldb, pos);
            for (int i = 0; i < l; ++i) nd[i] = cand_node(g, prop, u, j, d, pos[i]);
            nd[l] = u;
            nd[l + 1] = v;
        }
        __syncwarp();
        for (int i = 1; i < m; ++i)
            for (int c = lane; c < i; c += 32) {
                const int a = min(nd[i], nd[c]), b = max(nd[i], nd[c]);
                if (a == b) continue;
                const long long e = cidx(tp.prow, tp.p, a, b);
                if (tp.c64_valid[e] || !claim_byte(tp.c64_valid, e)) continue;
                const ull k = atomicAdd(tp.c64_list_len, 1ull);
                if (k < tp.c64_list_cap) tp.c64_list[k] = make_int2(a, b);
                else release_byte(tp.c64_valid, e);      // the list is full: formed on demand later
            }
        __syncwarp();
    }
}

// One CTA per listed pair: the dot product of the FP64 standardised columns over
// all 256 threads (a fixed summation order), then the entry, its mirror and both flags.
__global__ void __launch_bounds__(256) c64_fill_kernel(GraphDev g, TestParams tp, double *C64, int ldc)
{
    __shared__ double red[8];
    if (stopped(g.info) || !tp.lazy || !tp.c64_list || !tp.pair_seen) return;
    const ull nl = *tp.c64_list_len < tp.c64_list_cap ? *tp.c64_list_len : tp.c64_list_cap;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (ull k = blockIdx.x; k < nl; k += gridDim.x) {
        const int2 ab = tp.c64_list[k];
        const double *xa = tp.xs64 + (long long)ab.x * tp.ldk, *xb = tp.xs64 + (long long)ab.y * tp.ldk;
        const long long na = n_of(tp, ab.x), nh = na >> 1;
        const double2 *xa2 = reinterpret_cast<const double2 *>(xa), *xb2 = reinterpret_cast<const double2 *>(xb);
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 4
        for (long long t = threadIdx.x; t < nh; t += blockDim.x) {
            const double2 a2 = __ldg(xa2 + t), b2 = __ldg(xb2 + t);
            acc0 = fma(a2.x, b2.x, acc0);
            acc1 = fma(a2.y, b2.y, acc1);
        }
        if ((na & 1) && threadIdx.x == 0) acc0 = fma(xa[na - 1], xb[na - 1], acc0);
        double acc = acc0 + acc1;
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) red[w] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += red[i];
            const double val = sum / (double)na;
            C64[cidx(tp.prow, ldc, ab.x, ab.y)] = val;
            C64[cidx(tp.prow, ldc, ab.y, ab.x)] = val;
            __threadfence();
            tp.c64_valid[cidx(tp.prow, tp.p, ab.x, ab.y)] = 1;
            tp.c64_valid[cidx(tp.prow, tp.p, ab.y, ab.x)] = 1;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- small binomial table
// C(x, r) for x < SB_ROWS, r <= KC_MAX copied to shared memory, so that the
// unranking of a dropped set (at most KC_MAX positions of at most SB_ROWS - 1
// candidates) reads no global table: its binary searches are chains of
// dependent loads.
constexpr int SB_ROWS = PREC_MAX;
constexpr int SB_COLS = KC_MAX + 1;
__device__ __forceinline__ void load_small_binom(const GraphDev &g, ull *sb)
{
    for (int e = threadIdx.x; e < SB_ROWS * SB_COLS; e += blockDim.x) {
        const int x = e / SB_COLS, r = e - x * SB_COLS;
        sb[e] = x < g.ldb && r < g.ldb ? g.binom[(long long)x * g.ldb + r] : 0ull;
    }
}

// ---------------------------------------------------------------- complement path
// With P = corr[F,F]^{-1}, F = adj(u) u {u}, and the dropped set R
// (S = adj(u)\{v}\R, |R| = k = d - l), the {u,v} block of corr[T,T]^{-1},
// T = S u {u,v}, is Q = P_TT - P_TR P_RR^{-1} P_RT restricted to {u,v}
// (inverse of a principal submatrix); r = -Q_uv / sqrt(Q_uu Q_vv), and the
// Schur complement H of Sec. 4 is Q^{-1}: h11 = Q_vv/det, h22 = Q_uu/det.
// FP32 evaluation of one complement test with the proof that its decision is the
// FP64 one.  The test reads P_RR, P_Ru, P_Rv and the {u,v} block of P (FP64,
// rounded to FP32 on load).  Computed by Cholesky, the result is the exact
// Q = P_TT - P_TR P_RR^{-1} P_RT ({u,v} block) of P + dP with, to first order,
// |dP_ij| <= eps s_i s_j, s_i = sqrt(P_ii), eps = (4k + 8) eps32: the rounding
// of P, the backward errors of the factorisation, the two solves and the final
// dot products (rows of the factor and the solves have norms s_i, s_u, s_v).
// With X_a = P_RR^{-1} P_Ra (a in {u, v}) the change of Q is
//   dQ_ab = dP_ab - dP_aR X_b - X_a^T dP_Rb + X_a^T dP_RR X_b,
// so |dQ_ab| <= eps W_a W_b with W_a = s_a + sum_r s_r |X_ra|, and for
// r = -Q_uv / sqrt(Q_uu Q_vv)
//   |dr| <= eps (W_u W_v / sqrt(Q_uu Q_vv) + |r|/2 (W_u^2/Q_uu + W_v^2/Q_vv)).
// The expansion is used while eps W_a^2 / Q_aa and kap = k eps tr(D P_RR^{-1} D)
// (D = diag s_r; tr bounds the norm of the scaled inverse, hence the size of
// the higher-order terms relative to the first) stay below 0.05; the bound is
// doubled for those terms and 8 eps32 added for the final ratio and the FP32
// threshold.  Trusted: the |r| threshold r_q is cleared by more than that, the
// statistic lies at least `band` from q (as for the direct tests), and the
// test is far from the FP64 degeneracy rule (h11 = 1/(Q_uu (1 - r^2)) and h22
// at least 1000 times the floor).  Returns 0 trusted (indep set), 1 band,
// 2 guard; the FP64 evaluation decides the others.
__device__ __forceinline__ int comp_test_fp32(const double *P, const int (&sr)[KC_MAX], int su, int sv, int k,
                                              const TestParams &tp, float sqf, float rq, bool &indep)
{
    float L[KC_MAX][KC_MAX], yu[KC_MAX], yv[KC_MAX], sd[KC_MAX], ri[KC_MAX];
#pragma unroll
    for (int i = 0; i < KC_MAX; ++i) {
        yu[i] = yv[i] = sd[i] = ri[i] = 0.f;
#pragma unroll
        for (int c = 0; c < KC_MAX; ++c) L[i][c] = 0.f;
        if (i < k) {
            const double *Pi = P + (long long)sr[i] * PREC_MAX;
#pragma unroll
            for (int c = 0; c <= i; ++c) L[i][c] = (float)Pi[sr[c]];
            yu[i] = (float)Pi[su];
            yv[i] = (float)Pi[sv];
        }
    }
    const float Puu = (float)P[su * PREC_MAX + su], Pvv = (float)P[sv * PREC_MAX + sv];
    float Quv = (float)P[su * PREC_MAX + sv];
#pragma unroll
    for (int i = 0; i < KC_MAX; ++i) sd[i] = i < k ? sqrtf(fmaxf(L[i][i], 0.f)) : 0.f;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < KC_MAX; ++i) {
        if (i >= k || bad) continue;
#pragma unroll
        for (int c = 0; c < i; ++c) {
            float t = L[i][c];
#pragma unroll
            for (int q = 0; q < c; ++q) t = fmaf(-L[i][q], L[c][q], t);
            L[i][c] = t * ri[c];
        }
        float t = L[i][i];
#pragma unroll
        for (int q = 0; q < i; ++q) t = fmaf(-L[i][q], L[i][q], t);
        if (!(t > 0.f)) {
            bad = true;
            continue;
        }
        ri[i] = rsqrtf(t);
        float a = yu[i], b = yv[i];
#pragma unroll
        for (int q = 0; q < i; ++q) {
            a = fmaf(-L[i][q], yu[q], a);
            b = fmaf(-L[i][q], yv[q], b);
        }
        yu[i] = a * ri[i];
        yv[i] = b * ri[i];
    }
    if (bad) return 2;
    float Quu = Puu, Qvv = Pvv;
#pragma unroll
    for (int i = 0; i < KC_MAX; ++i) {
        Quu = fmaf(-yu[i], yu[i], Quu);
        Qvv = fmaf(-yv[i], yv[i], Qvv);
        Quv = fmaf(-yu[i], yv[i], Quv);
    }
    if (!(Quu > 0.f) || !(Qvv > 0.f)) return 2;
    // X_a = L^{-T} y_a in place (back substitution); W_a
    float Wu = sqrtf(Puu), Wv = sqrtf(Pvv);
#pragma unroll
    for (int i = KC_MAX - 1; i >= 0; --i) {
        if (i >= k) continue;
        float a = yu[i], b = yv[i];
#pragma unroll
        for (int q = i + 1; q < KC_MAX; ++q)
            if (q < k) {
                a = fmaf(-L[q][i], yu[q], a);
                b = fmaf(-L[q][i], yv[q], b);
            }
        yu[i] = a * ri[i];
        yv[i] = b * ri[i];
        Wu = fmaf(sd[i], fabsf(yu[i]), Wu);
        Wv = fmaf(sd[i], fabsf(yv[i]), Wv);
    }
    // tr(D P_RR^{-1} D) = sum_j s_j^2 |column j of L^{-1}|^2 (forward substitution per column)
    float tr = 0.f;
#pragma unroll
    for (int j = 0; j < KC_MAX; ++j) {
        if (j >= k) continue;
        float m[KC_MAX];
        float nj = 0.f;
#pragma unroll
        for (int i = 0; i < KC_MAX; ++i) {
            m[i] = 0.f;
            if (i < j || i >= k) continue;
            float t = i == j ? 1.f : 0.f;
#pragma unroll
            for (int q = 0; q < i; ++q)
                if (q >= j) t = fmaf(-L[i][q], m[q], t);
            m[i] = t * ri[i];
            nj = fmaf(m[i], m[i], nj);
        }
        tr = fmaf(sd[j] * sd[j], nj, tr);
    }
    const float eps = (4.0f * (float)k + 8.0f) * EPS32;
    const float kap = (float)k * eps * tr;
    const float iu = __frcp_rn(Quu), iv = __frcp_rn(Qvv);
    const float qu = eps * Wu * Wu * iu, qv = eps * Wv * Wv * iv;
    if (!(fmaxf(fmaxf(qu, qv), kap) <= 0.05f)) return 2;
    const float ih = rsqrtf(Quu * Qvv);
    const float a = fabsf(Quv * ih);
    const float dr = 2.0f * eps * (Wu * Wv * ih + 0.5f * a * (Wu * Wu * iu + Wv * Wv * iv)) + 8.0f * EPS32;
    if (!(dr <= tp.dr_max)) return 2;
    const float om = 1.0f - a * a;
    if (!(om > 8.0f * dr) || Quu * om > 1e9f || Qvv * om > 1e9f) return 2;
    const float gap = fabsf(a - rq), mn = fminf(a, rq);
    if (gap <= dr || sqf * gap < (float)tp.band * (1.0f - mn * mn)) return 1;
    indep = a <= rq;
    return 0;
}

constexpr int COMP_OFF_MAX = 2048;    // per-node offsets staged in shared memory up to this p
// The complement tests of CTA `cta` of `ncta`.  sb: the unranking table (loaded by
// the caller); soff: shared room for soff_cap per-node test offsets, used when they
// fit (the searches in both are chains of dependent loads).
// planned: soff already holds this CTA's own copy of the stage's offsets (soff[p] =
// the total) and the stage is unscored (the stage loop's stages have no direct tests).
// sdeg, sT: with planned, the degree and C(d, l) of every node (shared), so that a
// test is located without global loads.
__device__ __noinline__ void complement_body(const GraphDev &g, const TestParams &tp, const ull *sb, ull *soff,
                                                int soff_cap, int cta, int ncta, bool planned = false,
                                                const int *sdeg = nullptr, const ull *sT = nullptr)
{
    if (!planned && stopped(g.info)) return;
    const int l = g.info->l;
    const bool prop = !planned && stage_prop(g, l);
    const ull total = planned ? soff[g.p] : g.info->total_comp;
    if ((ull)cta >= total) return;                       // no test reaches this CTA
    const bool off_sm = planned || g.p < soff_cap;
    if (!planned) {
        if (off_sm)
            for (int i = threadIdx.x; i <= g.p; i += blockDim.x) soff[i] = g.cn_off[i];
        __syncthreads();
    }
    const ull *noff = off_sm ? soff : g.cn_off;
    // |r| threshold of the stage: z <= q  <=>  |r| <= tanh(q / sqrt(n - l - 3)) (from the
    // host's table); tests within a relative 1e-12 of it are decided by z itself, exactly
    // as the z form would
    const double rq = tp.rq_tab[l];
    // FP32 first (one problem; a batched handle's nodes differ in n): rq rounded to FP32
    const bool f32 = tp.comp_fp32 && !tp.nvec;
    const float sqf = sqrtf((float)(tp.n - l - 3)), rqf = (float)rq;
    ull nt = 0, ndg = 0, nfl = 0, nband = 0, nguard = 0;
    const ull nthr = (ull)ncta * blockDim.x;
    // tests are dealt CTA-first, so that a stage with a few thousand tests still
    // spreads its FP64 work (the bound of a test) over every SM
    for (ull t = (ull)threadIdx.x * ncta + cta; t < total; t += nthr) {
        int u, j, d;
        ull rank, T;
        if (sdeg) {
            u = (int)(upper_bound_dev(noff, (long long)g.p + 1, t) - 1);
            d = sdeg[u] - 1;
            T = sT[u];
            const ull w = t - noff[u], jj = w / T;
            j = (int)jj;
            rank = w - jj * T;
        } else {
            locate_test(g, noff, l, t, u, j, d, rank);
            T = g.binom[(long long)d * g.ldb + l];
        }
        const int v = g.nbr[nidx(g, u) + j];
        const int k = d - l;
        const int side = u > v;
        const int a = min(u, v), b = max(u, v);
        const ull key = ((ull)side << 62) | rank;
        ull *bp = g.best + pidx(g, a, b);
        const ull best0 = *(volatile ull *)bp;            // checked below, once the candidates are known
        int posR[KC_MAX];
        unrank_lex_fixed<KC_MAX>(T - 1 - rank, d, k, sb, SB_COLS, posR);   // complement of lex is reverse lex
        const double *P = g.prec + (long long)u * PREC_MAX * PREC_MAX;
        const short *ps = g.prec_pos + pidx(g, u, 0);
        const int su = ps[u], sv = ps[v];
        int sr[KC_MAX];
#pragma unroll
        for (int i = 0; i < KC_MAX; ++i) sr[i] = i < k ? ps[cand_node(g, prop, u, j, d, posR[i])] : 0x7fffffff;
        if (prop) sort_fixed<KC_MAX>(sr);                   // ascending slots (ids); unused entries last
        if (best0 < key) continue;                          // an earlier set of this pair separates
        nfl += (ull)(k * k * k) / 3 + 2ull * k * k + 6ull * k + 20;
        if (f32) {
            bool ind32 = false;
            const int tr32 = comp_test_fp32(P, sr, su, sv, k, tp, sqf, rqf, ind32);
            if (tr32 == 0) {
                ++nt;
                if (ind32) atomicMin(bp, key);
                continue;
            }
            if (tr32 == 1) ++nband;
            else ++nguard;
        }
        // every entry of P the test reads (P_RR lower triangle, P_Ru, P_Rv and the {u,v}
        // block) is loaded before the factorisation starts: one round of independent
        // loads instead of one per row
        double L[KC_MAX][KC_MAX], pu[KC_MAX], pv[KC_MAX];
#pragma unroll
        for (int i = 0; i < KC_MAX; ++i) {
            pu[i] = pv[i] = 0.0;
            if (i < k) {
                const double *Pi = P + (long long)sr[i] * PREC_MAX;
#pragma unroll
                for (int c = 0; c <= i; ++c) L[i][c] = Pi[sr[c]];
                pu[i] = Pi[su];
                pv[i] = Pi[sv];
            }
        }
        double Quu = P[su * PREC_MAX + su], Qvv = P[sv * PREC_MAX + sv], Quv = P[su * PREC_MAX + sv];
        // Cholesky of P_RR in place and the solves for P_Ru, P_Rv; every loop runs to
        // KC_MAX with guards so that L, the reciprocal pivots and y stay in registers
        double ri[KC_MAX], yu[KC_MAX], yv[KC_MAX];
        bool bad = false;
#pragma unroll
        for (int i = 0; i < KC_MAX; ++i) {
            yu[i] = yv[i] = 0.0;
            if (i >= k || bad) continue;
#pragma unroll
            for (int c = 0; c < i; ++c) {
                double s = L[i][c];
#pragma unroll
                for (int q = 0; q < c; ++q) s = fma(-L[i][q], L[c][q], s);
                L[i][c] = s * ri[c];
            }
            double s = L[i][i];
#pragma unroll
            for (int q = 0; q < i; ++q) s = fma(-L[i][q], L[i][q], s);
            if (!(s > 0.0)) {
                bad = true;
                continue;
            }
            ri[i] = rsqrt(s);
            double su_ = pu[i], sv_ = pv[i];
#pragma unroll
            for (int q = 0; q < i; ++q) {
                su_ = fma(-L[i][q], yu[q], su_);
                sv_ = fma(-L[i][q], yv[q], sv_);
            }
            yu[i] = su_ * ri[i];
            yv[i] = sv_ * ri[i];
        }
#pragma unroll
        for (int i = 0; i < KC_MAX; ++i) {
            Quu = fma(-yu[i], yu[i], Quu);
            Qvv = fma(-yv[i], yv[i], Qvv);
            Quv = fma(-yu[i], yv[i], Quv);
        }
        const double det = Quu * Qvv - Quv * Quv;
        const double h11 = Qvv / det, h22 = Quu / det;
        bool ind;
        if (bad || !(h11 > DEGEN) || !(h22 > DEGEN) || !(det > 0.0)) {
            ind = true;
            ++ndg;
        } else {
            const double r = -Quv * rsqrt(Quu * Qvv);
            const double ar = fabs(r);
            if (!tp.nvec && fabs(ar - rq) > 1e-12 * rq) {
                ind = ar < rq;
            } else {
                const double squ = sqrt((double)(n_of(tp, u) - l - 3));
                const double z = ar < 1.0 ? squ * fabs(atanh(r)) : INFINITY;
                ind = z <= tp.q;
            }
        }
        ++nt;
        if (ind) atomicMin(bp, key);
    }
    if (nt) {
        atomicAdd(&g.ctr->tests_executed, nt);
        atomicAdd(&g.ctr->complement_tests, nt);
        atomicAdd(&g.ctr->flops_comp, nfl);
    }
    if (ndg) atomicAdd(&g.ctr->degenerate, ndg);
    if (nband + nguard) atomicAdd(&g.ctr->redecided, nband + nguard);
    if (nband) atomicAdd(&g.ctr->band_hits, nband);
    if (nguard) atomicAdd(&g.ctr->guard_hits, nguard);
}

__global__ void __launch_bounds__(128) ci_complement_kernel(GraphDev g, TestParams tp)
{
    __shared__ ull sb[SB_ROWS * SB_COLS];
    __shared__ ull soff[COMP_OFF_MAX];
    if (stopped(g.info) || (ull)blockIdx.x >= g.info->total_comp) return;
    load_small_binom(g, sb);                             // the body's first barrier covers it
    complement_body(g, tp, sb, soff, COMP_OFF_MAX, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- neighbourhood precision blocks
// One CTA per node.  A maintained block drops the neighbours the last commit
// deleted (P <- P - P[:,w] P[w,:] / P_ww: the inverse of a principal
// submatrix); a requested block is built by a symmetric sweep of corr[F,F],
// F = adj(u) u {u} (ascending ids).
constexpr int PREC_CHUNKS = 8;        // CTAs sharing one node's block downdate
constexpr int PREC_RMAX = 64;         // removals applied in one block downdate (two per lane)
constexpr int PREC_SHARE_MIN = 16;    // from this many removals one CTA of the cluster factors P_RR

// One node per blockIdx.x, its kept rows split over blockIdx.y.  A maintained
// block drops the members the last commit deleted, R, all at once (the inverse
// of a principal submatrix):
//   P_TT <- P_TT - P_TR P_RR^{-1} P_RT      (T = the members kept).
// Every CTA factors P_RR = L D L^T (the same arithmetic in each), then each warp
// takes one of the CTA's kept rows i: y = P_RR^{-1} P_Ri by two triangular
// solves (lanes own entries of y), and P_ij -= y . P_Rj for the kept columns j.
// Only rows of R (never written here) and a warp's own row are read; the chunks
// of a node form one cluster, which meets once after every chunk has read the
// slot map, so that chunk 0 can retire R (slot map entry -1) at once; members
// retired earlier are skipped.  A requested block (chunk 0) is built by a
// symmetric sweep of corr[F,F], F = adj(u) u {u}.
// Node u, chunk `chunk` of `nchunks` (smd: the dynamic shared memory).  CL: the
// chunks of a node are one thread-block cluster (the kernel below), which shares
// a large factor through distributed shared memory and retires R in place; else
// every chunk with rows factors P_RR itself and prec_retire retires R once every
// chunk is done.
template <bool CL>
// need: the node's build request (-1: read it from the tail's flags in memory).
__device__ __forceinline__ void prec_body(const GraphDev &g, const TestParams &tp, const double *C64, int ldc, int u,
                                          int chunk, int nchunks, double *smd, int need = -1)
{
    if (stopped(g.info)) return;
    __shared__ int mem[PREC_MAX];
    __shared__ int bad, nrem;
    const int p = g.p;
    const int m0 = g.prec_m[u];
    // a maintained block loses exactly the neighbours the last degree pass found
    // deleted (its live members are the neighbours of the previous stage): none, no work
    if (m0 > 0 && g.dchg[u] == 0) return;
    if (m0 > 0) {
        int *rem = mem;
        __shared__ int keep[PREC_MAX];
        __shared__ int nkeep;
        double *P = g.prec + (long long)u * PREC_MAX * PREC_MAX;
        const int *pm = g.prec_mem + (long long)u * PREC_MAX;
        const short *pos = g.prec_pos + pidx(g, u, 0);
        const uint32_t *row = g.adj + (long long)u * g.W;
        // the block's slots: deleted by the last commit (R), kept (T: u and the members
        // still adjacent), or retired earlier; both lists in ascending slot order (one
        // slot per thread, m0 <= PREC_MAX < blockDim.x), by ballots and warp offsets
        __shared__ int wcnt[16], wkc[16];
        {
            const int sl = threadIdx.x, wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
            bool gone = false, kept = false;
            if (sl < m0) {
                const int w = pm[sl];
                if (w == u) {
                    kept = true;
                } else if (pos[w] >= 0) {
                    kept = (__ldcg(row + (w >> 5)) >> (w & 31)) & 1u;
                    gone = !kept;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, gone), balk = __ballot_sync(0xffffffffu, kept);
            if (ln == 0) {
                wcnt[wid] = __popc(bal);
                wkc[wid] = __popc(balk);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int acc = 0, acck = 0;
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                    const int c = wcnt[i], ck = wkc[i];
                    wcnt[i] = acc;
                    wkc[i] = acck;
                    acc += c;
                    acck += ck;
                }
                nrem = acc;
                nkeep = acck;
            }
            __syncthreads();
            const unsigned lt = (1u << ln) - 1u;
            if (gone) rem[wcnt[wid] + __popc(bal & lt)] = sl;
            if (kept) keep[wkc[wid] + __popc(balk & lt)] = sl;
        }
        __syncthreads();
        const int nr = nrem, nt = nkeep;
        if (nr == 0) return;
        if (chunk == 0 && threadIdx.x == 0) atomicAdd(&g.ctr->prec_downdates, 1ull);
        if (nr > PREC_RMAX) {
            // too many at once: drop the block; it is rebuilt if the node needs it again
            if (chunk == 0 && threadIdx.x == 0) g.prec_m[u] = -2;
            return;
        }
        if constexpr (CL) {
            // every chunk of the node's cluster has read the slot map (the exits above are
            // the same in all of them): chunk 0 retires R while the others go on
            cg::this_cluster().sync();
            if (chunk == 0)
                for (int i = threadIdx.x; i < nr; i += blockDim.x) g.prec_pos[pidx(g, u, pm[rem[i]])] = -1;
        }
        const int per = (nt + nchunks - 1) / nchunks;
        const int t0 = chunk * per, t1 = min(nt, t0 + per);
        // many removals in a cluster: rank 0 factors P_RR and the others copy the factor
        // (distributed shared memory); else every chunk with rows factors it itself
        const bool share = CL && nr >= PREC_SHARE_MIN;   // the same in every chunk
        if (!share && t0 >= t1) return;                // no kept rows in this chunk
        // P_RR = L D L^T, right-looking with one barrier per pivot: the trailing update of
        // pivot k reads the unscaled column k (times 1/D_k); column k-1 is scaled to L in
        // the same phase; thread 0 updates the next diagonal entry first and forms 1/D.
        double *A = smd;                         // nr x nr row-major: L below the diagonal
        double *rdv = A + nr * nr;               // 1/D
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        bool brk = false;
        if (!share || chunk == 0) {
        for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) {
            const int a2 = e / nr, b2 = e - a2 * nr;
            if (b2 <= a2) A[e] = P[rem[a2] * PREC_MAX + rem[b2]];
        }
        __syncthreads();
        // pivot flags alternate by parity: thread 0 writes the flag of pivot k+1 while
        // the other threads may still read the flag of pivot k
        __shared__ int badv[2];
        if (threadIdx.x == 0) {
            const double d = A[0];
            badv[0] = !(d > DEGEN);
            rdv[0] = rcp_newton(d);
        }
        for (int k = 0; k < nr; ++k) {
            __syncthreads();                     // column k and 1/D_k final
            if (badv[k & 1]) {                   // uniform: every thread reads the same flag
                brk = true;
                break;
            }
            if (k > 0)
                for (int i = k + threadIdx.x; i < nr; i += blockDim.x) A[i * nr + k - 1] *= rdv[k - 1];
            const double rk = rdv[k];
            // the trailing triangle k < c <= i < nr, flattened row by row over the threads
            // (entry e = r (r + 1) / 2 + c' for row k + 1 + r, column k + 1 + c'), so that a
            // warp's FP64 instructions carry 32 entries; entry 0, the next pivot, is thread 0's
            const int mt = nr - k - 1;
            for (int e = threadIdx.x; e < mt * (mt + 1) / 2; e += blockDim.x) {
                int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                if (r * (r + 1) / 2 > e) --r;
                else if ((r + 1) * (r + 2) / 2 <= e) ++r;
                const int i = k + 1 + r, c = k + 1 + (e - r * (r + 1) / 2);
                const double v = fma(-(A[i * nr + k] * rk), A[c * nr + k], A[i * nr + c]);
                A[i * nr + c] = v;
                if (e == 0) {                                // thread 0: the next pivot
                    badv[(k + 1) & 1] = !(v > DEGEN);
                    rdv[k + 1] = rcp_newton(v);
                }
            }
        }
        __syncthreads();
        }
        if constexpr (CL) {
            if (share) {
                __shared__ int fac_bad;
                if (chunk == 0 && threadIdx.x == 0) fac_bad = brk;
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();                                 // rank 0's factor and flag are ready
                if (chunk != 0) {
                    brk = *cl.map_shared_rank(&fac_bad, 0) != 0;
                    const double *A0 = cl.map_shared_rank(smd, 0);
                    if (!brk)
                        for (int e = threadIdx.x; e < nr * nr + nr; e += blockDim.x) smd[e] = A0[e];   // L, then 1/D
                }
                cl.sync();                                 // rank 0 keeps its shared memory until every copy is done
            }
        }
        if (brk) {
            // P_RR is a principal block of an SPD inverse; a pivot at the floor means the
            // block has lost accuracy: drop it (rebuilt from corr if the node needs it)
            if (chunk == 0 && threadIdx.x == 0) g.prec_m[u] = -2;
            return;
        }
        if (t0 >= t1) return;                          // no kept rows in this chunk
        // the entries P[rem[q]][keep[j]] every row of the update reads (rows of R are
        // never written here): staged once per CTA, all loads in flight together
        double *Sg = rdv + nr;                   // nr x nt
        for (int e = threadIdx.x; e < nr * nt; e += blockDim.x) {
            const int q = e / nt, j = e - q * nt;
            Sg[e] = P[(long long)rem[q] * PREC_MAX + keep[j]];
        }
        __syncthreads();
        const bool two = nr > 32;                // lanes hold y_q for q = lane, lane + 32
        for (int t = t0 + w; t < t1; t += nw) {
            double *Pi = P + (long long)keep[t] * PREC_MAX;
            double b0 = lane < nr ? Pi[rem[lane]] : 0.0;
            double b1 = two && lane + 32 < nr ? Pi[rem[lane + 32]] : 0.0;
            for (int k = 0; k < nr; ++k) {        // L z = b (unit lower)
                const double zk = __shfl_sync(0xffffffffu, k < 32 ? b0 : b1, k & 31);
                if (lane > k && lane < nr) b0 = fma(-A[lane * nr + k], zk, b0);
                if (two && lane + 32 > k && lane + 32 < nr) b1 = fma(-A[(lane + 32) * nr + k], zk, b1);
            }
            if (lane < nr) b0 *= rdv[lane];
            if (two && lane + 32 < nr) b1 *= rdv[lane + 32];
            for (int k = nr - 1; k > 0; --k) {    // L^T y = D^{-1} z
                const double yk = __shfl_sync(0xffffffffu, k < 32 ? b0 : b1, k & 31);
                if (lane < k) b0 = fma(-A[k * nr + lane], yk, b0);
                if (two && lane + 32 < k) b1 = fma(-A[k * nr + lane + 32], yk, b1);
            }
            // the kept columns in groups of 32 (lanes), two groups per pass; only the
            // groups the row has are issued (the FP64 pipe is the scarce one)
            for (int x0 = 0; 32 * x0 < nt; x0 += 2) {
                const int j0 = lane + 32 * x0, j1 = j0 + 32;
                const bool h1 = 32 * (x0 + 1) < nt;        // warp-uniform: a second group exists
                double a0 = j0 < nt ? Pi[keep[j0]] : 0.0;
                double a1 = h1 && j1 < nt ? Pi[keep[j1]] : 0.0;
#pragma unroll 4
                for (int q = 0; q < nr; ++q) {
                    const double yq = __shfl_sync(0xffffffffu, q < 32 ? b0 : b1, q & 31);
                    const double *Sq = Sg + q * nt;
                    if (j0 < nt) a0 = fma(-yq, Sq[j0], a0);
                    if (h1 && j1 < nt) a1 = fma(-yq, Sq[j1], a1);
                }
                if (j0 < nt) Pi[keep[j0]] = a0;
                if (h1 && j1 < nt) Pi[keep[j1]] = a1;
            }
        }
        if (chunk == 0 && threadIdx.x == 0)
            atomicAdd(&g.ctr->flops_prec, (ull)nr * nr * nr / 3 + 2ull * nt * nr * (nr + nt));
        return;
    }
    if (chunk != 0 || !(need < 0 ? g.prec_need[u] : need)) return;
    const int m = g.deg[u] + 1;
    if (threadIdx.x == 0) {
        bad = 0;
        int o = 0;
        const int *nb = g.nbr + nidx(g, u);
        const int dg = g.deg[u];
        bool placed = false;
        for (int i = 0; i < dg; ++i) {
            if (!placed && nb[i] > u) {
                mem[o++] = u;
                placed = true;
            }
            mem[o++] = nb[i];
        }
        if (!placed) mem[o++] = u;
    }
    __syncthreads();
    double *A = smd, *colk = A + m * m;
    for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5)
        for (int c = threadIdx.x & 31; c < m; c += 32) A[i * m + c] = C64[cidx(g.prow, ldc, mem[i], mem[c])];
    __syncthreads();
    sweep_inverse_block(A, m, m, colk, &bad);     // A = -corr[F,F]^{-1}
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            g.prec_m[u] = -1;
            g.prec_need[u] = 0;
        }
        return;
    }
    double *P = g.prec + (long long)u * PREC_MAX * PREC_MAX;
    // a block rebuilt after being dropped: clear the stale slot map first
    for (int w = threadIdx.x; w < p; w += blockDim.x) g.prec_pos[pidx(g, u, w)] = -1;
    __syncthreads();
    for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5)
        for (int c = threadIdx.x & 31; c < m; c += 32) P[i * PREC_MAX + c] = -A[i * m + c];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        g.prec_mem[(long long)u * PREC_MAX + i] = mem[i];
        g.prec_pos[pidx(g, u, mem[i])] = (short)i;
    }
    if (threadIdx.x == 0) {
        g.prec_m[u] = m;
        g.prec_need[u] = 0;
        atomicAdd(&g.ctr->flops_prec, (ull)m * m * m);
        atomicAdd(&g.ctr->prec_builds, 1ull);
    }
}

__global__ void __cluster_dims__(1, PREC_CHUNKS, 1) __launch_bounds__(512)
    prec_update_kernel(GraphDev g, TestParams tp, const double *C64, int ldc)
{
    extern __shared__ double smd[];
    prec_body<true>(g, tp, C64, ldc, blockIdx.x, blockIdx.y, PREC_CHUNKS, smd);
}

// After prec_body<false> of every chunk: the slots of node u's maintained block
// whose members the commit deleted leave the slot map (entry -1).  A dropped
// block (prec_m <= 0) keeps its stale map until it is rebuilt.
__device__ __forceinline__ void prec_retire(const GraphDev &g, int u)
{
    const int m0 = g.prec_m[u];
    if (m0 <= 0) return;
    const int *pm = g.prec_mem + (long long)u * PREC_MAX;
    short *pos = g.prec_pos + pidx(g, u, 0);
    const uint32_t *row = g.adj + (long long)u * g.W;
    for (int sl = threadIdx.x; sl < m0; sl += blockDim.x) {
        const int w = pm[sl];
        if (w != u && pos[w] >= 0 && !((row[w >> 5] >> (w & 31)) & 1u)) pos[w] = -1;
    }
}

// The first stage's blocks from the closed-form stage's inverse P = corr^{-1}: node
// u's block starts as all of P (every node a member, slot = id), and the downdate
// that follows drops the non-neighbours R = V \ F, which leaves corr[F,F]^{-1}
// (the inverse of a principal submatrix, as for every later deletion), F = adj(u)
// u {u}: a downdate of |R| members instead of a sweep of the whole neighbourhood.
// Nodes with more than PREC_RMAX non-neighbours keep the sweep build.
__global__ void __launch_bounds__(256) prec_seed_kernel(GraphDev g, const double *P, int ldp)
{
    const int u = blockIdx.x;
    const LevelInfo *I = g.info;
    const int p = g.p;
    if (stopped(I) || !I->stage_a_ran || !g.prec_need[u] || p - 1 - g.deg[u] > PREC_RMAX) return;
    double *B = g.prec + (long long)u * PREC_MAX * PREC_MAX;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e - i * p;
        B[(long long)i * PREC_MAX + j] = P[(long long)i * ldp + j];
    }
    for (int w = threadIdx.x; w < p; w += blockDim.x) {
        g.prec_mem[(long long)u * PREC_MAX + w] = w;
        g.prec_pos[pidx(g, u, w)] = (short)w;
    }
    if (threadIdx.x == 0) {
        g.prec_m[u] = p;
        g.prec_need[u] = 0;
        g.dchg[u] = p - 1 - g.deg[u];                  // the downdate's removals
        atomicAdd(&g.ctr->prec_builds, 1ull);
    }
}

// ---------------------------------------------------------------- commit
// End of stage l (PC-stable): delete every pair with a recorded key, store its
// first separating set (side, rank, and the expanded node list), reset the
// key, and count the tests of the sequential canonical order:
// key (0, rank) -> rank+1; key (1, rank) -> C(d_u,l) + rank+1; none -> both sides.
// The commit of CTA `cta` of `ncta` (sb: the small binomial table, loaded).
// soo: when given, a shared copy of the ordered-pair offsets (p+1 entries): the
// owner of a pair is found there instead of in the head's owner table.
__device__ __forceinline__ void commit_body(const GraphDev &g, int l_fixed, int explicit_sets, int count_canonical,
                                            const ull *sb, int cta, int ncta, const long long *soo = nullptr)
{
    const int l = l_fixed >= 0 ? l_fixed : g.info->l;
    const bool prop = stage_prop(g, l);
    const long long nop = g.info->n_opairs;
    const int p = g.p;
    const int lane = threadIdx.x & 31;
    ull removed = 0, canon = 0;
    // one ordered pair per thread (grid-stride in warp-aligned steps)
    for (long long base = cta * (long long)blockDim.x + (threadIdx.x & ~31); base < nop;
         base += (long long)ncta * blockDim.x) {
        const long long o = base + lane;
        bool expand = false, cut = false;                 // cut: this lane removes the edge (u, v)
        int su = 0, jj = 0, dd = 0, cu_ = 0, cv_ = 0, side_ = 0, j_ = 0, du_ = 0, dv_ = 0;
        long long e_ = 0;
        ull rank = 0, off = 0;
        if (o < nop) {
            // owner node: the head kernel's table inside the stage loop, else a search
            const int u = soo ? (int)(upper_bound_dev(soo, (long long)p + 1, o) - 1)
                              : l_fixed < 0 ? g.opu[o] : (int)(upper_bound_dev(g.ooff, (long long)p + 1, o) - 1);
            const int j = (int)(o - g.ooff[u]);
            const int v = g.nbr[nidx(g, u) + j];
            if (u < v) {
                const long long e = pidx(g, u, v);
                // every load of the pair before its first store (the compiler keeps
                // loads behind stores it cannot prove apart)
                const ull key = g.best[e];
                const int du = g.deg[u] - 1, dv = g.deg[v] - 1;
                const bool dof = !g.nvec || g.nvec[u] - l - 3 > 0;   // u and v share their instance
                const ull T0 = count_canonical && du >= l && dof ? g.binom[(long long)du * g.ldb + l] : 0ull;
                const ull T1 = count_canonical && dv >= l && dof ? g.binom[(long long)dv * g.ldb + l] : 0ull;
                g.best[e] = KEY_NONE;                     // ready for the next stage
                if (count_canonical) {
                    ull c;
                    if (key == KEY_NONE) c = sat_add(T0, T1);
                    else if ((key >> 62) == 0) c = key + 1;
                    else c = sat_add(T0, (key & ((1ull << 62) - 1)) + 1);
                    canon = sat_add(canon, c);
                }
                if (key != KEY_NONE) {
                    cut = true;
                    cu_ = u;
                    cv_ = v;
                    const int side = (int)(key >> 62);
                    rank = key & ((1ull << 62) - 1);
                    g.sep_level[e] = l;
                    g.sep_side[e] = side;
                    g.sep_rank[e] = (long long)rank;
                    ++removed;
                    side_ = side;
                    e_ = e;
                    j_ = j;
                    du_ = du;
                    dv_ = dv;
                }
            }
        }
        // room for the explicit sets in the sepset pool: one atomic per warp, each cutting
        // lane's offset from a scan of the lanes' set sizes
        if (cut && !explicit_sets) g.sep_off[e_] = -1;
        {
            const bool alloc = cut && explicit_sets;   // also at l = 0: an empty set, not V \ {u, v}
            const ull want = alloc ? (ull)l : 0ull;
            ull incl = want;
            for (int k = 1; k < 32; k <<= 1) {
                const ull y = __shfl_up_sync(0xffffffffu, incl, k);
                if (lane >= k) incl += y;
            }
            const ull wtot = __shfl_sync(0xffffffffu, incl, 31);
            ull wbase = 0;
            if (lane == 31 && wtot) wbase = atomicAdd(&g.ctr->pool_len, wtot);
            wbase = __shfl_sync(0xffffffffu, wbase, 31);
            if (alloc) {
                off = wbase + incl - want;
                g.sep_off[e_] = (long long)off;
                if ((long long)(off + l) > g.pool_cap) {
                    g.info->pool_overflow = 1;           // the host enlarges the pool and reruns
                    g.info->halt = 1;
                } else {
                    su = side_ ? cv_ : cu_;
                    jj = side_ ? lower_bound_int(g.nbr + nidx(g, cv_), dv_ + 1, cu_) : j_;
                    dd = side_ ? dv_ : du_;
                    expand = true;
                }
            }
        }
        // adjacency bits of the removed edges: the lanes of a warp hold consecutive
        // neighbours v of one node u, so their bits in row u share words -- one atomic
        // per word with the lanes' bits combined; row v's bit u per lane
        {
            const long long wu = cut ? (long long)cu_ * g.W + (cv_ >> 5) : -1ll - lane;
            const unsigned peers = __match_any_sync(0xffffffffu, wu);
            const unsigned bits = __reduce_or_sync(peers, cut ? 1u << (cv_ & 31) : 0u);
            if (cut && (int)(__ffs(peers) - 1) == lane) atomicAnd(g.adj + wu, ~bits);
            if (cut) atomicAnd(g.adj + (long long)cv_ * g.W + (cu_ >> 5), ~(1u << (cu_ & 31)));
        }
        // each lane expands its own removed pair (the pairs of a warp are consecutive
        // neighbours of one node, so removals cluster; one pair at a time per warp
        // serialised them)
        if (expand) {
            const int *nb = g.nbr + nidx(g, su);
            const int kd = dd - l;                        // dropped members
            if (kd <= KC_MAX && kd < l) {
                // through the complement: R = the kd dropped positions, at lex rank
                // C(dd,l) - 1 - rank among the kd-subsets; S = the rest, ascending
                int posR[KC_MAX], nodeR[KC_MAX];
                const ull T = g.binom[(long long)dd * g.ldb + l];
                const bool small_d = dd < SB_ROWS;
                unrank_lex_fixed<KC_MAX>(T - 1 - rank, dd, kd, small_d ? sb : g.binom, small_d ? SB_COLS : g.ldb,
                                         posR);
#pragma unroll
                for (int i = 0; i < KC_MAX; ++i) nodeR[i] = i < kd ? cand_node(g, prop, su, jj, dd, posR[i]) : -1;
                // the neighbour list in batches of 8 independent read-only loads (one
                // round trip per batch, not per neighbour: the pool stores follow them)
                int o2 = 0;
                for (int y0 = 0; y0 <= dd; y0 += 8) {
                    int wv[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) wv[k] = y0 + k <= dd ? __ldg(nb + y0 + k) : -1;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int y = y0 + k;
                        if (y > dd || y == jj) continue;
                        bool keep = true;
#pragma unroll
                        for (int i = 0; i < KC_MAX; ++i) keep &= nodeR[i] != wv[k];
                        if (keep) g.pool[off + o2++] = wv[k];
                    }
                }
            } else {
                ull r = rank;
                int x = 0;
                // C(a, b) from the shared table where it covers them (a < SB_ROWS, b < SB_COLS)
                auto bin = [&](int a, int b) -> ull {
                    return (a < SB_ROWS && b < SB_COLS) ? sb[a * SB_COLS + b] : g.binom[(long long)a * g.ldb + b];
                };
                int lg = 0;
                while ((1 << lg) < dd + 1) ++lg;
                if (l * lg < dd) {
                    // each position by a binary search (the walk below takes up to dd dependent
                    // loads): the sets whose i-th position lies in [x, y) number
                    // C(dd - x, l - i) - C(dd - y, l - i)
                    for (int i = 0; i < l; ++i) {
                        const int r1 = l - i;
                        const ull base = bin(dd - x, r1), target = base - r;
                        int lo = x, hi = dd - r1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (bin(dd - mid, r1) >= target) lo = mid;
                            else hi = mid - 1;
                        }
                        r -= base - bin(dd - lo, r1);
                        g.pool[off + i] = cand_node(g, prop, su, jj, dd, lo);
                        x = lo + 1;
                    }
                } else {
                    for (int i = 0; i < l; ++i) {
                        while (x < dd - (l - i)) {
                            const ull c = bin(dd - x - 1, l - i - 1);
                            if (r < c) break;
                            r -= c;
                            ++x;
                        }
                        g.pool[off + i] = cand_node(g, prop, su, jj, dd, x);
                        ++x;
                    }
                }
                if (prop) sort_small(g.pool + off, l);
            }
        }
    }
    // the counters: one atomic per warp (a stage's commit has up to p(p-1) threads)
    for (int k = 16; k > 0; k >>= 1) {
        removed += __shfl_xor_sync(0xffffffffu, removed, k);
        canon = sat_add(canon, __shfl_xor_sync(0xffffffffu, canon, k));
    }
    if (lane == 0) {
        if (removed) atomicAdd(&g.ctr->edges_removed, removed);
        if (canon) atomicAdd(&g.ctr->tests_canonical, canon);
    }
}

__global__ void commit_kernel(GraphDev g, int l_fixed, int explicit_sets, int count_canonical)
{
    if (stopped(g.info)) return;
    __shared__ ull sb[SB_ROWS * SB_COLS];
    load_small_binom(g, sb);
    __syncthreads();
    commit_body(g, l_fixed, explicit_sets, count_canonical, sb, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- stage loop in one kernel
// Every CTA of the stage loop plans stage l itself, as the head does: the
// complement and direct tests' per-node offsets in shared memory (soff, sdoff;
// entry p holds the total).  True when the stage is one for the loop: direct tests
// only of at most LOOP_MMAX - 2 members and outside the proposal's stages, nothing
// saturated, within the budget (the captured loop's head reports the others).
// sh: 64 words of scratch; sdeg, sT receive every node's degree and C(d, l).
__device__ __forceinline__ bool loop_stage_plan(const GraphDev &g, const TestParams &tp, int l, double budget,
                                                ull *soff, ull *sh, int *sdeg, ull *sT, ull *sdoff)
{
    const int t = threadIdx.x, p = g.p;                // p <= LOOP_PMAX < blockDim.x
    ull v[2] = {0ull, 0ull};
    bool sat = false;
    if (t < p) {
        const int dg = g.deg[t], d = dg - 1;
        const ull T = (dg > 0 && d >= l && dof_ok(tp, t, l)) ? g.binom[(long long)d * g.ldb + l] : 0ull;
        sdeg[t] = dg;
        sT[t] = T;
        const ull tot = sat_mul(T, (ull)dg);
        sat = tot == KEY_NONE;
        if (T && comp_eligible(d, l, tp) && g.prec_m[t] > 0) v[0] = tot;
        else v[1] = tot;
    }
    const int ssat = __syncthreads_or(sat);
    ull ex[2], tot[2];
    block_scan_sat<2>(v, ex, tot, sh);
    if (t < p) {
        soff[t] = ex[0];
        sdoff[t] = ex[1];
    }
    if (t == 0) {
        soff[p] = tot[0];
        sdoff[p] = tot[1];
    }
    __syncthreads();
    // direct tests only where the warp buffer holds them, where no proposal order could
    // apply (the captured loop scores such stages), and at most LOOP_DIRECT_ROUNDS per
    // warp of the grid (larger stages run faster on the small-stage kernels)
    const ull nwarps = (ull)gridDim.x * (blockDim.x >> 5);
    const bool direct_ok = tot[1] == 0 || (l + 2 <= LOOP_MMAX && tot[1] <= LOOP_DIRECT_ROUNDS * nwarps &&
                                           !(g.row_off && l >= 1 && l <= tp.learned_lmax));
    return !ssat && tot[0] != KEY_NONE && tot[1] != KEY_NONE && direct_ok &&
           (double)tot[0] + (double)tot[1] <= budget;
}

// Every CTA of the stage loop forms the tail's results it needs from the degrees
// of the new frozen graph (stage l just committed): the ordered-pair offsets
// (soo[p] = their total), and per node the precision-block request for the next
// stage min(l - 1, L*) (reversed order), as the tail does.  CTA 0's tail writes
// the same into memory for the captured loop.  sh: 32 words of scratch.
// Also the list of nodes whose blocks have work this stage (a maintained block whose
// node lost neighbours, or a build request): sact[0..*nact).
__device__ __forceinline__ void loop_tail_plan(const GraphDev &g, const TestParams &tp, int l, long long *soo,
                                               int *sneed, ull *sh, int *sact, int *nact)
{
    __shared__ int smx[32];
    const int t = threadIdx.x, p = g.p, lane = t & 31, w = t >> 5;
    const int dg = t < p ? __ldcg(g.deg + t) : 0;
    ull v[1] = {(ull)dg}, ex[1], tot[1];
    block_scan_sat<1>(v, ex, tot, sh);
    int mx = dg;
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) smx[w] = mx;
    if (t < p) soo[t] = (long long)ex[0];
    if (t == 0) soo[p] = (long long)tot[0];
    __syncthreads();
    int lmax = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) lmax = max(lmax, smx[i]);
    const int nl = min(l - 1, lmax - 1);
    bool act = false;
    if (t < p) {
        const int pm = g.prec_m[t];
        const int nd = nl >= 0 && dg > 0 && comp_eligible(dg - 1, nl, tp) && (pm == 0 || pm == -2);
        sneed[t] = nd;
        act = nd || (pm > 0 && __ldcg(g.dchg + t) != 0);
    }
    __syncthreads();                                    // sh free again
    ull va[1] = {act ? 1ull : 0ull}, exa[1], tota[1];
    block_scan_sat<1>(va, exa, tota, sh);
    if (act) sact[exa[0]] = t;
    if (t == 0) *nact = (int)tota[0];
    __syncthreads();
}

// Small problems in the reversed order (Algorithm 2) spend most of a stage on the
// latency of its launches, not on its tests.  This cooperative kernel runs the
// stages whose tests all take the complement path, one after the other, with a
// grid-wide barrier where the captured loop has a kernel boundary:
//   plan (every CTA: the head's offsets, in its shared memory), complement tests,
//   the previous stage's retirement of deleted block members | commit (the
//   owner of a pair found in a shared copy of the pair offsets) | degrees |
//   tail (CTA 0 into memory; every CTA forms the offsets and block requests it
//   needs itself) and precision downdates and builds.
// Stages with direct tests of at most LOOP_MMAX - 2 members run them too, a warp per
// test beside the complement tests.  It returns at the first stage it does not take
// (larger direct tests, or stages the proposal may score: the captured loop, whose
// head recomputes that stage, runs it and the rest), or when the search ends or halts.
// The exits are taken by all CTAs together: `done` and `halt` are written only in
// the commit and the last phase (the tail), each followed by a barrier, and every
// CTA plans the stage from the same data.  The stage l is read once per pass, at
// its start: the tail moves it on in the last phase.
// pre: first the first stage's block builds and downdates (the seeded blocks drop
// their non-neighbours), in place of the cluster kernel.
__global__ void __launch_bounds__(LOOP_THREADS, 1) stage_loop_kernel(GraphDev g, TestParams tp, const float *C32,
                                                                     const double *C64, int ldc, double budget,
                                                                     int cap, int chunks, int pre)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double lsm[];
    __shared__ ull sb[SB_ROWS * SB_COLS];
    __shared__ ull soff[LOOP_PMAX + 1];
    __shared__ ull sh[2 * 32];
    __shared__ long long soo[LOOP_PMAX + 1];
    __shared__ int sdeg[LOOP_PMAX];
    __shared__ ull sT[LOOP_PMAX];
    __shared__ ull sdoff[LOOP_PMAX + 1];
    __shared__ int sneed[LOOP_PMAX];
    __shared__ int sact[LOOP_PMAX];
    __shared__ int nact;
    LevelInfo *I = g.info;
    load_small_binom(g, sb);
    for (int i = threadIdx.x; i <= g.p; i += blockDim.x) soo[i] = g.ooff[i];   // the first stage's, from the tail
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwg = (int)((gridDim.x * blockDim.x) >> 5);
    if (pre) {
        // the tail scheduled the requests; every CTA lists the nodes with block work
        const int t = threadIdx.x;
        bool act = false;
        if (t < g.p) {
            const int nd = g.prec_need[t], pm = g.prec_m[t];
            sneed[t] = nd;
            act = nd || (pm > 0 && g.dchg[t] != 0);
        }
        ull va[1] = {act ? 1ull : 0ull}, exa[1], tota[1];
        block_scan_sat<1>(va, exa, tota, sh);
        if (act) sact[exa[0]] = t;
        if (t == 0) nact = (int)tota[0];
        __syncthreads();
        const int ch = max(1, min(chunks, (int)gridDim.x / max(1, nact)));
        for (int item = blockIdx.x; item < nact * ch; item += gridDim.x) {
            const int u = sact[item / ch];
            prec_body<false>(g, tp, C64, ldc, u, item % ch, ch, lsm, sneed[u]);
            __syncthreads();
        }
        grid.sync();
    }
    for (int it = 0; it <= g.p; ++it) {                 // one pass per stage, at most p stages
        if (stopped(I)) break;
        const int lcur = I->l;                          // moved on only by the tail below
        if (!loop_stage_plan(g, tp, lcur, budget, soff, sh, sdeg, sT, sdoff)) break;
        if (sdoff[g.p] > 0) {                           // the stage's direct tests, a warp each
            unsigned char *mine = (unsigned char *)lsm + (size_t)(threadIdx.x >> 5) * loop_direct_bytes();
            if (tp.precision == 0) loop_direct_body<true>(g, tp, lcur, sdoff, C32, C64, ldc, mine);
            else loop_direct_body<false>(g, tp, lcur, sdoff, C32, C64, ldc, mine);
        }
        complement_body(g, tp, sb, soff, LOOP_PMAX + 1, blockIdx.x, gridDim.x, true, sdeg, sT);
        // then the previous downdates' deletions leave the slot maps (the complement tests
        // read only the slots of current neighbours; repeating it is harmless)
        for (int u = blockIdx.x; u < g.p; u += gridDim.x) prec_retire(g, u);
        grid.sync();
        if (!stopped(I)) commit_body(g, -1, 1, 1, sb, blockIdx.x, gridDim.x, soo);
        grid.sync();
        if (!stopped(I))
            for (int u = gw; u < g.p; u += nwg) node_degree(g, u, lane, true);
        grid.sync();
        // the tail: CTA 0 in memory (next stage, loop end, offsets, requests), every
        // CTA for itself what the downdates and the next commit need
        if (blockIdx.x == 0) tail_body(g, tp, cap, 0, nullptr, 0, 0, 0, StageConds{}, true);
        loop_tail_plan(g, tp, lcur, soo, sneed, sh, sact, &nact);
        // the nodes with work only, each node's kept rows over as many CTAs as leave one
        // item per CTA (up to `chunks`): a CTA's items run one after the other
        const int ch = max(1, min(chunks, (int)gridDim.x / max(1, nact)));
        for (int item = blockIdx.x; item < nact * ch; item += gridDim.x) {
            const int u = sact[item / ch];
            prec_body<false>(g, tp, C64, ldc, u, item % ch, ch, lsm, sneed[u]);
            __syncthreads();                            // the body's shared arrays are reused
        }
        grid.sync();
    }
    // the last stage's deletions, also when the loop ran out of passes (no barrier
    // needed: nothing else runs in the kernel any more)
    for (int u = blockIdx.x; u < g.p; u += gridDim.x) prec_retire(g, u);
}

// ---------------------------------------------------------------- re-verification
// Every explicit separating set recorded in the sepset store is tested again in
// FP64 from the FP64 correlation matrix (one warp per removed pair); a set that
// does not come out independent sets the device status (PC_ERR_INTERNAL).
__global__ void __launch_bounds__(256) reverify_kernel(GraphDev g, TestParams tp, const float *C32,
                                                       const double *C64, int ldc, int mmax, int ms,
                                                       int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem_raw + (size_t)wib * per_warp_bytes;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)mmax * ms * sizeof(double));
    const int p = g.p;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    ull fails = 0;
    // nothing to re-test when no stage ran in the proposed order
    if (g.scored) {
        bool any = false;
        for (int l = lane; l <= mmax - 2 && l < p; l += 32) any |= g.scored[l] != 0;
        if (!__any_sync(0xffffffffu, any)) return;
    }
    // pair (a, b), a < b within a's instance: row a of the pair arrays, scanned 32
    // entries at a time by the lanes; the pairs to re-test are taken one by one
    for (long long a_ = gw; a_ < p; a_ += nw)
    for (int b0 = (int)a_ + 1, a = (int)a_, bend = g.blk_hi ? g.blk_hi[a] : p; b0 < bend; b0 += 32) {
        int lb = -1;
        long long ob = -1;
        bool need = false;
        if (b0 + lane < bend) {
            const long long e = pidx(g, a, b0 + lane);
            lb = g.sep_level[e];
            ob = g.sep_off[e];
            // an explicit set of a stage that ran in the proposed order (a plain-order
            // stage's set is the canonical one)
            need = lb >= 0 && ob >= 0 && lb + 2 <= mmax && !(g.scored && !g.scored[lb]);
        }
        for (unsigned m = __ballot_sync(0xffffffffu, need); m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            const int b = b0 + src;
            const int l = __shfl_sync(0xffffffffu, lb, src);
            const long long off = __shfl_sync(0xffffffffu, ob, src);
            if (lane == 0) {
                for (int i = 0; i < l; ++i) nd[i] = g.pool[off + i];
                nd[l] = a;
                nd[l + 1] = b;
            }
            __syncwarp();
            const double sq = sqrt((double)(n_of(tp, a) - l - 3));
            double r;
            float z;
            // FP32 under the trust rule (guard, bound, band), FP64 where it requires it
            // (FP64 throughout in the FP64 mode): the warp-per-test evaluation, members
            // in ascending order, independent of the kernel that found the set
            const bool ind = tp.precision == 0
                                 ? warp_test<true>(nd, l + 2, l, nullptr, C64, ldc, tp, sq, (float)sq, Mbuf, ms, acc, r, z)
                                 : warp_test<false>(nd, l + 2, l, C32, C64, ldc, tp, sq, (float)sq, Mbuf, ms, acc, r, z);
            if (!ind) ++fails;
            __syncwarp();
        }
    }
    if (lane == 0 && fails) g.ctr->status = 8;
}

// ---------------------------------------------------------------- raw batches
template <bool F64>
__global__ void __launch_bounds__(256) ci_list_kernel(const int *ij, const int *S, int l, long long b,
                                                      const float *C32, const double *C64, int ldc,
                                                      int p, TestParams tp, double *r_out,
                                                      uint8_t *indep_out, float *z_out,
                                                      DevCounters *ctr, const int *blk_lo,
                                                      const int *blk_hi, int ms, int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = l + 2;
    unsigned char *mine = smem_raw + (size_t)wib * per_warp_bytes;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)m * ms * sizeof(double));
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const double sq = sqrt((double)(tp.n - l - 3));
    const float sqf = (float)sq;
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    for (long long t = gw; t < b; t += nw) {
        bool okid = true;
        if (lane == 0) {
            for (int i = 0; i < l; ++i) nd[i] = S[t * l + i];
            nd[l] = ij[2 * t];
            nd[l + 1] = ij[2 * t + 1];
        }
        __syncwarp();
        for (int i = 0; i < m; ++i) okid = okid && nd[i] >= 0 && nd[i] < p;
        okid = okid && nd[l] != nd[l + 1];
        if (okid && blk_lo) {
            // batched problems: every node of a test must be in x's instance
            const int lo = blk_lo[nd[l]], hi = blk_hi[nd[l]];
            for (int i = 0; i < m; ++i) okid = okid && nd[i] >= lo && nd[i] < hi;
        }
        if (!okid) {
            if (lane == 0) ctr->status = 1;
            __syncwarp();
            continue;
        }
        double r;
        float z;
        ++acc.tests;
        const double sqt = tp.nvec ? sqrt((double)(n_of(tp, nd[l]) - l - 3)) : sq;
        bool ind = warp_test<F64>(nd, m, l, C32, C64, ldc, tp, sqt, tp.nvec ? (float)sqt : sqf, Mbuf, ms, acc,
                                  r, z);
        if (lane == 0) {
            if (r_out) r_out[t] = r;
            if (z_out) z_out[t] = z;
            if (indep_out) indep_out[t] = ind ? 1 : 0;
        }
        __syncwarp();
    }
    if (lane == 0) flush_acc(acc, ctr);
}

// ---------------------------------------------------------------- launchers
static int g_num_sms = 0;
static int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

// ---------------------------------------------------------------- path-restricted pools
// The candidate pool adj(G,i,j) intersected with path(G,i,j) of Algorithms 1 and 2
// (Sec. 2.1 notation): the neighbours of i or of j, other than i and j, that lie
// on some simple i-j path of the frozen graph.  A neighbour k of i lies on one iff
// k reaches j in the graph without i (then i, k, ..., j is such a path), a
// neighbour of j iff it reaches i without j.  comp[x * p + k] labels the
// connected component of k in the frozen graph without node x (-1 at k = x); one
// CTA per x, by frontier expansion over the adjacency bitset in shared memory.
// The labels' values do not matter, only their equality.
__global__ void __launch_bounds__(256) pp_components_kernel(GraphDev g, int *comp)
{
    extern __shared__ unsigned pp_bits[];
    const int p = g.p, W = g.W, x = blockIdx.x;
    unsigned *vis = pp_bits, *front = pp_bits + W, *nxt = pp_bits + 2 * W;
    __shared__ int start_s;
    int *cx = comp + (long long)x * p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        // nodes >= p and x itself count as visited
        unsigned v = 0;
        for (int b = 0; b < 32; ++b)
            if (w * 32 + b >= p || w * 32 + b == x) v |= 1u << b;
        vis[w] = v;
    }
    if (threadIdx.x == 0) cx[x] = -1;
    __syncthreads();
    for (int id = 0;; ++id) {
        // the lowest node not yet labelled starts the next component
        if (threadIdx.x == 0) {
            int st = -1;
            for (int w = 0; w < W && st < 0; ++w)
                if (~vis[w]) st = w * 32 + __ffs(~vis[w]) - 1;
            start_s = st;
        }
        __syncthreads();
        const int st = start_s;
        if (st < 0) break;
        for (int w = threadIdx.x; w < W; w += blockDim.x) front[w] = w == (st >> 5) ? 1u << (st & 31) : 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            vis[st >> 5] |= 1u << (st & 31);
            cx[st] = id;
        }
        __syncthreads();
        for (;;) {
            for (int w = threadIdx.x; w < W; w += blockDim.x) nxt[w] = 0u;
            __syncthreads();
            // every frontier node y: OR its adjacency row into nxt (a warp per word of front)
            for (int fw = warp; fw < W; fw += nwarps) {
                unsigned f = front[fw];
                while (f) {
                    const int y = fw * 32 + __ffs(f) - 1;
                    f &= f - 1;
                    const uint32_t *row = g.adj + (long long)y * W;
                    for (int w = lane; w < W; w += 32) {
                        const unsigned a = row[w];
                        if (a) atomicOr(&nxt[w], a);
                    }
                }
            }
            __syncthreads();
            int more = 0;
            for (int w = threadIdx.x; w < W; w += blockDim.x) {
                const unsigned nw = nxt[w] & ~vis[w];
                front[w] = nw;
                vis[w] |= nw;
                more |= nw != 0;
                for (unsigned m = nw; m; m &= m - 1) cx[w * 32 + __ffs(m) - 1] = id;
            }
            if (!__syncthreads_or(more)) break;
        }
    }
}

// The pool of the adjacent pair (a, b), ascending, into pool (one warp); returns its size.
__device__ __forceinline__ int pp_pool(const GraphDev &g, const int *comp, int a, int b, int *pool)
{
    const int p = g.p, lane = threadIdx.x & 31;
    const int *ca = comp + (long long)a * p, *cb = comp + (long long)b * p;
    const int la = ca[b], lb = cb[a];
    int dp = 0;
    for (int k0 = 0; k0 < p; k0 += 32) {
        const int k = k0 + lane;
        bool on = false;
        if (k < p && k != a && k != b) {
            const bool adj_a = (g.adj[(long long)a * g.W + (k >> 5)] >> (k & 31)) & 1u;
            const bool adj_b = (g.adj[(long long)b * g.W + (k >> 5)] >> (k & 31)) & 1u;
            on = (adj_a && ca[k] == la) || (adj_b && cb[k] == lb);
        }
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (on) pool[dp + __popc(m & ((1u << lane) - 1))] = k;
        dp += __popc(m);
    }
    __syncwarp();
    return dp;
}

// The adjacent pairs (a, b), a < b, one warp each: node a of the warp by a
// grid-stride over the nodes, then a's neighbours b > a in turn.
//   mode 0: the largest pool into *maxpool (the schedule's L*)
//   mode 1: stage l -- the pool's l-subsets in lexicographic order of positions in
//           the ascending pool (side 0), each an FP64 test by the warp; the first
//           independent one is the pair's separating set: key best[e] = rank,
//           level, side, rank and the explicit set recorded (the deletion waits for
//           the end of the stage, PC-stable).
// A stage whose scheduled tests (the sum of C(|pool|, l) over the pairs reached)
// pass `budget` stops with PC_ERR_BUDGET: pairs not yet started are skipped.
__global__ void __launch_bounds__(256) pp_search_kernel(GraphDev g, TestParams tp, const double *C64, int ldc,
                                                        const int *comp, int l, int mode, int *maxpool, int mmax,
                                                        int ms, int per_warp_bytes, double budget)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem_raw + (size_t)wib * per_warp_bytes;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)mmax * ms * sizeof(double));
    int *pos = nd + mmax;
    int *pool = pos + mmax;                              // p entries
    const int p = g.p, W = g.W;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const double sq = sqrt((double)(tp.n - l - 3));
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    int best_dp = -1;
    for (long long a_ = gw; a_ < p; a_ += nw) {
        const int a = (int)a_;
        for (int w = (a + 1) >> 5; w < W; ++w) {
            unsigned bits = g.adj[(long long)a * W + w];
            if (w == ((a + 1) >> 5)) bits &= ~0u << ((a + 1) & 31);
            while (bits) {
                const int b = w * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                const int dp = pp_pool(g, comp, a, b, pool);
                if (mode == 0) {
                    best_dp = max(best_dp, dp);
                    continue;
                }
                if (dp < l || l + 2 > mmax) continue;
                const ull T = g.binom[(long long)dp * g.ldb + l];
                ull sched = 0;
                if (lane == 0) sched = atomicAdd(&g.info->total_direct, T) + T;
                sched = __shfl_sync(0xffffffffu, sched, 0);
                if (T == KEY_NONE || (double)sched > budget || g.ctr->status) {
                    if (lane == 0) atomicExch(&g.ctr->status, 6);   // PC_ERR_BUDGET
                    continue;
                }
                if (lane == 0)
                    for (int i = 0; i < l; ++i) pos[i] = i;
                __syncwarp();
                const long long e = pidx(g, a, b);
                for (ull rank = 0; rank < T; ++rank) {
                    if (lane == 0) {
                        for (int i = 0; i < l; ++i) nd[i] = pool[pos[i]];
                        nd[l] = a;
                        nd[l + 1] = b;
                    }
                    __syncwarp();
                    double r;
                    float z;
                    ++acc.tests;
                    const bool ind = warp_test<true>(nd, l + 2, l, nullptr, C64, ldc, tp, sq, (float)sq, Mbuf, ms,
                                                     acc, r, z);
                    if (ind) {
                        if (lane == 0) {
                            const ull off = atomicAdd(&g.ctr->pool_len, (ull)l);
                            g.best[e] = rank;
                            g.sep_level[e] = l;
                            g.sep_side[e] = 0;
                            g.sep_rank[e] = (long long)rank;
                            g.sep_off[e] = (long long)off;
                            if ((long long)(off + l) > g.pool_cap) {
                                g.info->pool_overflow = 1;   // the host enlarges the pool and reruns
                            } else {
                                for (int i = 0; i < l; ++i) g.pool[off + i] = nd[i];
                            }
                        }
                        __syncwarp();
                        break;
                    }
                    if (lane == 0) lex_next_dyn(pos, l, dp);
                    __syncwarp();
                }
            }
        }
    }
    if (mode == 0) {
        for (int off = 16; off > 0; off >>= 1) best_dp = max(best_dp, __shfl_xor_sync(0xffffffffu, best_dp, off));
        if (lane == 0 && best_dp >= 0) atomicMax(maxpool, best_dp);
        return;
    }
    if (lane == 0) {
        flush_acc(acc, g.ctr);
        if (acc.tests) atomicAdd(&g.ctr->tests_canonical, acc.tests);
    }
}

// End of a path-pool stage: every pair with a recorded key loses its edge.
__global__ void pp_commit_kernel(GraphDev g)
{
    const int p = g.p;
    ull removed = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)p * p;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / p), b = (int)(t - (long long)a * p);
        if (b <= a) continue;
        const long long e = pidx(g, a, b);
        if (g.best[e] == KEY_NONE) continue;
        g.best[e] = KEY_NONE;
        atomicAnd(g.adj + (long long)a * g.W + (b >> 5), ~(1u << (b & 31)));
        atomicAnd(g.adj + (long long)b * g.W + (a >> 5), ~(1u << (a & 31)));
        ++removed;
    }
    if (removed) atomicAdd(&g.ctr->edges_removed, removed);
}

cudaError_t launch_pp_components(GraphDev g, int *comp, cudaStream_t s)
{
    pp_components_kernel<<<g.p, 256, (size_t)3 * g.W * sizeof(unsigned), s>>>(g, comp);
    note_launch();
    return cudaGetLastError();
}

// per-warp shared memory of the search: the (l+2) x (l+2) FP64 matrix, the test's
// node ids, the set positions and the pool (p ids)
static size_t pp_per_warp(int mmax, int p, int &ms)
{
    ms = mmax + 1;
    return ((size_t)mmax * ms * sizeof(double) + (2 * (size_t)mmax + (size_t)p) * sizeof(int) + 15) / 16 * 16;
}

cudaError_t launch_pp_search(GraphDev g, TestParams tp, const double *C64, int ldc, const int *comp, int l,
                             int mode, int *maxpool, double budget, cudaStream_t s)
{
    const int mmax = std::max(2, std::min(DIRECT_MMAX, l + 2));
    int ms;
    const size_t per = pp_per_warp(mmax, g.p, ms);
    int wpc = 8;
    while (wpc > 1 && (size_t)wpc * per > 96 * 1024) wpc >>= 1;
    const size_t smem = (size_t)wpc * per;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(pp_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min((g.p + wpc - 1) / wpc, num_sms() * 4));
    pp_search_kernel<<<blocks, wpc * 32, smem, s>>>(g, tp, C64, ldc, comp, l, mode, maxpool, mmax, ms, (int)per,
                                                    budget);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_pp_commit(GraphDev g, cudaStream_t s)
{
    pp_commit_kernel<<<num_sms() * 4, 256, 0, s>>>(g);
    note_launch();
    return cudaGetLastError();
}

// The adjacency bitset as a p x p 0/1 byte matrix (row-major), four bytes per thread.
__global__ void expand_adj_kernel(const uint32_t *adj, int p, int W, uint8_t *out)
{
    const long long total = (long long)p * p;
    for (long long q = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 4; q < total;
         q += (long long)gridDim.x * blockDim.x * 4) {
        uint32_t word = 0;
        for (int k = 0; k < 4 && q + k < total; ++k) {
            const long long e = q + k;
            const int u = (int)(e / p), v = (int)(e - (long long)u * p);
            word |= ((adj[(long long)u * W + (v >> 5)] >> (v & 31)) & 1u) << (8 * k);
        }
        if (q + 4 <= total && ((uintptr_t)(out + q) & 3) == 0) *(uint32_t *)(out + q) = word;
        else
            for (int k = 0; k < 4 && q + k < total; ++k) out[q + k] = (uint8_t)(word >> (8 * k));
    }
}

cudaError_t launch_expand_adj(GraphDev g, uint8_t *out, cudaStream_t s)
{
    expand_adj_kernel<<<num_sms() * 8, 256, 0, s>>>(g.adj, g.p, g.W, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_init_adj(GraphDev g, cudaStream_t s)
{
    long long tot = (long long)g.p * g.W;
    init_adj_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(g); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_level_degrees(GraphDev g, cudaStream_t s)
{
    degrees_kernel<<<(g.p * 32 + 255) / 256, 256, 0, s>>>(g); note_launch();
    return cudaGetLastError();
}

// One-CTA stage kernels (head, tail): one thread per node up to 1024 (fewer warps
// at each barrier for small p), else 1024 threads with several nodes each.
static int stage_threads(int p) { return p >= 1024 ? 1024 : std::max(32, (p + 31) / 32 * 32); }

cudaError_t launch_degrees_tail(GraphDev g, TestParams tp, int cap, cudaGraphConditionalHandle hc, int use_cond,
                                StageConds sc, cudaStream_t s)
{
    degrees_tail_kernel<<<(g.p * 32 + 255) / 256, 256, 0, s>>>(g, tp, cap, hc, use_cond, sc); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tail(GraphDev g, TestParams tp, int cap, int mode, const int *stagea_singular,
                        int stagea_launched, cudaGraphConditionalHandle hc, int use_cond, StageConds sc,
                        cudaStream_t s)
{
    tail_kernel<<<1, stage_threads(g.p), 0, s>>>(g, tp, cap, mode, stagea_singular, stagea_launched, hc, use_cond, sc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_head(GraphDev g, TestParams tp, double budget, int mmax_direct, StageConds sc, cudaStream_t s)
{
    head_kernel<<<1, stage_threads(g.p), 0, s>>>(g, tp, budget, mmax_direct, sc); note_launch();
    return cudaGetLastError();
}

static void direct_shape(int mmax, int &ms, int &per_warp, int &wpc)
{
    const int m = mmax;
    ms = m + 1;
    per_warp = (int)(((size_t)m * ms * sizeof(double) + 2 * (size_t)m * sizeof(int) + 15) / 16 * 16);
    wpc = 8;
    while (wpc > 1 && (size_t)wpc * per_warp > 96 * 1024) wpc >>= 1;
}

static int pow2_floor(int x)
{
    int r = 1;
    while (r * 2 <= x) r *= 2;
    return r;
}

cudaError_t launch_ci_direct(GraphDev g, TestParams tp, int mmax, const float *C32,
                             const double *C64, int ldc, cudaStream_t s)
{
    int ms, per_warp, wpc;
    direct_shape(mmax, ms, per_warp, wpc);
    wpc = std::min(wpc, pow2_floor(std::max(1, tp.direct_warps)));
    size_t smem = (size_t)wpc * per_warp;
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    // persistent grid: as many CTAs as can be resident (shared memory bound)
    int per_sm = (int)std::max<size_t>(1, std::min<size_t>(2048 / (wpc * 32), (200 * 1024) / smem));
    int blocks = num_sms() * per_sm;
    cudaError_t e;
    if (tp.precision == 0) {
        e = cudaFuncSetAttribute(ci_direct_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_direct_kernel<true><<<blocks, wpc * 32, smem, s>>>(g, tp, mmax, C32, C64, ldc, ms, per_warp); note_launch();
    } else {
        e = cudaFuncSetAttribute(ci_direct_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_direct_kernel<false><<<blocks, wpc * 32, smem, s>>>(g, tp, mmax, C32, C64, ldc, ms, per_warp); note_launch();
    }
    return cudaGetLastError();
}

// shared memory of the staged kernel: the row corr[u, adj(u)], the start
// positions of an item's rank rounds (shorts, L <= LANE_LMAX) and the block
size_t node_smem_bytes(int dmax)
{
    return (size_t)(NODE_DMAX + (NODE_ROUNDS_MAX * LANE_LMAX + 1) / 2 + dmax * dmax) * sizeof(float);
}

// resident CTAs per SM of the staged kernel instantiation (registers and shared
// memory), looked up once per instantiation and shared-memory size
template <int LO, int HI, bool PROP>
static int node_blocks_per_sm(size_t smem)
{
    static size_t cached_smem = 0;
    static int cached = 0;
    if (cached_smem != smem) {
        int nb = 0;
        cudaFuncSetAttribute(ci_node_kernel<LO, HI, PROP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ci_node_kernel<LO, HI, PROP>, NODE_THREADS, smem) !=
                cudaSuccess || nb < 1)
            nb = 1;
        cached = nb;
        cached_smem = smem;
    }
    return cached;
}

template <int LO, int HI, bool PROP>
static void lane_launch_p(GraphDev g, TestParams tp, const float *C32, int ldc, ull *queue, ull qcap, ull *qlen,
                          cudaStream_t s)
{
    ci_lane_kernel<LO, HI, PROP><<<num_sms() * tp.lane_blocks, 256, 0, s>>>(g, tp, C32, ldc, queue, qcap, qlen);
    note_launch();
    if (LO <= PAIRWARP_LMAX && tp.pair_warp) {
        ci_pairwarp_kernel<PROP><<<num_sms() * 4, 256, 0, s>>>(g, tp, C32, ldc, queue, qcap, qlen);
        note_launch();
    }
    if (HI >= 1 && tp.node_dmax > 0) {
        const size_t smem = node_smem_bytes(tp.node_dmax);
        const int per_sm = node_blocks_per_sm<LO, HI, PROP>(smem);
        ci_node_kernel<LO, HI, PROP><<<num_sms() * per_sm, NODE_THREADS, smem, s>>>(g, tp, C32, ldc, queue, qcap,
                                                                                   qlen);
        note_launch();
    }
}

template <int LO, int HI>
static void lane_launch(GraphDev g, TestParams tp, const float *C32, int ldc, ull *queue, ull qcap, ull *qlen,
                        bool prop, cudaStream_t s)
{
    if (prop) lane_launch_p<LO, HI, true>(g, tp, C32, ldc, queue, qcap, qlen, s);
    else lane_launch_p<LO, HI, false>(g, tp, C32, ldc, queue, qcap, qlen, s);
}

cudaError_t launch_ci_lane(GraphDev g, TestParams tp, const float *C32, const double *C64, int ldc,
                           unsigned long long *queue, unsigned long long qcap, unsigned long long *qlen,
                           int range, bool prop, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(qlen, 0, sizeof(ull), s);
    if (e != cudaSuccess) return e;
    if (range < 0 || range == 0) lane_launch<0, 2>(g, tp, C32, ldc, queue, qcap, qlen, prop, s);
    if (range < 0 || range == 1) lane_launch<3, 4>(g, tp, C32, ldc, queue, qcap, qlen, prop, s);
    if (range < 0 || range == 2) lane_launch<5, 6>(g, tp, C32, ldc, queue, qcap, qlen, prop, s);
    if (range < 0 || range == 3) lane_launch<7, 8>(g, tp, C32, ldc, queue, qcap, qlen, prop, s);
    if (range < 0 || range == 4) lane_launch<9, 10>(g, tp, C32, ldc, queue, qcap, qlen, prop, s);
    if (range < 0 || range == 5) lane_launch<11, 12>(g, tp, C32, ldc, queue, qcap, qlen, prop, s);
    int ms, per_warp, wpc;
    direct_shape(LANE_LMAX + 2, ms, per_warp, wpc);
    size_t smem = (size_t)wpc * per_warp;
    e = cudaFuncSetAttribute(ci_redecide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (tp.lazy && tp.c64_list && tp.pair_seen) {
        // the FP64 entries the queued tests need, formed in parallel before the FP64 pass
        e = cudaMemsetAsync(tp.c64_list_len, 0, sizeof(ull), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(tp.pair_seen, 0, tp.pair_seen_bytes, s);
        if (e != cudaSuccess) return e;
        c64_collect_kernel<<<num_sms() * 4, 256, 0, s>>>(g, tp, queue, qlen, qcap); note_launch();
        c64_fill_kernel<<<num_sms() * 4, 256, 0, s>>>(g, tp, const_cast<double *>(C64), ldc); note_launch();
    }
    ci_redecide_kernel<<<num_sms() * 4, wpc * 32, smem, s>>>(g, tp, C64, ldc, queue, qlen, qcap, ms, per_warp); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ci_complement(GraphDev g, TestParams tp, cudaStream_t s)
{
    ci_complement_kernel<<<num_sms() * 2, 128, 0, s>>>(g, tp); note_launch();
    return cudaGetLastError();
}

static size_t prec_smem_bytes(int p);

cudaError_t launch_prec_update(GraphDev g, TestParams tp, const double *C64, int ldc, cudaStream_t s)
{
    const size_t smem = prec_smem_bytes(g.p);
    cudaError_t e = cudaFuncSetAttribute(prec_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    prec_update_kernel<<<dim3(g.p, PREC_CHUNKS), 512, smem, s>>>(g, tp, C64, ldc); note_launch();
    return cudaGetLastError();
}

static size_t prec_smem_bytes(int p)
{
    const int mmax = std::min(p + 1, PREC_MAX);
    const size_t build = ((size_t)mmax * mmax + (size_t)mmax) * sizeof(double);
    // downdate: L (nr x nr), 1/D (nr) and the staged rows of R at the kept columns (nr x nt)
    const size_t down = ((size_t)PREC_RMAX * PREC_RMAX + (size_t)PREC_RMAX + (size_t)PREC_RMAX * mmax) *
                        sizeof(double);
    return std::max(build, down);
}

cudaError_t launch_prec_seed(GraphDev g, const double *P, int ldp, cudaStream_t s)
{
    if (g.p > PREC_MAX) return cudaErrorInvalidValue;
    prec_seed_kernel<<<g.p, 256, 0, s>>>(g, P, ldp); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stage_loop(GraphDev g, TestParams tp, const float *C32, const double *C64, int ldc,
                              double budget, int cap, int pre, cudaStream_t s)
{
    if (g.p > LOOP_PMAX) return cudaErrorInvalidValue;
    // the downdates' and builds' block, or the direct tests' warp buffers
    const size_t smem = std::max(prec_smem_bytes(g.p), (size_t)(LOOP_THREADS / 32) * loop_direct_bytes());
    cudaError_t e = cudaFuncSetAttribute(stage_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_loop_kernel, LOOP_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int grid = num_sms() * std::min(per_sm, 2);   // every CTA resident (cooperative launch)
    // a node's kept rows over PREC_CHUNKS CTAs (consecutive items: different SMs), so
    // that the FP64 work of a large downdate is spread
    int chunks = PREC_CHUNKS;
    void *args[] = {&g, &tp, (void *)&C32, (void *)&C64, &ldc, &budget, &cap, &chunks, &pre};
    e = cudaLaunchCooperativeKernel((const void *)stage_loop_kernel, dim3(grid), dim3(LOOP_THREADS), args, smem, s);
    note_launch();
    return e;
}

cudaError_t launch_commit(GraphDev g, long long n_opairs_cap, int l_fixed, int explicit_sets,
                          cudaStream_t s)
{
    long long cap = n_opairs_cap > 0 ? n_opairs_cap : 1;
    int blocks = (int)std::min<long long>((cap + 255) / 256, (long long)num_sms() * 8);
    commit_kernel<<<blocks, 256, 0, s>>>(g, l_fixed, explicit_sets, explicit_sets); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_reverify(GraphDev g, TestParams tp, const float *C32, const double *C64, int ldc, int lmax,
                            cudaStream_t s)
{
    // one warp's matrix holds the sets of the largest stage the search ran
    // (sets of more than 128 members are not re-tested)
    int mmax = std::max(2, std::min(std::min(g.p, 130), lmax + 2));
    int ms, per_warp, wpc;
    direct_shape(mmax, ms, per_warp, wpc);
    size_t smem = (size_t)wpc * per_warp;
    cudaError_t e = cudaFuncSetAttribute(reverify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    reverify_kernel<<<num_sms() * 2, wpc * 32, smem, s>>>(g, tp, C32, C64, ldc, mmax, ms, per_warp); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ci_list(const int *ij, const int *S, int l, long long b, const float *C32,
                           const double *C64, int ldc, int p, TestParams tp, double *r_out,
                           uint8_t *indep_out, float *z_out, DevCounters *ctr, const int *blk_lo,
                           const int *blk_hi, cudaStream_t s)
{
    int ms, per_warp, wpc;
    direct_shape(l + 2, ms, per_warp, wpc);
    size_t smem = (size_t)wpc * per_warp;
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    long long warps = b;
    int blocks = (int)std::min<long long>((warps + wpc - 1) / wpc, (long long)num_sms() * 16);
    if (blocks < 1) blocks = 1;
    cudaError_t e;
    if (tp.precision == 0) {
        e = cudaFuncSetAttribute(ci_list_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_list_kernel<true><<<blocks, wpc * 32, smem, s>>>(ij, S, l, b, C32, C64, ldc, p, tp, r_out,
                                                           indep_out, z_out, ctr, blk_lo, blk_hi, ms, per_warp); note_launch();
    } else {
        e = cudaFuncSetAttribute(ci_list_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_list_kernel<false><<<blocks, wpc * 32, smem, s>>>(ij, S, l, b, C32, C64, ldc, p, tp, r_out,
                                                            indep_out, z_out, ctr, blk_lo, blk_hi, ms, per_warp); note_launch();
    }
    return cudaGetLastError();
}

}  // namespace fpc
