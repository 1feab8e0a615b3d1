// orient.cu -- Phase II of Algorithm 1 (Algorithm 2 leaves it unchanged,
// Sec. 3.3): the skeleton is oriented from the separation sets.  First the
// unshielded colliders (i - k - j, i and j non-adjacent, k not in S(i,j):
// i -> k <- j), then rules R1-R4 repeated until none orients an edge.
//
// Order-free reading (the listing orders neither loop): every collider marks
// both of its edges at once, and the rules run in rounds -- each round tests
// every undirected edge against the marks of the previous round and applies all
// orientations it finds together.  An edge marked from both ends (two colliders,
// or both directions in one round) is bidirected.  R4 is read with X_k and X_j
// non-adjacent (the printed "X_k and X_l" contradicts its own X_k -> X_l).
//
// Marks are per-node bitsets over the instance's nodes:
//   AH[x] = {y : the edge {x,y} has an arrowhead at y}
//   AT[x] = {y : the edge {x,y} has an arrowhead at x}   (the transpose of AH)
// so that, with ADJ the skeleton's rows,
//   parents PA[x] = ADJ & AT & ~AH, children CH[x] = ADJ & AH & ~AT,
//   undirected UN[x] = ADJ & ~AH & ~AT,
// and each rule is a few word operations per 32 candidate nodes.
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>

namespace fpc {

namespace {

__device__ __forceinline__ void inst_words(const GraphDev &g, int x, int &lo, int &hi, int &w0, int &w1)
{
    lo = g.blk_lo ? g.blk_lo[x] : 0;
    hi = g.blk_hi ? g.blk_hi[x] : g.p;
    w0 = lo >> 5;
    w1 = (hi - 1) >> 5;
}

// Colliders: CTA i takes the nodes j > i of its instance, one warp per j; the
// lanes scan the words of ADJ[i] & ADJ[j] and look each common neighbour up in
// the recorded set (ascending) by binary search.
__global__ void __launch_bounds__(256) orient_colliders_kernel(GraphDev g, uint32_t *ah, uint32_t *at)
{
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int W = g.W;
    int lo, hi, w0, w1;
    inst_words(g, i, lo, hi, w0, w1);
    const uint32_t *Ai = g.adj + (long long)i * W;
    for (int j = i + 1 + wid; j < hi; j += nw) {
        if ((Ai[j >> 5] >> (j & 31)) & 1u) continue;         // adjacent: no triple
        const long long e = pidx(g, i, j);
        const int len = g.sep_level[e];
        const long long off = g.sep_off[e];
        if (len < 0 || off < 0) continue;                    // no record, or every other node (l = p-2)
        const int *S = g.pool + off;
        const uint32_t *Aj = g.adj + (long long)j * W;
        for (int w = w0 + lane; w <= w1; w += 32) {
            uint32_t m = Ai[w] & Aj[w];
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int k = (w << 5) + b;
                int l0 = 0, l1 = len;
                while (l0 < l1) {
                    const int mid = (l0 + l1) >> 1;
                    if (S[mid] < k) l0 = mid + 1;
                    else l1 = mid;
                }
                if (l0 < len && S[l0] == k) continue;        // k separates i and j: no collider
                atomicOr(ah + (long long)i * W + w, 1u << b);
                atomicOr(ah + (long long)j * W + w, 1u << b);
                atomicOr(at + (long long)k * W + (i >> 5), 1u << (i & 31));
                atomicOr(at + (long long)k * W + (j >> 5), 1u << (j & 31));
            }
        }
    }
}

// Is one of R1-R4 orienting the undirected edge a - b into a -> b?  Called by a
// whole warp (lanes split the words of the instance); the result is uniform.
__device__ bool rule_orients(const GraphDev &g, const uint32_t *ah, const uint32_t *at, int a, int b, int w0,
                             int w1)
{
    const int lane = threadIdx.x & 31, W = g.W;
    const uint32_t *Aa = g.adj + (long long)a * W, *Ab = g.adj + (long long)b * W;
    const uint32_t *Ha = ah + (long long)a * W, *Ta = at + (long long)a * W;
    const uint32_t *Hb = ah + (long long)b * W, *Tb = at + (long long)b * W;
    const int wb = b >> 5;
    const uint32_t bbit = 1u << (b & 31);
    // R1: some c -> a with c and b non-adjacent;  R2: a -> c -> b
    bool f = false;
    for (int w = w0 + lane; w <= w1; w += 32) {
        const uint32_t pa = Aa[w] & Ta[w] & ~Ha[w], cha = Aa[w] & Ha[w] & ~Ta[w];
        const uint32_t pb = Ab[w] & Tb[w] & ~Hb[w];
        uint32_t r1 = pa & ~Ab[w];
        if (w == wb) r1 &= ~bbit;
        f |= r1 != 0u || (cha & pb) != 0u;
    }
    if (__any_sync(0xffffffffu, f)) return true;
    // R3: a - c -> b and a - d -> b with c, d non-adjacent;
    // R4: a - c -> d -> b with c and b non-adjacent
    for (int w = w0; w <= w1; ++w) {                         // warp-uniform
        const uint32_t una = Aa[w] & ~Ha[w] & ~Ta[w];
        uint32_t C = una & Ab[w] & Tb[w] & ~Hb[w];
        uint32_t K = una & ~Ab[w];
        if (w == wb) K &= ~bbit;
        while (C) {
            const int cb = __ffs(C) - 1;
            C &= C - 1;
            const int c = (w << 5) + cb;
            const uint32_t *Ac = g.adj + (long long)c * W;
            bool h = false;
            for (int v = w0 + lane; v <= w1; v += 32) {
                uint32_t x = Aa[v] & ~Ha[v] & ~Ta[v] & Ab[v] & Tb[v] & ~Hb[v] & ~Ac[v];
                if (v == w) x &= ~(1u << cb);
                h |= x != 0u;
            }
            if (__any_sync(0xffffffffu, h)) return true;
        }
        while (K) {
            const int cb = __ffs(K) - 1;
            K &= K - 1;
            const int c = (w << 5) + cb;
            const uint32_t *Ac = g.adj + (long long)c * W, *Hc = ah + (long long)c * W, *Tc = at + (long long)c * W;
            bool h = false;
            for (int v = w0 + lane; v <= w1; v += 32)
                h |= (Ac[v] & Hc[v] & ~Tc[v] & Ab[v] & Tb[v] & ~Hb[v]) != 0u;
            if (__any_sync(0xffffffffu, h)) return true;
        }
    }
    return false;
}

// One round: a warp per node a, over the undirected edges a - b of the marks
// (ah, at); orientations go to (ah2, at2), which start as copies.
__global__ void __launch_bounds__(256) orient_rules_kernel(GraphDev g, const uint32_t *ah, const uint32_t *at,
                                                           uint32_t *ah2, uint32_t *at2, int *changed)
{
    const int lane = threadIdx.x & 31, W = g.W;
    const long long nwg = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long aa = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; aa < g.p; aa += nwg) {
        const int a = (int)aa;
        int lo, hi, w0, w1;
        inst_words(g, a, lo, hi, w0, w1);
        const uint32_t *Aa = g.adj + (long long)a * W, *Ha = ah + (long long)a * W, *Ta = at + (long long)a * W;
        for (int w = w0; w <= w1; ++w) {
            uint32_t un = Aa[w] & ~Ha[w] & ~Ta[w];
            while (un) {
                const int bb = __ffs(un) - 1;
                un &= un - 1;
                const int b = (w << 5) + bb;
                if (rule_orients(g, ah, at, a, b, w0, w1) && lane == 0) {
                    atomicOr(ah2 + (long long)a * W + w, 1u << bb);
                    atomicOr(at2 + (long long)b * W + (a >> 5), 1u << (a & 31));
                    *changed = 1;
                }
            }
        }
    }
}

// Codes per ordered pair: 0 no edge, 1 a - b, 2 a -> b, 3 a <- b, 4 a <-> b.
__global__ void orient_codes_kernel(GraphDev g, const uint32_t *ah, const uint32_t *at, int8_t *out)
{
    const long long p = g.p, tot = p * p;
    const int W = g.W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / p), b = (int)(e - (long long)a * p);
        const long long wi = (long long)a * W + (b >> 5);
        const uint32_t bit = 1u << (b & 31);
        int8_t c = 0;
        if (a != b && (g.adj[wi] & bit)) {
            const bool h = ah[wi] & bit, t = at[wi] & bit;
            c = (int8_t)(h ? (t ? 4 : 2) : (t ? 3 : 1));
        }
        out[e] = c;
    }
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

}  // namespace

cudaError_t launch_orient_colliders(GraphDev g, uint32_t *ah, uint32_t *at, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ah, 0, (size_t)g.p * g.W * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(at, 0, (size_t)g.p * g.W * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    orient_colliders_kernel<<<g.p, 256, 0, s>>>(g, ah, at); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_orient_round(GraphDev g, const uint32_t *ah, const uint32_t *at, uint32_t *ah2, uint32_t *at2,
                                int *changed, cudaStream_t s)
{
    const size_t bytes = (size_t)g.p * g.W * sizeof(uint32_t);
    cudaError_t e = cudaMemcpyAsync(ah2, ah, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(at2, at, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(changed, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<long long>(((long long)g.p * 32 + 255) / 256, (long long)sm_count() * 8);
    orient_rules_kernel<<<blocks, 256, 0, s>>>(g, ah, at, ah2, at2, changed); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_orient_codes(GraphDev g, const uint32_t *ah, const uint32_t *at, int8_t *out, cudaStream_t s)
{
    const long long tot = (long long)g.p * g.p;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, (long long)sm_count() * 16);
    orient_codes_kernel<<<blocks, 256, 0, s>>>(g, ah, at, out); note_launch();
    return cudaGetLastError();
}

}  // namespace fpc
