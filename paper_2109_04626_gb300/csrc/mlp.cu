// mlp.cu -- the conditioning-set proposal network (not in the paper): a
// member score s(u, v, k) for every candidate k of an ordered pair (u, v) at
// stage l, used to enumerate the likeliest separating sets first.
//
//   h1 = relu(W1 x + b1)  (16 -> 128),  h2 = relu(W2 h1 + b2)  (128 -> 128),
//   s = w3 . h2 + b3;     training loss: mean BCE(sigmoid(s), y).
//
// Forward on the tensor cores (tcgen05, BF16 operands, FP32 accumulators in
// TMEM): the CTA writes a 128-row tile of features into a SWIZZLE_128B K-major
// shared tile, one thread issues D1 = X W1^T (K = 16), the epilogue applies
// bias + ReLU and writes h1 (BF16) into the A operand of D2 = h1 W2^T
// (K = 128), and the second epilogue reduces h2 against w3.  Backward and Adam
// run on the CUDA cores in FP32 from the saved activations.
#include "internal.h"
#include "device_util.cuh"
#include "tc_util.cuh"

#include <cuda_bf16.h>

namespace fpc {

constexpr int NF = 16, NH = 128;
constexpr int NPARAM = NH * NF + NH + NH * NH + NH + NH + 1;   // 18817
constexpr int OFF_W1 = 0, OFF_B1 = NH * NF, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
constexpr int T_ROWS = 128;
constexpr int W1_TILE = 128 * 128;            // bytes: 128 rows x 64 bf16 (features in the first 16)
constexpr int W2_TILE = 128 * 128;            // bytes per 64-wide K tile
constexpr int A1_BYTES = 128 * 128;
constexpr int A2_BYTES = 2 * 128 * 128;
constexpr int MLP_SMEM = W1_TILE + 2 * W2_TILE + A1_BYTES + A2_BYTES + 1024;

// byte offset of element (row, col) of a 128-byte-row K-major tile with the
// 128-byte swizzle: the 16-byte chunk index is XORed with row mod 8
__device__ __forceinline__ int sw128_off(int row, int col_bf16)
{
    const int chunk = col_bf16 >> 3, within = col_bf16 & 7;
    return row * 128 + (((chunk ^ (row & 7)) << 4) | (within << 1));
}

// Member features of candidate k for the ordered pair (u, v) at stage l, from
// the FP32 correlation matrix: marginal correlations, first-order partial
// correlations, the first-order test statistic relative to the threshold,
// and the stage shape.
__device__ __forceinline__ void member_features_of(float cuv, float cuk, float cvk, int l, int d, float sqn_over_q,
                                                   float *f)
{
    const float e = 1e-6f;
    const float ruv_k = (cuv - cuk * cvk) * rsqrtf(fmaxf((1.f - cuk * cuk) * (1.f - cvk * cvk), e));
    const float ruk_v = (cuk - cuv * cvk) * rsqrtf(fmaxf((1.f - cuv * cuv) * (1.f - cvk * cvk), e));
    const float rvk_u = (cvk - cuv * cuk) * rsqrtf(fmaxf((1.f - cuv * cuv) * (1.f - cuk * cuk), e));
    f[0] = fabsf(cuv);
    f[1] = fabsf(cuk);
    f[2] = fabsf(cvk);
    f[3] = fabsf(cuk * cvk);
    f[4] = fabsf(ruv_k);
    f[5] = fabsf(ruk_v);
    f[6] = fabsf(rvk_u);
    f[7] = fminf(sqn_over_q * fabsf(ruv_k), 4.f);
    f[8] = fminf(sqn_over_q * fabsf(cuv), 4.f);
    f[9] = fminf(fmaxf(sqn_over_q * (fabsf(cuv) - fabsf(ruv_k)), -4.f), 4.f);
    f[10] = d > 0 ? (float)l / (float)d : 0.f;
    f[11] = log2f((float)d + 1.f) * 0.125f;
    f[12] = (float)l * (1.f / 16.f);
    f[13] = (cuv * cuk * cvk > 0.f) ? 1.f : 0.f;
    f[14] = 1.f;
    f[15] = 0.f;
}

__device__ __forceinline__ void member_features(const float *C, int ldc, const long long *prow, int u, int v, int k,
                                                int l, int d, float sqn_over_q, float *f)
{
    member_features_of(C[cidx(prow, ldc, u, v)], C[cidx(prow, ldc, u, k)], C[cidx(prow, ldc, v, k)], l, d,
                       sqn_over_q, f);
}

// Packs the FP32 master parameters into the swizzled BF16 B-operand tiles of
// W1 (128 x 64, features zero-padded) and W2 (two 128 x 64 K tiles).
// ... and W2 transposed (rows i, K = o) as the B operand of the backward
// product dL/dh1 = dL/da2 W2, after the forward's tiles.
__global__ void mlp_pack_kernel(const float *theta, uint8_t *wpack)
{
    const int o = blockIdx.x;            // output unit (row of the B operand)
    for (int c = threadIdx.x; c < 64; c += blockDim.x) {
        const float w = c < NF ? theta[OFF_W1 + o * NF + c] : 0.f;
        *(__nv_bfloat16 *)(wpack + sw128_off(o, c)) = __float2bfloat16_rn(w);
    }
    for (int c = threadIdx.x; c < NH; c += blockDim.x) {
        const int t = c >> 6;
        const __nv_bfloat16 w = __float2bfloat16_rn(theta[OFF_W2 + o * NH + c]);
        *(__nv_bfloat16 *)(wpack + W1_TILE + t * W2_TILE + sw128_off(o, c & 63)) = w;
        // element (i = c, K = o) of W2^T
        *(__nv_bfloat16 *)(wpack + W1_TILE + 2 * W2_TILE + (o >> 6) * W2_TILE + sw128_off(c, o & 63)) = w;
    }
}

// Where the rows of a forward pass come from.
struct MlpRows {
    // explicit features (R x 16 FP32), or ...
    const float *feats;
    long long R;
    // ... the candidates of the current stage: node u owns deg_u * (deg_u - 1)
    // rows starting at row_off[u] (pair j, candidate position x)
    const GraphDev *gp;
    const unsigned long long *row_off;
    const float *C32;
    int ldc;
    float sqn_over_q;
    const long long *nvec;   // batched problems: per-node samples (sqrt(n_u)/q per row)
    float inv_q;
};

// A candidate row of the current stage: node u (tracked by the caller, which
// walks it forward over consecutive rows), the pair's v, the candidate k.
struct RowRef {
    int u, v, k, d;
    bool ok;
};

__device__ __forceinline__ RowRef locate_row(const MlpRows &R, const GraphDev &g, long long row, long long nrows,
                                             int &ucur)
{
    RowRef r{0, 0, 0, 0, row < nrows};
    if (!r.ok) return r;
    while ((long long)R.row_off[ucur + 1] <= row) ++ucur;
    const int u = ucur, d = g.deg[u] - 1;
    const long long w = row - (long long)R.row_off[u];
    const int j = (int)(w / d), x = (int)(w - (long long)j * d);
    const int *nb = g.nbr + nidx(g, u);
    r.u = u;
    r.d = d;
    r.v = nb[j];
    r.k = nb[x + (x >= j)];
    return r;
}

// The correlations a row's features need (loaded one tile ahead of use).
struct RowVals {
    float cuv, cuk, cvk, sq;
    int d;
    bool ok;
};

__device__ __forceinline__ RowVals fetch_row(const MlpRows &R, const GraphDev &g, const RowRef &r)
{
    RowVals x{0.f, 0.f, 0.f, 0.f, r.d, r.ok};
    if (!r.ok) return x;
    x.cuv = R.C32[cidx(g.prow, R.ldc, r.u, r.v)];
    x.cuk = R.C32[cidx(g.prow, R.ldc, r.u, r.k)];
    x.cvk = R.C32[cidx(g.prow, R.ldc, r.v, r.k)];
    x.sq = R.nvec ? sqrtf((float)R.nvec[r.u]) * R.inv_q : R.sqn_over_q;
    return x;
}

// Forward pass over rows [0, R): scores s, and for training h1 (BF16), h2 (FP32).
// Each CTA takes a contiguous range of 128-row tiles.  For the rows of the
// current stage the next tile's indices are located while the first product
// runs and its correlations are requested before the second product's wait,
// so the gathers overlap the tensor-core work and the epilogues.
__global__ void __launch_bounds__(128, 2) mlp_forward_kernel(MlpRows rows, GraphDev g, const uint8_t *wpack,
                                                             const float *theta, float *scores,
                                                             __nv_bfloat16 *h1_out, float *h2_out, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sW1 = smem, *sW2 = smem + W1_TILE, *sA1 = sW2 + 2 * W2_TILE, *sA2 = sA1 + A1_BYTES;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float b1[NH], b2[NH], w3[NH];
    __shared__ float b3;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (!rows.feats && (g.info->done || g.info->halt)) return;
    const long long R = rows.feats ? rows.R : (long long)rows.row_off[g.p];
    const long long ntiles = (R + T_ROWS - 1) / T_ROWS;
    const long long tb = ntiles * blockIdx.x / gridDim.x, te = ntiles * (blockIdx.x + 1) / gridDim.x;
    // a stage without proposal rows (or a CTA without tiles) leaves before
    // loading the weights and allocating tensor memory
    if (tb >= te) return;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights (pre-swizzled) and vectors into shared memory; A1 zero-filled once
    for (int i = tid; i < (W1_TILE + 2 * W2_TILE) / 16; i += blockDim.x)
        ((uint4 *)smem)[i] = ((const uint4 *)wpack)[i];
    for (int i = tid; i < A1_BYTES / 16; i += blockDim.x) ((uint4 *)sA1)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < NH; i += blockDim.x) {
        b1[i] = theta[OFF_B1 + i];
        b2[i] = theta[OFF_B2 + i];
        w3[i] = theta[OFF_W3 + i];
    }
    if (tid == 0) b3 = theta[OFF_B3];
    if (warp == 0) tc_alloc(&tmem_base, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base, d1 = tmem, d2 = tmem + 128;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
    const int l = rows.feats ? 0 : g.info->l;
    unsigned phase = 0;
    bool ok = true;
    // the row this thread feeds into the first tile, located and fetched
    int ucur = 0;
    RowVals cur{};
    if (!rows.feats) {
        const long long r0 = tb * T_ROWS + tid;
        if (r0 < R) ucur = (int)(upper_bound_dev(rows.row_off, (long long)g.p + 1, (unsigned long long)r0) - 1);
        cur = fetch_row(rows, g, locate_row(rows, g, r0, R, ucur));
    }
    for (long long t = tb; t < te && ok; ++t) {
        const long long row = t * T_ROWS + tid;
        float f[NF];
        if (rows.feats) {
            if (row < R)
#pragma unroll
                for (int i = 0; i < NF; ++i) f[i] = rows.feats[row * NF + i];
            else
#pragma unroll
                for (int i = 0; i < NF; ++i) f[i] = 0.f;
        } else if (cur.ok) {
            member_features_of(cur.cuv, cur.cuk, cur.cvk, l, cur.d, cur.sq, f);
        } else {
#pragma unroll
            for (int i = 0; i < NF; ++i) f[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < NF; ++i) *(__nv_bfloat16 *)(sA1 + sw128_off(tid, i)) = __float2bfloat16_rn(f[i]);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            tc_mma(d1, sw128_desc(smem_u32(sA1)), sw128_desc(smem_u32(sW1)), idesc, 0u);
            tc_commit(&bar);
        }
        __syncwarp();
        // the next tile's row: indices now, correlations before the second wait
        RowRef nxt{0, 0, 0, 0, false};
        if (!rows.feats && t + 1 < te) nxt = locate_row(rows, g, row + T_ROWS, R, ucur);
        ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        tc_fence_after();
        // epilogue 1: h1 = relu(D1 + b1) -> BF16 into the A operand of layer 2
#pragma unroll 1
        for (int c0 = 0; c0 < NH; c0 += 32) {
            float v[32];
            tc_ld_32cols(d1 + lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // 8 columns: one 16-byte chunk of the swizzled row (and of h1's row)
                __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) hb[j] = __float2bfloat16_rn(fmaxf(v[q * 8 + j] + b1[c0 + q * 8 + j], 0.f));
                const int c = c0 + q * 8;
                *(uint4 *)(sA2 + (c >> 6) * (128 * 128) + sw128_off(tid, c & 63)) = *(const uint4 *)hb;
                if (h1_out && row < R) *(uint4 *)(h1_out + row * NH + c) = *(const uint4 *)hb;
            }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int tt = 0; tt < 2; ++tt)
                for (int ks = 0; ks < 4; ++ks)
                    tc_mma(d2, sw128_desc(smem_u32(sA2 + tt * 128 * 128) + ks * 32),
                           sw128_desc(smem_u32(sW2 + tt * W2_TILE) + ks * 32), idesc, (tt | ks) ? 1u : 0u);
            tc_commit(&bar);
        }
        __syncwarp();
        if (!rows.feats && t + 1 < te) cur = fetch_row(rows, g, nxt);
        ok = ok && mbar_wait(&bar, phase);
        phase ^= 1u;
        tc_fence_after();
        // epilogue 2: s = w3 . relu(D2 + b2) + b3
        float s = b3;
#pragma unroll 1
        for (int c0 = 0; c0 < NH; c0 += 32) {
            float v[32];
            tc_ld_32cols(d2 + lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float h = fmaxf(v[j] + b2[c0 + j], 0.f);
                s = fmaf(w3[c0 + j], h, s);
                if (h2_out && row < R) h2_out[row * NH + c0 + j] = h;
            }
        }
        if (row < R) scores[row] = s;
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 256);
    if (!ok && tid == 0) atomicExch(err, 7);   // a bounded wait expired
}

// Backward pass for rows [0, R) of a batch: per-CTA FP32 partial gradients in
// registers, added into grad (atomics once per CTA).  Uses the activations the
// forward pass saved (h1 BF16 as consumed by layer 2, h2 FP32) and the BF16
// weights the forward pass used.
__global__ void __launch_bounds__(256) mlp_backward_kernel(const float *feats, const float *labels,
                                                           const float *scores, const __nv_bfloat16 *h1,
                                                           const float *h2, long long R, float inv_b,
                                                           const float *theta, float *grad, double *loss)
{
    extern __shared__ float bsm[];
    float(*sdh2)[NH + 1] = (float(*)[NH + 1])bsm;                       // dL/dh2 (masked) of the tile
    float(*sh1)[NH + 1] = (float(*)[NH + 1])(bsm + T_ROWS * (NH + 1));   // h1, then dL/dh1
    float(*sW2)[NH + 1] = (float(*)[NH + 1])(bsm + 2 * T_ROWS * (NH + 1)); // W2 rounded to BF16
    float(*sx)[NF] = (float(*)[NF])(bsm + 2 * T_ROWS * (NH + 1) + NH * (NH + 1));
    float *sds = bsm + 2 * T_ROWS * (NH + 1) + NH * (NH + 1) + T_ROWS * NF;
    const int tid = threadIdx.x;
    for (int e = tid; e < NH * NH; e += blockDim.x)
        sW2[e / NH][e % NH] = __bfloat162float(__float2bfloat16_rn(theta[OFF_W2 + e]));
    // per-thread partials: dW2 entries (o, i) with o = tid/2, i in the half tid&1
    float gW2[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) gW2[i] = 0.f;
    float gW1[8], gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) gW1[i] = 0.f;
    double lsum = 0.0;
    const int o = tid >> 1, ih = (tid & 1) * 64;
    __syncthreads();
    for (long long t0 = (long long)blockIdx.x * T_ROWS; t0 < R; t0 += (long long)gridDim.x * T_ROWS) {
        const int nr = (int)(R - t0 < T_ROWS ? R - t0 : T_ROWS);
        for (int r = tid; r < T_ROWS; r += blockDim.x) {
            float ds = 0.f;
            if (r < nr) {
                const float s = scores[t0 + r], y = labels[t0 + r];
                ds = (1.f / (1.f + __expf(-s)) - y) * inv_b;
                lsum += (double)(fmaxf(s, 0.f) + log1pf(__expf(-fabsf(s))) - y * s);
            }
            sds[r] = ds;
        }
        for (int e = tid; e < T_ROWS * NH; e += blockDim.x) {
            const int r = e / NH, c = e % NH;
            float hv1 = 0.f, d2 = 0.f;
            if (r < nr) {
                hv1 = __bfloat162float(h1[(t0 + r) * NH + c]);
                const float hv2 = h2[(t0 + r) * NH + c];
                d2 = hv2 > 0.f ? 1.f : 0.f;
            }
            sh1[r][c] = hv1;
            sdh2[r][c] = d2;                     // mask for now; scaled below
        }
        for (int e = tid; e < T_ROWS * NF; e += blockDim.x) {
            const int r = e / NF, c = e % NF;
            sx[r][c] = r < nr ? __bfloat162float(__float2bfloat16_rn(feats[(t0 + r) * NF + c])) : 0.f;
        }
        __syncthreads();
        // dW3 / db3 (threads 0..127 own one unit each) and the masked dh2
        for (int e = tid; e < T_ROWS * NH; e += blockDim.x) {
            const int r = e / NH, c = e % NH;
            sdh2[r][c] *= sds[r] * theta[OFF_W3 + c];
        }
        if (tid < NH) {
            float a = 0.f;
            for (int r = 0; r < nr; ++r) a = fmaf(sds[r], h2[(t0 + r) * NH + tid], a);
            gw3 += a;
        }
        if (tid == 0)
            for (int r = 0; r < nr; ++r) gb3 += sds[r];
        __syncthreads();
        // dW2[o][i] += sum_r dh2[r][o] h1[r][i]; db2[o]
#pragma unroll 4
        for (int r = 0; r < nr; ++r) {
            const float a = sdh2[r][o];
#pragma unroll
            for (int i = 0; i < 64; ++i) gW2[i] = fmaf(a, sh1[r][ih + i], gW2[i]);
        }
        if ((tid & 1) == 0)
            for (int r = 0; r < nr; ++r) gb2 += sdh2[r][o];
        __syncthreads();
        // dh1[r][i] = sum_o dh2[r][o] W2[o][i], masked by h1 > 0 (stored into sh1)
        for (int e = tid; e < T_ROWS * NH; e += blockDim.x) {
            const int r = e / NH, i = e % NH;
            float a = 0.f;
            if (r < nr && sh1[r][i] > 0.f)
                for (int q = 0; q < NH; ++q) a = fmaf(sdh2[r][q], sW2[q][i], a);
            sh1[r][i] = a;                   // sh1 now holds dh1 (masked); each (r, i) is read and
                                             // written by the same thread only
        }
        __syncthreads();
        // dW1[i][f] += sum_r dh1[r][i] x[r][f]; db1[i]   (thread -> unit i = tid/2, 8 features)
        {
            const int iu = tid >> 1, f0 = (tid & 1) * 8;
            for (int r = 0; r < nr; ++r) {
                const float a = sh1[r][iu];
#pragma unroll
                for (int q = 0; q < 8; ++q) gW1[q] = fmaf(a, sx[r][f0 + q], gW1[q]);
                if ((tid & 1) == 0) gb1 += a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 64; ++i) atomicAdd(&grad[OFF_W2 + o * NH + ih + i], gW2[i]);
    if ((tid & 1) == 0) atomicAdd(&grad[OFF_B2 + o], gb2);
    {
        const int iu = tid >> 1, f0 = (tid & 1) * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) atomicAdd(&grad[OFF_W1 + iu * NF + f0 + q], gW1[q]);
        if ((tid & 1) == 0) atomicAdd(&grad[OFF_B1 + iu], gb1);
    }
    if (tid < NH) atomicAdd(&grad[OFF_W3 + tid], gw3);
    if (tid == 0) atomicAdd(&grad[OFF_B3], gb3);
    if (loss) {
        // block-level sum of the loss terms
        __shared__ double red[256];
        red[tid] = lsum;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        if (tid == 0) atomicAdd(loss, red[0]);
    }
}

// Backward pass on the tensor cores: BF16 operands, FP32 accumulators in TMEM.
// Per 128-row tile of the batch (thread t owns row t):
//   ds = (sigmoid(s) - y) / B,  dL/da2 = ds w3 (h2 > 0)            (FP32, then BF16)
//   dL/dh1 = dL/da2 W2  -> masked by h1 > 0                         (tensor core, then BF16)
//   dW2 += (dL/da2)^T h1,  dW1 += (dL/da1)^T x                      (tensor core, over the tiles)
// The products contract over the batch rows for the weight gradients, so their
// operands are written transposed (unit-major, rows along K) into K-major tiles.
// db2, db1 sum the BF16 signals the products read; dw3, db3 and the loss stay in
// FP32 from the saved h2.  dW2 and dW1 accumulate in TMEM across the CTA's tiles
// and are added into grad once per CTA.
constexpr int BWD_SMEM = 2 * W2_TILE + 4 * 2 * W2_TILE + 2 * 16 * 128 + 1024;

__global__ void __launch_bounds__(128, 1) mlp_backward_tc_kernel(const float *feats, const float *labels,
                                                                 const float *scores, const __nv_bfloat16 *h1,
                                                                 const float *h2, long long R, float inv_b,
                                                                 const float *theta, const uint8_t *wpack,
                                                                 float *grad, double *loss, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sW2T = smem;                              // B of dh1: rows i, K = o (two K chunks)
    uint8_t *sAdh2 = sW2T + 2 * W2_TILE;               // A of dh1: rows = batch rows, K = o
    uint8_t *sTdh2 = sAdh2 + 2 * W2_TILE;              // A of dW2: rows o, K = batch rows
    uint8_t *sTh1 = sTdh2 + 2 * W2_TILE;               // B of dW2: rows i, K = batch rows
    uint8_t *sTdh1 = sTh1 + 2 * W2_TILE;               // A of dW1: rows i, K = batch rows
    uint8_t *sTx = sTdh1 + 2 * W2_TILE;                // B of dW1: rows f (16), K = batch rows
    constexpr int XCH = 16 * 128;                      // bytes of one K chunk of sTx
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float w3s[NH];
    __shared__ double red[128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ntiles = (R + T_ROWS - 1) / T_ROWS;
    if ((long long)blockIdx.x >= ntiles) return;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < 2 * W2_TILE / 16; i += blockDim.x)
        ((uint4 *)sW2T)[i] = ((const uint4 *)(wpack + W1_TILE + 2 * W2_TILE))[i];
    for (int i = tid; i < NH; i += blockDim.x) w3s[i] = theta[OFF_W3 + i];
    if (warp == 0) tc_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base, d_dh1 = tmem, d_dW2 = tmem + 128, d_dW1 = tmem + 256;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    constexpr uint32_t idesc128 = idesc_bf16_f32(128, 128), idesc16 = idesc_bf16_f32(128, 16);
    unsigned phase = 0;
    bool ok = true, first = true;
    float gb1 = 0.f, gb2 = 0.f, gw3[4] = {0.f, 0.f, 0.f, 0.f}, gb3 = 0.f;
    double lsum = 0.0;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long r = tile * T_ROWS + tid;
        const bool valid = r < R;
        // the output signal and dL/da2 of this thread's row
        float ds = 0.f;
        if (valid) {
            const float sc = scores[r], y = labels[r];
            ds = (1.f / (1.f + __expf(-sc)) - y) * inv_b;
            lsum += (double)(fmaxf(sc, 0.f) + log1pf(__expf(-fabsf(sc))) - y * sc);
        }
        gb3 += ds;
#pragma unroll 1
        for (int c0 = 0; c0 < NH; c0 += 8) {
            float hv[8];
            if (valid) {
                const float4 a = *(const float4 *)(h2 + r * NH + c0), b = *(const float4 *)(h2 + r * NH + c0 + 4);
                hv[0] = a.x, hv[1] = a.y, hv[2] = a.z, hv[3] = a.w, hv[4] = b.x, hv[5] = b.y, hv[6] = b.z, hv[7] = b.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) hv[j] = 0.f;
            }
            __align__(16) __nv_bfloat16 db[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int o = c0 + j;
                db[j] = __float2bfloat16_rn(hv[j] > 0.f ? ds * w3s[o] : 0.f);
                *(__nv_bfloat16 *)(sTdh2 + (tid >> 6) * W2_TILE + sw128_off(o, tid & 63)) = db[j];
                // dw3[o] = sum over rows of ds h2[o]: warp sum, kept by lane o mod 32
                float v = ds * hv[j];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == (o & 31)) gw3[o >> 5] += v;
            }
            *(uint4 *)(sAdh2 + (c0 >> 6) * W2_TILE + sw128_off(tid, c0 & 63)) = *(const uint4 *)db;
        }
        // h1 (BF16 as saved) and x (rounded to BF16 as the forward read it), transposed
#pragma unroll 1
        for (int c0 = 0; c0 < NH; c0 += 8) {
            uint4 q = make_uint4(0, 0, 0, 0);
            if (valid) q = *(const uint4 *)(h1 + r * NH + c0);
            const __nv_bfloat16 *hb = (const __nv_bfloat16 *)&q;
#pragma unroll
            for (int j = 0; j < 8; ++j) *(__nv_bfloat16 *)(sTh1 + (tid >> 6) * W2_TILE + sw128_off(c0 + j, tid & 63)) = hb[j];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f)
            *(__nv_bfloat16 *)(sTx + (tid >> 6) * XCH + sw128_off(f, tid & 63)) =
                __float2bfloat16_rn(valid ? feats[r * NF + f] : 0.f);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int c = 0; c < 2; ++c)
                for (int ks = 0; ks < 4; ++ks) {
                    tc_mma(d_dh1, sw128_desc(smem_u32(sAdh2 + c * W2_TILE) + ks * 32),
                           sw128_desc(smem_u32(sW2T + c * W2_TILE) + ks * 32), idesc128, (c | ks) ? 1u : 0u);
                    tc_mma(d_dW2, sw128_desc(smem_u32(sTdh2 + c * W2_TILE) + ks * 32),
                           sw128_desc(smem_u32(sTh1 + c * W2_TILE) + ks * 32), idesc128,
                           (first && c == 0 && ks == 0) ? 0u : 1u);
                }
            tc_commit(&bar);
        }
        __syncwarp();
        ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        tc_fence_after();
        // db2[o = tid]: the BF16 signals of the tile, from the transposed tile
        {
            float a = 0.f;
            for (int k = 0; k < T_ROWS; ++k)
                a += __bfloat162float(*(const __nv_bfloat16 *)(sTdh2 + (k >> 6) * W2_TILE + sw128_off(tid, k & 63)));
            gb2 += a;
        }
        // dL/da1 = (dL/dh1) masked by h1 > 0, BF16, transposed into the A tile of dW1
#pragma unroll 1
        for (int c0 = 0; c0 < NH; c0 += 32) {
            float v[32];
            tc_ld_32cols(d_dh1 + lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int i = c0 + j;
                const float h = __bfloat162float(*(const __nv_bfloat16 *)(sTh1 + (tid >> 6) * W2_TILE +
                                                                         sw128_off(i, tid & 63)));
                *(__nv_bfloat16 *)(sTdh1 + (tid >> 6) * W2_TILE + sw128_off(i, tid & 63)) =
                    __float2bfloat16_rn(h > 0.f ? v[j] : 0.f);
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int c = 0; c < 2; ++c)
                for (int ks = 0; ks < 4; ++ks)
                    tc_mma(d_dW1, sw128_desc(smem_u32(sTdh1 + c * W2_TILE) + ks * 32),
                           sw128_desc(smem_u32(sTx + c * XCH) + ks * 32), idesc16,
                           (first && c == 0 && ks == 0) ? 0u : 1u);
            tc_commit(&bar);
        }
        __syncwarp();
        ok = ok && mbar_wait(&bar, phase);
        phase ^= 1u;
        tc_fence_after();
        // db1[i = tid] from the transposed BF16 tile
        {
            float a = 0.f;
            for (int k = 0; k < T_ROWS; ++k)
                a += __bfloat162float(*(const __nv_bfloat16 *)(sTdh1 + (k >> 6) * W2_TILE + sw128_off(tid, k & 63)));
            gb1 += a;
        }
        first = false;
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_after();
    if (ok && !first) {
        // dW2[o = lane of TMEM][i = column], dW1[i][f]
#pragma unroll 1
        for (int c0 = 0; c0 < NH; c0 += 32) {
            float v[32];
            tc_ld_32cols(d_dW2 + lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) atomicAdd(&grad[OFF_W2 + tid * NH + c0 + j], v[j]);
        }
        {
            float v[32];
            tc_ld_32cols(d_dW1 + lane_base, v);
#pragma unroll
            for (int f = 0; f < NF; ++f) atomicAdd(&grad[OFF_W1 + tid * NF + f], v[f]);
        }
        atomicAdd(&grad[OFF_B1 + tid], gb1);
        atomicAdd(&grad[OFF_B2 + tid], gb2);
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(&grad[OFF_W3 + k * 32 + lane], gw3[k]);
    }
    for (int off = 16; off > 0; off >>= 1) gb3 += __shfl_xor_sync(0xffffffffu, gb3, off);
    if (lane == 0) atomicAdd(&grad[OFF_B3], gb3);
    if (loss) {
        red[tid] = lsum;
        __syncthreads();
        for (int s2 = 64; s2 > 0; s2 >>= 1) {
            if (tid < s2) red[tid] += red[tid + s2];
            __syncthreads();
        }
        if (tid == 0) atomicAdd(loss, red[0]);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 512);
    if (!ok && tid == 0) atomicExch(err, 7);   // a bounded wait expired
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// theta -= lr * mhat / (sqrt(vhat) + eps).
__global__ void adam_kernel(float *theta, const float *grad, float *m, float *v, int n, float lr, float bc1,
                            float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g, vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// Per ordered pair (u, j) of a node with scored candidates: the permutation of
// its d candidate positions in descending score (ties: ascending position), as
// indices into nbr[u].  One warp per pair (its node from the stage's owner
// table): each lane holds the scores of positions lane, lane + 32, ... and
// counts, for each of them, the larger scores broadcast from the other lanes.
__global__ void perm_kernel(GraphDev g, const unsigned long long *row_off, const float *scores, short *perm)
{
    if (g.info->done || g.info->halt) return;
    if (row_off[g.p] == 0) return;                     // this stage runs in plain order
    const long long npairs = g.info->n_opairs;
    const int lane = threadIdx.x & 31;
    for (long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; o < npairs;
         o += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int u = g.opu[o];
        if (row_off[u + 1] == row_off[u]) continue;
        const int j = (int)(o - g.ooff[u]);
        const int d = g.deg[u] - 1;
        const long long base = (long long)row_off[u] + (long long)j * d;
        for (int x0 = 0; x0 < d; x0 += 32) {
            const int x = x0 + lane;
            const float sx = x < d ? scores[base + x] : 0.f;
            int rank = 0;
            for (int y0 = 0; y0 < d; y0 += 32) {
                const float sl = y0 + lane < d ? scores[base + y0 + lane] : 0.f;
                const int ny = d - y0 < 32 ? d - y0 : 32;
                for (int t = 0; t < ny; ++t) {
                    const float sy = __shfl_sync(0xffffffffu, sl, t);
                    const int y = y0 + t;
                    rank += (sy > sx) || (sy == sx && y < x);
                }
            }
            if (x < d) perm[base + rank] = (short)(x + (x >= j));   // index into nbr[u]
        }
    }
}

// ---------------------------------------------------------------- host side
int mlp_nparam() { return NPARAM; }
size_t mlp_pack_bytes() { return (size_t)W1_TILE + 4 * W2_TILE; }

cudaError_t launch_mlp_pack(const float *theta, uint8_t *wpack, cudaStream_t s)
{
    mlp_pack_kernel<<<NH, 64, 0, s>>>(theta, wpack);
    note_launch();
    return cudaGetLastError();
}

// forward pass: two CTAs per SM (97 KB shared memory and 256 TMEM columns each)
static int mlp_fwd_ctas(long long rows)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long tiles = (rows + T_ROWS - 1) / T_ROWS;
    long long c = tiles < 2ll * sms ? tiles : 2ll * sms;
    return (int)(c < 1 ? 1 : c);
}

static int mlp_ctas(long long rows)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long tiles = (rows + T_ROWS - 1) / T_ROWS;
    long long c = tiles < (long long)sms ? tiles : (long long)sms;
    return (int)(c < 1 ? 1 : c);
}

cudaError_t launch_mlp_forward_feats(const float *feats, long long R, const uint8_t *wpack, const float *theta,
                                     float *scores, __nv_bfloat16 *h1, float *h2, int *err, GraphDev g,
                                     cudaStream_t s)
{
    MlpRows rows{};
    rows.feats = feats;
    rows.R = R;
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM);
    if (e != cudaSuccess) return e;
    mlp_forward_kernel<<<mlp_fwd_ctas(R), 128, MLP_SMEM, s>>>(rows, g, wpack, theta, scores, h1, h2, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_score_stage(GraphDev g, const unsigned long long *row_off, long long rows_cap,
                                   const float *C32, int ldc, float sqn_over_q, float inv_q, const uint8_t *wpack,
                                   const float *theta, float *scores, short *perm, int *err, cudaStream_t s)
{
    MlpRows rows{};
    rows.feats = nullptr;
    rows.row_off = row_off;
    rows.C32 = C32;
    rows.ldc = ldc;
    rows.sqn_over_q = sqn_over_q;
    rows.nvec = g.nvec;
    rows.inv_q = inv_q;
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM);
    if (e != cudaSuccess) return e;
    mlp_forward_kernel<<<mlp_fwd_ctas(rows_cap), 128, MLP_SMEM, s>>>(rows, g, wpack, theta, scores, nullptr, nullptr, err);
    note_launch();
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    perm_kernel<<<sms * 4, 256, 0, s>>>(g, row_off, scores, perm);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward_tc(const float *feats, const float *labels, const float *scores,
                                   const __nv_bfloat16 *h1, const float *h2, long long R, float inv_b,
                                   const float *theta, const uint8_t *wpack, float *grad, double *loss, int *err,
                                   cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mlp_backward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BWD_SMEM);
    if (e != cudaSuccess) return e;
    mlp_backward_tc_kernel<<<mlp_ctas(R), 128, BWD_SMEM, s>>>(feats, labels, scores, h1, h2, R, inv_b, theta, wpack,
                                                              grad, loss, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *feats, const float *labels, const float *scores,
                                const __nv_bfloat16 *h1, const float *h2, long long R, float inv_b,
                                const float *theta, float *grad, double *loss, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)(2 * T_ROWS * (NH + 1) + NH * (NH + 1) + T_ROWS * NF + T_ROWS) * sizeof(float);
    e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mlp_backward_kernel<<<mlp_ctas(R), 256, smem, s>>>(feats, labels, scores, h1, h2, R, inv_b, theta, grad, loss);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam(float *theta, const float *grad, float *m, float *v, float lr, int step, cudaStream_t s)
{
    const float bc1 = 1.f - powf(0.9f, (float)step), bc2 = 1.f - powf(0.999f, (float)step);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(theta, grad, m, v, NPARAM, lr, bc1, bc2);
    note_launch();
    return cudaGetLastError();
}

// Member features for explicit quadruples (u, v, k, l | d << 16): candidate k
// of the ordered pair (u, v) at stage l with candidate-set size d.
__global__ void mlp_features_kernel(const int *quads, long long R, const float *C32, int ldc, const long long *prow,
                                    int p, long long n, const long long *nvec, float inv_q, float *feats, int *err)
{
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int u = quads[4 * r], v = quads[4 * r + 1], k = quads[4 * r + 2];
    const int l = quads[4 * r + 3] & 0xffff, d = (int)((unsigned)quads[4 * r + 3] >> 16);
    if (u < 0 || u >= p || v < 0 || v >= p || k < 0 || k >= p || u == v || k == u || k == v) {
        *err = 1;
        return;
    }
    float f[NF];
    member_features(C32, ldc, prow, u, v, k, l, d, sqrtf((float)(nvec ? nvec[u] : n)) * inv_q, f);
    for (int i = 0; i < NF; ++i) feats[r * NF + i] = f[i];
}

cudaError_t launch_mlp_features(const int *quads, long long R, const float *C32, int ldc, const long long *prow,
                                int p, long long n, const long long *nvec, double q, float *feats, int *err,
                                cudaStream_t s)
{
    mlp_features_kernel<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(quads, R, C32, ldc, prow, p, n, nvec,
                                                                      (float)(1.0 / q), feats, err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fpc
