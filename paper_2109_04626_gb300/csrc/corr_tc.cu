// corr_tc.cu -- split-precision BF16x3 correlation GEMM on the 5th-generation
// tensor cores (tcgen05, sm_103a): corr = Xs^T Xs / n (Sec. 4, the matrix corr).
//
// Each standardised value is split x = hi + lo with hi = bf16(x) and
// lo = bf16(x - hi); corr_ab ~ sum_t hi_a hi_b + hi_a lo_b + lo_a hi_b (the
// lo*lo term is below 2^-18 relative).  The three products of one K step go
// to the same FP32 accumulator in tensor memory (TMEM).
//
// One CTA computes one 128 x 64 tile (rows a of one 128-block, columns b of
// one 64-block, upper triangle) over a long K range.  The tensor core adds
// each MMA into its FP32 accumulator with a rounding error of order 2^-24 of
// the accumulator, so chains are kept short: samples go in rounds of four
// 64-sample K tiles, and within a round the four 16-sample K steps of every
// tile go to four separate accumulators (12 adds per chain).  Two sets of four
// accumulators (all 512 TMEM columns) alternate between rounds: while the
// tensor cores fill one set, the epilogue warps add the other into
// Kahan-compensated FP32 sums held in registers (the FP64 pipe of GB300 runs
// at 1/64 of FP32, so compensation is done in FP32).  Splits of K, a few per
// tile, are added in FP64 by a small reduction kernel in a fixed order.
//
//   warp 0 lane 0   TMA producer: A_hi, A_lo (128 rows) and B_hi, B_lo (64 rows)
//                   of 64 bf16 (128 B, SWIZZLE_128B) per stage, mbarrier tx-count
//   warp 1 lane 0   MMA issuer: 4 K steps x 3 products per K tile; a commit per
//                   stage frees it, a commit per round hands the set over
//   warps 2..5      epilogue: tcgen05.ld 32x32b of TMEM lane quadrant warp % 4
// Every mbarrier wait is bounded by a clock64 budget; on expiry the CTA
// records an error code, waits (bounded) for its issued copies and MMAs, frees
// its TMEM and returns.
#include "internal.h"
#include "tc_util.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace fpc {

constexpr int G_M = 128, G_N = 64, G_K = 64;              // tile; K in bf16 elements (128 B)
constexpr int G_STAGES = 4;
constexpr int G_A_BYTES = G_M * G_K * 2;                  // 16 KiB
constexpr int G_B_BYTES = G_N * G_K * 2;                  // 8 KiB
constexpr int G_STAGE_BYTES = 2 * G_A_BYTES + 2 * G_B_BYTES;   // A_hi, A_lo, B_hi, B_lo
constexpr int G_NACC = 4;                                 // accumulators of a set (one per K step)
constexpr int G_SET_COLS = G_NACC * G_N;                  // 256
constexpr int G_TMEM_COLS = 2 * G_SET_COLS;               // 512: two sets
constexpr int G_ROUND = 4;                                // K tiles per round
constexpr int G_THREADS = 192;

// upper-triangle tile t -> (row block bi, column block bj): columns b >= rows a
// somewhere in the tile, i.e. bj >= 2 bi (128-row and 64-column blocks)
__device__ __forceinline__ void g_tile(int t, int nb, int &bi, int &bj)
{
    bi = 0;
    while (t >= nb - 2 * bi) {
        t -= nb - 2 * bi;
        ++bi;
    }
    bj = 2 * bi + t;
}

__global__ void __launch_bounds__(G_THREADS, 1) corr_bf16x3_kernel(const __grid_constant__ CUtensorMap map_hi_a,
                                                                   const __grid_constant__ CUtensorMap map_lo_a,
                                                                   const __grid_constant__ CUtensorMap map_hi_b,
                                                                   const __grid_constant__ CUtensorMap map_lo_b,
                                                                   int p, int KT, int kt_per, float2 *part,
                                                                   int *err)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[G_STAGES], empty[G_STAGES], accf[2], accd[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int fail, issued_s, consumed_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = (p + G_N - 1) / G_N;
    int bi, bj;
    g_tile(blockIdx.x, nb, bi, bj);
    const int k0 = blockIdx.y * kt_per;
    const int nk = min(KT, k0 + kt_per) - k0;             // >= 1 by construction of the grid
    const int nrounds = (nk + G_ROUND - 1) / G_ROUND;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&accf[s], 1);                       // one commit per round
            mbar_init(&accd[s], 4);                       // one arrive per epilogue warp
        }
        mbar_init(&done, 1);
        fail = 0;
        issued_s = 0;
        consumed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc_alloc(&tmem_base, G_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            for (int i = 0; i < nk; ++i) {
                const int s = i % G_STAGES;
                const unsigned ph = (unsigned)(i / G_STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    atomicExch(&fail, 1);
                    break;
                }
                uint8_t *st = smem + s * G_STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], G_STAGE_BYTES);
                const int kx = (k0 + i) * G_K;
                tma_load_2d(st, &map_hi_a, &full[s], kx, bi * G_M);
                tma_load_2d(st + G_A_BYTES, &map_lo_a, &full[s], kx, bi * G_M);
                tma_load_2d(st + 2 * G_A_BYTES, &map_hi_b, &full[s], kx, bj * G_N);
                tma_load_2d(st + 2 * G_A_BYTES + G_B_BYTES, &map_lo_b, &full[s], kx, bj * G_N);
                issued_s = i + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer (single thread)
            constexpr uint32_t idesc = idesc_bf16_f32(G_M, G_N);
            for (int i = 0; i < nk; ++i) {
                const int r = i / G_ROUND, set = r & 1, first = (i % G_ROUND) == 0;
                if (first && r >= 2 && !mbar_wait(&accd[set], (unsigned)((r - 2) / 2) & 1u)) {
                    atomicExch(&fail, 1);                 // the set has not been drained
                    break;
                }
                const int s = i % G_STAGES;
                if (!mbar_wait(&full[s], (unsigned)(i / G_STAGES) & 1u)) {
                    atomicExch(&fail, 1);
                    break;
                }
                consumed_s = i + 1;
                tc_fence_after();
                const uint32_t base = smem_u32(smem + s * G_STAGE_BYTES);
#pragma unroll
                for (int k = 0; k < G_K / 16; ++k) {
                    const uint64_t ah = sw128_desc(base + k * 32);
                    const uint64_t al = sw128_desc(base + G_A_BYTES + k * 32);
                    const uint64_t bh = sw128_desc(base + 2 * G_A_BYTES + k * 32);
                    const uint64_t bl = sw128_desc(base + 2 * G_A_BYTES + G_B_BYTES + k * 32);
                    const uint32_t d = tmem + (uint32_t)(set * G_SET_COLS + k * G_N);
                    tc_mma(d, ah, bh, idesc, first ? 0u : 1u);
                    tc_mma(d, ah, bl, idesc, 1u);
                    tc_mma(d, al, bh, idesc, 1u);
                }
                tc_commit(&empty[s]);                     // frees the stage when these MMAs finish
                if ((i % G_ROUND) == G_ROUND - 1 || i == nk - 1) tc_commit(&accf[set]);
            }
            tc_commit(&done);                             // arrives when every issued MMA finished
        }
    } else {
        // ---- epilogue: rounds of TMEM -> registers, compensated FP32 sums
        const int q = warp & 3;                           // TMEM lane quadrant of this warp
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        float hs[G_N], hc[G_N];
#pragma unroll
        for (int c = 0; c < G_N; ++c) {
            hs[c] = 0.f;
            hc[c] = 0.f;
        }
        bool ok = true;
        for (int r = 0; r < nrounds && ok; ++r) {
            const int set = r & 1;
            // warp-uniform outcome: the TMEM loads below are warp-collective
            ok = __all_sync(0xffffffffu, mbar_wait(&accf[set], (unsigned)(r / 2) & 1u));
            if (!ok) {
                atomicExch(&fail, 1);
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < G_N; c0 += 32) {
                float v[32], w[32];
                tc_ld_32cols(lane_addr + (uint32_t)(set * G_SET_COLS + c0), v);
#pragma unroll 1
                for (int a = 1; a < G_NACC; ++a) {
                    tc_ld_32cols(lane_addr + (uint32_t)(set * G_SET_COLS + a * G_N + c0), w);
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] += w[j];
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {                // Kahan: sum hs, correction hc
                    const float y = v[j] - hc[c0 + j];
                    const float t = hs[c0 + j] + y;
                    hc[c0 + j] = (t - hs[c0 + j]) - y;
                    hs[c0 + j] = t;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accd[set]);           // the set may be reused
        }
        if (ok) {
            const int row = q * 32 + lane;
            float2 *out = part + (((size_t)blockIdx.y * gridDim.x + blockIdx.x) * G_M + row) * G_N;
#pragma unroll
            for (int c = 0; c < G_N; ++c) out[c] = make_float2(hs[c], -hc[c]);
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (fail) {
            // drain: every TMA copy this CTA issued lands before its shared memory is released
            for (int i = consumed_s; i < issued_s; ++i)
                mbar_wait(&full[i % G_STAGES], (unsigned)(i / G_STAGES) & 1u);
        }
        if (!mbar_wait(&done, 0u)) fail = 1;                 // every issued MMA finished
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, G_TMEM_COLS);
    if (threadIdx.x == 0 && fail) atomicExch(err, 7);     // PC_ERR_TIMEOUT
}

// Adds the K splits of each tile in FP64 (fixed order), scales by 1/n, writes
// the entry and its mirror; unit diagonal.
__global__ void __launch_bounds__(256) corr_tc_reduce_kernel(const float2 *part, int p, int ntiles,
                                                             int splits, long long n, float *C32, int ldc)
{
    const int nb = (p + G_N - 1) / G_N;
    int bi, bj;
    g_tile(blockIdx.x, nb, bi, bj);
    const double inv_n = 1.0 / (double)n;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < G_M * G_N; e += gridDim.y * blockDim.x) {
        const int r = e / G_N, c = e % G_N;
        const int a = bi * G_M + r, b = bj * G_N + c;
        if (a >= p || b >= p || a > b) continue;
        double sum = 0.0;
        for (int sp = 0; sp < splits; ++sp) {
            const float2 v = part[((size_t)sp * ntiles + blockIdx.x) * (G_M * G_N) + e];
            sum += (double)v.x + (double)v.y;
        }
        const float v = a == b ? 1.0f : (float)(sum * inv_n);
        C32[(long long)a * ldc + b] = v;
        C32[(long long)b * ldc + a] = v;
    }
}

// ---------------------------------------------------------------- host side
static std::once_flag g_tc_once;
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static bool g_tc_ok = false;

static void tc_init()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return;           // the kernels are compiled for sm_103a only
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    g_tc_ok = true;
}

bool tc_gemm_available()
{
    std::call_once(g_tc_once, tc_init);
    return g_tc_ok;
}

static int g_sms()
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// tiles of the upper triangle; K splits so that the grid is about one CTA per SM
static void tc_shape(long long n, int p, int &ntiles, int &splits, int &KT, int &kt_per)
{
    const int nb = (p + G_N - 1) / G_N;
    ntiles = 0;
    for (int bi = 0; 2 * bi < nb; ++bi) ntiles += nb - 2 * bi;
    KT = (int)((n + G_K - 1) / G_K);
    int sp = (g_sms() + ntiles / 2) / ntiles;
    sp = std::max(1, std::min(sp, KT));
    kt_per = (KT + sp - 1) / sp;
    splits = (KT + kt_per - 1) / kt_per;
}

size_t corr_bf16x3_ws_bytes(long long n, int p)
{
    int ntiles, splits, KT, kt_per;
    tc_shape(n, p, ntiles, splits, KT, kt_per);
    return (size_t)ntiles * splits * G_M * G_N * sizeof(float2) + 256;
}

static bool encode(CUtensorMap *map, const uint16_t *plane, long long ldk, int p, int box_rows)
{
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)p};         // innermost first: K, rows
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};                  // bytes between rows
    cuuint32_t box[2] = {G_K, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)plane, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_corr_bf16x3(const uint16_t *Xhi, const uint16_t *Xlo, long long n, long long ldk, int p,
                               float *C32, int ldc, float *ws, size_t ws_bytes, int *err, cudaStream_t s)
{
    if (!tc_gemm_available()) return cudaErrorNotSupported;
    // TMA: 16-byte aligned planes, row stride a multiple of 16 bytes, K offsets multiples of 64
    if (((uintptr_t)Xhi & 15) || ((uintptr_t)Xlo & 15) || (ldk * 2) % 16 || ldk % G_K)
        return cudaErrorInvalidValue;
    int ntiles, splits, KT, kt_per;
    tc_shape(n, p, ntiles, splits, KT, kt_per);
    if (ws_bytes < (size_t)ntiles * splits * G_M * G_N * sizeof(float2) || ((uintptr_t)ws & 7))
        return cudaErrorInvalidValue;
    CUtensorMap mha, mla, mhb, mlb;
    if (!encode(&mha, Xhi, ldk, p, G_M) || !encode(&mla, Xlo, ldk, p, G_M) || !encode(&mhb, Xhi, ldk, p, G_N) ||
        !encode(&mlb, Xlo, ldk, p, G_N))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)G_STAGES * G_STAGE_BYTES + 1024;
    cudaError_t e = cudaFuncSetAttribute(corr_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    corr_bf16x3_kernel<<<dim3(ntiles, splits), G_THREADS, smem, s>>>(mha, mla, mhb, mlb, p, KT, kt_per,
                                                                     (float2 *)ws, err);
    note_launch();
    corr_tc_reduce_kernel<<<dim3(ntiles, 8), 256, 0, s>>>((const float2 *)ws, p, ntiles, splits, n, C32, ldc);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fpc
