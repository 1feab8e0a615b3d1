// corr_tc.cu -- split-precision BF16x3 correlation GEMM on the 5th-generation
// tensor cores (tcgen05, sm_103a): corr = Xs^T Xs / n (Sec. 4, the matrix corr).
//
// Each standardised value is split x = hi + lo with hi = bf16(x) and
// lo = bf16(x - hi); corr_ab ~ sum_t hi_a hi_b + hi_a lo_b + lo_a hi_b (the
// lo*lo term is below 2^-18 relative).  The three products of one K step go
// to the same FP32 accumulator in tensor memory (TMEM).
//
// One CTA computes one 128 x 128 tile of the upper triangle over one K chunk
// of KT_PER_SPLIT * 64 = 256 samples.  The tensor core adds each MMA into its
// FP32 accumulator with a rounding error of order 2^-24 of the accumulator,
// so chains are kept short: the four 16-sample K steps of a 64-sample tile go
// to four separate accumulators (all 512 TMEM columns), i.e. 12 adds per chain,
// summed in the epilogue; K chunks are added in FP64 by a reduction kernel in
// a fixed order.
//
//   warp 0 lane 0  TMA producer: 4 boxes (A_hi, A_lo, B_hi, B_lo) of 128 rows
//                  x 64 bf16 (128 B, SWIZZLE_128B) per stage, mbarrier tx-count
//   warp 1 lane 0  MMA issuer: 4 K-steps of 16 x 3 products per stage, then
//                  tcgen05.commit -> the stage's "empty" barrier
//   warps 0..3     epilogue: tcgen05.ld 32x32b (warp w owns TMEM lanes 32w..)
// Every mbarrier wait is bounded by a clock64 budget; on expiry the CTA
// records an error code, waits (bounded) for its issued MMAs, frees its TMEM
// and returns.
#include "internal.h"
#include "tc_util.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace fpc {

constexpr int TC_M = 128, TC_N = 128, TC_K = 64;        // tile; K in bf16 elements (128 B)
constexpr int TC_STAGES = 3;
constexpr int TILE_BYTES = TC_M * TC_K * 2;             // 16 KiB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;             // A_hi, A_lo, B_hi, B_lo
constexpr int KT_PER_SPLIT = 4;                         // 256 samples per split
constexpr int N_ACC = 4;                                // TMEM accumulators (one per K-step slot)
constexpr int TMEM_COLS = N_ACC * TC_N;                 // 512: the whole tensor memory of the SM

__global__ void __launch_bounds__(128, 1) corr_bf16x3_kernel(const __grid_constant__ CUtensorMap map_hi,
                                                             const __grid_constant__ CUtensorMap map_lo,
                                                             int p, int KT, float *part, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ int fail, issued_s, consumed_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // upper-triangle tile index -> (bi, bj)
    const int nt = (p + TC_M - 1) / TC_M;
    int t = blockIdx.x, bi = 0;
    while (t >= nt - bi) {
        t -= nt - bi;
        ++bi;
    }
    const int bj = bi + t;
    const int k0 = blockIdx.y * KT_PER_SPLIT;
    const int nk = min(KT, k0 + KT_PER_SPLIT) - k0;      // >= 1 by construction of the grid

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fail = 0;
        issued_s = 0;
        consumed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            const unsigned ph = (unsigned)(i / TC_STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) {
                atomicExch(&fail, 1);
                break;
            }
            uint8_t *st = smem + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            const int kx = (k0 + i) * TC_K;
            tma_load_2d(st, &map_hi, &full[s], kx, bi * TC_M);
            tma_load_2d(st + TILE_BYTES, &map_lo, &full[s], kx, bi * TC_M);
            tma_load_2d(st + 2 * TILE_BYTES, &map_hi, &full[s], kx, bj * TC_M);
            tma_load_2d(st + 3 * TILE_BYTES, &map_lo, &full[s], kx, bj * TC_M);
            issued_s = i + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer (single thread)
        constexpr uint32_t idesc = idesc_bf16_f32(TC_M, TC_N);
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            const unsigned ph = (unsigned)(i / TC_STAGES) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                atomicExch(&fail, 1);
                break;
            }
            consumed_s = i + 1;
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
            for (int k = 0; k < TC_K / 16; ++k) {
                const uint64_t ah = sw128_desc(base + k * 32);
                const uint64_t al = sw128_desc(base + TILE_BYTES + k * 32);
                const uint64_t bh = sw128_desc(base + 2 * TILE_BYTES + k * 32);
                const uint64_t bl = sw128_desc(base + 3 * TILE_BYTES + k * 32);
                const uint32_t d = tmem + (uint32_t)(k * TC_N);
                tc_mma(d, ah, bh, idesc, i > 0 ? 1u : 0u);
                tc_mma(d, ah, bl, idesc, 1u);
                tc_mma(d, al, bh, idesc, 1u);
            }
            tc_commit(&empty[s]);                      // frees the stage when these MMAs finish
        }
        tc_commit(&done);                              // arrives when every issued MMA finished
    }
    __syncwarp();
    __syncthreads();
    if (fail && threadIdx.x == 0) {
        // drain: every TMA copy this CTA issued lands before its shared memory is released
        for (int i = consumed_s; i < issued_s; ++i)
            mbar_wait(&full[i % TC_STAGES], (unsigned)(i / TC_STAGES) & 1u);
    }

    // ---- epilogue: TMEM -> registers -> FP32 partial tile
    const bool ok = mbar_wait(&done, 0u);
    tc_fence_after();
    if (ok && !fail) {
        float *out = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (TC_M * TC_N);
        const int row = warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            float v[32], w[32];
            tc_ld_32cols(lane_addr + (uint32_t)c0, v);
#pragma unroll 1
            for (int a = 1; a < N_ACC; ++a) {
                tc_ld_32cols(lane_addr + (uint32_t)(a * TC_N + c0), w);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] += w[j];
            }
            float4 *dst = (float4 *)(out + (size_t)row * TC_N + c0);
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    if (threadIdx.x == 0 && (!ok || fail)) atomicExch(err, 7);   // PC_ERR_TIMEOUT
}

// Adds the K-chunk partials of each upper tile in FP64 (fixed order), scales
// by 1/n, writes the tile and its mirror into C32, unit diagonal.
__global__ void __launch_bounds__(256) corr_tc_reduce_kernel(const float *part, int p, int ntiles,
                                                             int splits, long long n, float *C32, int ldc)
{
    const int tile = blockIdx.x, nt = (p + TC_M - 1) / TC_M;
    int t = tile, bi = 0;
    while (t >= nt - bi) {
        t -= nt - bi;
        ++bi;
    }
    const int bj = bi + t;
    const double inv_n = 1.0 / (double)n;
    const int e0 = blockIdx.y * (TC_M * TC_N / 16), e1 = e0 + TC_M * TC_N / 16;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int r = e / TC_N, c = e % TC_N;
        const int a = bi * TC_M + r, b = bj * TC_N + c;
        if (a >= p || b >= p || (bi == bj && r > c)) continue;
        double sum = 0.0;
        for (int sp = 0; sp < splits; ++sp) sum += (double)part[((size_t)sp * ntiles + tile) * (TC_M * TC_N) + e];
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
    if (major != 10 || minor != 3) return;           // this build targets sm_103a only
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

static void tc_shape(long long n, int p, int &ntiles, int &splits, int &KT)
{
    const int nt = (p + TC_M - 1) / TC_M;
    ntiles = nt * (nt + 1) / 2;
    KT = (int)((n + TC_K - 1) / TC_K);
    splits = (KT + KT_PER_SPLIT - 1) / KT_PER_SPLIT;
}

size_t corr_bf16x3_ws_bytes(long long n, int p)
{
    int ntiles, splits, KT;
    tc_shape(n, p, ntiles, splits, KT);
    return (size_t)ntiles * splits * TC_M * TC_N * sizeof(float) + 256;
}

static bool encode(CUtensorMap *map, const uint16_t *plane, long long ldk, int p)
{
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)p};         // innermost first: K, rows
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};                  // bytes between rows
    cuuint32_t box[2] = {TC_K, TC_M};
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
    if (((uintptr_t)Xhi & 15) || ((uintptr_t)Xlo & 15) || (ldk * 2) % 16 || ldk % TC_K)
        return cudaErrorInvalidValue;
    int ntiles, splits, KT;
    tc_shape(n, p, ntiles, splits, KT);
    if (ws_bytes < (size_t)ntiles * splits * TC_M * TC_N * sizeof(float)) return cudaErrorInvalidValue;
    CUtensorMap mh, ml;
    if (!encode(&mh, Xhi, ldk, p) || !encode(&ml, Xlo, ldk, p)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)TC_STAGES * STAGE_BYTES + 1024;
    cudaError_t e = cudaFuncSetAttribute(corr_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    corr_bf16x3_kernel<<<dim3(ntiles, splits), 128, smem, s>>>(mh, ml, p, KT, ws, err);
    note_launch();
    corr_tc_reduce_kernel<<<dim3(ntiles, 16), 256, 0, s>>>(ws, p, ntiles, splits, n, C32, ldc);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fpc
