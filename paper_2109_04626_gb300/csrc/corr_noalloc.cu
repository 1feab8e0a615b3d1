// corr_noalloc.cu -- pc_corr_noalloc: the correlation step without any device
// allocation, for callers that cannot call cudaMalloc: applications whose
// device memory is reserved up front by their own pool or budget, and
// latency-critical loops in which a cudaMalloc would synchronise the device.
//
// Its only scratch -- the FP64 column means and reciprocal standard deviations
// -- lives in a file-scope __device__ array of fixed size.  Every GPU that
// loads the library holds that array (64 KiB) until the process exits.
#include "internal.h"
#include "../../include/fastpc.h"

#include <mutex>

namespace fpc {

constexpr int NOALLOC_MAXP = 4096;

// [0, NOALLOC_MAXP): column means; [NOALLOC_MAXP, 2*NOALLOC_MAXP): 1/sd.
static __device__ __align__(256) double g_noalloc_stats[2 * NOALLOC_MAXP];

// Device address of g_noalloc_stats per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[64] = {nullptr};

static cudaError_t noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_stats);   // with device `dev` current
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Gram matrix of the standardised columns read straight from X (row-major
// n x p), FP64 accumulation, upper-triangle 64x64 tiles mirrored, unit
// diagonal.  Standardisation is applied while the 32-row slab is staged.
template <typename T>
__global__ void __launch_bounds__(256) gram_raw_kernel(const T *__restrict__ X, long long n, int p,
                                                       long long ld, const double *stats,
                                                       double *C, long long ldc)
{
    constexpr int BT = 64, BK = 32;
    __shared__ double As[BK][BT + 1];
    __shared__ double Bs[BK][BT + 1];
    const double *mean = stats, *rsd = stats + NOALLOC_MAXP;
    int t = blockIdx.x, nt = (p + BT - 1) / BT, bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    const int bj = bi + t;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = bi * BT, b0 = bj * BT;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (long long k0 = 0; k0 < n; k0 += BK) {
        for (int e = threadIdx.x; e < BT * BK; e += 256) {
            int k = e / BT, c = e % BT;                    // row k of the slab, column c
            long long r = k0 + k;
            int ca = a0 + c, cb = b0 + c;
            As[k][c] = (r < n && ca < p) ? ((double)X[r * ld + ca] - mean[ca]) * rsd[ca] : 0.0;
            Bs[k][c] = (r < n && cb < p) ? ((double)X[r * ld + cb] - mean[cb]) * rsd[cb] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    const double inv_n = 1.0 / (double)n;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            int a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
            if (a >= p || b >= p) continue;
            double v = a == b ? 1.0 : acc[i][j] * inv_n;
            C[(long long)a * ldc + b] = v;
            C[(long long)b * ldc + a] = v;
        }
}

// True when p is device (or managed) memory of device `dev`, the device the
// kernels will run on: a buffer of another GPU is rejected before any launch.
static bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace fpc

extern "C" pc_status pc_corr_noalloc(const void *X, int32_t dtype, int64_t n, int32_t p, int64_t ld,
                                     double *C_out, int64_t ldc, void *stream)
{
    using namespace fpc;
    if (!X || !C_out || (dtype != PC_F32 && dtype != PC_F64)) return PC_ERR_ARG;
    if (n < 2 || n > (1ll << 31) || p < 1 || p > NOALLOC_MAXP || ld < p || ldc < p) return PC_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PC_ERR_ARG;                  // no usable device: nothing can be on it
    }
    if (!on_device(X, dev) || !on_device(C_out, dev)) return PC_ERR_ARG;
    double *stats = nullptr;
    if (noalloc_scratch(&stats) != cudaSuccess) return PC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // column statistics into the file-scope scratch (every call overwrites
    // entries 0..p-1 of both halves; nothing accumulates across calls)
    if (launch_col_stats(X, dtype, n, p, ld, stats, stats + NOALLOC_MAXP, s) != cudaSuccess)
        return PC_ERR_CUDA;
    const int nt = (p + 63) / 64;
    if (dtype == PC_F64)
        gram_raw_kernel<double><<<nt * (nt + 1) / 2, 256, 0, s>>>((const double *)X, n, p, ld, stats,
                                                                 C_out, ldc);
    else
        gram_raw_kernel<float><<<nt * (nt + 1) / 2, 256, 0, s>>>((const float *)X, n, p, ld, stats,
                                                                C_out, ldc);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
