// corr.cu -- column standardisation and the correlation matrix
// corr = Xs^T Xs / n (Sec. 4, the matrix corr): FP64 column statistics, FP64
// and FP32 Gram kernels on the CUDA cores, and the FP64 -> FP32 cast.
#include "internal.h"
#include <cuda_bf16.h>
#include <algorithm>

namespace fpc {

template <typename T>
__device__ __forceinline__ double ld_as_double(const T *p) { return (double)__ldg(p); }

// Column mean and reciprocal population standard deviation, two passes in FP64.
// Block: 32 columns x 8 row phases; a warp reads 32 consecutive columns of one row.
template <typename T>
__global__ void __launch_bounds__(256) col_stats_kernel(const T *__restrict__ X, long long n, int p,
                                                        long long ld, double *mean, double *rsd)
{
    __shared__ double red[8][33];
    __shared__ double mu_s[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + tx;
    const bool ok = col < p;
    double s = 0.0;
    if (ok)
        for (long long t = ty; t < n; t += 8) s += ld_as_double(X + t * ld + col);
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += red[k][tx];
        mu_s[tx] = a / (double)n;
    }
    __syncthreads();
    const double mu = mu_s[tx];
    double q = 0.0;
    if (ok)
        for (long long t = ty; t < n; t += 8) {
            double d = ld_as_double(X + t * ld + col) - mu;
            q += d * d;
        }
    red[ty][tx] = q;
    __syncthreads();
    if (ty == 0 && ok) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += red[k][tx];
        double var = a / (double)n;
        mean[col] = mu;
        rsd[col] = var > 0.0 ? 1.0 / sqrt(var) : 0.0;   // constant column -> zero column
    }
}

// Column statistics over row chunks: CTA (column tile, chunk) computes the
// chunk's count, mean and sum of squared deviations (two passes over the
// chunk); col_stats_merge adds the chunks in a fixed order with Chan's update
// M2 = M2a + M2b + (mb - ma)^2 na nb / (na + nb).  Population sd (1/n).
template <typename T>
__global__ void __launch_bounds__(256) col_stats_part_kernel(const T *__restrict__ X, long long n, int p,
                                                             long long ld, long long rows_per,
                                                             double *ws)
{
    __shared__ double red[8][33];
    __shared__ double mu_s[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + tx;
    const bool ok = col < p;
    const long long r0 = (long long)blockIdx.y * rows_per;
    const long long r1 = r0 + rows_per < n ? r0 + rows_per : n;
    const double cnt = (double)(r1 - r0);
    double s = 0.0;
    if (ok)
        for (long long t = r0 + ty; t < r1; t += 8) s += ld_as_double(X + t * ld + col);
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += red[k][tx];
        mu_s[tx] = cnt > 0 ? a / cnt : 0.0;
    }
    __syncthreads();
    const double mu = mu_s[tx];
    double q = 0.0;
    if (ok)
        for (long long t = r0 + ty; t < r1; t += 8) {
            double d = ld_as_double(X + t * ld + col) - mu;
            q += d * d;
        }
    red[ty][tx] = q;
    __syncthreads();
    if (ty == 0 && ok) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += red[k][tx];
        double *w = ws + (size_t)blockIdx.y * 3 * p;
        w[col] = cnt;
        w[p + col] = mu;
        w[2 * p + col] = a;
    }
}

// FP32 input: the same two-pass chunk statistics with the per-element work in
// FP32 (GB300 runs FP64 at 1/64 of FP32).  Runs of 8 elements are summed
// exactly as double-single (TwoSum into hi + lo) and each run is added to an
// FP64 accumulator; the deviation d = x - mean is formed exactly against the
// FP64 mean split into two floats and squared with FMA-exact products.  About
// 0.5 FP64 operations per element instead of 4; the results agree with FP64
// two-pass sums to about 1e-15 relative.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// x - (mh + ml) = sd + dl + dll exactly (mh + ml: an FP64 value split into floats)
__device__ __forceinline__ void dev_split(float x, float mh, float ml, float &sd, float &dl, float &dll)
{
    float e;
    two_sum_f(x, -mh, sd, e);
    two_sum_f(e, -ml, dl, dll);
}

constexpr int STAT_RUN = 8;

__global__ void __launch_bounds__(256) col_stats_part_f32_kernel(const float *__restrict__ X, long long n, int p,
                                                                 long long ld, long long rows_per, double *ws)
{
    __shared__ double red[8][33];
    __shared__ double mu_s[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + tx;
    const bool ok = col < p;
    const long long r0 = (long long)blockIdx.y * rows_per;
    const long long r1 = r0 + rows_per < n ? r0 + rows_per : n;
    const double cnt = (double)(r1 - r0);
    double S = 0.0;
    {
        float hi = 0.f, lo = 0.f;
        int k = 0;
        if (ok)
            for (long long t = r0 + ty; t < r1; t += 8) {
                float e;
                two_sum_f(hi, X[t * ld + col], hi, e);
                lo = __fadd_rn(lo, e);
                if (++k == STAT_RUN) {
                    S += (double)hi + (double)lo;
                    hi = lo = 0.f;
                    k = 0;
                }
            }
        S += (double)hi + (double)lo;
    }
    red[ty][tx] = S;
    __syncthreads();
    if (ty == 0) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += red[k][tx];
        mu_s[tx] = cnt > 0 ? a / cnt : 0.0;
    }
    __syncthreads();
    const double mu = mu_s[tx];
    const float mh = (float)mu, ml = (float)(mu - (double)mh);
    double Q = 0.0;
    {
        float hi = 0.f, lo = 0.f, sm = 0.f;
        int k = 0;
        if (ok)
            for (long long t = r0 + ty; t < r1; t += 8) {
                float sd, dl, dll, e;
                dev_split(X[t * ld + col], mh, ml, sd, dl, dll);
                const float pp = __fmul_rn(sd, sd);
                const float pe = __fmaf_rn(sd, sd, -pp);           // sd^2 = pp + pe exactly
                // d^2 - pp = pe + 2 sd (dl + dll) + (dl + dll)^2, to FP32 accuracy
                sm = __fadd_rn(sm, __fmaf_rn(dl, dl, __fmaf_rn(__fmul_rn(2.f, sd), __fadd_rn(dl, dll), pe)));
                two_sum_f(hi, pp, hi, e);
                lo = __fadd_rn(lo, e);
                if (++k == STAT_RUN) {
                    Q += (double)hi + ((double)lo + (double)sm);
                    hi = lo = sm = 0.f;
                    k = 0;
                }
            }
        Q += (double)hi + ((double)lo + (double)sm);
    }
    red[ty][tx] = Q;
    __syncthreads();
    if (ty == 0 && ok) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += red[k][tx];
        double *w = ws + (size_t)blockIdx.y * 3 * p;
        w[col] = cnt;
        w[p + col] = mu;
        w[2 * p + col] = a;
    }
}

__global__ void col_stats_merge_kernel(const double *ws, int chunks, int p, double *mean, double *rsd)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p) return;
    double na = 0.0, ma = 0.0, Ma = 0.0;
    for (int c = 0; c < chunks; ++c) {
        const double *w = ws + (size_t)c * 3 * p;
        const double nb = w[col], mb = w[p + col], Mb = w[2 * p + col];
        if (nb == 0.0) continue;
        const double nn = na + nb, dl = mb - ma, rn = 1.0 / nn;
        ma += dl * (nb * rn);
        Ma += Mb + dl * dl * (na * nb * rn);
        na = nn;
    }
    const double var = Ma / na;
    mean[col] = ma;
    rsd[col] = var > 0.0 ? 1.0 / sqrt(var) : 0.0;   // constant column -> zero column
}

// Xs = (X - mean) * rsd written K-major (column-major, row stride ldk = padded n)
// as FP64, FP32 and a BF16 hi/lo split (hi = bf16(x), lo = bf16(x - hi)).
// 32 x 32 tiles transposed through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) standardize_kernel(const T *__restrict__ X, long long n, int p,
                                                          long long ld, const double *mean,
                                                          const double *rsd, double *Xs64,
                                                          float *Xs32, uint16_t *Xhi,
                                                          uint16_t *Xlo, long long ldk)
{
    __shared__ double tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int col0 = blockIdx.x * 32;
    const long long row0 = (long long)blockIdx.y * 32;
    const int col = col0 + tx;
    const double mu = col < p ? mean[col] : 0.0, rs = col < p ? rsd[col] : 0.0;
    for (int k = 0; k < 4; ++k) {
        long long r = row0 + ty + 8 * k;
        double v = 0.0;
        if (r < n && col < p) v = (ld_as_double(X + r * ld + col) - mu) * rs;
        tile[ty + 8 * k][tx] = v;
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        int c = col0 + ty + 8 * k;
        long long r = row0 + tx;
        if (c < p && r < n) {
            double v = tile[tx][ty + 8 * k];
            long long o = (long long)c * ldk + r;
            if (Xs64) Xs64[o] = v;
            if (Xs32) Xs32[o] = (float)v;
            if (Xhi) {
                __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
                float rem = (float)(v - (double)__bfloat162float(hi));
                __nv_bfloat16 lo = __float2bfloat16_rn(rem);
                Xhi[o] = __bfloat16_as_ushort(hi);
                Xlo[o] = __bfloat16_as_ushort(lo);
            }
        }
    }
}

// FP32 input: Xs = (x - mean) * rsd formed in double-single FP32 (the FP64
// mean and 1/sd split into two floats; TwoSum and an FMA-exact product), so
// that the FP64 plane needs only hi + lo, the FP32 and BF16 planes none.
__global__ void __launch_bounds__(256) standardize_f32_kernel(const float *__restrict__ X, long long n, int p,
                                                              long long ld, const double *mean, const double *rsd,
                                                              double *Xs64, float *Xs32, uint16_t *Xhi,
                                                              uint16_t *Xlo, long long ldk)
{
    __shared__ float th[32][33], tl[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int col0 = blockIdx.x * 32;
    const long long row0 = (long long)blockIdx.y * 32;
    const int col = col0 + tx;
    const double mu = col < p ? mean[col] : 0.0, rs = col < p ? rsd[col] : 0.0;
    const float mh = (float)mu, ml = (float)(mu - (double)mh);
    const float rh = (float)rs, rl = (float)(rs - (double)rh);
    for (int k = 0; k < 4; ++k) {
        const long long r = row0 + ty + 8 * k;
        float vh = 0.f, vl = 0.f;
        if (r < n && col < p) {
            float sd, dl, dll;
            dev_split(X[r * ld + col], mh, ml, sd, dl, dll);          // x - mean = sd + dl + dll
            vh = __fmul_rn(sd, rh);
            const float ve = __fmaf_rn(sd, rh, -vh);               // sd * rh = vh + ve exactly
            vl = __fmaf_rn(__fadd_rn(dl, dll), rh, __fmaf_rn(sd, rl, ve));
        }
        th[ty + 8 * k][tx] = vh;
        tl[ty + 8 * k][tx] = vl;
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        const int c = col0 + ty + 8 * k;
        const long long r = row0 + tx;
        if (c < p && r < n) {
            const float vh = th[tx][ty + 8 * k], vl = tl[tx][ty + 8 * k];
            const long long o = (long long)c * ldk + r;
            if (Xs64) Xs64[o] = (double)vh + (double)vl;
            const float f = __fadd_rn(vh, vl);
            if (Xs32) Xs32[o] = f;
            if (Xhi) {
                const __nv_bfloat16 hi = __float2bfloat16_rn(f);
                const float rem = __fadd_rn(__fsub_rn(vh, __bfloat162float(hi)), vl);
                Xhi[o] = __bfloat16_as_ushort(hi);
                Xlo[o] = __bfloat16_as_ushort(__float2bfloat16_rn(rem));
            }
        }
    }
}

// Gram kernel C = Xs^T Xs / n on the CUDA cores, upper-triangle 64x64 tiles
// mirrored to the lower triangle, unit diagonal.  Xs is K-major: column a of
// Xs (= row a of Xs^T) is contiguous.  Acc is the accumulation type; for FP32
// inputs each 256-long K chunk is summed in FP32 and chunks are added in FP64.
template <typename T, typename Acc>
__global__ void __launch_bounds__(256) syrk_kernel(const T *__restrict__ Xs, long long n,
                                                   long long ldk, int p, T *C, int ldc)
{
    constexpr int BT = 64, BK = 32;
    __shared__ T As[BK][BT + 1];
    __shared__ T Bs[BK][BT + 1];
    // upper-triangular tile index -> (bi, bj), bi <= bj
    int t = blockIdx.x, nt = (p + BT - 1) / BT, bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    const int bj = bi + t;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = bi * BT, b0 = bj * BT;
    double accd[4][4];
    Acc acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) { accd[i][j] = 0.0; acc[i][j] = (Acc)0; }
    int chunk = 0;
    for (long long k0 = 0; k0 < n; k0 += BK) {
        // load 64 x 32 of each operand (K contiguous): thread -> (row, k)
        for (int e = threadIdx.x; e < BT * BK; e += 256) {
            int r = e / BK, k = e % BK;
            long long kk = k0 + k;
            int ra = a0 + r, rb = b0 + r;
            As[k][r] = (ra < p && kk < n) ? Xs[(long long)ra * ldk + kk] : (T)0;
            Bs[k][r] = (rb < p && kk < n) ? Xs[(long long)rb * ldk + kk] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < BK; ++k) {
            Acc av[4], bv[4];
            for (int i = 0; i < 4; ++i) av[i] = (Acc)As[k][ty * 4 + i];
            for (int j = 0; j < 4; ++j) bv[j] = (Acc)Bs[k][tx * 4 + j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
        if (++chunk == 8) {
            chunk = 0;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) { accd[i][j] += (double)acc[i][j]; acc[i][j] = (Acc)0; }
        }
    }
    const double inv_n = 1.0 / (double)n;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            int a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
            if (a >= p || b >= p) continue;
            double v = (accd[i][j] + (double)acc[i][j]) * inv_n;
            if (a == b) v = 1.0;
            C[(long long)a * ldc + b] = (T)v;
            C[(long long)b * ldc + a] = (T)v;
        }
}

// Split-K FP64 Gram: CTA (tile, split) accumulates K range
// [split*kchunk, min(n, (split+1)*kchunk)) of an upper-triangle 64x64 tile into
// ws[(split*ntiles + tile)][64][64]; syrk_reduce_kernel then adds the splits
// in a fixed order (deterministic), scales by 1/n, mirrors, sets the diagonal.
__global__ void __launch_bounds__(256) syrk_f64_split_kernel(const double *__restrict__ Xs, long long n,
                                                             long long ldk, int p, long long kchunk,
                                                             double *ws)
{
    constexpr int BT = 64, BK = 32;
    __shared__ double As[BK][BT + 1];
    __shared__ double Bs[BK][BT + 1];
    const int tile = blockIdx.x, nt = (p + BT - 1) / BT;
    int t = tile, bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    const int bj = bi + t;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = bi * BT, b0 = bj * BT;
    const long long kb = (long long)blockIdx.y * kchunk;
    const long long ke = kb + kchunk < n ? kb + kchunk : n;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (long long k0 = kb; k0 < ke; k0 += BK) {
        for (int e = threadIdx.x; e < BT * BK; e += 256) {
            int r = e / BK, k = e % BK;
            long long kk = k0 + k;
            int ra = a0 + r, rb = b0 + r;
            As[k][r] = (ra < p && kk < ke) ? Xs[(long long)ra * ldk + kk] : 0.0;
            Bs[k][r] = (rb < p && kk < ke) ? Xs[(long long)rb * ldk + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
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
    double *out = ws + ((size_t)blockIdx.y * gridDim.x + tile) * (BT * BT);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * BT + tx * 4 + j] = acc[i][j];
}

__global__ void __launch_bounds__(256) syrk_reduce_kernel(const double *ws, int p, int ntiles_total,
                                                          int splits, long long n, double *C, int ldc)
{
    constexpr int BT = 64;
    const int tile = blockIdx.x, nt = (p + BT - 1) / BT;
    const int e0 = blockIdx.y * (BT * BT / 8), e1 = e0 + BT * BT / 8;
    int t = tile, bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    const int bj = bi + t;
    const double inv_n = 1.0 / (double)n;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int r = e / BT, c = e % BT;
        const int a = bi * BT + r, b = bj * BT + c;
        if (a >= p || b >= p || (bi == bj && r > c)) continue;
        double sum = 0.0;
        for (int sp = 0; sp < splits; ++sp) sum += ws[((size_t)sp * ntiles_total + tile) * (BT * BT) + e];
        const double v = a == b ? 1.0 : sum * inv_n;
        C[(long long)a * ldc + b] = v;
        C[(long long)b * ldc + a] = v;
    }
}

static int g_sms = 0;
static int sm_count()
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 148;
    }
    return g_sms;
}

static void syrk_split_shape(long long n, int p, int &ntiles, int &splits, long long &kchunk)
{
    const int nt = (p + 63) / 64;
    ntiles = nt * (nt + 1) / 2;
    const long long kt = (n + 31) / 32;                   // 32-wide K steps
    long long sp = (2LL * sm_count() + ntiles - 1) / ntiles;
    if (sp > kt / 2) sp = kt / 2;
    if (sp < 1) sp = 1;
    kchunk = ((kt + sp - 1) / sp) * 32;
    splits = (int)((n + kchunk - 1) / kchunk);
}

size_t syrk_f64_ws_bytes(long long n, int p)
{
    int ntiles, splits;
    long long kchunk;
    syrk_split_shape(n, p, ntiles, splits, kchunk);
    return (size_t)ntiles * splits * 64 * 64 * sizeof(double);
}

// Lazy FP64 correlations: unit diagonal, no entry valid yet.
__global__ void c64_lazy_init_kernel(double *C64, int ldc, unsigned char *valid, int p)
{
    const long long tot = (long long)p * p;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(i / p), b = (int)(i % p);
        valid[i] = a == b;
        if (a == b) C64[(long long)a * ldc + a] = 1.0;
    }
}

cudaError_t launch_c64_lazy_init(double *C64, int ldc, unsigned char *valid, int p, cudaStream_t s)
{
    long long tot = (long long)p * p;
    c64_lazy_init_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, s>>>(C64, ldc, valid, p);
    note_launch();
    return cudaGetLastError();
}

__global__ void cast_kernel(const double *C64, float *C32, int p, int ldc)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long tot = (long long)p * ldc;
    if (i < tot) C32[i] = (float)C64[i];
}

// Batched problems: the same two steps on the diagonal block [o, o+pb) of a
// matrix whose validity flags have row stride P.
__global__ void c64_lazy_init_block_kernel(double *C64, int ldc, unsigned char *valid, int P, int o, int pb)
{
    const long long tot = (long long)pb * pb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int a = o + (int)(i / pb), b = o + (int)(i % pb);
        valid[(long long)a * P + b] = a == b;
        if (a == b) C64[(long long)a * ldc + a] = 1.0;
    }
}

__global__ void cast_block_kernel(const double *C64, float *C32, int ldc, int o, int pb)
{
    const long long tot = (long long)pb * pb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = (long long)(o + (int)(i / pb)) * ldc + o + (int)(i % pb);
        C32[e] = (float)C64[e];
    }
}

cudaError_t launch_c64_lazy_init_block(double *C64, int ldc, unsigned char *valid, int P, int o, int pb,
                                       cudaStream_t s)
{
    long long tot = (long long)pb * pb;
    c64_lazy_init_block_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, s>>>(
        C64, ldc, valid, P, o, pb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_cast_block(const double *C64, float *C32, int ldc, int o, int pb, cudaStream_t s)
{
    long long tot = (long long)pb * pb;
    cast_block_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, s>>>(C64, C32, ldc, o, pb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_col_stats(const void *X, int dtype, long long n, int p, long long ld,
                             double *mean, double *rsd, cudaStream_t s)
{
    dim3 g((p + 31) / 32);
    if (dtype == 1)
        col_stats_kernel<double><<<g, 256, 0, s>>>((const double *)X, n, p, ld, mean, rsd);
    else
        col_stats_kernel<float><<<g, 256, 0, s>>>((const float *)X, n, p, ld, mean, rsd);
    note_launch();
    return cudaGetLastError();
}

static void stats_shape(long long n, int &chunks, long long &rows_per)
{
    long long c = (n + 511) / 512;
    if (c > 128) c = 128;
    if (c < 1) c = 1;
    rows_per = (n + c - 1) / c;
    chunks = (int)((n + rows_per - 1) / rows_per);
}

size_t col_stats_ws_bytes(long long n, int p)
{
    int chunks;
    long long rows_per;
    stats_shape(n, chunks, rows_per);
    return (size_t)chunks * 3 * p * sizeof(double);
}

cudaError_t launch_col_stats_split(const void *X, int dtype, long long n, int p, long long ld,
                                   double *mean, double *rsd, double *ws, cudaStream_t s)
{
    int chunks;
    long long rows_per;
    stats_shape(n, chunks, rows_per);
    dim3 g((p + 31) / 32, chunks);
    if (dtype == 1)
        col_stats_part_kernel<double><<<g, 256, 0, s>>>((const double *)X, n, p, ld, rows_per, ws);
    else
        col_stats_part_f32_kernel<<<g, 256, 0, s>>>((const float *)X, n, p, ld, rows_per, ws);
    note_launch();
    col_stats_merge_kernel<<<(p + 31) / 32, 32, 0, s>>>(ws, chunks, p, mean, rsd); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_standardize(const void *X, int dtype, long long n, int p, long long ld,
                               const double *mean, const double *rsd, double *Xs64,
                               float *Xs32, uint16_t *Xhi, uint16_t *Xlo, long long ldk,
                               cudaStream_t s)
{
    dim3 g((p + 31) / 32, (unsigned)((n + 31) / 32));
    if (dtype == 1)
        standardize_kernel<double><<<g, 256, 0, s>>>((const double *)X, n, p, ld, mean, rsd,
                                                     Xs64, Xs32, Xhi, Xlo, ldk);
    else
        standardize_f32_kernel<<<g, 256, 0, s>>>((const float *)X, n, p, ld, mean, rsd, Xs64, Xs32, Xhi, Xlo, ldk);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_syrk_f64(const double *Xs, long long n, long long ldk, int p, double *C64,
                            int ldc, double *ws, size_t ws_bytes, cudaStream_t s)
{
    int ntiles, splits;
    long long kchunk;
    syrk_split_shape(n, p, ntiles, splits, kchunk);
    if (ws_bytes < (size_t)ntiles * splits * 64 * 64 * sizeof(double)) return cudaErrorInvalidValue;
    syrk_f64_split_kernel<<<dim3(ntiles, splits), 256, 0, s>>>(Xs, n, ldk, p, kchunk, ws); note_launch();
    syrk_reduce_kernel<<<dim3(ntiles, 8), 256, 0, s>>>(ws, p, ntiles, splits, n, C64, ldc); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_syrk_f32(const float *Xs, long long n, long long ldk, int p, float *C32,
                            int ldc, cudaStream_t s)
{
    int nt = (p + 63) / 64;
    syrk_kernel<float, float><<<nt * (nt + 1) / 2, 256, 0, s>>>(Xs, n, ldk, p, C32, ldc); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_cast_c(const double *C64, float *C32, int p, int ldc, cudaStream_t s)
{
    long long tot = (long long)p * ldc;
    cast_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C64, C32, p, ldc); note_launch();
    return cudaGetLastError();
}

}  // namespace fpc
