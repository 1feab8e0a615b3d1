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

// FP32 input (GB300 runs FP64 at 1/64 of FP32): the per-element work is FP32.
// Sums are kept exactly as double-single (TwoSum into hi + lo) and renormalised
// every few elements; FP64 is used only at the end of short runs and across
// warps and chunks.  The squares are taken about the float part mh of the FP64
// mean (x - mh exact by TwoSum, squared with FMA-exact products) and corrected
// by n (mean - mh)^2.  The results agree with FP64 two-pass sums to about 1e-15
// relative.
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

// float -> double without the FP64 pipe: the IEEE-754 binary32 fields moved into
// binary64 (exponent rebiased by 1023 - 127 = 896, fraction shifted by 52 - 23).
// Exact for normal numbers and zeros; subnormals, infinities and NaNs take the
// conversion instruction.
__device__ __forceinline__ double f2d(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (e == 0u || e == 0xffu) return (double)x;
    const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((b & 7u) << 29));
}

// Work layout of the FP32 statistics passes: CTA (column tile of ST_COLS, row
// chunk); lane l of a warp owns columns 4l..4l+3 of the tile (one 16-byte load
// per row), the 8 warps take every 8th row of the chunk, 4 rows per iteration.
constexpr int ST_THREADS = 256;
constexpr int ST_COLS = 128;

struct StatsLayout {
    int tiles, chunks;
    long long rows_per;
    size_t part_off, ticket_off, split_off, nmrs_off, bytes;
};

static StatsLayout stats_layout_f32(long long n, int p)
{
    StatsLayout L;
    L.tiles = (p + ST_COLS - 1) / ST_COLS;
    // about one wave of 4 CTAs per SM on 152 SMs, at least 64 rows per chunk
    long long rp = (n * L.tiles + 607) / 608;
    rp = (rp + 31) / 32 * 32;
    if (rp < 64) rp = 64;
    L.rows_per = rp;
    L.chunks = (int)std::max<long long>(1, (n + rp - 1) / rp);
    L.part_off = 0;
    L.ticket_off = (size_t)L.chunks * p * sizeof(double);
    L.split_off = (L.ticket_off + (size_t)L.tiles * sizeof(unsigned) + 15) / 16 * 16;
    L.nmrs_off = L.split_off + (size_t)p * sizeof(float4);
    L.bytes = L.nmrs_off + (size_t)p * sizeof(double);
    return L;
}

// 4 consecutive columns c..c+3 of row r (zeros past p, or for r < 0)
__device__ __forceinline__ void ld_row4(const float *__restrict__ X, long long ld, long long r, int c, int p,
                                        int vec, float (&v)[4])
{
    if (r < 0) {
        v[0] = v[1] = v[2] = v[3] = 0.f;
        return;
    }
    const float *q = X + r * ld + c;
    if (vec && c + 3 < p) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(q));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = c + k < p ? __ldg(q + k) : 0.f;
    }
}

// The last CTA of a column tile (ticket) adds the chunks' partials part[chunk][col]
// in a fixed order; returns true in that CTA, with tot[0..ST_COLS) the tile's totals.
__device__ __forceinline__ bool last_chunk_total(const double *part, int chunks, int p, unsigned *ticket,
                                                 double (*red)[ST_COLS], double *tot)
{
    __shared__ int amlast;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) amlast = atomicAdd(&ticket[blockIdx.x], 1u) == (unsigned)(chunks - 1);
    __syncthreads();
    if (!amlast) return false;
    __threadfence();
    const int cc = threadIdx.x % ST_COLS, h = threadIdx.x / ST_COLS;   // 2 halves of the chunks
    const int col = blockIdx.x * ST_COLS + cc;
    double s = 0.0;
    if (col < p)
        for (int ch = h; ch < chunks; ch += ST_THREADS / ST_COLS) s += __ldcg(part + (size_t)ch * p + col);
    red[h][cc] = s;
    __syncthreads();
    if (threadIdx.x < ST_COLS) tot[threadIdx.x] = red[0][threadIdx.x] + red[1][threadIdx.x];
    if (threadIdx.x == 0) ticket[blockIdx.x] = 0u;        // every CTA of the tile has taken its ticket
    __syncthreads();
    return true;
}

// Pass 1: column sums per chunk, then (last CTA of the tile) mean = sum / n and
// its float split (mh, ml) into split[col].xy.
__global__ void __launch_bounds__(ST_THREADS, 4) col_sum_f32_kernel(const float *__restrict__ X, long long n, int p,
                                                                long long ld, int vec, long long rows_per,
                                                                int chunks, double *part, unsigned *ticket,
                                                                double *mean, float4 *split)
{
    __shared__ double red[8][ST_COLS];
    __shared__ double tot[ST_COLS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * ST_COLS + 4 * lane;
    const long long r0 = (long long)blockIdx.y * rows_per;
    const long long r1 = r0 + rows_per < n ? r0 + rows_per : n;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long r = r0 + w; r < r1; r += 32) {
        float v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ld_row4(X, ld, r + 8 * u < r1 ? r + 8 * u : -1, c, p, vec, v[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float e;
                two_sum_f(hi[q], v[u][q], hi[q], e);
                lo[q] = __fadd_rn(lo[q], e);
            }
#pragma unroll
        for (int q = 0; q < 4; ++q) two_sum_f(hi[q], lo[q], hi[q], lo[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[w][4 * lane + q] = f2d(hi[q]) + f2d(lo[q]);
    __syncthreads();
    if (threadIdx.x < ST_COLS) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
        const int col = blockIdx.x * ST_COLS + threadIdx.x;
        if (col < p) part[(size_t)blockIdx.y * p + col] = s;
    }
    if (!last_chunk_total(part, chunks, p, ticket, red, tot)) return;
    if (threadIdx.x < ST_COLS) {
        const int col = blockIdx.x * ST_COLS + threadIdx.x;
        if (col < p) {
            const double mu = tot[threadIdx.x] / (double)n;
            mean[col] = mu;
            const float mh = (float)mu;
            split[col] = make_float4(mh, (float)(mu - (double)mh), 0.f, 0.f);
        }
    }
}

// Pass 2: A = sum (x - mh)^2 per chunk (the chunk was just read: mostly L2 hits);
// x - mh = sd + e exactly (TwoSum), (sd + e)^2 = pp + pe + 2 sd e + e^2 with
// sd^2 = pp + pe exact (FMA).  The last CTA of the tile forms
// M2 = sum (x - mean)^2 = A - n ml^2 (ml = mean - mh; no cancellation, ml is
// below half an FP32 ulp of the mean), rsd = 1/sd (population), its float split
// (rh, rl) into split[col].zw and nmrs[col] = -mean * rsd.  A constant column
// gets rsd = 0.
__global__ void __launch_bounds__(ST_THREADS, 4) col_m2_f32_kernel(const float *__restrict__ X, long long n, int p,
                                                                  long long ld, int vec, long long rows_per,
                                                                  int chunks, double *part, unsigned *ticket,
                                                                  const double *mean, double *rsd, float4 *split,
                                                                  double *nmrs)
{
    __shared__ double red[8][ST_COLS];
    __shared__ double tot[ST_COLS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * ST_COLS + 4 * lane;
    const long long r0 = (long long)blockIdx.y * rows_per;
    const long long r1 = r0 + rows_per < n ? r0 + rows_per : n;
    float mh[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) mh[q] = c + q < p ? split[c + q].x : 0.f;
    double Q[4] = {0.0, 0.0, 0.0, 0.0};
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f}, sm[4] = {0.f, 0.f, 0.f, 0.f};
    int runs = 0;
    for (long long r = r0 + w; r < r1; r += 32) {
        float v[4][4];
        bool in[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            in[u] = r + 8 * u < r1;
            ld_row4(X, ld, in[u] ? r + 8 * u : -1, c, p, vec, v[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!in[u]) continue;                            // a zero row is not a zero deviation
                float sd, e, ee;
                two_sum_f(v[u][q], -mh[q], sd, e);
                const float pp = __fmul_rn(sd, sd);
                const float pe = __fmaf_rn(sd, sd, -pp);
                sm[q] = __fadd_rn(sm[q], __fmaf_rn(e, e, __fmaf_rn(__fmul_rn(2.f, sd), e, pe)));
                two_sum_f(hi[q], pp, hi[q], ee);
                lo[q] = __fadd_rn(lo[q], ee);
            }
        if (++runs == 2) {                                       // 8 rows per column: into FP64
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Q[q] += f2d(hi[q]) + (f2d(lo[q]) + f2d(sm[q]));
                hi[q] = lo[q] = sm[q] = 0.f;
            }
            runs = 0;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[w][4 * lane + q] = Q[q] + (f2d(hi[q]) + (f2d(lo[q]) + f2d(sm[q])));
    __syncthreads();
    if (threadIdx.x < ST_COLS) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
        const int col = blockIdx.x * ST_COLS + threadIdx.x;
        if (col < p) part[(size_t)blockIdx.y * p + col] = s;
    }
    if (!last_chunk_total(part, chunks, p, ticket, red, tot)) return;
    if (threadIdx.x < ST_COLS) {
        const int col = blockIdx.x * ST_COLS + threadIdx.x;
        if (col < p) {
            const double mu = mean[col];
            float4 sp = split[col];
            const double ml = mu - (double)sp.x;
            const double m2 = tot[threadIdx.x] - (double)n * ml * ml;
            const double var = m2 / (double)n;
            const double rs = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
            rsd[col] = rs;
            const float rh = (float)rs;
            sp.z = rh;
            sp.w = (float)(rs - (double)rh);
            split[col] = sp;
            nmrs[col] = -(mu * rs);
        }
    }
}

// FP32 input: Xs = (x - mean) * rsd.  The FP64 plane is fma(x, rsd, -mean*rsd)
// (one FP64 operation per element; the constant error of -mean*rsd shifts a
// column by a constant, which changes a correlation only at second order because
// the column sums to zero).  The FP32 plane and the BF16 pair (hi = bf16(f),
// lo = bf16(rest)) come from the double-single FP32 value vh + vl formed against
// the float splits of mean and 1/sd.  64 x 64 tiles: 16-byte row reads into a
// column-major shared tile, then per column 64 consecutive rows written at once
// (two rows per lane).
constexpr int SD_T = 64;
__global__ void __launch_bounds__(256) standardize_f32_kernel(const float *__restrict__ X, long long n, int p,
                                                              long long ld, int vec, const float4 *__restrict__ split,
                                                              const double *__restrict__ rsd,
                                                              const double *__restrict__ nmrs, double *Xs64,
                                                              float *Xs32, uint16_t *Xhi, uint16_t *Xlo, long long ldk)
{
    __shared__ float tx[SD_T][SD_T + 2];                  // [column][row]
    const int col0 = blockIdx.x * SD_T;
    const long long row0 = (long long)blockIdx.y * SD_T;
    {
        const int cq = (threadIdx.x & 15) * 4, rg = threadIdx.x >> 4;   // 4 columns, rows rg + 16 i
        float v[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long r = row0 + rg + 16 * i;
            ld_row4(X, ld, r < n ? r : -1, col0 + cq, p, vec, v[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) tx[cq + q][rg + 16 * i] = v[i][q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long r = row0 + 2 * lane;                                    // rows r, r + 1
    if (r >= n) return;
    const bool both = r + 1 < n;
    for (int k = 0; k < SD_T / 8; ++k) {
        const int cc = w * (SD_T / 8) + k, c = col0 + cc;
        if (c >= p) break;
        const float2 x2 = *reinterpret_cast<const float2 *>(&tx[cc][2 * lane]);
        const float4 sp = split[c];                                         // mh, ml, rh, rl
        const long long o = (long long)c * ldk + r;                           // even: ldk and r are
        if (Xs64) {
            const double rs = rsd[c], b = nmrs[c];
            const double d0 = fma(f2d(x2.x), rs, b), d1 = fma(f2d(x2.y), rs, b);
            if (both) *reinterpret_cast<double2 *>(Xs64 + o) = make_double2(d0, d1);
            else Xs64[o] = d0;
        }
        if (!Xs32 && !Xhi) continue;
        float vh[2], vl[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            float sd, dl, dll;
            dev_split(t ? x2.y : x2.x, sp.x, sp.y, sd, dl, dll);            // x - mean = sd + dl + dll
            vh[t] = __fmul_rn(sd, sp.z);
            const float ve = __fmaf_rn(sd, sp.z, -vh[t]);                   // sd * rh = vh + ve exactly
            vl[t] = __fmaf_rn(__fadd_rn(dl, dll), sp.z, __fmaf_rn(sd, sp.w, ve));
        }
        const float f0 = __fadd_rn(vh[0], vl[0]), f1 = __fadd_rn(vh[1], vl[1]);
        if (Xs32) {
            if (both) *reinterpret_cast<float2 *>(Xs32 + o) = make_float2(f0, f1);
            else Xs32[o] = f0;
        }
        if (Xhi) {
            const __nv_bfloat16 a0 = __float2bfloat16_rn(f0), a1 = __float2bfloat16_rn(f1);
            const __nv_bfloat16 b0 = __float2bfloat16_rn(__fadd_rn(__fsub_rn(vh[0], __bfloat162float(a0)), vl[0]));
            const __nv_bfloat16 b1 = __float2bfloat16_rn(__fadd_rn(__fsub_rn(vh[1], __bfloat162float(a1)), vl[1]));
            if (both) {
                *reinterpret_cast<uint32_t *>(Xhi + o) =
                    (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(a1) << 16);
                *reinterpret_cast<uint32_t *>(Xlo + o) =
                    (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
            } else {
                Xhi[o] = __bfloat16_as_ushort(a0);
                Xlo[o] = __bfloat16_as_ushort(b0);
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
// [split*kchunk, min(n, (split+1)*kchunk)) of an upper-triangle BT x BT tile into
// ws[(split*ntiles + tile)][BT][BT]; syrk_reduce_kernel then adds the splits
// in a fixed order (deterministic), scales by 1/n, mirrors, sets the diagonal.
// BT 64 (4 x 4 outputs per thread) for large p; BT 32 (2 x 2) for p <= 128, where
// 64-wide tiles would pad the matrix to 128 and nearly double the FP64 work (the
// FP64 pipe is what bounds this kernel on GB300).
template <int BT>
__global__ void __launch_bounds__(256) syrk_f64_split_kernel(const double *__restrict__ Xs, long long n,
                                                             long long ldk, int p, long long kchunk,
                                                             double *ws)
{
    constexpr int BK = 32, RT = BT / 16;                 // RT x RT outputs per thread
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
    double acc[RT][RT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] = 0.0;
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
            double av[RT], bv[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) av[i] = As[k][ty * RT + i];
#pragma unroll
            for (int j = 0; j < RT; ++j) bv[j] = Bs[k][tx * RT + j];
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int j = 0; j < RT; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *out = ws + ((size_t)blockIdx.y * gridDim.x + tile) * (BT * BT);
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) out[(ty * RT + i) * BT + tx * RT + j] = acc[i][j];
}

template <int BT>
__global__ void __launch_bounds__(256) syrk_reduce_kernel(const double *ws, int p, int ntiles_total,
                                                          int splits, long long n, double *C, int ldc)
{
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

static int syrk_tile(int p) { return p <= 128 ? 32 : 64; }

static void syrk_split_shape(long long n, int p, int &ntiles, int &splits, long long &kchunk)
{
    const int bt = syrk_tile(p);
    const int nt = (p + bt - 1) / bt;
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
    const int bt = syrk_tile(p);
    return (size_t)ntiles * splits * bt * bt * sizeof(double);
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
    return std::max((size_t)chunks * 3 * p * sizeof(double), stats_layout_f32(n, p).bytes);
}

// FP64 input: per-chunk two-pass statistics and Chan's merge.  FP32 input: the
// two FP32 passes, each finished by its last CTA per column tile; the float
// splits of mean and 1/sd and -mean/sd are left in ws for launch_standardize.
cudaError_t launch_col_stats_split(const void *X, int dtype, long long n, int p, long long ld,
                                   double *mean, double *rsd, double *ws, cudaStream_t s)
{
    if (dtype == 1) {
        int chunks;
        long long rows_per;
        stats_shape(n, chunks, rows_per);
        dim3 g((p + 31) / 32, chunks);
        col_stats_part_kernel<double><<<g, 256, 0, s>>>((const double *)X, n, p, ld, rows_per, ws); note_launch();
        col_stats_merge_kernel<<<(p + 31) / 32, 32, 0, s>>>(ws, chunks, p, mean, rsd); note_launch();
        return cudaGetLastError();
    }
    const StatsLayout L = stats_layout_f32(n, p);
    char *base = reinterpret_cast<char *>(ws);
    double *part = reinterpret_cast<double *>(base + L.part_off);
    unsigned *ticket = reinterpret_cast<unsigned *>(base + L.ticket_off);
    float4 *split = reinterpret_cast<float4 *>(base + L.split_off);
    const int vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
    cudaError_t e = cudaMemsetAsync(ticket, 0, (size_t)L.tiles * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const dim3 g(L.tiles, L.chunks);
    col_sum_f32_kernel<<<g, ST_THREADS, 0, s>>>((const float *)X, n, p, ld, vec, L.rows_per, L.chunks, part, ticket,
                                                mean, split); note_launch();
    col_m2_f32_kernel<<<g, ST_THREADS, 0, s>>>((const float *)X, n, p, ld, vec, L.rows_per, L.chunks, part, ticket,
                                               mean, rsd, split, reinterpret_cast<double *>(base + L.nmrs_off));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_standardize(const void *X, int dtype, long long n, int p, long long ld,
                               const double *mean, const double *rsd, const double *stats_ws, double *Xs64,
                               float *Xs32, uint16_t *Xhi, uint16_t *Xlo, long long ldk,
                               cudaStream_t s)
{
    if (dtype == 1) {
        dim3 g((p + 31) / 32, (unsigned)((n + 31) / 32));
        standardize_kernel<double><<<g, 256, 0, s>>>((const double *)X, n, p, ld, mean, rsd,
                                                     Xs64, Xs32, Xhi, Xlo, ldk); note_launch();
        return cudaGetLastError();
    }
    const StatsLayout L = stats_layout_f32(n, p);
    const char *wsb = reinterpret_cast<const char *>(stats_ws);
    const float4 *split = reinterpret_cast<const float4 *>(wsb + L.split_off);
    const double *nmrs = reinterpret_cast<const double *>(wsb + L.nmrs_off);
    const int vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
    dim3 g((p + SD_T - 1) / SD_T, (unsigned)((n + SD_T - 1) / SD_T));
    standardize_f32_kernel<<<g, 256, 0, s>>>((const float *)X, n, p, ld, vec, split, rsd, nmrs, Xs64, Xs32, Xhi, Xlo,
                                             ldk);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_syrk_f64(const double *Xs, long long n, long long ldk, int p, double *C64,
                            int ldc, double *ws, size_t ws_bytes, cudaStream_t s)
{
    int ntiles, splits;
    long long kchunk;
    syrk_split_shape(n, p, ntiles, splits, kchunk);
    const int bt = syrk_tile(p);
    if (ws_bytes < (size_t)ntiles * splits * bt * bt * sizeof(double)) return cudaErrorInvalidValue;
    if (bt == 32) {
        syrk_f64_split_kernel<32><<<dim3(ntiles, splits), 256, 0, s>>>(Xs, n, ldk, p, kchunk, ws); note_launch();
        syrk_reduce_kernel<32><<<dim3(ntiles, 8), 256, 0, s>>>(ws, p, ntiles, splits, n, C64, ldc); note_launch();
    } else {
        syrk_f64_split_kernel<64><<<dim3(ntiles, splits), 256, 0, s>>>(Xs, n, ldk, p, kchunk, ws); note_launch();
        syrk_reduce_kernel<64><<<dim3(ntiles, 8), 256, 0, s>>>(ws, p, ntiles, splits, n, C64, ldc); note_launch();
    }
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
