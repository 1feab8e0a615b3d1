// level.cu -- one PC-stable stage of the skeleton search (Algorithm 1 lines
// 3-20 / Algorithm 2 lines 2-18) on the GPU.
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

namespace fpc {

typedef unsigned long long ull;

__device__ __forceinline__ ull sat_add(ull a, ull b)
{
    ull c = a + b;
    return c < a ? KEY_NONE : c;
}

// ---------------------------------------------------------------- degrees
__global__ void degrees_kernel(GraphDev g)
{
    const int lane = threadIdx.x & 31;
    const int u = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (u >= g.p) return;
    const uint32_t *row = g.adj + (long long)u * g.W;
    int base = 0;
    for (int w0 = 0; w0 < g.W; w0 += 32) {
        const int w = w0 + lane;
        uint32_t bits = (w < g.W) ? row[w] : 0u;
        const int c = __popc(bits);
        int incl = c;
        for (int off = 1; off < 32; off <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        int pos = base + incl - c;
        while (bits) {
            int t = __ffs(bits) - 1;
            g.nbr[(long long)u * g.p + pos++] = w * 32 + t;
            bits &= bits - 1;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        g.deg[u] = base;
        if (base > 0) atomicMax(&g.info->lstar, base - 1);
        atomicAdd(&g.info->edges, (ull)base);
    }
}

// exclusive scan of deg -> ooff[0..p], single CTA (p <= 4096)
__global__ void __launch_bounds__(1024) ooff_kernel(GraphDev g)
{
    __shared__ long long part[1024];
    const int p = g.p, t = threadIdx.x;
    const int per = (p + 1023) / 1024;
    const int s0 = t * per, s1 = min(p, s0 + per);
    long long sum = 0;
    for (int i = s0; i < s1; ++i) sum += g.deg[i];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        long long v = (t >= off) ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - sum;
    for (int i = s0; i < s1; ++i) {
        g.ooff[i] = run;
        run += g.deg[i];
    }
    if (t == 1023) {
        g.ooff[p] = part[1023];
        g.info->n_opairs = part[1023];
    }
}

// ---------------------------------------------------------------- complement eligibility
__device__ __forceinline__ bool comp_eligible(int d, int l, const TestParams &tp)
{
    const int k = d - l;
    return tp.reversed && tp.complement && d >= l && k <= KC_MAX && k < l && d + 2 <= PREC_MAX;
}

__global__ void prec_need_kernel(GraphDev g, TestParams tp, int l)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.p) return;
    const int dg = g.deg[u];
    const bool need = dg > 0 && comp_eligible(dg - 1, l, tp) && g.prec_m[u] == 0;
    g.prec_need[u] = need;
    if (need) atomicAdd(&g.info->n_build, 1);
}

__global__ void counts_kernel(GraphDev g, TestParams tp, int l)
{
    const long long nop = g.info->n_opairs;
    const int p = g.p;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nop;
         o += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(upper_bound_dev(g.ooff, (long long)p + 1, o) - 1);
        const int d = g.deg[u] - 1;
        const ull T = d >= l ? g.binom[(long long)d * (p + 1) + l] : 0ull;
        const bool comp = d >= l && comp_eligible(d, l, tp) && g.prec_m[u] > 0;
        g.tcnt[o] = comp ? 0ull : T;
        g.ccnt[o] = comp ? T : 0ull;
        if (T == KEY_NONE) g.info->saturated = 1;
    }
}

// ---------------------------------------------------------------- u64 saturating scan
constexpr int SCAN_T = 256, SCAN_PER = 16, SCAN_TILE = SCAN_T * SCAN_PER;

size_t scan_ws_bytes(long long n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 2) * sizeof(ull); }

__device__ __forceinline__ ull block_reduce_sat(ull v, ull *sh)
{
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = SCAN_T / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] = sat_add(sh[t], sh[t + s]);
        __syncthreads();
    }
    ull r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) scan_reduce_kernel(const ull *a, const long long *nptr,
                                                             ull *part)
{
    __shared__ ull sh[SCAN_T];
    const long long n = *nptr;
    const long long start = (long long)blockIdx.x * SCAN_TILE;
    ull s = 0;
    for (int i = 0; i < SCAN_PER; ++i) {
        long long idx = start + (long long)i * SCAN_T + threadIdx.x;
        if (idx < n) s = sat_add(s, a[idx]);
    }
    s = block_reduce_sat(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) scan_part_kernel(ull *part, int nb, ull *total)
{
    __shared__ ull sh[1024];
    const int t = threadIdx.x;
    ull carry = 0;
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int i = c0 + t;
        sh[t] = i < nb ? part[i] : 0ull;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            ull x = t >= off ? sh[t - off] : 0ull;
            __syncthreads();
            sh[t] = sat_add(sh[t], x);
            __syncthreads();
        }
        const ull excl = t ? sh[t - 1] : 0ull;
        if (i < nb) part[i] = sat_add(carry, excl);
        const ull blk = sh[1023];
        __syncthreads();
        carry = sat_add(carry, blk);
    }
    if (t == 0) *total = carry;
}

__global__ void __launch_bounds__(SCAN_T) scan_down_kernel(ull *a, const long long *nptr,
                                                           const ull *part, const ull *total)
{
    __shared__ ull tile[SCAN_TILE + SCAN_T];
    __shared__ ull sh[SCAN_T];
    const long long n = *nptr;
    const long long start = (long long)blockIdx.x * SCAN_TILE;
    if (start > n) return;
    for (int i = 0; i < SCAN_PER; ++i) {
        int li = i * SCAN_T + threadIdx.x;
        long long idx = start + li;
        tile[li + li / SCAN_PER] = idx < n ? a[idx] : 0ull;
    }
    __syncthreads();
    // thread t owns tile elements [t*PER, (t+1)*PER)
    const int t = threadIdx.x;
    ull s = 0;
    for (int i = 0; i < SCAN_PER; ++i) {
        int li = t * SCAN_PER + i;
        s = sat_add(s, tile[li + li / SCAN_PER]);
    }
    sh[t] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
        ull x = t >= off ? sh[t - off] : 0ull;
        __syncthreads();
        sh[t] = sat_add(sh[t], x);
        __syncthreads();
    }
    ull run = sat_add(part[blockIdx.x], t ? sh[t - 1] : 0ull);
    for (int i = 0; i < SCAN_PER; ++i) {
        int li = t * SCAN_PER + i;
        ull v = tile[li + li / SCAN_PER];
        tile[li + li / SCAN_PER] = run;
        run = sat_add(run, v);
    }
    __syncthreads();
    for (int i = 0; i < SCAN_PER; ++i) {
        int li = i * SCAN_T + threadIdx.x;
        long long idx = start + li;
        if (idx < n) a[idx] = tile[li + li / SCAN_PER];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a[n] = *total;
}

// exclusive scan of a[0..n) in place, a[n] = total (n read from device)
static cudaError_t scan_u64(ull *a, const long long *nptr, long long ncap, void *ws, ull *total_out,
                            cudaStream_t s)
{
    int nb = (int)((ncap + SCAN_TILE - 1) / SCAN_TILE);
    if (nb < 1) nb = 1;
    ull *part = (ull *)ws;
    ull *total = part + nb;
    scan_reduce_kernel<<<nb, SCAN_T, 0, s>>>(a, nptr, part); note_launch();
    scan_part_kernel<<<1, 1024, 0, s>>>(part, nb, total); note_launch();
    scan_down_kernel<<<nb, SCAN_T, 0, s>>>(a, nptr, part, total); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(total_out, total, sizeof(ull), cudaMemcpyDeviceToDevice, s);
}

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

__device__ __forceinline__ ull flops_direct(int l)
{
    ull L = (ull)l;
    return (L * L * L) / 3 + 2 * L * L + 6 * L + 10;
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
            for (int c = lane; c <= i; c += 32) M[i * ms + c] = C32[(long long)nd[i] * ldc + nd[c]];
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
            // error model of the FP32 evaluation: dr ~ (m eps32 + eps_C) / pmin
            const float dr = 2.0f * ((float)m * 5.96e-8f + 1.2e-7f) / pmin;
            const float omr = fmaxf(1.0f - rf * rf, 1e-3f);
            zf = fabsf(rf) < 1.0f ? sqf * fabsf(atanhf(rf)) : INFINITY;
            const float dz = sqf * dr / omr;
            if (dr > 5e-6f) {
                need64 = true;
                ++acc.guard;
            } else if (fabsf(zf - tp.qf) < (float)tp.band + 4.0f * dz) {
                need64 = true;
                ++acc.band;
            } else {
                indep = zf <= tp.qf;
                f32ok = true;
            }
        }
    }
    double r = rf;
    float z = zf;
    if (need64) {
        double *M = (double *)Mbuf;
        for (int i = 0; i < m; ++i)
            for (int c = lane; c <= i; c += 32) M[i * ms + c] = C64[(long long)nd[i] * ldc + nd[c]];
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

// ---------------------------------------------------------------- direct path (skeleton)
template <bool F64>
__global__ void __launch_bounds__(256) ci_direct_kernel(GraphDev g, TestParams tp, int l,
                                                        const float *C32, const double *C64,
                                                        int ldc, int ms, int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = l + 2, p = g.p;
    unsigned char *mine = smem_raw + (size_t)wib * per_warp_bytes;
    double *Mbuf = (double *)mine;
    int *nd = (int *)(mine + (size_t)m * ms * sizeof(double));
    int *pos = nd + m;
    const ull total = g.info->total_direct;
    const long long nop = g.info->n_opairs;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const double sq = sqrt((double)(tp.n - l - 3));
    const float sqf = (float)sq;
    WarpAcc acc = {0, 0, 0, 0, 0, 0, 0, 0.f};
    for (ull t = gw; t < total; t += nw) {
        const long long o = upper_bound_dev(g.tcnt, nop + 1, t) - 1;
        const ull rank = t - g.tcnt[o];
        const int u = (int)(upper_bound_dev(g.ooff, (long long)p + 1, o) - 1);
        const int j = (int)(o - g.ooff[u]);
        const int v = g.nbr[(long long)u * p + j];
        const int d = g.deg[u] - 1;
        const int side = u > v;
        const int a = min(u, v), b = max(u, v);
        const ull key = ((ull)side << 62) | rank;
        ull *bp = g.best + (long long)a * p + b;
        if (*(volatile ull *)bp < key) continue;   // an earlier set already separates
        if (lane == 0) {
            unrank_lex(rank, d, l, g.binom, p + 1, pos);
            for (int i = 0; i < l; ++i) {
                int x = pos[i];
                nd[i] = g.nbr[(long long)u * p + x + (x >= j)];
            }
            nd[l] = u;
            nd[l + 1] = v;
        }
        __syncwarp();
        double r;
        float z;
        ++acc.tests;
        bool ind = warp_test<F64>(nd, m, l, C32, C64, ldc, tp, sq, sqf, Mbuf, ms, acc, r, z);
        if (ind && lane == 0) atomicMin(bp, key);
        __syncwarp();
    }
    if (lane == 0) flush_acc(acc, g.ctr);
}

// ---------------------------------------------------------------- complement path
__global__ void __launch_bounds__(128) ci_complement_kernel(GraphDev g, TestParams tp, int l)
{
    const ull total = g.info->total_comp;
    const long long nop = g.info->n_opairs;
    const int p = g.p;
    const double sq = sqrt((double)(tp.n - l - 3));
    ull nt = 0, ndg = 0, nfl = 0;
    for (ull t = blockIdx.x * (ull)blockDim.x + threadIdx.x; t < total;
         t += (ull)gridDim.x * blockDim.x) {
        const long long o = upper_bound_dev(g.ccnt, nop + 1, t) - 1;
        const ull rank = t - g.ccnt[o];
        const int u = (int)(upper_bound_dev(g.ooff, (long long)p + 1, o) - 1);
        const int j = (int)(o - g.ooff[u]);
        const int v = g.nbr[(long long)u * p + j];
        const int d = g.deg[u] - 1;
        const int k = d - l;
        const int side = u > v;
        const int a = min(u, v), b = max(u, v);
        const ull key = ((ull)side << 62) | rank;
        ull *bp = g.best + (long long)a * p + b;
        if (*(volatile ull *)bp < key) continue;
        const ull T = g.binom[(long long)d * (p + 1) + l];
        int posR[KC_MAX];
        unrank_lex(T - 1 - rank, d, k, g.binom, p + 1, posR);   // complement of lex is reverse lex
        const double *P = g.prec + (long long)u * PREC_MAX * PREC_MAX;
        const short *ps = g.prec_pos + (long long)u * p;
        const int su = ps[u], sv = ps[v];
        int sr[KC_MAX];
        for (int i = 0; i < k; ++i) {
            int x = posR[i];
            sr[i] = ps[g.nbr[(long long)u * p + x + (x >= j)]];
        }
        double L[KC_MAX][KC_MAX], yu[KC_MAX], yv[KC_MAX];
        bool bad = false;
        for (int i = 0; i < k && !bad; ++i) {
            for (int c = 0; c <= i; ++c) {
                double s = P[sr[i] * PREC_MAX + sr[c]];
                for (int q = 0; q < c; ++q) s -= L[i][q] * L[c][q];
                if (c == i) {
                    if (!(s > 0.0)) { bad = true; break; }
                    L[i][i] = sqrt(s);
                } else {
                    L[i][c] = s / L[c][c];
                }
            }
            if (bad) break;
            double su_ = P[sr[i] * PREC_MAX + su], sv_ = P[sr[i] * PREC_MAX + sv];
            for (int q = 0; q < i; ++q) {
                su_ -= L[i][q] * yu[q];
                sv_ -= L[i][q] * yv[q];
            }
            yu[i] = su_ / L[i][i];
            yv[i] = sv_ / L[i][i];
        }
        double Quu = P[su * PREC_MAX + su], Qvv = P[sv * PREC_MAX + sv], Quv = P[su * PREC_MAX + sv];
        for (int i = 0; i < k; ++i) {
            Quu -= yu[i] * yu[i];
            Qvv -= yv[i] * yv[i];
            Quv -= yu[i] * yv[i];
        }
        const double det = Quu * Qvv - Quv * Quv;
        const double h11 = Qvv / det, h22 = Quu / det;
        bool ind;
        if (bad || !(h11 > DEGEN) || !(h22 > DEGEN) || !(det > 0.0)) {
            ind = true;
            ++ndg;
        } else {
            const double r = -Quv / sqrt(Quu * Qvv);
            const double z = fabs(r) < 1.0 ? sq * fabs(atanh(r)) : INFINITY;
            ind = z <= tp.q;
        }
        ++nt;
        nfl += (ull)(k * k * k) / 3 + 2ull * k * k + 6ull * k + 20;
        if (ind) atomicMin(bp, key);
    }
    if (nt) {
        atomicAdd(&g.ctr->tests_executed, nt);
        atomicAdd(&g.ctr->complement_tests, nt);
        atomicAdd(&g.ctr->flops_comp, nfl);
    }
    if (ndg) atomicAdd(&g.ctr->degenerate, ndg);
}

// ---------------------------------------------------------------- neighbourhood precision blocks
__global__ void __launch_bounds__(512) prec_build_kernel(GraphDev g, const double *C64, int ldc)
{
    const int u = blockIdx.x;
    if (!g.prec_need[u]) return;
    extern __shared__ double smd[];
    __shared__ int mem[PREC_MAX];
    __shared__ int bad;
    const int p = g.p;
    const int m = g.deg[u] + 1;
    if (threadIdx.x == 0) {
        bad = 0;
        int i = 0, o = 0;
        const int *nb = g.nbr + (long long)u * p;
        const int dg = g.deg[u];
        bool placed = false;
        for (; i < dg; ++i) {
            if (!placed && nb[i] > u) {
                mem[o++] = u;
                placed = true;
            }
            mem[o++] = nb[i];
        }
        if (!placed) mem[o++] = u;
    }
    __syncthreads();
    double *A = smd, *colk = A + m * m, *rowk = colk + m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, c = e - i * m;
        A[e] = C64[(long long)mem[i] * ldc + mem[c]];
    }
    __syncthreads();
    gj_inverse_block(A, m, m, colk, rowk, &bad);
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            g.prec_m[u] = -1;
            g.prec_need[u] = 0;
        }
        return;
    }
    double *P = g.prec + (long long)u * PREC_MAX * PREC_MAX;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, c = e - i * m;
        P[i * PREC_MAX + c] = A[e];
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        g.prec_mem[(long long)u * PREC_MAX + i] = mem[i];
        g.prec_pos[(long long)u * p + mem[i]] = (short)i;
    }
    if (threadIdx.x == 0) {
        g.prec_m[u] = m;
        g.prec_need[u] = 0;
        atomicAdd(&g.ctr->flops_prec, 2ull * (ull)m * m * m);
    }
}

// Remove the neighbours a stage deleted from each maintained block:
// P <- P - P[:,w] P[w,:] / P_ww drops w (inverse of a principal submatrix).
__global__ void __launch_bounds__(512) prec_downdate_kernel(GraphDev g)
{
    const int u = blockIdx.x;
    const int m = g.prec_m[u];
    if (m <= 0) return;
    __shared__ double colw[PREC_MAX];
    const int p = g.p;
    double *P = g.prec + (long long)u * PREC_MAX * PREC_MAX;
    const int *mem = g.prec_mem + (long long)u * PREC_MAX;
    short *pos = g.prec_pos + (long long)u * p;
    const uint32_t *row = g.adj + (long long)u * g.W;
    ull fl = 0;
    for (int s = 0; s < m; ++s) {
        const int w = mem[s];
        if (w == u || pos[w] < 0) continue;
        if ((row[w >> 5] >> (w & 31)) & 1u) continue;   // still adjacent
        for (int i = threadIdx.x; i < m; i += blockDim.x) colw[i] = P[i * PREC_MAX + s];
        __syncthreads();
        const double ipww = 1.0 / colw[s];
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = e / m, c = e - i * m;
            if (i != s && c != s) P[i * PREC_MAX + c] -= colw[i] * colw[c] * ipww;
        }
        __syncthreads();
        if (threadIdx.x == 0) pos[w] = -1;
        fl += 2ull * m * m;
        __syncthreads();
    }
    if (threadIdx.x == 0 && fl) atomicAdd(&g.ctr->flops_prec, fl);
}

// ---------------------------------------------------------------- commit
__global__ void commit_kernel(GraphDev g, int l, int explicit_sets, int count_canonical)
{
    const long long nop = g.info->n_opairs;
    const int p = g.p;
    ull removed = 0, canon = 0;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nop;
         o += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(upper_bound_dev(g.ooff, (long long)p + 1, o) - 1);
        const int j = (int)(o - g.ooff[u]);
        const int v = g.nbr[(long long)u * p + j];
        if (u > v) continue;
        const long long e = (long long)u * p + v;
        const ull key = g.best[e];
        const int jv = lower_bound_int(g.nbr + (long long)v * p, g.deg[v], u);
        const long long o2 = g.ooff[v] + jv;
        if (count_canonical) {
            const ull T0 = (g.tcnt[o + 1] - g.tcnt[o]) + (g.ccnt[o + 1] - g.ccnt[o]);
            const ull T1 = (g.tcnt[o2 + 1] - g.tcnt[o2]) + (g.ccnt[o2 + 1] - g.ccnt[o2]);
            ull c;
            if (key == KEY_NONE) c = sat_add(T0, T1);
            else if ((key >> 62) == 0) c = key + 1;
            else c = sat_add(T0, (key & ((1ull << 62) - 1)) + 1);
            canon = sat_add(canon, c);
        }
        if (key == KEY_NONE) continue;
        atomicAnd(g.adj + (long long)u * g.W + (v >> 5), ~(1u << (v & 31)));
        atomicAnd(g.adj + (long long)v * g.W + (u >> 5), ~(1u << (u & 31)));
        const int side = (int)(key >> 62);
        const ull rank = key & ((1ull << 62) - 1);
        g.sep_level[e] = l;
        g.sep_side[e] = side;
        g.sep_rank[e] = (long long)rank;
        ++removed;
        if (explicit_sets) {
            const ull off = atomicAdd(&g.ctr->pool_len, (ull)l);
            g.sep_off[e] = (long long)off;
            if ((long long)(off + l) > g.pool_cap) {
                g.ctr->status = 8;
                continue;
            }
            const int su = side ? v : u;
            const int jj = side ? jv : j;
            const int dd = g.deg[su] - 1;
            const int *nb = g.nbr + (long long)su * p;
            ull r = rank;
            int x = 0;
            for (int i = 0; i < l; ++i) {
                while (x < dd - (l - i)) {
                    ull c = g.binom[(long long)(dd - x - 1) * (p + 1) + (l - i - 1)];
                    if (r < c) break;
                    r -= c;
                    ++x;
                }
                g.pool[off + i] = nb[x + (x >= jj)];
                ++x;
            }
        } else {
            g.sep_off[e] = -1;
        }
    }
    if (removed) atomicAdd(&g.ctr->edges_removed, removed);
    if (canon) atomicAdd(&g.ctr->tests_canonical, canon);
}

// ---------------------------------------------------------------- raw batches
template <bool F64>
__global__ void __launch_bounds__(256) ci_list_kernel(const int *ij, const int *S, int l, long long b,
                                                      const float *C32, const double *C64, int ldc,
                                                      int p, TestParams tp, double *r_out,
                                                      uint8_t *indep_out, float *z_out,
                                                      DevCounters *ctr, int ms, int per_warp_bytes)
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
        if (!okid) {
            if (lane == 0) ctr->status = 1;
            __syncwarp();
            continue;
        }
        double r;
        float z;
        ++acc.tests;
        bool ind = warp_test<F64>(nd, m, l, C32, C64, ldc, tp, sq, sqf, Mbuf, ms, acc, r, z);
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

cudaError_t launch_level_degrees(GraphDev g, cudaStream_t s)
{
    degrees_kernel<<<(g.p * 32 + 255) / 256, 256, 0, s>>>(g); note_launch();
    ooff_kernel<<<1, 1024, 0, s>>>(g); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prec_need(GraphDev g, TestParams tp, int l, cudaStream_t s)
{
    prec_need_kernel<<<(g.p + 255) / 256, 256, 0, s>>>(g, tp, l); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_level_counts(GraphDev g, TestParams tp, int l, long long n_opairs_cap,
                                void *scan_ws, cudaStream_t s)
{
    long long cap = n_opairs_cap > 0 ? n_opairs_cap : 1;
    int blocks = (int)std::min<long long>((cap + 255) / 256, (long long)num_sms() * 16);
    counts_kernel<<<blocks, 256, 0, s>>>(g, tp, l); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_u64(g.tcnt, &g.info->n_opairs, cap, scan_ws, &g.info->total_direct, s);
    if (e != cudaSuccess) return e;
    return scan_u64(g.ccnt, &g.info->n_opairs, cap, scan_ws, &g.info->total_comp, s);
}

static void direct_shape(int l, int &ms, int &per_warp, int &wpc)
{
    const int m = l + 2;
    ms = m + 1;
    per_warp = (int)(((size_t)m * ms * sizeof(double) + 2 * (size_t)m * sizeof(int) + 15) / 16 * 16);
    wpc = 8;
    while (wpc > 1 && (size_t)wpc * per_warp > 96 * 1024) wpc >>= 1;
}

cudaError_t launch_ci_direct(GraphDev g, TestParams tp, int l, const float *C32,
                             const double *C64, int ldc, cudaStream_t s)
{
    int ms, per_warp, wpc;
    direct_shape(l, ms, per_warp, wpc);
    size_t smem = (size_t)wpc * per_warp;
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    int blocks = num_sms() * (wpc >= 8 ? 8 : 16 / wpc + 1);
    cudaError_t e;
    if (tp.precision == 0) {
        e = cudaFuncSetAttribute(ci_direct_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_direct_kernel<true><<<blocks, wpc * 32, smem, s>>>(g, tp, l, C32, C64, ldc, ms, per_warp); note_launch();
    } else {
        e = cudaFuncSetAttribute(ci_direct_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_direct_kernel<false><<<blocks, wpc * 32, smem, s>>>(g, tp, l, C32, C64, ldc, ms, per_warp); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_ci_complement(GraphDev g, TestParams tp, int l, cudaStream_t s)
{
    ci_complement_kernel<<<num_sms() * 8, 128, 0, s>>>(g, tp, l); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prec_build(GraphDev g, const double *C64, int ldc, cudaStream_t s)
{
    int mmax = std::min(g.p + 1, PREC_MAX);
    size_t smem = ((size_t)mmax * mmax + 2 * (size_t)mmax) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(prec_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    prec_build_kernel<<<g.p, 512, smem, s>>>(g, C64, ldc); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prec_downdate(GraphDev g, cudaStream_t s)
{
    prec_downdate_kernel<<<g.p, 512, 0, s>>>(g); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_commit(GraphDev g, TestParams tp, int l, long long n_opairs_cap,
                          int explicit_sets, cudaStream_t s)
{
    (void)tp;
    long long cap = n_opairs_cap > 0 ? n_opairs_cap : 1;
    int blocks = (int)std::min<long long>((cap + 255) / 256, (long long)num_sms() * 16);
    commit_kernel<<<blocks, 256, 0, s>>>(g, l, explicit_sets, explicit_sets); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ci_list(const int *ij, const int *S, int l, long long b, const float *C32,
                           const double *C64, int ldc, int p, TestParams tp, double *r_out,
                           uint8_t *indep_out, float *z_out, DevCounters *ctr, cudaStream_t s)
{
    int ms, per_warp, wpc;
    direct_shape(l, ms, per_warp, wpc);
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
                                                           indep_out, z_out, ctr, ms, per_warp); note_launch();
    } else {
        e = cudaFuncSetAttribute(ci_list_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ci_list_kernel<false><<<blocks, wpc * 32, smem, s>>>(ij, S, l, b, C32, C64, ldc, p, tp, r_out,
                                                            indep_out, z_out, ctr, ms, per_warp); note_launch();
    }
    return cudaGetLastError();
}

}  // namespace fpc
