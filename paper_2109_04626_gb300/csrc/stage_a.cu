// stage_a.cu -- the first stage of Algorithm 2 (l = p-2) in closed form.
// On the complete graph the only conditioning set of {u,v} is V\{u,v}; the
// Schur complement of Sec. 4 is then the inverse of the {u,v} block of
// P = corr^{-1}, so r_uv = -P_uv / sqrt(P_uu P_vv) and one FP64 inverse of
// corr decides every pair.
#include "internal.h"
#include "device_util.cuh"

#include <cooperative_groups.h>

namespace fpc {

namespace cg = cooperative_groups;

// The same symmetric sweep (A <- -A^{-1}, pivots in order, no exchanges) on a
// cluster of SA_CLUSTER CTAs, with one cluster barrier per sb pivots.  CTA r
// holds rows [r*rpc, (r+1)*rpc) in shared memory.  At the start of a group of
// pivots k0..k0+b-1 every CTA copies those rows (= columns, A stays symmetric), as
// their owners published them, through distributed shared memory; it then applies
// the group's pivots one after the other to its own rows and to its copies of
// the group's later rows -- the same operations on the same operands as their
// owners, so every copy of row k is the owner's row k when pivot k uses it.  The
// owners of the next group's rows publish them into the other of two buffers, and
// one cluster barrier ends the group (a reader of buffer g%2 is done with it
// before the barrier; it is written again only after the next one).  Each entry
// (i, j) is computed with the operands the one-CTA sweep uses for the pair {i, j},
// so the result is bit-identical to it; GB300's FP64 rate (about 2 FMA per clock
// per SM) is what the cluster multiplies, and the groups cut the barriers.
constexpr int SA_CLUSTER = 8;
constexpr int SA_SB_MAX = 8;
__global__ void __cluster_dims__(SA_CLUSTER, 1, 1) __launch_bounds__(256)
    inverse_cluster_kernel(double *A, int m, int lda, int sb, int *singular)
{
    extern __shared__ double smc[];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int rpc = (m + SA_CLUSTER - 1) / SA_CLUSTER;
    const int i0 = min(m, r * rpc), i1 = min(m, i0 + rpc), nr = i1 - i0;
    double *R = smc;                                   // own rows, row-major, m per row
    double *Pn = R + (size_t)rpc * m;                  // the group's rows, sb x m
    double *bc = Pn + (size_t)sb * m;                  // two broadcast buffers of sb rows (own rows only)
    for (int e = threadIdx.x; e < nr * m; e += blockDim.x) R[e] = A[(long long)(i0 + e / m) * lda + e % m];
    __syncthreads();
    for (int e = threadIdx.x; e < sb * m; e += blockDim.x) {       // own rows of group 0
        const int row = e / m;
        if (row < m && row >= i0 && row < i1) bc[e] = R[(size_t)(row - i0) * m + e % m];
    }
    bool bad = false;
    cl.sync();
    const int ng = (m + sb - 1) / sb;
    for (int gi = 0; gi < ng && !bad; ++gi) {
        const int k0 = gi * sb, b = min(sb, m - k0);
        const size_t buf = (size_t)(gi & 1) * sb * m;
        for (int e = threadIdx.x; e < b * m; e += blockDim.x)
            Pn[e] = cl.map_shared_rank(bc, (k0 + e / m) / rpc)[buf + e];
        __syncthreads();
        for (int q = 0; q < b; ++q) {
            const int k = k0 + q;
            const double *colk = Pn + (size_t)q * m;   // row k after pivots < k
            const double D = colk[k];
            if (!(D > DEGEN)) {                        // the same pivot in every CTA: a uniform exit
                bad = true;
                break;
            }
            const double iD = rcp_newton(D);
            // own rows, then the copies of the group's later rows, by the same formula:
            // a warp per row, lanes over its columns (no index division per entry)
            const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            const int nrows = nr + (b - 1 - q);
            for (int rr = threadIdx.x >> 5; rr < nrows; rr += nw) {
                const bool own = rr < nr;
                const int i = own ? i0 + rr : k + 1 + (rr - nr);
                double *row = own ? R + (size_t)rr * m : Pn + (size_t)(q + 1 + rr - nr) * m;
                const double ci = colk[i] * iD;
                for (int j = lane; j < m; j += 32) {
                    double v;
                    if (i == k) v = (j == k) ? -iD : colk[j] * iD;
                    else if (j == k) v = ci;
                    else if (i <= j) v = fma(-ci, colk[j], row[j]);
                    else v = fma(-(colk[j] * iD), colk[i], row[j]);
                    row[j] = v;
                }
            }
            __syncthreads();
        }
        if (!bad && gi + 1 < ng) {                     // publish own rows of the next group
            const int n0 = k0 + sb, nb2 = min(sb, m - n0);
            const size_t nbuf = (size_t)((gi + 1) & 1) * sb * m;
            for (int e = threadIdx.x; e < nb2 * m; e += blockDim.x) {
                const int row = n0 + e / m;
                if (row >= i0 && row < i1) bc[nbuf + e] = R[(size_t)(row - i0) * m + e % m];
            }
        }
        cl.sync();
    }
    cl.sync();                                         // no CTA leaves while another reads its buffers
    if (bad) {
        if (r == 0 && threadIdx.x == 0) *singular = 1;
        return;
    }
    for (int e = threadIdx.x; e < nr * m; e += blockDim.x) A[(long long)(i0 + e / m) * lda + e % m] = -R[e];
}

__global__ void __launch_bounds__(1024) inverse_smem_kernel(double *A, int m, int lda, int *singular)
{
    extern __shared__ double sm[];
    double *S = sm;                       // m x m
    double *colk = S + m * m;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) S[e] = A[(e / m) * (long long)lda + e % m];
    __syncthreads();
    sweep_inverse_block(S, m, m, colk, &bad);     // S = -A^{-1}
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) *singular = 1;
        return;
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) A[(e / m) * (long long)lda + e % m] = -S[e];
}

// Large m: one pivot per pair of launches, A in global memory.
__global__ void gj_save_kernel(const double *A, int m, int lda, int k, double *colk, double *rowk,
                               int *singular)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        colk[i] = A[(long long)i * lda + k];
        rowk[i] = A[(long long)k * lda + i];
    }
    if (i == 0 && !(A[(long long)k * lda + k] > DEGEN)) *singular = 1;
}

__global__ void gj_update_kernel(double *A, int m, int lda, int k, const double *colk,
                                 const double *rowk, const int *singular)
{
    if (*singular) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= m) return;
    const double ip = rcp_newton(rowk[k]);
    double v;
    if (i == k) v = (j == k) ? ip : rowk[j] * ip;
    else if (j == k) v = -colk[i] * ip;
    else v = A[(long long)i * lda + j] - colk[i] * rowk[j] * ip;
    A[(long long)i * lda + j] = v;
}

cudaError_t launch_inverse_spd(double *A, int m, int lda, double *work, int *singular,
                               cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(singular, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    // a cluster of SA_CLUSTER CTAs when the rows fit their shared memory, with the
    // largest block of pivots per barrier that fits beside them
    const size_t rpc = (size_t)(m + SA_CLUSTER - 1) / SA_CLUSTER;
    int sb = SA_SB_MAX;
    auto smem_of = [&](int b) { return (rpc * m + 3 * (size_t)b * m) * sizeof(double); };
    while (sb > 1 && smem_of(sb) > 200 * 1024) sb >>= 1;
    const size_t smem_c = smem_of(sb);
    if (m >= 32 && smem_c <= 200 * 1024) {
        e = cudaFuncSetAttribute(inverse_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
        if (e != cudaSuccess) return e;
        inverse_cluster_kernel<<<SA_CLUSTER, 256, smem_c, s>>>(A, m, lda, sb, singular); note_launch();
        return cudaGetLastError();
    }
    size_t smem = ((size_t)m * m + (size_t)m) * sizeof(double);
    if (smem <= 220 * 1024) {
        e = cudaFuncSetAttribute(inverse_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        inverse_smem_kernel<<<1, 1024, smem, s>>>(A, m, lda, singular); note_launch();
        return cudaGetLastError();
    }
    double *colk = work, *rowk = work + m;
    for (int k = 0; k < m; ++k) {
        gj_save_kernel<<<(m + 255) / 256, 256, 0, s>>>(A, m, lda, k, colk, rowk, singular); note_launch();
        gj_update_kernel<<<dim3((m + 255) / 256, m), 256, 0, s>>>(A, m, lda, k, colk, rowk,
                                                                   singular); note_launch();
    }
    return cudaGetLastError();
}

// Decide every pair {a<b} from P: h11 = P_bb/det, h22 = P_aa/det (the Schur
// complement of the pair given the rest), r = -P_ab/sqrt(P_aa P_bb),
// z = sqrt(n-p-1)|atanh r|; independent (or degenerate) pairs get key 0.
__global__ void stage_a_decide_kernel(const double *P, int p, int ldp, const int *singular,
                                      GraphDev g, TestParams tp)
{
    if (*singular) return;                 // corr numerically singular: the stage is skipped
    unsigned long long nt = 0, ndg = 0;
    const double sq = sqrt((double)(tp.n - p - 1));
    for (int a = blockIdx.y; a < p; a += gridDim.y)
        for (int b = a + 1 + blockIdx.x * blockDim.x + threadIdx.x; b < p;
             b += gridDim.x * blockDim.x) {
            double paa = P[(long long)a * ldp + a], pbb = P[(long long)b * ldp + b];
            double pab = P[(long long)a * ldp + b];
            double det = paa * pbb - pab * pab;
            double h11 = pbb / det, h22 = paa / det;
            bool degen = !(h11 > DEGEN) || !(h22 > DEGEN);
            bool ind;
            if (degen) {
                ind = true;
                ++ndg;
            } else {
                double r = -pab / sqrt(paa * pbb);
                double z = fabs(r) < 1.0 ? sq * fabs(atanh(r)) : INFINITY;
                ind = z <= tp.q;
            }
            ++nt;
            if (ind) g.best[pidx(g, a, b)] = 0ull;
        }
    if (nt) {
        atomicAdd(&g.ctr->tests_executed, nt);
        atomicAdd(&g.ctr->tests_canonical, nt);
        atomicAdd(&g.ctr->flops_stagea, nt * 12ull);
    }
    if (ndg) atomicAdd(&g.ctr->degenerate, ndg);
}

cudaError_t launch_stage_a_decide(const double *P, int p, int ldp, const int *singular,
                                  GraphDev g, TestParams tp, cudaStream_t s)
{
    dim3 grid((p + 255) / 256, p);
    stage_a_decide_kernel<<<grid, 256, 0, s>>>(P, p, ldp, singular, g, tp); note_launch();
    return cudaGetLastError();
}

}  // namespace fpc
