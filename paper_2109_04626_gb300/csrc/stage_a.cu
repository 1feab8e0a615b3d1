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
// cluster of SA_CLUSTER CTAs: CTA r holds rows [r*rpc, (r+1)*rpc) in shared
// memory.  At pivot k every CTA copies row k (= column k, A stays symmetric) from
// its owner's broadcast buffer through distributed shared memory and updates its
// own rows; the owner of row k+1 then publishes that row into the other of its two
// buffers, and one cluster barrier ends the pivot (a reader of buffer k%2 is done
// with it before the barrier; it is written again only after the next one).  Each
// entry (i, j) is computed with the operands the one-CTA sweep uses for the pair
// {i, j}, so the result is bit-identical to it; GB300's FP64 rate (about 2 FMA per
// clock per SM) is what the cluster multiplies.
constexpr int SA_CLUSTER = 8;
__global__ void __cluster_dims__(SA_CLUSTER, 1, 1) __launch_bounds__(256)
    inverse_cluster_kernel(double *A, int m, int lda, int *singular)
{
    extern __shared__ double smc[];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int rpc = (m + SA_CLUSTER - 1) / SA_CLUSTER;
    const int i0 = min(m, r * rpc), i1 = min(m, i0 + rpc), nr = i1 - i0;
    double *R = smc;                                   // own rows, row-major, m per row
    double *colk = smc + (size_t)rpc * m;              // this CTA's copy of row k
    double *bc = colk + m;                             // two broadcast rows (the owner's)
    for (int e = threadIdx.x; e < nr * m; e += blockDim.x) R[e] = A[(long long)(i0 + e / m) * lda + e % m];
    __syncthreads();
    if (i0 == 0 && nr > 0)
        for (int j = threadIdx.x; j < m; j += blockDim.x) bc[j] = R[j];
    bool bad = false;
    cl.sync();
    for (int k = 0; k < m; ++k) {
        const int owner = k / rpc;
        const double *rowk = cl.map_shared_rank(bc, owner) + (size_t)(k & 1) * m;
        for (int j = threadIdx.x; j < m; j += blockDim.x) colk[j] = rowk[j];
        __syncthreads();
        const double D = colk[k];
        if (!(D > DEGEN)) {                            // the same pivot in every CTA: a uniform exit
            bad = true;
            break;
        }
        const double iD = rcp_newton(D);
        for (int e = threadIdx.x; e < nr * m; e += blockDim.x) {
            const int i = i0 + e / m, j = e - (e / m) * m;
            double v;
            if (i == k) v = (j == k) ? -iD : colk[j] * iD;
            else if (j == k) v = colk[i] * iD;
            else if (i <= j) v = fma(-(colk[i] * iD), colk[j], R[e]);
            else v = fma(-(colk[j] * iD), colk[i], R[e]);
            R[e] = v;
        }
        __syncthreads();
        if (k + 1 < m && k + 1 >= i0 && k + 1 < i1)      // publish row k+1, as updated by pivot k
            for (int j = threadIdx.x; j < m; j += blockDim.x)
                bc[(size_t)((k + 1) & 1) * m + j] = R[(size_t)(k + 1 - i0) * m + j];
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
    // a cluster of SA_CLUSTER CTAs when the rows fit their shared memory (at m = 95 it
    // takes 0.29 ms against 0.46 ms for the one-CTA sweep)
    const size_t smem_c = ((size_t)((m + SA_CLUSTER - 1) / SA_CLUSTER) * m + 3 * (size_t)m) * sizeof(double);
    if (m >= 32 && smem_c <= 200 * 1024) {
        e = cudaFuncSetAttribute(inverse_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
        if (e != cudaSuccess) return e;
        inverse_cluster_kernel<<<SA_CLUSTER, 256, smem_c, s>>>(A, m, lda, singular); note_launch();
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
