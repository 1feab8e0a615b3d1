// device_util.cuh -- small device helpers shared by the kernels of libfastpc.
#pragma once
#include "internal.h"

namespace fpc {

// Index of the pair (a, c) in a per-pair array, of a's neighbour list, and of
// the entry (a, c) of a correlation matrix (see GraphDev::prow).
__device__ __forceinline__ long long pidx(const GraphDev &g, int a, int c)
{
    return g.prow ? __ldg(g.prow + a) + c : (long long)a * g.p + c;
}
__device__ __forceinline__ long long nidx(const GraphDev &g, int a)
{
    return g.nrow ? __ldg(g.nrow + a) : (long long)a * g.p;
}
__device__ __forceinline__ long long cidx(const long long *prow, int ldc, int a, int c)
{
    return prow ? __ldg(prow + a) + c : (long long)a * ldc + c;
}

// 1/v for a pivot v (v > 0 in FP32 range once it passes the DEGEN floor) by two
// Newton-Raphson steps x <- x + x (1 - v x) from the FP32 reciprocal: each step
// squares the relative error (2^-23 -> 2^-46 -> below the FP64 rounding), so x is
// within two units in the last place of 1/v, without the IEEE division's slow
// path (a long FP64 sequence, and GB300's FP64 pipe is narrow) on a pivot chain.
__device__ __forceinline__ double rcp_newton(double v)
{
    double x = (double)__frcp_rn((float)v);
    x = fma(x, fma(-v, x, 1.0), x);
    x = fma(x, fma(-v, x, 1.0), x);
    return x;
}

// Symmetric sweep of every pivot of an SPD matrix in shared memory:
// A <- -A^{-1}.  Pivot k is used without row exchanges, so it equals the
// conditional variance of k given 0..k-1 (the degeneracy test of the oracle's
// elimination).  Step k: D = A_kk, A_ij -= A_ik A_kj / D (i, j != k),
// A_ik = A_ki = A_ik / D, A_kk = -1/D.  The matrix stays symmetric, so each
// thread updates one upper-triangle entry and mirrors it (m^3/2 FMAs).
// One CTA, blockDim.x a multiple of 32.  Sets *bad if a pivot is <= DEGEN.
__device__ __forceinline__ void sweep_inverse_block(double *A, int m, int lda, double *colk, int *bad)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
    for (int k = 0; k < m; ++k) {
        const double D = A[k * lda + k];
        if (!(D > DEGEN)) {
            if (threadIdx.x == 0) *bad = 1;
            return;                                   // uniform: all threads read the same pivot
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) colk[i] = A[i * lda + k];
        __syncthreads();
        const double iD = rcp_newton(D);
        for (int i = ty; i < m; i += ny) {
            const double ci = colk[i] * iD;
            for (int j = i + tx; j < m; j += 32) {
                double v;
                if (i == k) v = (j == k) ? -iD : colk[j] * iD;
                else if (j == k) v = ci;
                else v = fma(-ci, colk[j], A[i * lda + j]);
                A[i * lda + j] = v;
                A[j * lda + i] = v;
            }
        }
        __syncthreads();
    }
}

// Lexicographic unranking: positions pos[0..l) (ascending, in 0..d-1) of the
// rank-th l-subset of d items.  The number of subsets whose i-th position is
// x (positions before it fixed) is C(d-x-1, l-i-1), and by the hockey-stick
// identity those with i-th position in [x0, x1) number C(d-x0, l-i) -
// C(d-x1, l-i).  Each position is therefore either walked to (O(d) steps in
// total, best when l is close to d) or found by binary search (O(l log d)
// steps, best for small l).  binom is the (ldb x ldb) saturating table; rank
// must be < C(d, l), in which case no table entry read here saturates.
__device__ __forceinline__ void unrank_lex(unsigned long long rank, int d, int l,
                                           const unsigned long long *binom, int ldb, int *pos)
{
    int lg = 0;
    while ((1 << lg) < d + 1) ++lg;
    if (l * lg < d) {
        int x = 0;
        for (int i = 0; i < l; ++i) {
            const int r1 = l - i;                              // size of the remaining subset
            const unsigned long long base = __ldg(binom + (long long)(d - x) * ldb + r1);
            const unsigned long long target = base - rank;     // want C(d-x', r1) >= target
            int lo = x, hi = d - r1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(binom + (long long)(d - mid) * ldb + r1) >= target) lo = mid;
                else hi = mid - 1;
            }
            pos[i] = lo;
            rank -= base - __ldg(binom + (long long)(d - lo) * ldb + r1);
            x = lo + 1;
        }
        return;
    }
    int x = 0;
    for (int i = 0; i < l; ++i) {
        // x never passes d-(l-i): there C(l-i-1, l-i-1) = 1 > any valid remainder
        while (x < d - (l - i)) {
            unsigned long long c = __ldg(binom + (long long)(d - x - 1) * ldb + (l - i - 1));
            if (rank < c) break;
            rank -= c;
            ++x;
        }
        pos[i] = x++;
    }
}

// unrank_lex with the positions in a fixed-size array (l <= KM): the loops run
// to the compile-time bound with guards, so pos stays in registers.  Same
// positions as unrank_lex; entries from l on are 0.  binom (row stride ldb) may
// be a shared-memory copy of the table's first columns (plain loads).
template <int KM>
__device__ __forceinline__ void unrank_lex_fixed(unsigned long long rank, int d, int l,
                                                 const unsigned long long *binom, int ldb, int (&pos)[KM])
{
    int lg = 0;
    while ((1 << lg) < d + 1) ++lg;
    const bool search = l * lg < d;
    int x = 0;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        pos[i] = 0;
        if (i >= l) continue;
        const int r1 = l - i;                                  // size of the remaining subset
        if (search) {
            const unsigned long long base = binom[(long long)(d - x) * ldb + r1];
            const unsigned long long target = base - rank;
            int lo = x, hi = d - r1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (binom[(long long)(d - mid) * ldb + r1] >= target) lo = mid;
                else hi = mid - 1;
            }
            pos[i] = lo;
            rank -= base - binom[(long long)(d - lo) * ldb + r1];
            x = lo + 1;
        } else {
            while (x < d - r1) {
                const unsigned long long c = binom[(long long)(d - x - 1) * ldb + (r1 - 1)];
                if (rank < c) break;
                rank -= c;
                ++x;
            }
            pos[i] = x++;
        }
    }
}

// Ascending sort of a fixed-size register array (odd-even transposition
// network: compile-time indices only).
template <int KM>
__device__ __forceinline__ void sort_fixed(int (&a)[KM])
{
#pragma unroll
    for (int r = 0; r < KM; ++r)
#pragma unroll
        for (int i = r & 1; i + 1 < KM; i += 2) {
            const int x = a[i], y = a[i + 1];
            a[i] = min(x, y);
            a[i + 1] = max(x, y);
        }
}

// First index i in [0, len) with a[i] > key (len if none).
template <typename T>
__device__ __forceinline__ long long upper_bound_dev(const T *a, long long len, T key)
{
    long long lo = 0, hi = len;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (a[mid] > key) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// First index i in [0, len) with a[i] >= key.
__device__ __forceinline__ int lower_bound_int(const int *a, int len, int key)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void atomic_max_float_pos(unsigned int *addr, float v)
{
    // v >= 0: IEEE order equals unsigned order of the bit patterns
    atomicMax(addr, __float_as_uint(v));
}

}  // namespace fpc
