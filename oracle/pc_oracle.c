/*
 * pc_oracle.c -- plain, slow FP64 CPU oracle for the PC-stable skeleton search
 * of "A Fast PC Algorithm with Reversed-order Pruning and A Parallelization
 * Strategy" (Zhang, Tian, Johnson, Zhang, Jiang; arXiv 2109.04626).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every routine states the passage of the paper it follows.  Readings of
 * passages that are silent, garbled or ambiguous are marked "Reading Rn".
 *
 * Arithmetic is IEEE FP64 throughout.  Loops follow the paper's order; the
 * only parallelism is OpenMP over the (frozen, hence independent) edges of
 * one PC-stable level, which changes no result (Sec. 2.2.2: PC-stable defers
 * deletions to the end of a stage, so tests within a stage see the same graph).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_REVERSED        1   /* Algorithm 2 schedule (l descending)        */
#define ORACLE_NONSTABLE       2   /* Algorithm 1/2 with stable = False           */
#define ORACLE_ONESIDED_I      4   /* test S from adj(i)\{j} only, i<j            */
#define ORACLE_ONESIDED_J      8   /* test S from adj(j)\{i} only, i<j            */
#define ORACLE_STAGEA_GENERIC 16   /* reversed: run l=p-2 through enumeration     */
#define ORACLE_NO_STAGEA      32   /* reversed: skip the l=p-2 stage entirely     */
#define ORACLE_POPULATION     64   /* CI by |r| <= tol instead of Fisher z        */
#define ORACLE_PATHPOOL      128   /* one pool per pair: adj(G,a,b) on a-b paths  */

/* Degeneracy floor (Reading R8): a conditional variance at or below this
 * value means the variable is (numerically) determined by the conditioning
 * set; such a test is declared independent with r := 0. */
#define ORACLE_DEGEN 1e-12

/* ------------------------------------------------------------------------ */
/* Inverse standard normal CDF: Wichura (1988), Algorithm AS 241 (PPND16),
 * Applied Statistics 37(3):477-484.  Used for the threshold
 * Phi^{-1}(1 - alpha/2) of the Fisher-z test (Sec. 2.2.2, Eq. 1 and the
 * rule that replaces the independence query of Algorithm 1).             */
double oracle_norm_ppf(double p)
{
    static const double a[8] = {
        3.3871328727963666080e0, 1.3314166789178437745e+2,
        1.9715909503065514427e+3, 1.3731693765509461125e+4,
        4.5921953931549871457e+4, 6.7265770927008700853e+4,
        3.3430575583588128105e+4, 2.5090809287301226727e+3};
    static const double b[8] = {
        1.0, 4.2313330701600911252e+1,
        6.8718700749205790830e+2, 5.3941960214247511077e+3,
        2.1213794301586595867e+4, 3.9307895800092710610e+4,
        2.8729085735721942674e+4, 5.2264952788528545610e+3};
    static const double c[8] = {
        1.42343711074968357734e0, 4.63033784615654529590e0,
        5.76949722146069140550e0, 3.64784832476320460504e0,
        1.27045825245236838258e0, 2.41780725177450611770e-1,
        2.27238449892691845833e-2, 7.74545014278341407640e-4};
    static const double d[8] = {
        1.0, 2.05319162663775882187e0,
        1.67638483018380384940e0, 6.89767334985100004550e-1,
        1.48103976427480074590e-1, 1.51986665636164571966e-2,
        5.47593808499534494600e-4, 1.05075007164441684324e-9};
    static const double e[8] = {
        6.65790464350110377720e0, 5.46378491116411436990e0,
        1.78482653991729133580e0, 2.96560571828504891230e-1,
        2.65321895265761230930e-2, 1.24266094738807843860e-3,
        2.71155556874348757815e-5, 2.01033439929228813265e-7};
    static const double f[8] = {
        1.0, 5.99832206555887937690e-1,
        1.36929880922735805310e-1, 1.48753612908506148525e-2,
        7.86869131145613259100e-4, 1.84631831751005468180e-5,
        1.42151175831644588870e-7, 2.04426310338993978564e-15};
    const double *num, *den;
    double q = p - 0.5, r, x, val;
    if (!(p > 0.0 && p < 1.0)) return NAN;
    if (fabs(q) <= 0.425) {
        r = 0.180625 - q * q;
        num = a; den = b; x = r;
        val = 0.0;
        double nn = 0.0, dd = 0.0;
        for (int k = 7; k >= 0; --k) { nn = nn * x + num[k]; dd = dd * x + den[k]; }
        return q * nn / dd;
    }
    r = (q < 0.0) ? p : 1.0 - p;
    r = sqrt(-log(r));
    if (r <= 5.0) { x = r - 1.6; num = c; den = d; }
    else          { x = r - 5.0; num = e; den = f; }
    {
        double nn = 0.0, dd = 0.0;
        for (int k = 7; k >= 0; --k) { nn = nn * x + num[k]; dd = dd * x + den[k]; }
        val = nn / dd;
    }
    return (q < 0.0) ? -val : val;
}

/* ------------------------------------------------------------------------ */
/* Pearson correlation matrix corr = {rho_ij} (Sec. 4, definition of corr),
 * by two-pass summation: column means first, then centred cross products.
 * X is row-major n x p.  C is row-major p x p with the diagonal set to 1.
 * Reading R18: a constant column (zero sum of squares) has correlation 0 with
 * every other column (its standardised values are all zero).               */
void oracle_pearson(const double *X, int64_t n, int32_t p, double *C)
{
    double *D = (double *)malloc(sizeof(double) * (size_t)n * (size_t)p);
    double *ss = (double *)malloc(sizeof(double) * (size_t)p);
    for (int32_t a = 0; a < p; ++a) {
        double s = 0.0;
        for (int64_t t = 0; t < n; ++t) s += X[t * p + a];
        double mu = s / (double)n;
        double q = 0.0;
        for (int64_t t = 0; t < n; ++t) {
            double dv = X[t * p + a] - mu;
            D[(size_t)a * n + t] = dv;      /* column-major centred copy */
            q += dv * dv;
        }
        ss[a] = q;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t a = 0; a < p; ++a) {
        C[(size_t)a * p + a] = 1.0;
        for (int32_t b = a + 1; b < p; ++b) {
            double s = 0.0;
            const double *da = D + (size_t)a * n, *db = D + (size_t)b * n;
            for (int64_t t = 0; t < n; ++t) s += da[t] * db[t];
            double r = (ss[a] > 0.0 && ss[b] > 0.0) ? s / sqrt(ss[a] * ss[b]) : 0.0;
            C[(size_t)a * p + b] = r;
            C[(size_t)b * p + a] = r;
        }
    }
    free(D);
    free(ss);
}

/* ------------------------------------------------------------------------ */
/* Partial correlation r_{uv.S} from the Schur complement of Sec. 4:
 *   H = H0 - H1 H2^{-1} H1^T,   rho = h12 / sqrt(h11 h22),
 * with H0 = corr[{u,v},{u,v}], H1 = corr[{u,v},S], H2 = corr[S,S].
 * H2^{-1} H1^T is formed by Gauss-Jordan elimination on [H2 | H1^T].
 * H2 is a principal block of a correlation matrix (symmetric positive
 * semi-definite), so elimination runs without row exchanges (Reading R8):
 * the k-th pivot is then the conditional variance of S_k given S_1..S_{k-1}.
 * Returns 1 (degenerate) when a pivot, h11 or h22 is <= ORACLE_DEGEN, else 0.
 * ldc is the row stride of C.                                               */
int oracle_partial_corr(const double *C, int32_t ldc, int32_t u, int32_t v,
                        const int32_t *S, int32_t l, double *r_out,
                        double *h11_out, double *h22_out)
{
    int32_t w = l + 2;                    /* augmented width */
    double *A = (double *)malloc(sizeof(double) * (size_t)(l > 0 ? l : 1) * (size_t)w);
    int degen = 0;
    for (int32_t i = 0; i < l; ++i) {
        for (int32_t j = 0; j < l; ++j) A[i * w + j] = C[(size_t)S[i] * ldc + S[j]];
        A[i * w + l]     = C[(size_t)S[i] * ldc + u];
        A[i * w + l + 1] = C[(size_t)S[i] * ldc + v];
    }
    for (int32_t k = 0; k < l && !degen; ++k) {
        double piv = A[k * w + k];
        if (!(piv > ORACLE_DEGEN)) { degen = 1; break; }
        double inv = 1.0 / piv;
        for (int32_t j = 0; j < w; ++j) A[k * w + j] *= inv;
        for (int32_t i = 0; i < l; ++i) {
            if (i == k) continue;
            double f = A[i * w + k];
            if (f == 0.0) continue;
            for (int32_t j = 0; j < w; ++j) A[i * w + j] -= f * A[k * w + j];
        }
    }
    double h11 = 0, h22 = 0, h12 = 0, r = 0;
    if (!degen) {
        /* H = H0 - H1 * Y, Y = H2^{-1} H1^T = columns l, l+1 of A */
        h11 = C[(size_t)u * ldc + u];
        h22 = C[(size_t)v * ldc + v];
        h12 = C[(size_t)u * ldc + v];
        for (int32_t k = 0; k < l; ++k) {
            double cu = C[(size_t)u * ldc + S[k]], cv = C[(size_t)v * ldc + S[k]];
            double yu = A[k * w + l], yv = A[k * w + l + 1];
            h11 -= cu * yu;
            h22 -= cv * yv;
            h12 -= cu * yv;
        }
        if (!(h11 > ORACLE_DEGEN) || !(h22 > ORACLE_DEGEN)) degen = 1;
        else r = h12 / sqrt(h11 * h22);
    }
    free(A);
    if (degen) r = 0.0;
    if (r_out) *r_out = r;
    if (h11_out) *h11_out = h11;
    if (h22_out) *h22_out = h22;
    return degen;
}

/* Fisher-z statistic sqrt(n-l-3)*|arctanh r| (Eq. 1 and the rule that
 * replaces Algorithm 1's independence query; the absolute value follows that rule,
 * Reading R5).  |r| >= 1 gives +inf (dependent). */
static double fisher_z(double r, int64_t n, int32_t l)
{
    if (!(fabs(r) < 1.0)) return INFINITY;
    return sqrt((double)(n - l - 3)) * fabs(atanh(r));
}

/* One Gaussian CI test.  Independent (returns 1) iff the test is degenerate
 * or z <= q (equality counts as independent, Reading R6).  In population
 * mode (tol >= 0) the rule is |r| <= tol instead. */
int oracle_ci_test(const double *C, int32_t ldc, int64_t n, double q, double tol,
                   int32_t u, int32_t v, const int32_t *S, int32_t l,
                   double *r_out, double *z_out, int *degen_out)
{
    double r;
    int degen = oracle_partial_corr(C, ldc, u, v, S, l, &r, NULL, NULL);
    double z = degen ? 0.0 : fisher_z(r, n, l);
    int indep;
    if (degen) indep = 1;
    else if (tol >= 0.0) indep = fabs(r) <= tol;
    else indep = z <= q;
    if (r_out) *r_out = r;
    if (z_out) *z_out = z;
    if (degen_out) *degen_out = degen;
    return indep;
}

/* ------------------------------------------------------------------------ */
/* Precision matrix P = corr^{-1} by Gauss-Jordan elimination without row
 * exchanges (corr is symmetric positive definite).  Returns 1 if a pivot is
 * <= ORACLE_DEGEN (numerically singular corr), else 0. */
int oracle_precision(const double *C, int32_t p, double *P)
{
    int32_t w = 2 * p;
    double *A = (double *)malloc(sizeof(double) * (size_t)p * (size_t)w);
    for (int32_t i = 0; i < p; ++i)
        for (int32_t j = 0; j < w; ++j)
            A[(size_t)i * w + j] = (j < p) ? C[(size_t)i * p + j] : (double)(j - p == i);
    int singular = 0;
    for (int32_t k = 0; k < p; ++k) {
        double piv = A[(size_t)k * w + k];
        if (!(piv > ORACLE_DEGEN)) { singular = 1; break; }
        double inv = 1.0 / piv;
        for (int32_t j = 0; j < w; ++j) A[(size_t)k * w + j] *= inv;
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < p; ++i) {
            if (i == k) continue;
            double f = A[(size_t)i * w + k];
            if (f == 0.0) continue;
            for (int32_t j = 0; j < w; ++j) A[(size_t)i * w + j] -= f * A[(size_t)k * w + j];
        }
    }
    if (!singular)
        for (int32_t i = 0; i < p; ++i)
            for (int32_t j = 0; j < p; ++j) P[(size_t)i * p + j] = A[(size_t)i * w + p + j];
    free(A);
    return singular;
}

/* ------------------------------------------------------------------------ */
/* Skeleton search (Phase I).                                                */

typedef struct {
    int32_t p;
    int64_t n;
    uint8_t *adj;          /* p*p final skeleton                              */
    int32_t *sep_level;    /* p*p; -1 = edge kept                              */
    int32_t *sep_side;     /* 0: S from adj(min)\{max}; 1: from adj(max)\{min} */
    int64_t *sep_rank;     /* lexicographic rank of S within its side         */
    int64_t *sep_off;      /* offset into pool; -1: S = V\{u,v} (l = p-2)      */
    int32_t *pool;
    int64_t pool_len, pool_cap;
    int64_t *tests_level;  /* tests executed at each level 0..p-2             */
    int64_t *removed_level;/* edges removed at each level                     */
    int64_t tests_total;
    int64_t degenerate;
    int32_t stageA_ran;
    int32_t n_levels;      /* number of levels visited (in order)             */
    int32_t *level_seq;
} oracle_result;

static void pool_push(oracle_result *R, const int32_t *s, int32_t l)
{
    if (R->pool_len + l > R->pool_cap) {
        int64_t cap = R->pool_cap ? R->pool_cap : 1024;
        while (cap < R->pool_len + l) cap *= 2;
        R->pool = (int32_t *)realloc(R->pool, sizeof(int32_t) * (size_t)cap);
        R->pool_cap = cap;
    }
    memcpy(R->pool + R->pool_len, s, sizeof(int32_t) * (size_t)l);
    R->pool_len += l;
}

/* Neighbour lists of a graph, ascending node ids. */
static void build_nbrs(const uint8_t *adj, int32_t p, int32_t *deg, int32_t *nbr)
{
    for (int32_t u = 0; u < p; ++u) {
        int32_t d = 0;
        for (int32_t w = 0; w < p; ++w)
            if (adj[(size_t)u * p + w]) nbr[(size_t)u * p + d++] = w;
        deg[u] = d;
    }
}

/* Enumerate the size-l subsets of cand \ {excl} (cand ascending, length dc)
 * in lexicographic order of positions; stop at the first independent one.
 * Returns 1 if found (rank, positions -> nodes written to S_out).  The test
 * count is added to *ntests.  The inner search over S of Algorithms 1 and 2. */
static int search_side(const double *C, int32_t p, int64_t n, double q, double tol,
                       int32_t u, int32_t v, const int32_t *nb, int32_t dn, int32_t l,
                       int64_t *ntests, int64_t *rank_out, int32_t *S_out,
                       int64_t *ndegen)
{
    int32_t cand[dn > 0 ? dn : 1];
    int32_t d = 0;
    for (int32_t k = 0; k < dn; ++k) if (nb[k] != v) cand[d++] = nb[k];
    if (d < l) return 0;
    int32_t idx[l > 0 ? l : 1];
    int32_t S[l > 0 ? l : 1];
    for (int32_t k = 0; k < l; ++k) idx[k] = k;
    int64_t rank = 0;
    for (;;) {
        for (int32_t k = 0; k < l; ++k) S[k] = cand[idx[k]];
        int degen = 0;
        int ind = oracle_ci_test(C, p, n, q, tol, u, v, S, l, NULL, NULL, &degen);
        ++*ntests;
        if (degen) ++*ndegen;
        if (ind) {
            *rank_out = rank;
            memcpy(S_out, S, sizeof(int32_t) * (size_t)l);
            return 1;
        }
        /* lexicographic successor of idx over {0..d-1} */
        int32_t i = l - 1;
        while (i >= 0 && idx[i] == d - l + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int32_t j = i + 1; j < l; ++j) idx[j] = idx[j - 1] + 1;
        ++rank;
    }
    return 0;
}

/* comp[x*p + k]: the connected component of node k in the frozen graph with
 * node x removed (-1 at k = x).  Depth-first over the adjacency matrix. */
static void components_without(const uint8_t *adj, int32_t p, int32_t *comp)
{
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p > 0 ? p : 1));
    for (int32_t x = 0; x < p; ++x) {
        int32_t *c = comp + (size_t)x * p;
        for (int32_t k = 0; k < p; ++k) c[k] = -1;
        int32_t id = 0;
        for (int32_t s0 = 0; s0 < p; ++s0) {
            if (s0 == x || c[s0] >= 0) continue;
            int32_t top = 0;
            stack[top++] = s0;
            c[s0] = id;
            while (top) {
                int32_t y = stack[--top];
                for (int32_t z = 0; z < p; ++z)
                    if (z != x && c[z] < 0 && adj[(size_t)y * p + z]) { c[z] = id; stack[top++] = z; }
            }
            ++id;
        }
    }
    free(stack);
}

/* The candidate pool of the pair {a,b} in the paper's notation,
 * adj(G,a,b) intersected with path(G,a,b) (Sec. 2.1 definitions, used by
 * Algorithms 1 and 2): the nodes adjacent to a or to b, other than a and b,
 * that lie on some simple a-b path of the frozen graph.  A neighbour k of a
 * lies on one iff k reaches b without passing through a (then a, k, ..., b is
 * such a path), a neighbour of b iff it reaches a without passing through b.
 * Written ascending to pool; returns its size. */
static int32_t path_pool(const uint8_t *adj, int32_t p, const int32_t *comp, int32_t a, int32_t b,
                         int32_t *pool)
{
    const int32_t *ca = comp + (size_t)a * p, *cb = comp + (size_t)b * p;
    int32_t d = 0;
    for (int32_t k = 0; k < p; ++k) {
        if (k == a || k == b) continue;
        int on = (adj[(size_t)a * p + k] && ca[k] == ca[b]) || (adj[(size_t)b * p + k] && cb[k] == cb[a]);
        if (on) pool[d++] = k;
    }
    return d;
}

/* One stage l with the adjacency frozen at its start (PC-stable: the stage
 * body of Algorithm 1 with stable = True).  Edges {a,b}, a<b, are tested on
 * side 0 (S from adj(a)\{b}) and, if that finds no separating set, side 1
 * (S from adj(b)\{a}) -- Reading R1/R2.  Deletions are applied at the end. */
static void stable_level(oracle_result *R, const double *C, uint8_t *adj, int32_t p,
                         int64_t n, double q, double tol, int32_t l, int flags)
{
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)p * (size_t)p);
    build_nbrs(adj, p, deg, nbr);
    int64_t E = 0;
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = a + 1; b < p; ++b) E += adj[(size_t)a * p + b] != 0;
    int32_t *ea = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E ? E : 1));
    int32_t *eb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E ? E : 1));
    int64_t e = 0;
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = a + 1; b < p; ++b)
            if (adj[(size_t)a * p + b]) { ea[e] = a; eb[e] = b; ++e; }
    int32_t lw = l > 0 ? l : 1;
    int32_t *found = (int32_t *)calloc((size_t)(E ? E : 1), sizeof(int32_t));
    int32_t *fside = (int32_t *)calloc((size_t)(E ? E : 1), sizeof(int32_t));
    int64_t *frank = (int64_t *)calloc((size_t)(E ? E : 1), sizeof(int64_t));
    int32_t *fS = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E ? E : 1) * (size_t)lw);
    int64_t *ft = (int64_t *)calloc((size_t)(E ? E : 1), sizeof(int64_t));
    int64_t *fd = (int64_t *)calloc((size_t)(E ? E : 1), sizeof(int64_t));
    int32_t *comp = NULL;
    if (flags & ORACLE_PATHPOOL) {
        comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)p * (size_t)p);
        components_without(adj, p, comp);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < E; ++k) {
        int32_t a = ea[k], b = eb[k];
        int64_t rank = 0;
        int got = 0;
        if (flags & ORACLE_PATHPOOL) {
            /* one pool for the pair, searched once (side 0) */
            int32_t pool[p];
            int32_t dp = path_pool(adj, p, comp, a, b, pool);
            got = search_side(C, p, n, q, tol, a, b, pool, dp, l, &ft[k], &rank, fS + (size_t)k * lw, &fd[k]);
            if (got) { found[k] = 1; fside[k] = 0; frank[k] = rank; }
            continue;
        }
        if (!(flags & ORACLE_ONESIDED_J))
            got = search_side(C, p, n, q, tol, a, b, nbr + (size_t)a * p, deg[a], l,
                              &ft[k], &rank, fS + (size_t)k * lw, &fd[k]);
        if (got) { found[k] = 1; fside[k] = 0; frank[k] = rank; continue; }
        if (!(flags & ORACLE_ONESIDED_I))
            got = search_side(C, p, n, q, tol, b, a, nbr + (size_t)b * p, deg[b], l,
                              &ft[k], &rank, fS + (size_t)k * lw, &fd[k]);
        if (got) { found[k] = 1; fside[k] = 1; frank[k] = rank; }
    }
    for (int64_t k = 0; k < E; ++k) {
        R->tests_level[l] += ft[k];
        R->degenerate += fd[k];
        if (!found[k]) continue;
        int32_t a = ea[k], b = eb[k];
        size_t ab = (size_t)a * p + b, ba = (size_t)b * p + a;
        adj[ab] = adj[ba] = 0;
        R->sep_level[ab] = R->sep_level[ba] = l;
        R->sep_side[ab] = R->sep_side[ba] = fside[k];
        R->sep_rank[ab] = R->sep_rank[ba] = frank[k];
        R->sep_off[ab] = R->sep_off[ba] = R->pool_len;
        pool_push(R, fS + (size_t)k * lw, l);
        R->removed_level[l]++;
    }
    free(deg); free(nbr); free(ea); free(eb); free(found); free(fside);
    free(frank); free(fS); free(ft); free(fd); free(comp);
}

/* One stage l of the original (order-dependent) PC: an edge is deleted as
 * soon as a separating set is found (Algorithm 1 with stable = False), so
 * later pairs see the current graph.  Sequential by construction. */
static void nonstable_level(oracle_result *R, const double *C, uint8_t *adj, int32_t p,
                            int64_t n, double q, double tol, int32_t l, int flags)
{
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(l > 0 ? l : 1));
    int32_t *comp = (flags & ORACLE_PATHPOOL) ? (int32_t *)malloc(sizeof(int32_t) * (size_t)p * (size_t)p) : NULL;
    int dirty = 1;
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = a + 1; b < p; ++b) {
            size_t ab = (size_t)a * p + b, ba = (size_t)b * p + a;
            if (!adj[ab]) continue;
            int64_t rank = 0, nt = 0, nd = 0;
            int got = 0, side = 0;
            if (comp) {
                /* the pair's pool in the graph as it is now (deletions are immediate) */
                if (dirty) { components_without(adj, p, comp); dirty = 0; }
                int32_t dp = path_pool(adj, p, comp, a, b, nb);
                got = search_side(C, p, n, q, tol, a, b, nb, dp, l, &nt, &rank, S, &nd);
                dirty = got;
            }
            for (int s = 0; s < 2 && !got && !comp; ++s) {
                if (s == 0 && (flags & ORACLE_ONESIDED_J)) continue;
                if (s == 1 && (flags & ORACLE_ONESIDED_I)) continue;
                int32_t u = s ? b : a, v = s ? a : b, dn = 0;
                for (int32_t w = 0; w < p; ++w) if (adj[(size_t)u * p + w]) nb[dn++] = w;
                got = search_side(C, p, n, q, tol, u, v, nb, dn, l, &nt, &rank, S, &nd);
                side = s;
            }
            R->tests_level[l] += nt;
            R->degenerate += nd;
            if (got) {
                adj[ab] = adj[ba] = 0;
                R->sep_level[ab] = R->sep_level[ba] = l;
                R->sep_side[ab] = R->sep_side[ba] = side;
                R->sep_rank[ab] = R->sep_rank[ba] = rank;
                R->sep_off[ab] = R->sep_off[ba] = R->pool_len;
                pool_push(R, S, l);
                R->removed_level[l]++;
            }
        }
    free(nb);
    free(S);
    free(comp);
}

/* Largest candidate-set size max |adj(u)\{v}| over adjacent ordered pairs. */
static int32_t max_cand(const uint8_t *adj, int32_t p)
{
    int32_t best = -1;
    for (int32_t u = 0; u < p; ++u) {
        int32_t d = 0;
        for (int32_t w = 0; w < p; ++w) d += adj[(size_t)u * p + w] != 0;
        if (d > 0 && d - 1 > best) best = d - 1;
    }
    return best;
}

/* The largest pool of an adjacent pair (ORACLE_PATHPOOL), -1 without edges. */
static int32_t max_path_pool(const uint8_t *adj, int32_t p)
{
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)p * (size_t)p);
    int32_t *pool = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    components_without(adj, p, comp);
    int32_t best = -1;
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = a + 1; b < p; ++b)
            if (adj[(size_t)a * p + b]) {
                int32_t d = path_pool(adj, p, comp, a, b, pool);
                if (d > best) best = d;
            }
    free(comp);
    free(pool);
    return best;
}

/* Size of the largest candidate set of the current graph: adj(u)\{v} over
 * adjacent ordered pairs, or the pair pools with ORACLE_PATHPOOL. */
static int32_t largest_candidates(const uint8_t *adj, int32_t p, int flags)
{
    return (flags & ORACLE_PATHPOOL) ? max_path_pool(adj, p) : max_cand(adj, p);
}

/* The stage l = p-2 of Algorithm 2 in closed form: on the complete graph the
 * only conditioning set of {u,v} is S = V\{u,v}, and the Schur complement of
 * Sec. 4 then equals the inverse of the {u,v} block of P = corr^{-1}:
 *   h11 = P_vv/det, h22 = P_uu/det, h12 = -P_uv/det,  r = -P_uv/sqrt(P_uu P_vv).
 * One test per unordered pair (both sides would test the same S). */
static void stage_a(oracle_result *R, const double *C, uint8_t *adj, int32_t p,
                    int64_t n, double q, double tol)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)p * (size_t)p);
    if (oracle_precision(C, p, P)) { free(P); return; }
    R->stageA_ran = 1;
    int32_t l = p - 2;
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = a + 1; b < p; ++b) {
            double paa = P[(size_t)a * p + a], pbb = P[(size_t)b * p + b];
            double pab = P[(size_t)a * p + b];
            double det = paa * pbb - pab * pab;
            double h11 = pbb / det, h22 = paa / det;
            int degen = !(h11 > ORACLE_DEGEN) || !(h22 > ORACLE_DEGEN);
            int ind;
            if (degen) { ind = 1; R->degenerate++; }
            else {
                double r = -pab / sqrt(paa * pbb);
                if (tol >= 0.0) ind = fabs(r) <= tol;
                else ind = fisher_z(r, n, l) <= q;
            }
            R->tests_level[l]++;
            if (ind) {
                size_t ab = (size_t)a * p + b, ba = (size_t)b * p + a;
                R->sep_level[ab] = R->sep_level[ba] = l;
                R->sep_side[ab] = R->sep_side[ba] = 0;
                R->sep_rank[ab] = R->sep_rank[ba] = 0;
                R->sep_off[ab] = R->sep_off[ba] = -1;
                R->removed_level[l]++;
            }
        }
    /* deferred deletion (stable) */
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = 0; b < p; ++b)
            if (a != b && R->sep_level[(size_t)a * p + b] == l) adj[(size_t)a * p + b] = 0;
    free(P);
}

/* Phase I skeleton.  C: p x p correlation (row-major), n samples, q the
 * Fisher-z threshold, tol >= 0 selects population mode, max_level < 0 means
 * no cap.  Schedules:
 *  conventional (Algorithm 1): l = 0,1,... while some adjacent ordered pair
 *    has |adj(u)\{v}| >= l (Algorithm 1's early termination), l <= cap;
 *  reversed (Algorithm 2): the stage l = p-2 first (closed form, Reading R4),
 *    then l = min(cap, L*) and l <- min(l-1, L*) down to 0, where L* is the
 *    largest candidate-set size in the current graph (levels no pair can use
 *    are empty and are skipped; Algorithm 2 has no early termination).
 * Levels are also capped at n-4 so that n-l-3 > 0 (Reading R9).            */
/* A result on the complete graph, no separating sets yet. */
static oracle_result *result_new(int32_t p, int64_t n)
{
    oracle_result *R = (oracle_result *)calloc(1, sizeof(oracle_result));
    R->p = p; R->n = n;
    size_t pp = (size_t)p * (size_t)p;
    R->adj = (uint8_t *)malloc(pp);
    R->sep_level = (int32_t *)malloc(sizeof(int32_t) * pp);
    R->sep_side = (int32_t *)calloc(pp, sizeof(int32_t));
    R->sep_rank = (int64_t *)calloc(pp, sizeof(int64_t));
    R->sep_off = (int64_t *)calloc(pp, sizeof(int64_t));
    R->tests_level = (int64_t *)calloc((size_t)p + 1, sizeof(int64_t));
    R->removed_level = (int64_t *)calloc((size_t)p + 1, sizeof(int64_t));
    R->level_seq = (int32_t *)calloc((size_t)p + 1, sizeof(int32_t));
    for (size_t k = 0; k < pp; ++k) { R->sep_level[k] = -1; R->adj[k] = 1; }
    for (int32_t a = 0; a < p; ++a) R->adj[(size_t)a * p + a] = 0;
    return R;
}

oracle_result *oracle_skeleton(const double *C, int32_t p, int64_t n, double q, double tol,
                               int32_t max_level, int flags)
{
    oracle_result *R = result_new(p, n);
    if (p < 2) return R;
    int32_t cap = p - 2;
    if (max_level >= 0 && max_level < cap) cap = max_level;
    if (n - 4 < cap) cap = (int32_t)(n - 4);
    int nonstable = flags & ORACLE_NONSTABLE;
    if (!(flags & ORACLE_REVERSED)) {
        for (int32_t l = 0; l <= cap; ++l) {
            if (largest_candidates(R->adj, p, flags) < l) break;
            R->level_seq[R->n_levels++] = l;
            if (nonstable) nonstable_level(R, C, R->adj, p, n, q, tol, l, flags);
            else stable_level(R, C, R->adj, p, n, q, tol, l, flags);
        }
    } else {
        int32_t l;
        if (!(flags & (ORACLE_STAGEA_GENERIC | ORACLE_NO_STAGEA)) && n - p - 1 > 0) {
            stage_a(R, C, R->adj, p, n, q, tol);
            if (R->stageA_ran) R->level_seq[R->n_levels++] = p - 2;
        }
        l = cap;
        if (R->stageA_ran && l > p - 3) l = p - 3;
        int32_t ls = largest_candidates(R->adj, p, flags);
        if (ls < l) l = ls;
        while (l >= 0) {
            R->level_seq[R->n_levels++] = l;
            if (nonstable) nonstable_level(R, C, R->adj, p, n, q, tol, l, flags);
            else stable_level(R, C, R->adj, p, n, q, tol, l, flags);
            int32_t nl = l - 1;
            ls = largest_candidates(R->adj, p, flags);
            if (ls < nl) nl = ls;
            l = nl;
        }
    }
    for (int32_t l = 0; l <= p; ++l) R->tests_total += R->tests_level[l];
    return R;
}

/* Algorithm 3, the batched form of Algorithm 2: stage l = p-2 down to 0; the
 * loop reaches the adjacent pairs {a,b}, a<b, in order, forms each pair's pool
 * adj(G,a,b) intersected with path(G,a,b) (Reading R19) from the graph as it is
 * when the pair is reached, and queues its l-subsets in lexicographic order;
 * whenever `batch` tests are queued they are decided together and the edges
 * found independent are deleted at once.  Readings (R20): the partial batch is
 * flushed at the end of every stage (the listing resets its counter per stage
 * and flushes only after the last one, which would drop tests); a pair deleted
 * by an earlier batch queues no further subsets; within a batch a pair's first
 * independent test in queue order gives its separating set (side 0, the rank
 * of the set in its pool).  Empty stages are skipped as in Reading R4, and
 * stage p-2 is enumerated (no closed form: deletions inside it change later
 * pools). */
typedef struct {
    int32_t a, b;
    int64_t rank;
} batch_entry;

static void flush_batch(oracle_result *R, const double *C, uint8_t *adj, int32_t p, int64_t n, double q,
                        double tol, int32_t l, const batch_entry *E, const int32_t *ES, int64_t m,
                        int *dirty)
{
    int32_t lw = l > 0 ? l : 1;
    for (int64_t t = 0; t < m; ++t) {
        int32_t a = E[t].a, b = E[t].b;
        size_t ab = (size_t)a * p + b, ba = (size_t)b * p + a;
        int degen = 0;
        int ind = oracle_ci_test(C, p, n, q, tol, a, b, ES + (size_t)t * lw, l, NULL, NULL, &degen);
        R->tests_level[l]++;
        if (degen) R->degenerate++;
        if (!ind || R->sep_level[ab] == l) continue;   /* dependent, or already separated here */
        R->sep_level[ab] = R->sep_level[ba] = l;
        R->sep_side[ab] = R->sep_side[ba] = 0;
        R->sep_rank[ab] = R->sep_rank[ba] = E[t].rank;
        R->sep_off[ab] = R->sep_off[ba] = R->pool_len;
        pool_push(R, ES + (size_t)t * lw, l);
        R->removed_level[l]++;
    }
    for (int64_t t = 0; t < m; ++t) {
        size_t ab = (size_t)E[t].a * p + E[t].b, ba = (size_t)E[t].b * p + E[t].a;
        if (R->sep_level[ab] == l && adj[ab]) { adj[ab] = adj[ba] = 0; *dirty = 1; }
    }
}

oracle_result *oracle_skeleton_batched(const double *C, int32_t p, int64_t n, double q, double tol,
                                       int32_t max_level, int64_t batch)
{
    oracle_result *R = result_new(p, n);
    if (p < 2 || batch < 1) return R;
    int32_t cap = p - 2;
    if (max_level >= 0 && max_level < cap) cap = max_level;
    if (n - 4 < cap) cap = (int32_t)(n - 4);
    uint8_t *adj = R->adj;
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)p * (size_t)p);
    int32_t *pool = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    int64_t ecap = 1024;
    batch_entry *E = (batch_entry *)malloc(sizeof(batch_entry) * (size_t)ecap);
    int32_t *ES = (int32_t *)malloc(sizeof(int32_t) * (size_t)ecap * (size_t)(p > 0 ? p : 1));
    int32_t l = cap;
    int32_t ls = max_path_pool(adj, p);
    if (ls < l) l = ls;
    while (l >= 0) {
        R->level_seq[R->n_levels++] = l;
        int32_t lw = l > 0 ? l : 1;
        int64_t m = 0;
        int dirty = 1;
        for (int32_t a = 0; a < p; ++a)
            for (int32_t b = a + 1; b < p; ++b) {
                if (!adj[(size_t)a * p + b]) continue;
                if (dirty) { components_without(adj, p, comp); dirty = 0; }
                int32_t d = path_pool(adj, p, comp, a, b, pool);
                if (d < l) continue;
                int32_t idx[lw];
                for (int32_t k = 0; k < l; ++k) idx[k] = k;
                for (int64_t rank = 0;; ++rank) {
                    if (!adj[(size_t)a * p + b]) break;        /* deleted by an earlier batch */
                    if (m == ecap) {
                        ecap *= 2;
                        E = (batch_entry *)realloc(E, sizeof(batch_entry) * (size_t)ecap);
                        ES = (int32_t *)realloc(ES, sizeof(int32_t) * (size_t)ecap * (size_t)(p > 0 ? p : 1));
                    }
                    E[m].a = a; E[m].b = b; E[m].rank = rank;
                    for (int32_t k = 0; k < l; ++k) ES[(size_t)m * lw + k] = pool[idx[k]];
                    if (++m == batch) {
                        flush_batch(R, C, adj, p, n, q, tol, l, E, ES, m, &dirty);
                        m = 0;
                    }
                    int32_t i = l - 1;
                    while (i >= 0 && idx[i] == d - l + i) --i;
                    if (i < 0) break;
                    ++idx[i];
                    for (int32_t j = i + 1; j < l; ++j) idx[j] = idx[j - 1] + 1;
                }
            }
        if (m) flush_batch(R, C, adj, p, n, q, tol, l, E, ES, m, &dirty);
        int32_t nl = l - 1;
        ls = max_path_pool(adj, p);
        if (ls < nl) nl = ls;
        l = nl;
    }
    for (int32_t k = 0; k <= p; ++k) R->tests_total += R->tests_level[k];
    free(comp); free(pool); free(E); free(ES);
    return R;
}

void oracle_result_free(oracle_result *R)
{
    if (!R) return;
    free(R->adj); free(R->sep_level); free(R->sep_side); free(R->sep_rank);
    free(R->sep_off); free(R->pool); free(R->tests_level); free(R->removed_level);
    free(R->level_seq); free(R);
}

/* Flat accessors for the Python wrapper (ctypes). */
void oracle_result_copy(const oracle_result *R, uint8_t *adj, int32_t *sep_level,
                        int32_t *sep_side, int64_t *sep_rank, int64_t *sep_off,
                        int64_t *tests_level, int64_t *removed_level, int32_t *level_seq)
{
    size_t pp = (size_t)R->p * (size_t)R->p;
    memcpy(adj, R->adj, pp);
    memcpy(sep_level, R->sep_level, sizeof(int32_t) * pp);
    memcpy(sep_side, R->sep_side, sizeof(int32_t) * pp);
    memcpy(sep_rank, R->sep_rank, sizeof(int64_t) * pp);
    memcpy(sep_off, R->sep_off, sizeof(int64_t) * pp);
    memcpy(tests_level, R->tests_level, sizeof(int64_t) * ((size_t)R->p + 1));
    memcpy(removed_level, R->removed_level, sizeof(int64_t) * ((size_t)R->p + 1));
    memcpy(level_seq, R->level_seq, sizeof(int32_t) * ((size_t)R->p + 1));
}

int64_t oracle_result_pool_len(const oracle_result *R) { return R->pool_len; }
void oracle_result_pool(const oracle_result *R, int32_t *out)
{
    if (R->pool_len) memcpy(out, R->pool, sizeof(int32_t) * (size_t)R->pool_len);
}
void oracle_result_scalars(const oracle_result *R, int64_t *out4)
{
    out4[0] = R->tests_total;
    out4[1] = R->degenerate;
    out4[2] = R->stageA_ran;
    out4[3] = R->n_levels;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Phase II of Algorithm 1 (Sec. 3.3: Algorithm 2 leaves it unchanged): the
 * skeleton is oriented from the separation sets, first the unshielded
 * colliders, then rules R1-R4 repeated until none orients an edge.
 *
 * Edge marks: mk[a*p+b] = 1 iff the edge {a,b} carries an arrowhead at b.
 * a - b: no mark on either end; a -> b: mk[a*p+b] only; both: a <-> b.
 * Output codes per ordered pair: 0 no edge, 1 a - b, 2 a -> b, 3 a <- b,
 * 4 a <-> b.
 *
 * Reading R15: the listing orders neither loop.  Every collider found marks
 * both of its edges at once (an edge marked from both ends by two colliders
 * is bidirected); the rules run in rounds, each evaluating R1-R4 on every
 * undirected edge against the marks at the start of the round and then
 * applying all orientations found (found in both directions: bidirected),
 * until a round orients nothing.
 * Reading R16: R4 as printed requires X_k -> X_l and calls X_k, X_l
 * non-adjacent; read as X_k and X_j non-adjacent (the published form of the
 * rule, Meek 1995).                                                         */

static int ph2_dir(const uint8_t *adj, const uint8_t *mk, int32_t p, int32_t x, int32_t y)
{   /* x -> y */
    return adj[(size_t)x * p + y] && mk[(size_t)x * p + y] && !mk[(size_t)y * p + x];
}

static int ph2_und(const uint8_t *adj, const uint8_t *mk, int32_t p, int32_t x, int32_t y)
{   /* x - y */
    return adj[(size_t)x * p + y] && !mk[(size_t)x * p + y] && !mk[(size_t)y * p + x];
}

/* Does one of R1-R4 (Algorithm 1, Phase II) change the undirected edge a - b
 * into a -> b?  Returns the rule number, or 0.  The paper's letters: the edge
 * oriented is X_i - X_j with X_i = a, X_j = b for R2-R4, and X_j - X_k with
 * X_j = a, X_k = b for R1.                                                  */
static int ph2_rule(const uint8_t *adj, const uint8_t *mk, int32_t p, int32_t a, int32_t b)
{
    /* R1: X_i -> X_j, X_i and X_k non-adjacent */
    for (int32_t c = 0; c < p; ++c)
        if (c != b && ph2_dir(adj, mk, p, c, a) && !adj[(size_t)c * p + b]) return 1;
    /* R2: X_i -> X_k -> X_j */
    for (int32_t c = 0; c < p; ++c)
        if (ph2_dir(adj, mk, p, a, c) && ph2_dir(adj, mk, p, c, b)) return 2;
    /* R3: X_i - X_k -> X_j and X_i - X_l -> X_j, X_k and X_l non-adjacent */
    for (int32_t c = 0; c < p; ++c) {
        if (!(ph2_und(adj, mk, p, a, c) && ph2_dir(adj, mk, p, c, b))) continue;
        for (int32_t d = c + 1; d < p; ++d)
            if (ph2_und(adj, mk, p, a, d) && ph2_dir(adj, mk, p, d, b) && !adj[(size_t)c * p + d]) return 3;
    }
    /* R4: X_i - X_k -> X_l and X_k -> X_l -> X_j, X_k and X_j non-adjacent */
    for (int32_t c = 0; c < p; ++c) {
        if (c == b || !ph2_und(adj, mk, p, a, c) || adj[(size_t)c * p + b]) continue;
        for (int32_t d = 0; d < p; ++d)
            if (ph2_dir(adj, mk, p, c, d) && ph2_dir(adj, mk, p, d, b)) return 4;
    }
    return 0;
}

/* R1-R4 in rounds (Reading R15) on the marks mk, in place.  Returns the number
 * of rounds that oriented at least one edge.                                */
int32_t oracle_meek(const uint8_t *adj, uint8_t *mk, int32_t p)
{
    const size_t pp = (size_t)p * p;
    uint8_t *next = (uint8_t *)malloc(pp ? pp : 1);
    int32_t rounds = 0;
    for (;;) {
        int changed = 0;
        memcpy(next, mk, pp);
        for (int32_t a = 0; a < p; ++a)
            for (int32_t b = 0; b < p; ++b)
                if (a != b && ph2_und(adj, mk, p, a, b) && ph2_rule(adj, mk, p, a, b)) {
                    next[(size_t)a * p + b] = 1;
                    changed = 1;
                }
        memcpy(mk, next, pp);
        if (!changed) break;
        ++rounds;
    }
    free(next);
    return rounds;
}

/* Unshielded colliders (Algorithm 1, Phase II, its first step): for every pair of
 * non-adjacent vertices i < j and every common neighbour k, k not in S(i,j)
 * puts arrowheads at k on i - k and j - k (Reading R15).  S(i,j) is given as
 * sep_off[i*p+j]: an offset into pool with sep_len[i*p+j] members, -1 for
 * "every other node" (the closed-form stage l = p-2), -2 when no set was
 * recorded (no collider is decided from such a pair).                       */
void oracle_vstructures(const uint8_t *adj, int32_t p, const int64_t *sep_off, const int32_t *sep_len,
                        const int32_t *pool, uint8_t *mk)
{
    memset(mk, 0, (size_t)p * p);
    for (int32_t i = 0; i < p; ++i)
        for (int32_t j = i + 1; j < p; ++j) {
            if (adj[(size_t)i * p + j]) continue;
            const int64_t off = sep_off[(size_t)i * p + j];
            if (off < 0) continue;                      /* every other node, or none */
            const int32_t len = sep_len[(size_t)i * p + j];
            for (int32_t k = 0; k < p; ++k) {
                if (k == i || k == j || !adj[(size_t)i * p + k] || !adj[(size_t)j * p + k]) continue;
                int in_s = 0;
                for (int32_t t = 0; t < len; ++t) in_s |= pool[off + t] == k;
                if (!in_s) {
                    mk[(size_t)i * p + k] = 1;
                    mk[(size_t)j * p + k] = 1;
                }
            }
        }
}

/* Marks -> codes (0 none, 1 a - b, 2 a -> b, 3 a <- b, 4 a <-> b). */
void oracle_codes(const uint8_t *adj, const uint8_t *mk, int32_t p, int8_t *out)
{
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = 0; b < p; ++b) {
            const size_t e = (size_t)a * p + b, t = (size_t)b * p + a;
            int8_t c = 0;
            if (a != b && adj[e]) c = (int8_t)(mk[e] ? (mk[t] ? 4 : 2) : (mk[t] ? 3 : 1));
            out[e] = c;
        }
}

/* The whole Phase II: colliders, rules, codes.  Returns the rule rounds.    */
int32_t oracle_orient(const uint8_t *adj, int32_t p, const int64_t *sep_off, const int32_t *sep_len,
                      const int32_t *pool, int8_t *out)
{
    const size_t pp = (size_t)p * p;
    uint8_t *mk = (uint8_t *)malloc(pp > 0 ? pp : 1);
    oracle_vstructures(adj, p, sep_off, sep_len, pool, mk);
    const int32_t rounds = oracle_meek(adj, mk, p);
    oracle_codes(adj, mk, p, out);
    free(mk);
    return rounds;
}
