"""The FP32 trust rule of the CI tests (no GPU needed).

A test is evaluated in FP32 from FP32 correlations; its decision is trusted
only when the rule below says that the FP64 decision of Eq. 1 (Sec. 2.2.2,
evaluated in r: |r| <= tanh(q / sqrt(n-l-3))) is the same.  The computed
trailing block is the exact Schur complement of corr + E, E the correlation
step's entry errors (|E_ij| <= eps_C) plus the backward error of the FP32
Cholesky (<= 4 m eps32 per entry: the factor's rows have unit norm).  With b_u,
b_v the regression coefficients of u and v on S, to first order

  |dr| <= eps (A_u A_v / sqrt(h11 h22) + |r|/2 (A_u^2/h11 + A_v^2/h22)),
  A = 1 + |b|_1,  eps = eps_C + 4 m eps32,

doubled for the higher-order terms, which are kept small by requiring
eps A^2/h <= 0.05 and m eps |corr_SS^{-1}| <= 0.05.  A test is trusted when
|r| clears the threshold by more than the doubled bound and z lies at least the
band from q.  The small-stage kernel bounds A and |corr_SS^{-1}| from the
prefix factor it keeps (|Lp^{-1}|_F^2, the prefix coefficients) and the border
member's pivot; the warp-per-test kernel forms b_u and b_v exactly.

This file emulates both in float32, in the kernels' order of operations
(separate multiply and subtract where the kernel fuses them: a different
rounding of the same size), on random correlation blocks (some near singular)
with n chosen so that the FP64 statistic lies within 1 % of the threshold, and
checks that every trusted decision equals the FP64 one and that the FP32 r lies
within the rule's bound of the FP64 r -- with correlations exact in FP32 and
with errors of the full allowance eps_C = 1e-6 on every entry, at every n.
The bound itself is pinned in FP64 against exact perturbations.  The
split-precision product is emulated too: on SEM data of the workloads' recipes
its entry errors stay below the 1e-6 allowance."""
import math
import statistics

import numpy as np
import pytest

f32 = np.float32
E32 = 5.96e-8
GUARD, BAND = 1e-3, 1e-3


def _rsqrt(x):
    return f32(1.0) / np.sqrt(f32(x), dtype=f32)


def _trust(eps_c, m, sqf, rq, a, h11, h22, ih, Au, Av, kap, dr_max=1.0):
    """(verdict 0 trusted / 1 band / 2 guard, doubled bound) -- fp32_trust."""
    eps = f32(eps_c + 4.0 * m * E32)
    i11, i22 = f32(1) / h11, f32(1) / h22
    if max(eps * Au * Au * i11, eps * Av * Av * i22, kap) > 0.05:
        return 2, None
    dr = f32(2) * eps * (Au * Av * ih + f32(0.5) * a * (Au * Au * i11 + Av * Av * i22)) + f32(8 * E32)
    if dr > dr_max:
        return 2, dr
    gap, mn = abs(a - rq), min(a, rq)
    if gap <= dr or sqf * gap < f32(BAND) * (f32(1) - mn * mn):
        return 1, dr
    return 0, dr


def lane_test_fp32(C32, L, eps_c, sqf, rq):
    """The small-stage kernel's bordered test.  Nodes 0, 1 are u, v; 2 .. L the
    prefix; L+1 the border member.  Returns (kind, |r|, independent, bound) with kind
    "trusted", "queued" or "dependent"."""
    K = max(L - 1, 0)
    m = L + 2
    sp = list(range(2, 2 + K))
    s = 1 + L
    Lp, rd = {}, [f32(0)] * max(K, 1)
    lu, lv = [f32(0)] * max(K, 1), [f32(0)] * max(K, 1)
    pmin, bad = f32(1e30), False
    for i in range(K):
        dd = f32(1)
        for c in range(i):
            t = f32(C32[sp[i], sp[c]])
            for c2 in range(c):
                t = f32(t - f32(Lp[i, c2] * Lp[c, c2]))
            t = f32(t * rd[c])
            Lp[i, c] = t
            dd = f32(dd - f32(t * t))
        pmin = min(pmin, dd)
        bad |= not dd > 1e-12
        rl = _rsqrt(max(dd, f32(1e-30)))
        rd[i] = rl
        Lp[i, i] = f32(dd * rl)
        tu, tv = f32(C32[0, sp[i]]), f32(C32[1, sp[i]])
        for c in range(i):
            tu = f32(tu - f32(lu[c] * Lp[i, c]))
            tv = f32(tv - f32(lv[c] * Lp[i, c]))
        lu[i], lv[i] = f32(tu * rl), f32(tv * rl)
    # prefix terms: F = |Lp^{-1}|_F^2 by columns, the prefix coefficients' l1 norms
    F = f32(0)
    for c in range(K):
        z = {c: rd[c]}
        F = f32(F + z[c] * z[c])
        for k in range(c + 1, K):
            t = f32(0)
            for j in range(c, k):
                t = f32(t + f32(Lp[k, j] * z[j]))
            z[k] = f32(-t * rd[k])
            F = f32(F + z[k] * z[k])
    BuP = BvP = f32(0)
    bu_, bv_ = {}, {}
    for k in range(K - 1, -1, -1):
        tu, tv = lu[k], lv[k]
        for j in range(k + 1, K):
            tu = f32(tu - f32(Lp[j, k] * bu_[j]))
            tv = f32(tv - f32(Lp[j, k] * bv_[j]))
        bu_[k], bv_[k] = f32(tu * rd[k]), f32(tv * rd[k])
        BuP, BvP = f32(BuP + abs(bu_[k])), f32(BvP + abs(bv_[k]))
    sKF = np.sqrt(f32(K) * F, dtype=f32)
    h11, h22, h12 = f32(1), f32(1), f32(C32[0, 1])
    for i in range(K):
        h11 = f32(h11 - f32(lu[i] * lu[i]))
        h22 = f32(h22 - f32(lv[i] * lv[i]))
        h12 = f32(h12 - f32(lu[i] * lv[i]))
    x, bsu, bsv, gs = f32(1), f32(0), f32(0), f32(0)
    if L > 0:
        ls, xb = [f32(0)] * max(K, 1), f32(1)
        for i in range(K):
            t = f32(C32[s, sp[i]])
            for c in range(i):
                t = f32(t - f32(ls[c] * Lp[i, c]))
            t = f32(t * rd[i])
            ls[i] = t
            xb = f32(xb - f32(t * t))
        cu, cv = f32(C32[s, 0]), f32(C32[s, 1])
        for i in range(K):
            cu = f32(cu - f32(lu[i] * ls[i]))
            cv = f32(cv - f32(lv[i] * ls[i]))
        pmin = min(pmin, xb)
        bad |= not xb > 1e-12
        rx = f32(1) / max(xb, f32(1e-30))
        h11 = f32(h11 - f32(f32(cu * cu) * rx))
        h22 = f32(h22 - f32(f32(cv * cv) * rx))
        h12 = f32(h12 - f32(f32(cu * cv) * rx))
        x = max(xb, f32(1e-30))
        bsu, bsv = abs(f32(cu * rx)), abs(f32(cv * rx))
        gs = f32(sKF * np.sqrt(max(f32(1) - xb, f32(0)), dtype=f32)) if K > 0 else f32(0)
    pmin = min(pmin, h11, h22)
    bad |= not h11 > 1e-12 or not h22 > 1e-12
    if bad or pmin < GUARD:
        return "queued", None, None, None
    ih = _rsqrt(f32(h11 * h22))
    a = abs(f32(h12 * ih))
    Au = f32(1 + BuP + bsu * f32(1 + gs))
    Av = f32(1 + BvP + bsv * f32(1 + gs))
    eps = f32(eps_c + 4.0 * m * E32)
    kap = f32(m * eps * f32(F + 1)) / x
    t, dr = _trust(eps_c, m, sqf, rq, a, h11, h22, ih, Au, Av, kap)
    if t:
        return "queued", a, None, dr
    return ("trusted" if a < 1 else "dependent"), a, bool(a <= rq), dr


def warp_test_fp32(C32, L, eps_c, sqf, rq, dr_max=1.0):
    """The warp-per-test kernel: Cholesky of the (S, u, v) block in the order S..., u, v
    (column scaling by 1/sqrt(pivot), then the trailing update), the regression
    coefficients by back substitution.  Node order here: S = 2 .. L+1, u = 0, v = 1."""
    order = list(range(2, 2 + L)) + [0, 1]
    m = L + 2
    M = C32[np.ix_(order, order)].astype(f32).copy()
    pmin = f32(1e30)
    for k in range(L):
        piv = M[k, k]
        pmin = min(pmin, piv)
        if not piv > 1e-12:
            return "queued", None, None, None
        rl = f32(1) / np.sqrt(piv, dtype=f32)
        for i in range(k + 1, m):
            M[i, k] = f32(M[i, k] * rl)
        for i in range(k + 1, m):
            for c in range(k + 1, i + 1):
                M[i, c] = f32(M[i, c] - f32(M[i, k] * M[c, k]))
    h11, h22, h12 = M[L, L], M[L + 1, L + 1], M[L + 1, L]
    pmin = min(pmin, h11, h22)
    if not (h11 > 1e-12 and h22 > 1e-12) or pmin < GUARD:
        return "queued", None, None, None
    yu, yv = M[L, :L].copy(), M[L + 1, :L].copy()
    su = sv = f32(0)
    for k in range(L - 1, -1, -1):
        rl = _rsqrt(M[k, k])
        bu, bv = f32(yu[k] * rl), f32(yv[k] * rl)
        su, sv = f32(su + abs(bu)), f32(sv + abs(bv))
        for j in range(k):
            yu[j] = f32(yu[j] - f32(M[k, j] * bu))
            yv[j] = f32(yv[j] - f32(M[k, j] * bv))
    rf = f32(h12 / np.sqrt(f32(h11 * h22), dtype=f32))
    a = abs(rf)
    ih = _rsqrt(f32(h11 * h22))
    t, dr = _trust(eps_c, m, sqf, rq, a, h11, h22, ih, f32(1 + su), f32(1 + sv), f32(0), dr_max)
    if t:
        return "queued", a, None, dr
    return ("trusted" if a < 1 else "dependent"), a, bool(a <= rq), dr


def _block(rng, m, extra=(1, 40)):
    k = m + int(rng.integers(*extra))          # few samples: some blocks near singular
    A = rng.standard_normal((k, m)) @ (np.eye(m) + 0.5 * rng.standard_normal((m, m)))
    return np.corrcoef(A, rowvar=False)


def _cases(seed, count, entry_err, eps_c, nmin=0, lmax=12, kernel=lane_test_fp32):
    rng = np.random.default_rng(seed)
    q = -statistics.NormalDist().inv_cdf(0.005)
    out = []
    while len(out) < count:
        L = int(rng.integers(0, lmax + 1))
        m = L + 2
        C = _block(rng, m)
        E = np.triu(rng.uniform(-entry_err, entry_err, (m, m)), 1)
        C32 = (C + E + E.T).astype(f32)
        np.fill_diagonal(C32, 1)
        P = np.linalg.inv(C)
        r64 = -P[0, 1] / math.sqrt(P[0, 0] * P[1, 1])
        if abs(r64) < 1e-6:
            continue
        n = int(round((q / math.atanh(abs(r64))) ** 2 * (1 + rng.uniform(-0.01, 0.01)) + L + 3))
        if n < nmin or n - L - 3 <= 0:
            continue
        sq = math.sqrt(n - L - 3)
        z64 = sq * abs(math.atanh(r64))
        kind, a, ind, dr = kernel(C32, L, eps_c, f32(sq), f32(math.tanh(q / sq)))
        out.append((kind, a, ind, z64 <= q, z64, sq, q, abs(r64), dr))
    return out


REGIMES = [("correlations exact in FP32", 0.0, 1.2e-7, 0),
           ("entry errors of 1e-6 on every entry, every n", 1e-6, 1e-6, 0),
           ("entry errors of 1e-6 on every entry, n >= 1000", 1e-6, 1e-6, 1000)]


@pytest.mark.parametrize("kernel", [lane_test_fp32, warp_test_fp32], ids=["small_stage", "warp_per_test"])
@pytest.mark.parametrize("regime", REGIMES, ids=["exact", "1e-6_all_n", "1e-6_n_ge_1000"])
def test_trusted_fp32_decisions_equal_fp64(regime, kernel):
    label, entry_err, eps_c, nmin = regime
    rows = _cases(11, 700, entry_err, eps_c, nmin, kernel=kernel)
    trusted = [r for r in rows if r[0] == "trusted"]
    assert len(trusted) > 0.2 * len(rows), label    # near the threshold the rule still trusts many
    assert any(r[0] == "queued" for r in rows)        # and sends others to FP64
    for kind, a, ind, ind64, z64, sq, q, r64, dr in trusted:
        assert ind == ind64, label
        # the FP32 |r| lies within the rule's bound of the FP64 |r|
        assert abs(float(a) - r64) <= float(dr), label


def test_error_bound_holds_for_exact_perturbations():
    # the first-order bound (without rounding terms) against exact FP64 arithmetic:
    # r of corr + E for random symmetric E with |E_ij| <= eps never moves further than
    # eps (A_u A_v / sqrt(h11 h22) + |r|/2 (A_u^2/h11 + A_v^2/h22)) from r of corr
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(400):
        L = int(rng.integers(0, 13))
        m = L + 2
        C = _block(rng, m)
        S, u, v = list(range(2, m)), 0, 1
        Css = C[np.ix_(S, S)]
        bu = np.linalg.solve(Css, C[S, u]) if L else np.zeros(0)
        bv = np.linalg.solve(Css, C[S, v]) if L else np.zeros(0)
        h11 = 1 - C[u, S] @ bu
        h22 = 1 - C[v, S] @ bv
        h12 = C[u, v] - C[u, S] @ bv
        r = h12 / math.sqrt(h11 * h22)
        Au, Av = 1 + np.abs(bu).sum(), 1 + np.abs(bv).sum()
        eps = 1e-9 * min(1.0, h11 / Au ** 2, h22 / Av ** 2)
        bound = eps * (Au * Av / math.sqrt(h11 * h22) + abs(r) / 2 * (Au ** 2 / h11 + Av ** 2 / h22))
        for _ in range(3):
            E = np.triu(rng.uniform(-eps, eps, (m, m)), 1)
            P = np.linalg.inv(C + E + E.T)
            r2 = -P[0, 1] / math.sqrt(P[0, 0] * P[1, 1])
            worst = max(worst, abs(r2 - r) / bound)
    assert worst <= 1.02                            # first order: equality up to O(eps^2)


def test_raw_tests_keep_r_within_their_bar():
    # pc_ci_batch returns r itself: FP32 is trusted there only when the bound is
    # <= 5e-6, which keeps |r32 - r64| inside the 1e-5 parity bar (blocks of
    # better conditioning than above, as most raw tests are)
    rng = np.random.default_rng(17)
    q = -statistics.NormalDist().inv_cdf(0.005)
    kept = 0
    for _ in range(600):
        L = int(rng.integers(0, 13))
        m = L + 2
        C = _block(rng, m, (40, 400))
        E = np.triu(rng.uniform(-1e-6, 1e-6, (m, m)), 1)
        C32 = (C + E + E.T).astype(f32)
        np.fill_diagonal(C32, 1)
        P = np.linalg.inv(C)
        r64 = -P[0, 1] / math.sqrt(P[0, 0] * P[1, 1])
        sq = math.sqrt(20000 - L - 3)
        kind, a, ind, dr = warp_test_fp32(C32, L, 1e-6, f32(sq), f32(math.tanh(q / sq)), dr_max=5e-6)
        if kind != "queued":
            kept += 1
            assert abs(float(a) - abs(r64)) <= 5e-6
    assert kept >= 10                                  # the rest went to FP64


def _bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), kept as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def _corr_bf16x3(Xs, ktile=64):
    """The split-precision product: X = hi + lo in BF16, hi*hi + hi*lo + lo*hi summed in
    FP32 within a tile of samples, compensated (Kahan) sums across tiles."""
    hi = _bf16(Xs)
    lo = _bf16(Xs.astype(np.float32) - hi)
    n, p = Xs.shape
    acc = np.zeros((p, p), np.float32)
    comp = np.zeros((p, p), np.float32)
    for k0 in range(0, n, ktile):
        H, Lo = hi[k0:k0 + ktile], lo[k0:k0 + ktile]
        part = (H.T @ H + H.T @ Lo + Lo.T @ H).astype(np.float32)
        y = part - comp
        t = acc + y
        comp = (t - acc) - y
        acc = t
    return acc / np.float32(n)


@pytest.mark.parametrize("shape", [(95, 5000, 0.3), (200, 20000, None)])
def test_bf16x3_entry_errors_stay_below_the_allowance(shape):
    # on SEM data of the workloads' recipes the split-precision correlations stay
    # below the eps_C = 1e-6 entry-error allowance of the trust rule
    from paper_2109_04626_gb300 import sem
    p, n, prob = shape
    rng = np.random.Generator(np.random.PCG64(77))
    dag, W, order = sem.er_dag(p, prob if prob else 10.0 / (p - 1), rng)
    X = sem.sample(W, order, n, rng)
    Xs = (X - X.mean(0)) / X.std(0)
    C64 = Xs.T @ Xs / n
    E = np.abs(_corr_bf16x3(Xs).astype(np.float64) - C64)
    np.fill_diagonal(E, 0.0)
    assert E.max() < 5e-7                     # half the allowance
    assert np.median(E[np.triu_indices(p, 1)]) < 1e-7


# --------------------------------------------------------------------------- complement tests
# The reversed order's high stages test (u, v | S) with S = F \ {u, v} \ R, |R| = k
# small, from the FP64 precision block P = corr[F,F]^{-1}:  Q = P_TT - P_TR P_RR^{-1}
# P_RT on {u, v} is the inverse of corr[T,T] there (T = F \ R), r = -Q_uv /
# sqrt(Q_uu Q_vv).  In FP32 (P rounded on load) the result is that of P + dP,
# |dP_ij| <= eps s_i s_j (s_i = sqrt(P_ii), eps = (4k + 8) eps32), and to first order
#   |dr| <= eps (W_u W_v / sqrt(Q_uu Q_vv) + |r|/2 (W_u^2/Q_uu + W_v^2/Q_vv)),
#   W_a = s_a + sum_r s_r |X_ra|,  X_a = P_RR^{-1} P_Ra,
# used while eps W_a^2/Q_aa and k eps tr(D P_RR^{-1} D) stay below 0.05, doubled,
# plus 8 eps32.

def comp_test_fp32(P, R, u, v, sqf, rq, dr_max=1.0):
    """The complement kernel's FP32 evaluation in its order of operations (R: the
    dropped slots in ascending order, u and v: slots of the pair)."""
    k = len(R)
    L = np.zeros((k, k), f32)
    yu = np.array([P[r, u] for r in R], dtype=f32)
    yv = np.array([P[r, v] for r in R], dtype=f32)
    for i in range(k):
        for c in range(i + 1):
            L[i, c] = f32(P[R[i], R[c]])
    sd = np.array([np.sqrt(max(L[i, i], f32(0)), dtype=f32) for i in range(k)], dtype=f32)
    ri = np.zeros(k, f32)
    for i in range(k):
        for c in range(i):
            t = L[i, c]
            for q in range(c):
                t = f32(t - f32(L[i, q] * L[c, q]))
            L[i, c] = f32(t * ri[c])
        t = L[i, i]
        for q in range(i):
            t = f32(t - f32(L[i, q] * L[i, q]))
        if not t > 0:
            return "queued", None, None, None
        ri[i] = _rsqrt(t)
        a, b = yu[i], yv[i]
        for q in range(i):
            a = f32(a - f32(L[i, q] * yu[q]))
            b = f32(b - f32(L[i, q] * yv[q]))
        yu[i], yv[i] = f32(a * ri[i]), f32(b * ri[i])
    Quu, Qvv, Quv = f32(P[u, u]), f32(P[v, v]), f32(P[u, v])
    for i in range(k):
        Quu = f32(Quu - f32(yu[i] * yu[i]))
        Qvv = f32(Qvv - f32(yv[i] * yv[i]))
        Quv = f32(Quv - f32(yu[i] * yv[i]))
    if not (Quu > 0 and Qvv > 0):
        return "queued", None, None, None
    Wu, Wv = np.sqrt(f32(P[u, u]), dtype=f32), np.sqrt(f32(P[v, v]), dtype=f32)
    for i in range(k - 1, -1, -1):
        a, b = yu[i], yv[i]
        for q in range(i + 1, k):
            a = f32(a - f32(L[q, i] * yu[q]))
            b = f32(b - f32(L[q, i] * yv[q]))
        yu[i], yv[i] = f32(a * ri[i]), f32(b * ri[i])
        Wu = f32(Wu + f32(sd[i] * abs(yu[i])))
        Wv = f32(Wv + f32(sd[i] * abs(yv[i])))
    tr = f32(0)
    for j in range(k):
        m = np.zeros(k, f32)
        nj = f32(0)
        for i in range(j, k):
            t = f32(1) if i == j else f32(0)
            for q in range(j, i):
                t = f32(t - f32(L[i, q] * m[q]))
            m[i] = f32(t * ri[i])
            nj = f32(nj + f32(m[i] * m[i]))
        tr = f32(tr + f32(f32(sd[j] * sd[j]) * nj))
    eps = f32((4.0 * k + 8.0) * E32)
    kap = f32(f32(k) * eps * tr)
    iu, iv = f32(1) / Quu, f32(1) / Qvv
    if not max(eps * Wu * Wu * iu, eps * Wv * Wv * iv, kap) <= 0.05:
        return "queued", None, None, None
    ih = _rsqrt(f32(Quu * Qvv))
    a = abs(f32(Quv * ih))
    dr = f32(2) * eps * (Wu * Wv * ih + f32(0.5) * a * (Wu * Wu * iu + Wv * Wv * iv)) + f32(8 * E32)
    if not dr <= dr_max:
        return "queued", a, None, dr
    om = f32(1) - a * a
    if not om > 8 * dr or Quu * om > 1e9 or Qvv * om > 1e9:
        return "queued", a, None, dr
    gap, mn = abs(a - rq), min(a, rq)
    if gap <= dr or sqf * gap < f32(BAND) * (f32(1) - mn * mn):
        return "queued", a, None, dr
    return "trusted", a, bool(a <= rq), dr


def _comp_case(rng):
    """A neighbourhood block F (slot 0 = u, slot 1 = v), a dropped set R of k slots
    and the FP64 r of (u, v | F \\ {u, v} \\ R) from corr directly."""
    k = int(rng.integers(1, 9))
    m = k + 2 + int(rng.integers(0, 30))
    C = _block(rng, m, (1, 60))
    P = np.linalg.inv(C)
    R = sorted(int(x) for x in rng.choice(np.arange(2, m), size=k, replace=False))
    T = [i for i in range(m) if i not in R]
    Q = np.linalg.inv(C[np.ix_(T, T)])
    r64 = -Q[0, 1] / math.sqrt(Q[0, 0] * Q[1, 1])
    return C, P, R, r64, len(T) - 2


def test_trusted_fp32_complement_decisions_equal_fp64():
    rng = np.random.default_rng(23)
    q = -statistics.NormalDist().inv_cdf(0.005)
    rows = []
    while len(rows) < 700:
        C, P, R, r64, L = _comp_case(rng)
        if abs(r64) < 1e-6 or abs(r64) > 0.999:
            continue
        n = int(round((q / math.atanh(abs(r64))) ** 2 * (1 + rng.uniform(-0.01, 0.01)) + L + 3))
        if n - L - 3 <= 0:
            continue
        sq = math.sqrt(n - L - 3)
        z64 = sq * abs(math.atanh(r64))
        kind, a, ind, dr = comp_test_fp32(P, R, 0, 1, f32(sq), f32(math.tanh(q / sq)))
        rows.append((kind, a, ind, z64 <= q, abs(r64), dr))
    trusted = [x for x in rows if x[0] == "trusted"]
    assert len(trusted) > 0.2 * len(rows)            # within 1 % of the threshold many are still decided
    assert any(x[0] == "queued" for x in rows)        # and others go to FP64
    for kind, a, ind, ind64, r64, dr in trusted:
        assert ind == ind64
        assert abs(float(a) - r64) <= float(dr)


def test_trusted_fp32_complement_far_from_threshold():
    # at the workloads' sizes most complement tests are far from the threshold:
    # there nearly all are decided in FP32, and the decisions are the FP64 ones
    rng = np.random.default_rng(29)
    q = -statistics.NormalDist().inv_cdf(0.005)
    n_trusted = n_all = 0
    while n_all < 400:
        C, P, R, r64, L = _comp_case(rng)
        n = int(rng.integers(500, 20000))
        sq = math.sqrt(n - L - 3)
        kind, a, ind, dr = comp_test_fp32(P, R, 0, 1, f32(sq), f32(math.tanh(q / sq)))
        n_all += 1
        if kind == "trusted":
            n_trusted += 1
            assert ind == (sq * abs(math.atanh(r64)) <= q)
            assert abs(float(a) - abs(r64)) <= float(dr)
    assert n_trusted > 0.6 * n_all


def test_complement_bound_holds_for_exact_perturbations():
    # the first-order bound (no rounding terms) against exact FP64 arithmetic:
    # perturbing P by symmetric dP with |dP_ij| <= eps s_i s_j moves r by at most
    # eps (W_u W_v / sqrt(Q_uu Q_vv) + |r|/2 (W_u^2/Q_uu + W_v^2/Q_vv))
    rng = np.random.default_rng(31)
    worst = 0.0
    for _ in range(300):
        C, P, R, r64, L = _comp_case(rng)
        m = P.shape[0]
        X = np.linalg.solve(P[np.ix_(R, R)], P[np.ix_(R, [0, 1])])
        Q = P[np.ix_([0, 1], [0, 1])] - P[np.ix_([0, 1], R)] @ X
        r = -Q[0, 1] / math.sqrt(Q[0, 0] * Q[1, 1])
        s = np.sqrt(np.diag(P))
        Wu = s[0] + s[R] @ np.abs(X[:, 0])
        Wv = s[1] + s[R] @ np.abs(X[:, 1])
        eps = 1e-9 * min(1.0, Q[0, 0] / Wu ** 2, Q[1, 1] / Wv ** 2)
        bound = eps * (Wu * Wv / math.sqrt(Q[0, 0] * Q[1, 1]) + abs(r) / 2 * (Wu ** 2 / Q[0, 0] + Wv ** 2 / Q[1, 1]))
        for _ in range(3):
            E = np.triu(rng.uniform(-eps, eps, (m, m)), 1)
            E = E + E.T + np.diag(rng.uniform(-eps, eps, m))
            P2 = P + E * np.outer(s, s)
            X2 = np.linalg.solve(P2[np.ix_(R, R)], P2[np.ix_(R, [0, 1])])
            Q2 = P2[np.ix_([0, 1], [0, 1])] - P2[np.ix_([0, 1], R)] @ X2
            r2 = -Q2[0, 1] / math.sqrt(Q2[0, 0] * Q2[1, 1])
            worst = max(worst, abs(r2 - r) / bound)
        assert abs(r - r64) <= 1e-9 * max(1.0, abs(r64))   # the complement identity itself
    assert worst <= 1.02
