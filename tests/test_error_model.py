"""The FP32 error model of the small-stage kernel's test (no GPU needed).

The kernel borders a Cholesky factor of the set's first l-1 members with the
last one in FP32 and trusts the decision only when the smallest pivot clears the
guard, the bound dr = 2(m eps32 + eps_C) / pivot stays below 1e-4, and |z - q|
clears band + 4 sqrt(n-l-3) dr / (1 - r^2) (Sec. 2.2.2 test, evaluated in r).
This file emulates that arithmetic in float32, in the kernel's order of
operations (separate multiply and subtract where the kernel fuses them: a
different rounding of the same size), on random correlation blocks of random
conditioning, with n chosen so that the FP64 statistic lies within 1 % of the
threshold.  Every decision the model trusts must equal the FP64 decision, with
the FP32 statistic's error well inside the distance to the threshold: for
correlations exact in FP32 (the FP32 GEMM and cast paths, eps_C = 1.2e-7) and
for entry errors of 2e-7 (the size the BF16x3 tensor-core GEMM typically leaves).
The split-precision product itself is emulated too: on SEM data of the workloads'
recipes its entry errors stay below the level at which the model stops holding."""
import math
import statistics

import numpy as np
import pytest

f32 = np.float32
GUARD, BAND, DR_MAX = 1e-3, 1e-3, 1e-4


def _rsqrt(x):
    return f32(1.0) / np.sqrt(f32(x), dtype=f32)


def lane_test_fp32(C32, L, eps_c, sqf, rq):
    """Nodes 0, 1 are u, v; 2 .. L the prefix; L+1 the border member.  Returns
    (kind, |r|, independent) with kind "trusted", "queued" or "dependent"."""
    K = L - 1
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
        tu, tv = f32(C32[0, sp[i]]), f32(C32[1, sp[i]])
        for c in range(i):
            tu = f32(tu - f32(lu[c] * Lp[i, c]))
            tv = f32(tv - f32(lv[c] * Lp[i, c]))
        lu[i], lv[i] = f32(tu * rl), f32(tv * rl)
    h11, h22, h12 = f32(1), f32(1), f32(C32[0, 1])
    for i in range(K):
        h11 = f32(h11 - f32(lu[i] * lu[i]))
        h22 = f32(h22 - f32(lv[i] * lv[i]))
        h12 = f32(h12 - f32(lu[i] * lv[i]))
    ls, x = [f32(0)] * max(K, 1), f32(1)
    for i in range(K):
        t = f32(C32[s, sp[i]])
        for c in range(i):
            t = f32(t - f32(ls[c] * Lp[i, c]))
        t = f32(t * rd[i])
        ls[i] = t
        x = f32(x - f32(t * t))
    cu, cv = f32(C32[s, 0]), f32(C32[s, 1])
    for i in range(K):
        cu = f32(cu - f32(lu[i] * ls[i]))
        cv = f32(cv - f32(lv[i] * ls[i]))
    pmin = min(pmin, x)
    bad |= not x > 1e-12
    rx = f32(1) / max(x, f32(1e-30))
    h11 = f32(h11 - f32(f32(cu * cu) * rx))
    h22 = f32(h22 - f32(f32(cv * cv) * rx))
    h12 = f32(h12 - f32(f32(cu * cv) * rx))
    pmin = min(pmin, h11, h22)
    bad |= not h11 > 1e-12 or not h22 > 1e-12
    e = f32(2.0) * (f32(L + 2) * f32(5.96e-8) + f32(eps_c))
    if bad or pmin < GUARD or e > DR_MAX * pmin:
        return "queued", None, None
    a = abs(f32(h12 * _rsqrt(f32(h11 * h22))))
    if a >= 1:
        return "dependent", a, False
    D = max(f32(1) - a * a, f32(1e-3))
    mn = min(a, rq)
    w = f32(1) - mn * mn
    if sqf * abs(a - rq) * D * pmin < f32(BAND) * D * w * pmin + f32(4) * sqf * e * w:
        return "queued", a, None
    return "trusted", a, bool(a <= rq)


def _cases(seed, count, entry_err, eps_c, nmin=0):
    rng = np.random.default_rng(seed)
    q = -statistics.NormalDist().inv_cdf(0.005)
    out = []
    while len(out) < count:
        L = int(rng.integers(1, 9))
        m = L + 2
        k = m + int(rng.integers(1, 40))            # few samples: some blocks near singular
        A = rng.standard_normal((k, m)) @ (np.eye(m) + 0.5 * rng.standard_normal((m, m)))
        C = np.corrcoef(A, rowvar=False)
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
        kind, a, ind = lane_test_fp32(C32, L, eps_c, f32(sq), f32(math.tanh(q / sq)))
        out.append((kind, a, ind, z64 <= q, z64, sq, q))
    return out


@pytest.mark.parametrize("regime", [("correlations exact in FP32", 0.0, 1.2e-7, 0),
                                    ("entry errors of 2e-7, n >= 1000", 2e-7, 1e-6, 1000)])
def test_trusted_fp32_decisions_equal_fp64(regime):
    label, entry_err, eps_c, nmin = regime
    rows = _cases(11, 2500 if nmin == 0 else 300, entry_err, eps_c, nmin)
    trusted = [r for r in rows if r[0] == "trusted"]
    assert len(trusted) > 0.2 * len(rows)             # near the threshold the model still trusts many
    assert any(r[0] == "queued" for r in rows)        # and queues some for FP64
    for kind, a, ind, ind64, z64, sq, q in trusted:
        assert ind == ind64, label
        # the FP32 statistic's error stays well inside the distance to the threshold
        assert abs(sq * math.atanh(float(a)) - z64) < 0.5 * abs(z64 - q), label


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
def test_bf16x3_entry_errors_stay_below_the_models_breakdown(shape):
    # on SEM data of the workloads' recipes the split-precision correlations stay well
    # below the +-5e-7 entry error from which the emulated model stops holding
    from paper_2109_04626_gb300 import sem
    p, n, prob = shape
    rng = np.random.Generator(np.random.PCG64(77))
    dag, W, order = sem.er_dag(p, prob if prob else 10.0 / (p - 1), rng)
    X = sem.sample(W, order, n, rng)
    Xs = (X - X.mean(0)) / X.std(0)
    C64 = Xs.T @ Xs / n
    E = np.abs(_corr_bf16x3(Xs).astype(np.float64) - C64)
    np.fill_diagonal(E, 0.0)
    assert E.max() < 5e-7
    assert np.median(E[np.triu_indices(p, 1)]) < 1e-7
