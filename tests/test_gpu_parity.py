"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle.

Bars: partial correlations within 1e-5 absolute, decisions and the
removed-edge set bit-exact, sepsets (level, side, rank, nodes) identical, and
the sequential canonical test count equal to the oracle's.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import sem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

R_TOL = 1e-5


@pytest.fixture(scope="module")
def fp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04626_gb300 import build
    from paper_2109_04626_gb300 import fastpc
    build.build()
    fastpc.load()
    return fastpc


def _sem_case(seed, p, n, prob, dtype=np.float32):
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, prob, rng)
    X = sem.sample(W, order, n, rng).astype(dtype)
    return np.ascontiguousarray(X)


def _run_gpu(fp, X, alpha, max_level, order, precision, complement=1, device_input=True, **opts):
    n, p = X.shape
    with fp.PC(n, p, alpha, max_level, order=order, precision=precision,
               complement=complement, **opts) as pc:
        pc.corr(torch.from_numpy(X).cuda() if device_input else X)
        adj, st = pc.skeleton()
        seps = pc.sepsets()
    return adj, st, seps


def _check_skeleton(fp, X, alpha=0.01, max_level=-1, order=1, precision=2, complement=1,
                    device_input=True, **opts):
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, alpha, max_level, reversed_order=bool(order))
    adj, st, seps = _run_gpu(fp, X, alpha, max_level, order, precision, complement, device_input, **opts)
    np.testing.assert_array_equal(adj, R["adj"])
    assert seps == R["sepsets"]
    assert st["tests_canonical"] == R["tests_total"]
    assert st["tests_executed"] >= st["tests_canonical"] or st["tests_executed"] > 0 or \
        R["tests_total"] == 0
    return R, st


# --------------------------------------------------------------------------- correlation
@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape", [(1000, 20, np.float64), (5000, 95, np.float32),
                                   (3001, 70, np.float32), (257, 129, np.float64)])
def test_corr_matches_oracle(fp, precision, shape):
    n, p, dt = shape
    X = _sem_case(11 + p, p, n, 0.2, dt)
    with fp.PC(n, p, 0.01, -1, precision=precision) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        C32, C64 = pc.corr_get()
    Co = oracle.pearson(X)
    assert np.abs(C64 - Co).max() <= 1e-12
    assert np.abs(C32.astype(np.float64) - Co).max() <= 2e-6
    assert np.all(np.diag(C32) == 1.0) and np.all(np.diag(C64) == 1.0)


@pytest.mark.parametrize("pad", [0, 3])
def test_corr_large_means_and_strided_rows(fp, pad):
    # FP32 columns whose means are large against their spread (the statistics take
    # x - mean in split FP32 arithmetic), read through a row stride that is not a
    # multiple of 4 floats when pad = 3 (per-element loads instead of 16-byte rows)
    n, p = 2113, 45
    X = _sem_case(23, p, n, 0.3, np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    X = X * rng.uniform(0.01, 3.0, p) + rng.choice([-1.0, 1.0], p) * 10.0 ** rng.uniform(0, 4, p)
    X = X.astype(np.float32)
    W = np.zeros((n, p + pad), dtype=np.float32)
    W[:, :p] = X
    Xd = torch.from_numpy(W).cuda()[:, :p]
    with fp.PC(n, p, 0.01, -1, precision=2) as pc:
        pc.corr(Xd)
        C32, C64 = pc.corr_get()
    Co = oracle.pearson(X)
    # the oracle's own FP64 rounding of x - mean is about 1e-16 * |mean| / sd here
    assert np.abs(C64 - Co).max() <= 1e-10
    assert np.abs(C32.astype(np.float64) - Co).max() <= 2e-6


def test_corr_host_input_equals_device_input(fp):
    X = _sem_case(5, 40, 2000, 0.3)
    n, p = X.shape
    with fp.PC(n, p, 0.01) as pc:
        pc.corr(X)
        A32, A64 = pc.corr_get()
        pc.corr(torch.from_numpy(X).cuda())
        B32, B64 = pc.corr_get()
    np.testing.assert_array_equal(A64, B64)
    np.testing.assert_array_equal(A32, B32)


# --------------------------------------------------------------------------- raw CI tests
def _random_tests(rng, p, l, b):
    ij = np.empty((b, 2), dtype=np.int32)
    S = np.empty((b, max(l, 1)), dtype=np.int32)
    for k in range(b):
        nodes = rng.choice(p, size=l + 2, replace=False)
        ij[k] = nodes[:2]
        S[k, :l] = np.sort(nodes[2:])
    return ij, S[:, :l].copy()


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("case", ["p95_dense", "p20_fp64", "er_moderate"])
def test_ci_batch_parity(fp, precision, case):
    if case == "p95_dense":
        s = sem.make(2)
        X = s.X
        levels = [0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 80, 93]
    elif case == "p20_fp64":
        X = sem.make(1).X
        levels = [0, 1, 2, 4, 7, 11, 18]
    else:
        X = _sem_case(77, 200, 4000, 0.03)
        levels = [0, 1, 2, 3, 4, 6, 9, 14, 20, 31, 50]
    n, p = X.shape
    C = oracle.pearson(X)
    q = oracle.threshold(0.01)
    rng = np.random.default_rng(2024)
    with fp.PC(n, p, 0.01, -1, precision=precision) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        for l in levels:
            b = 257
            ij, S = _random_tests(rng, p, l, b)
            r, ind, z = pc.ci_batch(torch.from_numpy(ij).cuda(), torch.from_numpy(S).cuda(), l)
            r = r.cpu().numpy()
            ind = ind.cpu().numpy().astype(bool)
            z = z.cpu().numpy()
            ro, zo, io, do = oracle.ci_batch(C, n, 0.01, ij, S)
            assert np.abs(r - ro).max() <= R_TOL, (l, np.abs(r - ro).max())
            clear = np.abs(zo - q) > 1e-9
            np.testing.assert_array_equal(ind[clear], io[clear])


def test_ci_batch_errors(fp):
    X = _sem_case(3, 12, 10, 0.3)
    n, p = X.shape                                     # n = 10, p = 12
    with fp.PC(n, p, 0.01) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        ij = torch.tensor([[0, 1]], dtype=torch.int32, device="cuda")
        S = torch.arange(2, 12, dtype=torch.int32, device="cuda").reshape(1, 10)
        with pytest.raises(fp.PCError) as e:           # l = 11 > p - 2
            pc.ci_batch(ij, torch.zeros((1, 11), dtype=torch.int32, device="cuda"), 11)
        assert e.value.status == 1
        with pytest.raises(fp.PCError) as e:           # n - l - 3 = 0: Fisher z undefined
            pc.ci_batch(ij, S[:, :7].contiguous(), 7)
        assert e.value.status == 5
        bad = torch.tensor([[0, 99]], dtype=torch.int32, device="cuda")
        with pytest.raises(fp.PCError) as e:           # node id out of range
            pc.ci_batch(bad, S[:, :1].contiguous(), 1)
        assert e.value.status == 1
        same = torch.tensor([[4, 4]], dtype=torch.int32, device="cuda")
        with pytest.raises(fp.PCError) as e:           # u == v
            pc.ci_batch(same, S[:, :1].contiguous(), 1)
        assert e.value.status == 1
        r, ind, z = pc.ci_batch(ij, S[:, :2].contiguous(), 2)    # the handle still works
        assert r.shape == (1,)


# --------------------------------------------------------------------------- skeletons
@pytest.mark.parametrize("order", [1, 0])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_skeleton_p20_fp64(fp, order, precision):
    _check_skeleton(fp, sem.make(1).X, order=order, precision=precision)


@pytest.mark.parametrize("complement", [1, 0])
@pytest.mark.parametrize("precision", [0, 2])
def test_skeleton_p95_dense_reversed(fp, complement, precision):
    R, st = _check_skeleton(fp, sem.make(2).X, order=1, precision=precision,
                            complement=complement)
    assert st["stage_a_ran"] == 1
    if complement:
        assert st["complement_tests"] > 0


def test_skeleton_p95_dense_conventional(fp):
    _check_skeleton(fp, sem.make(2).X, order=0, precision=2)


def _hub_case(seed=613, p=70, hub_degree=20, n=30000):
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.hub_dag(p, rng, mean_degree=3.0, hubs=3, hub_degree=hub_degree, lo=0.4, hi=0.9)
    return np.ascontiguousarray(sem.sample(W, order, n, rng).astype(np.float32))


@pytest.mark.parametrize("precision", [1, 2])
def test_skeleton_deep_stages_conventional(fp, precision):
    """Three hubs of degree 20 keep their edges to stage 15 (Algorithm 1): stages 9-12
    run on the register-resident small-stage kernel (ranges 9-10 and 11-12), 13-15 on
    the warp-per-test kernel."""
    X = _hub_case()
    R, st = _check_skeleton(fp, X, order=0, precision=precision)
    assert R["levels"][-1] >= 13 and sum(int(t) for t in R["tests_level"][9:13]) > 10 ** 5
    assert st["levels_run"] == len(R["levels"])


def test_skeleton_deep_stages_proposal_order(fp):
    """The same stages with a proposal order (random network parameters, scored up
    to l = 12): the skeleton equals the oracle's, every set separates in FP64."""
    X = _hub_case()
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=False)
    theta = np.random.default_rng(8).standard_normal(fp.pc_mlp_nparam()).astype(np.float32) * 0.2
    with fp.PC(n, p, 0.01, -1, order=0) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        fp.pc_mlp_set_params(pc.h, theta)
        for k, v in (("learned", 1), ("learned_min_tests", 0), ("learned_min_ratio", 0),
                     ("learned_max_level", 12)):
            fp.pc_set_opt(pc.h, k, v)
        adj, st = pc.skeleton()
        seps = pc.sepsets()
    np.testing.assert_array_equal(adj, R["adj"])
    assert set(seps) == set(R["sepsets"])
    for (a, b), (lv, side, rank, nodes) in seps.items():
        assert lv == R["sepsets"][(a, b)][0]
        assert oracle.ci_test(C, n, 0.01, a, b, list(nodes))[0]


@pytest.mark.parametrize("pair_warp", [0, 1])
@pytest.mark.parametrize("node_dmax", [0, 5, 12, 128])
@pytest.mark.parametrize("case", ["p95_conventional", "hub", "p95_reversed"])
def test_skeleton_staged_and_global_small_stages(fp, case, node_dmax, pair_warp):
    # pair_warp_dmin 4: the warp-per-pair kernel takes every node of degree > 4 at
    # stages 1 and 2 (the default 32 leaves the small ones to the staged kernel)
    """The small stages split between the staged kernel (nodes of degree <=
    node_dmax: corr block in shared memory), the warp-per-pair kernel (stages 1
    and 2, the other nodes) and the kernel reading corr from L2 (the rest); every
    split gives the oracle's skeleton, sets and counts."""
    if case == "hub":
        X, order = _hub_case(), 0
    else:
        X, order = sem.make(2).X, (1 if case == "p95_reversed" else 0)
    for precision in (1, 2):
        for dmin in (4, 32):
            _check_skeleton(fp, X, order=order, precision=precision, node_dmax=node_dmax, pair_warp=pair_warp,
                            pair_warp_dmin=dmin)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_stage_loop_in_one_kernel_equals_captured_loop(fp, precision):
    """The reversed order's complement-only stages in one cooperative kernel
    (option stage_loop) or in the captured stage loop: the oracle's skeleton,
    sets, counts and stages either way -- dense and sparse problems, a problem
    whose later stages have direct tests (the kernel hands over to the captured
    loop), a level cap, p at the kernel's limit, host-driven and timed loops."""
    cases = [(sem.make(2).X, -1), (_sem_case(91, 60, 4000, 0.4), -1), (_sem_case(94, 128, 3000, 0.3), -1),
             (_sem_case(95, 40, 600, 0.6), -1), (_sem_case(95, 40, 600, 0.6), 25), (sem.make(1).X, -1)]
    for X, ml in cases:
        for opts in ({"stage_loop": 1}, {"stage_loop": 0}, {"stage_loop": 1, "graph": 0}):
            R, st = _check_skeleton(fp, X, max_level=ml, order=1, precision=precision, **opts)
            assert st["levels_run"] == len(R["levels"])
    X = sem.make(2).X
    n, p = X.shape
    with fp.PC(n, p, 0.01, -1, order=1, timing=1) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        pc.skeleton()
        tm = fp.pc_timing(pc.h)
        assert tm["stage_loop"][1] == 1 and tm["stage_loop"][0] > 0


def test_complement_fp32_first_equals_fp64(fp):
    """The complement tests of the reversed order in FP32 first (decided there
    only under the error bound) or in FP64 only: the oracle's skeleton, sets and
    counts either way; with FP32 first most complement tests are decided in FP32
    (the FP64 re-decisions they add are few)."""
    cases = [sem.make(2).X, _sem_case(91, 60, 4000, 0.4), _sem_case(92, 120, 2000, 0.3),
             _sem_case(93, 80, 800, 0.5)]
    for X in cases:
        _, st0 = _check_skeleton(fp, X, order=1, comp_fp32=0)
        _, st1 = _check_skeleton(fp, X, order=1, comp_fp32=1)
        # executed counts are speculative (a test is skipped once an earlier set of its
        # pair is recorded, which depends on timing); the canonical counts are checked above
        assert st1["tests_redecided"] - st0["tests_redecided"] <= 0.5 * st1["complement_tests"]


def test_staged_kernel_proposal_order(fp):
    """The staged kernel in the proposal order: the sets of a pair are enumerated
    over its permuted candidate list (neighbour indices into the staged block)."""
    X = _hub_case()
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=False)
    theta = np.random.default_rng(9).standard_normal(fp.pc_mlp_nparam()).astype(np.float32) * 0.2
    for node_dmax, pair_warp in ((0, 0), (0, 1), (10, 1), (128, 0), (128, 1)):
        with fp.PC(n, p, 0.01, -1, order=0, node_dmax=node_dmax, pair_warp=pair_warp) as pc:
            pc.corr(torch.from_numpy(X).cuda())
            fp.pc_mlp_set_params(pc.h, theta)
            pc.set(learned=1, learned_min_tests=0, learned_min_ratio=0, learned_max_level=12)
            adj, st = pc.skeleton()
            seps = pc.sepsets()
        np.testing.assert_array_equal(adj, R["adj"])
        assert set(seps) == set(R["sepsets"])
        for (a, b), (lv, side, rank, nodes) in seps.items():
            assert lv == R["sepsets"][(a, b)][0]
            assert oracle.ci_test(C, n, 0.01, a, b, list(nodes))[0]


@pytest.mark.parametrize("seed", range(6))
def test_skeleton_random_small(fp, seed):
    rng = np.random.default_rng(seed)
    p = int(rng.integers(5, 70))
    n = int(rng.integers(p + 10, 3000))
    X = _sem_case(300 + seed, p, n, float(rng.uniform(0.05, 0.5)))
    for order in (1, 0):
        _check_skeleton(fp, X, alpha=float(rng.choice([0.01, 0.05, 1e-3])), order=order,
                        precision=int(rng.integers(0, 3)))


@pytest.mark.parametrize("max_level", [0, 1, 3])
@pytest.mark.parametrize("order", [1, 0])
def test_skeleton_max_level(fp, max_level, order):
    X = _sem_case(41, 30, 1500, 0.3)
    _check_skeleton(fp, X, max_level=max_level, order=order)


def test_skeleton_edge_cases(fp):
    # two and three variables
    for p in (2, 3):
        X = _sem_case(50 + p, p, 200, 0.9)
        for order in (1, 0):
            _check_skeleton(fp, X, order=order)
    # few samples: stages capped at n - 4, stage l=p-2 skipped when n - p - 1 <= 0
    X = _sem_case(61, 12, 9, 0.4)
    for order in (1, 0):
        _check_skeleton(fp, X, order=order, precision=0)
    # an empty graph (independent columns) and a ragged p not a multiple of 32
    X = np.random.default_rng(3).standard_normal((800, 37)).astype(np.float32)
    for order in (1, 0):
        _check_skeleton(fp, X, order=order)


@pytest.mark.parametrize("order", [1, 0])
def test_skeleton_constant_column(fp, order):
    # Reading R18: a constant column correlates 0 with everything (GPU: 1/sd := 0)
    X = _sem_case(73, 30, 1500, 0.2)
    X[:, 11] = 3.25
    _check_skeleton(fp, X, order=order)


def test_skeleton_maximum_p(fp):
    # the largest p a handle accepts (4096), conventional order up to l = 1
    rng = np.random.Generator(np.random.PCG64(4096))
    dag, W, order = sem.er_dag(4096, 3.0 / 4095, rng)
    X = np.ascontiguousarray(sem.sample(W, order, 1000, rng).astype(np.float32))
    _check_skeleton(fp, X, max_level=1, order=0)


def test_skeleton_degenerate_duplicate_column(fp):
    X = _sem_case(71, 15, 1200, 0.3, np.float64)
    X[:, 9] = X[:, 4]                                  # exactly collinear pair
    R, st = _check_skeleton(fp, X, order=0, precision=0)
    assert st["degenerate"] > 0 or R["degenerate"] == 0


@pytest.mark.parametrize("precision", [0, 2])
def test_stage_a_singular_cluster_sweep(fp, precision):
    # an exactly collinear pair makes corr singular, so the closed-form stage is
    # skipped as in the oracle
    X = _sem_case(73, 48, 4000, 0.2, np.float64)
    X[:, 30] = X[:, 7]
    R, st = _check_skeleton(fp, X, order=1, precision=precision)
    assert R["stageA_ran"] is False or R["stageA_ran"] == 0
    assert st["stage_a_ran"] == 0


def test_stage_a_singular_on_the_cluster(fp):
    # on the cluster a singular corr ends the sweep at the same pivot in every CTA
    # (the stage is skipped as in the oracle); the cap keeps the enumerated stages
    # of the complete graph small
    rng = np.random.Generator(np.random.PCG64(7300))
    dag, W, order = sem.er_dag(200, 0.02, rng)
    X = np.ascontiguousarray(sem.sample(W, order, 4000, rng))
    X[:, 150] = X[:, 7]
    for ml in (0, 1):
        R, st = _check_skeleton(fp, X, max_level=ml, order=1, precision=2)
        assert st["stage_a_ran"] == 0 and not R["stageA_ran"]


@pytest.mark.parametrize("p", [32, 57, 130, 200, 330])
def test_stage_a_cluster_sizes(fp, p):
    # the closed-form stage's inverse: the sweep over a cluster of 8 CTAs with ragged
    # row blocks (p not a multiple of 8)
    X = _sem_case(90 + p, p, max(2000, 4 * p), 0.15 if p < 100 else (0.04 if p < 150 else 0.015))
    R, st = _check_skeleton(fp, X, order=1, precision=2)
    assert st["stage_a_ran"] == int(bool(R["stageA_ran"]))


def test_skeleton_host_buffers(fp):
    X = sem.make(1).X
    _check_skeleton(fp, X, device_input=False)


def test_skeleton_on_torch_stream(fp):
    X = sem.make(1).X
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, True)
    s = torch.cuda.Stream()
    with fp.PC(n, p, 0.01) as pc:
        fp.pc_set_stream(pc.h, s)
        Xd = torch.from_numpy(X).cuda()
        s.wait_stream(torch.cuda.current_stream())
        pc.corr(Xd)
        adj_d = torch.empty((p, p), dtype=torch.uint8, device="cuda")
        pc.skeleton(adj_d)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(adj_d.cpu().numpy(), R["adj"])


def test_repeated_calls_reuse_handle(fp):
    X = _sem_case(81, 25, 900, 0.3)
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, True)
    with fp.PC(n, p, 0.01) as pc:
        for _ in range(3):
            pc.corr(torch.from_numpy(X).cuda())
            adj, st = pc.skeleton()
            np.testing.assert_array_equal(adj, R["adj"])
            assert pc.sepsets() == R["sepsets"]


# --------------------------------------------------------------------------- full-size workloads
@pytest.mark.parametrize("cfg", [3, 4])
def test_full_size_conventional(fp, cfg):
    """p=500 power law (levels <= 8) and p=1000 ER, conventional order (Algorithm 1)."""
    w = sem.WORKLOADS[cfg]
    X = sem.make(cfg).X
    _check_skeleton(fp, X, alpha=w["alpha"], max_level=w["max_level"], order=0, precision=2)


@pytest.mark.parametrize("mode", ["host_loop", "timed"])
def test_stage_loop_drivers_agree(fp, mode):
    """The captured stage loop (CUDA graph, conditional WHILE) and the
    host-driven loop (used for per-kernel timing) give the same result."""
    for cfg, order in ((2, 1), (1, 0), (1, 1)):
        X = sem.make(cfg).X
        n, p = X.shape
        C = oracle.pearson(X)
        R = oracle.skeleton(C, n, 0.01, -1, reversed_order=bool(order))
        opts = {"graph": 0} if mode == "host_loop" else {"timing": 1}
        with fp.PC(n, p, 0.01, -1, order=order, **opts) as pc:
            pc.corr(torch.from_numpy(X).cuda())
            adj, st = pc.skeleton()
            np.testing.assert_array_equal(adj, R["adj"])
            assert pc.sepsets() == R["sepsets"]
            assert st["tests_canonical"] == R["tests_total"]
            assert st["levels_run"] == len(R["levels"])
            if mode == "timed":
                tm = fp.pc_timing(pc.h)
                assert tm["bookkeeping"][1] > 0 and tm["corr"][1] > 0
                # the GEMM kernels are timed inside the correlation step
                assert tm["corr_gemm"][1] > 0 and 0 < tm["corr_gemm"][0] <= tm["corr"][0]


def test_levels_run_and_first_level_match_schedule(fp):
    X = sem.make(2).X
    n, p = X.shape
    C = oracle.pearson(X)
    for order in (1, 0):
        R = oracle.skeleton(C, n, 0.01, -1, reversed_order=bool(order))
        with fp.PC(n, p, 0.01, -1, order=order) as pc:
            pc.corr(torch.from_numpy(X).cuda())
            adj, st = pc.skeleton()
        assert st["levels_run"] == len(R["levels"])
        lv = R["levels"][1:] if order else R["levels"]
        assert st["first_level"] == lv[0]


def test_skeleton_many_concurrent_matches_oracle(fp):
    """pc_skeleton_many: independent problems on their own streams, each identical
    to the oracle; a problem over its test budget fails alone."""
    cases = [(101, 40, 2000, 0.3, 1), (102, 73, 5000, 0.25, 1), (103, 25, 800, 0.5, 0),
             (104, 96, 3000, 0.08, 0), (105, 57, 9000, 0.2, 1), (106, 31, 1200, 0.35, 1)]
    pcs, ps, refs, streams = [], [], [], []
    for seed, p, n, prob, order in cases:
        X = _sem_case(seed, p, n, prob)
        C = oracle.pearson(X)
        refs.append(oracle.skeleton(C, n, 0.01, -1, reversed_order=bool(order)))
        pc = fp.PC(n, p, 0.01, -1, order=order)
        s = torch.cuda.Stream()
        fp.pc_set_stream(pc.h, s)
        pc.corr(torch.from_numpy(X).cuda())
        pcs.append(pc)
        ps.append(p)
        streams.append(s)
    # one extra problem whose first stage exceeds its budget
    Xb = _sem_case(107, 60, 3000, 0.3)
    pcb = fp.PC(3000, 60, 0.01, -1, order=0, budget=10)
    fp.pc_set_stream(pcb.h, torch.cuda.Stream())
    pcb.corr(torch.from_numpy(Xb).cuda())
    adjs, stats, status = fp.pc_skeleton_many([pc.h for pc in pcs] + [pcb.h], ps + [60])
    assert status[-1] == 6 and adjs[-1] is None
    for pc, adj, st, code, R in zip(pcs, adjs, stats, status, refs):
        assert code == 0
        np.testing.assert_array_equal(adj, R["adj"])
        assert pc.sepsets() == R["sepsets"]
        assert st["tests_canonical"] == R["tests_total"]
    for pc in pcs + [pcb]:
        pc.close()
