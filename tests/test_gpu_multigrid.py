"""GPU parity of the multigrid-preconditioned solves (qpat_params.multigrid)
against the CPU FP64 oracle, through the C ABI.

The preconditioner changes the iteration, not the solution: every solve
still stops at |b - A x| <= pcg_rtol |b| = 1e-13 |b|, so the bars are those
of the persistent PCG (tests/test_gpu_parity.py): 1e-10 relative L2 for the
K solves and their J s, J^T t (cond(K) < 1e3), and the normwise backward
error plus 10 cond(M_delta) 1e-13 for M_delta.  Multigrid 1 runs the
V-cycle in FP64, multigrid 2 runs the K cycle in FP32 under FP64 CG.
"""
import numpy as np
import pytest

import oracle as O
import qpat_synth as S
from tests.gpu_common import Case, rel, small_cases
from tests.test_gpu_parity import cond_mdelta

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu

CASES = dict(small_cases())
CASES["cube24_K4"] = S.small_config(24, 16.0, 4, 5)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(CASES[request.param])
    c.lib = Q.qpat_mesh(c.xyz, c.tets, patch_nodes=64 if c.N > 64 else 32)
    yield c
    c.lib.close()


def _mg(mg, **kw):
    return Q.qpat_default_params(multigrid=mg, **kw)


@pytest.mark.parametrize("mg", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_forward(case, mg, precision):
    case.lib.reset_stats()
    phi, h = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, _mg(mg, precision=precision))
    assert rel(phi, case.phi) < 1e-10
    assert rel(h, case.h) < 1e-10
    # a handful of V-cycles instead of hundreds of Jacobi steps
    assert case.lib.stats()["pcg_iters"] <= 40


@pytest.mark.parametrize("mg", [1, 2])
def test_jvp_vjp_pair(case, mg):
    rng = np.random.default_rng(5)
    s = rng.standard_normal(2 * case.N)
    t = rng.standard_normal((case.K, case.N))
    prm = _mg(mg)
    out = Q.qpat_jvp(case.lib, case.kappa, case.mu, case.phi, s, case.w, prm)
    assert rel(out, O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)) < 1e-10
    ref = O.vjp(case.om, case.kappa, case.mu, case.phi, t, case.w, case.fac)
    out = Q.qpat_vjp(case.lib, case.kappa, case.mu, case.phi, t, case.w, prm)
    assert rel(out[:case.N], ref[:case.N]) < 1e-10
    assert rel(out[case.N:], ref[case.N:]) < 1e-10
    if case.K <= 8:
        oj, ov = Q.qpat_jvp_vjp_pair(case.lib, case.kappa, case.mu, case.phi, s, t, case.w, prm)
        assert rel(oj, O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)) < 1e-10
        assert rel(ov, ref) < 1e-10


@pytest.mark.parametrize("prior,q", [(0, 1.0), (1, 1.0), (1, 2.0)])
def test_prior_solve(case, prior, q):
    rng = np.random.default_rng(13)
    N = case.N
    kt = 0.3 * rng.standard_normal(N)
    mt = np.log(case.mu / case.mu.mean())
    rhs = rng.standard_normal(2 * N)
    T, ba, delta = 1e-2, 0.7, 1e-6
    Md = O.prior_matrix(case.om, kt, mt, T, ba, delta, prior=prior, q=q)
    ref = O.Factor(Md).solve(rhs)
    case.lib.reset_stats()
    out = Q.qpat_prior_solve(case.lib, kt, mt, rhs, _mg(1, T=T, b_over_a=ba, delta=delta, prior=prior, prior_q=q))
    Anorm = abs(Md).sum(axis=0).max()
    eta = np.linalg.norm(Md @ out - rhs, 1) / (Anorm * np.linalg.norm(out, 1) + np.linalg.norm(rhs, 1))
    assert eta < 1e-13
    assert rel(out, ref) < max(10 * cond_mdelta(Md, delta) * 1e-13, 1e-10)


def test_runs_are_bit_identical(case):
    """Fixed-order set-up and reductions: the same call twice gives the same bits."""
    prm = _mg(1)
    a, _ = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, prm)
    b, _ = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, prm)
    np.testing.assert_array_equal(a, b)


def test_hierarchy_shape(case):
    Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, _mg(1))
    rows = case.lib.multigrid_levels()
    assert rows[0] == case.N and rows[-1] <= 128
    assert rows == Q.qpat_multigrid_host_info(case.xyz, case.tets, patch_nodes=64 if case.N > 64 else 32)


def test_initial_guess(case):
    """A guess changes the work, not the accuracy (same absolute target)."""
    dev = torch.device("cuda")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    phi = torch.empty((case.K, case.N), dtype=torch.float64, device=dev)
    h = torch.empty_like(phi)
    guess = case.phi * (1 + 1e-3 * np.random.default_rng(3).standard_normal(case.phi.shape))
    Q.qpat_forward_guess_dev(case.lib, T(case.kappa), T(case.mu), T(case.flux), T(guess), phi, h, _mg(1))
    torch.cuda.synchronize()
    assert rel(phi.cpu().numpy(), case.phi) < 1e-10


def test_parameter_checks(case):
    for bad in (dict(multigrid=3), dict(multigrid=1, mg_degree=9), dict(multigrid=1, mg_ratio=0.5)):
        with pytest.raises(Q.QpatError):
            Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, Q.qpat_default_params(**bad))


def test_graph_loop_equals_host_loop(case):
    """Without timing the CG iterations run as a captured graph whose "while"
    node is driven by the device; with timing on they are launched from the
    host one by one.  The same kernels on the same data: the same bits and
    the same iteration count."""
    prm = _mg(1)
    case.lib.reset_stats()
    a, _ = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, prm)
    ia = case.lib.stats()["pcg_iters"]
    case.lib.set_timing(True)
    try:
        case.lib.reset_stats()
        b, _ = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, prm)
        ib = case.lib.stats()["pcg_iters"]
        ms, launches = case.lib.multigrid_fine_time()
    finally:
        case.lib.set_timing(False)
    np.testing.assert_array_equal(a, b)
    assert ia == ib
    if len(case.lib.multigrid_levels()) > 1:
        assert launches == ib and ms > 0.0


def test_iteration_cap_and_restart(case):
    """A cap below the need ends the graph loop with QPAT_ENOCONV; the next
    solve on the same handle is exact again."""
    if case.N <= 128:
        pytest.skip("one level: the exact coarse solve converges at once")
    with pytest.raises(Q.QpatError):
        Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, _mg(1, max_pcg_iter=1))
    phi, _ = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, _mg(1))
    assert rel(phi, case.phi) < 1e-10
