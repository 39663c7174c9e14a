"""GPU parity of the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances (relative L2 per field):
  operator apply FP64      1e-13  (summation order only)
  operator apply FP32      2e-6   (FP32 coordinates and arithmetic)
  forward, J s, J^T t      1e-10  (FP64 PCG and FP32 PCG + FP64 refinement,
                                   both to a relative residual of 1e-13;
                                   error <= cond(K) * 1e-13 with cond(K) < 1e3)
  M_delta^-1               bounded by cond(M_delta) * 1e-12 (computed per case)
"""
import numpy as np
import pytest

import oracle as O
import qpat_synth as S
from tests.gpu_common import Case, rel, small_cases

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu

CASES = small_cases()


def cond_mdelta(Md, delta):
    """cond(M_delta) = lambda_max / delta: M_delta = blkdiag(M(kt), (b/a) M(mt))
    + delta I with both stiffness blocks symmetric positive semi-definite and
    annihilating the constants (natural boundary condition), so delta is its
    smallest eigenvalue exactly; lambda_max comes from a Lanczos run."""
    import scipy.sparse.linalg as spla
    lmax = spla.eigsh(Md, k=1, which="LA", return_eigenvectors=False, tol=1e-6)[0]
    return lmax / delta


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    _need_gpu()
    c = Case(CASES[request.param])
    c.lib = Q.qpat_mesh(c.xyz, c.tets, patch_nodes=64 if c.N > 64 else 32)
    yield c
    c.lib.close()


def _params(precision=0, **kw):
    return Q.qpat_default_params(precision=precision, **kw)


def test_mesh_faces_and_flux(case):
    np.testing.assert_array_equal(case.lib.faces(), case.om.faces)
    if hasattr(case.cfg, "illuminations"):
        for k, il in enumerate(case.cfg.illuminations):
            f = Q.qpat_flux_side(case.lib, il.center, il.axis, il.ref, case.cfg.R, il.theta0, il.half_w, il.amp)
            np.testing.assert_array_equal(f != 0, case.flux[k] != 0)
            # the two sides evaluate the centroid angle in a different order
            np.testing.assert_allclose(f, case.flux[k], rtol=1e-13, atol=1e-15)
        return
    for k, p in enumerate(case.cfg.patches):
        f = Q.qpat_flux_patch(case.lib, p.center, p.normal, p.half_w, p.amp)
        np.testing.assert_array_equal(f, case.flux[k])


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6), (2, 1e-13), (3, 2e-6)])
@pytest.mark.parametrize("R", [1, 3, 4, 8])
def test_apply_K(case, precision, tol, R):
    rng = np.random.default_rng(R)
    x = rng.standard_normal((case.N, R))
    y_ref = case.Kmat @ x
    dev = torch.device("cuda")
    xt = torch.tensor(x, device=dev)
    yt = torch.empty_like(xt)
    Q.qpat_apply_K_dev(case.lib, torch.tensor(case.kappa, device=dev), torch.tensor(case.mu, device=dev), xt, yt,
                       precision)
    torch.cuda.synchronize()
    assert rel(yt.cpu().numpy(), y_ref) < tol


# pcg_variant 1: two grid reductions per PCG iteration, 2: one (Chronopoulos-Gear),
# 3: two, with the operator streamed through a shared-memory ring by bulk copies
@pytest.mark.parametrize("precision,fp32_op,variant", [(0, 0, 1), (0, 0, 2), (0, 0, 3), (1, 0, 1), (1, 1, 1),
                                                       (1, 1, 2), (1, 1, 3)])
def test_forward(case, precision, fp32_op, variant):
    phi, h = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux,
                            _params(precision, fp32_operator=fp32_op, pcg_variant=variant))
    assert rel(phi, case.phi) < 1e-10
    assert rel(h, case.h) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_jvp(case, precision):
    rng = np.random.default_rng(5)
    s = rng.standard_normal(2 * case.N)
    ref = O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)
    out = Q.qpat_jvp(case.lib, case.kappa, case.mu, case.phi, s, case.w, _params(precision))
    assert rel(out, ref) < 1e-10
    out1 = Q.qpat_jvp(case.lib, case.kappa, case.mu, case.phi, s, None, _params(precision))
    assert rel(out1, O.jvp(case.om, case.kappa, case.mu, case.phi, s, None, case.fac)) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_vjp(case, precision):
    rng = np.random.default_rng(6)
    t = rng.standard_normal((case.K, case.N))
    ref = O.vjp(case.om, case.kappa, case.mu, case.phi, t, case.w, case.fac)
    out = Q.qpat_vjp(case.lib, case.kappa, case.mu, case.phi, t, case.w, _params(precision))
    assert rel(out[:case.N], ref[:case.N]) < 1e-10
    assert rel(out[case.N:], ref[case.N:]) < 1e-10


def test_adjoint_identity_on_gpu(case):
    rng = np.random.default_rng(7)
    v = rng.standard_normal(2 * case.N)
    t = rng.standard_normal((case.K, case.N))
    a = np.sum(Q.qpat_jvp(case.lib, case.kappa, case.mu, case.phi, v, case.w) * t)
    b = v @ Q.qpat_vjp(case.lib, case.kappa, case.mu, case.phi, t, case.w)
    assert abs(a - b) <= 1e-10 * abs(a)


def test_pair_matches_separate_calls(case):
    if case.K > 8:
        pytest.skip("pair needs K <= 8")
    dev = torch.device("cuda")
    rng = np.random.default_rng(8)
    s = rng.standard_normal(2 * case.N)
    t = rng.standard_normal((case.K, case.N))
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    oj = torch.empty((case.K, case.N), dtype=torch.float64, device=dev)
    ov = torch.empty(2 * case.N, dtype=torch.float64, device=dev)
    Q.qpat_jvp_vjp_pair_dev(case.lib, T(case.kappa), T(case.mu), T(case.phi), T(case.w), T(s), T(t), oj, ov)
    torch.cuda.synchronize()
    assert rel(oj.cpu().numpy(), O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)) < 1e-10
    assert rel(ov.cpu().numpy(), O.vjp(case.om, case.kappa, case.mu, case.phi, t, case.w, case.fac)) < 1e-10


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_prior_solve(case, precision, variant):
    rng = np.random.default_rng(9)
    N = case.N
    kt = 0.3 * rng.standard_normal(N)
    mt = np.log(case.mu / case.mu.mean())
    rhs = rng.standard_normal(2 * N)
    T, ba, delta = 1e-2, 0.7, 1e-6
    Md = O.prior_matrix(case.om, kt, mt, T, ba, delta)
    ref = O.Factor(Md).solve(rhs)
    p = _params(precision, T=T, b_over_a=ba, delta=delta, pcg_rtol=1e-13, pcg_variant=variant)
    out = Q.qpat_prior_solve(case.lib, kt, mt, rhs, p)
    # the PCG stops on its recursive residual (1e-13); the true residual of
    # an operator with cond ~1e6-1e9 drifts above it by up to ~eps * cond, so
    # the bar is the normwise backward error
    Anorm = abs(Md).sum(axis=0).max()
    eta = np.linalg.norm(Md @ out - rhs, 1) / (Anorm * np.linalg.norm(out, 1) + np.linalg.norm(rhs, 1))
    assert eta < 1e-13
    tol = 10 * cond_mdelta(Md, delta) * 1e-13
    assert rel(out, ref) < max(tol, 1e-10)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_forward_k_padding_and_zero_flux(case, variant):
    # a zero illumination next to real ones: padded / inactive RHS stay exactly 0
    fl = np.vstack([case.flux, np.zeros_like(case.flux[:1])])
    if fl.shape[0] > 16:
        pytest.skip("K too large")
    phi, _ = Q.qpat_forward(case.lib, case.kappa, case.mu, fl, _params(0, pcg_variant=variant))
    assert np.all(phi[-1] == 0.0)
    assert rel(phi[:-1], case.phi) < 1e-10


def test_launch_counter_counts_the_solve(case):
    n0 = Q.qpat_launch_count()
    Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux)
    assert Q.qpat_launch_count() - n0 >= 2   # at least assembly + one PCG launch


@pytest.mark.parametrize("q", [1.0, 0.5, 2.0])
def test_prior_solve_tvq(case, q):
    """M_delta of the smoothed TV^q prior (Sec. 3's alternative r(t)) solved on
    the GPU against the oracle's sparse LU; q = 2 is the plain Laplacian."""
    rng = np.random.default_rng(11)
    N = case.N
    kt = 0.3 * rng.standard_normal(N)
    mt = np.log(case.mu / case.mu.mean())
    rhs = rng.standard_normal(2 * N)
    T, ba, delta = 1e-2, 0.7, 1e-6
    Md = O.prior_matrix(case.om, kt, mt, T, ba, delta, prior=1, q=q)
    ref = O.Factor(Md).solve(rhs)
    out = Q.qpat_prior_solve(case.lib, kt, mt, rhs,
                             _params(0, T=T, b_over_a=ba, delta=delta, pcg_rtol=1e-13, prior=1, prior_q=q))
    # TV^q weights reach T^(q-2) (up to 1e3 here), so cond(M_delta) ~ 1e9-1e10
    # and the true residual of a solve stopped on its recursive residual sits
    # ~eps cond above it; the bar is the normwise backward error instead
    Anorm = abs(Md).sum(axis=0).max()
    eta = np.linalg.norm(Md @ out - rhs, 1) / (Anorm * np.linalg.norm(out, 1) + np.linalg.norm(rhs, 1))
    assert eta < 1e-13
    tol = 10 * cond_mdelta(Md, delta) * 1e-13
    assert rel(out, ref) < max(tol, 1e-10)


def test_prior_parameter_checks(case):
    with pytest.raises(Q.QpatError):
        Q.qpat_prior_solve(case.lib, np.zeros(case.N), np.zeros(case.N), np.ones(2 * case.N),
                           _params(0, prior=1, prior_q=2.5))


def test_mixed_precision_falls_back_to_fp64_outside_fp32_range(case):
    """kappa and mu scaled by 1e40 (beyond the FP32 range; K = 1e40 (S + M)
    up to the Robin term, still well conditioned in FP64) make the FP32
    operator infinite: the inner PCG reports a breakdown and the solve is
    redone by the FP64 PCG, so the mixed path returns the FP64 answer."""
    kap, mu = case.kappa * 1e40, case.mu * 1e40
    ref, _ = Q.qpat_forward(case.lib, kap, mu, case.flux, _params(0))
    case.lib.reset_stats()
    out, _ = Q.qpat_forward(case.lib, kap, mu, case.flux, _params(1, fp32_operator=1))
    assert case.lib.stats()["fp64_fallbacks"] >= 1
    assert rel(out, ref) < 1e-10


@pytest.mark.parametrize("restart", [0, 1])
def test_mixed_precision_reliable_updates_and_restarts(case, restart):
    """Both forms of the FP32 + FP64 refinement solve (reliable updates that
    keep the FP32 search direction, or a fresh inner PCG per sweep) reach the
    FP64 answer: forward and the pair of J products."""
    p = _params(1, fp32_operator=1, mixed_restart=restart)
    phi, h = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, p)
    assert rel(phi, case.phi) < 1e-10
    rng = np.random.default_rng(12)
    s = rng.standard_normal(2 * case.N)
    out = Q.qpat_jvp(case.lib, case.kappa, case.mu, case.phi, s, case.w, p)
    assert rel(out, O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)) < 1e-10


@pytest.mark.parametrize("deg", [1, 2, 4, 8])
def test_prior_solve_poly_preconditioner(case, deg):
    """The patch-local Chebyshev preconditioner (block Jacobi over the CTA
    patches, a degree-deg polynomial per block) changes the iteration, not
    the solution: the M_delta solve meets the Jacobi bars, and on Kuhn cubes
    of a few hundred nodes or more it needs no more iterations than Jacobi."""
    rng = np.random.default_rng(13)
    N = case.N
    kt = 0.3 * rng.standard_normal(N)
    mt = np.log(case.mu / case.mu.mean())
    rhs = rng.standard_normal(2 * N)
    T, ba, delta = 1e-2, 0.7, 1e-6
    Md = O.prior_matrix(case.om, kt, mt, T, ba, delta)
    ref = O.Factor(Md).solve(rhs)
    iters = {}
    for d in (0, deg):
        case.lib.reset_stats()
        out = Q.qpat_prior_solve(case.lib, kt, mt, rhs,
                                 _params(0, T=T, b_over_a=ba, delta=delta, pcg_rtol=1e-13, prior_poly_degree=d))
        iters[d] = case.lib.stats()["pcg_iters"]
        Anorm = abs(Md).sum(axis=0).max()
        eta = np.linalg.norm(Md @ out - rhs, 1) / (Anorm * np.linalg.norm(out, 1) + np.linalg.norm(rhs, 1))
        assert eta < 1e-13
        tol = 10 * cond_mdelta(Md, delta) * 1e-13
        assert rel(out, ref) < max(tol, 1e-10)
    # on a handful of nodes CG needs only a few steps either way; on the
    # mapped cylinder mesh the stiffness has positive off-diagonal entries,
    # the Gershgorin interval is wider and a low degree may not pay
    if N > 400 and not hasattr(case.cfg, "illuminations"):
        assert iters[deg] <= iters[0]


@pytest.mark.parametrize("precision,fp32_op,variant", [(0, 0, 1), (0, 0, 2), (1, 1, 1), (1, 0, 1)])
@pytest.mark.parametrize("deg", [0, 1, 3])
def test_forward_and_pair_poly_preconditioner(case, precision, fp32_op, variant, deg):
    """K solves with Jacobi (deg 0) or the patch-local Chebyshev
    preconditioner (FP64 PCG and the FP32 inner PCG of the refinement;
    variants and operators without it fall back to Jacobi) reach the
    oracle's forward field and J products."""
    p = _params(precision, fp32_operator=fp32_op, pcg_variant=variant, poly_degree=deg)
    phi, h = Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, p)
    assert rel(phi, case.phi) < 1e-10
    assert rel(h, case.h) < 1e-10
    rng = np.random.default_rng(14)
    s = rng.standard_normal(2 * case.N)
    t = rng.standard_normal((case.K, case.N))
    oj = Q.qpat_jvp(case.lib, case.kappa, case.mu, case.phi, s, case.w, p)
    assert rel(oj, O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)) < 1e-10
    ov = Q.qpat_vjp(case.lib, case.kappa, case.mu, case.phi, t, case.w, p)
    assert rel(ov, O.vjp(case.om, case.kappa, case.mu, case.phi, t, case.w, case.fac)) < 1e-10


def test_poly_degree_checks(case):
    for kw in ({"poly_degree": 9}, {"prior_poly_degree": -1}):
        with pytest.raises(Q.QpatError):
            Q.qpat_forward(case.lib, case.kappa, case.mu, case.flux, _params(0, **kw))


def test_local_entry_counts(case):
    """Couplings inside a patch (what the patch-local preconditioner applies)
    are a subset of the stored entries; with the whole mesh in one patch
    they are all of them."""
    lib = case.lib
    assert 0 < lib.local_entries <= lib.entries
    assert 0 < lib.prior_local_entries <= lib.prior_entries
    if case.N <= 1024:
        one = Q.qpat_mesh(case.xyz, case.tets, patch_nodes=32 * (-(-case.N // 32)))
        try:
            assert one.local_entries == one.entries
            assert one.prior_local_entries == one.prior_entries
        finally:
            one.close()


def test_runs_are_bit_identical(case):
    """The element kernels sum colour by colour and the PCG reduces in a
    fixed order, so repeated calls (and a second mesh handle built from the
    same input) give bit-identical fields and the same iteration counts."""
    rng = np.random.default_rng(15)
    N = case.N
    s = rng.standard_normal(2 * N)
    t = rng.standard_normal((case.K, N))
    kt = 0.3 * rng.standard_normal(N)
    mt = np.log(case.mu / case.mu.mean())
    rhs = rng.standard_normal(2 * N)
    other = Q.qpat_mesh(case.xyz, case.tets, patch_nodes=64 if case.N > 64 else 32)
    try:
        runs = []
        for lib in (case.lib, case.lib, other):
            lib.reset_stats()
            out = []
            for prec in (0, 1):
                p = _params(prec, fp32_operator=1)
                out += list(Q.qpat_forward(lib, case.kappa, case.mu, case.flux, p))
                out.append(Q.qpat_jvp(lib, case.kappa, case.mu, case.phi, s, case.w, p))
                out.append(Q.qpat_vjp(lib, case.kappa, case.mu, case.phi, t, case.w, p))
            out.append(Q.qpat_prior_solve(lib, kt, mt, rhs, _params(0, T=1e-2, b_over_a=0.7)))
            runs.append((out, lib.stats()["pcg_iters"]))
        for out, iters in runs[1:]:
            assert iters == runs[0][1]
            for a, b in zip(out, runs[0][0]):
                np.testing.assert_array_equal(a, b)
    finally:
        other.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pair_host_entry(case, precision):
    """qpat_jvp_vjp_pair (host pointers, one 2K-RHS block solve) against the
    oracle's J s and J^T t."""
    if case.K > 8:
        pytest.skip("the pair takes K <= 8")
    rng = np.random.default_rng(16)
    s = rng.standard_normal(2 * case.N)
    t = rng.standard_normal((case.K, case.N))
    oj, ov = Q.qpat_jvp_vjp_pair(case.lib, case.kappa, case.mu, case.phi, s, t, case.w,
                                 _params(precision, fp32_operator=1))
    assert rel(oj, O.jvp(case.om, case.kappa, case.mu, case.phi, s, case.w, case.fac)) < 1e-10
    assert rel(ov, O.vjp(case.om, case.kappa, case.mu, case.phi, t, case.w, case.fac)) < 1e-10
