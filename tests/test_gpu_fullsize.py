"""Parity at the benchmark's full sizes -- the 64^3 cube (Config 1, 4
illuminations) and the bench's 128^3 workload (Config 4, 8 illuminations,
the 16-RHS pair) -- in the launch configurations bench.py times.  The
oracle's sparse factorisation is too slow here, so each result is checked
through a property that holds at any size, using only the oracle's assembled
matrices:
  K x against the oracle CSR product,
  the forward residual |K phi - f| / |f| with the oracle K and f,
  the J s solve residual |K x - (G1 kappa s1 + G2 mu s2)| with the oracle G,
  the adjoint identity <J s, t> = <s, J^T t> of the paired launch,
  the M_delta solve's normwise backward error against the oracle's M_delta.
The linearisation point phi handed to J s and J^T t is a seeded smooth
positive field (the formulas hold for any phi), not a GPU result.
"""
import numpy as np
import pytest

import oracle as O
import qpat_synth as S
from tests.gpu_common import Case, rel

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu


def smooth_phi(xyz, K, L, seed):
    """K seeded smooth positive fields on the nodes (decaying away from a
    random face, with a gentle random modulation)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(K):
        ax, side = int(rng.integers(0, 3)), int(rng.integers(0, 2))
        d = xyz[:, ax] if side == 0 else L - xyz[:, ax]
        mod = 1.0 + 0.2 * np.sin(2 * np.pi * xyz @ rng.uniform(-1, 1, 3) / L)
        out.append(np.exp(-d / (0.2 * L)) * mod + 1e-3)
    return np.stack(out)


@pytest.fixture(scope="module", params=["c1_cube64", "c4_cube128"])
def big(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(S.config(request.param), solve=False)
    c.name = request.param
    c.lib = Q.qpat_mesh(c.xyz, c.tets)
    dev = torch.device("cuda")
    c.T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    c.phi = smooth_phi(c.xyz, c.K, c.cfg.L, 5)
    # the bench's headline: FP64 CG with the FP64 multigrid cycle ("mg1"); its
    # other arms: the K cycle in FP32 ("mg2"), the persistent FP64 PCG with
    # Jacobi K solves (0) and FP32 PCG inside FP64 refinement (1)
    c.prm = {0: Q.qpat_default_params(precision=0, poly_degree=0),
             1: Q.qpat_default_params(precision=1, fp32_operator=1),
             "mg1": Q.qpat_default_params(precision=0, multigrid=1),
             "mg2": Q.qpat_default_params(precision=0, multigrid=2)}
    yield c
    c.lib.close()


def test_apply_full_size(big):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((big.N, 4))
    y = torch.empty((big.N, 4), dtype=torch.float64, device="cuda")
    Q.qpat_apply_K_dev(big.lib, big.T(big.kappa), big.T(big.mu), big.T(x), y, 0)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), big.Kmat @ x) < 1e-13


@pytest.mark.parametrize("precision", [0, 1, "mg1", "mg2"])
def test_forward_residual_full_size(big, precision):
    dev = "cuda"
    phi = torch.empty((big.K, big.N), dtype=torch.float64, device=dev)
    h = torch.empty_like(phi)
    Q.qpat_forward_dev(big.lib, big.T(big.kappa), big.T(big.mu), big.T(big.flux), phi, h, big.prm[precision])
    torch.cuda.synchronize()
    ph = phi.cpu().numpy()
    for k in range(big.K):
        f = O.load_vector(big.om, big.flux[k])
        assert np.linalg.norm(big.Kmat @ ph[k] - f) / np.linalg.norm(f) < 1e-12
    np.testing.assert_allclose(h.cpu().numpy(), big.mu * ph, rtol=1e-15)


@pytest.mark.parametrize("precision", [0, "mg1"])
def test_jvp_solve_residual_full_size(big, precision):
    rng = np.random.default_rng(2)
    s = 0.1 * rng.standard_normal(2 * big.N)
    N = big.N
    out = torch.empty((big.K, N), dtype=torch.float64, device="cuda")
    Q.qpat_jvp_dev(big.lib, big.T(big.kappa), big.T(big.mu), big.T(big.phi), None, big.T(s), out, big.prm[precision])
    torch.cuda.synchronize()
    Js = out.cpu().numpy()
    for k in sorted({0, big.K - 1}):
        x = (Js[k] - big.phi[k] * big.mu * s[N:]) / big.mu
        rhs = (O.G1_matrix(big.om, big.phi[k]) @ (big.kappa * s[:N])
               + O.G2_matrix(big.om, big.phi[k]) @ (big.mu * s[N:]))
        assert np.linalg.norm(big.Kmat @ x - rhs) / np.linalg.norm(rhs) < 1e-11


@pytest.mark.parametrize("precision", [0, 1, "mg1", "mg2"])
def test_pair_adjoint_identity_full_size(big, precision):
    rng = np.random.default_rng(3)
    N = big.N
    s = rng.standard_normal(2 * N)
    t = rng.standard_normal((big.K, N))
    w = 1.0 / (0.01 * np.abs(big.mu * big.phi) + 1e-6)
    oj = torch.empty((big.K, N), dtype=torch.float64, device="cuda")
    ov = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    Q.qpat_jvp_vjp_pair_dev(big.lib, big.T(big.kappa), big.T(big.mu), big.T(big.phi), big.T(w), big.T(s), big.T(t),
                            oj, ov, big.prm[precision])
    torch.cuda.synchronize()
    a = float(np.sum(oj.cpu().numpy() * t))
    b = float(s @ ov.cpu().numpy())
    assert abs(a - b) <= 1e-10 * abs(a)


@pytest.mark.parametrize("deg", [0, 2])
def test_prior_solve_full_size(big, deg):
    """The M_delta solve as bench.py times it (two blocks, lagged weights of
    log(kappa / median), log(mu / median), library T, b/a, delta; degree 2 is
    the default, 0 Jacobi): normwise backward error against the oracle's
    M_delta, and the two preconditioners agree within the conditioning of the
    solve (they run the same system to the same residual)."""
    N = big.N
    kt = np.log(big.kappa / np.median(big.kappa))
    mt = np.log(big.mu / np.median(big.mu))
    rhs = np.random.default_rng(123).standard_normal(2 * N)
    prm = Q.qpat_default_params(prior_poly_degree=deg)
    out = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    big.lib.reset_stats()
    Q.qpat_prior_solve_dev(big.lib, big.T(kt), big.T(mt), big.T(rhs), out, prm)
    torch.cuda.synchronize()
    iters = big.lib.stats()["pcg_iters"]
    x = out.cpu().numpy()
    Md = O.prior_matrix(big.om, kt, mt, prm.T, prm.b_over_a, prm.delta)
    Anorm = abs(Md).sum(axis=0).max()
    eta = np.linalg.norm(Md @ x - rhs, 1) / (Anorm * np.linalg.norm(x, 1) + np.linalg.norm(rhs, 1))
    assert eta < 1e-13
    if not hasattr(big, "prior_x"):
        big.prior_x = {}
    big.prior_x[deg] = (x, iters)
    if len(big.prior_x) == 2:
        (x0, it0), (x2, it2) = big.prior_x[0], big.prior_x[2]
        assert rel(x2, x0) < 1e-8
        assert it2 < 0.7 * it0   # the patch-local polynomial roughly halves the count (64^3: 1400 -> 680)


def test_prior_solve_multigrid_full_size(big):
    """The M_delta solve of the bench's headline (multigrid cycle, FP64):
    normwise backward error against the oracle's M_delta, and the solution
    of the persistent degree-2 PCG within the conditioning of the solve."""
    N = big.N
    kt = np.log(big.kappa / np.median(big.kappa))
    mt = np.log(big.mu / np.median(big.mu))
    rhs = np.random.default_rng(123).standard_normal(2 * N)
    out = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    prm = big.prm["mg1"]
    Q.qpat_prior_solve_dev(big.lib, big.T(kt), big.T(mt), big.T(rhs), out, prm)
    torch.cuda.synchronize()
    x = out.cpu().numpy()
    Md = O.prior_matrix(big.om, kt, mt, prm.T, prm.b_over_a, prm.delta)
    Anorm = abs(Md).sum(axis=0).max()
    eta = np.linalg.norm(Md @ x - rhs, 1) / (Anorm * np.linalg.norm(x, 1) + np.linalg.norm(rhs, 1))
    assert eta < 1e-13
    ref = torch.empty_like(out)
    Q.qpat_prior_solve_dev(big.lib, big.T(kt), big.T(mt), big.T(rhs), ref, Q.qpat_default_params())
    torch.cuda.synchronize()
    assert rel(x, ref.cpu().numpy()) < 1e-8
