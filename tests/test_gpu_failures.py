"""Failure detection on the GPU, in forms that fault, trap or hang nothing:
every wait of the persistent solvers is bounded and returns a status the
host reads, iteration caps return a code, and inputs outside the model's
domain are refused before any kernel uses them.  After each failure the same
mesh handle (and CUDA context) must still solve correctly."""
import numpy as np
import pytest

import oracle as O
import qpat_synth as S
from tests.gpu_common import Case, rel

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(S.small_config(13, 12.0, 3, 3), patch_nodes=64)
    lib = Q.qpat_mesh(c.xyz, c.tets, patch_nodes=64)     # 35 patches: many CTAs meet at each barrier
    yield c, lib
    lib.close()


def _check_still_solves(c, lib, precision=0):
    phi, _ = Q.qpat_forward(lib, c.kappa, c.mu, c.flux, Q.qpat_default_params(precision=precision))
    assert rel(phi, c.phi) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_grid_barrier_wait_runs_out_and_returns_etimeout(case, precision):
    """A grid-barrier poll limit of 1 makes every CTA that waits for the last
    arrival give up at once: the solver sets QPAT_ETIMEOUT, every CTA
    leaves the persistent kernel, and the host reports the code."""
    c, lib = case
    prm = Q.qpat_default_params(precision=precision, barrier_spin_limit=1)
    with pytest.raises(Q.QpatError) as ei:
        Q.qpat_forward(lib, c.kappa, c.mu, c.flux, prm)
    assert ei.value.code == Q.QPAT_ETIMEOUT
    _check_still_solves(c, lib, precision)


def test_prior_solve_barrier_timeout(case):
    c, lib = case
    rng = np.random.default_rng(3)
    kt, mt = 0.1 * rng.standard_normal(c.N), 0.1 * rng.standard_normal(c.N)
    with pytest.raises(Q.QpatError) as ei:
        Q.qpat_prior_solve(lib, kt, mt, rng.standard_normal(2 * c.N), Q.qpat_default_params(barrier_spin_limit=1))
    assert ei.value.code == Q.QPAT_ETIMEOUT
    z = np.zeros(c.N)                  # M_delta = Laplacian + delta I: cond ~ 1e6, error ~ 1e-7
    b = rng.standard_normal(2 * c.N)
    x = Q.qpat_prior_solve(lib, z, z, b, Q.qpat_default_params(T=1e-2))
    assert rel(x, O.prior_solve(c.om, z, z, b, 1e-2)) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_iteration_cap_returns_enoconv(case, precision):
    c, lib = case
    with pytest.raises(Q.QpatError) as ei:
        Q.qpat_forward(lib, c.kappa, c.mu, c.flux, Q.qpat_default_params(precision=precision, max_pcg_iter=2))
    assert ei.value.code == Q.QPAT_ENOCONV
    _check_still_solves(c, lib, precision)


@pytest.mark.parametrize("what", ["kappa_nan", "kappa_zero", "mu_negative", "mu_inf"])
def test_coefficients_outside_the_model_are_refused(case, what):
    """Eq. (1) needs kappa, mu positive and bounded: a NaN, zero, negative or
    infinite nodal value is refused with QPAT_EINVAL (forward, J s, J^T t)."""
    c, lib = case
    kap, mu = c.kappa.copy(), c.mu.copy()
    i = c.N // 3
    if what == "kappa_nan":
        kap[i] = np.nan
    elif what == "kappa_zero":
        kap[i] = 0.0
    elif what == "mu_negative":
        mu[i] = -0.01
    else:
        mu[i] = np.inf
    prm = Q.qpat_default_params()
    for call in (lambda: Q.qpat_forward(lib, kap, mu, c.flux, prm),
                 lambda: Q.qpat_jvp(lib, kap, mu, c.phi, np.ones(2 * c.N), None, prm),
                 lambda: Q.qpat_vjp(lib, kap, mu, c.phi, np.ones((c.K, c.N)), None, prm)):
        with pytest.raises(Q.QpatError) as ei:
            call()
        assert ei.value.code == Q.QPAT_EINVAL
        assert "positive and finite" in str(ei.value)
    _check_still_solves(c, lib)


def test_non_finite_log_parameters_and_bad_data_are_refused(case):
    c, lib = case
    kt = np.zeros(c.N)
    kt[5] = np.nan
    with pytest.raises(Q.QpatError) as ei:
        Q.qpat_prior_solve(lib, kt, np.zeros(c.N), np.ones(2 * c.N), Q.qpat_default_params())
    assert ei.value.code == Q.QPAT_EINVAL
    chi = c.h.copy()
    sig = 0.01 * np.abs(c.h) + 1e-6
    bad_sig = sig.copy()
    bad_sig[0, 0] = 0.0
    bad_chi = chi.copy()
    bad_chi[0, 1] = np.nan
    prm = Q.qpat_default_params(max_lin=1, max_lsqr=1)
    for ch, sg in ((chi, bad_sig), (bad_chi, sig)):
        with pytest.raises(Q.QpatError) as ei:
            Q.qpat_reconstruct(lib, c.flux, ch, sg, prm, (0.3, 0.01))
        assert ei.value.code == Q.QPAT_EINVAL
    with pytest.raises(Q.QpatError) as ei:
        Q.qpat_reconstruct(lib, c.flux, chi, sig, Q.qpat_default_params(lsqr_reorth=2), (0.3, 0.01))
    assert ei.value.code == Q.QPAT_EINVAL
    _check_still_solves(c, lib)
