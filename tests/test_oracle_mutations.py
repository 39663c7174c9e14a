"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch each of them.  Each mutation is applied with monkeypatch and undone
after the test."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.qpat_oracle as Q
import tests.test_oracle_pins as P


def _fails(fn):
    try:
        fn()
    except AssertionError:
        return True
    return False


def test_flipped_g1_sign_is_caught(monkeypatch):
    orig = Q.G1_matrix
    monkeypatch.setattr(Q, "G1_matrix", lambda m, phi: -orig(m, phi))
    assert _fails(P.test_jvp_matches_central_differences)


def test_dropped_direct_mu_term_is_caught(monkeypatch):
    orig = Q.jvp

    def bad(mesh, kappa, mu, phi, s, w=None, factor=None):
        N = mesh.N
        out = orig(mesh, kappa, mu, phi, s, w, factor)
        phi2 = np.atleast_2d(phi)
        return out - phi2 * mu * s[N:] * (1 if w is None else w)
    import oracle
    monkeypatch.setattr(Q, "jvp", bad)
    monkeypatch.setattr(oracle, "jvp", bad)
    assert _fails(P.test_jvp_matches_central_differences)


def test_untransposed_g1_in_vjp_is_caught(monkeypatch):
    orig = Q.G1_matrix

    class Wrap:
        def __init__(self, M):
            self.M = M

        @property
        def T(self):
            return self.M            # "forgets" the transpose

        def __matmul__(self, x):
            return self.M @ x
    monkeypatch.setattr(Q, "G1_matrix", lambda m, phi: Wrap(orig(m, phi)))
    assert _fails(P.test_adjoint_identity)


def test_wrong_robin_factor_is_caught(monkeypatch):
    orig = Q.assemble_robin
    monkeypatch.setattr(Q, "assemble_robin", lambda m: 2.0 * orig(m))
    assert _fails(P.test_manufactured_solution_second_order)


def test_wrong_mass_weight_is_caught(monkeypatch):
    def bad_w3():
        W = np.zeros((4, 4, 4))
        for i in range(4):
            for j in range(4):
                for k in range(4):
                    W[i, j, k] = 1 / 20 if (i == j == k) else 1 / 120
        return W
    monkeypatch.setattr(Q, "_w3_tet", bad_w3)
    assert _fails(P.test_weighted_mass_matches_independent_quadrature)


def test_wrong_gradient_index_is_caught(monkeypatch):
    orig = Q.tet_geometry

    def bad(xyz, tets):
        vol, g = orig(xyz, tets)
        return vol, g[:, [0, 2, 1, 3], :]        # swapped local indices
    monkeypatch.setattr(Q, "tet_geometry", bad)
    assert _fails(P.test_kuhn_laplacian_is_seven_point_stencil)


def test_tvq_exponent_off_by_one_is_caught(monkeypatch):
    # r'(t)/t computed as (t^2 + T^2)^(q/2) instead of (t^2 + T^2)^(q/2 - 1)
    monkeypatch.setattr(Q, "tvq_rprime", lambda t, T, q: t * (t * t + T * T) ** (q / 2.0))
    assert _fails(P.test_tvq_weights_closed_forms_and_derivative)


def test_tvq_missing_chain_rule_factor_is_caught(monkeypatch):
    # d/dt (t^2 + T^2)^(q/2) / q taken without the inner derivative 2t / 2 = t
    monkeypatch.setattr(Q, "tvq_rprime", lambda t, T, q: (t * t + T * T) ** (q / 2.0 - 1.0))
    assert _fails(P.test_tvq_weights_closed_forms_and_derivative)


def test_dropped_j_beta_in_linearised_data_is_caught(monkeypatch):
    # y~ = w (chi - h) instead of w (chi - h + J beta): an increment solve
    monkeypatch.setattr(Q, "linearised_data", lambda chi, h, Jb, w: (w * (chi - h)).ravel())
    assert _fails(P.test_linearisation_step_is_krylov_minimiser_of_the_linearised_problem)
    assert _fails(P.test_step_zero_is_krylov_minimiser_in_kappa_alone)


def test_unwhitened_linearised_data_is_caught(monkeypatch):
    monkeypatch.setattr(Q, "linearised_data", lambda chi, h, Jb, w: (chi - h + Jb).ravel())
    assert _fails(P.test_linearisation_step_is_krylov_minimiser_of_the_linearised_problem)


def test_step_zero_over_both_blocks_is_caught(monkeypatch):
    # step 0 solving for (kappa_tilde, mu_tilde) and keeping the first block
    def bad(mesh, kap, mu, phi, h, fac, chi, w, kt, P_):
        N = mesh.N
        beta = np.concatenate([kt, np.log(mu / mu.mean())])
        r = Q.linearisation_step(mesh, kap, mu, phi, h, fac, chi, w, beta, P_)
        r.x = r.x[:N]
        return r
    import oracle
    monkeypatch.setattr(Q, "step_zero", bad)
    monkeypatch.setattr(oracle, "step_zero", bad)
    assert _fails(P.test_step_zero_is_krylov_minimiser_in_kappa_alone)


def _init_mu_variant(kind):
    def f(chi, phi0, mu0):
        r = phi0 / chi if kind == "inverted" else chi / phi0
        m = np.sum(r, axis=0) if kind == "sum" else np.mean(r, axis=0)
        m = np.where(m > 0, m, mu0)
        lo, hi = (10.0 * mu0, 0.1 * mu0) if kind == "swapped" else (0.1 * mu0, 10.0 * mu0)
        m = np.minimum(np.maximum(m, lo), hi)
        return np.log(m / mu0)
    return f


@pytest.mark.parametrize("kind", ["sum", "inverted", "swapped"])
def test_init_mu_mistakes_are_caught(monkeypatch, kind):
    import oracle
    monkeypatch.setattr(Q, "init_mu", _init_mu_variant(kind))
    monkeypatch.setattr(oracle, "init_mu", _init_mu_variant(kind))
    assert _fails(P.test_init_mu_hand_computed_case)
    if kind != "swapped":
        assert _fails(P.test_init_mu_recovers_mu_when_data_is_mu_times_phi0)
