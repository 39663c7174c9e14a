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
