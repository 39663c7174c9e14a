"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

None of these compares the oracle with itself: each check uses a closed form,
an invariant, an independent quadrature, finite differences, a textbook
element matrix or dense linear algebra, chosen so that a dropped term, a wrong
sign or index or a transposed operand in the oracle fails at least one of
them (see test_oracle_mutations.py, which plants such mistakes).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import qpat_synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden_tet():
    blocks = {}
    cur = None
    with open(os.path.join(GOLDEN, "reference_tet_p1.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line[0].isalpha():
                cur = line
                blocks[cur] = []
            else:
                blocks[cur].append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def ref_tet_mesh():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    return O.Mesh(xyz, np.array([[0, 1, 2, 3]]))


def small_mesh(n=5, L=2.0):
    return O.Mesh(*S.kuhn_cube(n, L))


# ---------------------------------------------------------------- element level

def test_reference_tet_stiffness_and_mass_match_textbook():
    g = read_golden_tet()
    m = ref_tet_mesh()
    S1 = O.assemble_stiffness(m, np.ones(1)).toarray()
    M1 = O.assemble_weighted_mass(m, np.ones(4)).toarray()
    np.testing.assert_allclose(6 * S1, g["stiffness_times_6"], atol=1e-14)
    np.testing.assert_allclose(120 * M1, g["mass_times_120"], atol=1e-14)
    # the orientation of the vertices must not matter
    m2 = O.Mesh(m.xyz, np.array([[0, 2, 1, 3]]))
    np.testing.assert_allclose(O.assemble_stiffness(m2, np.ones(1)).toarray(), S1, atol=1e-15)


def _duffy_rule(order=5):
    """Quadrature on the reference tet by the collapsed-coordinate (Duffy) map of
    a Gauss-Legendre tensor rule: independent of the factorial simplex formula."""
    x, w = np.polynomial.legendre.leggauss(order)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    pts, wts = [], []
    for a, wa in zip(x, w):
        for b, wb in zip(x, w):
            for c, wc in zip(x, w):
                # (a, b, c) in the unit cube -> tet
                X = a
                Y = b * (1 - a)
                Z = c * (1 - a) * (1 - b)
                jac = (1 - a) ** 2 * (1 - b)
                pts.append((X, Y, Z))
                wts.append(wa * wb * wc * jac)
    return np.array(pts), np.array(wts)


def test_weighted_mass_matches_independent_quadrature():
    rng = np.random.default_rng(3)
    xyz = rng.uniform(-1, 1, size=(4, 3))
    m = O.Mesh(xyz, np.array([[0, 1, 2, 3]]))
    c = rng.uniform(0.5, 2.0, size=4)
    Mc = O.assemble_weighted_mass(m, c).toarray()
    pts, wts = _duffy_rule()
    lam = np.column_stack([1 - pts.sum(1), pts])          # reference barycentrics
    scale = 6 * m.vol[0]                                  # |det| of the affine map
    ch = lam @ c
    Q = np.einsum("q,q,qi,qj->ij", wts * scale, ch, lam, lam)
    np.testing.assert_allclose(Mc, Q, rtol=1e-13, atol=1e-15)


def test_g1_matches_independent_quadrature():
    rng = np.random.default_rng(4)
    xyz = rng.uniform(-1, 1, size=(4, 3))
    m = O.Mesh(xyz, np.array([[0, 1, 2, 3]]))
    phi = rng.standard_normal(4)
    G1 = O.G1_matrix(m, phi).toarray()
    pts, wts = _duffy_rule()
    lam = np.column_stack([1 - pts.sum(1), pts])
    gphi = phi @ m.grads[0]
    gi = m.grads[0] @ gphi                                  # grad phi . grad lambda_i
    Q = -np.einsum("q,i,qj->ij", wts * 6 * m.vol[0], gi, lam)
    np.testing.assert_allclose(G1, Q, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- mesh level

def test_kuhn_mesh_counts_and_measures():
    for n, L in [(2, 1.0), (5, 2.0), (11, 20.0)]:
        m = small_mesh(n, L)
        assert m.N == n ** 3 and m.E == 6 * (n - 1) ** 3
        assert m.F == 12 * (n - 1) ** 2
        assert abs(m.vol.sum() - L ** 3) < 1e-12 * L ** 3
        assert abs(m.farea.sum() - 6 * L ** 2) < 1e-12 * L ** 2
        assert np.allclose(m.vol, (L / (n - 1)) ** 3 / 6)


def test_stiffness_row_sums_vanish_and_mass_totals():
    m = small_mesh(6, 3.0)
    rng = np.random.default_rng(0)
    Sc = O.assemble_stiffness(m, rng.uniform(0.1, 1, m.E))
    assert np.abs(Sc @ np.ones(m.N)).max() < 1e-13
    one = np.ones(m.N)
    assert abs(one @ (O.assemble_weighted_mass(m, one) @ one) - 27.0) < 1e-12
    assert abs(one @ (O.assemble_robin(m) @ one) - 0.5 * 54.0) < 1e-12


def test_kuhn_laplacian_is_seven_point_stencil():
    """On the Kuhn (Freudenthal) triangulation the P1 Laplacian stiffness equals
    h times the 7-point finite-difference Laplacian: an independent textbook
    fact that pins grad(lambda) and the assembly indices."""
    n, L = 6, 5.0
    h = L / (n - 1)
    m = small_mesh(n, L)
    A = O.assemble_stiffness(m, np.ones(m.E)).tocsr()
    i, j, k = 2, 3, 2
    row = i + n * (j + n * k)
    r = A.getrow(row).toarray().ravel()
    expect = np.zeros(m.N)
    expect[row] = 6 * h
    for d in (1, n, n * n):
        expect[row + d] = -h
        expect[row - d] = -h
    np.testing.assert_allclose(r, expect, atol=1e-13)


def test_system_matrix_spd():
    m = small_mesh(4, 2.0)
    rng = np.random.default_rng(1)
    K = O.system_matrix(m, rng.uniform(0.2, 0.4, m.N), rng.uniform(0.01, 0.03, m.N)).toarray()
    np.testing.assert_allclose(K, K.T, atol=1e-15)
    assert np.linalg.eigvalsh(K).min() > 0


def test_load_vector_total_and_patch_area():
    cfg = S.config("c0_cube11")
    m = O.Mesh(*cfg.mesh())
    p = cfg.patches[0]
    fl = O.flux_patch(m, p.center, p.normal, p.half_w, 1.0)
    assert abs((fl * m.farea).sum() - 100.0) < 1e-9      # 10 x 10 mm patch
    f = O.load_vector(m, fl)
    assert abs(f.sum() - 2 * 100.0) < 1e-9               # 2 * integral of Phi


# ---------------------------------------------------------------- forward model

def _manufactured_error(n, L=2.0, kap=0.3, mu=0.05):
    m = small_mesh(n, L)
    a = math.sqrt(mu / kap) * np.array([1.0, 2.0, 2.0]) / 3.0
    exact = np.exp(m.xyz @ a)
    # Robin data 1/4 phi + 1/2 kappa nu.grad(phi) at every boundary node,
    # one value per (face, vertex) because nu changes between faces
    W = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 12.0
    f = np.zeros(m.N)
    p = m.xyz[m.faces]
    nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    cen = p.mean(axis=1)
    out = np.sign(((cen - L / 2) * nrm).sum(1))
    nrm *= out[:, None]
    for fi in range(m.F):
        vals = exact[m.faces[fi]] * (0.25 + 0.5 * kap * (nrm[fi] @ a))
        f[m.faces[fi]] += 2.0 * m.farea[fi] * (W @ vals)
    K = O.system_matrix(m, np.full(m.N, kap), np.full(m.N, mu))
    ph = O.Factor(K).solve(f)
    M = O.assemble_weighted_mass(m, np.ones(m.N))
    e = ph - exact
    return math.sqrt(e @ (M @ e))


def test_manufactured_solution_second_order():
    errs = [_manufactured_error(n) for n in (5, 9, 17, 33)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    # halving h divides the L2 error by 4 (observed: 4.16, 4.07, 4.02)
    assert all(3.8 < r < 4.3 for r in ratios), ratios
    assert abs(ratios[-1] - 4.0) < 0.1, ratios


def _manufactured_error_cylinder(n, R=1.0, H=2.0, kap=0.3, mu=0.05):
    """As _manufactured_error on the mapped cylinder mesh (Test 1 geometry):
    the Robin data is exact on the polygonal domain the mesh covers, so the
    P1 error must still fall as h^2."""
    m = O.Mesh(*S.cylinder_mesh(n, n, R, H))
    a = math.sqrt(mu / kap) * np.array([1.0, 2.0, 2.0]) / 3.0
    exact = np.exp(m.xyz @ a)
    W = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 12.0
    f = np.zeros(m.N)
    p = m.xyz[m.faces]
    nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    cen = p.mean(axis=1)
    out = np.sign(((cen - np.array([0.0, 0.0, H / 2])) * nrm).sum(1))   # convex body
    nrm *= out[:, None]
    for fi in range(m.F):
        vals = exact[m.faces[fi]] * (0.25 + 0.5 * kap * (nrm[fi] @ a))
        f[m.faces[fi]] += 2.0 * m.farea[fi] * (W @ vals)
    K = O.system_matrix(m, np.full(m.N, kap), np.full(m.N, mu))
    e = O.Factor(K).solve(f) - exact
    return math.sqrt(e @ (O.assemble_weighted_mass(m, np.ones(m.N)) @ e))


def test_manufactured_solution_second_order_on_cylinder():
    errs = [_manufactured_error_cylinder(n) for n in (5, 9, 17, 33)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.3 < r < 4.7 for r in ratios), ratios
    assert abs(ratios[-1] - 4.0) < 0.3, ratios


def test_cylinder_mesh_measures_and_side_flux_converge():
    """Volume -> pi R^2 H (error O(h^2)), side area -> 2 pi R H (inscribed
    polygons); the side illumination's total flux sum Phi_F |F| -> R H / 2, the
    integral of cos(4 (theta - theta0)) over [theta0 - pi/8, theta0 + pi/8]
    times R H; faces outside the lit band or on the caps carry no flux."""
    R, H = 10.0, 8.0
    prev = None
    for n in (9, 17, 33):
        m = O.Mesh(*S.cylinder_mesh(n, 5, R, H))
        vol_err = abs(m.vol.sum() - np.pi * R * R * H) / (np.pi * R * R * H)
        radial = np.linalg.norm(m.xyz[m.faces][..., :2], axis=2)
        side = np.all(np.abs(radial - R) <= 1e-9 * R, axis=1)
        area_err = abs(m.farea[side].sum() - 2 * np.pi * R * H) / (2 * np.pi * R * H)
        errs = []
        for k in range(4):
            fl = O.flux_side(m, (0, 0, 0), (0, 0, 1), (1, 0, 0), R, k * np.pi / 2)
            assert np.all(fl[~side] == 0.0) and fl.min() >= 0.0 and fl.max() <= 1.0
            errs.append(abs((fl * m.farea).sum() - R * H / 2) / (R * H / 2))
        cur = (vol_err, area_err, max(errs))
        if prev is not None:
            # volume O(h^2); side nodes are not equally spaced in angle
            # (square rings), so the side area and flux fall less regularly
            assert cur[0] < prev[0] / 3.5 and cur[1] < prev[1] / 1.8 and cur[2] < prev[2] / 1.9, (prev, cur)
        prev = cur
    assert prev[0] < 2e-3 and prev[1] < 2e-3 and prev[2] < 1e-2
    # the four illuminations are rotations of each other: equal totals
    tot = [(O.flux_side(m, (0, 0, 0), (0, 0, 1), (1, 0, 0), R, k * np.pi / 2) * m.farea).sum() for k in range(4)]
    np.testing.assert_allclose(tot, tot[0], rtol=1e-12)


def test_load_vector_nodal_matches_face_constant_for_constant_flux():
    m = small_mesh(5, 2.0)
    nod = np.ones(m.N)
    np.testing.assert_allclose(O.load_vector_nodal(m, nod), O.load_vector(m, np.ones(m.F)), atol=1e-14)


# ---------------------------------------------------------------- Jacobian

def _state(cfg_n=6, K=2, seed=5):
    cfg = S.small_config(cfg_n, 10.0, K, seed)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    kap, mu = cfg.coefficients(xyz)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    fac = O.Factor(O.system_matrix(m, kap, mu))
    phi, h = O.forward(m, kap, mu, fl, fac)
    return m, kap, mu, fl, fac, phi, h


def test_jvp_matches_central_differences():
    m, kap, mu, fl, fac, phi, h = _state()
    rng = np.random.default_rng(11)
    s = rng.standard_normal(2 * m.N)
    Js = O.jvp(m, kap, mu, phi, s, None, fac)
    eps = 1e-4
    N = m.N
    def H(sig):
        return O.measure(m, kap * np.exp(sig * eps * s[:N]), mu * np.exp(sig * eps * s[N:]), fl)
    fd = (H(1) - H(-1)) / (2 * eps)
    assert np.linalg.norm(fd - Js) / np.linalg.norm(Js) < 1e-7


def test_adjoint_identity():
    m, kap, mu, fl, fac, phi, h = _state(K=3)
    rng = np.random.default_rng(12)
    v = rng.standard_normal(2 * m.N)
    t = rng.standard_normal((3, m.N))
    w = rng.uniform(0.5, 2.0, (3, m.N))
    lhs = np.sum(O.jvp(m, kap, mu, phi, v, w, fac) * t)
    rhs = v @ O.vjp(m, kap, mu, phi, t, w, fac)
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1e-300)


def test_dense_jacobian_tiny_mesh():
    """Column-by-column J of a tiny mesh against the dense formula
    diag(mu) K^-1 [G1 diag(kappa), G2 diag(mu)] + [0, diag(phi mu)] built
    with numpy dense inverses."""
    cfg = S.small_config(3, 2.0, 1, 7)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    kap, mu = cfg.coefficients(xyz)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    phi, _ = O.forward(m, kap, mu, fl)
    N = m.N
    Kd = O.system_matrix(m, kap, mu).toarray()
    G1 = O.G1_matrix(m, phi[0]).toarray()
    G2 = O.G2_matrix(m, phi[0]).toarray()
    Kinv = np.linalg.inv(Kd)
    Jd = np.hstack([np.diag(mu) @ Kinv @ G1 @ np.diag(kap),
                    np.diag(mu) @ Kinv @ G2 @ np.diag(mu) + np.diag(phi[0] * mu)])
    cols = np.stack([O.jvp(m, kap, mu, phi, e)[0] for e in np.eye(2 * N)], axis=1)
    np.testing.assert_allclose(cols, Jd, rtol=1e-10, atol=1e-13 * np.abs(Jd).max())
    # and its transpose through vjp
    rows = np.stack([O.vjp(m, kap, mu, phi, e[None, :]) for e in np.eye(N)], axis=0)
    np.testing.assert_allclose(rows, Jd, rtol=1e-10, atol=1e-13 * np.abs(Jd).max())
    # G2 is symmetric, as the transpose formula uses
    np.testing.assert_allclose(G2, G2.T, atol=1e-15)


# ---------------------------------------------------------------- prior

def test_lagged_weight_is_rprime_over_t():
    """c_u |grad u| = r'(|grad u|) with r' from central differences of the
    Perona-Malik r of Eq. (10), for a linear u with known gradient."""
    m = small_mesh(4, 3.0)
    T = 5e-3
    for gnorm in (1e-4, 3e-3, 5e-3, 0.2):
        g = gnorm * np.array([2.0, -1.0, 2.0]) / 3.0
        u = m.xyz @ g
        c = O.lagged_weights(m, u, T)
        r = lambda t: 0.5 * T ** 2 * np.log1p((t / T) ** 2)
        e = 1e-6 * gnorm
        rp = (r(gnorm + e) - r(gnorm - e)) / (2 * e)
        np.testing.assert_allclose(c * gnorm, rp, rtol=1e-8)
    assert np.all(O.lagged_weights(m, np.zeros(m.N), T) == 1.0)


def test_prior_operator_psd_kernel_and_delta():
    m = small_mesh(4, 2.0)
    rng = np.random.default_rng(2)
    u = 0.3 * rng.standard_normal(m.N)
    Mu = O.assemble_stiffness(m, O.lagged_weights(m, u, 5e-3)).toarray()
    assert np.abs(Mu @ np.ones(m.N)).max() < 1e-13
    ev = np.linalg.eigvalsh(Mu)
    assert ev.min() >= -1e-14 * ev.max()
    assert np.sum(ev < 1e-12 * ev.max()) == 1            # one-dimensional kernel
    delta = 1e-6
    Md = O.prior_matrix(m, u, -u, 5e-3, 0.7, delta).toarray()
    evd = np.linalg.eigvalsh(Md)
    assert evd.min() >= delta * (1 - 1e-9)
    # u = 0: c = 1, M(0) is the plain P1 Laplacian stiffness
    np.testing.assert_allclose(
        O.prior_matrix(m, np.zeros(m.N), np.zeros(m.N), 1e-3, 1.0, 0.0).toarray()[:m.N, :m.N],
        O.assemble_stiffness(m, np.ones(m.E)).toarray(), atol=1e-14)


def test_tvq_weights_closed_forms_and_derivative():
    """Smoothed TV^q (the alternative priors named in Sec. 3): q = 1 gives the
    lagged-diffusivity weight of smoothed total variation, 1/sqrt(t^2 + T^2)
    (the fixed-point weight of Vogel and Oman); q = 2 gives weight 1 for any u
    (the plain P1 Laplacian stiffness, a textbook case); for every q the weight
    times t is the derivative of r (central differences), and the t = 0
    value is T^(q - 2)."""
    m = small_mesh(4, 3.0)
    T = 5e-3
    rng = np.random.default_rng(4)
    u = 0.2 * rng.standard_normal(m.N)
    g = np.einsum("ek,ekd->ed", u[m.tets], m.grads)
    t = np.linalg.norm(g, axis=1)
    np.testing.assert_allclose(O.lagged_weights(m, u, T, prior=1, q=1.0), 1.0 / np.sqrt(t ** 2 + T ** 2),
                               rtol=1e-13)
    np.testing.assert_allclose(O.lagged_weights(m, u, T, prior=1, q=2.0), 1.0, rtol=1e-15)
    np.testing.assert_allclose(
        O.prior_matrix(m, u, -u, T, 1.0, 0.0, prior=1, q=2.0).toarray()[:m.N, :m.N],
        O.assemble_stiffness(m, np.ones(m.E)).toarray(), atol=1e-14)
    for q in (0.5, 1.0, 1.5):
        assert np.all(O.lagged_weights(m, np.zeros(m.N), T, prior=1, q=q) == T ** (q - 2.0))
        for gnorm in (1e-4, 5e-3, 0.2):
            gv = gnorm * np.array([2.0, -1.0, 2.0]) / 3.0
            c = O.lagged_weights(m, m.xyz @ gv, T, prior=1, q=q)
            e = 1e-4 * gnorm          # truncation O(e^2) vs roundoff eps r / e
            rp = (O.tvq_r(gnorm + e, T, q) - O.tvq_r(gnorm - e, T, q)) / (2 * e)
            np.testing.assert_allclose(c * gnorm, rp, rtol=1e-6)
    # the lagged operator keeps M 1 = 0, PSD with a 1-D kernel, and M_delta >= delta
    Mu = O.assemble_stiffness(m, O.lagged_weights(m, u, T, prior=1, q=0.7)).toarray()
    assert np.abs(Mu @ np.ones(m.N)).max() < 1e-9 * np.abs(Mu).max()
    ev = np.linalg.eigvalsh(Mu)
    assert ev.min() >= -1e-13 * ev.max() and np.sum(ev < 1e-12 * ev.max()) == 1
    evd = np.linalg.eigvalsh(O.prior_matrix(m, u, -u, T, 0.7, 1e-6, prior=1, q=0.7).toarray())
    assert evd.min() >= 1e-6 * (1 - 1e-6)


# ---------------------------------------------------------------- LSQR

def _dense_problem(mrows=40, ncols=12, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((mrows, ncols))
    B = rng.standard_normal((ncols, ncols))
    P = B @ B.T + 0.5 * np.eye(ncols)
    b = rng.standard_normal(mrows)
    return A, P, b


def test_lsqr_iterate_is_krylov_minimiser():
    A, P, b = _dense_problem()
    Pinv = np.linalg.inv(P)
    for m in (1, 3, 6):
        res = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, m,
                           fixed_counts=True)
        # x in P^-1 K_m(A^T A P^-1, A^T b): basis by repeated products
        basis = []
        r = A.T @ b
        for _ in range(m):
            basis.append(Pinv @ r)
            r = A.T @ (A @ (Pinv @ r))
        V = np.linalg.qr(np.stack(basis, 1))[0]
        y = np.linalg.lstsq(A @ V, b, rcond=None)[0]
        xbest = V @ y
        np.testing.assert_allclose(res.x, xbest, rtol=1e-9, atol=1e-11)
        assert abs(res.phibar[-1] - np.linalg.norm(A @ res.x - b)) < 1e-9 * np.linalg.norm(b)


def test_lsqr_full_rank_gives_least_squares_and_scaling_invariance():
    A, P, b = _dense_problem(seed=1)
    Pinv = np.linalg.inv(P)
    n = A.shape[1]
    # n rounds are exact in exact arithmetic; finite precision needs a few more
    res = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, 4 * n,
                       fixed_counts=True)
    xls = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(res.x, xls, rtol=1e-8)
    res2 = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p / 7.0, b, 4,
                        fixed_counts=True)
    res1 = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, 4,
                        fixed_counts=True)
    np.testing.assert_allclose(res2.x, res1.x, rtol=1e-11)


def test_lsqr_stopping_rule():
    A, P, b = _dense_problem(200, 60, seed=2)
    Pinv = np.linalg.inv(P)
    res = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, 60,
                       m0=5, tau=0.05)
    assert res.stop_rule
    m = res.iters
    assert 1 - res.phibar[m] / res.phibar[m - 5] <= 0.05
    for k in range(6, m):
        assert 1 - res.phibar[k] / res.phibar[k - 5] > 0.05


# ---------------------------------------------------------------- Algorithm 1

def test_fit_background_recovers_constant_coefficients():
    cfg = S.small_config(5, 10.0, 2, 3)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    kap0, mu0 = 0.27, 0.012
    h = O.measure(m, np.full(m.N, kap0), np.full(m.N, mu0), fl)
    w = 1.0 / np.maximum(0.01 * np.abs(h), 1e-12)
    k, mm = O.fit_background(m, fl, h, w, grid=7, gn_steps=15)
    assert abs(k / kap0 - 1) < 1e-6 and abs(mm / mu0 - 1) < 1e-6


def test_reconstruct_decreases_residual_and_error():
    cfg = S.small_config(7, 12.0, 2, 9)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    kap_t, mu_t = cfg.coefficients(xyz)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    h = O.measure(m, kap_t, mu_t, fl)
    sig = 0.01 * np.abs(h) + 1e-12
    chi = h + sig * S.noise_draws(1, h.shape)
    par = O.QpatParams(T=1e-3, max_lin=3, max_lsqr=20)
    k0m0 = (float(np.median(kap_t)), float(np.median(mu_t)))
    kap, mu, rep = O.reconstruct(m, fl, chi, sig, par, k0m0)
    assert rep.linearisations >= 2
    assert all(rep.residuals[i + 1] < rep.residuals[i] for i in range(len(rep.residuals) - 1))
    e_mu = np.linalg.norm(mu - mu_t) / np.linalg.norm(mu_t)
    e_mu0 = np.linalg.norm(k0m0[1] - mu_t) / np.linalg.norm(mu_t)
    assert e_mu < e_mu0


def test_reconstruct_resume_equals_one_run():
    """Checkpoint / resume of Algorithm 1: step 1 restarts from beta^(l)
    alone, so stopping after l linearisations and resuming from (kappa_0,
    mu_0, beta^(l), l) reproduces the uninterrupted run exactly; resuming
    without the background constants is refused."""
    cfg = S.small_config(7, 12.0, 2, 9)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    kap_t, mu_t = cfg.coefficients(xyz)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    h = O.measure(m, kap_t, mu_t, fl)
    sig = 0.01 * np.abs(h) + 1e-12
    chi = h + sig * S.noise_draws(1, h.shape)
    k0m0 = (float(np.median(kap_t)), float(np.median(mu_t)))
    full = O.reconstruct(m, fl, chi, sig, O.QpatParams(T=1e-2, max_lin=4, max_lsqr=8, fixed_counts=True), k0m0)
    part = O.reconstruct(m, fl, chi, sig, O.QpatParams(T=1e-2, max_lin=2, max_lsqr=8, fixed_counts=True), k0m0)
    assert part[2].linearisations == 2 and part[2].accepted_last
    rest = O.reconstruct(m, fl, chi, sig, O.QpatParams(T=1e-2, max_lin=4, max_lsqr=8, fixed_counts=True), k0m0,
                         beta_in=part[2].beta, lin_done=part[2].linearisations)
    assert rest[2].linearisations == full[2].linearisations
    np.testing.assert_array_equal(rest[0], full[0])
    np.testing.assert_array_equal(rest[1], full[1])
    np.testing.assert_array_equal(rest[2].beta, full[2].beta)
    assert rest[2].residuals == full[2].residuals[1:]   # continues the history after beta^(2)
    with pytest.raises(ValueError):
        O.reconstruct(m, fl, chi, sig, O.QpatParams(), None, beta_in=part[2].beta, lin_done=2)


def test_reconstruct_step_halving_option():
    """The step-halving option (not in the paper; off by default) only
    changes what happens to a step that Algorithm 1 would reject: the accepted
    prefix of a default run is reproduced exactly, every accepted step lowers
    the residual, and on the Test 2 stand-in (two opposite illuminations),
    where the default run's kappa-only step 0 diverges, it stays bounded and
    fits the data to the noise level."""
    cfg = S.small_config(7, 12.0, 2, 9)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    kap_t, mu_t = cfg.coefficients(xyz)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    h = O.measure(m, kap_t, mu_t, fl)
    sig = 0.01 * np.abs(h) + 1e-12
    chi = h + sig * S.noise_draws(1, h.shape)
    k0m0 = (float(np.median(kap_t)), float(np.median(mu_t)))
    # (the plain LSQR recurrence, whose default run stops at a rejected step here)
    d = O.reconstruct(m, fl, chi, sig, O.QpatParams(T=1e-3, max_lin=5, max_lsqr=50, lsqr_reorth=False), k0m0)[2]
    hv = O.reconstruct(m, fl, chi, sig, O.QpatParams(T=1e-3, max_lin=5, max_lsqr=50, step_halvings=4,
                                                     lsqr_reorth=False), k0m0)[2]
    assert not d.accepted_last                                  # the default run stops at a rejected step
    assert hv.residuals[:len(d.residuals)] == d.residuals        # same accepted prefix, bit for bit
    assert hv.linearisations > d.linearisations
    assert all(b < a for a, b in zip(hv.residuals, hv.residuals[1:]))

    co = S.Test2Config(9, ("btm", "top"))
    x2, t2 = co.mesh()
    m2 = O.Mesh(x2, t2)
    k2, mu2 = co.coefficients(x2)
    fl2 = np.stack([O.flux_patch(m2, p.center, p.normal, p.half_w, p.amp) for p in co.patches])
    h2 = O.measure(m2, k2, mu2, fl2)
    s2 = 0.01 * np.abs(h2) + 1e-3 * np.abs(h2).max()
    c2 = h2 + s2 * S.noise_draws(3, h2.shape)
    kd, _, rd = O.reconstruct(m2, fl2, c2, s2, O.QpatParams(lsqr_reorth=False))
    kh, _, rh = O.reconstruct(m2, fl2, c2, s2, O.QpatParams(step_halvings=6, lsqr_reorth=False))
    assert np.abs(np.log(kd / rd.kappa0)).max() > 20          # default: step 0 diverges
    assert np.abs(np.log(kh / rh.kappa0)).max() < 2
    assert rh.residuals[-1] < 1.5 * np.sqrt(h2.size)           # whitened noise level sqrt(K N)


# ---------------------------------------------------------------- Algorithm 1 pieces

def test_init_mu_hand_computed_case():
    """mu_init of Algorithm 1 with the multi-illumination rule of Sec. 4 on a
    hand-computed K = 2 case (mu_0 = 0.01): node 0 averages 0.02/1 and
    0.06/2 to 0.025; node 1 averages to 0.2 and is clipped to 10 mu_0; node 2
    averages to -0.02 (not positive: mu_0); node 3 averages to 1e-5 and is
    clipped to mu_0 / 10.  Expected mu_tilde = log(mu_init / mu_0), written
    out by hand."""
    chi = np.array([[0.02, 0.3, -0.05, 1e-5],
                    [0.06, 0.1, 0.01, 1e-5]])
    phi0 = np.array([[1.0, 1.0, 1.0, 1.0],
                     [2.0, 1.0, 1.0, 1.0]])
    got = O.init_mu(chi, phi0, 0.01)
    expect = np.array([math.log(2.5), math.log(10.0), 0.0, math.log(0.1)])
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-14)


def test_init_mu_recovers_mu_when_data_is_mu_times_phi0():
    """The motivation of mu_init (Eqs. (2), (4)): if every illumination's data
    is chi^(k) = mu o phi0^(k) with the same mu, the average of chi/phi0 is
    mu and mu_tilde_init = log(mu / mu_0) exactly, for any positive phi0^(k)."""
    rng = np.random.default_rng(4)
    mu0 = 0.012
    mu = mu0 * np.exp(rng.uniform(-1.5, 1.5, 50))
    phi0 = rng.uniform(0.1, 3.0, (3, 50))
    got = O.init_mu(mu[None, :] * phi0, phi0, mu0)
    np.testing.assert_allclose(got, np.log(mu / mu0), rtol=0, atol=1e-13)


def _fd_jacobian(m, fl, k0, m0, beta, eps=1e-5):
    """Column-by-column Jacobian of beta -> h(kappa_0 e^kt, mu_0 e^mt) (K N x 2N)
    by central differences of the forward model alone (no jvp code)."""
    N = m.N
    cols = []
    for j in range(2 * N):
        hs = []
        for sgn in (1.0, -1.0):
            b = beta.copy()
            b[j] += sgn * eps
            hs.append(O.measure(m, k0 * np.exp(b[:N]), m0 * np.exp(b[N:]), fl).ravel())
        cols.append((hs[0] - hs[1]) / (2 * eps))
    return np.stack(cols, axis=1)


def _tiny_linearisation():
    cfg = S.small_config(3, 6.0, 3, 13)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    fl = np.stack([O.flux_patch(m, p.center, p.normal, p.half_w) for p in cfg.patches])
    N = m.N
    k0, m0 = 0.3, 0.012
    rng = np.random.default_rng(21)
    beta = 0.3 * rng.standard_normal(2 * N)                       # beta^(l), away from 0
    beta_true = beta + 0.2 * rng.standard_normal(2 * N)
    h_true = O.measure(m, k0 * np.exp(beta_true[:N]), m0 * np.exp(beta_true[N:]), fl)
    sig = 0.01 * np.abs(h_true) + 1e-3 * np.abs(h_true).max()
    chi = h_true + sig * S.noise_draws(5, h_true.shape)
    return m, fl, k0, m0, beta, chi, 1.0 / sig


def _krylov_minimiser(A, Pinv, b, m):
    """argmin |A x - b| over x in P^-1 K_m(A^T A P^-1, A^T b), from an
    orthonormal basis (each new vector orthogonalised twice) and a dense
    least-squares solve."""
    Vb = []
    r = A.T @ b
    for _ in range(m):
        v = Pinv @ r
        for _ in range(2):
            for q in Vb:
                v = v - (q @ v) * q
        Vb.append(v / np.linalg.norm(v))
        r = A.T @ (A @ v)
    V = np.stack(Vb, 1)
    return V @ np.linalg.lstsq(A @ V, b, rcond=None)[0]


def test_linearisation_step_is_krylov_minimiser_of_the_linearised_problem():
    """Steps 1-3 of Algorithm 1 on a 27-node mesh with K = 3: after m LSQR
    rounds the candidate beta^(l+1) minimises |A beta - y~| over
    M_delta^-1 K_m(A^T A M_delta^-1, A^T y~), with A = Gamma^-1/2 J,
    y~ = Gamma^-1/2 (chi - h(beta^(l)) + J beta^(l)) and M_delta built from
    beta^(l) (Eqs. (11), (16), (19), (21)), all formed here with dense numpy
    algebra and J from central differences of the forward model alone.
    Dropping the + J beta^(l) term of y~ (an increment solve instead of
    Gauss-Newton for beta), the whitening, or building M_delta elsewhere
    fails it."""
    m, fl, k0, m0, beta, chi, w = _tiny_linearisation()
    N = m.N
    kap, mu = k0 * np.exp(beta[:N]), m0 * np.exp(beta[N:])
    fac = O.Factor(O.system_matrix(m, kap, mu))
    phi, h = O.forward(m, kap, mu, fl, fac)
    Jd = _fd_jacobian(m, fl, k0, m0, beta)
    A = w.ravel()[:, None] * Jd
    ytil = w.ravel() * (chi.ravel() - h.ravel() + Jd @ beta)
    T = 1e-2
    Md = O.prior_matrix(m, beta[:N], beta[N:], T, 1.0, 1e-6).toarray()
    Pinv = np.linalg.inv(Md)
    for rounds in (1, 3, 5):
        P = O.QpatParams(T=T, max_lsqr=rounds, fixed_counts=True, lsqr_reorth=True)
        res = O.linearisation_step(m, kap, mu, phi, h, fac, chi, w, beta, P)
        expect = _krylov_minimiser(A, Pinv, ytil, rounds)
        assert np.linalg.norm(res.x - expect) <= 1e-6 * np.linalg.norm(expect), rounds
    # the + J beta^(l) term changes this problem's answer by O(1)
    alt = _krylov_minimiser(A, Pinv, w.ravel() * (chi.ravel() - h.ravel()), 5)
    assert np.linalg.norm(alt - expect) > 0.1 * np.linalg.norm(expect)


def test_step_zero_is_krylov_minimiser_in_kappa_alone():
    """Step 0 of Sec. 5 is the same problem in kappa_tilde alone: A = Gamma^-1/2
    J_kappa, y^ = Gamma^-1/2 (chi - h + J_kappa kappa_tilde_init) and the
    prior M(kappa_tilde_init) + delta I of the kappa block; the result after
    m rounds is that Krylov minimiser (dense numpy, J from central
    differences).  Solving for both blocks, or dropping
    J_kappa kappa_tilde_init, fails it."""
    m, fl, k0, m0, beta, chi, w = _tiny_linearisation()
    N = m.N
    kt = beta[:N]
    kap, mu = k0 * np.exp(kt), m0 * np.exp(beta[N:])
    fac = O.Factor(O.system_matrix(m, kap, mu))
    phi, h = O.forward(m, kap, mu, fl, fac)
    Jk = _fd_jacobian(m, fl, k0, m0, beta)[:, :N]
    A = w.ravel()[:, None] * Jk
    yhat = w.ravel() * (chi.ravel() - h.ravel() + Jk @ kt)
    T = 1e-2
    Mk = O.prior_matrix(m, kt, np.zeros(N), T, 1.0, 1e-6).toarray()[:N, :N]
    Pinv = np.linalg.inv(Mk)
    for rounds in (1, 3, 5):
        P = O.QpatParams(T=T, max_lsqr=rounds, fixed_counts=True, lsqr_reorth=True)
        res = O.step_zero(m, kap, mu, phi, h, fac, chi, w, kt, P)
        assert res.x.shape == (N,)
        expect = _krylov_minimiser(A, Pinv, yhat, rounds)
        assert np.linalg.norm(res.x - expect) <= 1e-6 * np.linalg.norm(expect), rounds
    alt = _krylov_minimiser(A, Pinv, w.ravel() * (chi.ravel() - h.ravel()), 5)
    assert np.linalg.norm(alt - expect) > 0.1 * np.linalg.norm(expect)


def test_lsqr_reorth_keeps_krylov_minimiser_where_plain_recurrence_drifts():
    """LSQR with full reorthogonalisation follows exact arithmetic: on a
    problem whose P has one direction 1e6 above the rest (as M_delta^-1 has
    the constant mode, 1/delta), its m-th iterate stays the minimiser over
    P^-1 K_m(A^T A P^-1, A^T b) (basis built by dense projection with full
    orthogonalisation) for m up to 24, and it equals the plain recurrence in
    the first rounds, where that has not yet lost orthogonality."""
    rng = np.random.default_rng(31)
    mrows, ncols = 120, 60
    A = rng.standard_normal((mrows, ncols)) @ np.diag(np.logspace(0, -3, ncols))
    Qm = np.linalg.qr(rng.standard_normal((ncols, ncols)))[0]
    lam = np.logspace(-1, 1, ncols)
    lam[0] = 1e-6                                   # the 1/delta-like direction of P^-1
    P = Qm @ np.diag(lam) @ Qm.T
    Pinv = Qm @ np.diag(1.0 / lam) @ Qm.T
    b = rng.standard_normal(mrows)
    for m in (3, 12, 24):
        res = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, m,
                           fixed_counts=True, reorth=True)
        # orthonormal basis of the Krylov space, each new vector orthogonalised twice
        Vb = []
        r = A.T @ b
        for _ in range(m):
            v = Pinv @ r
            for _ in range(2):
                for q in Vb:
                    v = v - (q @ v) * q
            Vb.append(v / np.linalg.norm(v))
            r = A.T @ (A @ v)
        V = np.stack(Vb, 1)
        xbest = V @ np.linalg.lstsq(A @ V, b, rcond=None)[0]
        assert np.linalg.norm(A @ res.x - b) <= np.linalg.norm(A @ xbest - b) * (1 + 1e-8)
        assert np.linalg.norm(res.x - xbest) <= 1e-6 * np.linalg.norm(xbest)
        assert abs(res.phibar[-1] - np.linalg.norm(A @ res.x - b)) < 1e-9 * np.linalg.norm(b)
    plain = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, 2, fixed_counts=True)
    ro = O.lsqr_prior(lambda v: A @ v, lambda u: A.T @ u, lambda p: Pinv @ p, b, 2, fixed_counts=True, reorth=True)
    assert np.linalg.norm(ro.x - plain.x) <= 1e-8 * np.linalg.norm(plain.x)


def test_jacobi_pcg_matches_sparse_lu():
    """The oracle's iterative stand-in for large meshes: Jacobi PCG to a
    relative residual of 1e-13 agrees with the SuperLU solve within the
    residual bound (cond x 1e-13) on the system matrix K and on M_delta, for
    several right-hand sides at once, and in slices of iterations."""
    cfg = S.small_config(9, 10.0, 3, 2)
    xyz, tets = cfg.mesh()
    m = O.Mesh(xyz, tets)
    kap, mu = cfg.coefficients(xyz)
    rng = np.random.default_rng(5)
    A = O.system_matrix(m, kap, mu)
    B = rng.standard_normal((m.N, 3))
    X = O.JacobiPcg(A).solve(B)
    Xd = np.stack([O.Factor(A).solve(B[:, j]) for j in range(3)], 1)
    assert np.linalg.norm(X - Xd) <= 1e-10 * np.linalg.norm(Xd)
    assert np.linalg.norm(B - A @ X) <= 1.01e-13 * np.linalg.norm(B) * np.sqrt(3)
    kt, mt = 0.2 * rng.standard_normal(m.N), 0.2 * rng.standard_normal(m.N)
    P = O.prior_matrix(m, kt, mt, 1e-2, 1.0, 1e-6)
    b = rng.standard_normal(2 * m.N)
    cg = O.JacobiPcg(P)
    cg.start(b)
    n = 0
    while not cg.advance(7):
        n += 1
    x = cg.result()
    lam = np.linalg.eigvalsh(P.toarray())
    xd = O.Factor(P).solve(b)
    assert n > 3 and x.shape == b.shape
    assert np.linalg.norm(x - xd) <= 1e-13 * (lam[-1] / lam[0]) * np.linalg.norm(xd) * 10
