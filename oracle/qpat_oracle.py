"""CPU FP64 oracle of the QPAT reconstruction -- TEST INFRASTRUCTURE ONLY.

Plain, slow and obviously correct: every operator is an assembled scipy CSR
matrix built from exact P1 integrals, every inverse is a sparse LU solve
(SuperLU, a library primitive), and LSQR / Algorithm 1 follow the paper's
steps in its order and notation.  Only `tests/`, `__graft_entry__.smoke()` and
the CPU-baseline / reference leg of `bench.py` may use it.  It shares no code,
table or constant with the CUDA path.

Paper sections used:
  Eq. (1)   Robin BVP of the diffusion approximation
  Eq. (2)   H = mu * phi;   Eq. (7) nodal h_n = mu_n phi_n
  Eq. (3)   derivative variational problem (Lemma 1)
  Eq. (4)-(5) log parametrisation with P1 coefficient vectors
  Eq. (10)  Perona-Malik r(t);  Eq. (14) lagged-diffusivity operator M(u)
  Eq. (16), (19) block prior M and M_delta = M + delta I
  Eq. (21)-(22) priorconditioned LSQR and its stopping rule
  Algorithm 1 (with step 0 of Sec. 5) and the multi-illumination rule of Sec. 4
  Appendix: weak form, G(1), G(2), J s and J^T t

Every function states which of these it follows.  Where the paper is silent
the reading taken is written in the docstring.

Pinned by tests/test_oracle_*.py against closed forms, invariants, finite
differences, dense brute force and textbook reference-element matrices.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "Mesh", "QpatParams", "tet_geometry", "boundary_faces", "face_areas",
    "int_bary_tet", "int_bary_tri", "assemble_stiffness", "assemble_weighted_mass",
    "assemble_robin", "load_vector", "load_vector_nodal", "flux_patch", "flux_side", "system_matrix", "Factor",
    "JacobiPcg",
    "forward", "G1_matrix", "G2_matrix", "jvp", "vjp", "lagged_weights", "tvq_r", "tvq_rprime",
    "prior_matrix", "prior_solve", "lsqr_prior", "fit_background", "init_mu",
    "linearised_data", "step_zero", "linearisation_step",
    "reconstruct", "measure", "nonlinear_residual", "simulate_data",
]


# --------------------------------------------------------------------------
# Mesh geometry (Sec. 3, Eq. (5): P1 basis on a tetrahedral partition)
# --------------------------------------------------------------------------

def tet_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Volumes |T| and barycentric gradients grad(lambda_i) of every tet.

    With vertices p0..p3 and the edge matrix D (rows p_i - p0, i = 1..3),
    x - p0 = D^T (lambda_1, lambda_2, lambda_3), so grad(lambda_i) is column i
    of D^{-1} and grad(lambda_0) = -(sum of the other three).  |T| = |det D|/6.
    Returns vol (E,), grads (E, 4, 3).
    """
    p = xyz[tets]                        # E x 4 x 3
    D = p[:, 1:, :] - p[:, :1, :]        # E x 3 x 3, rows = edges
    det = np.linalg.det(D)
    Dinv = np.linalg.inv(D)              # columns are grad(lambda_1..3)
    g123 = np.transpose(Dinv, (0, 2, 1))  # E x 3 x 3, row i = grad lambda_{i+1}
    g0 = -g123.sum(axis=1, keepdims=True)
    grads = np.concatenate([g0, g123], axis=1)
    vol = np.abs(det) / 6.0
    return vol, grads


def boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Boundary triangles of a conforming tet mesh, in canonical order.

    A face (vertex triple) is on the boundary iff exactly one tet has it.
    Each face is returned with its vertices sorted ascending, and the faces
    are sorted lexicographically: this canonical order is the one in which
    per-face flux arrays are given.
    """
    f = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                        tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]], axis=0)
    f = np.sort(f, axis=1)
    uniq, counts = np.unique(f, axis=0, return_counts=True)
    return uniq[counts == 1].astype(np.int64)


def face_areas(xyz: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """|F| = half the norm of the cross product of two edges."""
    a = xyz[faces[:, 1]] - xyz[faces[:, 0]]
    b = xyz[faces[:, 2]] - xyz[faces[:, 0]]
    return 0.5 * np.linalg.norm(np.cross(a, b), axis=1)


def int_bary_tet(alpha) -> float:
    """Exact integral over a tet of prod lambda_i^alpha_i, divided by |T|:
    3! prod(alpha_i!) / (sum(alpha) + 3)!  (standard simplex formula)."""
    num = 6 * np.prod([math.factorial(a) for a in alpha])
    return num / math.factorial(sum(alpha) + 3)


def int_bary_tri(alpha) -> float:
    """Exact integral over a triangle of prod lambda_i^alpha_i, divided by
    |F|: 2! prod(alpha_i!) / (sum(alpha) + 2)!."""
    num = 2 * np.prod([math.factorial(a) for a in alpha])
    return num / math.factorial(sum(alpha) + 2)


def _w3_tet() -> np.ndarray:
    """W[i, j, k] = (1/|T|) * integral of lambda_i lambda_j lambda_k."""
    W = np.zeros((4, 4, 4))
    for i in range(4):
        for j in range(4):
            for k in range(4):
                a = [0, 0, 0, 0]
                a[i] += 1
                a[j] += 1
                a[k] += 1
                W[i, j, k] = int_bary_tet(a)
    return W


def _w1_tet() -> np.ndarray:
    """(1/|T|) * integral of lambda_i  (= 1/4)."""
    return np.array([int_bary_tet([1 if q == i else 0 for q in range(4)]) for i in range(4)])


def _w2_tri() -> np.ndarray:
    W = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            a = [0, 0, 0]
            a[i] += 1
            a[j] += 1
            W[i, j] = int_bary_tri(a)
    return W


@dataclasses.dataclass
class Mesh:
    """Tet mesh with the geometry the FE assembly needs (Sec. 3, Eq. (5))."""
    xyz: np.ndarray
    tets: np.ndarray

    def __post_init__(self):
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float64)
        self.tets = np.ascontiguousarray(self.tets, dtype=np.int64)
        self.vol, self.grads = tet_geometry(self.xyz, self.tets)
        self.faces = boundary_faces(self.tets)
        self.farea = face_areas(self.xyz, self.faces)

    @property
    def N(self) -> int:
        return self.xyz.shape[0]

    @property
    def E(self) -> int:
        return self.tets.shape[0]

    @property
    def F(self) -> int:
        return self.faces.shape[0]


def _coo_assemble(N, conn, local):
    """Sum local (E x m x m) matrices into an N x N CSR matrix."""
    m = conn.shape[1]
    rows = np.repeat(conn, m, axis=1).ravel()
    cols = np.tile(conn, (1, m)).ravel()
    return sp.coo_matrix((local.ravel(), (rows, cols)), shape=(N, N)).tocsr()


# --------------------------------------------------------------------------
# FE operators (Appendix, weak form of Eq. (1); Eq. (3); Eq. (14))
# --------------------------------------------------------------------------

def assemble_stiffness(mesh: Mesh, c_elem: np.ndarray) -> sp.csr_matrix:
    """S(c)_ij = sum_T c_T |T| grad(lambda_i) . grad(lambda_j) for an
    element-constant coefficient c_T (E,)."""
    loc = np.einsum("e,eid,ejd->eij", mesh.vol * c_elem, mesh.grads, mesh.grads)
    return _coo_assemble(mesh.N, mesh.tets, loc)


def elem_mean_integral(mesh: Mesh, c_nodal: np.ndarray) -> np.ndarray:
    """(1/|T|) integral over T of the P1 interpolant of nodal c:
    sum_k c_k (1/|T|) integral lambda_k."""
    return c_nodal[mesh.tets] @ _w1_tet()


def assemble_kappa_stiffness(mesh: Mesh, kappa: np.ndarray) -> sp.csr_matrix:
    """integral kappa_h grad(phi_i) . grad(phi_j) with P1 kappa_h: since the
    gradients are constant on T this is S(c) with c_T the exact element
    mean of kappa_h."""
    return assemble_stiffness(mesh, elem_mean_integral(mesh, kappa))


def assemble_weighted_mass(mesh: Mesh, c_nodal: np.ndarray) -> sp.csr_matrix:
    """M(c)_ij = integral c_h lambda_i lambda_j for the P1 interpolant c_h:
    sum_T |T| sum_k c_k W[i, j, k] with the exact simplex weights W."""
    W = _w3_tet()
    loc = mesh.vol[:, None, None] * np.einsum("ijk,ek->eij", W, c_nodal[mesh.tets])
    return _coo_assemble(mesh.N, mesh.tets, loc)


def assemble_robin(mesh: Mesh) -> sp.csr_matrix:
    """Boundary term (1/2) integral_{dOmega} phi v of the weak form
    (Appendix): B_ij = 1/2 sum_F |F| (1/|F|) integral lambda_i lambda_j."""
    W = _w2_tri()
    loc = 0.5 * mesh.farea[:, None, None] * W[None, :, :]
    return _coo_assemble(mesh.N, mesh.faces, loc)


def load_vector(mesh: Mesh, flux_face: np.ndarray) -> np.ndarray:
    """f_i = 2 integral_{dOmega} Phi lambda_i (Appendix) for a face-constant
    flux Phi_F given in canonical face order: 2 sum_F Phi_F |F| / 3."""
    w1 = np.array([int_bary_tri([1 if q == i else 0 for q in range(3)]) for i in range(3)])
    f = np.zeros(mesh.N)
    contrib = 2.0 * (flux_face * mesh.farea)[:, None] * w1[None, :]
    np.add.at(f, mesh.faces, contrib)
    return f


def load_vector_nodal(mesh: Mesh, flux_nodal: np.ndarray) -> np.ndarray:
    """f_i = 2 integral_{dOmega} Phi_h lambda_i for the P1 boundary
    interpolant Phi_h of nodal flux values (used for manufactured data)."""
    W = _w2_tri()
    loc = 2.0 * mesh.farea[:, None] * (flux_nodal[mesh.faces] @ W.T)
    f = np.zeros(mesh.N)
    np.add.at(f, mesh.faces, loc)
    return f


def flux_patch(mesh: Mesh, center, normal, half_w: float, amp: float = 1.0,
               tol: float = 1e-9) -> np.ndarray:
    """Face-constant flux of a square boundary patch (Sec. 5, Test 2
    characteristic functions).  Reading: a boundary face is lit (Phi_F = amp)
    iff all three vertices lie on the plane through `center` with normal
    `normal` and the face centroid lies in the closed square of half width
    `half_w` around `center` (infinity norm over the tangent axes)."""
    c = np.asarray(center, dtype=np.float64)
    nv = np.asarray(normal, dtype=np.float64)
    scale = np.max(np.ptp(mesh.xyz, axis=0))
    p = mesh.xyz[mesh.faces]                     # F x 3 x 3
    on_plane = np.all(np.abs((p - c) @ nv) <= tol * scale, axis=1)
    cen = p.mean(axis=1) - c
    tang = cen - np.outer(cen @ nv, nv)
    inside = np.max(np.abs(tang), axis=1) <= half_w + tol * scale
    return np.where(on_plane & inside, amp, 0.0)


def flux_side(mesh: Mesh, center, axis, ref, radius: float, theta0: float,
              half_w: float = np.pi / 8, amp: float = 1.0, tol: float = 1e-9) -> np.ndarray:
    """Face-constant flux through the curved side of a cylinder (Sec. 5,
    Test 1): Phi(theta) = amp cos(pi/2 (theta - theta0) / half_w) for
    |theta - theta0| <= half_w (the paper's cos(4 (theta - theta0)) on
    [theta0 - pi/8, theta0 + pi/8]), homogeneous along the axis.  Reading: a
    boundary face belongs to the side iff its three vertices lie at distance
    `radius` from the axis (line through `center` along `axis`); it takes
    the value of Phi at the polar angle of its centroid, measured about the
    axis from the direction `ref` (projected off the axis)."""
    c = np.asarray(center, dtype=np.float64)
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    e1 = np.asarray(ref, dtype=np.float64)
    e1 = e1 - (e1 @ a) * a
    e1 = e1 / np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    scale = np.max(np.ptp(mesh.xyz, axis=0))
    p = mesh.xyz[mesh.faces] - c                     # F x 3 x 3
    radial = p - (p @ a)[..., None] * a
    on_side = np.all(np.abs(np.linalg.norm(radial, axis=2) - radius) <= tol * scale, axis=1)
    cen = p.mean(axis=1)
    theta = np.arctan2(cen @ e2, cen @ e1)
    d = np.angle(np.exp(1j * (theta - theta0)))      # wrapped to (-pi, pi]
    lit = on_side & (np.abs(d) <= half_w)
    return np.where(lit, amp * np.cos(0.5 * np.pi * d / half_w), 0.0)


def system_matrix(mesh: Mesh, kappa: np.ndarray, mu: np.ndarray) -> sp.csr_matrix:
    """FE matrix K(kappa, mu) of the weak form of Eq. (1) (Appendix):
    integral (kappa grad phi . grad v + mu phi v) + 1/2 integral_{dOmega} phi v."""
    return (assemble_kappa_stiffness(mesh, kappa)
            + assemble_weighted_mass(mesh, mu)
            + assemble_robin(mesh)).tocsr()


class Factor:
    """Exact sparse solve with a fixed matrix (SuperLU factorisation)."""

    def __init__(self, A: sp.spmatrix):
        self.A = A.tocsc()
        self.lu = spla.splu(self.A, permc_spec="MMD_AT_PLUS_A")

    def solve(self, b: np.ndarray) -> np.ndarray:
        return self.lu.solve(np.asarray(b, dtype=np.float64))


class JacobiPcg:
    """Textbook Jacobi-preconditioned conjugate gradients for a symmetric
    positive definite A, several right-hand sides at once (each column its
    own CG), stopped per column at |b - A x| <= rtol |b| (the recursive
    residual).  The stand-in for Factor where a sparse factorisation of A is
    out of reach (millions of 3D finite-element unknowns); same .solve(b)
    interface.  The iteration can advance in slices (start / advance) so
    that a caller can time bounded parts of one solve."""

    def __init__(self, A: sp.spmatrix, rtol: float = 1e-13, maxit: int = 200000):
        self.A = A.tocsr()
        self.dinv = 1.0 / self.A.diagonal()
        self.rtol = rtol
        self.maxit = maxit

    def start(self, B: np.ndarray):
        B = np.asarray(B, dtype=np.float64)
        self.one = B.ndim == 1
        B = B.reshape(B.shape[0], -1)
        self.x = np.zeros_like(B)
        self.r = B.copy()
        self.z = self.dinv[:, None] * self.r
        self.p = self.z.copy()
        self.rz = np.einsum("ij,ij->j", self.r, self.z)
        self.stop2 = (self.rtol ** 2) * np.einsum("ij,ij->j", B, B)
        self.active = np.einsum("ij,ij->j", self.r, self.r) > self.stop2
        self.iters = np.zeros(B.shape[1], dtype=np.int64)

    def advance(self, n: int) -> bool:
        """Up to n CG iterations of every unconverged column; True when all
        columns have converged."""
        for _ in range(n):
            a = np.flatnonzero(self.active)
            if a.size == 0:
                return True
            p = self.p[:, a]
            q = self.A @ p
            alpha = self.rz[a] / np.einsum("ij,ij->j", p, q)
            self.x[:, a] += alpha * p
            r = self.r[:, a] - alpha * q
            self.r[:, a] = r
            z = self.dinv[:, None] * r
            rz_new = np.einsum("ij,ij->j", r, z)
            self.p[:, a] = z + (rz_new / self.rz[a]) * p
            self.rz[a] = rz_new
            self.iters[a] += 1
            done = np.einsum("ij,ij->j", r, r) <= self.stop2[a]
            self.active[a[done]] = False
            if self.iters.max() >= self.maxit:
                raise RuntimeError("JacobiPcg: iteration cap reached")
        return not self.active.any()

    def result(self) -> np.ndarray:
        return self.x[:, 0].copy() if self.one else self.x.copy()

    def solve(self, b: np.ndarray) -> np.ndarray:
        self.start(b)
        while not self.advance(1000):
            pass
        return self.result()


# --------------------------------------------------------------------------
# Forward model and matrix-free Jacobian (Appendix)
# --------------------------------------------------------------------------

def forward(mesh: Mesh, kappa, mu, flux: np.ndarray, factor: Optional[Factor] = None):
    """phi^(k) = K^{-1} f^(k) and h^(k) = mu * phi^(k) (Appendix; Eq. (7)).

    flux: K x F face fluxes.  Returns (phi, h), each K x N."""
    flux = np.atleast_2d(flux)
    if factor is None:
        factor = Factor(system_matrix(mesh, kappa, mu))
    phi = np.stack([factor.solve(load_vector(mesh, fk)) for fk in flux])
    return phi, mu[None, :] * phi


def measure(mesh: Mesh, kappa, mu, flux):
    """h(kappa, mu) for all illuminations (K x N)."""
    return forward(mesh, kappa, mu, flux)[1]


def G1_matrix(mesh: Mesh, phi: np.ndarray) -> sp.csr_matrix:
    """G(1)_ij = - integral phi_j grad(varphi) . grad(phi_i) (Appendix):
    - sum_T grad(varphi_h)|_T . grad(lambda_i) * integral_T lambda_j."""
    gphi = np.einsum("ek,ekd->ed", phi[mesh.tets], mesh.grads)   # E x 3
    a = np.einsum("ed,eid->ei", gphi, mesh.grads)                 # E x 4 (row i)
    w1 = _w1_tet()
    loc = -(mesh.vol[:, None, None] * a[:, :, None] * w1[None, None, :])
    return _coo_assemble(mesh.N, mesh.tets, loc)


def G2_matrix(mesh: Mesh, phi: np.ndarray) -> sp.csr_matrix:
    """G(2)_ij = - integral phi_j varphi phi_i (Appendix)."""
    return -assemble_weighted_mass(mesh, phi)


def _wts(w, K, N):
    return np.ones((K, N)) if w is None else np.broadcast_to(w, (K, N))


def jvp(mesh: Mesh, kappa, mu, phi, s, w=None, factor: Optional[Factor] = None):
    """(w o J s) for the stacked illuminations (Appendix):

    J s = diag(mu) K^{-1} (G(1) diag(kappa) s1 + G(2) diag(mu) s2)
          + diag(varphi) diag(mu) s2,  per illumination.
    s = [s1; s2] in R^{2N} (derivative w.r.t. the log parameters, Eq. (4)).
    Returns K x N."""
    phi = np.atleast_2d(phi)
    K, N = phi.shape
    if factor is None:
        factor = Factor(system_matrix(mesh, kappa, mu))
    s1, s2 = s[:N], s[N:]
    out = np.empty((K, N))
    for k in range(K):
        rhs = G1_matrix(mesh, phi[k]) @ (kappa * s1) + G2_matrix(mesh, phi[k]) @ (mu * s2)
        out[k] = mu * factor.solve(rhs) + phi[k] * mu * s2
    return out * _wts(w, K, N)


def vjp(mesh: Mesh, kappa, mu, phi, t, w=None, factor: Optional[Factor] = None):
    """J^T (w o t) summed over the stacked illuminations (Appendix):

    J^T t = blkdiag(kappa, mu) ( [G(1)^T; G(2)] K^{-1} diag(mu) t + [0; diag(varphi) t] ),
    using the symmetry of K and G(2).  t: K x N.  Returns 2N."""
    phi = np.atleast_2d(phi)
    K, N = phi.shape
    t = np.atleast_2d(t) * _wts(w, K, N)
    if factor is None:
        factor = Factor(system_matrix(mesh, kappa, mu))
    o1 = np.zeros(N)
    o2 = np.zeros(N)
    for k in range(K):
        z = factor.solve(mu * t[k])
        o1 += G1_matrix(mesh, phi[k]).T @ z
        o2 += G2_matrix(mesh, phi[k]) @ z + phi[k] * t[k]
    return np.concatenate([kappa * o1, mu * o2])


# --------------------------------------------------------------------------
# Lagged-diffusivity prior (Eqs. (10), (14), (16), (19))
# --------------------------------------------------------------------------

def pm_rprime(t, T):
    """r'(t) for the Perona-Malik r(t) = 1/2 T^2 log(1 + (t/T)^2) of Eq. (10)."""
    return t / (1.0 + (t / T) ** 2)


def tvq_r(t, T, q):
    """Smoothed TV^q, one of the alternatives to Eq. (10) named in Sec. 3:
    r(t) = (t^2 + T^2)^(q/2) / q (q = 1: smoothed total variation; the
    smoothing T makes r continuously differentiable at t = 0, as Eq. (9)
    requires)."""
    return (t * t + T * T) ** (q / 2.0) / q


def tvq_rprime(t, T, q):
    """d/dt of tvq_r: t (t^2 + T^2)^(q/2 - 1)."""
    return t * (t * t + T * T) ** (q / 2.0 - 1.0)


def lagged_weights(mesh: Mesh, u: np.ndarray, T: float, prior: int = 0, q: float = 1.0) -> np.ndarray:
    """c_u = r'(|grad u|) / |grad u| on every tet (Eq. (14)); grad u is
    constant on a tet for P1 u.  prior 0: Perona-Malik (Eq. (10)); prior 1:
    smoothed TV^q (tvq_r).  At |grad u| = 0 the limit value is used: 1 for
    Perona-Malik, T^(q-2) for TV^q."""
    g = np.einsum("ek,ekd->ed", u[mesh.tets], mesh.grads)
    t = np.linalg.norm(g, axis=1)
    nz = t > 0
    if prior == 0:
        c = np.ones_like(t)
        c[nz] = pm_rprime(t[nz], T) / t[nz]
    else:
        c = np.full_like(t, T ** (q - 2.0))
        c[nz] = tvq_rprime(t[nz], T, q) / t[nz]
    return c


def prior_matrix(mesh: Mesh, kt, mt, T: float, b_over_a: float, delta: float, prior: int = 0, q: float = 1.0):
    """M_delta = blkdiag(M(kt), (b/a) M(mt)) + delta I (Eqs. (16), (19)), with
    M(u) the FE matrix of -div(c_u grad) with natural boundary condition."""
    Mk = assemble_stiffness(mesh, lagged_weights(mesh, kt, T, prior, q))
    Mm = assemble_stiffness(mesh, lagged_weights(mesh, mt, T, prior, q))
    M = sp.block_diag([Mk, b_over_a * Mm], format="csr")
    return (M + delta * sp.identity(2 * mesh.N, format="csr")).tocsr()


def prior_solve(mesh: Mesh, kt, mt, rhs, T: float, b_over_a: float = 1.0,
                delta: float = 1e-6, prior: int = 0, q: float = 1.0):
    """x = M_delta^{-1} rhs (the one prior solve of each LSQR round, Sec. 4)."""
    return Factor(prior_matrix(mesh, kt, mt, T, b_over_a, delta, prior, q)).solve(rhs)


# --------------------------------------------------------------------------
# Priorconditioned LSQR (Eqs. (21)-(22))
# --------------------------------------------------------------------------

BREAKDOWN = 1e-12   # relative size below which a Golub-Kahan direction counts as zero


@dataclasses.dataclass
class LsqrResult:
    x: np.ndarray
    phibar: List[float]      # |A x_m - b| estimates, m = 0..iters
    iters: int
    stop_rule: bool


def lsqr_prior(A: Callable, AT: Callable, Pinv: Callable, b: np.ndarray,
               max_iter: int, m0: int = 10, tau: float = 1e-2,
               fixed_counts: bool = False, reorth: bool = False) -> LsqrResult:
    """LSQR for min |A L^{-1} xt - b|, x = L^{-1} xt, L^T L = P, started from
    xt = 0 and carried out in x-space so that only P^{-1} = M_delta^{-1} is
    applied, once per round (Eq. (21), Sec. 4).

    Golub-Kahan bidiagonalisation of A L^{-1} written with p = A^T u,
    v = P^{-1} p / alpha (x-space direction), q = p / alpha:
      beta u = A v - alpha u,   alpha^2 = p . P^{-1} p with p = A^T u - beta q,
    followed by the plane rotation that keeps the QR factor of the
    bidiagonal matrix, giving |A x_m - b| = phibar_m.
    Stops when r_m = 1 - phibar_m / phibar_{m-m0} <= tau for m > m0
    (Eq. (22)), or after max_iter rounds; with fixed_counts it always runs
    max_iter rounds.  phibar is the residual estimate of Eq. (22).

    reorth: full reorthogonalisation (a numerical realisation of the same
    method, not a change of it).  In exact arithmetic the u's are
    orthonormal and the v's are P-orthonormal (v_i . P v_j = delta_ij, with
    q_j = P v_j), so subtracting their components again changes nothing; in
    floating point it stops the loss of orthogonality that otherwise lets
    the 1/delta mode of M_delta^-1 re-enter every few rounds.  Each new
    u-hat is projected off all earlier u's and each new p off all earlier
    v's (p -= (v_j . p) q_j, which P-orthogonalises z = P^-1 p), both by
    classical Gram-Schmidt applied twice."""
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return LsqrResult(np.zeros_like(np.asarray(AT(b))), [0.0], 0, False)
    u = b / beta
    p = AT(u)
    x = np.zeros_like(p)
    z = Pinv(p)
    alpha = math.sqrt(max(float(p @ z), 0.0))
    if alpha == 0.0:
        return LsqrResult(x, [beta], 0, False)
    v = z / alpha
    q = p / alpha
    wd = v.copy()
    phibar = beta
    rhobar = alpha
    hist = [phibar]
    m = 0
    stopped = False
    U, V, Qb = [u], [v], [q]
    while m < max_iter:
        m += 1
        av = A(v)
        uh = av - alpha * u
        if reorth:
            for _ in range(2):
                uh = uh - np.stack(U, axis=1) @ (np.stack(U, axis=0) @ uh)
        beta = np.linalg.norm(uh)
        # breakdown: a new direction that vanishes against the scale of the
        # product that made it ends the bidiagonalisation; the rotation
        # below then completes the exact least-squares solution over the
        # Krylov space and the iteration stops
        done = beta <= BREAKDOWN * np.linalg.norm(av)
        if done:
            beta = 0.0
            alpha = 0.0
        else:
            u = uh / beta
            atu = AT(u)
            p = atu - beta * q
            if reorth:
                for _ in range(2):
                    p = p - np.stack(Qb, axis=1) @ (np.stack(V, axis=0) @ p)
            if np.linalg.norm(p) <= BREAKDOWN * np.linalg.norm(atu):
                done = True
                alpha = 0.0
            else:
                z = Pinv(p)
                alpha = math.sqrt(max(float(p @ z), 0.0))
                if alpha > 0:
                    v = z / alpha
                    q = p / alpha
                else:
                    done = True
        if reorth:
            U.append(u)
            V.append(v)
            Qb.append(q)
        rho = math.hypot(rhobar, beta)
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi_m = c * phibar
        phibar = s * phibar
        x = x + (phi_m / rho) * wd
        wd = v - (theta / rho) * wd
        hist.append(phibar)
        if done:
            break
        if not fixed_counts and m > m0:
            r_m = 1.0 - hist[m] / hist[m - m0]
            if r_m <= tau:
                stopped = True
                break
    return LsqrResult(x, hist, m, stopped)


# --------------------------------------------------------------------------
# Algorithm 1 (with step 0 and several illuminations)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class QpatParams:
    """Free parameters of Algorithm 1 (defaults: Sec. 4, end)."""
    T: float = 5e-3
    b_over_a: float = 1.0
    delta: float = 1e-6
    tau: float = 1e-2
    m0: int = 10
    max_lin: int = 5          # linearisations, step 0 included
    max_lsqr: int = 50
    fixed_counts: bool = False
    fit_grid: int = 9
    fit_gn_steps: int = 10
    prior: int = 0            # 0: Perona-Malik (Eq. (10)); 1: smoothed TV^q (tvq_r)
    prior_q: float = 1.0
    # Not in the paper (an option, off by default): before rejecting a step
    # in step 4, try beta + 2^-j (beta_new - beta) for j = 1..step_halvings;
    # step 0's update is then also accepted only if it lowers the residual
    # (first of x, x/2, ...; otherwise kappa_tilde_init is kept).
    step_halvings: int = 0
    # LSQR with full reorthogonalisation (lsqr_prior, reorth): the iterates of
    # exact arithmetic, to rounding (the reading of step 3's LSQR).  False
    # runs the plain recurrence, which loses orthogonality after a few tens
    # of rounds: on the 11^3 cube one 50-round sweep then moves by 1e-2 - 6e-2
    # under 1e-13 perturbations of the solves (reorthogonalised: ~1e-12).
    lsqr_reorth: bool = True


def nonlinear_residual(chi, h, w) -> float:
    """|Gamma^{-1/2} (chi - h)| with Gamma^{-1/2} = diag(w) (Algorithm 1, step 4)."""
    return float(np.linalg.norm((w * (chi - h)).ravel()))


FIT_KAPPA_RANGE = (0.05, 2.0)
FIT_MU_RANGE = (1e-3, 0.1)


def fit_background(mesh: Mesh, flux, chi, w, grid: int = 9, gn_steps: int = 10):
    """(kappa_0, mu_0) minimising |Gamma^{-1/2}(chi - h(log k 1, log m 1))|
    (Algorithm 1, preamble).  The paper does not name the optimiser; the
    reading: a grid x grid log-spaced search over kappa in [0.05, 2] mm and
    mu in [1e-3, 0.1] mm^-1 (first minimum in row-major (kappa, mu) order),
    then up to `gn_steps` Gauss-Newton steps in (log kappa, log mu) using the
    two Jacobian columns J [1;0] and J [0;1], each step halved up to 5 times
    until the residual decreases (else the search stops)."""
    N = mesh.N
    ks = np.exp(np.linspace(math.log(FIT_KAPPA_RANGE[0]), math.log(FIT_KAPPA_RANGE[1]), grid))
    ms = np.exp(np.linspace(math.log(FIT_MU_RANGE[0]), math.log(FIT_MU_RANGE[1]), grid))

    def resid(a, b):
        kap = np.full(N, math.exp(a))
        mu = np.full(N, math.exp(b))
        fac = Factor(system_matrix(mesh, kap, mu))
        phi, h = forward(mesh, kap, mu, flux, fac)
        return nonlinear_residual(chi, h, w), kap, mu, phi, fac

    best = None
    for i, kv in enumerate(ks):
        for j, mv in enumerate(ms):
            r = resid(math.log(kv), math.log(mv))[0]
            if best is None or r < best[0]:
                best = (r, math.log(kv), math.log(mv))
    r0, a, b = best
    for _ in range(gn_steps):
        r0, kap, mu, phi, fac = resid(a, b)
        ones, zeros = np.ones(N), np.zeros(N)
        ja = jvp(mesh, kap, mu, phi, np.concatenate([ones, zeros]), w, fac).ravel()
        jb = jvp(mesh, kap, mu, phi, np.concatenate([zeros, ones]), w, fac).ravel()
        h = mu[None, :] * phi
        res = (w * (chi - h)).ravel()
        Amat = np.stack([ja, jb], axis=1)
        d = np.linalg.solve(Amat.T @ Amat, Amat.T @ res)
        step = 1.0
        accepted = False
        for _h in range(6):
            r1 = resid(a + step * d[0], b + step * d[1])[0]
            if r1 < r0:
                a, b = a + step * d[0], b + step * d[1]
                accepted = True
                break
            step *= 0.5
        if not accepted:
            break
    return math.exp(a), math.exp(b)


def init_mu(chi, phi0, mu0):
    """mu_init = (1/K) sum_k chi^(k) / phi0^(k) (Algorithm 1 with the
    multi-illumination rule of Sec. 4); mu_tilde = log(mu_init / mu0).
    Reading (the paper assumes phi0 > 0): a P1 solution can undershoot to
    phi0 <= 0 far from the sources, so where the average is not positive
    mu_init = mu0, and mu_init is then clipped into [mu0 / 10, 10 mu0]."""
    mu_init = np.mean(chi / phi0, axis=0)
    mu_init = np.where(mu_init > 0, mu_init, mu0)
    mu_init = np.clip(mu_init, 0.1 * mu0, 10.0 * mu0)
    return np.log(mu_init / mu0)


def simulate_data(cfg, noise_seed: int, floor: float = 1e-3):
    """Synthetic measurement of Sec. 5 (Test 1): h on the nested 2x finer
    mesh, injected onto the coarse nodes (the interpolation P), plus Gaussian
    noise eta_i ~ N(0, sigma_i^2) with sigma_i = 0.01 |h_i|.  Reading: sigma
    gets a floor of `floor` x max|h| so that Gamma stays positive definite
    where the P1 data is ~0.  cfg is a qpat_synth.Config.
    Returns (chi, sigma, h), each K x N on the coarse nodes."""
    import qpat_synth as S
    xf, tf = S.kuhn_cube(2 * cfg.n - 1, cfg.L)
    mf = Mesh(xf, tf)
    kf, muf = cfg.coefficients(xf)
    flf = np.stack([flux_patch(mf, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
    hf = measure(mf, kf, muf, flf)
    h = hf[:, S.fine_to_coarse_index(cfg.n)]
    sig = 0.01 * np.abs(h) + floor * np.abs(h).max()
    chi = h + sig * S.noise_draws(noise_seed, h.shape)
    return chi, sig, h


@dataclasses.dataclass
class ReconReport:
    kappa0: float
    mu0: float
    residuals: List[float]           # nonlinear residual at each accepted beta
    lsqr_iters: List[int]
    lsqr_phibar: List[List[float]]
    linearisations: int
    accepted_last: bool
    beta: Optional[np.ndarray] = None  # final beta^(l) = [kappa_tilde, mu_tilde]


def linearised_data(chi, h, Jbeta, w) -> np.ndarray:
    """y~ = Gamma^{-1/2} (chi - h(beta^(l)) + J^(l) beta^(l)), stacked over the
    illuminations (Algorithm 1, step 1; the y^(l) of Eq. (11)).  chi, h, Jbeta
    and the whitening w = diag(Gamma^{-1/2}) are K x N; returns K N."""
    return (w * (chi - h + Jbeta)).ravel()


def step_zero(mesh: Mesh, kap, mu, phi, h, fac, chi, w, kt, P: QpatParams) -> LsqrResult:
    """Step 0 of Sec. 5 (Test 1): with J_kappa the Jacobian w.r.t. kappa_tilde
    alone at (kappa_tilde_init, mu_tilde_init), y^ = Gamma^{-1/2}(chi - h +
    J_kappa kappa_tilde_init) and the prior M_delta(kappa_tilde_init) =
    M(kappa_tilde_init) + delta I of the kappa block only, LSQR from zero.
    kap, mu, phi, h and the factor of K belong to beta_init.  Returns the LSQR
    result; its x is the new kappa_tilde_init."""
    K, N = np.atleast_2d(chi).shape
    zeros = np.zeros(N)
    Jk = jvp(mesh, kap, mu, phi, np.concatenate([kt, zeros]), None, fac)
    yhat = linearised_data(chi, h, Jk, w)
    Mk = Factor(assemble_stiffness(mesh, lagged_weights(mesh, kt, P.T, P.prior, P.prior_q))
                + P.delta * sp.identity(N, format="csr"))
    A0 = lambda v: jvp(mesh, kap, mu, phi, np.concatenate([v, zeros]), w, fac).ravel()
    AT0 = lambda u: vjp(mesh, kap, mu, phi, u.reshape(K, N), w, fac)[:N]
    return lsqr_prior(A0, AT0, Mk.solve, yhat, P.max_lsqr, P.m0, P.tau, P.fixed_counts, P.lsqr_reorth)


def linearisation_step(mesh: Mesh, kap, mu, phi, h, fac, chi, w, beta, P: QpatParams) -> LsqrResult:
    """Steps 1-3 of Algorithm 1 at beta^(l) (kap, mu, phi, h and the factor of
    K belong to beta^(l)): y~ of step 1, M_delta = blkdiag(M(kappa_tilde^(l)),
    (b/a) M(mu_tilde^(l))) + delta I of step 2 (Eqs. (16), (19)), and the
    priorconditioned LSQR of step 3 from zero (Eqs. (21)-(22)).  Returns the
    LSQR result; its x is the candidate beta^(l+1) that step 4 tests."""
    K, N = np.atleast_2d(chi).shape
    Jb = jvp(mesh, kap, mu, phi, beta, None, fac)
    ytil = linearised_data(chi, h, Jb, w)
    Pfac = Factor(prior_matrix(mesh, beta[:N], beta[N:], P.T, P.b_over_a, P.delta, P.prior, P.prior_q))
    A = lambda v: jvp(mesh, kap, mu, phi, v, w, fac).ravel()
    AT = lambda u: vjp(mesh, kap, mu, phi, u.reshape(K, N), w, fac)
    return lsqr_prior(A, AT, Pfac.solve, ytil, P.max_lsqr, P.m0, P.tau, P.fixed_counts, P.lsqr_reorth)


def reconstruct(mesh: Mesh, flux, chi, sigma, params: QpatParams,
                kappa0_mu0=None, beta_in=None, lin_done: int = 0):
    """Algorithm 1 with step 0 (Sec. 5, Test 1) for K stacked illuminations.

    flux: K x F, chi and sigma: K x N (Gamma = diag(sigma^2), so
    Gamma^{-1/2} = diag(1/sigma)).  Linearisations are counted as in Sec. 5
    (step 0 is the first).  Returns (kappa, mu, report); report.beta is the
    final beta^(l).  Resume: step 1 of Algorithm 1 starts from beta^(l)
    alone, so with beta_in (needs kappa0_mu0 and lin_done >= 1) the
    initialisation and step 0 are skipped and the loop continues from
    beta^(l) = beta_in with lin_done linearisations counted."""
    chi = np.atleast_2d(chi)
    w = 1.0 / np.atleast_2d(sigma)
    K, N = chi.shape
    P = params
    if beta_in is not None and (kappa0_mu0 is None or lin_done < 1):
        raise ValueError("resuming needs kappa0_mu0 and lin_done >= 1")
    if kappa0_mu0 is None:
        k0, m0_ = fit_background(mesh, flux, chi, w, P.fit_grid, P.fit_gn_steps)
    else:
        k0, m0_ = float(kappa0_mu0[0]), float(kappa0_mu0[1])

    def coeffs(beta):
        return k0 * np.exp(beta[:N]), m0_ * np.exp(beta[N:])

    rep = ReconReport(k0, m0_, [], [], [], 0, True)
    if beta_in is not None:
        # resume at step 1 from beta^(l)
        beta = np.array(beta_in, dtype=np.float64)
        rep.linearisations = int(lin_done)
    else:
        # initialisation
        ones = np.ones(N)
        fac0 = Factor(system_matrix(mesh, k0 * ones, m0_ * ones))
        phi0, _ = forward(mesh, k0 * ones, m0_ * ones, flux, fac0)
        mt = init_mu(chi, phi0, m0_)
        kt = np.zeros(N)

        # step 0: LSQR for kappa only, prior M_delta(kt_init)
        kap, mu = k0 * np.exp(kt), m0_ * np.exp(mt)
        fac = Factor(system_matrix(mesh, kap, mu))
        phi, h = forward(mesh, kap, mu, flux, fac)
        res0 = step_zero(mesh, kap, mu, phi, h, fac, chi, w, kt, P)
        rep.lsqr_iters.append(res0.iters)
        rep.lsqr_phibar.append(res0.phibar)
        rep.linearisations = 1
        if P.step_halvings > 0:
            # option: keep the first of x, x/2, ... that lowers the residual at beta_init
            r_init = nonlinear_residual(chi, h, w)
            kt_acc = kt
            for j in range(P.step_halvings + 1):
                kt_c = kt + res0.x if j == 0 else kt + res0.x * 0.5 ** j
                kc, mc = k0 * np.exp(kt_c), m0_ * np.exp(mt)
                _, hc = forward(mesh, kc, mc, flux, Factor(system_matrix(mesh, kc, mc)))
                if nonlinear_residual(chi, hc, w) < r_init:
                    kt_acc = kt_c
                    break
            kt = kt_acc
        else:
            kt = kt + res0.x
        beta = np.concatenate([kt, mt])

    # step 1 needs h(beta^(l))
    kap, mu = coeffs(beta)
    fac = Factor(system_matrix(mesh, kap, mu))
    phi, h = forward(mesh, kap, mu, flux, fac)
    r_cur = nonlinear_residual(chi, h, w)
    rep.residuals.append(r_cur)

    while rep.linearisations < P.max_lin:
        # steps 1-3: linearise at beta^(l), lagged M_delta, priorconditioned LSQR
        res = linearisation_step(mesh, kap, mu, phi, h, fac, chi, w, beta, P)
        rep.lsqr_iters.append(res.iters)
        rep.lsqr_phibar.append(res.phibar)
        rep.linearisations += 1
        beta_new = res.x
        # step 4: accept only if the nonlinear residual decreased (option:
        # first try the shorter steps beta + 2^-j (beta_new - beta))
        for j in range(P.step_halvings + 1):
            cand = beta_new if j == 0 else beta + (beta_new - beta) * 0.5 ** j
            kap_n, mu_n = coeffs(cand)
            fac_n = Factor(system_matrix(mesh, kap_n, mu_n))
            phi_n, h_n = forward(mesh, kap_n, mu_n, flux, fac_n)
            r_new = nonlinear_residual(chi, h_n, w)
            if r_new < r_cur:
                beta_new = cand
                break
        if r_new >= r_cur:
            rep.accepted_last = False
            break
        beta, kap, mu, fac, phi, h, r_cur = beta_new, kap_n, mu_n, fac_n, phi_n, h_n, r_new
        rep.residuals.append(r_cur)
    kap, mu = coeffs(beta)
    rep.beta = beta
    return kap, mu, rep
