"""Seeded synthetic inputs for the QPAT reconstruction hot path.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
only geometry and random draws -- the Kuhn cube mesh, phantom coefficient
fields, boundary-patch descriptions, noise draws and random vectors.  It
evaluates nothing of the method itself: no finite-element matrix, no solve, no
Jacobian.  Random numbers that the method consumes (the measurement noise of
Sec. 5, eq. for chi_i = h_i + eta_i) are drawn here and passed in as inputs.

The paper's own meshes and phantoms (Sec. 5, Tests 1 and 2, Tables 1-2) are
not available, so these seeded stand-ins reproduce their structure: a cube
body, boundary-patch illuminations given as characteristic functions (Test 2),
piecewise-constant spherical inclusions in mu_a and mu_s', 1 % Gaussian noise
and data simulated on a finer nested mesh (Sec. 5, footnote to Eq. (7)).
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "kuhn_cube", "fine_to_coarse_index", "Sphere", "Patch", "Config",
    "spheres_phantom", "blob_phantom", "config", "noise_draws",
    "random_vector", "kappa_from_optics", "CONFIG_NAMES",
    "cylinder_mesh", "SideIllumination", "CylinderConfig", "cylinder_config",
    "wavelength_optics",
]


def kuhn_cube(n: int, L: float) -> Tuple[np.ndarray, np.ndarray]:
    """Structured tetrahedral mesh of the cube [0, L]^3 with n nodes per side.

    Node (i, j, k) sits at (i, j, k) * L / (n - 1) and has index
    i + n * (j + n * k).  Each voxel is split into the 6 Kuhn tetrahedra that
    share its (0,0,0)-(1,1,1) diagonal: for every permutation (a, b, c) of the
    axes the tet is o, o + e_a, o + e_a + e_b, o + 1.  The mesh is conforming;
    orientation is left as generated (half the tets are negatively oriented),
    consumers orient them themselves.

    Returns xyz (N x 3 float64) and tets (E x 4 int32), N = n^3,
    E = 6 (n - 1)^3.
    """
    if n < 2:
        raise ValueError("kuhn_cube needs n >= 2")
    h = L / (n - 1)
    g = np.arange(n, dtype=np.float64) * h
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)

    m = n - 1
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    base = (ii + n * (jj + n * kk)).ravel().astype(np.int64)
    stride = np.array([1, n, n * n], dtype=np.int64)
    tets = []
    for perm in itertools.permutations(range(3)):
        a, b, _ = perm
        v0 = base
        v1 = base + stride[a]
        v2 = v1 + stride[b]
        v3 = base + stride.sum()
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    # voxel-major order: the 6 tets of a voxel are consecutive
    tets = np.stack(tets, axis=1).reshape(-1, 4)
    return xyz, tets.astype(np.int32)


def fine_to_coarse_index(n: int) -> np.ndarray:
    """Indices, in the (2n-1)^3 nested fine Kuhn mesh, of the n^3 coarse nodes.

    The fine mesh refines every coarse voxel into 8 voxels, so coarse node
    (i, j, k) coincides with fine node (2i, 2j, 2k).  Injection through this
    index is the interpolation P of Sec. 5 (Test 1) on nested grids.
    """
    nf = 2 * n - 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return (2 * i + nf * (2 * j + nf * 2 * k)).ravel().astype(np.int64)


@dataclasses.dataclass
class Sphere:
    center: Tuple[float, float, float]
    radius: float
    mua: float | None = None      # absorption inside (None = background)
    mus: float | None = None      # reduced scattering inside (None = background)


@dataclasses.dataclass
class Patch:
    """A square illumination patch on a face of the cube (Sec. 5, Test 2).

    `axis` is the face normal axis (0, 1, 2), `side` is 0 for the face at
    coordinate 0 and 1 for the face at coordinate L.  `center` is the patch
    centre (3 coordinates, the normal one lying on the face), `half_w` its
    half width along both tangent axes and `amp` the flux amplitude.
    A boundary triangle is lit (flux = amp) when all its vertices lie on the
    face and its centroid lies in the closed square; otherwise its flux is 0.
    """
    axis: int
    side: int
    center: Tuple[float, float, float]
    half_w: float
    amp: float = 1.0

    @property
    def normal(self) -> Tuple[float, float, float]:
        v = [0.0, 0.0, 0.0]
        v[self.axis] = 1.0 if self.side == 1 else -1.0
        return tuple(v)


def kappa_from_optics(mua: np.ndarray, mus: np.ndarray) -> np.ndarray:
    """Diffusion coefficient kappa = 1 / (3 (mu_a + mu_s')) of the phantom."""
    return 1.0 / (3.0 * (mua + mus))


def spheres_phantom(xyz: np.ndarray, spheres: Sequence[Sphere],
                    mua_bg: float, mus_bg: float):
    """Nodal mu_a, mu_s' of a background with spherical inclusions.

    A node takes the inclusion value when it lies in the closed ball; later
    spheres overwrite earlier ones.
    """
    N = xyz.shape[0]
    mua = np.full(N, mua_bg)
    mus = np.full(N, mus_bg)
    for s in spheres:
        inside = np.sum((xyz - np.asarray(s.center)) ** 2, axis=1) <= s.radius ** 2
        if s.mua is not None:
            mua[inside] = s.mua
        if s.mus is not None:
            mus[inside] = s.mus
    return mua, mus


def blob_phantom(xyz: np.ndarray, rng: np.random.Generator, L: float,
                 nblobs: int = 20, sig=(2.0, 6.0),
                 mua_range=(0.005, 0.05), mus_range=(0.5, 2.0)):
    """Log-normal blob fields: exp of a Gaussian-blob sum mapped into ranges.

    Each field is g(x) = sum_b a_b exp(-|x - c_b|^2 / (2 s_b^2)) with
    a_b ~ N(0, 1), c_b ~ U[0, L]^3, s_b ~ U[sig]; g is affinely mapped onto
    [log lo, log hi] and exponentiated.
    """
    def field(lo, hi):
        c = rng.uniform(0.0, L, size=(nblobs, 3))
        s = rng.uniform(sig[0], sig[1], size=nblobs)
        a = rng.standard_normal(nblobs)
        g = np.zeros(xyz.shape[0])
        for b in range(nblobs):
            d2 = np.sum((xyz - c[b]) ** 2, axis=1)
            g += a[b] * np.exp(-d2 / (2.0 * s[b] ** 2))
        gmin, gmax = g.min(), g.max()
        t = (g - gmin) / max(gmax - gmin, 1e-300)
        return np.exp(np.log(lo) + t * (np.log(hi) - np.log(lo)))
    mua = field(*mua_range)
    mus = field(*mus_range)
    return mua, mus


@dataclasses.dataclass
class Config:
    name: str
    n: int
    L: float
    patches: List[Patch]
    spheres: List[Sphere]
    mua_bg: float = 0.01
    mus_bg: float = 1.0
    blobs: bool = False
    seed: int = 0

    @property
    def N(self) -> int:
        return self.n ** 3

    @property
    def E(self) -> int:
        return 6 * (self.n - 1) ** 3

    @property
    def K(self) -> int:
        return len(self.patches)

    def mesh(self):
        return kuhn_cube(self.n, self.L)

    def optics(self, xyz: np.ndarray):
        """Nodal (mu_a, mu_s') of the phantom on the given nodes."""
        if self.blobs:
            return blob_phantom(xyz, np.random.default_rng(self.seed), self.L)
        return spheres_phantom(xyz, self.spheres, self.mua_bg, self.mus_bg)

    def coefficients(self, xyz: np.ndarray):
        """Nodal (kappa, mu) with mu = mu_a and kappa = 1 / (3 (mu_a + mu_s'))."""
        mua, mus = self.optics(xyz)
        return kappa_from_optics(mua, mus), mua


def _face_patches(L: float, half_w: float, faces) -> List[Patch]:
    out = []
    for axis, side in faces:
        c = [L / 2.0] * 3
        c[axis] = L if side == 1 else 0.0
        out.append(Patch(axis, side, tuple(c), half_w))
    return out


def _random_spheres(rng, L, count, rmin, rmax, first_mus=2.0):
    out = []
    margin = L / 4.0
    for i in range(count):
        c = tuple(rng.uniform(margin, L - margin, size=3))
        r = rng.uniform(rmin, rmax) if rmax > rmin else rmin
        mua = rng.uniform(0.02, 0.03)
        out.append(Sphere(c, r, mua=mua, mus=first_mus if i == 0 else None))
    return out


CONFIG_NAMES = ("c0_cube11", "c1_cube64", "c2_cube96", "c4_cube128")


def config(name: str, seed: int | None = None) -> Config:
    """Synthetic workloads standing in for the paper's test cases.

    c0_cube11  : 20 mm cube, 11^3 nodes, 2 spheres r = 3 mm (mu_a in
                 [0.02, 0.03], mu_s' = 2 in the first), 1 top-face 10 x 10 mm
                 patch.
    c1_cube64  : 40 mm cube, 64^3 nodes, 6 spheres r in [3, 6] mm, 4 patches
                 (top, bottom, +x, -x), 20 x 20 mm each.
    c2_cube96  : 40 mm cube, 96^3 nodes, blob fields, 8 patches (6 faces and
                 two off-centre on +-z).
    c4_cube128 : 40 mm cube, 128^3 nodes, blob fields, 8 patches.
    Seeds default to 1000 * config index.
    """
    if name == "c0_cube11":
        s = 0 if seed is None else seed
        rng = np.random.default_rng(s)
        L = 20.0
        spheres = []
        for i in range(2):
            c = tuple(rng.uniform(5.0, 15.0, size=3))
            spheres.append(Sphere(c, 3.0, mua=rng.uniform(0.02, 0.03),
                                  mus=2.0 if i == 0 else None))
        return Config(name, 11, L, _face_patches(L, 5.0, [(2, 1)]), spheres, seed=s)
    if name == "c1_cube64":
        s = 1000 if seed is None else seed
        rng = np.random.default_rng(s)
        L = 40.0
        spheres = _random_spheres(rng, L, 6, 3.0, 6.0)
        return Config(name, 64, L,
                      _face_patches(L, 10.0, [(2, 1), (2, 0), (0, 1), (0, 0)]),
                      spheres, seed=s)
    if name in ("c2_cube96", "c4_cube128"):
        s = (2000 if name == "c2_cube96" else 4000) if seed is None else seed
        L = 40.0
        n = 96 if name == "c2_cube96" else 128
        patches = _face_patches(L, 10.0, [(2, 1), (2, 0), (0, 1), (0, 0), (1, 1), (1, 0)])
        patches.append(Patch(2, 1, (L / 4, L / 4, L), 6.0))
        patches.append(Patch(2, 0, (3 * L / 4, 3 * L / 4, 0.0), 6.0))
        return Config(name, n, L, patches, [], blobs=True, seed=s)
    raise KeyError(name)


def small_config(n: int, L: float, K: int, seed: int) -> Config:
    """A small cube (used for parity at oracle-friendly sizes): `n` nodes per
    side, K face patches cycling top, bottom, +x, -x, +y, -y, two random
    spheres."""
    rng = np.random.default_rng(seed)
    spheres = _random_spheres(rng, L, 2, L / 8, L / 6)
    faces = [(2, 1), (2, 0), (0, 1), (0, 0), (1, 1), (1, 0)]
    patches = _face_patches(L, L / 4, [faces[k % 6] for k in range(K)])
    return Config(f"cube{n}_K{K}", n, L, patches, spheres, seed=seed)


def uneven_batch(count: int = 32, seed: int = 3000, nmin: int = 16, nmax: int = 48) -> List[Config]:
    """Independent problems of uneven size: cubes of n ~ U{nmin..nmax} nodes
    per side (L = 20 mm), K ~ U{1..4} face patches, 2-5 random spheres."""
    rng = np.random.default_rng(seed)
    faces = [(2, 1), (2, 0), (0, 1), (0, 0)]
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        K = int(rng.integers(1, 5))
        L = 20.0
        spheres = _random_spheres(rng, L, int(rng.integers(2, 6)), 2.0, 4.0)
        out.append(Config(f"batch{i}_n{n}_K{K}", n, L, _face_patches(L, 5.0, faces[:K]), spheres,
                          seed=seed + i))
    return out


# ---------------------------------------------------------------- Test 2 stand-in

TEST2_FACES = {"btm": (2, 0), "top": (2, 1), "rgt": (0, 1), "bck": (1, 1)}


def test2_phantom(xyz: np.ndarray, L: float = 11.0, half_thick: float = 0.5, half_width: float = 1.0):
    """Nodal (kappa, mu) of the Test 2 target of Sec. 5 on the cube [0, L]^3
    (the paper centres it at the origin; here centre = (L/2, L/2, L/2)).

    mu: background 0.015, a spherical shell 4 <= r <= 5 at 0.02, and a
    cross-shaped inclusion lying along the plane z = x at 0.01 (the cross
    wins where they meet).  kappa: background 0.3, a ball r <= 3 at 0.2, and
    a cross along the plane z = -x at 0.4 (the cross wins).  The paper shows
    the crosses only in figures; here a cross is a plus sign of two bars,
    half width `half_width`, lying in its plane (one along y, one along the
    in-plane diagonal, both through the centre and across the cube), with
    half thickness `half_thick` normal to the plane.
    """
    p = np.asarray(xyz, dtype=np.float64) - L / 2.0
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    r = np.sqrt(x * x + y * y + z * z)
    s2 = np.sqrt(2.0)

    def cross(normal_dist, inplane):
        return (np.abs(normal_dist) <= half_thick) & ((np.abs(inplane) <= half_width) | (np.abs(y) <= half_width))

    cross_mu = cross((z - x) / s2, (x + z) / s2)     # plane z = x
    cross_kappa = cross((z + x) / s2, (x - z) / s2)  # plane z = -x
    mu = np.full(p.shape[0], 0.015)
    mu[(r >= 4.0) & (r <= 5.0)] = 0.02
    mu[cross_mu] = 0.01
    kappa = np.full(p.shape[0], 0.3)
    kappa[r <= 3.0] = 0.2
    kappa[cross_kappa] = 0.4
    return kappa, mu


@dataclasses.dataclass
class Test2Config:
    """Test 2 of Sec. 5 on a Kuhn cube of n^3 nodes over [0, 11]^3 mm, lit
    through whole faces (characteristic functions, amplitude 1): any subset
    of btm (z = 0), top (z = L), rgt (x = L) and bck (y = L)."""
    n: int
    illum: Tuple[str, ...] = ("btm",)
    L: float = 11.0

    @property
    def name(self) -> str:
        return f"test2_n{self.n}_" + "+".join(self.illum)

    @property
    def N(self) -> int:
        return self.n ** 3

    @property
    def K(self) -> int:
        return len(self.illum)

    @property
    def patches(self) -> List[Patch]:
        return _face_patches(self.L, self.L / 2.0, [TEST2_FACES[f] for f in self.illum])

    def mesh(self):
        return kuhn_cube(self.n, self.L)

    def coefficients(self, xyz: np.ndarray):
        return test2_phantom(xyz, self.L)


def noise_draws(seed: int, shape) -> np.ndarray:
    """Standard normal draws for the measurement noise eta (Sec. 5, Test 1):
    chi = h + 0.01 |h| * xi with xi from here."""
    return np.random.default_rng(seed).standard_normal(shape)


def random_vector(seed: int, shape) -> np.ndarray:
    """Seeded standard-normal test vector."""
    return np.random.default_rng(seed).standard_normal(shape)


# ------------------------------------------------------------------ cylinder (Test 1 geometry)

def cylinder_mesh(n: int, nz: int, R: float, H: float) -> Tuple[np.ndarray, np.ndarray]:
    """Tetrahedral mesh of the cylinder {x^2 + y^2 <= R^2, 0 <= z <= H}.

    A Kuhn grid with n x n x nz nodes on [-1, 1]^2 x [0, H] is mapped onto
    the cylinder by sending each square ring max(|x|, |y|) = s to the circle
    of radius s R along rays from the axis: (x, y) -> R s (x, y) / |(x, y)|.
    The map is a homeomorphism, so the mesh stays conforming; tets take many
    shapes and the side is a polygonal approximation of the circle whose
    boundary nodes lie exactly at radius R.  Node and tet numbering follow
    the Kuhn grid (x fastest).  Orientation is left as generated.
    """
    if n < 3 or nz < 2:
        raise ValueError("cylinder_mesh needs n >= 3 and nz >= 2")
    g = np.linspace(-1.0, 1.0, n)
    gz = np.linspace(0.0, H, nz)
    zz, yy, xx = np.meshgrid(gz, g, g, indexing="ij")
    x, y = xx.ravel(), yy.ravel()
    s = np.maximum(np.abs(x), np.abs(y))
    rho = np.hypot(x, y)
    f = np.where(rho > 0, s / np.where(rho > 0, rho, 1.0), 0.0) * R
    xyz = np.stack([x * f, y * f, zz.ravel()], axis=1)
    m, mz = n - 1, nz - 1
    kk, jj, ii = np.meshgrid(np.arange(mz), np.arange(m), np.arange(m), indexing="ij")
    base = (ii + n * (jj + n * kk)).ravel().astype(np.int64)
    stride = np.array([1, n, n * n], dtype=np.int64)
    tets = []
    for perm in itertools.permutations(range(3)):
        a, b, _ = perm
        v1 = base + stride[a]
        tets.append(np.stack([base, v1, v1 + stride[b], base + stride.sum()], axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4)
    return xyz, tets.astype(np.int32)


@dataclasses.dataclass
class SideIllumination:
    """Photon flux through the curved side of the cylinder (Sec. 5, Test 1):
    homogeneous along the axis, centred at polar angle theta0, non-zero for
    |theta - theta0| <= half_w with amplitude amp cos(pi/2 (theta - theta0) /
    half_w) (half_w = pi/8 gives the paper's cos(4 (theta - theta0))).  The
    polar angle is measured about `axis` through `center`, from `ref`."""
    theta0: float
    half_w: float = np.pi / 8
    amp: float = 1.0
    center: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    axis: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    ref: Tuple[float, float, float] = (1.0, 0.0, 0.0)


@dataclasses.dataclass
class CylinderConfig:
    name: str
    n: int
    nz: int
    R: float
    H: float
    illuminations: List[SideIllumination]
    spheres: List[Sphere]
    mua_bg: float = 0.01
    mus_bg: float = 1.0
    seed: int = 0

    @property
    def N(self) -> int:
        return self.n * self.n * self.nz

    @property
    def K(self) -> int:
        return len(self.illuminations)

    def mesh(self):
        return cylinder_mesh(self.n, self.nz, self.R, self.H)

    def optics(self, xyz: np.ndarray):
        return spheres_phantom(xyz, self.spheres, self.mua_bg, self.mus_bg)

    def coefficients(self, xyz: np.ndarray):
        mua, mus = self.optics(xyz)
        return kappa_from_optics(mua, mus), mua


def cylinder_config(n: int, nz: int, R: float, H: float, K: int, seed: int) -> CylinderConfig:
    """Test 1 stand-in: cylinder of radius R and height H, K side
    illuminations at theta0 = (k - 1) pi / 2 (k = 1..K, cycling), two random
    spherical inclusions inside radius R/2 (the paper's Test 1 targets are
    not available)."""
    rng = np.random.default_rng(seed)
    spheres = []
    for i in range(2):
        r0 = rng.uniform(0.0, 0.5 * R)
        t0 = rng.uniform(0.0, 2 * np.pi)
        c = (r0 * np.cos(t0), r0 * np.sin(t0), rng.uniform(0.3 * H, 0.7 * H))
        spheres.append(Sphere(c, rng.uniform(0.15, 0.25) * R, mua=rng.uniform(0.02, 0.03),
                              mus=2.0 if i == 0 else None))
    ill = [SideIllumination(theta0=(k % 4) * np.pi / 2) for k in range(K)]
    return CylinderConfig(f"cyl{n}x{nz}_K{K}", n, nz, R, H, ill, spheres, seed=seed)


# ------------------------------------------------------------------ several wavelengths

def wavelength_optics(cfg, xyz: np.ndarray, wavelengths_nm: Sequence[float], seed: int = 0):
    """Nodal (kappa, mu) of the phantom at several wavelengths (the paper's
    remark that the extension to multiple wavelengths is straightforward):
    absorption mu_a(x) scaled by a seeded smooth spectrum per wavelength
    (factors in [0.5, 1.5]), reduced scattering mu_s'(x) following the
    usual power law (lambda / 800 nm)^(-1.2).  Returns a list of (kappa, mu)
    pairs, one per wavelength."""
    rng = np.random.default_rng(seed)
    mua, mus = cfg.optics(xyz)
    c = rng.uniform(0.0, 2 * np.pi, size=2)
    out = []
    for lam in wavelengths_nm:
        a = 1.0 + 0.5 * np.sin(c[0] + lam / 60.0) * np.cos(c[1] + lam / 170.0)
        s = (lam / 800.0) ** (-1.2)
        mua_l, mus_l = mua * a, mus * s
        out.append((kappa_from_optics(mua_l, mus_l), mua_l))
    return out
