"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point declared in include/qpat.h, and its host mesh preparation
(boundary faces in canonical order, locality permutation, CTA patches)
agrees with the oracle's mesh processing.  No GPU compute is called."""
import os
import re

import numpy as np
import pytest

import oracle as O
import qpat_synth as S
import paper_1512_02796_gb300 as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "qpat.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qpat_[A-Za-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = Q.load()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(Q.exported_names()) == set(names)


def test_default_params_follow_the_paper():
    p = Q.qpat_default_params()
    assert p.T == 5e-3 and p.delta == 1e-6 and p.b_over_a == 1.0
    assert p.m0 == 10 and p.tau == 1e-2
    # library choices, not the paper's: degree-2 patch-local Chebyshev preconditioners
    assert p.poly_degree == 2 and p.prior_poly_degree == 2


@pytest.mark.parametrize("n,L,pn", [(2, 1.0, 32), (5, 2.0, 32), (11, 20.0, 64), (11, 20.0, 512), (17, 4.0, 96)])
def test_host_mesh_faces_match_oracle_and_patches_verify(n, L, pn):
    xyz, tets = S.kuhn_cube(n, L)
    info, faces, perm = Q.qpat_mesh_host_info(xyz, tets, pn)
    of = O.boundary_faces(tets)
    assert info["F"] == of.shape[0] == 12 * (n - 1) ** 2
    np.testing.assert_array_equal(faces, of)
    assert np.array_equal(np.sort(perm), np.arange(n ** 3))
    assert info["P"] == -(-n ** 3 // pn)
    assert info["patch_tets"] >= 6 * (n - 1) ** 3
    assert info["max_own"] <= pn + 32     # balanced whole 32-node slices
    # element colours (checked inside: no two tets of a colour share an owned
    # node): at least the 6 tets around the cube diagonal, at least the 24 around
    # an interior node once a patch owns one, few enough for one barrier each
    assert 6 <= info["max_tet_colours"] <= 64
    if n >= 5:
        assert info["max_tet_colours"] >= 24


@pytest.mark.parametrize("n,nz,pn", [(5, 4, 32), (9, 6, 64), (17, 9, 256)])
def test_host_mesh_cylinder_faces_match_oracle_and_patches_verify(n, nz, pn):
    """The mapped cylinder (Test 1 geometry): tets of many shapes, a curved
    side; the host preparation (faces, order, patches, assembled pattern) is
    checked by the library's structure validator and against the oracle."""
    xyz, tets = S.cylinder_mesh(n, nz, 10.0, 8.0)
    info, faces, perm = Q.qpat_mesh_host_info(xyz, tets, pn)
    of = O.boundary_faces(tets)
    np.testing.assert_array_equal(faces, of)
    assert info["F"] == of.shape[0] == 4 * (n - 1) * (nz - 1) * 2 + 2 * 2 * (n - 1) ** 2
    assert np.array_equal(np.sort(perm), np.arange(xyz.shape[0]))
    assert info["max_own"] <= pn + 32


def test_prior_stiffness_pattern_drops_exact_zero_couplings():
    """Kuhn tets couple their face- and body-diagonal edges with exactly zero
    gradient product, so the prior's stiffness pattern keeps the 7-point
    stencil (6 neighbours + diagonal per interior row) of the 15-entry full
    pattern; the counts match the oracle's assembled matrices (the dense
    brute-force check of which zeros are exact)."""
    n = 6
    xyz, tets = S.kuhn_cube(n, 5.0)
    info, _, _ = Q.qpat_mesh_host_info(xyz, tets, 64)
    m = O.Mesh(xyz, tets)
    Kfull = O.system_matrix(m, np.ones(m.N), np.ones(m.N))
    Mstiff = O.assemble_stiffness(m, np.ones(m.E)).tocsr()
    Mstiff.data[np.abs(Mstiff.data) < 1e-12 * np.abs(Mstiff.data).max()] = 0.0
    Mstiff.eliminate_zeros()
    assert info["nnz"] == Kfull.nnz
    assert info["prior_nnz"] == Mstiff.nnz == 7 * n ** 3 - 6 * n * n
    # on the mapped cylinder the pattern is a subset (checked by the library) and
    # keeps every coupling the oracle's stiffness has
    xyz, tets = S.cylinder_mesh(7, 5, 10.0, 8.0)
    info, _, _ = Q.qpat_mesh_host_info(xyz, tets, 64)
    m = O.Mesh(xyz, tets)
    Ms = O.assemble_stiffness(m, np.ones(m.E)).tocsr()
    Ms.data[np.abs(Ms.data) < 1e-12 * np.abs(Ms.data).max()] = 0.0
    Ms.eliminate_zeros()
    assert info["prior_nnz"] >= Ms.nnz


def test_host_mesh_random_relabelled_mesh():
    """Faces are canonical in caller ids whatever the node numbering and tet
    orientation."""
    xyz, tets = S.kuhn_cube(6, 3.0)
    rng = np.random.default_rng(0)
    p = rng.permutation(xyz.shape[0])
    inv = np.argsort(p)
    xyz2 = xyz[p]
    tets2 = inv[tets]
    for e in range(tets2.shape[0]):
        tets2[e] = tets2[e][rng.permutation(4)]
    info, faces, _ = Q.qpat_mesh_host_info(xyz2, tets2.astype(np.int32), 64)
    np.testing.assert_array_equal(faces, O.boundary_faces(tets2))


def test_host_mesh_rejects_bad_input():
    xyz, tets = S.kuhn_cube(3, 1.0)
    bad = tets.copy()
    bad[0, 0] = xyz.shape[0]
    with pytest.raises(Q.QpatError):
        Q.qpat_mesh_host_info(xyz, bad, 32)
    flat = tets.copy()
    flat[0] = [0, 1, 2, 2]        # degenerate tet
    with pytest.raises(Q.QpatError):
        Q.qpat_mesh_host_info(xyz, flat, 32)
    with pytest.raises(Q.QpatError):
        Q.qpat_mesh_host_info(xyz, tets, 8)   # patch size below the minimum


def test_launch_counter_is_callable_without_a_gpu():
    # a host-side counter: no kernel has been launched by the CPU test process
    assert Q.qpat_launch_count() >= 0


def test_params_struct_layout_matches_the_header():
    """The ctypes mirror of qpat_params has the C struct's size: the library's
    qpat_default_params clears exactly sizeof(qpat_params) bytes (memset
    first), so with a guard area behind the mirror's size the last byte of
    the struct is written and the guard is left alone."""
    import ctypes
    n = ctypes.sizeof(Q.qpat_params)
    buf = (ctypes.c_ubyte * (n + 32))(*([0xAB] * (n + 32)))
    Q.load().qpat_default_params(ctypes.cast(buf, ctypes.POINTER(Q.qpat_params)))
    import struct
    assert bytes(buf[n - 8:n]) == struct.pack("<d", 30.0)   # mg_ratio, the last field
    assert all(b == 0xAB for b in buf[n:])
    p = Q.qpat_default_params()
    assert p.lsqr_reorth == 1 and p.barrier_spin_limit == 0
    assert p.multigrid == 0 and p.mg_degree == 1 and p.mg_ratio == 30.0


def test_host_output_arrays_are_checked_before_any_call():
    """Caller-supplied host outputs (e.g. pinned buffers) must be contiguous,
    writable float64 of the right shape; the binding refuses others before it
    reaches the library."""
    import types
    m = types.SimpleNamespace(N=4, handle=None)
    x = np.zeros(4)
    for bad in (np.empty(7), np.empty(8, dtype=np.float32), np.empty(16)[::2]):
        with pytest.raises(ValueError):
            Q.qpat_prior_solve(m, x, x, np.zeros(8), out=bad)
    ro = np.empty(8)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        Q.qpat_prior_solve(m, x, x, np.zeros(8), out=ro)
    phi = np.ones((2, 4))
    with pytest.raises(ValueError):
        Q.qpat_jvp_vjp_pair(m, x, x, phi, np.zeros(8), phi, None, out_jv=np.empty((3, 4)), out_vjp=np.empty(8))
    with pytest.raises(ValueError):
        Q.qpat_jvp_vjp_pair(m, x, x, phi, np.zeros(8), phi, None, out_jv=np.empty((2, 4)), out_vjp=np.empty(4))


@pytest.mark.parametrize("n,prior", [(6, 0), (11, 0), (11, 1), (17, 0), (17, 1), (24, 1)])
def test_multigrid_plan_invariants_on_cubes(n, prior):
    """The smoothed-aggregation plan (aggregates, P, R = P^T, the slots of
    A P and P^T A P, symmetric coarse patterns) passes the library's own
    invariant check, coarsens by a clear factor per level and ends at <= 128
    rows."""
    xyz, tets = S.kuhn_cube(n, 10.0)
    rows = Q.qpat_multigrid_host_info(xyz, tets, prior=bool(prior))
    assert rows[0] == n ** 3
    assert rows[-1] <= 128
    for a, b in zip(rows, rows[1:]):
        assert b <= a / 4


def test_multigrid_plan_on_cylinder_and_tiny_meshes():
    xyz, tets = S.cylinder_mesh(9, 6, 5.0, 10.0)
    for prior in (False, True):
        rows = Q.qpat_multigrid_host_info(xyz, tets, prior=prior)
        assert rows[0] == xyz.shape[0] and rows[-1] <= 128
    xyz, tets = S.kuhn_cube(3, 1.0)          # 27 nodes: the fine level is the coarsest
    assert Q.qpat_multigrid_host_info(xyz, tets) == [27]


def test_multigrid_plan_independent_of_caller_numbering():
    """The library reorders nodes itself (Morton order), so the multigrid plan
    of a randomly relabelled mesh with shuffled tet vertices has the same
    level sizes as the original, and passes the same invariant checks."""
    xyz, tets = S.kuhn_cube(14, 5.0)
    rng = np.random.default_rng(4)
    p = rng.permutation(xyz.shape[0])
    inv = np.argsort(p)
    tets2 = inv[tets]
    for e in range(tets2.shape[0]):
        tets2[e] = tets2[e][rng.permutation(4)]
    for prior in (False, True):
        a = Q.qpat_multigrid_host_info(xyz, tets, prior=prior)
        b = Q.qpat_multigrid_host_info(xyz[p], tets2.astype(np.int32), prior=prior)
        assert a == b and a[-1] <= 128 and len(a) >= 2
