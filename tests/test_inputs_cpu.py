"""Seeded synthetic inputs: the Test 2 stand-in target and its illuminations
(Sec. 5, Test 2), checked against the values and supports the paper states."""
import numpy as np
import pytest

import oracle as O
import qpat_synth as S


@pytest.mark.parametrize("pt,kappa,mu", [
    ((0.0, 0.0, 0.0), 0.4, 0.01),       # centre: both crosses (the crosses win)
    ((2.0, 0.0, 0.0), 0.2, 0.015),      # inside the kappa ball, off both cross planes
    ((4.5, 0.0, 0.0), 0.3, 0.02),       # in the mu shell 4 <= r <= 5
    ((2.0, 0.0, 2.0), 0.2, 0.01),       # on the plane z = x (mu cross), in the kappa ball
    ((2.0, 0.0, -2.0), 0.4, 0.015),     # on the plane z = -x (kappa cross)
    ((3.0, 3.0, -3.0), 0.3, 0.015),     # on z = -x but outside both bars of the cross
    ((5.0, 5.0, 5.0), 0.3, 0.015),      # background corner
])
def test_test2_phantom_values(pt, kappa, mu):
    L = 11.0
    xyz = np.asarray([pt]) + L / 2.0
    k, m = S.test2_phantom(xyz, L)
    assert k[0] == kappa and m[0] == mu


def test_test2_levels_and_supports():
    cfg = S.Test2Config(21, ("btm", "rgt", "top", "bck"))
    xyz, _ = cfg.mesh()
    k, m = cfg.coefficients(xyz)
    assert set(np.unique(k)) == {0.2, 0.3, 0.4}
    assert set(np.unique(m)) == {0.01, 0.015, 0.02}
    # the two crosses are mirror images under x -> -x (about the centre)
    mirror = xyz.copy()
    mirror[:, 0] = cfg.L - mirror[:, 0]
    km, mm = cfg.coefficients(mirror)
    np.testing.assert_array_equal(k == 0.4, mm == 0.01)


@pytest.mark.parametrize("faces", [("btm",), ("btm", "rgt"), ("btm", "top", "bck")])
def test_test2_whole_face_illuminations(faces):
    """Each illumination is the characteristic function of one whole face:
    all 2 (n-1)^2 boundary triangles of that face, amplitude 1, nothing else."""
    cfg = S.Test2Config(6, faces)
    xyz, tets = cfg.mesh()
    om = O.Mesh(xyz, tets)
    for f, p in zip(faces, cfg.patches):
        phi = O.flux_patch(om, p.center, p.normal, p.half_w, p.amp)
        axis, side = S.TEST2_FACES[f]
        on_face = np.all(np.isclose(om.xyz[om.faces][:, :, axis], side * cfg.L), axis=1)
        np.testing.assert_array_equal(phi != 0, on_face)
        assert np.count_nonzero(phi) == 2 * (cfg.n - 1) ** 2
        assert np.all(phi[phi != 0] == 1.0)
