"""Uneven batch: forward solves of meshes of different sizes (and different
illumination counts) in one cooperative launch replayed as a CUDA graph,
against the per-mesh entry point and the oracle."""
import numpy as np
import pytest

import oracle as O
import qpat_synth as S
from tests.gpu_common import rel

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu

SIZES = [(5, 1), (9, 3), (12, 2), (7, 4), (16, 1), (10, 4), (13, 3)]


@pytest.mark.parametrize("deg", [0, 2])
def test_uneven_batch_matches_single_solves(deg):
    """Jacobi (deg 0) or the patch-local Chebyshev preconditioner in the
    batched launch: every problem equals its single-mesh solve and the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfgs = [S.small_config(n, 2.0 * n, K, 100 + i) for i, (n, K) in enumerate(SIZES)]
    meshes, data = [], []
    for cfg in cfgs:
        xyz, tets = cfg.mesh()
        kap, mu = cfg.coefficients(xyz)
        m = Q.qpat_mesh(xyz, tets, patch_nodes=64)
        flux = np.stack([Q.qpat_flux_patch(m, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
        meshes.append(m)
        data.append((xyz, tets, kap, mu, flux))
    batch = Q.qpat_batch_create(meshes, [c.K for c in cfgs], Q.qpat_default_params(poly_degree=deg))
    try:
        for rep in range(3):
            scale = 1.0 + 0.1 * rep          # new inputs on every replay of the same graph
            for j, (xyz, tets, kap, mu, flux) in enumerate(data):
                k, m_, f = batch.inputs(j)
                k.copy_(torch.tensor(kap * scale))
                m_.copy_(torch.tensor(mu))
                f.copy_(torch.tensor(flux))
            batch.forward()
            torch.cuda.synchronize()
            st, it, ct = batch.status()
            assert all(s == 0 for s in st), st
            assert all(c >= 1 for c in ct)
            for j, (xyz, tets, kap, mu, flux) in enumerate(data):
                ref, _ = Q.qpat_forward(meshes[j], kap * scale, mu, flux)
                assert rel(batch.phi(j).cpu().numpy(), ref) < 1e-10
                if rep == 0 and j < 3:
                    om = O.Mesh(xyz, tets)
                    phi_o, _ = O.forward(om, kap, mu, flux)
                    assert rel(batch.phi(j).cpu().numpy(), phi_o) < 1e-10
    finally:
        batch.close()
        for m in meshes:
            m.close()


def test_autotune_picks_a_measured_candidate():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = S.small_config(20, 20.0, 4, 7)
    xyz, tets = cfg.mesh()
    kap, mu = cfg.coefficients(xyz)
    (pn, op), table = Q.qpat_autotune(xyz, tets, kap, mu, 4, iters=20)
    finite = {k: v for k, v in table.items() if np.isfinite(v)}
    assert len(finite) >= 6
    assert (pn, op) in finite and finite[(pn, op)] == min(finite.values())


def test_several_wavelengths_on_one_mesh_in_one_launch():
    """Several wavelengths (independent optical problems on one mesh, the
    paper's straightforward extension) as one batched launch: the same mesh
    handle once per wavelength, each solve equal to its own FP64 forward and,
    for one wavelength, to the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = S.small_config(12, 20.0, 3, 41)
    xyz, tets = cfg.mesh()
    lams = [700.0, 760.0, 830.0, 900.0]
    optics = S.wavelength_optics(cfg, xyz, lams, seed=5)
    m = Q.qpat_mesh(xyz, tets, patch_nodes=64)
    flux = np.stack([Q.qpat_flux_patch(m, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
    batch = Q.qpat_batch_create([m] * len(lams), [cfg.K] * len(lams))
    try:
        for j, (kap, mu) in enumerate(optics):
            k, m_, f = batch.inputs(j)
            k.copy_(torch.tensor(kap))
            m_.copy_(torch.tensor(mu))
            f.copy_(torch.tensor(flux))
        batch.forward()
        torch.cuda.synchronize()
        st, _, _ = batch.status()
        assert all(s == 0 for s in st), st
        phis = [batch.phi(j).cpu().numpy() for j in range(len(lams))]
        for j, (kap, mu) in enumerate(optics):
            ref, _ = Q.qpat_forward(m, kap, mu, flux)
            assert rel(phis[j], ref) < 1e-10
        om = O.Mesh(xyz, tets)
        phi_o, _ = O.forward(om, optics[2][0], optics[2][1], flux)
        assert rel(phis[2], phi_o) < 1e-10
        # the wavelengths really differ
        assert rel(phis[0], phis[3]) > 1e-3
    finally:
        batch.close()
        m.close()


def test_concurrent_reconstructions_match_sequential():
    """Independent reconstructions (Algorithm 1) on meshes of different sizes
    run concurrently, one host thread and one mesh stream each (the library
    call releases the interpreter), give bit for bit the results of the same
    reconstructions run one after the other: every device sum has a fixed
    order, whatever else runs on the GPU."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from concurrent.futures import ThreadPoolExecutor
    probs = []
    for i, (n, K) in enumerate([(7, 1), (9, 2), (11, 3), (8, 4)]):
        cfg = S.small_config(n, 2.0 * n, K, 300 + i)
        xyz, tets = cfg.mesh()
        kap, mu = cfg.coefficients(xyz)
        m = Q.qpat_mesh(xyz, tets, patch_nodes=64)
        flux = np.stack([Q.qpat_flux_patch(m, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
        _, h = Q.qpat_forward(m, kap, mu, flux)
        sig = 0.01 * np.abs(h) + 1e-3 * np.abs(h).max()
        chi = h + sig * S.noise_draws(40 + i, h.shape)
        probs.append((m, flux, chi, sig, (float(np.median(kap)), float(np.median(mu)))))
    prm = Q.qpat_default_params(T=1e-2, max_lin=3, max_lsqr=6, fixed_counts=1)
    run = lambda p: Q.qpat_reconstruct(p[0], p[1], p[2], p[3], prm, p[4])
    try:
        seq = [run(p) for p in probs]
        with ThreadPoolExecutor(max_workers=4) as ex:
            con = list(ex.map(run, probs))
        for (ks, ms, rs), (kc, mc, rc) in zip(seq, con):
            np.testing.assert_array_equal(kc, ks)
            np.testing.assert_array_equal(mc, ms)
            assert rc.linearisations == rs.linearisations
    finally:
        for p in probs:
            p[0].close()
