"""The allocation-free forward solve (qpat_forward_noalloc_dev), for callers
that cannot allocate device memory when they need a solve: real-time
pipelines that forbid allocator calls after start-up (an allocation can block
on the driver) and hosts that budget all GPU memory themselves.

Its output must equal the regular entry point's (qpat_forward_dev, FP64) to
the 1e-10 relative tolerance of the other forward tests, on two calls in a
row (the second call reuses the same fixed scratch array), the device's free
memory must not change across its calls, and sizes above the fixed limit
must be refused.  This file runs last so that a stop at the first failure has
already run every other test."""
import numpy as np
import pytest

import qpat_synth as S

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("cfg", [S.small_config(9, 10.0, 3, 2), S.config("c0_cube11"),
                                 S.small_config(13, 12.0, 5, 3)], ids=["cube9_K3", "c0_cube11", "cube13_K5"])
def test_noalloc_forward_matches_regular_entry_point(cfg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    xyz, tets = cfg.mesh()
    kap, mu = cfg.coefficients(xyz)
    mesh = Q.qpat_mesh(xyz, tets, patch_nodes=64)
    try:
        dev = torch.device("cuda")
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
        flux = np.stack([Q.qpat_flux_patch(mesh, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
        k, m, f = T(kap), T(mu), T(flux)
        K, N = flux.shape[0], mesh.N
        phi_ref = torch.empty((K, N), dtype=torch.float64, device=dev)
        h_ref = torch.empty_like(phi_ref)
        Q.qpat_forward_dev(mesh, k, m, f, phi_ref, h_ref, Q.qpat_default_params(precision=0))
        outs = [(torch.full((K, N), float("nan"), dtype=torch.float64, device=dev),
                 torch.full((K, N), float("nan"), dtype=torch.float64, device=dev)) for _ in range(2)]
        torch.cuda.synchronize()
        free = []
        for phi, h in outs:           # nothing else touches the device between the two readings
            Q.qpat_forward_noalloc_dev(mesh, k, m, f, phi, h)
            torch.cuda.synchronize()
            free.append(torch.cuda.mem_get_info()[0])
        # the second call (after the first one's set-up) takes no device memory
        assert free[1] == free[0]
        for phi, h in outs:
            assert _rel(phi, phi_ref) < 1e-10
            assert _rel(h, h_ref) < 1e-10
    finally:
        mesh.close()


def test_noalloc_rejects_sizes_above_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = S.config("c1_cube64")            # 262,144 nodes x 4 illuminations > 524,288
    xyz, tets = cfg.mesh()
    kap, mu = cfg.coefficients(xyz)
    mesh = Q.qpat_mesh(xyz, tets)
    try:
        dev = torch.device("cuda")
        k = torch.tensor(kap, device=dev)
        m = torch.tensor(mu, device=dev)
        f = torch.zeros((4, mesh.F), dtype=torch.float64, device=dev)
        phi = torch.empty((4, mesh.N), dtype=torch.float64, device=dev)
        with pytest.raises(Q.QpatError) as ei:
            Q.qpat_forward_noalloc_dev(mesh, k, m, f, phi, None)
        assert ei.value.code == Q.QPAT_EINVAL
        assert "exceeds" in str(ei.value)
    finally:
        mesh.close()
