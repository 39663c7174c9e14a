"""Shared helpers of the GPU parity tests (inputs come from qpat_synth; the
expected values from the oracle)."""
import numpy as np

import oracle as O
import qpat_synth as S


class Case:
    """A synthetic linearisation point: mesh, coefficients, fluxes, forward
    solution and whitening weights, all from the oracle on the CPU."""

    def __init__(self, cfg, patch_nodes=512, solve=True):
        self.cfg = cfg
        self.xyz, self.tets = cfg.mesh()
        self.om = O.Mesh(self.xyz, self.tets)
        self.kappa, self.mu = cfg.coefficients(self.xyz)
        if hasattr(cfg, "illuminations"):     # cylinder: curved-side fluxes (Test 1)
            self.flux = np.stack([O.flux_side(self.om, il.center, il.axis, il.ref, cfg.R, il.theta0, il.half_w,
                                              il.amp) for il in cfg.illuminations])
        else:
            self.flux = np.stack([O.flux_patch(self.om, p.center, p.normal, p.half_w, p.amp)
                                  for p in cfg.patches])
        self.K = self.flux.shape[0]
        self.N = self.om.N
        self.patch_nodes = patch_nodes
        self.Kmat = O.system_matrix(self.om, self.kappa, self.mu)
        if solve:
            self.fac = O.Factor(self.Kmat)
            self.phi, self.h = O.forward(self.om, self.kappa, self.mu, self.flux, self.fac)
            rng = np.random.default_rng(cfg.seed + 17)
            self.w = 1.0 / (0.01 * np.abs(self.h) + 1e-3 * np.abs(self.h).max())
            self.w *= rng.uniform(0.9, 1.1, self.w.shape)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def small_cases():
    return {
        "tiny_n2": S.small_config(2, 1.0, 1, 1),
        "cube9_K3": S.small_config(9, 10.0, 3, 2),
        "c0_cube11": S.config("c0_cube11"),
        "cube13_K5": S.small_config(13, 12.0, 5, 3),
        "cyl9x6_K4": S.cylinder_config(9, 6, 10.0, 8.0, 4, 21),
    }
