"""Thin Python binding of the C ABI in include/qpat.h (argument marshalling only).

Every function keeps the C name.  Host-pointer calls take numpy arrays and
return numpy arrays; `*_dev` calls take CUDA torch tensors (float64,
contiguous) and run on the current torch stream.  All computation happens in
libqpat.so; there is no fallback: a missing library or a failing call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int32_p = ctypes.POINTER(ctypes.c_int32)
_c_int64_p = ctypes.POINTER(ctypes.c_int64)

QPAT_OK, QPAT_EINVAL, QPAT_ENOCONV, QPAT_EBREAKDOWN, QPAT_ETIMEOUT, QPAT_ECUDA, QPAT_ENOMEM = 0, -1, -2, -3, -4, -5, -6


class qpat_params(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_double), ("b_over_a", ctypes.c_double), ("delta", ctypes.c_double),
        ("tau", ctypes.c_double), ("m0", ctypes.c_int), ("max_lin", ctypes.c_int),
        ("max_lsqr", ctypes.c_int), ("fixed_counts", ctypes.c_int), ("precision", ctypes.c_int),
        ("max_pcg_iter", ctypes.c_int), ("pcg_rtol", ctypes.c_double), ("fit_grid", ctypes.c_int),
        ("fit_gn_steps", ctypes.c_int), ("patch_nodes", ctypes.c_int), ("fp32_operator", ctypes.c_int),
        ("pcg_variant", ctypes.c_int), ("prior", ctypes.c_int), ("mixed_restart", ctypes.c_int),
        ("poly_degree", ctypes.c_int), ("prior_poly_degree", ctypes.c_int), ("step_halvings", ctypes.c_int),
        ("prior_q", ctypes.c_double), ("lsqr_reorth", ctypes.c_int), ("barrier_spin_limit", ctypes.c_int64),
        ("multigrid", ctypes.c_int), ("mg_degree", ctypes.c_int), ("mg_ratio", ctypes.c_double),
    ]


class qpat_report(ctypes.Structure):
    _fields_ = [
        ("kappa0", ctypes.c_double), ("mu0", ctypes.c_double), ("linearisations", ctypes.c_int),
        ("accepted_last", ctypes.c_int), ("lsqr_iters", ctypes.c_int * 32),
        ("residuals", ctypes.c_double * 33), ("pcg_iters", ctypes.c_int64), ("solves", ctypes.c_int64),
        ("refinements", ctypes.c_int64), ("ms_total", ctypes.c_double),
    ]


class QpatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qpat error {code}: {msg}")
        self.code = code


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libqpat.so (building it first if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libqpat.so not built at {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    sig = {
        "qpat_default_params": (None, [ctypes.POINTER(qpat_params)]),
        "qpat_last_error": (ctypes.c_char_p, []),
        "qpat_launch_count": (ctypes.c_int64, []),
        "qpat_mesh": (ctypes.c_int, [_c_double_p, ctypes.c_int64, _c_int32_p, ctypes.c_int64, ctypes.POINTER(vp)]),
        "qpat_mesh_ex": (ctypes.c_int, [_c_double_p, ctypes.c_int64, _c_int32_p, ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(vp)]),
        "qpat_mesh_free": (None, [vp]),
        "qpat_mesh_host_info": (ctypes.c_int, [_c_double_p, ctypes.c_int64, _c_int32_p, ctypes.c_int64,
                                               ctypes.c_int, _c_int64_p, _c_int32_p, _c_int32_p]),
        "qpat_mesh_num_nodes": (ctypes.c_int64, [vp]),
        "qpat_mesh_num_tets": (ctypes.c_int64, [vp]),
        "qpat_mesh_num_faces": (ctypes.c_int64, [vp]),
        "qpat_mesh_num_patches": (ctypes.c_int64, [vp]),
        "qpat_mesh_num_entries": (ctypes.c_int64, [vp]),
        "qpat_mesh_num_prior_entries": (ctypes.c_int64, [vp]),
        "qpat_mesh_num_local_entries": (ctypes.c_int64, [vp, ctypes.c_int]),
        "qpat_mesh_faces": (ctypes.c_int, [vp, _c_int32_p]),
        "qpat_mesh_permutation": (ctypes.c_int, [vp, _c_int32_p]),
        "qpat_mesh_stats": (ctypes.c_int, [vp, _c_int64_p]),
        "qpat_mesh_fp64_fallbacks": (ctypes.c_int64, [vp]),
        "qpat_mesh_rhs_iterations": (ctypes.c_int64, [vp]),
        "qpat_mesh_multigrid_levels": (ctypes.c_int, [vp, ctypes.c_int, _c_int64_p, ctypes.c_int]),
        "qpat_mesh_multigrid_fine_time": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), _c_int64_p]),
        "qpat_multigrid_host_info": (ctypes.c_int, [_c_double_p, ctypes.c_int64, _c_int32_p, ctypes.c_int64, ctypes.c_int,
                                                    ctypes.c_int, _c_int64_p, ctypes.c_int]),
        "qpat_mesh_reset_stats": (ctypes.c_int, [vp]),
        "qpat_mesh_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "qpat_mesh_pcg_time": (ctypes.c_int, [vp, _c_double_p]),
        "qpat_flux_side": (ctypes.c_int, [vp, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, _c_double_p]),
        "qpat_flux_patch": (ctypes.c_int, [vp, _c_double_p, _c_double_p, ctypes.c_double, ctypes.c_double,
                                           _c_double_p]),
        "qpat_apply_K_dev": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp, vp]),
        "qpat_forward": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), _c_double_p, _c_double_p, ctypes.c_int,
                                        _c_double_p, _c_double_p, _c_double_p]),
        "qpat_forward_dev": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), vp, vp, ctypes.c_int, vp, vp, vp, vp]),
        "qpat_forward_noalloc_dev": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, ctypes.c_double, ctypes.c_int,
                                                    vp, vp, vp]),
        "qpat_forward_guess_dev": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), vp, vp, ctypes.c_int, vp, vp,
                                                  vp, vp, vp]),
        "qpat_jvp": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), _c_double_p, _c_double_p, ctypes.c_int,
                                    _c_double_p, _c_double_p, _c_double_p, _c_double_p]),
        "qpat_jvp_dev": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), vp, vp, ctypes.c_int, vp, vp, vp, vp, vp]),
        "qpat_vjp": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), _c_double_p, _c_double_p, ctypes.c_int,
                                    _c_double_p, _c_double_p, _c_double_p, _c_double_p]),
        "qpat_vjp_dev": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), vp, vp, ctypes.c_int, vp, vp, vp, vp, vp]),
        "qpat_jvp_vjp_pair_dev": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), vp, vp, ctypes.c_int, vp, vp, vp,
                                                 vp, vp, vp, vp]),
        "qpat_jvp_vjp_pair": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), _c_double_p, _c_double_p, ctypes.c_int,
                                             _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                             _c_double_p]),
        "qpat_prior_solve": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), _c_double_p, _c_double_p, _c_double_p,
                                            _c_double_p]),
        "qpat_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(qpat_params), ctypes.POINTER(vp)]),
        "qpat_batch_buffers": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                              ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "qpat_batch_forward": (ctypes.c_int, [vp, vp]),
        "qpat_batch_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]),
        "qpat_batch_free": (None, [vp]),
        "qpat_unet_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(vp)]),
        "qpat_unet_free": (None, [vp]),
        "qpat_unet_num_params": (ctypes.c_int64, [vp]),
        "qpat_unet_get_params": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "qpat_unet_set_params": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "qpat_unet_features_dev": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, ctypes.c_double, vp, vp]),
        "qpat_unet_predict_dev": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp]),
        "qpat_unet_train_dev": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_float,
                                               ctypes.POINTER(ctypes.c_float), vp]),
        "qpat_unet_set_log_output": (ctypes.c_int, [vp, ctypes.c_double]),
        "qpat_unet_grad_dev": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(ctypes.c_float), vp]),
        "qpat_unet_to_double_dev": (ctypes.c_int, [vp, ctypes.c_int64, vp, vp]),
        "qpat_conv3d_bf16_dev": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                vp, vp, vp]),
        "qpat_conv3d_bf16_wgrad_dev": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                                      vp]),
        "qpat_conv3d_bf16_wgrad_scratch": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "qpat_conv3d_set_engine": (ctypes.c_int, [ctypes.c_int]),
        "qpat_conv3d_tc_timeouts": (ctypes.c_int, []),
        "qpat_autotune": (ctypes.c_int, [_c_double_p, ctypes.c_int64, _c_int32_p, ctypes.c_int64, _c_double_p,
                                         _c_double_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), _c_double_p, ctypes.POINTER(ctypes.c_int)]),
        "qpat_prior_solve_dev": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), vp, vp, vp, vp, vp]),
        "qpat_reconstruct": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), ctypes.c_int, _c_double_p,
                                            _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                            ctypes.POINTER(qpat_report)]),
        "qpat_reconstruct_ex": (ctypes.c_int, [vp, ctypes.POINTER(qpat_params), ctypes.c_int, _c_double_p,
                                               _c_double_p, _c_double_p, _c_double_p, _c_double_p, ctypes.c_int,
                                               _c_double_p, _c_double_p, _c_double_p, ctypes.POINTER(qpat_report)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_names() -> Sequence[str]:
    return [
        "qpat_default_params", "qpat_last_error", "qpat_launch_count", "qpat_mesh", "qpat_mesh_ex", "qpat_mesh_free",
        "qpat_mesh_host_info", "qpat_mesh_num_nodes", "qpat_mesh_num_tets", "qpat_mesh_num_faces", "qpat_mesh_num_patches",
        "qpat_mesh_num_entries", "qpat_mesh_num_prior_entries", "qpat_mesh_num_local_entries",
        "qpat_mesh_faces", "qpat_mesh_permutation", "qpat_mesh_stats", "qpat_mesh_fp64_fallbacks",
        "qpat_mesh_rhs_iterations", "qpat_mesh_multigrid_levels", "qpat_mesh_multigrid_fine_time", "qpat_multigrid_host_info", "qpat_mesh_reset_stats",
        "qpat_mesh_set_timing", "qpat_mesh_pcg_time",
        "qpat_flux_patch", "qpat_flux_side", "qpat_apply_K_dev", "qpat_forward", "qpat_forward_dev", "qpat_forward_noalloc_dev",
        "qpat_forward_guess_dev",
        "qpat_jvp", "qpat_jvp_dev",
        "qpat_vjp", "qpat_vjp_dev", "qpat_jvp_vjp_pair_dev", "qpat_jvp_vjp_pair", "qpat_prior_solve", "qpat_prior_solve_dev",
        "qpat_batch_create", "qpat_batch_buffers", "qpat_batch_forward", "qpat_batch_status", "qpat_batch_free",
        "qpat_autotune", "qpat_reconstruct", "qpat_reconstruct_ex",
        "qpat_unet_create", "qpat_unet_free", "qpat_unet_num_params", "qpat_unet_get_params", "qpat_unet_set_params",
        "qpat_unet_features_dev", "qpat_unet_predict_dev", "qpat_unet_train_dev", "qpat_unet_grad_dev",
        "qpat_unet_set_log_output",
        "qpat_unet_to_double_dev",
        "qpat_conv3d_bf16_dev", "qpat_conv3d_bf16_wgrad_dev", "qpat_conv3d_bf16_wgrad_scratch",
        "qpat_conv3d_set_engine", "qpat_conv3d_tc_timeouts",
    ]


class UNet:
    """Owning wrapper of qpat_unet_t (see include/qpat.h)."""

    def __init__(self, n: int, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().qpat_unet_create(int(n), int(seed), ctypes.byref(h)))
        self.handle = h
        self.n = int(n)

    def num_params(self) -> int:
        return int(load().qpat_unet_num_params(self.handle))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(load().qpat_unet_get_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().qpat_unet_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def predict(self, x, y):
        """x: (B, n^3, 3) float32 CUDA tensor -> y (B, n^3) float32."""
        _check(load().qpat_unet_predict_dev(self.handle, _tpf(x), x.shape[0], _tpf(y), _stream()))
        return y

    def train_step(self, x, t, lr: float) -> float:
        loss = ctypes.c_float()
        _check(load().qpat_unet_train_dev(self.handle, _tpf(x), _tpf(t), x.shape[0], float(lr), ctypes.byref(loss),
                                          _stream()))
        return float(loss.value)

    def set_log_output(self, floor: float):
        """floor > 0: learn log(max(phi, floor)) and predict exp of the output."""
        _check(load().qpat_unet_set_log_output(self.handle, float(floor)))

    def grad(self, x, t):
        """(loss, gradient) of the mean squared error of samples x against
        targets t, in the parameter layout of get_params; no update."""
        g = np.empty(self.num_params(), dtype=np.float32)
        loss = ctypes.c_float()
        _check(load().qpat_unet_grad_dev(self.handle, _tpf(x), _tpf(t), x.shape[0],
                                         g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss),
                                         _stream()))
        return float(loss.value), g

    def close(self):
        if getattr(self, "handle", None):
            load().qpat_unet_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tpf(t):
    """float32 / bf16 contiguous CUDA tensor pointer."""
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("device calls take contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def qpat_unet_features_dev(mesh: Mesh, kappa, mu, flux, h: float, x):
    K = flux.shape[0]
    _check(load().qpat_unet_features_dev(mesh.handle, _tp(kappa), _tp(mu), K, _tp(flux), float(h), _tpf(x),
                                         _stream()))
    return x


def qpat_unet_to_double_dev(y, out):
    _check(load().qpat_unet_to_double_dev(_tpf(y), int(y.numel()), _tp(out), _stream()))
    return out


def qpat_conv3d_set_engine(engine: int):
    """0: tcgen05 tensor cores where the shape allows (default); 1: mma.sync only."""
    _check(load().qpat_conv3d_set_engine(int(engine)))


def qpat_conv3d_tc_timeouts() -> int:
    return int(load().qpat_conv3d_tc_timeouts())


def qpat_conv3d_bf16_dev(x, w, bias, cout: int, relu: bool, n: int, out, out_f32=None):
    cin = x.shape[-1]
    _check(load().qpat_conv3d_bf16_dev(_tpf(x), int(cin), _tpf(w), _tpf(bias), int(cout), 1 if relu else 0, int(n),
                                       _tpf(out), _tpf(out_f32), _stream()))
    return out


def qpat_conv3d_bf16_wgrad_dev(x, dy, n: int, dw, db, partial):
    _check(load().qpat_conv3d_bf16_wgrad_dev(_tpf(x), int(x.shape[-1]), _tpf(dy), int(dy.shape[-1]), int(n),
                                             _tpf(dw), _tpf(db), _tpf(partial), _stream()))
    return dw, db


def qpat_conv3d_bf16_wgrad_scratch(n: int, cin: int, cout: int) -> int:
    return int(load().qpat_conv3d_bf16_wgrad_scratch(int(n), int(cin), int(cout)))


def qpat_autotune(xyz, tets, kappa, mu, K: int, iters: int = 30):
    """Best (patch_nodes, fp32_operator) for this mesh and K, and the timing
    table {(patch_nodes, fp32_operator): microseconds per FP32 PCG iteration}."""
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    bp, bo, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    us = np.zeros(16)
    _check(load().qpat_autotune(_dp(xyz), xyz.shape[0], tets.ctypes.data_as(_c_int32_p), tets.shape[0],
                                _dp(_f64(kappa)), _dp(_f64(mu)), int(K), int(iters), ctypes.byref(bp),
                                ctypes.byref(bo), _dp(us), ctypes.byref(nc)))
    cands = [0, 128, 256, 512, 1024]
    table = {(c, op): float(us[2 * i + op]) for i, c in enumerate(cands) for op in (0, 1)}
    return (bp.value, bo.value), table


def _check(rc: int):
    if rc != QPAT_OK:
        msg = load().qpat_last_error().decode(errors="replace")
        raise QpatError(rc, msg)


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_c_double_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def qpat_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().qpat_launch_count())


def qpat_default_params(**overrides) -> qpat_params:
    p = qpat_params()
    load().qpat_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Mesh:
    """Owning wrapper of a qpat_mesh_t handle."""

    def __init__(self, xyz, tets, patch_nodes: Optional[int] = None):
        lib = load()
        xyz = _f64(xyz)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        h = ctypes.c_void_p()
        if patch_nodes is None:
            _check(lib.qpat_mesh(_dp(xyz), xyz.shape[0], tets.ctypes.data_as(_c_int32_p), tets.shape[0],
                                 ctypes.byref(h)))
        else:
            _check(lib.qpat_mesh_ex(_dp(xyz), xyz.shape[0], tets.ctypes.data_as(_c_int32_p), tets.shape[0],
                                    patch_nodes, ctypes.byref(h)))
        self.handle = h
        self.N = int(lib.qpat_mesh_num_nodes(h))
        self.E = int(lib.qpat_mesh_num_tets(h))
        self.F = int(lib.qpat_mesh_num_faces(h))
        self.P = int(lib.qpat_mesh_num_patches(h))
        self.entries = int(lib.qpat_mesh_num_entries(h))
        self.prior_entries = int(lib.qpat_mesh_num_prior_entries(h))
        # couplings inside a patch (what the patch-local preconditioner applies)
        self.local_entries = int(lib.qpat_mesh_num_local_entries(h, 0))
        self.prior_local_entries = int(lib.qpat_mesh_num_local_entries(h, 1))

    def close(self):
        if getattr(self, "handle", None):
            load().qpat_mesh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def faces(self) -> np.ndarray:
        out = np.empty((self.F, 3), dtype=np.int32)
        _check(load().qpat_mesh_faces(self.handle, out.ctypes.data_as(_c_int32_p)))
        return out

    def permutation(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int32)
        _check(load().qpat_mesh_permutation(self.handle, out.ctypes.data_as(_c_int32_p)))
        return out

    def stats(self) -> dict:
        out = np.zeros(4, dtype=np.int64)
        _check(load().qpat_mesh_stats(self.handle, out.ctypes.data_as(_c_int64_p)))
        return {"pcg_iters": int(out[0]), "solves": int(out[1]), "refinements": int(out[2]),
                "launches": int(out[3]), "fp64_fallbacks": int(load().qpat_mesh_fp64_fallbacks(self.handle)),
                "rhs_iters": int(load().qpat_mesh_rhs_iterations(self.handle))}

    def reset_stats(self):
        _check(load().qpat_mesh_reset_stats(self.handle))

    def multigrid_fine_time(self):
        """(ms, launches) of the fine-level smoothing launches of the
        multigrid cycles since the last reset (timing on)."""
        ms = ctypes.c_double()
        n = np.zeros(1, dtype=np.int64)
        _check(load().qpat_mesh_multigrid_fine_time(self.handle, ctypes.byref(ms), n.ctypes.data_as(_c_int64_p)))
        return float(ms.value), int(n[0])

    def multigrid_levels(self, prior: bool = False) -> list:
        """Rows of each level of the multigrid hierarchy of the K (or prior)
        pattern, finest first; [] before the first multigrid solve."""
        rows = np.zeros(16, dtype=np.int64)
        n = load().qpat_mesh_multigrid_levels(self.handle, 1 if prior else 0, rows.ctypes.data_as(_c_int64_p), 16)
        if n < 0:
            _check(n)
        return [int(r) for r in rows[:min(n, 16)]]

    def set_timing(self, on: bool = True):
        _check(load().qpat_mesh_set_timing(self.handle, 1 if on else 0))

    def pcg_time_ms(self) -> float:
        v = ctypes.c_double()
        _check(load().qpat_mesh_pcg_time(self.handle, ctypes.byref(v)))
        return float(v.value)


def qpat_mesh(xyz, tets, patch_nodes: Optional[int] = None) -> Mesh:
    """Mesh handle; patch_nodes=None lets the library balance the patches
    over the GPU's resident CTAs (qpat_mesh), an int calls qpat_mesh_ex."""
    return Mesh(xyz, tets, patch_nodes)


def qpat_mesh_host_info(xyz, tets, patch_nodes: int = 512):
    """Host-only mesh preparation check; returns (info dict, faces, perm)."""
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    info = np.zeros(11, dtype=np.int64)
    lib = load()
    # first call sizes the face array
    _check(lib.qpat_mesh_host_info(_dp(xyz), xyz.shape[0], tets.ctypes.data_as(_c_int32_p), tets.shape[0],
                                   patch_nodes, info.ctypes.data_as(_c_int64_p), None, None))
    faces = np.empty((int(info[0]), 3), dtype=np.int32)
    perm = np.empty(xyz.shape[0], dtype=np.int32)
    _check(lib.qpat_mesh_host_info(_dp(xyz), xyz.shape[0], tets.ctypes.data_as(_c_int32_p), tets.shape[0],
                                   patch_nodes, info.ctypes.data_as(_c_int64_p), faces.ctypes.data_as(_c_int32_p),
                                   perm.ctypes.data_as(_c_int32_p)))
    keys = ["F", "P", "max_touched", "max_own", "max_ptets", "max_pfaces", "patch_tets", "patch_faces",
            "nnz", "prior_nnz", "max_tet_colours"]
    return dict(zip(keys, (int(v) for v in info))), faces, perm


def qpat_multigrid_host_info(xyz, tets, prior: bool = False, patch_nodes: int = 512) -> list:
    """Host-only check of the multigrid hierarchy's plan for the mesh's K (or
    prior) pattern; returns the rows of each level, finest first."""
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    rows = np.zeros(16, dtype=np.int64)
    n = load().qpat_multigrid_host_info(_dp(xyz), xyz.shape[0], tets.ctypes.data_as(_c_int32_p), tets.shape[0],
                                        patch_nodes, 1 if prior else 0, rows.ctypes.data_as(_c_int64_p), 16)
    if n < 0:
        _check(n)
    return [int(r) for r in rows[:min(n, 16)]]


def qpat_flux_side(mesh: Mesh, center, axis, ref, radius: float, theta0: float, half_w: float = math.pi / 8,
                   amp: float = 1.0) -> np.ndarray:
    """Per-face flux (canonical face order) through the curved side of a
    cylinder, cos(pi/2 (theta - theta0) / half_w) on |theta - theta0| <= half_w."""
    out = np.empty(mesh.F)
    _check(load().qpat_flux_side(mesh.handle, _dp(_f64(center)), _dp(_f64(axis)), _dp(_f64(ref)), float(radius),
                                 float(theta0), float(half_w), float(amp), _dp(out)))
    return out


def qpat_flux_patch(mesh: Mesh, center, normal, half_w: float, amp: float = 1.0) -> np.ndarray:
    c = _f64(center)
    n = _f64(normal)
    out = np.empty(mesh.F)
    _check(load().qpat_flux_patch(mesh.handle, _dp(c), _dp(n), float(half_w), float(amp), _dp(out)))
    return out


def _pp(params):
    return ctypes.byref(params) if params is not None else None


# ------------------------------------------------------------------ host calls

def qpat_forward(mesh: Mesh, kappa, mu, flux, params: Optional[qpat_params] = None):
    flux = _f64(np.atleast_2d(flux))
    K = flux.shape[0]
    kappa, mu = _f64(kappa), _f64(mu)
    phi = np.empty((K, mesh.N))
    h = np.empty((K, mesh.N))
    _check(load().qpat_forward(mesh.handle, _pp(params), _dp(kappa), _dp(mu), K, _dp(flux), _dp(phi), _dp(h)))
    return phi, h


def qpat_jvp(mesh: Mesh, kappa, mu, phi, s, w=None, params: Optional[qpat_params] = None):
    phi = _f64(np.atleast_2d(phi))
    K = phi.shape[0]
    w = None if w is None else _f64(np.broadcast_to(w, phi.shape))
    out = np.empty((K, mesh.N))
    _check(load().qpat_jvp(mesh.handle, _pp(params), _dp(_f64(kappa)), _dp(_f64(mu)), K, _dp(phi), _dp(w),
                           _dp(_f64(s)), _dp(out)))
    return out


def qpat_vjp(mesh: Mesh, kappa, mu, phi, t, w=None, params: Optional[qpat_params] = None):
    phi = _f64(np.atleast_2d(phi))
    K = phi.shape[0]
    t = _f64(np.broadcast_to(t, phi.shape))
    w = None if w is None else _f64(np.broadcast_to(w, phi.shape))
    out = np.empty(2 * mesh.N)
    _check(load().qpat_vjp(mesh.handle, _pp(params), _dp(_f64(kappa)), _dp(_f64(mu)), K, _dp(phi), _dp(w),
                           _dp(t), _dp(out)))
    return out


def qpat_jvp_vjp_pair(mesh: Mesh, kappa, mu, phi, s, t, w=None, params: Optional[qpat_params] = None,
                      out_jv=None, out_vjp=None):
    """One J s and one J^T t (host arrays) as a single 2K-RHS block solve;
    returns (w o J s (K x N), J^T (w o t) (2N)), written into out_jv / out_vjp
    when given (contiguous float64 host arrays, e.g. pinned)."""
    phi = _f64(np.atleast_2d(phi))
    K = phi.shape[0]
    t = _f64(np.broadcast_to(t, phi.shape))
    w = None if w is None else _f64(np.broadcast_to(w, phi.shape))
    oj = np.empty((K, mesh.N)) if out_jv is None else out_jv
    ov = np.empty(2 * mesh.N) if out_vjp is None else out_vjp
    if oj.shape != (K, mesh.N) or ov.shape != (2 * mesh.N,) or oj.dtype != np.float64 or ov.dtype != np.float64 \
            or not (oj.flags.c_contiguous and ov.flags.c_contiguous and oj.flags.writeable and ov.flags.writeable):
        raise ValueError("qpat_jvp_vjp_pair: out_jv must be K x N and out_vjp 2N contiguous float64")
    _check(load().qpat_jvp_vjp_pair(mesh.handle, _pp(params), _dp(_f64(kappa)), _dp(_f64(mu)), K, _dp(phi), _dp(w),
                                    _dp(_f64(s)), _dp(t), _dp(oj), _dp(ov)))
    return oj, ov


def qpat_prior_solve(mesh: Mesh, kt, mt, rhs, params: Optional[qpat_params] = None, out=None):
    out = np.empty(2 * mesh.N) if out is None else out
    if out.shape != (2 * mesh.N,) or out.dtype != np.float64 or not (out.flags.c_contiguous and out.flags.writeable):
        raise ValueError("qpat_prior_solve: out must be a contiguous float64 array of 2N")
    _check(load().qpat_prior_solve(mesh.handle, _pp(params), _dp(_f64(kt)), _dp(_f64(mt)), _dp(_f64(rhs)),
                                   _dp(out)))
    return out


def qpat_reconstruct_ex(mesh: Mesh, flux, chi, sigma, params: Optional[qpat_params] = None, kappa0_mu0=None,
                        beta_in=None, lin_done: int = 0):
    """Algorithm 1 with checkpoint / resume: returns (kappa, mu, beta, report);
    beta_in / lin_done resume a run at step 1 (see include/qpat.h)."""
    flux = _f64(np.atleast_2d(flux))
    K = flux.shape[0]
    chi = _f64(np.atleast_2d(chi))
    sigma = _f64(np.broadcast_to(sigma, chi.shape))
    k0 = None if kappa0_mu0 is None else _f64(kappa0_mu0)
    b_in = None if beta_in is None else _f64(beta_in)
    kappa = np.empty(mesh.N)
    mu = np.empty(mesh.N)
    beta = np.empty(2 * mesh.N)
    rep = qpat_report()
    _check(load().qpat_reconstruct_ex(mesh.handle, _pp(params), K, _dp(flux), _dp(chi), _dp(sigma), _dp(k0),
                                      _dp(b_in), int(lin_done), _dp(kappa), _dp(mu), _dp(beta), ctypes.byref(rep)))
    return kappa, mu, beta, rep


def qpat_reconstruct(mesh: Mesh, flux, chi, sigma, params: Optional[qpat_params] = None, kappa0_mu0=None):
    flux = _f64(np.atleast_2d(flux))
    K = flux.shape[0]
    chi = _f64(np.atleast_2d(chi))
    sigma = _f64(np.broadcast_to(sigma, chi.shape))
    k0 = None if kappa0_mu0 is None else _f64(kappa0_mu0)
    kappa = np.empty(mesh.N)
    mu = np.empty(mesh.N)
    rep = qpat_report()
    _check(load().qpat_reconstruct(mesh.handle, _pp(params), K, _dp(flux), _dp(chi), _dp(sigma), _dp(k0),
                                   _dp(kappa), _dp(mu), ctypes.byref(rep)))
    return kappa, mu, rep


# ------------------------------------------------------------------ device calls (torch)

def _tp(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous()):
        raise ValueError("device calls take contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def qpat_apply_K_dev(mesh: Mesh, kappa, mu, x, y, precision: int = 0):
    R = 1 if x.dim() == 1 else x.shape[1]
    _check(load().qpat_apply_K_dev(mesh.handle, precision, _tp(kappa), _tp(mu), R, _tp(x), _tp(y), _stream()))
    return y


def qpat_forward_dev(mesh: Mesh, kappa, mu, flux, phi, h, params: Optional[qpat_params] = None):
    K = flux.shape[0]
    _check(load().qpat_forward_dev(mesh.handle, _pp(params), _tp(kappa), _tp(mu), K, _tp(flux), _tp(phi), _tp(h),
                                   _stream()))
    return phi, h


def qpat_forward_guess_dev(mesh: Mesh, kappa, mu, flux, phi0, phi, h, params: Optional[qpat_params] = None):
    K = flux.shape[0]
    _check(load().qpat_forward_guess_dev(mesh.handle, _pp(params), _tp(kappa), _tp(mu), K, _tp(flux), _tp(phi0),
                                         _tp(phi), _tp(h), _stream()))
    return phi, h


def qpat_forward_noalloc_dev(mesh: Mesh, kappa, mu, flux, phi, h, rtol: float = 1e-13, max_iter: int = 20000):
    """Forward solve whose scratch lives in the library's fixed device array
    (no device allocation in the call); see include/qpat.h for the limit."""
    K = flux.shape[0]
    _check(load().qpat_forward_noalloc_dev(mesh.handle, _tp(kappa), _tp(mu), K, _tp(flux), float(rtol),
                                           int(max_iter), _tp(phi), _tp(h), _stream()))
    return phi, h


def qpat_jvp_dev(mesh: Mesh, kappa, mu, phi, w, s, out, params: Optional[qpat_params] = None):
    K = phi.shape[0]
    _check(load().qpat_jvp_dev(mesh.handle, _pp(params), _tp(kappa), _tp(mu), K, _tp(phi), _tp(w), _tp(s),
                               _tp(out), _stream()))
    return out


def qpat_vjp_dev(mesh: Mesh, kappa, mu, phi, w, t, out, params: Optional[qpat_params] = None):
    K = phi.shape[0]
    _check(load().qpat_vjp_dev(mesh.handle, _pp(params), _tp(kappa), _tp(mu), K, _tp(phi), _tp(w), _tp(t),
                               _tp(out), _stream()))
    return out


def qpat_jvp_vjp_pair_dev(mesh: Mesh, kappa, mu, phi, w, s, t, out_jv, out_vjp,
                          params: Optional[qpat_params] = None):
    K = phi.shape[0]
    _check(load().qpat_jvp_vjp_pair_dev(mesh.handle, _pp(params), _tp(kappa), _tp(mu), K, _tp(phi), _tp(w),
                                        _tp(s), _tp(t), _tp(out_jv), _tp(out_vjp), _stream()))
    return out_jv, out_vjp


def qpat_prior_solve_dev(mesh: Mesh, kt, mt, rhs, out, params: Optional[qpat_params] = None):
    _check(load().qpat_prior_solve_dev(mesh.handle, _pp(params), _tp(kt), _tp(mt), _tp(rhs), _tp(out),
                                       _stream()))
    return out


# ------------------------------------------------------------------ uneven batches

class _DevArray:
    """Zero-copy view of a library-owned float64 device buffer."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}


class Batch:
    """Owning wrapper of a qpat_batch_t: forward solves of several meshes in
    one cooperative launch, replayed as a CUDA graph (see include/qpat.h)."""

    def __init__(self, meshes, K, params: Optional[qpat_params] = None):
        import torch
        lib = load()
        n = len(meshes)
        arr = (ctypes.c_void_p * n)(*[m.handle for m in meshes])
        ks = (ctypes.c_int * n)(*[int(k) for k in K])
        h = ctypes.c_void_p()
        _check(lib.qpat_batch_create(n, arr, ks, _pp(params), ctypes.byref(h)))
        self.handle = h
        self.meshes = list(meshes)
        self.K = [int(k) for k in K]
        self.views = []
        for j, m in enumerate(meshes):
            p = [ctypes.c_void_p() for _ in range(4)]
            _check(lib.qpat_batch_buffers(h, j, *[ctypes.byref(x) for x in p]))
            shapes = [(m.N,), (m.N,), (self.K[j], m.F), (self.K[j], m.N)]
            self.views.append([torch.as_tensor(_DevArray(x.value, s), device="cuda") for x, s in zip(p, shapes)])

    def inputs(self, j):
        """(kappa, mu, flux) device tensors of problem j, to be filled in place."""
        return tuple(self.views[j][:3])

    def phi(self, j):
        return self.views[j][3]

    def forward(self):
        _check(load().qpat_batch_forward(self.handle, _stream()))

    def status(self):
        n = len(self.meshes)
        st, it, ct = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)()
        _check(load().qpat_batch_status(self.handle, st, it, ct))
        return list(st), list(it), list(ct)

    def close(self):
        if getattr(self, "handle", None):
            self.views = []
            load().qpat_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qpat_batch_create(meshes, K, params: Optional[qpat_params] = None) -> Batch:
    return Batch(meshes, K, params)
