"""bench.py's roofline arithmetic for the multigrid headline, on the CPU:
the algorithmic work per launch of the fine-level smoothing kernel, the
achieved rate from the summed CUDA-event time, the fraction of the peak, and
that a stored ncu traffic figure is used only while the kernel sources keep
the hash recorded beside it."""
import json
import types

import pytest

import bench


def _fake(N=1000, entries=15000, prior_entries=7000, K=8):
    mesh = types.SimpleNamespace(entries=entries, prior_entries=prior_entries)
    return {"mesh": mesh, "N": N, "K": K}


def _acc(fine_ms, fine_launches, ms=10.0):
    return {"ms": ms, "iters": fine_launches, "rhs_iters": 16 * fine_launches, "launches": 1,
            "fine_ms": fine_ms, "fine_launches": fine_launches}


def test_fine_smoothing_work_and_rate():
    d = _fake()
    prm = types.SimpleNamespace(multigrid=1)
    acc = {"pair": _acc(2.0, 4), "prior": _acc(1.0, 4)}
    kern, peak = bench.mg_kernel_table(d, prm, acc, sm_mhz=2070.0, nsm=152, hbm_peak=6000.0, step_ms_total=20.0)
    R, N, E = 16, 1000, 15000
    assert kern["pair"]["flops_per_launch"] == 2 * E * R + 6 * N * R
    assert kern["pair"]["bytes_per_launch"] == 12 * E + 2 * N + 5 * 8 * R * N + 8 * N
    # 4 launches in 2 ms
    assert kern["pair"]["achieved_tflops"] == pytest.approx(4 * (2 * E * R + 6 * N * R) / 2e-3 / 1e12)
    assert kern["pair"]["us_per_launch"] == pytest.approx(500.0)
    assert peak == pytest.approx(2 * 152 * 2.07e9 * 2 / 1e12)     # 2 FMA per SM per cycle
    assert kern["pair"]["fp64_frac"] == pytest.approx(kern["pair"]["achieved_tflops"] / peak)
    # the prior: two value sets, R = 2
    assert kern["prior"]["flops_per_launch"] == 2 * 7000 * 2 + 6 * N * 2
    # FP32 cycle: 4-byte values, judged against HBM
    kern32, _ = bench.mg_kernel_table(d, types.SimpleNamespace(multigrid=2), acc, 2070.0, 152, 6000.0, 20.0)
    assert kern32["pair"]["arith"] == "fp32"
    assert kern32["pair"]["bytes_per_launch"] == 8 * E + 2 * N + 5 * 4 * R * N + 4 * N
    roof = bench.mg_roofline(kern32, "pair", peak, 6000.0, "measured", 2070.0, 152, "no_such_workload")
    assert roof["bound"] == "hbm" and roof["frac"] == pytest.approx(kern32["pair"]["achieved_gbs"] / 6000.0)
    assert roof["traffic"] is None


def test_traffic_only_with_matching_sources(tmp_path, monkeypatch):
    d = _fake()
    acc = {"pair": _acc(2.0, 4), "prior": _acc(1.0, 4)}
    kern, peak = bench.mg_kernel_table(d, types.SimpleNamespace(multigrid=1), acc, 2070.0, 152, 6000.0, 20.0)
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # a fixed hash stands for the current kernel sources
    monkeypatch.setattr(bench, "kernel_source_sha1", lambda files=None: "abc")
    entry = {"kernels": {"pair_fp64": {"dram_bytes_per_launch": 123}}}
    (prof / "k_cheb_w_traffic.json").write_text(json.dumps(dict(entry, source_sha1="abc")))
    assert bench.mg_roofline(kern, "pair", peak, 6000.0, "measured", 2070.0, 152, "w")["traffic"] == 123
    (prof / "k_cheb_w_traffic.json").write_text(json.dumps(dict(entry, source_sha1="other")))
    assert bench.mg_roofline(kern, "pair", peak, 6000.0, "measured", 2070.0, 152, "w")["traffic"] is None
