"""Host logic of the bench's roofline figures (no GPU): the whole-step bound
from its definition (method flops / tensor peak, 40 bytes per pt-field and
substep / HBM peak, right-hand-side operations / FP32 pipe), and the DRAM
traffic that is reported only while the capture's source hash matches."""

import os

import pytest

import bench

W = {"name": "ks_33x48x96", "n_r": 33, "n_theta": 48, "n_phi": 96, "L": 46, "n_fields": 50}


def test_whole_step_bound_by_hand():
    hbm, bf16, mhz, ms = 6800.0, 1700.0, 2000.0, 4.0
    b = bench._whole_step_bound(W, ms, hbm, bf16, mhz)
    P = 33 * 48 * 96
    units = 4 * P * 50
    t_tensor = (66 + 16 * 48 + 2 * 47) * units / 1.7e15
    t_hbm = 40 * units / 6.8e12
    t_alu = 4 * P * (bench.RHS_OPS_PER_POINT + 750) * bench.FF_INSTR_PER_OP / (152 * 128 * 2.0e9)
    assert b["t_tensor_ms"] == pytest.approx(t_tensor * 1e3)
    assert b["t_hbm_ms"] == pytest.approx(t_hbm * 1e3)
    assert b["t_rhs_alu_ms"] == pytest.approx(t_alu * 1e3)
    assert b["t_bound_ms"] == pytest.approx((max(t_tensor, t_hbm) + t_alu) * 1e3)
    assert b["frac"] == pytest.approx(b["t_bound_ms"] / ms)
    # 928 method flops per pt-field and substep on this shell
    assert 66 + 16 * 48 + 2 * 47 == 928


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    text = open(os.path.join(bench.ROOT, "profiles", "k_op_tc_dram_ks_33x48x96.md")).read()
    val, src = bench._op_traffic(W)
    if bench._op_sources_sha() in text:
        assert val is not None and val > 1e9, src
    else:
        assert val is None and "stale" in src
    # a capture on other sources is reported as stale, not used
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_op_tc_dram_ks_33x48x96.md").write_text(
        text.replace(bench._op_sources_sha(), "0" * 64))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_op_sources_sha", lambda: "1" * 64)
    val, src = bench._op_traffic(W)
    assert val is None and "stale" in src
    # no capture for a workload: no traffic
    val, src = bench._op_traffic(dict(W, name="other"))
    assert val is None
