"""Host-side arithmetic of bench.py's reports (no GPU): the phase shares and
the gather-phase DRAM rate derived from them, the traffic record's key, and
the oracle baselines' schedule."""

import argparse
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _clk(gather, exact, other):
    names = ("setup", "gather", "exact", "select", "thresholds", "decide_compact", "output")
    rounds = dict.fromkeys(names, 0)
    rounds.update(gather=gather, exact=exact, select=other)
    return {"rounds": rounds, "round0": dict.fromkeys(names[:6], 0) | {"gather": other}}


def _args(**kw):
    a = argparse.Namespace(storage="f32", share=False, block=1, cpu_c_alpha=None, B0=None, B=None, grow=None)
    for key, v in kw.items():
        setattr(a, key, v)
    return a


def test_phase_shares_and_gather_rate(monkeypatch):
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: bench.TRAFFIC_CAPTURE["sha1"])
    rec = bench.TRAFFIC_CAPTURE["records"][0]
    cfg = rec["config"]
    opts = {key: cfg[key] for key in ("c_alpha", "B0", "B", "grow", "threads")}
    w = dict(bench.WORKLOAD, nq=cfg["nq"])
    out = bench.phase_report(_clk(600, 200, 100), opts, _args(), w)
    sh = out["phase_clock_shares"]
    assert sh["rounds"]["gather"] == pytest.approx(600 / 1000) and sh["round0"]["gather"] == pytest.approx(0.1)
    assert out["phase_clocks_total"] == 1000
    g = out["gather_phase_dram"]
    want = (rec["rounds_bytes"] - 4.0 * w["n"] * w["nq"]) / (rec["rounds_ms"] * 1e-3 * 0.8) / 1e9
    assert g["share"] == pytest.approx(0.8) and g["gbs_at_least"] == pytest.approx(want, rel=1e-3)
    assert g["frac_at_least"] == pytest.approx(want / g["peak"], rel=1e-3)


@pytest.mark.parametrize("change", [dict(opt="B0", val=32), dict(arg="storage", val="bf16"), dict(arg="share", val=True),
                                    dict(arg="block", val=8), dict(w="nq", val=64), dict(sha="0" * 40)])
def test_gather_rate_only_for_the_captured_configuration(change, monkeypatch):
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: bench.TRAFFIC_CAPTURE["sha1"])
    cfg = bench.TRAFFIC_CAPTURE["records"][0]["config"]
    opts = {key: cfg[key] for key in ("c_alpha", "B0", "B", "grow", "threads")}
    w = dict(bench.WORKLOAD, nq=cfg["nq"])
    args = _args()
    if "opt" in change:
        opts[change["opt"]] = change["val"]
    elif "arg" in change:
        setattr(args, change["arg"], change["val"])
    elif "w" in change:
        w[change["w"]] = change["val"]
    else:  # kernel sources changed since the capture
        monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: change["sha"])
    assert "gather_phase_dram" not in bench.phase_report(_clk(6, 2, 1), opts, args, w)


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    """The traffic record stays valid across comment-only edits, and only those."""
    src = os.path.join(bench.ROOT, "paper_1902_09465_gb300", "csrc")
    d = tmp_path / "paper_1902_09465_gb300" / "csrc"
    d.mkdir(parents=True)
    texts = {f: open(os.path.join(src, f)).read() for f in ("adaptive_kernel.cuh", "knn_common.cuh")}
    for f, t in texts.items():
        (d / f).write_text(t)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_sha1()
    (d / "knn_common.cuh").write_text("// a note\n/* a block\n comment */\n\n" + texts["knn_common.cuh"] + "\n// end\n")
    assert bench.kernel_sources_sha1() == h0
    (d / "knn_common.cuh").write_text(texts["knn_common.cuh"] + "\nconstexpr int kUnused = 1;\n")
    assert bench.kernel_sources_sha1() != h0


def test_oracle_schedule_follows_the_gpu_arm():
    line_cfg = {"workload": "w", "c_alpha": 3e-4, "B0": 16, "B": 16, "grow": 0, "threads_per_query": 1024}
    assert bench.oracle_schedule(_args(), line_cfg) == {"c_alpha": 3e-4, "B0": 16, "B": 16, "grow": 0}
    assert bench.oracle_schedule(_args()) == bench.REFERENCE_SCHEDULE
    assert bench.oracle_schedule(_args(B0=4, cpu_c_alpha=1e-2))["B0"] == 4
    assert bench.oracle_schedule(_args(B0=4, cpu_c_alpha=1e-2))["c_alpha"] == 1e-2


def test_cpu_baseline_reports_model_and_single_core_rate():
    from paper_1902_09465_gb300 import synth
    X, Q = synth.pixel_mixture(2000, 64, 8, seed=1)
    r = bench.cpu_baseline(_args(), budget_s=0.5, X=X, Q=Q)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert isinstance(r["cpu_model"], str) and r["cpu_model"]
    st = r["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "queries" in st["sample"]


def test_roofline_picks_the_longer_kernel_and_keeps_both():
    hbm = {"bound": "hbm", "kernel": "rounds"}
    alu = {"bound": "alu", "kernel": "round0"}
    r = bench.roofline_of(hbm, alu, 2.1, 2.0, {"ms": 4.1})
    assert r["bound"] == "alu" and r["kernel"] == "round0"
    assert r["kernels"] == {"round0_kernel": alu, "adaptive_rounds_kernel": hbm} and r["call"] == {"ms": 4.1}
    r = bench.roofline_of(hbm, alu, 1.0, 2.0, {})
    assert r["bound"] == "hbm" and r["kernel"] == "rounds"


def test_alu_peak_counts_forty_multiplies_per_block():
    # 152 SMs x 64 multiply-adds per clock x 2.07 GHz / 40 = 503.4 G blocks/s
    assert abs(bench.alu_peak_blocks(152, 2070.0) - 503.424) < 1e-3
