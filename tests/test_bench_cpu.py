"""The bench's host-side helpers on CPU: strict-JSON output (no NaN / Infinity)
and the command-line flags of the benchmark contract."""

import json
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_finite_json_replaces_non_finite_values():
    import bench
    line = {"value": 1.5, "check": {"primal_res": math.nan, "dual_res": math.inf}, "list": [1.0, -math.inf, 2],
            "n": 3, "s": "x"}
    out = json.dumps(bench.finite_json(line), allow_nan=False)   # raises on NaN / Infinity
    back = json.loads(out)
    assert back["check"] == {"primal_res": None, "dual_res": None}
    assert back["list"] == [1.0, None, 2] and back["value"] == 1.5 and back["n"] == 3 and back["s"] == "x"


@pytest.mark.parametrize("argv", [[], ["--gpus", "4", "--steps", "7", "--warmup", "3"],
                                  ["--impl", "reference", "--steps", "2", "--warmup", "1"],
                                  ["--prior", "stv", "--storage", "bf16", "--no-batched"]])
def test_flags_parse(argv, monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    a = bench.parse()
    assert a.gpus >= 1 and a.steps >= 1 and a.warmup >= 0
    if not argv:
        assert a.gpus == 1 and a.warmup >= 3 and a.impl == "native" and a.prior == "tv" and a.storage == "fp32"


def test_compact_line_keeps_the_contract_and_ends_with_the_forms():
    """The printed line carries the contract's keys and ends with every
    form's headline numbers, within the last 1500 characters of the output."""
    import bench
    line = {"metric": "m", "value": 2484.0367963, "unit": "iters/s", "n_gpus": 1, "steps": 20, "warmup": 5,
            "ms_per_step": 40.25705, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "gpu_launches": 6140, "config": bench.config_obj("tv", "fp32"),
            "roofline": {"bound": "hbm", "achieved": 6663.46, "peak": 6785.9, "unit": "GB/s", "frac": 0.98,
                         "traffic": 2255654712},
            "cpu_baseline": bench.cpu_baseline_obj(dict(sample_iters=100, ncols=2, prologue_s=0.58,
                                                        iters_per_s=0.948), "tv"),
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 7},
            "e2e": {"value": 2414.2, "unit": "iters/s", "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
            "tuning": {"long": "x" * 400},
            "variants": {"dft": 2298.1, "haar2": 2357.0}, "stv_step": {"ms_per_iter": 0.365, "frac_hbm": 0.45},
            "batched": {"value": 77.2, "ms_per_batch": 828.6, "hbm_gbs_inverse_stream": 5230.0,
                        "peak_bps": 6.7859e12, "recons_per_s_with_plan": 8.1, "plan_s_total": 7.0, "slices": 64,
                        "iters_per_slice": 80, "note": "y" * 300},
            "precision": {"workload": "z" * 200, "fp16": {"iters_per_s": 403.6, "inverse_frac": 0.76,
                                                          "inverse_share": 0.44}},
            "grad": {"forward_ms": 12.05, "backward_ms": 18.93, "backward_over_forward": 1.57,
                     "forward_frac": 0.67, "backward_frac": 0.77}}
    out = bench.compact_line(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "roofline", "cpu_baseline",
              "e2e", "clocks", "gpu_launches", "config"):
        assert k in out, k
    assert "tuning" not in out and list(out)[-1] == "forms"
    text = json.dumps(bench.finite_json(out), separators=(",", ":"))
    tail = text[-1500:]
    for k in ('"batched"', '"precision"', '"grad"', '"variants_iters_s"', '"fwd_frac"', '"recons_s"'):
        assert k in tail, k
    assert out["forms"]["batched"]["frac"] == pytest.approx(5230.0e9 / 6.7859e12, rel=1e-2)
