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
