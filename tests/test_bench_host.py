"""Host logic of bench.py, no GPU: the fixed-parameter parser, the arithmetic dtype of a
precision mode, the per-field error measure (with the velocity error against the largest
component), the roofline breakdown of profile tallies, the source-keyed traffic table and
the reference arm's JSON line on a small workload."""
import io
import json
import os
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402
from paper_2603_21869_gb300 import cases  # noqa: E402


def test_parse_params_takes_five_to_seven_values():
    assert bench.parse_params("2,2,1,0,1") == (2, 2, 1, 0, 1, 0, 0)
    assert bench.parse_params("3,3,2,4,0,1") == (3, 3, 2, 4, 0, 1, 0)
    assert bench.parse_params("2,2,1,0,1,0,1") == (2, 2, 1, 0, 1, 0, 1)
    for bad in ("2,2,1,0", "1,2,3,4,5,6,7,8"):
        with pytest.raises(SystemExit):
            bench.parse_params(bad)


def test_arith_dtype_is_the_arithmetic_type():
    assert bench.arith_dtype("f64") == "f64"
    assert bench.arith_dtype("f32") == "f32"
    assert bench.arith_dtype("bf16") == "f32"   # BF16 only stores the multigrid corrections


def test_field_errors_scale_velocity_by_the_largest_component():
    shape = (4, 3, 2)
    ref = {f: np.zeros(shape) for f in cases.FIELDS}
    got = {f: np.zeros(shape) for f in cases.FIELDS}
    for f in cases.FIELDS:
        ref[f][:] = 1.0
    ref["u"][:] = 10.0
    ref["v"][:] = 0.01
    got["u"][:] = 10.0
    got["v"][:] = 0.01 + 1e-4            # 1 % of v, 1e-5 of the speed
    for f in ("w", "p", "T", "k", "omega"):
        got[f][:] = ref[f]
    e = bench.field_errors(got, ref)
    assert e["v"] == pytest.approx(1e-2, rel=1e-9)
    assert e["velocity"] == pytest.approx(1e-5, rel=1e-9)
    assert e["u"] == 0.0 and e["p"] == 0.0


def test_breakdown_picks_the_largest_site_and_its_bytes_per_launch(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (6000.0, "measured"))
    prof = {"sweep_L0": {"ms": 20.0, "launches": 10, "bytes": 1.0e11},
            "fcg_L0": {"ms": 30.0, "launches": 5, "bytes": 1.2e11},
            "explicit": {"ms": 5.0, "launches": 1, "bytes": 1.0e9}}
    bd = bench.breakdown(prof, 2, {"fcg_L0": 2.0e10})
    r = bd["roofline"]
    assert r["kernel"] == "fcg_L0" and r["launches"] == 5
    assert r["bytes_per_launch"] == pytest.approx(2.4e10)
    assert r["achieved"] == pytest.approx(1.2e11 / 0.030 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["traffic"] == 2.0e10
    # the V-cycle figure counts the multigrid sites only (sweeps, residuals, transfers, coarse CTA)
    assert bd["vcycle"]["gbs"] == pytest.approx(1.0e11 / 0.020 / 1e9)
    assert bd["kernels"]["explicit"]["ms_per_step"] == pytest.approx(2.5)


def test_traffic_is_reported_only_for_the_source_it_was_measured_on():
    sha = bench._src_sha("mg_kernels.cu")
    table = {("room", "bf16", "fcg_L0"): {"bytes": 1.0, "src": "mg_kernels.cu", "sha": sha},
             ("room", "f32", "fcg_L0"): {"bytes": 2.0, "src": "mg_kernels.cu", "sha": "0" * 16}}
    assert bench.traffic_for(table, ("room", "bf16", "fcg_L0")) == 1.0
    assert bench.traffic_for(table, ("room", "f32", "fcg_L0")) is None
    assert bench.traffic_for(table, ("channel", "f32", "sweep_L0")) is None
    # the committed entries name a source file that exists
    for t in bench.TRAFFIC.values():
        assert len(bench._src_sha(t["src"])) == 16


def test_reference_arm_prints_its_line_with_the_given_steps():
    spec = cases.heated_channel_3d(16, 8, 8, mg_levels=2, fixed_vcycles=2)
    args = SimpleNamespace(steps=2, warmup=1)
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(args, spec, "a 16x8x8 channel", 0, 1, "channel")
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "cell-steps/s" and line["unit"] == "cell-steps/s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["higher_is_better"] is True
