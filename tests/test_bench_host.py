"""Host logic of bench.py (no GPU): the algorithmic bytes per point-step of
each composition, and the committed DRAM counters being used only for the
kernels and kernel plan they were taken with."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_per_point_step(bench):
    # one read + one write of 5 complex values per pass; 2D: 2 passes per
    # (N, L) pair, 3D: 4; TS2 one pair per step, TS4 three
    assert bench.bytes_per_point_step(2, "ts2", "f32") == (160, 80)
    assert bench.bytes_per_point_step(2, "ts4", "f32") == (480, 80)
    assert bench.bytes_per_point_step(3, "ts2", "f32") == (320, 80)
    assert bench.bytes_per_point_step(3, "ts4", "f32") == (960, 80)
    assert bench.bytes_per_point_step(3, "ts2", "f32", (5, 1, 1)) == (160, 80)   # xy-plane pass
    assert bench.bytes_per_point_step(2, "ts2", "f64") == (320, 160)


def test_committed_traffic_matches_its_kernels_and_plan(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        tr = json.load(f)
    plans = tr["plans"]
    if tr["csrc_sha256_16"] != bench.csrc_hash():
        # the kernels changed since the capture: the bench reports no traffic
        assert bench.measured_traffic("2d512_ts4_f32", "xpass", plans["2d512_ts4_f32"]) is None
        pytest.skip("pass kernels changed since the committed DRAM counters")
    for key, val in tr["bytes_per_launch"].items():
        wl, kern = key.split(":")
        assert bench.measured_traffic(wl, kern, plans[wl]) == val
        # within 15% of the algorithmic one read + one write of the field
        n, L, prm, scheme, dt, prec, batch = bench.WORKLOADS[wl]
        alg = 2 * batch * 5 * n[0] * n[1] * (8 if prec == "f32" else 16)
        assert 0.8 * alg < val < 1.15 * alg
    for key in list(tr["thread_instr_per_point"]) + list(tr["dp_instr_per_point"]):
        wl, kern = key.split(":")
        assert wl in plans
    plan = plans["2d512_ts4_f32"]
    other = [v + 1 if k == 0 else v for k, v in enumerate(plan)]
    assert bench.measured_traffic("2d512_ts4_f32", "xpass", other) is None
    assert bench.measured_instr("2d512_ts4_f64", "xpass", plans["2d512_ts4_f64"],
                                "dp_instr_per_point") == tr["dp_instr_per_point"]["2d512_ts4_f64:xpass"]
