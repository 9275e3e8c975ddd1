"""The substep schedule the library issues (sgp_substep_plan, host only, no
GPU) against the compositions of Sec. 3.3 as the oracle takes them step by
step: every entry of the library's list is a run of consecutive substeps of
the oracle's sequence of the same kind (merged at step boundaries), with the
summed step and, for a nonlinear flow, the time at which every merged
substep acts; the flows alternate, their counts and total times are those
of the scheme, and bad arguments are refused."""
import os

import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import sgp

SCHEMES = ["ts2", "ts4", "ts2_lnl", "ts4_l"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(sgp.LIB_PATH):
        from paper_2603_25282_gb300 import build
        build.build()


def _oracle_substeps(scheme, n, dt):
    """(kind, delta, time) of every substep of n oracle steps: a nonlinear
    flow acts at the current time, a linear one starts there and advances
    it; step s starts at s dt."""
    out = []
    for s in range(n):
        tcur = s * dt
        for kind, coef in O.substep_sequence(scheme):
            out.append((kind, coef * dt, tcur))
            if kind == "L":
                tcur += coef * dt
    return out


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_plan_is_the_merged_oracle_sequence(scheme, n):
    dt = 1e-3
    plan = sgp.substep_plan(scheme, n, dt)
    orc = _oracle_substeps(scheme, n, dt)
    per_step = len(O.substep_sequence(scheme))
    assert len(plan) == (per_step - 1) * n + 1           # one merge per step boundary
    assert all(a[0] != b[0] for a, b in zip(plan, plan[1:]))
    tol = 1e-15 * max(1, n)
    j = 0
    for kind, delta, toff in plan:
        acc, first = 0.0, j
        while abs(acc - delta) > tol:
            assert j < len(orc) and orc[j][0] == kind, (kind, delta, j)
            if kind == "N":
                assert abs(orc[j][2] - toff) < tol      # acts at the entry's time
            acc += orc[j][1]
            j += 1
        assert j > first
        if kind == "L":
            assert abs(orc[first][2] - toff) < tol      # starts at the entry's time
    assert j == len(orc)
    for k in ("N", "L"):
        assert abs(sum(d for kk, d, _ in plan if kk == k) - n * dt) < tol


def test_plan_edge_cases_and_errors():
    assert sgp.substep_plan("ts4", 0, 1e-3) == []
    for bad in [dict(scheme=7, nsteps=1, dt=1e-3), dict(scheme="ts2", nsteps=-1, dt=1e-3),
                dict(scheme="ts2", nsteps=1, dt=0.0), dict(scheme="ts2", nsteps=1, dt=float("nan"))]:
        with pytest.raises(sgp.SgpError, match="EINVAL"):
            sgp.substep_plan(bad["scheme"], bad["nsteps"], bad["dt"])
