"""Every kernel variant (tile and radix schedules) against the FP64 oracle,
and the autotuner's contract: it leaves the state unchanged, picks an
existing variant per axis, and the tuned plan still matches the oracle.

Tolerances as the main parity tests: FP64 relative l2 <= 1e-10, FP32
<= 1e-5 after a few tens of steps (the FP32 error grows like the square
root of the number of passes; 1e-4 is the 1000-step bound).
"""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu

PRM = dict(omega=0.6, gamma=1.2, c0=200.0, c1=-2.0, c2=3.0, gx=1.0, gy=1.2, gz=1.5)


def _run(n, L, prec, variants, psi, nsteps, dt, scheme):
    c = sgp.Context(n, L, prec=prec)
    c.set_params(**PRM)
    c.set_plan(variants)
    assert c.get_plan()[:len(n)] == list(variants)
    dt_ = np.complex64 if prec == "f32" else np.complex128
    c.set_state(psi[None].astype(dt_).copy(), 0.0)
    c.step(nsteps, dt, scheme)
    out = c.get_state()[0].astype(np.complex128)
    c.close()
    return out


def _oracle(n, L, psi, nsteps, dt, scheme):
    pr = O.Propagator(O.Grid(n, L), O.Params(**PRM))
    return pr.run(psi, 0.0, dt, nsteps, scheme)[0]


CASES_2D = [((64, 48), (8.0, 6.0)), ((256, 32), (12.0, 4.0)), ((96, 128), (7.0, 9.0))]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("n,L", CASES_2D)
def test_every_variant_2d(prec, tol, n, L):
    psi = inputs.gaussian_random_phase(n, L, seed=3, amp=0.5)
    nsteps, dt = 20, 1e-3
    ref = _oracle(n, L, psi, nsteps, dt, "ts4")
    for vx in range(sgp.N_VARIANTS):
        for vy in range(sgp.N_VARIANTS):
            if not (sgp.variant_exists(prec, n[0], vx) and sgp.variant_exists(prec, n[1], vy)):
                continue
            if vx != vy and vx != 0 and vy != 0:
                continue            # every variant on each axis, paired with 0 or itself
            out = _run(n, L, prec, (vx, vy), psi, nsteps, dt, "ts4")
            assert O.rel_l2(out, ref) < tol, (vx, vy, O.rel_l2(out, ref))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_every_variant_3d(prec, tol):
    n, L = (32, 48, 64), (5.0, 6.0, 7.0)
    psi = inputs.gaussian_random_phase(n, L, seed=4, amp=0.5)
    nsteps, dt = 10, 1e-3
    ref = _oracle(n, L, psi, nsteps, dt, "ts2")
    for v in range(sgp.N_VARIANTS):
        plan = [v if sgp.variant_exists(prec, n[a], v) else 0 for a in range(3)]
        out = _run(n, L, prec, plan, psi, nsteps, dt, "ts2")
        assert O.rel_l2(out, ref) < tol, (plan, O.rel_l2(out, ref))


def test_set_plan_rejects_missing_variant():
    c = sgp.Context((96, 64), 8.0, prec="f32")
    with pytest.raises(sgp.SgpError):
        c.set_plan((sgp.N_VARIANTS, 0))      # no such variant
    with pytest.raises(sgp.SgpError):
        c.set_plan((0, -1))
    assert c.get_plan() == [0, 0, 0]
    c.set_plan((3, 3))         # 12 elements per thread (N = 96), radix-4 plan (N = 64)
    assert c.get_plan() == [3, 3, 0]
    c.close()
    c = sgp.Context((64, 64), 8.0, prec="f64")
    with pytest.raises(sgp.SgpError):
        c.set_plan((0, 3))         # radix-4 variant is FP32 only
    c.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_autotune_keeps_state_and_matches_oracle(prec):
    n, L = (128, 96), (8.0, 6.0)
    psi = inputs.gaussian_random_phase(n, L, seed=5, amp=0.5)
    c = sgp.Context(n, L, prec=prec, batch=2)
    c.set_params(**PRM)
    dt_ = np.complex64 if prec == "f32" else np.complex128
    both = np.stack([psi, psi]).astype(dt_)
    c.set_state(both.copy(), 0.0)
    plan, ms = c.autotune(reps=5, force=True, timings=True)
    assert np.array_equal(c.get_state(), both)            # the state is untouched
    for a in range(2):
        assert sgp.variant_exists(prec, n[a], plan[a])
        assert ms[a][plan[a]] is not None and ms[a][plan[a]] > 0
        for v in range(sgp.N_VARIANTS):
            timed = (sgp.variant_exists(prec, n[a], v) and not (a == 0 and v == 4)
                     and not (a != 0 and v == 6))
            assert (ms[a][v] is not None) == timed
    assert ms[2] == [None] * sgp.N_VARIANTS
    assert c.autotune(reps=5) == plan                     # cached
    c.step(20, 1e-3, "ts4")
    out = c.get_state().astype(np.complex128)
    ref = _oracle(n, L, psi, 20, 1e-3, "ts4")
    tol = 1e-10 if prec == "f64" else 1e-5
    for m in range(2):
        assert O.rel_l2(out[m], ref) < tol
    c.close()


def test_ensemble_autotune_then_step():
    grids = [((64, 64), 8.0), ((96, 96), 8.0), ((64, 64), 8.0)]
    ens = sgp.Ensemble(grids, prec="f32")
    ens.set_params([PRM] * 3)
    psis = [inputs.gaussian_random_phase(g[0], g[1], seed=10 + i, amp=0.5) for i, g in enumerate(grids)]
    for i, p in enumerate(psis):
        ens.set_member_state(i, p.astype(np.complex64))
    ens.autotune(reps=3, force=True)
    ens.step(10, 1e-3, "ts2")
    for i, (n, L) in enumerate(grids):
        ref = O.Propagator(O.Grid(n, L), O.Params(**PRM)).run(psis[i], 0.0, 1e-3, 10, "ts2")[0]
        assert O.rel_l2(ens.get_member_state(i).astype(np.complex128), ref) < 1e-5
    ens.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,L,steps", [((256, 256), 8.0, 130), ((96, 64), (7.0, 5.0), 12),
                                       ((48, 32, 64), (6.0, 5.0, 7.0), 6)])
def test_variant6_against_variant2(prec, n, L, steps):
    """x-pass variant 6 (the rows of variant 2, the nonlinear flow shared by
    all threads of the CTA) takes every line and point through the
    arithmetic of variant 2 (130 steps replay a captured 64-step graph
    twice).  FP64: the fields agree to rounding (the compiler may fuse the
    other product of a sum of two products in another kernel).  FP32: the
    flow's small-angle
    form is chosen per warp, and a warp holds other points here, so the
    fields differ at the level of FP32 rounding: variant 6 is as close to
    the FP64 field as variant 2 is."""
    psi = inputs.gaussian_random_phase(n, L, seed=8, amp=0.5)
    rest = [0] * (len(n) - 1)
    a = _run(n, L, prec, [2] + rest, psi, steps, 1e-3, "ts4" if len(n) == 2 else "ts2")
    b = _run(n, L, prec, [6] + rest, psi, steps, 1e-3, "ts4" if len(n) == 2 else "ts2")
    assert np.isfinite(a).all()
    if prec == "f64":
        assert O.rel_l2(b, a) < 1e-12
    else:
        ref = _run(n, L, "f64", [0] * len(n), psi, steps, 1e-3, "ts4" if len(n) == 2 else "ts2")
        ea, eb = O.rel_l2(a, ref), O.rel_l2(b, ref)
        assert eb < 1e-4 and eb <= 1.5 * ea + 1e-7, (ea, eb)
