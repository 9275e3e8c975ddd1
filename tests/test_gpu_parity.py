"""Parity of the CUDA propagator (through the C ABI) with the FP64 oracle.

Tolerances: FP64 path relative l2 <= 1e-10 against the oracle; FP32 path
<= 1e-4 after 1000 steps with mass drift <= 1e-5.  Sizes span several CTA
tiles, rectangular grids, radix-3 lengths, batches and 3D; the full-size
512^2 TS4 workload is compared on its first steps.
"""
import math

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs
from paper_2603_25282_gb300 import sgp

pytestmark = pytest.mark.gpu


def _params(**kw):
    base = dict(omega=0.5, gamma=1.0, c0=100.0, c1=-1.0, c2=1.0, gx=1.0, gy=1.0, gz=1.0)
    base.update(kw)
    return base


def _ctx(n, L, prec="f64", batch=1, **prm):
    c = sgp.Context(n, L, batch=batch, prec=prec)
    c.set_params(**prm)
    return c


def _gpu_run(n, L, prm, psi, nsteps, dt, scheme, prec="f64", t0=0.0):
    c = _ctx(n, L, prec, **prm)
    dt_ = np.complex64 if prec == "f32" else np.complex128
    c.set_state(np.ascontiguousarray(psi[None].astype(dt_)), t0)
    c.step(nsteps, dt, scheme)
    out = c.get_state()[0].astype(np.complex128)
    t = c.t
    c.close()
    return out, t


def _oracle_run(n, L, prm, psi, nsteps, dt, scheme, t0=0.0):
    g = O.Grid(n, L)
    pr = O.Propagator(g, O.Params(**prm))
    return pr.run(psi, t0, dt, nsteps, scheme)


# ----------------------------------------------------------------------------
# single substeps
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,L", [((64, 64), 8.0), ((48, 96), (6.0, 9.0)), ((16, 32), (3.0, 4.0))])
def test_nonlinear_substep_f64(n, L):
    prm = _params(omega=0.7, gx=1.3, gy=0.8, c1=-3.0, c2=4.0)
    psi = inputs.gaussian_random_phase(n, L, seed=1, amp=1.5)
    c = _ctx(n, L, "f64", **prm)
    c.set_state(psi[None].copy(), 0.37)
    c.substep("nonlinear", 0.013)
    out = c.get_state()[0]
    ref = O.nonlinear_substep(psi, O.Grid(n, L), O.Params(**prm), 0.013, 0.37)
    assert O.rel_l2(out, ref) < 1e-13


@pytest.mark.parametrize("delta", [0.02, -0.011])
@pytest.mark.parametrize("n,L", [((64, 64), 8.0), ((96, 48), (9.0, 6.0)), ((32, 16), (4.0, 3.0))])
def test_linear_substep_f64(n, L, delta):
    prm = _params(omega=0.6, gamma=1.3)
    psi = inputs.gaussian_random_phase(n, L, seed=2, amp=1.5)
    c = _ctx(n, L, "f64", **prm)
    c.set_state(psi[None].copy(), 0.0)
    c.substep("linear", delta)
    out = c.get_state()[0]
    assert abs(c.t - delta) < 1e-15
    ref = O.linear_substep(psi, O.Grid(n, L), O.Params(**prm), delta)
    assert O.rel_l2(out, ref) < 1e-12


def test_linear_substep_zero_soc_zero_rotation_f64():
    """Degenerate lambda = 0 mode (Omega = 0, gamma = 0) and gamma = 0 alone."""
    n, L = (32, 32), 5.0
    psi = inputs.gaussian_random_phase(n, L, seed=3, amp=1.0)
    for prm in (_params(omega=0.0, gamma=0.0), _params(omega=0.4, gamma=0.0),
                _params(omega=0.0, gamma=0.9)):
        c = _ctx(n, L, "f64", **prm)
        c.set_state(psi[None].copy(), 0.0)
        c.substep("linear", 0.05)
        ref = O.linear_substep(psi, O.Grid(n, L), O.Params(**prm), 0.05)
        assert O.rel_l2(c.get_state()[0], ref) < 1e-12
        c.close()


# ----------------------------------------------------------------------------
# whole steps, FP64
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
@pytest.mark.parametrize("n,L", [((64, 64), 8.0), ((96, 48), (8.0, 6.0)), ((16, 16), 4.0),
                                 ((128, 32), (12.0, 5.0))])
def test_steps_f64_match_oracle(n, L, scheme):
    prm = _params(omega=0.5, gamma=1.0, gx=1.2, gy=0.9)
    psi = inputs.gaussian_random_phase(n, L, seed=4, amp=0.5)
    out, t = _gpu_run(n, L, prm, psi, 20, 2e-3, scheme, "f64", t0=0.1)
    ref, tr = _oracle_run(n, L, prm, psi, 20, 2e-3, scheme, t0=0.1)
    assert abs(t - tr) < 1e-14
    assert O.rel_l2(out, ref) < 1e-10


def test_config1_full_run_f64():
    """2D 64^2 on [-8,8]^2, Omega = 0.5, gamma = 1, c = (100, -1, 1), TS2,
    dt = 1e-3, 1000 steps, seeded Gaussian with 0.01 random phase."""
    n, L = (64, 64), 8.0
    prm = _params()
    psi = inputs.gaussian_random_phase(n, L, seed=1, amp=0.01)
    out, _ = _gpu_run(n, L, prm, psi, 1000, 1e-3, "ts2", "f64")
    ref, _ = _oracle_run(n, L, prm, psi, 1000, 1e-3, "ts2")
    assert O.rel_l2(out, ref) < 1e-10


def test_split_calls_equal_one_call_f64():
    n, L = (32, 32), 6.0
    prm = _params(gx=1.1)
    psi = inputs.gaussian_random_phase(n, L, seed=5, amp=0.3)
    a, ta = _gpu_run(n, L, prm, psi, 40, 1e-3, "ts4")
    c = _ctx(n, L, "f64", **prm)
    c.set_state(psi[None].copy(), 0.0)
    c.step(15, 1e-3, "ts4")
    c.step(25, 1e-3, "ts4")
    assert abs(c.t - ta) < 1e-15
    assert O.rel_l2(c.get_state()[0], a) < 1e-13


def test_batch_members_are_independent_f64():
    n, L = (48, 32), (6.0, 5.0)
    prm = _params(gx=1.2)
    psis = [inputs.gaussian_random_phase(n, L, seed=s, amp=0.4) for s in (7, 8, 9)]
    c = _ctx(n, L, "f64", batch=3, **prm)
    c.set_state(np.stack(psis), 0.0)
    c.step(10, 2e-3, "ts2")
    out = c.get_state()
    for k, psi in enumerate(psis):
        ref, _ = _oracle_run(n, L, prm, psi, 10, 2e-3, "ts2")
        assert O.rel_l2(out[k], ref) < 1e-10


@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
@pytest.mark.parametrize("n,L", [((16, 16, 32), (4.0, 4.0, 5.0)), ((32, 48, 16), (5.0, 6.0, 3.0))])
def test_steps_3d_f64_match_oracle(n, L, scheme):
    prm = _params(omega=0.7, gamma=1.0, c0=50.0, c1=-2.0, c2=5.0, gx=1.0, gy=1.2, gz=2.0)
    psi = inputs.gaussian_random_phase(n, L, seed=10, amp=0.5)
    out, _ = _gpu_run(n, L, prm, psi, 5, 2e-3, scheme, "f64")
    ref, _ = _oracle_run(n, L, prm, psi, 5, 2e-3, scheme)
    assert O.rel_l2(out, ref) < 1e-10


# ----------------------------------------------------------------------------
# FP32 path
# ----------------------------------------------------------------------------
def test_f32_1000_steps_accuracy_and_mass():
    n, L = (64, 64), 8.0
    prm = _params()
    psi = inputs.gaussian_random_phase(n, L, seed=1, amp=0.01)
    out, _ = _gpu_run(n, L, prm, psi, 1000, 1e-3, "ts2", "f32")
    ref, _ = _oracle_run(n, L, prm, psi, 1000, 1e-3, "ts2")
    err = O.rel_l2(out, ref)
    g = O.Grid(n, L)
    m0 = g.cell * np.sum(np.abs(psi) ** 2)
    m1 = g.cell * np.sum(np.abs(out) ** 2)
    assert err < 1e-4, err
    assert abs(m1 - m0) < 1e-5, (m0, m1)


def test_f32_ts4_full_size_first_steps():
    """512^2 on [-16,16]^2, Omega = 0.9, gamma = 1.5, c = (1000,-5,10), TS4,
    dt = 5e-4: the first two steps against the oracle (FP32 within 1e-5), in
    every kernel plan the autotuner chooses between for this grid."""
    n, L = (512, 512), 16.0
    prm = _params(omega=0.9, gamma=1.5, c0=1000.0, c1=-5.0, c2=10.0)
    psi = inputs.gaussian_random_phase(n, L, seed=2, amp=0.01)
    ref, _ = _oracle_run(n, L, prm, psi, 2, 5e-4, "ts4")
    out64, _ = _gpu_run(n, L, prm, psi, 2, 5e-4, "ts4", "f64")
    assert O.rel_l2(out64, ref) < 1e-10
    vs = [v for v in range(sgp.N_VARIANTS) if sgp.variant_exists("f32", 512, v)]
    for plan in [(vx, vy) for vx in vs for vy in vs]:
        c = _ctx(n, L, "f32", **prm)
        c.set_plan(plan)
        c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
        c.step(2, 5e-4, "ts4")
        out32 = c.get_state()[0].astype(np.complex128)
        c.close()
        assert O.rel_l2(out32, ref) < 1e-5, plan


# ----------------------------------------------------------------------------
# observables
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,L", [((64, 64), 8.0), ((48, 96), (6.0, 9.0))])
def test_observables_f64_match_oracle(n, L):
    prm = _params(omega=0.4, gamma=0.8, c0=30.0, c1=-2.0, c2=3.0, gx=1.2, gy=0.9)
    psi = inputs.gaussian_random_phase(n, L, seed=11, amp=1.0)
    psi[0] *= 1.3
    c = _ctx(n, L, "f64", **prm)
    c.set_state(psi[None].copy(), 0.7)
    ob = c.observables()[0]
    ref = O.observables(psi, O.Grid(n, L), O.Params(**prm), 0.7)
    for k in ("mass", "energy", "magnetization", "lz", "e_kin", "e_pot", "e_rot", "e_int", "e_soc"):
        assert abs(ob[k] - ref[k]) < 1e-10 * max(1.0, abs(ref[k])), (k, ob[k], ref[k])
    for a, b in zip(ob["comp_mass"], ref["comp_mass"]):
        assert abs(a - b) < 1e-12
    for a, b in zip(ob["width2"], ref["width2"]):
        assert abs(a - b) < 1e-10 * max(1.0, abs(b))


def test_observables_3d_f64_match_oracle():
    n, L = (16, 32, 16), (4.0, 5.0, 4.0)
    prm = _params(omega=0.4, gamma=0.8, gz=1.7)
    psi = inputs.gaussian_random_phase(n, L, seed=12, amp=1.0)
    c = _ctx(n, L, "f64", **prm)
    c.set_state(psi[None].copy(), 0.2)
    ob = c.observables()[0]
    ref = O.observables(psi, O.Grid(n, L), O.Params(**prm), 0.2)
    for k in ("mass", "energy", "lz", "e_kin", "e_soc"):
        assert abs(ob[k] - ref[k]) < 1e-10 * max(1.0, abs(ref[k])), (k, ob[k], ref[k])
    assert abs(ob["width2"][2] - ref["width2"][2]) < 1e-10


# ----------------------------------------------------------------------------
# edge cases and errors
# ----------------------------------------------------------------------------
def test_zero_steps_is_a_noop_and_errors_are_reported():
    n, L = (32, 32), 4.0
    c = _ctx(n, L, "f64", **_params())
    with pytest.raises(sgp.SgpError, match="ESTATE"):
        c.step(1, 1e-3)
    psi = inputs.gaussian_random_phase(n, L, seed=3)
    c.set_state(psi[None].copy(), 0.0)
    c.step(0, 1e-3)
    assert np.array_equal(c.get_state()[0], psi)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.step(1, -1e-3)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.step(1, float("nan"))
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.set_params(omega=float("inf"))


def test_zero_field_stays_zero():
    n, L = (32, 32), 4.0
    c = _ctx(n, L, "f32", **_params())
    z = np.zeros((1, 5, 32, 32), np.complex64)
    c.set_state(z, 0.0)
    c.step(3, 1e-3, "ts4")
    assert np.array_equal(c.get_state(), z)
    ob = c.observables()[0]
    assert ob["mass"] == 0.0 and ob["energy"] == 0.0


# ----------------------------------------------------------------------------
# per-member parameters, graph replay, ensembles of different grids
# ----------------------------------------------------------------------------
def test_per_member_parameters_f64():
    n, L = (48, 32), (6.0, 5.0)
    plist = [_params(omega=0.2, gamma=0.5, c0=40.0, gx=1.1),
             _params(omega=0.7, gamma=1.4, c0=90.0, c1=2.0, gy=0.8),
             _params(omega=0.2, gamma=0.5, c0=10.0, c2=-3.0)]
    psis = [inputs.gaussian_random_phase(n, L, seed=30 + k, amp=0.4) for k in range(3)]
    c = sgp.Context(n, L, batch=3, prec="f64")
    c.set_params_batch(plist)
    c.set_state(np.stack(psis), 0.0)
    c.step(12, 2e-3, "ts4")
    out = c.get_state()
    obs = c.observables()
    for k in range(3):
        ref, t = _oracle_run(n, L, plist[k], psis[k], 12, 2e-3, "ts4")
        assert O.rel_l2(out[k], ref) < 1e-10
        r = O.observables(ref, O.Grid(n, L), O.Params(**plist[k]), t)
        assert abs(obs[k]["energy"] - r["energy"]) < 1e-10 * max(1, abs(r["energy"]))


@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
def test_graph_replay_matches_direct_issue_and_oracle(scheme):
    n, L = (32, 32), 6.0
    prm = _params(gx=1.2, gy=0.9)
    psi = inputs.gaussian_random_phase(n, L, seed=15, amp=0.3)
    outs = []
    for graphs in (True, False):
        c = sgp.Context(n, L, prec="f64")
        c.set_params(**prm)
        c.set_graphs(graphs)
        c.set_state(psi[None].copy(), 0.0)
        c.step(150, 1e-3, scheme)          # 2 graph chunks of 64 + 22 direct
        outs.append(c.get_state()[0])
        assert abs(c.t - 0.15) < 1e-14
        c.close()
    assert O.rel_l2(outs[0], outs[1]) < 1e-13
    ref, _ = _oracle_run(n, L, prm, psi, 150, 1e-3, scheme)
    assert O.rel_l2(outs[0], ref) < 1e-10


def test_ensemble_of_different_grids_f64():
    grids = [((32, 32), 6.0), ((48, 48), 7.0), ((32, 32), 6.0), ((64, 32), (8.0, 5.0))]
    rng = np.random.default_rng(5)
    plist = [_params(omega=float(rng.uniform(0, 0.9)), gamma=float(rng.uniform(0, 2)),
                     c0=float(rng.uniform(50, 200)), c1=float(rng.uniform(-5, 5)),
                     c2=float(rng.uniform(0, 10))) for _ in grids]
    psis = [inputs.gaussian_random_phase(n, L, seed=50 + k, amp=0.3) for k, (n, L) in enumerate(grids)]
    with sgp.Ensemble(grids, prec="f64") as ens:
        assert ens.groups == 3
        ens.set_params(plist)
        for k, psi in enumerate(psis):
            ens.set_member_state(k, psi.copy(), 0.0)
        ens.step(70, 1e-3, "ts2")           # one graph chunk of 64 + 6 direct
        obs = ens.observables()
        for k, ((n, L), psi) in enumerate(zip(grids, psis)):
            ref, t = _oracle_run(n, L, plist[k], psi, 70, 1e-3, "ts2")
            assert O.rel_l2(ens.get_member_state(k), ref) < 1e-10
            r = O.observables(ref, O.Grid(n, L), O.Params(**plist[k]), t)
            assert abs(obs[k]["mass"] - r["mass"]) < 1e-12


@pytest.mark.parametrize("n,L", [((96, 96), 6.0), ((192, 192), 6.0)])
def test_fp32_mass_drift_on_radix3_lengths(n, L):
    """FP32 mass over 1000 TS4 steps on grids of length 3*2^k (plans with a
    radix-6 stage and twiddles at multiples of 30 degrees), trap on: the
    drift stays at the power-of-two level (it was ~1e-5 when the twiddle
    product lost its correction against exact +-1/2 components)."""
    prm = _params(c0=0.0, c1=0.0, c2=0.0, gamma=0.0, omega=0.2)
    c = _ctx(n, L, "f32", **prm)
    psi = inputs.ini_example3(n, L)
    c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
    m0 = c.observables()[0]["mass"]
    c.step(1000, 1e-3, "ts4")
    m1 = c.observables()[0]["mass"]
    c.close()
    assert abs(m1 / m0 - 1) < 5e-6


# ----------------------------------------------------------------------------
# compositions with the linear flow outside (Sec. 3.3, the other reading)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", ["ts2_lnl", "ts4_l"])
@pytest.mark.parametrize("n,L", [((64, 48), (8.0, 6.0)), ((96, 64), (9.0, 8.0))])
def test_linear_outer_schemes_f64(scheme, n, L):
    prm = _params(omega=0.6, gamma=1.1, gx=1.0, gy=1.3, c1=-2.0, c2=3.0)
    psi = inputs.gaussian_random_phase(n, L, seed=21, amp=0.5)
    out, t = _gpu_run(n, L, prm, psi, 20, 2e-3, scheme, "f64")
    ref, tr = _oracle_run(n, L, prm, psi, 20, 2e-3, scheme)
    assert abs(t - tr) < 1e-14
    assert O.rel_l2(out, ref) < 1e-10


@pytest.mark.parametrize("scheme", ["ts2_lnl", "ts4_l"])
def test_linear_outer_schemes_3d_and_f32(scheme):
    n, L = (32, 32, 48), (5.0, 5.0, 6.0)
    prm = _params(omega=0.5, gamma=0.8, gz=1.5)
    psi = inputs.gaussian_random_phase(n, L, seed=22, amp=0.5)
    ref, _ = _oracle_run(n, L, prm, psi, 10, 2e-3, scheme)
    out64, _ = _gpu_run(n, L, prm, psi, 10, 2e-3, scheme, "f64")
    assert O.rel_l2(out64, ref) < 1e-10
    out32, _ = _gpu_run(n, L, prm, psi, 10, 2e-3, scheme, "f32")
    assert O.rel_l2(out32, ref) < 1e-5


@pytest.mark.parametrize("scheme", ["ts2_lnl", "ts4_l"])
def test_linear_outer_schemes_graph_replay(scheme):
    """200 steps (graph replays of 64-step chunks, where the chunks meet the
    linear substeps are not merged) against the oracle."""
    n, L = (48, 48), 6.0
    prm = _params(omega=0.4, gamma=0.9)
    psi = inputs.gaussian_random_phase(n, L, seed=23, amp=0.5)
    out, _ = _gpu_run(n, L, prm, psi, 200, 1e-3, scheme, "f64")
    ref, _ = _oracle_run(n, L, prm, psi, 200, 1e-3, scheme)
    assert O.rel_l2(out, ref) < 1e-10


# ----------------------------------------------------------------------------
# full-size 3D workload, checkpoint/resume, health check
# ----------------------------------------------------------------------------
def test_3d_128_full_size_first_steps():
    """128^3 on [-8,8]^3, Omega = 0.7, gamma = 1, c = (500, -2, 5), gz = 2:
    the first two TS2 and TS4 steps against the oracle (FP64 within 1e-10,
    FP32 within 1e-5)."""
    n, L = (128, 128, 128), 8.0
    prm = _params(omega=0.7, gamma=1.0, c0=500.0, c1=-2.0, c2=5.0, gz=2.0)
    psi = inputs.gaussian_random_phase(n, L, seed=4, amp=0.01)
    for scheme in ("ts2", "ts4"):
        ref, _ = _oracle_run(n, L, prm, psi, 2, 1e-3, scheme)
        out64, _ = _gpu_run(n, L, prm, psi, 2, 1e-3, scheme, "f64")
        assert O.rel_l2(out64, ref) < 1e-10, scheme
        for v in range(sgp.N_VARIANTS):          # every plan the autotuner tries per axis
            c = _ctx(n, L, "f32", **prm)
            c.set_plan((v, v, v) if v != 5 else (5, 1, 1))   # variant 5: the xy-plane pass
            c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
            c.step(2, 1e-3, scheme)
            out32 = c.get_state()[0].astype(np.complex128)
            c.close()
            assert O.rel_l2(out32, ref) < 1e-5, (scheme, v)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_save_and_resume_is_bitwise(prec, tmp_path):
    """A run of 150 + 150 TS4 steps in one context equals 150 steps, the
    state and time saved to a file, a fresh context loaded from it and 150
    more steps, bit for bit (the resumed context replays the same chunks)."""
    n, L = (48, 64), (6.0, 8.0)
    prm = _params(gx=1.1, gy=0.9)
    dt_ = np.complex64 if prec == "f32" else np.complex128
    psi = inputs.gaussian_random_phase(n, L, seed=41, amp=0.4)[None].astype(dt_)
    a = _ctx(n, L, prec, **prm)
    a.set_state(psi.copy(), 0.0)
    a.step(150, 1e-3, "ts4")
    np.save(tmp_path / "state.npy", a.get_state())
    np.save(tmp_path / "t.npy", np.array([a.t]))
    a.step(150, 1e-3, "ts4")
    b = _ctx(n, L, prec, **prm)
    b.set_state(np.load(tmp_path / "state.npy"), float(np.load(tmp_path / "t.npy")[0]))
    b.step(150, 1e-3, "ts4")
    assert b.t == a.t
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_health_check_passes_and_matches_unchecked_run():
    n, L = (64, 64), 8.0
    prm = _params()
    psi = inputs.gaussian_random_phase(n, L, seed=42, amp=0.01)[None].astype(np.complex64)
    outs = []
    for every in (0, 100):
        c = _ctx(n, L, "f32", **prm)
        c.set_health_check(every, 1e-5)
        c.set_state(psi.copy(), 0.0)
        c.step(300, 1e-3, "ts4")
        assert abs(c.t - 0.3) < 1e-14
        outs.append(c.get_state()[0].astype(np.complex128))
        c.close()
    # the chunks of the checked run end and restart the step sequence, so the
    # two runs differ by FP32 rounding only
    assert O.rel_l2(outs[0], outs[1]) < 2e-5
    ref, _ = _oracle_run(n, L, prm, psi[0].astype(np.complex128), 300, 1e-3, "ts4")
    assert O.rel_l2(outs[1], ref) < 1e-4


def test_health_check_reports_nonfinite_and_drift():
    n, L = (32, 32), 4.0
    c = _ctx(n, L, "f32", batch=2, **_params())
    psi = inputs.gaussian_random_phase(n, L, seed=43, amp=0.3).astype(np.complex64)
    bad = psi.copy()
    bad[1, 3, 4] = np.nan
    c.set_health_check(5, 1e-5)
    c.set_state(np.stack([psi, bad]), 0.0)
    with pytest.raises(sgp.SgpError, match="ENONFINITE") as e:
        c.step(20, 1e-3, "ts2")
    assert "member 1" in str(e.value)
    # a tolerance of zero: the first check after the first chunk fails
    # (FP32 rounding moves the mass) and the time has advanced one chunk
    c.set_health_check(5, 0.0)
    c.set_state(np.stack([psi, psi]), 0.0)
    with pytest.raises(sgp.SgpError, match="EDRIFT") as e:
        c.step(20, 1e-3, "ts2")
    assert "member 0" in str(e.value)
    assert abs(c.t - 5e-3) < 1e-15
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.set_health_check(-1, 1e-5)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.set_health_check(10, float("nan"))
    c.set_health_check(0, 0.0)                   # off again
    c.step(20, 1e-3, "ts2")
    c.close()


def test_ensemble_observables_report_a_nonfinite_member():
    grids = [((32, 32), 6.0), ((48, 48), 7.0), ((32, 32), 6.0)]
    with sgp.Ensemble(grids, prec="f32") as ens:
        ens.set_params([_params()] * 3)
        for k, (n, L) in enumerate(grids):
            psi = inputs.gaussian_random_phase(n, L, seed=80 + k, amp=0.3).astype(np.complex64)
            if k == 2:
                psi[1, 5, 5] = np.nan
            ens.set_member_state(k, psi, 0.0)
        with pytest.raises(sgp.SgpError, match="ENONFINITE.*member 2"):
            ens.observables()
