"""x-pass variant 5: the xy-plane pass of 3D FP32 grids with NX = NY (one
thread-block cluster per z plane, the y transforms done inside it, the
plane handed between the CTAs through distributed shared memory).

Each line takes the arithmetic of the x-pass and the y-line pass of the
same elements per thread, so plan (5, v, w) must equal plan (1, v, w) bit
for bit for v in {0, 1, 2, 4}: TS2 and TS4, captured graphs (runs longer
than two 64-step chunks), single substeps, member windows of
sgp_step_host, several members with their own parameters, NZ different
from NX.  Against the FP64 oracle directly at 64^3 (FP32 tolerance of the
other variant tests, 1e-5), and the gradients of a recorded run (forward
through the plane pass, backward through the unfused passes) equal those of
variant 1.
"""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu

PRM = dict(omega=0.6, gamma=1.2, c0=200.0, c1=-2.0, c2=3.0, gx=1.0, gy=1.2, gz=1.5)


def _plist(batch):
    rng = np.random.default_rng(17)
    return [dict(omega=float(rng.uniform(0.1, 0.9)), gamma=float(rng.uniform(0.5, 1.5)),
                 c0=float(rng.uniform(50, 300)), c1=float(rng.uniform(-3, 3)),
                 c2=float(rng.uniform(0, 5)), gx=1.0, gy=1.2, gz=1.4) for _ in range(batch)]


def _states(n, L, batch):
    return np.stack([inputs.gaussian_random_phase(n, L, seed=90 + m, amp=0.4)
                     for m in range(batch)]).astype(np.complex64)


def _run(n, L, batch, plan, steps, scheme, host=False, chunks=1, graphs=True):
    c = sgp.Context(n, L, batch=batch, prec="f32")
    c.set_params_batch(_plist(batch))
    c.set_graphs(graphs)
    c.set_plan(plan)
    assert c.get_plan() == list(plan)
    psi = _states(n, L, batch)
    l0 = c.launch_count()
    if host:
        out = c.step_host(psi, 0.0, steps, 1e-3, scheme, chunks=chunks)
    else:
        c.set_state(psi, 0.0)
        l0 = c.launch_count()
        c.step(steps, 1e-3, scheme)
        out = c.get_state()
    c.synchronize()
    launches = c.launch_count() - l0
    c.close()
    return out, launches


@pytest.mark.parametrize("n,L,batch", [((128, 128, 128), 8.0, 1), ((64, 64, 64), 6.0, 3),
                                       ((128, 128, 64), (8.0, 8.0, 6.0), 2),
                                       ((64, 64, 96), (6.0, 6.0, 7.0), 2)])
@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
def test_plane_pass_equals_variant1(n, L, batch, scheme):
    a, la = _run(n, L, batch, (1, 1, 1), 5, scheme)
    b, lb = _run(n, L, batch, (5, 1, 1), 5, scheme)
    assert np.isfinite(a).all()
    assert np.array_equal(a, b)
    # no y-line passes: two launches per linear/nonlinear pair instead of four
    pairs = 5 if scheme == "ts2" else 15
    assert la - lb == 2 * pairs


@pytest.mark.parametrize("vy", [0, 2, 4])
def test_plane_pass_with_other_y_variants(vy):
    """The y axis's own variant does not enter the steps (only its E = 8
    twiddle table); every E = 8 y variant gives the same field."""
    n, L = (64, 64, 64), 6.0
    a, _ = _run(n, L, 2, (1, vy, 0), 4, "ts2")
    b, _ = _run(n, L, 2, (5, vy, 0), 4, "ts2")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("graphs", [True, False])
def test_plane_pass_in_captured_graphs(graphs):
    """130 steps: two replays of a captured 64-step graph and two eager
    steps (or all eager)."""
    n, L = (64, 64, 64), 6.0
    a, _ = _run(n, L, 2, (1, 0, 0), 130, "ts2", graphs=graphs)
    b, _ = _run(n, L, 2, (5, 0, 0), 130, "ts2", graphs=graphs)
    assert np.isfinite(a).all()
    assert np.array_equal(a, b)


def test_plane_pass_member_windows():
    """sgp_step_host steps member groups through member windows."""
    n, L = (64, 64, 32), (6.0, 6.0, 5.0)
    a, _ = _run(n, L, 5, (1, 0, 0), 6, "ts4")
    b, _ = _run(n, L, 5, (5, 0, 0), 6, "ts4", host=True, chunks=3)
    assert np.array_equal(a, b)


def test_plane_pass_substeps():
    """sgp_substep: a linear substep is x forward, the linear flow and x
    inverse; with variant 5 the x-passes carry the y transforms."""
    n, L = (64, 64, 64), 6.0
    res = []
    for plan in ((1, 0, 0), (5, 0, 0)):
        c = sgp.Context(n, L, batch=2, prec="f32")
        c.set_params_batch(_plist(2))
        c.set_plan(plan)
        c.set_state(_states(n, L, 2), 0.3)
        c.substep("linear", 2e-3)
        c.substep("nonlinear", -1e-3)
        c.substep("linear", -5e-4)
        res.append(c.get_state())
        c.close()
    assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
def test_plane_pass_matches_oracle(scheme):
    n, L = (64, 64, 64), (6.0, 6.0, 7.0)
    psi = inputs.gaussian_random_phase(n, L, seed=4, amp=0.5)
    nsteps, dt = 10, 1e-3
    ref = O.Propagator(O.Grid(n, L), O.Params(**PRM)).run(psi, 0.0, dt, nsteps, scheme)[0]
    c = sgp.Context(n, L, prec="f32")
    c.set_params(**PRM)
    c.set_plan((5, 0, 0))
    c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
    c.step(nsteps, dt, scheme)
    out = c.get_state()[0].astype(np.complex128)
    c.close()
    assert O.rel_l2(out, ref) < 1e-5


def test_plane_pass_gradients_equal_variant1():
    """The record runs its steps through the plane pass, the backward sweep
    through the unfused passes: the same states, so the same gradients."""
    n, L, batch = (64, 64, 64), 6.0, 2
    res = []
    for plan in ((1, 0, 0), (5, 0, 0)):
        c = sgp.Context(n, L, batch=batch, prec="f32")
        c.set_params_batch(_plist(batch))
        c.set_plan(plan)
        c.set_state(_states(n, L, batch), 0.0)
        c.record(20, 1e-3, "ts2", interval=6)
        g_t = np.conj(c.get_state())
        g0, dp = c.backward(g_t)
        c.close()
        res.append((g0, dp))
    assert np.isfinite(res[0][0]).all()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_plane_pass_rejected_where_it_does_not_exist():
    assert not sgp.variant_exists("f32", 128, 5)     # a grid-level variant
    cases = [((64, 64), "f32", (5, 0)),                # 2D
             ((96, 96, 64), "f32", (5, 0, 0)),         # NX = 96
             ((64, 128, 64), "f32", (5, 0, 0)),        # NX != NY
             ((64, 64, 64), "f64", (5, 0, 0)),         # FP64
             ((64, 64, 64), "f32", (0, 5, 0)),         # not the x axis
             ((64, 64, 64), "f32", (0, 0, 5))]
    for n, prec, plan in cases:
        c = sgp.Context(n, 6.0, prec=prec)
        with pytest.raises(sgp.SgpError):
            c.set_plan(plan)
        assert c.get_plan() == [0, 0, 0]
        c.close()


def test_autotuner_times_the_plane_pass():
    n, L = (64, 64, 64), 6.0
    c = sgp.Context(n, L, batch=2, prec="f32")
    c.set_params_batch(_plist(2))
    psi = _states(n, L, 2)
    c.set_state(psi, 0.0)
    plan, ms = c.autotune(reps=3, force=True, timings=True)
    assert ms[0][5] is not None and ms[0][5] > 0
    assert ms[1][5] is None and ms[2][5] is None
    assert np.array_equal(c.get_state(), psi)
    c.close()
