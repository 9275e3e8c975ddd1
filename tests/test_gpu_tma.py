"""Line-pass variant 4 (the tile brought into shared memory by tensor
copies) against variant 1, whose geometry and arithmetic it shares: bit for
bit in 2D and 3D (y and z lines), with a ragged last tile (zero-filled
columns past the grid's edge), several members (the member coordinate of
the tensor map), member windows of sgp_step_host (a first member other than
0), the autotuner's scratch field, and every line length that has lines of
more than 256 elements (several boxes per line)."""
import numpy as np
import pytest

from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _plist(batch):
    rng = np.random.default_rng(11)
    return [dict(omega=float(rng.uniform(0.1, 0.9)), gamma=float(rng.uniform(0.5, 1.5)),
                 c0=float(rng.uniform(50, 300)), c1=float(rng.uniform(-3, 3)),
                 c2=float(rng.uniform(0, 5)), gx=1.0, gy=1.2, gz=1.4) for _ in range(batch)]


def _states(n, L, batch):
    return np.stack([inputs.gaussian_random_phase(n, L, seed=80 + m, amp=0.4)
                     for m in range(batch)]).astype(np.complex64)


def _run(n, L, batch, plan, steps, scheme, host=False, chunks=1):
    c = sgp.Context(n, L, batch=batch, prec="f32")
    c.set_params_batch(_plist(batch))
    c.set_plan(plan)
    psi = _states(n, L, batch)
    if host:
        out = c.step_host(psi, 0.0, steps, 1e-3, scheme, chunks=chunks)
    else:
        c.set_state(psi, 0.0)
        c.step(steps, 1e-3, scheme)
        out = c.get_state()
    c.synchronize()
    c.close()
    return out


@pytest.mark.parametrize("n,L,batch", [((512, 512), 16.0, 2), ((48, 64), (6.0, 8.0), 3),
                                       ((96, 384), (8.0, 12.0), 2), ((64, 768), (6.0, 16.0), 1),
                                       ((32, 1024), (4.0, 16.0), 1)])
def test_variant4_equals_variant1_2d(n, L, batch):
    a = _run(n, L, batch, (1, 1), 7, "ts4")
    b = _run(n, L, batch, (1, 4), 7, "ts4")
    assert np.isfinite(a).all()
    assert np.array_equal(a, b)


def test_variant4_equals_variant1_3d():
    n, L = (32, 48, 64), (5.0, 6.0, 7.0)
    a = _run(n, L, 2, (1, 1, 1), 5, "ts2")
    b = _run(n, L, 2, (1, 4, 4), 5, "ts2")
    assert np.isfinite(a).all()
    assert np.array_equal(a, b)


def test_variant4_member_windows():
    """sgp_step_host steps groups of members through member windows: the
    tensor coordinate of a group's first member is not 0."""
    n, L = (128, 96), (8.0, 6.0)
    a = _run(n, L, 5, (1, 1), 6, "ts2")
    b = _run(n, L, 5, (1, 4), 6, "ts2", host=True, chunks=3)
    assert np.array_equal(a, b)


def test_autotuner_times_variant4_on_its_scratch_field():
    """The autotuner runs each variant on a scratch copy: the tensor map
    must follow the field buffer (the state must stay untouched)."""
    n, L = (256, 256), 8.0
    c = sgp.Context(n, L, batch=2, prec="f32")
    c.set_params_batch(_plist(2))
    psi = _states(n, L, 2)
    c.set_state(psi, 0.0)
    c.set_plan((0, 4))
    c.step(2, 1e-3, "ts2")                   # the map of the context's own field exists now
    before = c.get_state()
    plan, ms = c.autotune(reps=3, force=True, timings=True)
    assert ms[1][4] is not None and ms[0][4] is None
    assert np.array_equal(c.get_state(), before)
    c.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_variant4_in_the_adjoint_sweep(graphs):
    """The adjoint sweep runs line passes on its own buffers (the recomputed
    segment states, the adjoint state and its transform): the tensor map
    follows each of them.  Gradients with the line pass of variant 4 equal
    those of variant 1 bit for bit, with graph replay and eagerly."""
    n, L, batch = (256, 256), 8.0, 2
    res = []
    for plan in ((0, 1), (0, 4)):
        c = sgp.Context(n, L, batch=batch, prec="f32")
        c.set_params_batch(_plist(batch))
        c.set_graphs(graphs)
        c.set_plan(plan)
        psi = _states(n, L, batch)
        c.set_state(psi, 0.0)
        c.record(30, 1e-3, "ts2", interval=7)        # five segments, the last one short
        g_t = np.conj(c.get_state())
        g0, dp = c.backward(g_t)
        c.close()
        res.append((g0, dp))
    assert np.isfinite(res[0][0]).all() and np.isfinite(res[0][1]).all()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_variant4_in_captured_graphs():
    """A run of 130 steps replays a captured 64-step graph twice: the
    tensor-copy kernels inside it equal variant 1 bit for bit."""
    n, L = (512, 512), 16.0
    a = _run(n, L, 1, (0, 1), 130, "ts2")
    b = _run(n, L, 1, (0, 4), 130, "ts2")
    assert np.isfinite(a).all()
    assert np.array_equal(a, b)
