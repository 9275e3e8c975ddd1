"""sgp_step_host (host buffers in and out, the copies of the other member
groups overlapped with the steps of one) against the same run through
sgp_set_state / sgp_step / sgp_get_state: bit-identical results for every
split of the batch (uneven groups included), per-member parameters (the
member window into the per-member tables), 2D and 3D, both precisions,
in-place buffers; the time, the state left on the device, and the errors.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu


def _plist(batch):
    rng = np.random.default_rng(7)
    return [dict(omega=float(rng.uniform(0.1, 0.9)), gamma=float(rng.uniform(0.5, 1.5)),
                 c0=float(rng.uniform(50, 200)), c1=float(rng.uniform(-3, 3)),
                 c2=float(rng.uniform(0, 5)), gx=1.0, gy=1.2, gz=1.5) for _ in range(batch)]


def _states(n, L, batch, dtype):
    return np.stack([inputs.gaussian_random_phase(n, L, seed=60 + m, amp=0.4)
                     for m in range(batch)]).astype(dtype)


def _pinned(a):
    return torch.from_numpy(a).pin_memory()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,L,scheme,nsteps", [((64, 48), (8.0, 6.0), "ts4", 7),
                                               ((32, 32, 16), (5.0, 5.0, 4.0), "ts2", 5)])
def test_step_host_equals_set_step_get(prec, n, L, scheme, nsteps):
    batch = 5
    dtype = np.complex64 if prec == "f32" else np.complex128
    psi = _states(n, L, batch, dtype)
    c = sgp.Context(n, L, batch=batch, prec=prec)
    c.set_params_batch(_plist(batch))
    c.set_state(psi.copy(), 0.3)
    c.step(nsteps, 1e-3, scheme)
    ref = c.get_state()
    t_ref = c.t
    for chunks in (1, 2, 3, 5):
        out = torch.empty(psi.shape, dtype=torch.complex64 if prec == "f32" else torch.complex128).pin_memory()
        c.step_host(_pinned(psi), 0.3, nsteps, 1e-3, scheme, chunks=chunks, out=out)
        assert np.array_equal(out.numpy(), ref), chunks
        assert c.t == t_ref
        assert np.array_equal(c.get_state(), ref)      # the state stays on the device
    c.close()


def test_step_host_in_place_pageable_and_continuation():
    n, L, batch = (48, 48), 6.0, 4
    psi = _states(n, L, batch, np.complex64)
    prm = _plist(batch)
    a = sgp.Context(n, L, batch=batch, prec="f32")
    a.set_params_batch(prm)
    a.set_state(psi.copy(), 0.0)
    a.step(20, 1e-3, "ts4")
    ref = a.get_state()
    b = sgp.Context(n, L, batch=batch, prec="f32")
    b.set_params_batch(prm)
    buf = psi.copy()                                   # pageable, in and out the same
    b.step_host(buf, 0.0, 10, 1e-3, "ts4", chunks=3, out=buf)
    b.step(10, 1e-3, "ts4")                            # continues from the device state
    # 10 + 10 steps in two calls: the step sequence restarts at the call
    # boundary, so the comparison is at the FP32 level
    out = b.get_state()
    for m in range(batch):
        assert O.rel_l2(out[m].astype(np.complex128), ref[m].astype(np.complex128)) < 2e-6
    assert abs(b.t - 0.02) < 1e-15
    a.close()
    b.close()


def test_step_host_errors():
    c = sgp.Context((32, 32), 4.0, batch=2, prec="f32")
    psi = _states((32, 32), 4.0, 2, np.complex64)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.step_host(psi, 0.0, 1, 1e-3, chunks=0)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.step_host(psi, 0.0, 1, 1e-3, chunks=3)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        c.step_host(psi, float("nan"), 1, 1e-3, chunks=1)
    with pytest.raises(ValueError):
        c.step_host(torch.from_numpy(psi).cuda(), 0.0, 1, 1e-3, chunks=1)
    out = c.step_host(psi, 0.0, 0, 1e-3, chunks=2)     # zero steps: a round trip
    assert np.array_equal(out, psi)
    c.close()


def test_ensemble_step_host_equals_member_calls():
    grids = [((32, 32), 6.0), ((48, 48), 7.0), ((32, 32), 6.0), ((64, 32), (8.0, 5.0))]
    plist = _plist(len(grids))
    psis = [inputs.gaussian_random_phase(n, L, seed=70 + k, amp=0.3).astype(np.complex64)
            for k, (n, L) in enumerate(grids)]
    with sgp.Ensemble(grids, prec="f32") as a, sgp.Ensemble(grids, prec="f32") as b:
        a.set_params(plist)
        b.set_params(plist)
        for k, p in enumerate(psis):
            a.set_member_state(k, p.copy(), 0.2)
        a.step(9, 1e-3, "ts4")
        ref = [a.get_member_state(k) for k in range(len(grids))]
        srcs = [torch.from_numpy(p).pin_memory() for p in psis]
        outs = b.step_host(srcs, 0.2, 9, 1e-3, "ts4")
        for k in range(len(grids)):
            assert np.array_equal(outs[k], ref[k]), k
            assert np.array_equal(b.get_member_state(k), ref[k])
        inplace = [p.copy() for p in psis]                 # pageable, in place
        b.step_host(inplace, 0.2, 9, 1e-3, "ts4", outs=inplace)
        for k in range(len(grids)):
            assert np.array_equal(inplace[k], ref[k])
        with pytest.raises(sgp.SgpError, match="EINVAL"):
            b.step_host(psis, float("inf"), 1, 1e-3)


def test_ensemble_step_host_page_locked_copies_in_one_launch():
    """Every buffer page-locked: each direction is one copy launch reading or
    writing the host buffers through their device mapping (two launches more
    than with pageable buffers); the results equal the per-member calls bit
    for bit, also in place and with grids of the persistent kernel.  One
    pageable buffer among them sends the call back to per-member copies."""
    grids = [((64, 64), 8.0), ((128, 128), 8.0), ((96, 96), 8.0), ((64, 64), 8.0), ((256, 256), 8.0)]
    plist = _plist(len(grids))
    psis = [inputs.gaussian_random_phase(n, L, seed=90 + k, amp=0.3).astype(np.complex64)
            for k, (n, L) in enumerate(grids)]
    with sgp.Ensemble(grids, prec="f32") as a, sgp.Ensemble(grids, prec="f32") as b:
        a.set_params(plist)
        b.set_params(plist)
        for k, p in enumerate(psis):
            a.set_member_state(k, p.copy(), 0.1)
        a.step(5, 1e-3, "ts2")
        ref = [a.get_member_state(k) for k in range(len(grids))]
        # pageable buffers: per-member copies
        l0 = b.launch_count()
        outs = b.step_host([p.copy() for p in psis], 0.1, 5, 1e-3, "ts2")
        lp = b.launch_count() - l0
        for k in range(len(grids)):
            assert np.array_equal(outs[k], ref[k]), k
        # page-locked in and out
        srcs = [torch.from_numpy(p.copy()).pin_memory() for p in psis]
        pouts = [torch.empty(p.shape, dtype=torch.complex64).pin_memory() for p in psis]
        l0 = b.launch_count()
        b.step_host(srcs, 0.1, 5, 1e-3, "ts2", outs=pouts)
        assert b.launch_count() - l0 == lp + 2
        for k in range(len(grids)):
            assert np.array_equal(pouts[k].numpy(), ref[k]), k
            assert np.array_equal(srcs[k].numpy(), psis[k])          # inputs untouched
        # page-locked, in place
        b.step_host(srcs, 0.1, 5, 1e-3, "ts2", outs=srcs)
        for k in range(len(grids)):
            assert np.array_equal(srcs[k].numpy(), ref[k]), k
        # one pageable output among page-locked buffers
        mixed = list(pouts)
        mixed[2] = np.empty(psis[2].shape, dtype=np.complex64)
        srcs = [torch.from_numpy(p.copy()).pin_memory() for p in psis]
        l0 = b.launch_count()
        b.step_host(srcs, 0.1, 5, 1e-3, "ts2", outs=mixed)
        assert b.launch_count() - l0 == lp
        assert np.array_equal(mixed[2], ref[2])
        assert np.array_equal(mixed[4].numpy(), ref[4])
