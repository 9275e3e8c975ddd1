"""sgp_observables_static, the allocation-free observables entry point,
against the context-based sgp_observables.

The entry point serves callers that cannot allocate device memory when they
need the observables: their device memory is reserved by another
allocator's pool, or they run on a path where cudaMalloc's implicit device
synchronisation is not acceptable.  It keeps all of its scratch in
fixed-size device arrays inside the library, shared by every call, so the
test makes calls in a row with different shapes and precisions: what one
call leaves in the scratch must not leak into the next.

The test holds on its own: it passes alone in a fresh process and after
the other tests (the first call on the device is the entry point's set-up,
made inside the test).  The file name puts it last in a run.
"""
import numpy as np
import pytest

from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu

KEYS = ("mass", "energy", "magnetization", "lz", "e_kin", "e_pot", "e_rot", "e_int", "e_soc")
PRM = dict(omega=0.4, gamma=0.8, c0=30.0, c1=-2.0, c2=3.0, gx=1.2, gy=0.9, gz=1.5)


def _reference(n, L, batch, prec, fields, t):
    """Observables of the same fields through a context (sgp_observables)."""
    with sgp.Context(n, L, batch=batch, prec=prec) as c:
        c.set_params(**PRM)
        c.set_state(np.ascontiguousarray(fields), t)
        return c.observables()


def _static(n, L, batch, prec, dev, t):
    return sgp.observables_static(n, L, dev.data_ptr(), batch=batch, prec=prec, t=t,
                                  device=0, stream=None, **PRM)


def _fields(n, L, batch, prec, seed):
    dt = np.complex64 if prec == "f32" else np.complex128
    f = np.stack([inputs.gaussian_random_phase(n, L, seed=seed + m, amp=1.0) for m in range(batch)])
    f[:, 0] *= 1.3
    return f.astype(dt)


def _check(got, ref):
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        for k in KEYS:
            assert abs(g[k] - r[k]) < 1e-10 * max(1.0, abs(r[k])), (k, g[k], r[k])
        for a, b in zip(g["comp_mass"], r["comp_mass"]):
            assert abs(a - b) < 1e-12 * max(1.0, abs(b))
        for a, b in zip(g["width2"], r["width2"]):
            assert abs(a - b) < 1e-10 * max(1.0, abs(b))


def test_static_observables_match_context_and_allocate_nothing():
    """Calls in a row, with different shapes and precisions, each made twice,
    match the context observables; after the first call on the device (the
    set-up, which loads the kernels and the fixed scratch) the device's free
    memory does not change across the calls, and sgp_last_error(NULL) is
    empty after each successful call."""
    torch = pytest.importorskip("torch")
    cases = [
        ((64, 64), 8.0, 2, "f64", 0.7),
        ((48, 96), (6.0, 9.0), 1, "f32", 0.3),
        ((16, 32, 16), (4.0, 5.0, 4.0), 3, "f64", 0.2),
        ((128, 128), 8.0, 4, "f32", 0.5),
        ((64, 64), 8.0, 2, "f64", 0.7),
    ]
    # references through contexts, and every device field, before measuring
    refs, devs = [], []
    for i, (n, L, batch, prec, t) in enumerate(cases):
        f = _fields(n, L, batch, prec, seed=40 + 10 * i)
        refs.append(_reference(n, L, batch, prec, f, t))
        devs.append(torch.from_numpy(np.ascontiguousarray(f)).to("cuda:0"))
    torch.cuda.synchronize()
    n, L, batch, prec, t = cases[0]
    _check(_static(n, L, batch, prec, devs[0], t), refs[0])      # set-up call
    free0 = torch.cuda.mem_get_info(0)[0]
    for (n, L, batch, prec, t), dev, ref in zip(cases, devs, refs):
        for _ in range(2):
            _check(_static(n, L, batch, prec, dev, t), ref)
            assert sgp.lib().sgp_last_error(None).decode() == ""
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0


def test_static_observables_reject_oversized_requests():
    """Both requests are refused by the size checks before any kernel runs
    (the buffer passed is real but far too small for them)."""
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        sgp.observables_static((64, 64), 8.0, buf.data_ptr(), batch=65, prec="f64")
    with pytest.raises(sgp.SgpError, match="EINVAL"):          # > 2^19 partial sums
        sgp.observables_static((1024, 1024, 1024), 8.0, buf.data_ptr(), batch=1, prec="f64")
