"""Caller-supplied device allocator (sgp_set_allocator) with PyTorch's
caching allocator: contexts take their memory from torch's pool and give it
back on destroy, results are bit-identical to the cudaMalloc path, the
adjoint's checkpoints come from the pool too, and an allocator that fails
makes creation return SGP_ENOMEM.  The default allocator is restored after
every test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu

PRM = dict(omega=0.6, gamma=1.0, c0=200.0, c1=-2.0, c2=3.0, gx=1.0, gy=1.2)


def _run(n, L, psi, steps):
    c = sgp.Context(n, L, prec="f32")
    c.set_params(**PRM)
    c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
    c.step(steps, 1e-3, "ts4")
    out = c.get_state()
    c.close()
    return out


def test_torch_pool_owns_the_context_memory():
    n, L = (256, 256), 8.0
    psi = inputs.gaussian_random_phase(n, L, seed=1, amp=0.01)
    ref = _run(n, L, psi, 130)                       # cudaMalloc path (graphs included)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    try:
        sgp.use_torch_allocator(True)
        c = sgp.Context(n, L, prec="f32")
        grown = torch.cuda.memory_allocated() - base
        assert grown >= 5 * n[0] * n[1] * 8          # at least the field
        c.set_params(**PRM)
        c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
        c.step(130, 1e-3, "ts4")
        assert torch.cuda.memory_allocated() - base > grown   # tables from the pool too
        out = c.get_state()
        c.close()
        assert torch.cuda.memory_allocated() == base  # all of it given back
    finally:
        sgp.use_torch_allocator(False)
    assert np.array_equal(out, ref)


def test_torch_pool_serves_the_adjoint_checkpoints():
    n, L = (64, 64), 8.0
    psi = inputs.gaussian_random_phase(n, L, seed=2, amp=0.3)
    rng = np.random.default_rng(3)
    gT = (rng.standard_normal((1, 5) + n) + 1j * rng.standard_normal((1, 5) + n)).astype(np.complex64)
    res = []
    for torch_pool in (False, True):
        try:
            sgp.use_torch_allocator(torch_pool)
            c = sgp.Context(n, L, prec="f32")
            c.set_params(**PRM)
            c.set_state(psi[None].astype(np.complex64).copy(), 0.0)
            before = torch.cuda.memory_allocated()
            c.record(50, 1e-3, "ts2")
            res.append(c.backward(gT))
            if torch_pool:
                assert torch.cuda.memory_allocated() > before
            c.close()
        finally:
            sgp.use_torch_allocator(False)
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_failing_allocator_reports_enomem():
    calls = []

    def _alloc(size, device, stream, user):
        calls.append(size)
        return None

    keep = (sgp.ALLOC_FN(_alloc), sgp.FREE_FN(lambda *a: None))
    try:
        assert sgp.lib().sgp_set_allocator(keep[0], keep[1], None) == 0
        with pytest.raises(sgp.SgpError, match="ENOMEM"):
            sgp.Context((64, 64), 8.0, prec="f32")
        assert calls
    finally:
        sgp.use_torch_allocator(False)
    c = sgp.Context((64, 64), 8.0, prec="f32")     # the default is back
    c.close()


def test_misaligned_allocator_block_is_refused_and_freed():
    """A block that is not 16-byte aligned is handed back at once and the
    creation fails as for a failed allocation; no kernel touches it."""
    held, freed = {}, []

    def _alloc(size, device, stream, user):
        t = torch.empty(size + 64, dtype=torch.uint8, device="cuda:%d" % device)
        p = t.data_ptr() + 8
        held[p] = t
        return p

    def _free(p, device, stream, user):
        freed.append(p)
        held.pop(p, None)

    keep = (sgp.ALLOC_FN(_alloc), sgp.FREE_FN(_free))
    try:
        assert sgp.lib().sgp_set_allocator(keep[0], keep[1], None) == 0
        with pytest.raises(sgp.SgpError, match="ENOMEM.*misaligned"):
            sgp.Context((64, 64), 8.0, prec="f32")
        assert freed and not held
    finally:
        sgp.use_torch_allocator(False)
