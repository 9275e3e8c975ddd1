"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI:
the largest line length along each axis, the FP32 nonlinear flow on both
sides of its small-angle switches, and the persistent ensemble kernel at
its largest line lengths.
"""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu


def _run(n, L, prm, psi, steps, dt, scheme, prec):
    c = sgp.Context(n, L, batch=1, prec=prec)
    c.set_params(**prm)
    c.set_state(np.ascontiguousarray(psi[None].astype(c.dtype)), 0.0)
    c.step(steps, dt, scheme)
    out = c.get_state()[0].astype(np.complex128)
    c.close()
    return out


@pytest.mark.parametrize("n,L", [((1024, 48), (16.0, 6.0)), ((48, 1024), (6.0, 16.0)),
                                 ((16, 16, 256), (4.0, 4.0, 12.0))])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-5)])
def test_largest_line_length_along_each_axis(n, L, prec, tol):
    """N = 1024 (the longest compiled line) along x (the x-pass) and along y
    (the line pass with the mix); N = 256 along z in 3D."""
    prm = dict(omega=0.5, gamma=1.2, c0=80.0, c1=-2.0, c2=3.0, gx=1.1, gy=0.9, gz=1.3)
    psi = inputs.gaussian_random_phase(n, L, seed=31, amp=0.3)
    out = _run(n, L, prm, psi, 3, 2e-3, "ts4", prec)
    ref = O.Propagator(O.Grid(n, L), O.Params(**prm)).run(psi, 0.0, 2e-3, 3, "ts4")[0]
    assert O.rel_l2(out, ref) < tol, O.rel_l2(out, ref)


@pytest.mark.parametrize("c1,c2,delta", [
    (-1.0, 1.0, 1e-3),       # spin rotation |K| << 3.5e-3: the Taylor form, singlet series
    (-40.0, 1.0, 0.02),      # |K| well above the switch: the exact SU(2) form
    (0.0, 0.0, 0.01),        # no spin and no singlet terms: only the phase
    (-3.0, 60.0, 0.02),      # singlet angle above the series range: the square-root form
])
def test_fp32_nonlinear_substep_on_both_sides_of_the_switches(c1, c2, delta):
    """One FP32 nonlinear substep against the FP64 oracle to FP32 accuracy on a
    field whose local spin density varies over the grid, so that some warps
    take the small-angle forms and some the exact ones.  The tolerance is
    FP32 rounding of angles up to a few radians (the input is rounded to FP32
    on both sides)."""
    n, L = (64, 64), 6.0
    prm = dict(omega=0.3, gamma=0.0, c0=50.0, c1=c1, c2=c2, gx=1.2, gy=0.8, gz=1.0)
    psi = inputs.gaussian_random_phase(n, L, seed=41, amp=1.0) * 2.0
    c = sgp.Context(n, L, prec="f32")
    c.set_params(**prm)
    c.set_state(psi[None].astype(np.complex64).copy(), 0.4)
    c.substep("nonlinear", delta)
    out = c.get_state()[0].astype(np.complex128)
    c.close()
    ref = O.nonlinear_substep(psi.astype(np.complex64).astype(np.complex128), O.Grid(n, L),
                              O.Params(**prm), delta, 0.4)
    assert O.rel_l2(out, ref) < 2e-6, O.rel_l2(out, ref)


def test_persistent_kernel_at_its_largest_line_lengths():
    """Members of 384^2 and 512^2 (the largest sides the persistent kernel is
    compiled for) beside a 64^2 one: bit for bit the per-group launches."""
    grids = [((512, 512), 16.0), ((384, 384), 12.0), ((64, 64), 8.0), ((512, 512), 16.0)]
    prms = [dict(omega=0.9, gamma=1.5, c0=1000.0, c1=-5.0, c2=10.0),
            dict(omega=0.4, gamma=0.7, c0=300.0, c1=2.0, c2=1.0),
            dict(omega=0.2, gamma=1.0, c0=100.0, c1=-1.0, c2=1.0),
            dict(omega=0.6, gamma=0.2, c0=800.0, c1=-3.0, c2=4.0)]
    out = []
    for persistent in (True, False):
        ens = sgp.Ensemble(grids, prec="f32")
        ens.set_params(prms)
        if not persistent:
            ens.set_persistent(False)
        assert ens.persistent == persistent
        for i, (n, L) in enumerate(grids):
            ens.set_member_state(i, inputs.gaussian_random_phase(n, L, seed=50 + i, amp=0.01)
                                 .astype(np.complex64))
        ens.step(66, 5e-4, "ts4")
        out.append([ens.get_member_state(i) for i in range(len(grids))])
        ens.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
