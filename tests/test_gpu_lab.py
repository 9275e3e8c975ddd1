"""Lab-frame output (sgp_get_state_lab, Eq. (RSDA2)) against the oracle's
mapping: every quadrant of the rotation angle (quarter turns + shears), FP64
to 1e-12 and FP32 to 1e-5 relative l2, 3D about z, per-member Omega, after
propagation, and the square-grid rule for quarter turns.
"""
import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu


def _lab(n, L, prec, omega, t, psi, batch_psis=None, omegas=None):
    batch = 1 if batch_psis is None else len(batch_psis)
    c = sgp.Context(n, L, prec=prec, batch=batch)
    if omegas is None:
        c.set_params(omega=omega, gamma=1.0)
    else:
        c.set_params_batch([dict(omega=w, gamma=1.0) for w in omegas])
    dt = np.complex64 if prec == "f32" else np.complex128
    src = (psi[None] if batch_psis is None else np.stack(batch_psis)).astype(dt)
    c.set_state(src.copy(), t)
    out = c.get_state_lab().astype(np.complex128)
    assert np.array_equal(c.get_state(), src)          # the state is untouched
    c.close()
    return out


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("t", [0.3, 1.2, 2.5, 4.4, 7.7])
def test_lab_frame_2d_every_quadrant(prec, tol, t):
    n, L, omega = (64, 64), 8.0, 0.9
    psi = inputs.gaussian_random_phase(n, L, seed=1, amp=0.01)
    out = _lab(n, L, prec, omega, t, psi)[0]
    ref = O.lab_frame_field(psi, O.Grid(n, L), omega, t)
    assert O.rel_l2(out, ref) < tol


@pytest.mark.parametrize("n,L", [((96, 96), 9.0), ((128, 128), 10.0)])
def test_lab_frame_radix3_and_larger_f64(n, L):
    psi = inputs.gaussian_random_phase(n, L, seed=2, amp=0.3)
    out = _lab(n, L, "f64", 0.7, 3.3, psi)[0]
    ref = O.lab_frame_field(psi, O.Grid(n, L), 0.7, 3.3)
    assert O.rel_l2(out, ref) < 1e-12


def test_lab_frame_3d_about_z():
    n, L = (32, 32, 16), (6.0, 6.0, 5.0)
    psi = inputs.gaussian_random_phase(n, L, seed=3, amp=0.01)
    out = _lab(n, L, "f64", 0.8, 2.6, psi)[0]
    ref = O.lab_frame_field(psi, O.Grid(n, L), 0.8, 2.6)
    assert O.rel_l2(out, ref) < 1e-12


def test_lab_frame_per_member_omega():
    n, L = (64, 64), 8.0
    psis = [inputs.gaussian_random_phase(n, L, seed=s, amp=0.01) for s in (4, 5, 6)]
    omegas = [0.2, 0.9, -0.6]
    out = _lab(n, L, "f64", None, 2.0, None, psis, omegas)
    for m in range(3):
        ref = O.lab_frame_field(psis[m], O.Grid(n, L), omegas[m], 2.0)
        assert O.rel_l2(out[m], ref) < 1e-12


def test_lab_frame_after_propagation():
    n, L = (64, 64), 8.0
    prm = dict(omega=0.9, gamma=1.0, c0=100.0, c1=-1.0, c2=1.0, gx=1.0, gy=1.2, gz=1.0)
    psi = inputs.gaussian_random_phase(n, L, seed=7, amp=0.01)
    c = sgp.Context(n, L, prec="f64")
    c.set_params(**prm)
    c.set_state(psi[None].copy(), 0.0)
    c.step(200, 1e-2, "ts4")
    out = c.get_state_lab()[0]
    c.close()
    rot, T = O.Propagator(O.Grid(n, L), O.Params(**prm)).run(psi, 0.0, 1e-2, 200, "ts4")
    ref = O.lab_frame_field(rot, O.Grid(n, L), prm["omega"], T)
    assert O.rel_l2(out, ref) < 1e-10


def test_lab_frame_rectangular_grid():
    n, L = (64, 48), (8.0, 6.0)
    psi = inputs.gaussian_random_phase(n, L, seed=8, amp=0.01)
    # |Omega t| = 0.5 < pi/4: shears only, any grid
    out = _lab(n, L, "f64", 0.5, 1.0, psi)[0]
    ref = O.lab_frame_field(psi, O.Grid(n, L), 0.5, 1.0)
    assert O.rel_l2(out, ref) < 1e-12
    # a quarter turn is needed: refused on a non-square grid
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        _lab(n, L, "f64", 0.5, 4.0, psi)
