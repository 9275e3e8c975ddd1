"""Pins of the oracle's lab-frame mapping (Eqs. (RSDA1), (RSDA2)) and of the
rotating-frame reading of Algorithm 1 (CPU only).

* the rotation by shears against a Gaussian rotated in closed form, in every
  quadrant (quarter turns + shears), in 2D and about z in 3D;
* exact unitarity of the mapping;
* RSDA1 undoes RSDA2;
* the printed Algorithm 1, run literally in the lab frame (mapping in and
  out every step, trap V(x)), against the rotating-frame oracle mapped to
  the lab frame at the end: the two agree to spectral accuracy with an
  anisotropic trap, which pins the frame reading (the nonlinear flow takes
  V(R(t)x) in the rotating frame).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs


def _gauss(X, c, k):
    r2 = sum((x - cc) ** 2 for x, cc in zip(X, c))
    return np.exp(-r2) * np.exp(1j * k * X[0])


@pytest.mark.parametrize("theta", [0.3, -0.7, 1.2, 2.9, -2.2, 4.5, math.pi / 4, -math.pi / 4])
def test_rotation_by_shears_matches_closed_form_2d(theta):
    g = O.Grid((64, 64), 8.0)
    X = g.coords()
    f = _gauss(X, (0.7, -0.4), 0.3)
    out = O.rotate_rsda(np.stack([f] * 5), g, theta)
    c, s = math.cos(theta), math.sin(theta)
    Y = (c * X[0] - s * X[1], s * X[0] + c * X[1])
    assert np.abs(out[0] - _gauss(Y, (0.7, -0.4), 0.3)).max() < 1e-13


def test_rotation_by_shears_3d_about_z():
    g = O.Grid((64, 64, 16), (8.0, 8.0, 5.0))
    X = g.coords()
    f = _gauss(X, (0.5, 0.2, -0.3), 0.2)
    th = 2.4
    out = O.rotate_rsda(np.stack([f] * 5), g, th)
    c, s = math.cos(th), math.sin(th)
    Y = (c * X[0] - s * X[1], s * X[0] + c * X[1], X[2])
    assert np.abs(out[2] - _gauss(Y, (0.5, 0.2, -0.3), 0.2)).max() < 1e-12


def test_mapping_is_unitary_and_rsda1_inverts_rsda2():
    g = O.Grid((64, 64), 8.0)
    rng = np.random.default_rng(1)
    noise = rng.standard_normal((5, 64, 64)) + 1j * rng.standard_normal((5, 64, 64))
    lab = O.lab_frame_field(noise, g, 0.9, 1.7)
    assert abs(np.vdot(lab, lab).real / np.vdot(noise, noise).real - 1.0) < 1e-13
    phi = inputs.gaussian_random_phase((64, 64), 8.0, seed=3, amp=0.01)
    for t in (0.4, 1.7, 3.1):           # no quarter turn, one, two
        back = O.rotating_frame_field(O.lab_frame_field(phi, g, 0.9, t), g, 0.9, t)
        assert O.rel_l2(back, phi) < 1e-12


def test_lab_phase_factor():
    # a state concentrated in one component picks up exp(i l Omega t)
    g = O.Grid((64, 64), 8.0)
    X = g.coords()
    f = np.exp(-0.5 * (X[0] ** 2 + X[1] ** 2))    # radial: rotation leaves it
    Phi = np.zeros((5, 64, 64), complex)
    for comp in range(5):
        Phi[comp] = f
    lab = O.lab_frame_field(Phi, g, 0.5, 0.8)
    for comp, l in enumerate((2, 1, 0, -1, -2)):
        assert np.abs(lab[comp] - np.exp(1j * l * 0.4) * f).max() < 1e-13


def _algorithm1_vs_rotating(prm, nsteps, tau=5e-3, n=(64, 64), L=8.0):
    g = O.Grid(n, L)
    psi0 = inputs.gaussian_random_phase(n, L, seed=7, amp=0.3)
    lab = psi0.copy()
    props = O.mode_propagators(g, prm, tau)
    t = 0.0
    for _ in range(nsteps):
        lab = O.algorithm1_lab_step(lab, g, prm, t, tau, props)
        t += tau
    rot, T = O.Propagator(g, prm).run(psi0, 0.0, tau, nsteps, "ts2")
    return O.rel_l2(O.lab_frame_field(rot, g, prm.omega, T), lab), O.rel_l2(rot, lab)


PRM_A1 = O.Params(omega=0.8, gamma=0.6, c0=60.0, c1=-1.5, c2=2.0, gx=1.0, gy=1.3)


def test_algorithm1_in_the_lab_frame_matches_the_rotating_frame():
    # linear flow and the anisotropic trap over 40 steps: the mapping in and
    # out every step is exact to rounding for this smooth state
    lin = dataclasses.replace(PRM_A1, c0=0.0, c1=0.0, c2=0.0)
    err, frame = _algorithm1_vs_rotating(lin, 40)
    assert err < 1e-11
    assert frame > 1e-2            # without the final mapping they differ at O(1)
    # the full flow: agreement to spectral accuracy over a few steps (the
    # nonlinear phase builds fine structure that the per-step
    # re-interpolation of the literal algorithm resolves less well over
    # many steps at this grid)
    err, _ = _algorithm1_vs_rotating(PRM_A1, 2)
    assert err < 1e-9
