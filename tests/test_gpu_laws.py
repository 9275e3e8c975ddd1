"""Dynamical laws of Sec. 2 on the GPU path, Example 3 set-up: c = (120, 1, 1),
Omega = 0.2, the Example 3 initial data, [-24, 24]^2, TS4 with tau = 1e-3 up
to t = 12, FP32 fields (FP64 sums), observables every 10 steps, on the
example's grid h = 1/16 (N = 768 = 3 * 256).  Three cases, as in the paper's
example:

  (i)   gamma = 0, isotropic trap: mass, magnetization and <L_z> conserved;
        delta_r(t) follows Eq. (delta_r) (real radially symmetric data, so
        its first derivative at 0 vanishes) and delta_x = delta_y;
  (ii)  gamma = 0.9: mass and energy conserved; dM/dt from central
        differences of the series equals the magnetization law evaluated on
        the state;
  (iii) gamma = 0, gamma_x = 1.3: mass and magnetization conserved;
        d<L_z>/dt equals (gamma_x^2 - gamma_y^2) int x y rho (Lemma, lab
        coordinates).

Tolerances are FP32-level: mass to 1e-5 relative over the 12 000 steps
(the FP32 bound of the method's FP32 form is a mass drift of 1e-5 per 1000
steps, so this is 12 times tighter), magnetization to 5e-6 of the mass,
laws to 2e-3 of the rate's scale (central differences over 0.02 in time),
sums in FP64.
"""
import math

import numpy as np
import pytest

from paper_2603_25282_gb300 import inputs, sgp
from tests import lab_rk4

pytestmark = pytest.mark.gpu

N, L, TAU, T_END, EVERY = 768, 24.0, 1e-3, 12.0, 10
S6H = math.sqrt(6.0) / 2.0


def _series(gamma, gx, probe_times=()):
    prm = dict(omega=0.2, gamma=gamma, c0=120.0, c1=1.0, c2=1.0, gx=gx, gy=1.0)
    c = sgp.Context((N, N), L, prec="f32")
    c.set_params(**prm)
    psi0 = inputs.ini_example3((N, N), L)
    c.set_state(psi0[None].astype(np.complex64).copy(), 0.0)
    obs = [c.observables()[0]]
    states = {}
    nsteps = int(round(T_END / TAU))
    probe_steps = {int(round(t / TAU)): t for t in probe_times}
    for s in range(EVERY, nsteps + 1, EVERY):
        c.step(EVERY, TAU, "ts4")
        obs.append(c.observables()[0])
        if s in probe_steps:
            states[probe_steps[s]] = c.get_state()[0].astype(np.complex128)
    c.close()
    t = np.array([o["t"] for o in obs])
    return prm, t, obs, states


def _col(obs, key):
    return np.array([o[key] for o in obs])


def _rate(t, y, tp):
    k = int(np.argmin(np.abs(t - tp)))
    return (y[k + 1] - y[k - 1]) / (t[k + 1] - t[k - 1])


@pytest.fixture(scope="module")
def case_i():
    return _series(0.0, 1.0)


def test_case_i_conservation(case_i):
    prm, t, obs, _ = case_i
    mass = _col(obs, "mass")
    assert np.abs(mass / mass[0] - 1).max() < 1e-5
    M = _col(obs, "magnetization")
    assert np.abs(M - M[0]).max() < 5e-6 * mass[0]
    lz = _col(obs, "lz")
    assert np.abs(lz - lz[0]).max() < 1e-5
    e = _col(obs, "energy")
    assert np.abs(e / e[0] - 1).max() < 1e-5


def test_case_i_width_law(case_i):
    prm, t, obs, _ = case_i
    wx = _col(obs, "width2")[:, 0]
    wy = _col(obs, "width2")[:, 1]
    dr = wx + wy
    e0, lz0 = obs[0]["energy"], obs[0]["lz"]
    law = (e0 + prm["omega"] * lz0) * (1 - np.cos(2 * t)) + dr[0] * np.cos(2 * t)
    assert np.abs(dr - law).max() < 1e-4 * np.abs(law).max()
    assert np.abs(wx - wy).max() < 1e-5 * dr.max()
    # period pi of the breathing mode (twice the trap frequency)
    assert dr.max() > 1.01 * dr.min()


def test_case_ii_magnetization_law():
    probes = (1.0, 4.0, 8.0)
    prm, t, obs, states = _series(0.9, 1.0, probes)
    mass = _col(obs, "mass")
    assert np.abs(mass / mass[0] - 1).max() < 1e-5
    e = _col(obs, "energy")
    assert np.abs(e / e[0] - 1).max() < 1e-4
    M = _col(obs, "magnetization")
    h = 2.0 * L / N

    def Lminus(f):
        dx, dy = lab_rk4.grad(f, L, L)
        return 1j * dy - dx
    cj = np.conj
    scale = np.abs(np.diff(M) / np.diff(t)).max()
    assert scale > 1e-3                          # the magnetization does move
    for tp in probes:
        phi = states[tp]
        dens = (cj(phi[0]) * Lminus(phi[1]) - phi[4] * Lminus(cj(phi[3]))
                + S6H * cj(phi[1]) * Lminus(phi[2]) - S6H * phi[3] * Lminus(cj(phi[2])))
        law = 2 * prm["gamma"] * np.real(1j * h * h * np.sum(dens))
        rate = _rate(t, M, tp)
        assert abs(rate - law) < 2e-3 * scale, (tp, rate, law)


def test_case_iii_angular_momentum_law():
    probes = (1.0, 4.0, 8.0)
    prm, t, obs, states = _series(0.0, 1.3, probes)
    mass = _col(obs, "mass")
    assert np.abs(mass / mass[0] - 1).max() < 1e-5
    M = _col(obs, "magnetization")
    assert np.abs(M - M[0]).max() < 5e-6 * mass[0]
    lz = _col(obs, "lz")
    h = 2.0 * L / N
    x = -L + h * np.arange(N)
    X, Y = np.meshgrid(x, x, indexing="xy")
    scale = np.abs(np.diff(lz) / np.diff(t)).max()
    assert scale > 1e-3
    for tp in probes:
        phi = states[tp]
        co, si = math.cos(prm["omega"] * tp), math.sin(prm["omega"] * tp)
        xl, yl = co * X + si * Y, -si * X + co * Y
        rho = np.sum(np.abs(phi) ** 2, axis=0)
        law = (prm["gx"] ** 2 - 1.0) * h * h * np.sum(xl * yl * rho)
        rate = _rate(t, lz, tp)
        assert abs(rate - law) < 2e-3 * scale, (tp, rate, law)
