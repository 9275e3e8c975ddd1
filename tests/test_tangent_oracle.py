"""Pins of the tangent-linear oracle gradient (oracle/sgp_tangent.py).

It is a second, independent FP64 oracle gradient: forward-mode dual numbers
through the oracle's substeps, against the central finite differences of
oracle/sgp_grad.py (which it must match to their truncation error, and which
must converge to it at second order), a block-matrix exponential for the
derivative of the per-mode matrix of Sec. 3.1, the closed form of the
objective's gradient with no steps, and the invariance of J under a global
phase.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import sgp_grad as G
from oracle import sgp_oracle as O
from oracle import sgp_tangent as TL
from paper_2603_25282_gb300 import inputs

PRM = O.Params(omega=0.6, gamma=1.0, c0=400.0, c1=-3.0, c2=5.0, gx=1.0, gy=1.3)


def _setup(n, L, seed):
    psi0 = inputs.gaussian_random_phase(n, L, seed=seed, amp=0.3)
    c, w = inputs.density_target(n, L, seed=seed + 1)
    return psi0, c, w


def test_dual_forward_pass_reproduces_the_oracle():
    n, L = (16, 16), 8.0
    psi0, c, w = _setup(n, L, 31)
    grid = O.Grid(n, L)
    J, _ = TL.directional_derivative(psi0, grid, PRM, 2e-3, 4, "ts4", c, w)
    ref = G.objective(psi0, grid, PRM, 2e-3, 4, "ts4", c, w)
    assert abs(J - ref) <= 1e-12 * abs(ref)


def test_daleckii_krein_equals_block_matrix_exponential():
    """d exp(i delta Q)[dQ] is the upper-right block of exp of the block
    matrix [[i delta Q, i delta dQ], [0, i delta Q]] (scipy.linalg.expm)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(5)
    for k in range(6):
        nup, nuq = rng.uniform(-5, 5, size=2)
        Om, ga = rng.uniform(-1.5, 1.5), rng.uniform(-2, 2)
        if k == 0:
            Om = 0.0              # lambda = 0 at the origin mode: degenerate spectrum
            nup = nuq = 0.0
        Q = O.q_matrix(nup, nuq, Om, ga)
        dQ = 0.7 * O.q_matrix(nup, nuq, 1.0, 0.0) - 0.4 * O.q_matrix(nup, nuq, 0.0, 1.0)
        delta = rng.uniform(-0.4, 0.4)
        E, dE = TL.expm_hermitian_tangent(Q, dQ, delta)
        Z = np.zeros((10, 10), complex)
        Z[:5, :5] = Z[5:, 5:] = 1j * delta * Q
        Z[:5, 5:] = 1j * delta * dQ
        B = scipy_linalg.expm(Z)
        assert np.abs(E - B[:5, :5]).max() < 1e-13
        assert np.abs(dE - B[:5, 5:]).max() < 1e-13


@pytest.mark.parametrize("scheme,nsteps", [("ts2", 5), ("ts4", 3), ("ts2_lnl", 4), ("ts4_l", 3)])
def test_tangent_matches_central_differences_2d(scheme, nsteps):
    n, L, dt = (16, 16), 8.0, 2e-3
    psi0, c, w = _setup(n, L, 41)
    grid = O.Grid(n, L)
    rng = np.random.default_rng(42)
    dirs = [rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape) for _ in range(2)]
    tl_d, tl_p = TL.gradient_tangent(psi0, grid, PRM, dt, nsteps, scheme, c, w, directions=dirs)
    fd_d, fd_p = G.gradient_fd(psi0, grid, PRM, dt, nsteps, scheme, c, w, directions=dirs,
                               params=TL.PARAMS)
    for a, b in zip(tl_d, fd_d):
        assert abs(a - b) <= 1e-6 * abs(b), (a, b)
    scale = max(abs(v) for v in fd_p.values())
    for name in TL.PARAMS:
        assert abs(tl_p[name] - fd_p[name]) <= 1e-7 * scale, (name, tl_p[name], fd_p[name])


def test_tangent_matches_central_differences_3d():
    n, L, dt = (8, 8, 8), 5.0, 2e-3
    prm = dataclasses.replace(PRM, gz=1.7)
    psi0, c, w = _setup(n, L, 51)
    grid = O.Grid(n, L)
    V = np.random.default_rng(52).standard_normal(psi0.shape) * (1 + 0.5j)
    tl_d, tl_p = TL.gradient_tangent(psi0, grid, prm, dt, 3, "ts2", c, w, directions=[V])
    fd_d, fd_p = G.gradient_fd(psi0, grid, prm, dt, 3, "ts2", c, w, directions=[V],
                               params=TL.PARAMS)
    assert abs(tl_d[0] - fd_d[0]) <= 1e-6 * abs(fd_d[0])
    scale = max(abs(v) for v in fd_p.values())
    for name in TL.PARAMS:
        assert abs(tl_p[name] - fd_p[name]) <= 1e-7 * scale, name


def test_central_differences_converge_to_tangent_at_second_order():
    """FD(h) - tangent = O(h^2): halving h divides the gap by about 4, for a
    parameter and for a state direction (the 1e-6 tolerance above is the
    FD truncation error at h = 1e-5, not a gap in the tangent)."""
    n, L, dt = (16, 16), 8.0, 2e-3
    psi0, c, w = _setup(n, L, 61)
    grid = O.Grid(n, L)
    _, exact = TL.directional_derivative(psi0, grid, PRM, dt, 4, "ts2", c, w, dprm={"omega": 1.0})

    def J(om):
        return G.objective(psi0, grid, dataclasses.replace(PRM, omega=om), dt, 4, "ts2", c, w)
    gaps = []
    for h in (0.04, 0.02):
        fd = (J(PRM.omega + h) - J(PRM.omega - h)) / (2 * h)
        gaps.append(abs(fd - exact))
    assert 3.5 < gaps[0] / gaps[1] < 4.5, gaps
    V = np.random.default_rng(62).standard_normal(psi0.shape) * (1 - 1j)
    _, exact = TL.directional_derivative(psi0, grid, PRM, dt, 4, "ts2", c, w, dPhi0=V)

    def Js(P):
        return G.objective(P, grid, PRM, dt, 4, "ts2", c, w)
    gaps = [abs(G.fd_state(Js, psi0, V, h) - exact) for h in (4e-4, 2e-4)]
    assert 3.5 < gaps[0] / gaps[1] < 4.5, gaps


def test_global_phase_direction_has_zero_derivative():
    n, L = (16, 16), 8.0
    psi0, c, w = _setup(n, L, 71)
    grid = O.Grid(n, L)
    _, d = TL.directional_derivative(psi0, grid, PRM, 2e-3, 4, "ts4", c, w, dPhi0=1j * psi0)
    _, ref = TL.directional_derivative(psi0, grid, PRM, 2e-3, 4, "ts4", c, w, dPhi0=psi0)
    assert abs(d) < 1e-11 * abs(ref)


def test_no_steps_closed_form():
    """With zero steps J = h^d sum (|phi|^2 - rho_l(R(T) x))^2 at T = t0:
    dJ along V is Re sum conj(4 h^d (|phi|^2 - tgt) phi) V, and dJ/dOmega
    comes from the target's frame alone."""
    n, L, T = (16, 16), 8.0, 0.3
    psi0, c, w = _setup(n, L, 81)
    grid = O.Grid(n, L)
    V = np.random.default_rng(82).standard_normal(psi0.shape) + 0.3j
    _, d = TL.directional_derivative(psi0, grid, PRM, 1e-3, 0, "ts2", c, w, dPhi0=V, t0=T)
    tgt = G.target_density(grid, PRM.omega, T, c, w)
    g = 4.0 * grid.cell * (np.abs(psi0) ** 2 - tgt) * psi0
    assert abs(d - float(np.real(np.vdot(g, V)))) < 1e-12 * abs(d)
    _, dom = TL.directional_derivative(psi0, grid, PRM, 1e-3, 0, "ts2", c, w, dprm={"omega": 1.0}, t0=T)
    X = grid.coords()
    co, si = math.cos(PRM.omega * T), math.sin(PRM.omega * T)
    Y = G.rotated_coords(grid, PRM.omega, T)
    dY = [T * (-si * X[0] + co * X[1]), T * (-co * X[0] - si * X[1])]
    dtgt = np.stack([tgt[m] * sum(-2.0 * (Y[a] - c[m][a]) * dY[a] for a in range(2)) for m in range(5)])
    ref = grid.cell * float(np.sum(-2.0 * (np.abs(psi0) ** 2 - tgt) * dtgt))
    assert abs(dom - ref) < 1e-12 * abs(ref)
    for name in ("gamma", "c0", "c1", "c2"):
        assert TL.directional_derivative(psi0, grid, PRM, 1e-3, 0, "ts2", c, w,
                                         dprm={name: 1.0}, t0=T)[1] == 0.0
