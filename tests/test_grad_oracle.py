"""Pins of the FP64 oracle gradient and of the identities the adjoint kernels
rest on (CPU only).

The oracle gradient (oracle/sgp_grad.py) is a central finite difference of
the oracle propagator.  It is pinned against a closed form, against its own
second-order convergence and against the global-phase invariance of J.  The
identity pins check, on the oracle's substeps, the facts the hand-written
adjoint uses: time reversal of both flows, the symplectic form of the
nonlinear flow's vector-Jacobian product, the parameter derivatives of the
nonlinear flow as vector fields at its output (its four parts commute), and
the derivative of exp(i a.f) used for the linear flow's Omega and gamma.
"""
import dataclasses
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import sgp_grad as G
from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs

PRM = O.Params(omega=0.6, gamma=1.0, c0=400.0, c1=-1.0, c2=2.0, gx=1.0, gy=1.0)
PRM_ANISO = dataclasses.replace(PRM, gy=1.3, c1=-3.0, c2=7.0)


def _setup(n=16, L=8.0, seed=5):
    grid = O.Grid((n, n), L)
    psi0 = inputs.gaussian_random_phase((n, n), L, seed=seed, amp=0.3)
    centres, weights = inputs.density_target((n, n), L, seed=seed + 1)
    return grid, psi0, centres, weights


def _rand_dir(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_target_mass_is_one():
    grid, _, c, w = _setup()
    tgt = G.target_density(grid, 0.0, 0.0, c, w)
    assert abs(grid.cell * tgt.sum() - 1.0) < 1e-12


def test_fd_matches_closed_form_without_steps():
    # J(Phi) with no steps: dJ/dRe + i dJ/dIm = 4 h^d (|phi|^2 - rho) phi
    grid, psi0, c, w = _setup()
    tgt = G.target_density(grid, PRM.omega, 0.0, c, w)
    g = 4.0 * grid.cell * (np.abs(psi0) ** 2 - tgt) * psi0
    for k in range(3):
        V = _rand_dir(psi0.shape, 10 + k)
        exact = float(np.real(np.vdot(g, V)))
        dirs, _ = G.gradient_fd(psi0, grid, PRM, 1e-3, 0, "ts2", c, w, directions=[V], params=())
        # central-difference truncation ~ h^2 |V|^2 |d^3 J|: about 1e-8 relative here
        assert abs(dirs[0] - exact) <= 1e-6 * abs(exact)


def test_fd_omega_closed_form_without_steps():
    # with no steps J depends on Omega only through R(T) at T = t0
    grid, psi0, c, w = _setup()
    t0 = 0.37
    X = grid.coords()
    co, si = math.cos(PRM.omega * t0), math.sin(PRM.omega * t0)
    Y = G.rotated_coords(grid, PRM.omega, t0)
    dY = [t0 * (-si * X[0] + co * X[1]), t0 * (-co * X[0] - si * X[1])]
    tgt = G.target_density(grid, PRM.omega, t0, c, w)
    dtgt = np.stack([tgt[m] * sum(-2.0 * (Y[a] - c[m][a]) * dY[a] for a in range(2))
                     for m in range(5)])
    exact = grid.cell * float(np.sum(-2.0 * (np.abs(psi0) ** 2 - tgt) * dtgt))
    _, pars = G.gradient_fd(psi0, grid, PRM, 1e-3, 0, "ts2", c, w, params=("omega",), t0=t0)
    assert abs(pars["omega"] - exact) <= 1e-8 * abs(exact)


def test_fd_second_order_convergence():
    grid, psi0, c, w = _setup(n=16)
    V = _rand_dir(psi0.shape, 3) * 0.1
    J = lambda P: G.objective(P, grid, PRM_ANISO, 2e-3, 3, "ts2", c, w)
    d = [G.fd_state(J, psi0, V, h) for h in (4e-2, 2e-2, 1e-2)]
    r = (d[0] - d[1]) / (d[1] - d[2])
    assert 3.5 < r < 4.5, r


def test_fd_global_phase_invariance():
    grid, psi0, c, w = _setup()
    dirs, _ = G.gradient_fd(psi0, grid, PRM_ANISO, 2e-3, 3, "ts2", c, w,
                            directions=[1j * psi0, _rand_dir(psi0.shape, 4)], params=())
    assert abs(dirs[0]) < 1e-7 * abs(dirs[1])


# --------------------------------------------------------------------------
# identities used by the adjoint kernels
# --------------------------------------------------------------------------
def _small_state(seed=1, n=4):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((5, n, n)) + 1j * rng.standard_normal((5, n, n))) * 0.3


@pytest.mark.parametrize("d", [1e-3, 0.07, -0.2])
def test_nonlinear_flow_time_reversal(d):
    grid = O.Grid((4, 4), 8.0)
    phi = _small_state()
    out = O.nonlinear_substep(phi, grid, PRM_ANISO, d, 0.7)
    back = O.nonlinear_substep(out, grid, PRM_ANISO, -d, 0.7)
    assert np.abs(back - phi).max() < 1e-12


def test_linear_flow_time_reversal():
    grid = O.Grid((8, 8), 8.0)
    phi = _rand_dir((5, 8, 8), 2)
    back = O.linear_substep(O.linear_substep(phi, grid, PRM, 0.05), grid, PRM, -0.05)
    assert np.abs(back - phi).max() < 1e-12


def _jvp(f, P, V, eps=1e-6):
    return (f(P + eps * V) - f(P - eps * V)) / (2 * eps)


def test_nonlinear_vjp_is_inverse_flow_jvp():
    # real adjoint of DN(Phi) applied to g equals -i DN_{-d}(N(Phi))[i g]
    grid = O.Grid((2, 2), 8.0)
    phi = _small_state(n=2)
    d, t = 0.13, 0.7
    N = lambda P, dd=d: O.nonlinear_substep(P, grid, PRM_ANISO, dd, t)
    out = N(phi)
    g = _rand_dir(phi.shape, 7)
    n = phi.size
    J = np.zeros((2 * n, 2 * n))
    for k in range(2 * n):
        e = np.zeros(2 * n)
        e[k] = 1.0
        dv = _jvp(N, phi, (e[:n] + 1j * e[n:]).reshape(phi.shape)).ravel()
        J[:, k] = np.concatenate([dv.real, dv.imag])
    gt = J.T @ np.concatenate([g.real.ravel(), g.imag.ravel()])
    gt = (gt[:n] + 1j * gt[n:]).reshape(phi.shape)
    gs = -1j * _jvp(lambda P: N(P, -d), out, 1j * g)
    assert np.abs(gt - gs).max() < 1e-7 * np.abs(gt).max()


def _spin_apply(Fx, Fy, Fz, v):
    return O.spin_dot(Fx, Fy, Fz, v)


def test_nonlinear_parameter_derivatives_are_vector_fields_at_output():
    # d N_d(phi)/dp = d X_p(N_d(phi)): X_c0 = -i rho psi, X_c1 = -i (F.f) psi,
    # X_c2 = -i A00 A conj(psi), X_Omega = -i t (gx^2 - gy^2) x_r y_r psi
    grid = O.Grid((4, 4), 8.0)
    phi = _small_state(3)
    d, t = 0.09, 0.8
    prm = PRM_ANISO
    out = O.nonlinear_substep(phi, grid, prm, d, t)
    rho, Fx, Fy, Fz, _, A00 = O.local_densities(out)
    X = grid.coords()
    co, si = math.cos(prm.omega * t), math.sin(prm.omega * t)
    xr, yr = co * X[0] + si * X[1], -si * X[0] + co * X[1]
    fields = {
        "c0": -1j * rho * out,
        "c1": -1j * _spin_apply(Fx, Fy, Fz, out),
        "c2": -1j * A00 * O.const_matvec(O.AMAT, np.conj(out)),
        "omega": -1j * t * (prm.gx ** 2 - prm.gy ** 2) * xr * yr * out,
    }
    for name, Xp in fields.items():
        fd = G.fd_param(lambda p: O.nonlinear_substep(phi, grid, p, d, t), prm, name, 1e-6)
        assert np.abs(fd - d * Xp).max() < 1e-7 * max(1.0, np.abs(d * Xp).max()), name


def omega_left(a, da):
    """Left-trivialised derivative of exp(i a.f): d exp = i (w.f) exp."""
    th = float(np.linalg.norm(a))
    if th == 0.0:
        return np.array(da, dtype=float)
    ah = a / th
    par = ah * (ah @ da)
    return par + math.sin(th) / th * (da - par) - (1.0 - math.cos(th)) / th * np.cross(ah, da)


def test_dexp_left_jacobian():
    F = [O.FX, O.FY, O.FZ]
    rng = np.random.default_rng(2)
    E = lambda a: sl.expm(1j * sum(a[k] * F[k] for k in range(3)))
    for a in (rng.standard_normal(3) * 0.9, np.array([0.0, 0.0, 2.5]), rng.standard_normal(3) * 1e-3):
        da = rng.standard_normal(3)
        lhs = (E(a + 1e-6 * da) - E(a - 1e-6 * da)) / 2e-6
        w = omega_left(a, da)
        rhs = 1j * sum(w[k] * F[k] for k in range(3)) @ E(a)
        assert np.abs(lhs - rhs).max() < 1e-8


def test_linear_parameter_derivative_by_modes():
    # d L_d(Phi)/dp = inverse[ i (w_p . f) (L_d Phi)^ ] per mode, with
    # a = d (-gamma nu_y, gamma nu_x, -Omega), w_p = omega_left(a, da/dp)
    grid = O.Grid((8, 8), 6.0)
    phi = _rand_dir((5, 8, 8), 9)
    d = 0.3
    out = O.linear_substep(phi, grid, PRM, d)
    hat = O.forward(out, grid)
    nux, nuy = grid.wavenumbers()
    F = [O.FX, O.FY, O.FZ]
    for name in ("omega", "gamma"):
        res = np.zeros_like(hat)
        for iy in range(8):
            for ix in range(8):
                a = d * np.array([-PRM.gamma * nuy[iy, ix], PRM.gamma * nux[iy, ix], -PRM.omega])
                da = d * (np.array([0.0, 0.0, -1.0]) if name == "omega"
                          else np.array([-nuy[iy, ix], nux[iy, ix], 0.0]))
                w = omega_left(a, da)
                M = 1j * sum(w[k] * F[k] for k in range(3))
                res[:, iy, ix] = M @ hat[:, iy, ix]
        pred = O.inverse(res, grid)
        fd = G.fd_param(lambda p: O.linear_substep(phi, grid, p, d), PRM, name, 1e-6)
        assert np.abs(fd - pred).max() < 1e-7 * np.abs(pred).max(), name
