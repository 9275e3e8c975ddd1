"""FP64 oracle gradient of a terminal-time objective of the propagator.

TEST INFRASTRUCTURE ONLY, under the same rule as ``sgp_oracle``: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
it; it imports nothing from the product.

Objective (the density-misfit workload): for the rotating-frame field Phi at
time T,
    J = h^d sum_{l, j} (|phi_l(x_j, T)|^2 - rho_l(R(T) x_j))^2,
with rho_l(y) = w_l exp(-|y - c_l|^2) and R(t) the rotation of Eq. (mapping)
(the same R as in the trap, Sec. 2), so J compares the lab-frame density
with a lab-frame target and depends on Omega through the frame as well as
through the dynamics.

Gradients are central finite differences of J composed with the oracle's own
propagator (Sec. 3.3 compositions, unmerged substeps): the definition of a
derivative, with no reverse-mode or adjoint arithmetic here.  Conventions:
the state gradient is dJ/dRe Psi + i dJ/dIm Psi, so the directional
derivative along a complex direction V is Re sum conj(g) V; parameter
derivatives are plain partial derivatives.  The pins in
``tests/test_grad_oracle.py`` check the finite differences against a closed
form (no steps), their second-order convergence and the global-phase
invariance of J.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import sgp_oracle as O


def rotated_coords(grid, omega, t):
    """R(t) x at every grid point: (x cos + y sin, -x sin + y cos[, z])."""
    X = grid.coords()
    co, si = math.cos(omega * t), math.sin(omega * t)
    out = [co * X[0] + si * X[1], -si * X[0] + co * X[1]]
    if grid.dim == 3:
        out.append(X[2])
    return out


def target_density(grid, omega, t, centres, weights):
    """rho_l(R(t) x_j) for the five components, shape (5,) + grid.shape."""
    Y = rotated_coords(grid, omega, t)
    rho = np.empty((5,) + grid.shape)
    for comp in range(5):
        r2 = sum((y - c) ** 2 for y, c in zip(Y, centres[comp]))
        rho[comp] = weights[comp] * np.exp(-r2)
    return rho


def misfit(PhiT, grid, omega, T, centres, weights):
    """J of the module docstring for a terminal field PhiT at time T."""
    tgt = target_density(grid, omega, T, centres, weights)
    return grid.cell * float(np.sum((np.abs(PhiT) ** 2 - tgt) ** 2))


def objective(Phi0, grid, prm, tau, nsteps, scheme, centres, weights, t0=0.0):
    """J after nsteps of the composition from Phi0 at time t0."""
    prop = O.Propagator(grid, prm)
    PhiT, T = prop.run(np.asarray(Phi0, dtype=np.complex128), t0, tau, nsteps, scheme)
    return misfit(PhiT, grid, prm.omega, T, centres, weights)


def fd_state(fun, Phi0, V, h):
    """Central difference of fun along the complex direction V."""
    return (fun(Phi0 + h * V) - fun(Phi0 - h * V)) / (2.0 * h)


def fd_param(fun_of_prm, prm, name, h):
    """Central difference of fun_of_prm in the parameter ``name``."""
    v = getattr(prm, name)
    up = dataclasses.replace(prm, **{name: v + h})
    dn = dataclasses.replace(prm, **{name: v - h})
    return (fun_of_prm(up) - fun_of_prm(dn)) / (2.0 * h)


def gradient_fd(Phi0, grid, prm, tau, nsteps, scheme, centres, weights,
                directions=(), params=("omega", "gamma", "c1"), h_state=1e-5,
                h_param=1e-5, t0=0.0):
    """Oracle directional and parameter derivatives of J.

    Returns (dirs, pars): dirs[k] = dJ along directions[k] (equal to
    Re sum conj(g) V_k for the state gradient g), pars[name] = dJ/dname.
    """
    def J_state(P):
        return objective(P, grid, prm, tau, nsteps, scheme, centres, weights, t0)

    def J_prm(p):
        return objective(Phi0, grid, p, tau, nsteps, scheme, centres, weights, t0)

    dirs = [fd_state(J_state, Phi0, V, h_state) for V in directions]
    pars = {name: fd_param(J_prm, prm, name, h_param) for name in params}
    return dirs, pars
