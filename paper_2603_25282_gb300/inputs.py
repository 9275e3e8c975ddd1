"""Seeded synthetic initial data and parameter sets.

This module holds input generation only: it contains none of the propagator's
arithmetic and imports neither the CUDA library nor any reference code.  Both
the GPU path and the CPU oracle are fed from here.

Arrays are complex128 of shape (5, ny, nx) or (5, nz, ny, nx) with the
component order l = 2, 1, 0, -1, -2 and x fastest; grids are x_j = -L + j h,
h = 2L/N (Sec. 3.1).
"""
from __future__ import annotations

import math

import numpy as np


def coords(n, L):
    """Broadcast coordinate arrays (X, Y[, Z]) on the periodic grid."""
    n = tuple(int(v) for v in n)
    if np.isscalar(L):
        L = (float(L),) * len(n)
    axes = [-Lk + np.arange(N) * (2.0 * Lk / N) for Lk, N in zip(L, n)]
    g = np.meshgrid(*axes[::-1], indexing="ij")
    return tuple(g[::-1]), tuple(2.0 * Lk / N for Lk, N in zip(L, n))


def _normalise(psi, h):
    mass = float(np.prod(h)) * float(np.sum(np.abs(psi) ** 2))
    return psi / math.sqrt(mass)


def gaussian_random_phase(n, L, seed, amp=0.01, nmodes=8, kmax=3):
    """Gaussian exp(-|x|^2/2) in every component times exp(i amp theta_l(x)).

    theta_l is a smooth band-limited random field:
    sum_k u_k cos(pi (m_k x + n_k y [+ o_k z]) / L + phi_k), u_k ~ U[-1, 1],
    m, n, o integers in [-kmax, kmax], phi_k ~ U[0, 2 pi), drawn per component
    from numpy's PCG64 stream seeded with ``seed``.  Normalised so that
    h^d sum |Psi|^2 = 1.
    """
    X, h = coords(n, L)
    Ls = (float(L),) * len(n) if np.isscalar(L) else tuple(L)
    rng = np.random.default_rng(seed)
    r2 = sum(x * x for x in X)
    G = np.exp(-0.5 * r2)
    psi = np.empty((5,) + X[0].shape, dtype=np.complex128)
    for comp in range(5):
        theta = np.zeros_like(G)
        for _ in range(nmodes):
            u = rng.uniform(-1.0, 1.0)
            ks = rng.integers(-kmax, kmax + 1, size=len(n))
            ph = rng.uniform(0.0, 2.0 * math.pi)
            arg = sum(math.pi * float(k) * x / Lk for k, x, Lk in zip(ks, X, Ls))
            theta += u * np.cos(arg + ph)
        psi[comp] = G * np.exp(1j * amp * theta)
    return _normalise(psi, h)


def ini_example1(n, L):
    """Initial data (ini1) of Example 1/2: psi_{+-2} = psi_{+-1} = phi,
    psi_0 = 2 phi, phi = exp(-|x|^2/2) / (sqrt(8) pi^(d/4)).  Not renormalised
    (the paper's own normalisation gives mass 1 in the continuum)."""
    X, h = coords(n, L)
    d = len(n)
    r2 = sum(x * x for x in X)
    phi = np.exp(-0.5 * r2) / (math.sqrt(8.0) * math.pi ** (d / 4.0))
    return np.stack([phi, phi, 2 * phi, phi, phi]).astype(np.complex128)


def ini_example3(n, L):
    """Initial data of Example 3: psi_{+-2} = psi_{+-1} = phi,
    psi_0 = 6 sqrt(7) phi, phi = exp(-|x|^2/8) / (32 sqrt(pi))."""
    X, h = coords(n, L)
    r2 = sum(x * x for x in X)
    phi = np.exp(-r2 / 8.0) / (32.0 * math.sqrt(math.pi))
    return np.stack([phi, phi, 6 * math.sqrt(7.0) * phi, phi, phi]).astype(np.complex128)


def vortex_state(n, L, weights=(1, 0, 0, 0, 0)):
    """(x + i y) exp(-|x|^2/2) in the weighted components, normalised to mass 1
    (a state with <L_z> = 1 in the continuum)."""
    X, h = coords(n, L)
    r2 = sum(x * x for x in X)
    f = (X[0] + 1j * X[1]) * np.exp(-0.5 * r2)
    psi = np.stack([w * f for w in weights]).astype(np.complex128)
    return _normalise(psi, h)


def random_field(n, seed, scale=1.0):
    """Unstructured complex normal field (for transform and adjoint checks)."""
    rng = np.random.default_rng(seed)
    shp = (5,) + tuple(int(v) for v in n)[::-1]
    return scale * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))


def ensemble_members(count, seed, sides=(64, 96, 128, 192, 256)):
    """Seeded ensemble of independent 2D runs (sizes and parameters).

    Side from ``sides``; Omega ~ U[0, 0.9], gamma ~ U[0, 2], c0 ~ U[50, 1000],
    c1 ~ U[-5, 5], c2 ~ U[0, 10]; domain half-width 8; isotropic unit trap.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append(dict(n=int(rng.choice(sides)), L=8.0,
                        omega=float(rng.uniform(0.0, 0.9)),
                        gamma=float(rng.uniform(0.0, 2.0)),
                        c0=float(rng.uniform(50.0, 1000.0)),
                        c1=float(rng.uniform(-5.0, 5.0)),
                        c2=float(rng.uniform(0.0, 10.0)),
                        gx=1.0, gy=1.0, gz=1.0, seed=int(seed) * 100003 + i))
    return out


def density_target(n, L, seed):
    """Seeded target of the terminal density misfit (the adjoint workload).

    Component l gets rho_l(x) = w_l exp(-|x - c_l|^2), i.e. G(x - c_l)^2 with
    G = exp(-|x|^2/2), centre c_l ~ U[-1/2, 1/2]^d (PCG64 seeded with
    ``seed``) and w_l such that h^d sum_j rho_l(x_j) = 1/5 on the grid, so the
    five targets carry mass 1 together.  Returns (centres (5, d), weights (5,)).
    The objective evaluates rho_l at the rotated point R(T) x itself.
    """
    X, h = coords(n, L)
    rng = np.random.default_rng(seed)
    d = len(X)
    centres = rng.uniform(-0.5, 0.5, size=(5, d))
    cell = float(np.prod(h))
    weights = np.empty(5)
    for comp in range(5):
        r2 = sum((x - c) ** 2 for x, c in zip(X, centres[comp]))
        weights[comp] = 0.2 / (cell * float(np.sum(np.exp(-r2))))
    return centres, weights
