"""Pins of the FP64 oracle's 3D branch and of its transform at the line
lengths the kernels run.

Each test checks the oracle against something other than itself: the
brute-force DFT sum of Sec. 3.1, exact solutions of the free and harmonic
problems in 3D (the kinetic factor with nu_z, the trap term gamma_z^2 z^2),
the separation of the 3D linear flow into the 2D flow (Q built from nu_x,
nu_y only, Sec. 3.1's remark on 3D) times the 1D free flow along z, the
conservation lemmas of Sec. 3.4, closed-form observables of Sec. 2 with an
anisotropic trap (width2[2], the gamma_z potential), the separation of the
SOC energy into x-y slices, and the temporal orders of Sec. 3.3 in 3D.
"""
import math

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs


def _dft_matrix(N, L):
    """K[p, j] = exp(-i nu_p (x_j + L)) of Sec. 3.1, p in FFT order."""
    p = np.array([k if k < N // 2 else k - N for k in range(N)], dtype=float)
    x = -L + np.arange(N) * (2.0 * L / N)
    return np.exp(-1j * np.outer(np.pi * p / L, x + L))


@pytest.mark.parametrize("nx,ny", [(96, 4), (128, 2), (6, 192)])
def test_forward_is_the_printed_sum_at_kernel_lengths(nx, ny):
    """The oracle's transform (numpy.fft) against the printed sum built
    entry by entry, at the radix-3 and power-of-two lengths of the kernels."""
    L = (3.0, 5.0)
    g = O.Grid((nx, ny), L)
    rng = np.random.default_rng(nx + ny)
    phi = rng.normal(size=(5, ny, nx)) + 1j * rng.normal(size=(5, ny, nx))
    Kx, Ky = _dft_matrix(nx, L[0]), _dft_matrix(ny, L[1])
    ref = np.einsum("qk,ckj,pj->cqp", Ky, phi, Kx) / (nx * ny)
    assert np.abs(O.forward(phi, g) - ref).max() < 1e-13 * np.abs(ref).max() * math.log2(nx * ny)
    back = O.inverse(ref, g)
    assert np.abs(back - phi).max() < 1e-12


def test_forward_3d_is_the_printed_sum():
    n, L = (6, 4, 8), (1.5, 2.0, 2.5)
    g = O.Grid(n, L)
    rng = np.random.default_rng(9)
    phi = rng.normal(size=(5, 8, 4, 6)) + 1j * rng.normal(size=(5, 8, 4, 6))
    Kx, Ky, Kz = (_dft_matrix(N, Lv) for N, Lv in zip(n, L))
    ref = np.einsum("rl,qk,pj,clkj->crqp", Kz, Ky, Kx, phi) / np.prod(n)
    assert np.abs(O.forward(phi, g) - ref).max() < 1e-14 * np.abs(ref).max() * 8
    assert np.abs(O.inverse(O.forward(phi, g), g) - phi).max() < 1e-13


def test_free_gaussian_3d_with_rotation_is_exact():
    """V = 0, c = 0, gamma = 0: phi_l(t) = e^{-i l Omega t} (1+it)^{-3/2}
    exp(-|x|^2 / (2(1+it))), the free Schroedinger Gaussian in 3D (the
    kinetic factor of Eq. (sl1) with nu_z)."""
    n, L = (48, 48, 48), 10.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.6, gamma=0.0, gx=0.0, gy=0.0, gz=0.0)
    X, Y, Z = g.coords()
    r2 = X ** 2 + Y ** 2 + Z ** 2
    phi0 = np.stack([np.exp(-0.5 * r2)] * 5).astype(complex)
    T = 1.0
    out, t = O.Propagator(g, p).run(phi0, 0.0, 0.5, 2, "ts2")
    free = np.exp(-r2 / (2 * (1 + 1j * T))) * (1 + 1j * T) ** -1.5
    ref = np.stack([np.exp(-1j * l * 0.6 * T) * free for l in (2, 1, 0, -1, -2)])
    assert abs(t - T) < 1e-15
    assert np.abs(out - ref).max() < 1e-10


def test_3d_linear_flow_separates_into_2d_flow_and_free_z_flow():
    """SOC and rotation on, c = V = 0: for phi(x, y, z) = f(x, y) G(z) the 3D
    flow is [2D flow of f] (1+it)^{-1/2} exp(-z^2 / (2(1+it))), because Q
    involves nu_x, nu_y only and the kinetic factor separates."""
    n2, L2 = (24, 24), 8.0
    nz, Lz = 48, 10.0
    p = O.Params(omega=0.4, gamma=0.8, gx=0.0, gy=0.0, gz=0.0)
    f = inputs.gaussian_random_phase(n2, L2, seed=7, amp=0.5)
    g3 = O.Grid(n2 + (nz,), (L2, L2, Lz))
    z = -Lz + np.arange(nz) * (2 * Lz / nz)
    phi0 = f[:, None, :, :] * np.exp(-0.5 * z * z)[None, :, None, None]
    T = 0.6
    out3, _ = O.Propagator(g3, p).run(phi0, 0.0, 0.2, 3, "ts4")
    out2, _ = O.Propagator(O.Grid(n2, L2), p).run(f, 0.0, 0.2, 3, "ts4")
    gz = np.exp(-z * z / (2 * (1 + 1j * T))) * (1 + 1j * T) ** -0.5
    ref = out2[:, None, :, :] * gz[None, :, None, None]
    assert O.rel_l2(out3, ref) < 1e-11


def test_anisotropic_ground_state_3d():
    """c = 0, gamma = 0, trap (1, 1, 2), Omega = 0.7: the ground state
    G = pi^{-1/2} (2/pi)^{1/4} exp(-(x^2 + y^2)/2 - z^2) has energy
    (1 + 1 + 2)/2 = 2 and is invariant under rotations about z, so the
    rotating-frame field is phi_l(t) = e^{-i l Omega t} e^{-2 i t} G; TS2
    and TS4 reach it at their orders (the trap with gamma_z at the mapped
    point, Eq. (harmonic))."""
    n, L = (32, 32, 32), 6.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.7, gamma=0.0, gx=1.0, gy=1.0, gz=2.0)
    X, Y, Z = g.coords()
    G0 = math.pi ** -0.5 * (2 / math.pi) ** 0.25 * np.exp(-0.5 * (X ** 2 + Y ** 2) - Z ** 2)
    phi0 = np.stack([G0] * 5).astype(complex)
    T = 0.4
    ref = np.stack([np.exp(-1j * l * 0.7 * T - 2j * T) * G0 for l in (2, 1, 0, -1, -2)])
    pr = O.Propagator(g, p)
    err = {}
    for sch in ("ts2", "ts4"):
        err[sch] = [O.rel_l2(pr.run(phi0, 0.0, T / k, k, sch)[0], ref) for k in (8, 16)]
    assert err["ts4"][1] < 1e-6
    assert 1.9 < math.log2(err["ts2"][0] / err["ts2"][1]) < 2.1
    assert 3.7 < math.log2(err["ts4"][0] / err["ts4"][1]) < 4.3


def test_mass_and_magnetization_conserved_3d():
    n, L = (16, 16, 16), 6.0
    g = O.Grid(n, L)
    phi = inputs.gaussian_random_phase(n, L, seed=17, amp=0.5)
    phi[0] *= 1.5
    p_soc = O.Params(omega=0.5, gamma=0.9, c0=60, c1=-2, c2=3, gx=1.2, gy=0.9, gz=1.6)
    out, t = O.Propagator(g, p_soc).run(phi, 0.0, 0.01, 10, "ts4")
    assert abs(O.observables(out, g, p_soc, t)["mass"] - O.observables(phi, g, p_soc, 0.0)["mass"]) < 1e-13
    p0 = O.Params(omega=0.5, gamma=0.0, c0=60, c1=-2, c2=3, gx=1.2, gy=0.9, gz=1.6)
    out, t = O.Propagator(g, p0).run(phi, 0.0, 0.01, 10, "ts4")
    m0 = O.observables(phi, g, p0, 0.0)["magnetization"]
    assert abs(m0) > 0.1
    assert abs(O.observables(out, g, p0, t)["magnetization"] - m0) < 1e-13


def test_observables_3d_anisotropic_closed_forms():
    """psi = prod_a (w_a/pi)^{1/4} exp(-w_a x_a^2 / 2) in l = 2, w = (1.2,
    1.2, 2.5), trap (1.1, 1.1, 1.7): mass 1, M = 2, kinetic sum(w)/4,
    potential sum(gamma_a^2 / (4 w_a)), widths 1/(2 w_a) (width2[2] along
    z), interaction (c0/2 + 2 c1) int rho^2 with int rho^2 = prod
    sqrt(w_a / (2 pi)); the vortex (x + iy) e^{-(x^2+y^2)/2}/sqrt(pi) times
    the z factor has <L_z> = 1 and kinetic 1 + w_z/4."""
    n, L = (64, 64, 64), 7.0      # rho^2 along z is exp(-5 z^2): h = 0.22 resolves it
    g = O.Grid(n, L)
    X, Y, Z = g.coords()
    w = (1.2, 1.2, 2.5)
    G = np.ones(X.shape)
    for wa, Xa in zip(w, (X, Y, Z)):
        G = G * (wa / math.pi) ** 0.25 * np.exp(-0.5 * wa * Xa ** 2)
    phi = np.zeros((5,) + G.shape, complex)
    phi[0] = G
    p = O.Params(omega=0.4, c0=7.0, c1=2.0, gx=1.1, gy=1.1, gz=1.7)
    ob = O.observables(phi, g, p, 0.9)
    rho2 = np.prod([math.sqrt(wa / (2 * math.pi)) for wa in w])
    assert abs(ob["mass"] - 1) < 1e-12
    assert abs(ob["magnetization"] - 2) < 1e-12
    assert abs(ob["e_kin"] - sum(w) / 4) < 1e-11
    assert abs(ob["e_pot"] - sum(ga ** 2 / (4 * wa) for ga, wa in zip((1.1, 1.1, 1.7), w))) < 1e-11
    for a in range(3):
        assert abs(ob["width2"][a] - 1 / (2 * w[a])) < 1e-11
    assert abs(ob["e_int"] - (3.5 + 2 * 2.0) * rho2) < 1e-11
    assert abs(ob["lz"]) < 1e-13
    gz = (w[2] / math.pi) ** 0.25 * np.exp(-0.5 * w[2] * Z ** 2)
    v = np.zeros_like(phi)
    v[0] = (X + 1j * Y) * np.exp(-0.5 * (X ** 2 + Y ** 2)) / math.sqrt(math.pi) * gz
    ob = O.observables(v, g, p, 0.3)
    assert abs(ob["lz"] - 1.0) < 1e-11
    assert abs(ob["e_kin"] - (1.0 + w[2] / 4)) < 1e-11
    assert abs(ob["e_rot"] + 0.4) < 1e-11


def test_soc_and_transverse_kinetic_energy_separate_into_slices():
    """The SOC operator and the x-y kinetic energy act slice by slice: the 3D
    oracle's SOC energy is h_z times the sum of the 2D oracle's SOC energies
    of the z-slices (the 2D form is pinned against the physical-space
    operator in test_oracle_pins)."""
    n, L = (16, 20, 12), (5.0, 6.0, 4.0)
    g3 = O.Grid(n, L)
    g2 = O.Grid(n[:2], L[:2])
    p = O.Params(gamma=0.7)
    phi = inputs.gaussian_random_phase(n, L, seed=19, amp=2.0)
    e3 = O.observables(phi, g3, p, 0.0)["e_soc"]
    hz = 2 * L[2] / n[2]
    e2 = sum(O.observables(phi[:, k], g2, p, 0.0)["e_soc"] for k in range(n[2]))
    assert abs(e3 - hz * e2) < 1e-12 * max(1.0, abs(e3))


def test_temporal_orders_3d():
    n, L = (16, 16, 16), 6.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.3, gamma=0.5, c0=30, c1=-1, c2=1, gx=1.0, gy=1.2, gz=1.5)
    phi = inputs.gaussian_random_phase(n, L, seed=23, amp=0.2)
    pr = O.Propagator(g, p)
    T = 0.2
    ref, _ = pr.run(phi, 0.0, T / 160, 160, "ts4")
    for sch, order in (("ts2", 2), ("ts4", 4)):
        e = [O.rel_l2(pr.run(phi, 0.0, T / k, k, sch)[0], ref) for k in (10, 20)]
        assert abs(math.log2(e[0] / e[1]) - order) < 0.2, (sch, e)
