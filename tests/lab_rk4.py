"""Independent check method for the oracle: classical RK4 in time with Fourier
spectral derivatives in space, applied to the full lab-frame equation
Eq. (CGPEs) of Sec. 1 (rotation term -Omega L_z kept in physical space, SOC
operators L_+- = i d_y +- d_x, the printed F.f matrix with F_+- entries, the
singlet term c2 A00 A conj(Psi)).

It shares no step with the splitting method: no rotating frame, no exact
subflows, no composition.  Used only by the oracle pin tests.
"""
import math

import numpy as np

S6 = math.sqrt(6.0) / 2.0


def _k(n, L):
    return np.pi * np.fft.fftfreq(n, d=1.0 / n) / L


def grad(f, Lx, Ly):
    """(d_x f, d_y f) of arrays shaped (..., ny, nx)."""
    ny, nx = f.shape[-2:]
    kx = _k(nx, Lx)[None, :]
    ky = _k(ny, Ly)[:, None]
    F = np.fft.fft2(f)
    return np.fft.ifft2(1j * kx * F), np.fft.ifft2(1j * ky * F)


def laplacian(f, Lx, Ly):
    ny, nx = f.shape[-2:]
    kx = _k(nx, Lx)[None, :]
    ky = _k(ny, Ly)[:, None]
    return np.fft.ifft2(-(kx ** 2 + ky ** 2) * np.fft.fft2(f))


def rhs(psi, X, Y, Lx, Ly, p):
    """d/dt Psi = -i [ (H0 + c1 F.f - gamma S) Psi + c2 A00 A conj(Psi) ]."""
    p2, p1, p0, m1, m2 = psi
    rho = np.sum(np.abs(psi) ** 2, axis=0)
    Fz = 2 * abs(p2) ** 2 + abs(p1) ** 2 - abs(m1) ** 2 - 2 * abs(m2) ** 2
    Fp = 2 * (np.conj(p2) * p1 + np.conj(m1) * m2) + math.sqrt(6) * (
        np.conj(p1) * p0 + np.conj(p0) * m1)
    Fm = np.conj(Fp)
    A00 = (2 * p2 * m2 - 2 * p1 * m1 + p0 * p0) / math.sqrt(5)
    V = 0.5 * (p["gx"] ** 2 * X ** 2 + p["gy"] ** 2 * Y ** 2)
    dx, dy = grad(psi, Lx, Ly)
    Lp = 1j * dy + dx            # L_+
    Lm = 1j * dy - dx            # L_-
    Lzpsi = -1j * (X * dy - Y * dx)
    H0 = -0.5 * laplacian(psi, Lx, Ly) + (V + p["c0"] * rho) * psi - p["omega"] * Lzpsi
    # (F.f) Psi with the printed matrix (rows of F.f in Sec. 1)
    Ff = np.stack([
        2 * Fz * p2 + Fm * p1,
        Fp * p2 + Fz * p1 + S6 * Fm * p0,
        S6 * Fp * p1 + S6 * Fm * m1,
        S6 * Fp * p0 - Fz * m1 + Fm * m2,
        Fp * m1 - 2 * Fz * m2])
    # S Psi with the printed SOC matrix
    SP = np.stack([
        Lm[1],
        Lp[0] + S6 * Lm[2],
        S6 * Lp[1] + S6 * Lm[3],
        S6 * Lp[2] + Lm[4],
        Lp[3]])
    # A conj(Psi): A_ij = (-1)^(i-1) delta_{i+j,6}/sqrt5
    AcP = np.stack([np.conj(m2), -np.conj(m1), np.conj(p0), -np.conj(p1),
                    np.conj(p2)]) / math.sqrt(5)
    return -1j * (H0 + p["c1"] * Ff - p["gamma"] * SP + p["c2"] * A00 * AcP)


def integrate(psi, X, Y, Lx, Ly, p, T, dt):
    n = int(round(T / dt))
    for _ in range(n):
        k1 = rhs(psi, X, Y, Lx, Ly, p)
        k2 = rhs(psi + 0.5 * dt * k1, X, Y, Lx, Ly, p)
        k3 = rhs(psi + 0.5 * dt * k2, X, Y, Lx, Ly, p)
        k4 = rhs(psi + dt * k3, X, Y, Lx, Ly, p)
        psi = psi + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return psi


def trig_interp(f, Lx, Ly, xq, yq):
    """Evaluate the Fourier interpolant of grid data f (ny, nx) on [-L, L)^2
    at the points (xq, yq) (same-shaped arrays), by direct summation."""
    ny, nx = f.shape
    F = np.fft.fft2(f) / (nx * ny)
    kx = _k(nx, Lx)
    ky = _k(ny, Ly)
    ex = np.exp(1j * np.multiply.outer(xq + Lx, kx))    # (..., nx)
    ey = np.exp(1j * np.multiply.outer(yq + Ly, ky))    # (..., ny)
    # sum_q sum_p F[q, p] ey[q] ex[p]
    return np.einsum("...q,qp,...p->...", ey, F, ex)
