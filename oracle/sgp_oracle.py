"""FP64 CPU oracle for the compact splitting Fourier spectral propagator of the
rotating spin-orbit-coupled spin-2 Gross-Pitaevskii system (arXiv 2603.25282).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (the CUDA library and its Python binding) never
imports, calls or links it, and this module imports nothing from the product.

The oracle is deliberately plain: numpy FP64, whole-array operations, no
blocking, no fusion, no merging of adjacent substeps.  Library primitives used
as single steps: ``numpy.fft`` (the discrete Fourier transform of Sec. 3.1,
pinned against a brute-force DFT in the tests) and ``numpy.linalg.eigh`` (the
Hermitian eigendecomposition that defines the matrix exponential
``exp(i delta Q)`` of Sec. 3.1, pinned against the paper's printed closed form).

Conventions (all from Sec. 3.1, "Fourier spectral method" paragraph):
  * state array shape ``(5, ny, nx)`` (2D) or ``(5, nz, ny, nx)`` (3D),
    component order l = 2, 1, 0, -1, -2 (Sec. 1, the vector Psi);
  * grid x_j = -L + j h, h = 2L/N, N even;
  * Fourier index p in [-N/2, N/2-1] stored in FFT order, nu_p = pi p / L;
  * forward transform carries the 1/N factor per axis, the inverse none.

Frame: the oracle evolves the rotating-frame field Phi of Eq. (mapping),
phi_l(x, t) = exp(-i l Omega t) psi_l(R(t) x, t).  The linear flow is Eq.
(linearEQ2) (Laplace + SOC + Omega f_z); the nonlinear flow is Eq. (nonlEQ1)
with the trap evaluated at the mapped point R(t) x, which is Algorithm 1's
nonlinear substep written in the rotating frame (the phase factor commutes with
the spin rotation and leaves A00 unchanged).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQ6H = math.sqrt(6.0) / 2.0
SQ5 = math.sqrt(5.0)
MS = np.array([2, 1, 0, -1, -2], dtype=np.float64)   # l for component index 0..4


# --------------------------------------------------------------------------
# Spin-2 matrices and singlet matrix (Sec. 1, definitions after Eq. (harmonic))
# --------------------------------------------------------------------------
def spin2_matrices():
    """Return (f_x, f_y, f_z), the spin-2 matrices printed in Sec. 1."""
    fx = np.array([[0, 1, 0, 0, 0],
                   [1, 0, SQ6H, 0, 0],
                   [0, SQ6H, 0, SQ6H, 0],
                   [0, 0, SQ6H, 0, 1],
                   [0, 0, 0, 1, 0]], dtype=np.complex128)
    fy = 1j * np.array([[0, -1, 0, 0, 0],
                        [1, 0, -SQ6H, 0, 0],
                        [0, SQ6H, 0, -SQ6H, 0],
                        [0, 0, SQ6H, 0, -1],
                        [0, 0, 0, 1, 0]], dtype=np.complex128)
    fz = np.diag([2.0, 1.0, 0.0, -1.0, -2.0]).astype(np.complex128)
    return fx, fy, fz


def singlet_matrix():
    """A_ij = (-1)^(i-1) delta_{i+j,6} / sqrt(5), i, j = 1..5 (Sec. 1)."""
    A = np.zeros((5, 5), dtype=np.complex128)
    for i in range(1, 6):
        j = 6 - i
        A[i - 1, j - 1] = (-1.0) ** (i - 1) / SQ5
    return A


FX, FY, FZ = spin2_matrices()
AMAT = singlet_matrix()


# --------------------------------------------------------------------------
# Parameters and grid (Sec. 1 Eq. (CGPEs), Eq. (harmonic); Sec. 3.1 grids)
# --------------------------------------------------------------------------
@dataclass
class Params:
    """Physical parameters of Eq. (CGPEs) with the harmonic trap (harmonic)."""
    omega: float = 0.0      # angular velocity Omega
    gamma: float = 0.0      # SOC strength gamma
    c0: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    gx: float = 1.0         # trap frequencies gamma_x, gamma_y, gamma_z
    gy: float = 1.0
    gz: float = 1.0


@dataclass
class Grid:
    """Uniform periodic grid on [-L, L]^d (Sec. 3.1, sets I_N, T_N, G).

    ``n`` and ``L`` are given in (x, y[, z]) order; arrays are stored with x
    as the last (fastest) axis.
    """
    n: tuple
    L: tuple
    dim: int = field(init=False)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        if np.isscalar(self.L):
            self.L = (float(self.L),) * len(self.n)
        self.L = tuple(float(v) for v in self.L)
        self.dim = len(self.n)
        for N in self.n:
            if N % 2:
                raise ValueError("N must be even (Sec. 3.1)")

    @property
    def h(self):
        return tuple(2.0 * L / N for L, N in zip(self.L, self.n))

    @property
    def cell(self):
        return float(np.prod(self.h))

    def coords(self):
        """Physical coordinates x_j = -L + j h, broadcast to the array shape."""
        axes = [-L + np.arange(N) * (2.0 * L / N) for L, N in zip(self.L, self.n)]
        # array axis order is (z, y, x); meshgrid with indexing='ij' on reversed
        grids = np.meshgrid(*axes[::-1], indexing="ij")
        return tuple(grids[::-1])     # (X, Y[, Z]) each of array shape

    def wavenumbers(self):
        """nu_p = pi p / L for p in FFT order, broadcast to the array shape."""
        axes = []
        for L, N in zip(self.L, self.n):
            p = np.fft.fftfreq(N, d=1.0 / N)      # 0..N/2-1, -N/2..-1
            axes.append(np.pi * p / L)
        grids = np.meshgrid(*axes[::-1], indexing="ij")
        return tuple(grids[::-1])

    @property
    def shape(self):
        return tuple(self.n[::-1])


# --------------------------------------------------------------------------
# Discrete Fourier transforms (Sec. 3.1, the two displayed sums)
# --------------------------------------------------------------------------
def _spatial_axes(grid):
    return tuple(range(-grid.dim, 0))


def forward(phi, grid):
    """phi_hat_p = (1/N^d) sum_j phi_j exp(-i nu_p (x_j + L)) per component."""
    return np.fft.fftn(phi, axes=_spatial_axes(grid)) / float(np.prod(grid.n))


def inverse(phihat, grid):
    """phi_j = sum_p phi_hat_p exp(+i nu_p (x_j + L)) per component."""
    return np.fft.ifftn(phihat, axes=_spatial_axes(grid)) * float(np.prod(grid.n))


def naive_dft_1d(x, sign=-1):
    """Brute-force O(N^2) DFT sum_j x_j exp(sign 2 pi i p j / N), p = 0..N-1.

    Used only to pin ``numpy.fft`` to the definition in the tests.
    """
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[-1]
    out = np.zeros_like(x)
    for p in range(N):
        acc = 0.0 + 0.0j
        for j in range(N):
            acc += x[..., j] * complex(math.cos(2 * math.pi * p * j / N),
                                       sign * math.sin(2 * math.pi * p * j / N))
        out[..., p] = acc
    return out


# --------------------------------------------------------------------------
# Linear subflow (Sec. 3.1, Eqs. (linearEQ2), (linearEQ3), (sl1))
# --------------------------------------------------------------------------
def q_matrix(nu_x, nu_y, omega, gamma):
    """Q of Sec. 3.1: A_hat = |nu|^2/2 I - Q, a = -nu_q - i nu_p.

    nu_p is the x-wavenumber, nu_q the y-wavenumber.  Arrays broadcast; the
    result has shape (..., 5, 5).
    """
    nu_x = np.asarray(nu_x, dtype=np.float64)
    nu_y = np.asarray(nu_y, dtype=np.float64)
    a = -nu_y - 1j * nu_x
    ab = np.conj(a)
    shp = np.broadcast(nu_x, nu_y).shape
    Q = np.zeros(shp + (5, 5), dtype=np.complex128)
    Q[..., 0, 0] = -2 * omega
    Q[..., 1, 1] = -omega
    Q[..., 3, 3] = omega
    Q[..., 4, 4] = 2 * omega
    Q[..., 0, 1] = gamma * a
    Q[..., 1, 0] = gamma * ab
    Q[..., 1, 2] = SQ6H * gamma * a
    Q[..., 2, 1] = SQ6H * gamma * ab
    Q[..., 2, 3] = SQ6H * gamma * a
    Q[..., 3, 2] = SQ6H * gamma * ab
    Q[..., 3, 4] = gamma * a
    Q[..., 4, 3] = gamma * ab
    return Q


def expm_hermitian(Q, delta):
    """exp(i delta Q) for Hermitian Q (stacked), via its eigendecomposition."""
    w, V = np.linalg.eigh(Q)
    ph = np.exp(1j * delta * w)
    return np.einsum("...ij,...j,...kj->...ik", V, ph, np.conj(V))


def mode_propagators(grid, prm, delta):
    """Per-mode matrix exp(-i|nu|^2 delta/2) exp(i delta Q) of Eq. (sl1).

    Q depends on (nu_x, nu_y) only (also in 3D, Remark on the 3D extension);
    the kinetic factor uses the full |nu|^2.  Shape: grid.shape + (5, 5).
    """
    nus = grid.wavenumbers()
    E = expm_hermitian(q_matrix(nus[0], nus[1], prm.omega, prm.gamma), delta)
    nu2 = sum(nu * nu for nu in nus)
    return E * np.exp(-0.5j * nu2 * delta)[..., None, None]


def linear_substep(Phi, grid, prm, delta, props=None):
    """Exact flow of Eq. (linearEQ2) over time delta, via Eq. (sl1)."""
    if props is None:
        props = mode_propagators(grid, prm, delta)
    Ph = forward(Phi, grid)
    Ph = np.moveaxis(props @ np.moveaxis(Ph, 0, -1)[..., None], -2, 0)[..., 0]
    return inverse(Ph, grid)


# --------------------------------------------------------------------------
# Nonlinear subflow (Sec. 3.2, Eq. (nonlEQ1) and its solution (solution2))
# --------------------------------------------------------------------------
def trap_rotated(grid, prm, t):
    """V(R(t) x) with R(t) of Eq. (mapping) and V of Eq. (harmonic)."""
    co, si = math.cos(prm.omega * t), math.sin(prm.omega * t)
    X = grid.coords()
    xr = co * X[0] + si * X[1]
    yr = -si * X[0] + co * X[1]
    V = prm.gx ** 2 * xr ** 2 + prm.gy ** 2 * yr ** 2
    if grid.dim == 3:
        V = V + prm.gz ** 2 * X[2] ** 2
    return 0.5 * V


def local_densities(Phi):
    """rho, F = (F_x, F_y, F_z), F_+ and A00 at every point (Sec. 1)."""
    p2, p1, p0, m1, m2 = Phi
    rho = np.sum(np.abs(Phi) ** 2, axis=0)
    Fz = 2 * abs(p2) ** 2 + abs(p1) ** 2 - abs(m1) ** 2 - 2 * abs(m2) ** 2
    Fp = 2 * (np.conj(p2) * p1 + np.conj(m1) * m2) + math.sqrt(6.0) * (
        np.conj(p1) * p0 + np.conj(p0) * m1)
    A00 = (2 * p2 * m2 - 2 * p1 * m1 + p0 * p0) / SQ5
    return rho, Fp.real, Fp.imag, Fz, Fp, A00


def spin2_exp_poly(Fx, Fy, Fz, kappa_over_F):
    """exp(-i c1 delta F.f) by the quartic polynomial printed after (solution2).

    ``kappa_over_F`` = c1 * delta, so kappa = c1 |F| delta.  Returns per-point
    5x5 matrices, shape (..., 5, 5).  Points with |F| = 0 get the identity.
    """
    Fn = np.sqrt(Fx * Fx + Fy * Fy + Fz * Fz)
    safe = np.where(Fn > 0, Fn, 1.0)
    M = (Fx[..., None, None] * FX + Fy[..., None, None] * FY
         + Fz[..., None, None] * FZ) / safe[..., None, None]
    k = kappa_over_F * Fn
    M2 = M @ M
    M3 = M2 @ M
    M4 = M3 @ M
    eye = np.broadcast_to(np.eye(5, dtype=np.complex128), M.shape)
    c1 = np.asarray(1j * (np.sin(2 * k) / 6 - 4 * np.sin(k) / 3))
    c2 = np.asarray(4 * np.cos(k) / 3 - np.cos(2 * k) / 12 - 5.0 / 4.0)
    c3 = np.asarray(1j * (np.sin(k) / 3 - np.sin(2 * k) / 6))
    c4 = np.asarray(np.cos(2 * k) / 12 - np.cos(k) / 3 + 0.25)
    U = (eye + c1[..., None, None] * M + c2[..., None, None] * M2
         + c3[..., None, None] * M3 + c4[..., None, None] * M4)
    return np.where((Fn > 0)[..., None, None], U, eye)


def const_matvec(M, v):
    """M v at every point for a constant 5x5 matrix M and a (5, ...) field."""
    return (M @ v.reshape(5, -1)).reshape(v.shape)


def spin_dot(Fx, Fy, Fz, v):
    """(F.f) v = (F_x f_x + F_y f_y + F_z f_z) v at every point."""
    return Fx * const_matvec(FX, v) + Fy * const_matvec(FY, v) + Fz * const_matvec(FZ, v)


def apply_spin2_exp_poly(Fx, Fy, Fz, kappa_over_F, v):
    """exp(-i c1 delta F.f) v with the quartic polynomial printed after
    (solution2), the powers of M = F.f/|F| applied to v one at a time.
    Points with |F| = 0 are left unchanged."""
    Fn = np.sqrt(Fx * Fx + Fy * Fy + Fz * Fz)
    safe = np.where(Fn > 0, Fn, 1.0)
    k = kappa_over_F * Fn
    c1 = 1j * (np.sin(2 * k) / 6 - 4 * np.sin(k) / 3)
    c2 = 4 * np.cos(k) / 3 - np.cos(2 * k) / 12 - 5.0 / 4.0
    c3 = 1j * (np.sin(k) / 3 - np.sin(2 * k) / 6)
    c4 = np.cos(2 * k) / 12 - np.cos(k) / 3 + 0.25
    out = v.copy()
    Mv = v
    for ck in (c1, c2, c3, c4):
        Mv = spin_dot(Fx, Fy, Fz, Mv) / safe
        out = out + ck * Mv
    return np.where(Fn > 0, out, v)


def nonlinear_substep(Phi, grid, prm, delta, t):
    """Exact solution (solution2) of Eq. (nonlEQ1) over time delta at time t.

    rho and F are frozen (Eqs. after (nonlEQ1)); the singlet part is the
    zeta-system solution with S = sqrt((rho/5)^2 - |A00|^2/5); the spin part
    is the quartic polynomial; the scalar phase carries V(R(t)x) and
    (c0 + c2/5) rho.
    """
    rho, Fx, Fy, Fz, Fp, A00 = local_densities(Phi)
    S2 = (rho / 5.0) ** 2 - np.abs(A00) ** 2 / 5.0
    S = np.sqrt(np.maximum(S2, 0.0))
    arg = prm.c2 * S * delta
    safeS = np.where(S > 0, S, 1.0)
    sinc = np.where(S > 0, np.sin(arg) / safeS, prm.c2 * delta)
    ABar = const_matvec(AMAT, np.conj(Phi))
    b = np.cos(arg) * Phi + 1j * sinc * (rho / 5.0 * Phi - A00 * ABar)
    b = apply_spin2_exp_poly(Fx, Fy, Fz, prm.c1 * delta, b)
    V = trap_rotated(grid, prm, t)
    return np.exp(-1j * delta * (V + (prm.c0 + prm.c2 / 5.0) * rho)) * b


# --------------------------------------------------------------------------
# Compositions (Sec. 3.3, the coefficient lists and Algorithm 1)
# --------------------------------------------------------------------------
CBRT2 = 2.0 ** (1.0 / 3.0)
TS4_A1 = 1.0 / (2.0 * (2.0 - CBRT2))
TS4_A2 = (1.0 - CBRT2) / (2.0 * (2.0 - CBRT2))
TS4_B1 = 1.0 / (2.0 - CBRT2)
TS4_B2 = -CBRT2 / (2.0 - CBRT2)


def substep_sequence(scheme):
    """Ordered list of ('N' | 'L', coefficient) for one step.

    TS2: N(tau/2) L(tau) N(tau/2) -- Algorithm 1.
    TS4: N(a1) L(b1) N(a2) L(b2) N(a2) L(b1) N(a1) -- the fourth-order
    coefficients of Sec. 3.3 with the nonlinear flow taking the a_j.
    The same compositions with the roles of the two flows exchanged (the
    other reading of Sec. 3.3's coefficient list, equally valid):
    TS2_LNL: L(tau/2) N(tau) L(tau/2);
    TS4_L:   L(a1) N(b1) L(a2) N(b2) L(a2) N(b1) L(a1).
    """
    if scheme == "ts2":
        return [("N", 0.5), ("L", 1.0), ("N", 0.5)]
    if scheme == "ts4":
        return [("N", TS4_A1), ("L", TS4_B1), ("N", TS4_A2), ("L", TS4_B2),
                ("N", TS4_A2), ("L", TS4_B1), ("N", TS4_A1)]
    if scheme == "ts2_lnl":
        return [("L", 0.5), ("N", 1.0), ("L", 0.5)]
    if scheme == "ts4_l":
        return [("L", TS4_A1), ("N", TS4_B1), ("L", TS4_A2), ("N", TS4_B2),
                ("L", TS4_A2), ("N", TS4_B1), ("L", TS4_A1)]
    raise ValueError(scheme)


class Propagator:
    """Time stepper over the rotating-frame field; caches per-delta matrices
    (Remark 3.1: the mode matrices depend only on Omega, gamma and the
    substep size)."""

    def __init__(self, grid, prm):
        self.grid = grid
        self.prm = prm
        self._props = {}

    def props(self, delta):
        key = float(delta)
        if key not in self._props:
            self._props[key] = mode_propagators(self.grid, self.prm, delta)
        return self._props[key]

    def step(self, Phi, t, tau, scheme="ts2"):
        """One step of TS2/TS4 from time t; t advances only in the L substeps."""
        tcur = t
        for kind, coef in substep_sequence(scheme):
            d = coef * tau
            if kind == "N":
                Phi = nonlinear_substep(Phi, self.grid, self.prm, d, tcur)
            else:
                Phi = linear_substep(Phi, self.grid, self.prm, d, self.props(d))
                tcur = tcur + d
        return Phi, t + tau

    def run(self, Phi, t, tau, nsteps, scheme="ts2"):
        for _ in range(nsteps):
            Phi, t = self.step(Phi, t, tau, scheme)
        return Phi, t


# --------------------------------------------------------------------------
# Observables (Sec. 2: mass, energy, magnetization, <L_z>, widths)
# --------------------------------------------------------------------------
def spectral_derivative(phi, grid, axis):
    """d/dx_axis by the Fourier spectral method (axis 0 = x, 1 = y, 2 = z)."""
    nu = grid.wavenumbers()[axis]
    return inverse(1j * nu * forward(phi, grid), grid)


def observables(Phi, grid, prm, t):
    """Mass, energy, magnetization, <L_z>, component masses, widths at time t.

    All integrals are h^d-weighted grid sums of the rotating-frame field; the
    quantities are the lab-frame ones of Sec. 2 (mass, rho-terms, |grad|^2,
    <L_z> and the SOC term are invariant under the mapping (mapping); the trap
    and the widths use the mapped point R(t) x).
    """
    cell = grid.cell
    rho, Fx, Fy, Fz, Fp, A00 = local_densities(Phi)
    comp_mass = cell * np.sum(np.abs(Phi) ** 2, axis=tuple(range(1, grid.dim + 1)))
    mass = float(np.sum(comp_mass))
    magnet = float(np.sum(MS * comp_mass))
    X = grid.coords()
    dx = spectral_derivative(Phi, grid, 0)
    dy = spectral_derivative(Phi, grid, 1)
    lz = float(np.real(cell * np.sum(np.conj(Phi) * (-1j) * (X[0] * dy - X[1] * dx))))
    # kinetic and SOC energies via Parseval in Fourier space (Eq. for E(t), Sec. 2)
    Ph = forward(Phi, grid)
    nus = grid.wavenumbers()
    nu2 = sum(nu * nu for nu in nus)
    vol = float(np.prod([2.0 * L for L in grid.L]))
    e_kin = float(vol * np.sum(0.5 * nu2 * np.abs(Ph) ** 2))
    Ssym = q_matrix(nus[0], nus[1], 0.0, 1.0)          # symbol of the SOC matrix S
    soc = np.einsum("i...,...ij,j...->...", np.conj(Ph), Ssym, Ph)
    e_soc = float(-prm.gamma * vol * np.real(np.sum(soc)))
    V = trap_rotated(grid, prm, t)
    e_pot = float(cell * np.sum(V * rho))
    e_rot = -prm.omega * lz
    e_c0 = float(cell * np.sum(0.5 * prm.c0 * rho ** 2))
    e_c1 = float(cell * np.sum(0.5 * prm.c1 * (Fx ** 2 + Fy ** 2 + Fz ** 2)))
    e_c2 = float(cell * np.sum(0.5 * prm.c2 * np.abs(A00) ** 2))
    co, si = math.cos(prm.omega * t), math.sin(prm.omega * t)
    xr = co * X[0] + si * X[1]
    yr = -si * X[0] + co * X[1]
    w2 = [float(cell * np.sum(xr ** 2 * rho)), float(cell * np.sum(yr ** 2 * rho)),
          float(cell * np.sum(X[2] ** 2 * rho)) if grid.dim == 3 else 0.0]
    energy = e_kin + e_pot + e_rot + e_c0 + e_c1 + e_c2 + e_soc
    return dict(t=t, mass=mass, energy=energy, magnetization=magnet, lz=lz,
                comp_mass=comp_mass, width2=w2, e_kin=e_kin, e_pot=e_pot,
                e_rot=e_rot, e_int=e_c0 + e_c1 + e_c2, e_soc=e_soc)


def rel_l2(a, b):
    """Relative discrete l2 error ||a - b|| / ||b|| over all components."""
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def component_errors(a, ref):
    """E_l = ||psi_ref_l - psi_l|| / ||psi_ref_l|| (Sec. 4.1), l = 2..-2."""
    out = []
    for l in range(5):
        out.append(float(np.linalg.norm((a[l] - ref[l]).ravel())
                         / np.linalg.norm(ref[l].ravel())))
    return out


# --------------------------------------------------------------------------
# Lab-frame output by rotation-shear decomposition (Sec. 3.1, Eqs. (RSDA1),
# (RSDA2)); test infrastructure like the rest of this module
# --------------------------------------------------------------------------
def shear(f, grid, axis, coef_times_other):
    """exp(c(x) d_axis) f: translate every line along `axis` (0 = x, 1 = y)
    by c, where c varies with the other coordinate: c = coef_times_other,
    an array broadcast to the grid.  In Fourier space along the line the
    mode nu_p is multiplied by exp(i nu_p c) (a translation by c)."""
    nu = grid.wavenumbers()[axis]
    ax = -1 - axis                     # array axis of the line
    fh = np.fft.fft(f, axis=ax)
    fh = fh * np.exp(1j * nu * coef_times_other)
    return np.fft.ifft(fh, axis=ax)


def rotate_quarter(f, k):
    """g(x) = f(R_{k pi/2} x) exactly on a square periodic grid, R_a the
    counter-clockwise rotation by a; x_j = -L + j h, so -x_j = x_{(N-j) mod N}."""
    k %= 4
    out = f
    for _ in range(k):
        # g(x, y) = f(-y, x):  G[iy, ix] = A[ix, (N - iy) mod N]
        n = out.shape[-1]
        idx = (-np.arange(n)) % n
        out = np.swapaxes(out, -1, -2)[..., idx, :]
    return out


def rotate_rsda(f, grid, theta):
    """g(x) = f(R_theta x) (R_theta counter-clockwise) by exact quarter turns
    and the three shears of Eq. (RSDA2) for the remaining angle in
    [-pi/4, pi/4]: exp(a y d_x) exp(b x d_y) exp(a y d_x) with
    a = -tan(theta_r / 2), b = sin(theta_r).  Quarter turns need a square
    grid (equal N and L in x and y)."""
    k = int(np.round(theta / (0.5 * math.pi)))
    thr = theta - k * 0.5 * math.pi
    if k % 4:
        if grid.n[0] != grid.n[1] or grid.L[0] != grid.L[1]:
            raise ValueError("quarter turns need a square grid")
        f = rotate_quarter(f, k)
    X = grid.coords()
    a = -math.tan(0.5 * thr)
    b = math.sin(thr)
    g = shear(f, grid, 0, a * X[1])
    g = shear(g, grid, 1, b * X[0])
    return shear(g, grid, 0, a * X[1])


def lab_frame_field(Phi, grid, omega, t):
    """psi_l(x, t) = exp(i l Omega t) phi_l(R(t)^T x, t), the inverse of the
    mapping (mapping), evaluated on the grid as in Eq. (RSDA2)."""
    th = omega * t
    g = rotate_rsda(Phi, grid, th)
    return np.exp(1j * MS * th).reshape((5,) + (1,) * grid.dim) * g


def rotating_frame_field(Psi, grid, omega, t):
    """phi_l(x, t) = exp(-i l Omega t) psi_l(R(t) x, t), Eq. (RSDA1)."""
    th = omega * t
    g = rotate_rsda(Psi, grid, -th)
    return np.exp(-1j * MS * th).reshape((5,) + (1,) * grid.dim) * g


def lab_trap(grid, prm):
    """V(x) of Eq. (harmonic) in the lab frame."""
    X = grid.coords()
    V = prm.gx ** 2 * X[0] ** 2 + prm.gy ** 2 * X[1] ** 2
    if grid.dim == 3:
        V = V + prm.gz ** 2 * X[2] ** 2
    return 0.5 * V


def lab_nonlinear_substep(Psi, grid, prm, delta):
    """Eq. (solution2) in the lab frame (trap V(x)): the rotating-frame flow
    with the rotation angle set to zero."""
    p0 = Params(**{**prm.__dict__, "omega": 0.0})
    return nonlinear_substep(Psi, grid, p0, delta, 0.0)


def algorithm1_lab_step(Psi, grid, prm, t, tau, props=None):
    """One step of Algorithm 1 as printed, in the lab frame: N(tau/2) with
    V(x), the mapping (RSDA1) at t, the linear flow (sl1) over tau, the
    inverse mapping (RSDA2) at t + tau, N(tau/2)."""
    Psi = lab_nonlinear_substep(Psi, grid, prm, 0.5 * tau)
    Phi = rotating_frame_field(Psi, grid, prm.omega, t)
    Phi = linear_substep(Phi, grid, prm, tau, props)
    Psi = lab_frame_field(Phi, grid, prm.omega, t + tau)
    return lab_nonlinear_substep(Psi, grid, prm, 0.5 * tau)
