"""Tangent-linear (forward-mode) FP64 oracle gradient of the propagator.

TEST INFRASTRUCTURE ONLY, under the same rule as ``sgp_oracle``: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
it; it imports nothing from the product.

Every quantity of the oracle's substeps is carried as a dual number
a + eps * a' with eps^2 = 0 (class ``Dual``), so one pass of the substeps
gives the exact derivative of the terminal objective along one direction
(a state direction and/or a parameter seed), with no finite-difference
truncation and no reverse sweep.  The field is complex and the flows are not
holomorphic (they contain conj and |.|^2), but every operation is either
holomorphic in its arguments or a conjugation, so a complex value with a
complex tangent, where conj maps the tangent to its conjugate, carries the
exact real derivative.

The substeps follow the oracle step by step, in the paper's order:
  * L(delta), Sec. 3.1 Eq. (sl1): forward DFT, the per-mode matrix
    exp(-i |nu|^2 delta/2) exp(i delta Q), inverse DFT.  The derivative of
    exp(i delta Q) in Omega and gamma is the Daleckii-Krein formula for a
    function of a Hermitian matrix: with Q = V diag(w) V^H,
    d exp(i delta Q) = V (G o (V^H dQ V)) V^H, G_jk the divided difference
    of exp(i delta w) at w_j, w_k (i delta exp(i delta w_j) when equal);
    dQ/dOmega = -f_z, dQ/dgamma = Q at Omega = 0, gamma = 1.
  * N(delta) at time t, Sec. 3.2 Eq. (solution2): singlet rotation, the
    quartic spin polynomial printed after (solution2), the scalar phase with
    V(R(t) x) (R depends on Omega, Eq. (mapping)).
  * the compositions of Sec. 3.3 (``sgp_oracle.substep_sequence``).
The objective is ``sgp_grad.misfit`` (its target depends on Omega through
R(T)).  Conventions match ``sgp_grad``: the derivative along a complex state
direction V equals Re sum conj(g) V for the state gradient g.

Pins: ``tests/test_tangent_oracle.py`` (finite differences converge to it
at second order, the Daleckii-Krein derivative against a block-matrix
exponential, global-phase invariance, the closed form with no steps).
"""
from __future__ import annotations

import math

import numpy as np

from . import sgp_grad as G
from . import sgp_oracle as O

PARAMS = ("omega", "gamma", "c0", "c1", "c2")


class Dual:
    """a + eps a' (eps^2 = 0) over numpy arrays or scalars."""

    __slots__ = ("v", "d")
    __array_priority__ = 1000    # numpy operands defer to Dual's operators

    def __init__(self, v, d=None):
        self.v = v
        self.d = np.zeros_like(v) if d is None else d

    def __add__(self, o):
        o = lift(o)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = lift(o)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return lift(o) - self

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __mul__(self, o):
        o = lift(o)
        return Dual(self.v * o.v, self.d * o.v + self.v * o.d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = lift(o)
        q = self.v / o.v
        return Dual(q, (self.d - q * o.d) / o.v)

    def __rtruediv__(self, o):
        return lift(o) / self

    def __pow__(self, k):
        if k != 2:
            raise ValueError("only squares are needed")
        return self * self

    def __getitem__(self, idx):
        return Dual(self.v[idx], self.d[idx])

    @property
    def real(self):
        return Dual(np.real(self.v), np.real(self.d))


def lift(x):
    return x if isinstance(x, Dual) else Dual(x, np.zeros_like(np.asarray(x, dtype=np.result_type(x, 0.0))))


def conj(x):
    return Dual(np.conj(x.v), np.conj(x.d))


def abs2(x):
    return (x * conj(x)).real


def sqrt(x):
    r = np.sqrt(x.v)
    return Dual(r, x.d / (2.0 * r))


def sin(x):
    return Dual(np.sin(x.v), np.cos(x.v) * x.d)


def cos(x):
    return Dual(np.cos(x.v), -np.sin(x.v) * x.d)


def exp(x):
    e = np.exp(x.v)
    return Dual(e, e * x.d)


def dsum(x, axis=None):
    return Dual(np.sum(x.v, axis=axis), np.sum(x.d, axis=axis))


def where(cond, a, b):
    a, b = lift(a), lift(b)
    return Dual(np.where(cond, a.v, b.v), np.where(cond, a.d, b.d))


def stack(xs):
    return Dual(np.stack([x.v for x in xs]), np.stack([x.d for x in xs]))


def const_matvec(M, x):
    """M x at every point for a constant 5x5 M and a (5, ...) dual field."""
    return Dual(O.const_matvec(M, x.v), O.const_matvec(M, x.d))


def forward(x, grid):
    return Dual(O.forward(x.v, grid), O.forward(x.d, grid))


def inverse(x, grid):
    return Dual(O.inverse(x.v, grid), O.inverse(x.d, grid))


# --------------------------------------------------------------------------
# linear subflow (Sec. 3.1, Eq. (sl1)) with the Daleckii-Krein derivative
# --------------------------------------------------------------------------
def _phi1(z):
    """(e^z - 1)/z, stable for small |z| (Taylor series below 1e-3)."""
    z = np.asarray(z, dtype=np.complex128)
    small = np.abs(z) < 1e-3
    zs = np.where(small, 1.0, z)
    direct = (np.exp(zs) - 1.0) / zs
    series = 1.0 + z / 2.0 + z * z / 6.0 + z ** 3 / 24.0
    return np.where(small, series, direct)


def expm_hermitian_tangent(Q, dQ, delta):
    """exp(i delta Q) and its derivative along dQ (stacked Hermitian Q)."""
    w, V = np.linalg.eigh(Q)
    ph = np.exp(1j * delta * w)
    E = np.einsum("...ij,...j,...kj->...ik", V, ph, np.conj(V))
    # divided differences of f(w) = exp(i delta w):
    # f[w_j, w_k] = exp(i delta w_k) i delta phi1(i delta (w_j - w_k))
    wj = w[..., :, None]
    wk = w[..., None, :]
    Gm = np.exp(1j * delta * wk) * (1j * delta) * _phi1(1j * delta * (wj - wk))
    B = np.conj(np.swapaxes(V, -1, -2)) @ dQ @ V
    dE = V @ (Gm * B) @ np.conj(np.swapaxes(V, -1, -2))
    return E, dE


def mode_propagators(grid, omega, gamma, delta):
    """Dual per-mode matrices exp(-i|nu|^2 delta/2) exp(i delta Q(Omega, gamma))."""
    nus = grid.wavenumbers()
    Q = O.q_matrix(nus[0], nus[1], omega.v, gamma.v)
    dQ = omega.d * O.q_matrix(nus[0], nus[1], 1.0, 0.0) + gamma.d * O.q_matrix(nus[0], nus[1], 0.0, 1.0)
    E, dE = expm_hermitian_tangent(Q, dQ, delta)
    kin = np.exp(-0.5j * sum(nu * nu for nu in nus) * delta)[..., None, None]
    return Dual(E * kin, dE * kin)


def linear_substep(Phi, grid, omega, gamma, delta):
    """Dual of ``sgp_oracle.linear_substep``."""
    P = mode_propagators(grid, omega, gamma, delta)
    Ph = forward(Phi, grid)
    vv = np.moveaxis(Ph.v, 0, -1)[..., None]
    dd = np.moveaxis(Ph.d, 0, -1)[..., None]
    out_v = np.moveaxis(P.v @ vv, -2, 0)[..., 0]
    out_d = np.moveaxis(P.d @ vv + P.v @ dd, -2, 0)[..., 0]
    return inverse(Dual(out_v, out_d), grid)


# --------------------------------------------------------------------------
# nonlinear subflow (Sec. 3.2, Eq. (solution2))
# --------------------------------------------------------------------------
def local_densities(Phi):
    """Dual rho, F_x, F_y, F_z, A00 (Sec. 1 definitions)."""
    p2, p1, p0, m1, m2 = (Phi[k] for k in range(5))
    rho = abs2(p2) + abs2(p1) + abs2(p0) + abs2(m1) + abs2(m2)
    Fz = 2.0 * abs2(p2) + abs2(p1) - abs2(m1) - 2.0 * abs2(m2)
    Fp = 2.0 * (conj(p2) * p1 + conj(m1) * m2) + math.sqrt(6.0) * (conj(p1) * p0 + conj(p0) * m1)
    Fx = Dual(np.real(Fp.v), np.real(Fp.d))
    Fy = Dual(np.imag(Fp.v), np.imag(Fp.d))
    A00 = (2.0 * p2 * m2 - 2.0 * p1 * m1 + p0 * p0) / O.SQ5
    return rho, Fx, Fy, Fz, A00


def _singlet_factors(u, a):
    """cos(a sqrt(u)) and sin(a sqrt(u))/sqrt(u) as duals of u >= 0 (both
    are analytic in u; the series is used where sqrt(u) a is below 1e-4)."""
    av = a.v if isinstance(a, Dual) else a
    small = abs(av) * np.sqrt(np.maximum(u.v, 0.0)) < 1e-4
    us = Dual(np.where(small, 1.0, np.maximum(u.v, 0.0)), np.where(small, 0.0, u.d))
    s = sqrt(us)
    c_direct = cos(a * s)
    sc_direct = sin(a * s) / s
    # series in u: cos = 1 - a^2 u/2 + a^4 u^2/24, sin(a s)/s = a - a^3 u/6 + a^5 u^2/120
    a2 = a * a
    c_ser = 1.0 - a2 * u / 2.0 + a2 * a2 * u * u / 24.0
    sc_ser = a - a * a2 * u / 6.0 + a * a2 * a2 * u * u / 120.0
    return where(small, c_ser, c_direct), where(small, sc_ser, sc_direct)


def spin_dot(Fx, Fy, Fz, v):
    """(F.f) v at every point (dual)."""
    return Fx * const_matvec(O.FX, v) + Fy * const_matvec(O.FY, v) + Fz * const_matvec(O.FZ, v)


def trap_rotated(grid, prm, t):
    """Dual V(R(t) x) (Eq. (harmonic) at the mapped point of Eq. (mapping))."""
    X = grid.coords()
    th = prm["omega"] * t
    co, si = cos(th), sin(th)
    xr = co * X[0] + si * X[1]
    yr = co * X[1] - si * X[0]
    V = prm["gx"] ** 2 * (xr * xr) + prm["gy"] ** 2 * (yr * yr)
    if grid.dim == 3:
        V = V + prm["gz"] ** 2 * X[2] ** 2
    return 0.5 * V


def nonlinear_substep(Phi, grid, prm, delta, t):
    """Dual of ``sgp_oracle.nonlinear_substep``."""
    rho, Fx, Fy, Fz, A00 = local_densities(Phi)
    # singlet part: S^2 = (rho/5)^2 - |A00|^2/5 (clamped at 0, as the oracle)
    S2 = (rho * rho) / 25.0 - abs2(A00) / 5.0
    S2 = where(S2.v > 0, S2, 0.0)
    cosS, sincS = _singlet_factors(S2, prm["c2"] * delta)
    ABar = const_matvec(O.AMAT, conj(Phi))
    b = cosS * Phi + 1j * sincS * (rho / 5.0 * Phi - A00 * ABar)
    # spin part: exp(-i c1 delta F.f) by the printed quartic polynomial
    Fn = sqrt(Fx * Fx + Fy * Fy + Fz * Fz)
    k = prm["c1"] * delta * Fn
    coef = (1j * (sin(2.0 * k) / 6.0 - 4.0 * sin(k) / 3.0),
            4.0 * cos(k) / 3.0 - cos(2.0 * k) / 12.0 - 5.0 / 4.0,
            1j * (sin(k) / 3.0 - sin(2.0 * k) / 6.0),
            cos(2.0 * k) / 12.0 - cos(k) / 3.0 + 0.25)
    out = b
    Mv = b
    for ck in coef:
        Mv = spin_dot(Fx, Fy, Fz, Mv) / Fn
        out = out + ck * Mv
    # scalar phase with the trap at the mapped point
    V = trap_rotated(grid, prm, t)
    return exp(-1j * delta * (V + (prm["c0"] + prm["c2"] / 5.0) * rho)) * out


# --------------------------------------------------------------------------
# compositions (Sec. 3.3) and the objective
# --------------------------------------------------------------------------
def step(Phi, grid, prm, t, tau, scheme):
    tcur = t
    for kind, c in O.substep_sequence(scheme):
        d = c * tau
        if kind == "N":
            Phi = nonlinear_substep(Phi, grid, prm, d, tcur)
        else:
            Phi = linear_substep(Phi, grid, prm["omega"], prm["gamma"], d)
            tcur = tcur + d
    return Phi, t + tau


def misfit(PhiT, grid, omega, T, centres, weights):
    """Dual of ``sgp_grad.misfit``: h^d sum (|phi|^2 - rho_l(R(T) x))^2."""
    X = grid.coords()
    th = omega * T
    co, si = cos(th), sin(th)
    Y = [co * X[0] + si * X[1], co * X[1] - si * X[0]]
    if grid.dim == 3:
        Y.append(lift(X[2]))
    tgt = []
    for comp in range(5):
        r2 = lift(0.0)
        for y, c in zip(Y, centres[comp]):
            r2 = r2 + (y - c) * (y - c)
        tgt.append(weights[comp] * exp(-r2))
    diff = abs2(PhiT) - stack(tgt)
    J = dsum(diff * diff) * grid.cell
    return J


def directional_derivative(Phi0, grid, prm, tau, nsteps, scheme, centres, weights,
                           dPhi0=None, dprm=None, t0=0.0):
    """J and dJ along the seed (dPhi0, dprm): dPhi0 a complex state direction,
    dprm a dict of parameter tangents (names of ``PARAMS``)."""
    Phi0 = np.asarray(Phi0, dtype=np.complex128)
    dPhi0 = np.zeros_like(Phi0) if dPhi0 is None else np.asarray(dPhi0, dtype=np.complex128)
    dprm = dprm or {}
    p = {name: Dual(float(getattr(prm, name)), float(dprm.get(name, 0.0))) for name in PARAMS}
    for name in ("gx", "gy", "gz"):
        p[name] = float(getattr(prm, name))
    Phi = Dual(Phi0, dPhi0)
    t = t0
    for _ in range(nsteps):
        Phi, t = step(Phi, grid, p, t, tau, scheme)
    J = misfit(Phi, grid, p["omega"], t, centres, weights)
    return float(np.real(J.v)), float(np.real(J.d))


def gradient_tangent(Phi0, grid, prm, tau, nsteps, scheme, centres, weights,
                     directions=(), params=PARAMS, t0=0.0):
    """Directional derivatives along ``directions`` and the partial
    derivatives in ``params``, one tangent pass each (same return layout as
    ``sgp_grad.gradient_fd``)."""
    dirs = [directional_derivative(Phi0, grid, prm, tau, nsteps, scheme, centres, weights,
                                   dPhi0=V, t0=t0)[1] for V in directions]
    pars = {name: directional_derivative(Phi0, grid, prm, tau, nsteps, scheme, centres, weights,
                                         dprm={name: 1.0}, t0=t0)[1] for name in params}
    return dirs, pars


# the objective itself, for cross-checks with sgp_grad
objective = G.objective
