"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a
brute-force definition, a closed form printed in the paper, an independent
integrator (RK4) of the defining equation, a conservation lemma, a dynamical
law of Sec. 2, or the errors printed in Table 1.
"""
import math
import os

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs
from tests import lab_rk4

S6H = math.sqrt(6.0) / 2.0


# ----------------------------------------------------------------------------
# transforms (Sec. 3.1)
# ----------------------------------------------------------------------------
def test_forward_is_the_printed_sum_bruteforce():
    """forward() equals (1/N^2) sum_jk phi_jk e^{-i nu_p (x_j+L)} e^{-i nu_q (y_k+L)}."""
    g = O.Grid((6, 4), (1.5, 2.0))
    rng = np.random.default_rng(3)
    phi = rng.normal(size=(5, 4, 6)) + 1j * rng.normal(size=(5, 4, 6))
    X, Y = g.coords()
    NX, NY = g.wavenumbers()
    out = np.zeros_like(phi)
    for qi in range(4):
        for pi_ in range(6):
            nup, nuq = NX[qi, pi_], NY[qi, pi_]
            ker = np.exp(-1j * nup * (X + 1.5)) * np.exp(-1j * nuq * (Y + 2.0))
            out[:, qi, pi_] = np.sum(phi * ker, axis=(1, 2)) / 24.0
    assert np.abs(O.forward(phi, g) - out).max() < 1e-14
    assert np.abs(O.inverse(O.forward(phi, g), g) - phi).max() < 1e-14


def test_wavenumbers_nyquist_and_order():
    g = O.Grid((8,), (2.0,))
    (nu,) = g.wavenumbers()
    assert np.allclose(nu, np.pi / 2.0 * np.array([0, 1, 2, 3, -4, -3, -2, -1]))


def test_naive_dft_helper_matches_fft_1d():
    x = np.random.default_rng(1).normal(size=12) + 0j
    assert np.abs(O.naive_dft_1d(x) - np.fft.fft(x)).max() < 1e-12


# ----------------------------------------------------------------------------
# spin-2 algebra (Sec. 1, Sec. 3.2)
# ----------------------------------------------------------------------------
def test_spin2_algebra():
    fx, fy, fz = O.FX, O.FY, O.FZ
    for M in (fx, fy, fz):
        assert np.abs(M - M.conj().T).max() == 0
    assert np.abs(fx @ fy - fy @ fx - 1j * fz).max() < 1e-15
    assert np.abs(fy @ fz - fz @ fy - 1j * fx).max() < 1e-15
    assert np.abs(fz @ fx - fx @ fz - 1j * fy).max() < 1e-15
    assert np.abs(fx @ fx + fy @ fy + fz @ fz - 6 * np.eye(5)).max() < 1e-14
    A = O.AMAT
    assert np.abs(A @ A - np.eye(5) / 5).max() < 1e-16
    rng = np.random.default_rng(0)
    psi = rng.normal(size=5) + 1j * rng.normal(size=5)
    for M in (fx, fy, fz):          # Psi^T A f_alpha Psi = 0 (Sec. 3.2)
        assert abs(psi @ A @ M @ psi) < 1e-13
    F = rng.normal(size=3)          # (F.conj(f)) A + A (F.f) = 0 (Sec. 3.2)
    Ff = F[0] * fx + F[1] * fy + F[2] * fz
    assert np.abs(np.conj(Ff) @ A + A @ Ff).max() < 1e-14


def test_local_densities_match_printed_components():
    rng = np.random.default_rng(7)
    psi = rng.normal(size=(5, 3)) + 1j * rng.normal(size=(5, 3))
    rho, Fx, Fy, Fz, Fp, A00 = O.local_densities(psi)
    for k in range(3):
        v = psi[:, k]
        assert abs(Fx[k] - np.real(v.conj() @ O.FX @ v)) < 1e-13
        assert abs(Fy[k] - np.real(v.conj() @ O.FY @ v)) < 1e-13
        assert abs(Fz[k] - np.real(v.conj() @ O.FZ @ v)) < 1e-13
        assert abs(A00[k] - v @ O.AMAT @ v) < 1e-13


# ----------------------------------------------------------------------------
# linear subflow (Sec. 3.1)
# ----------------------------------------------------------------------------
def printed_expm_iTQ(nup, nuq, Om, ga, tau):
    """The closed form of e^{i tau Q} printed in Sec. 3.1 (c_jk, xi, lambda,
    eta_1..eta_4), entries a^{k-j} c_jk above and conj(a)^{j-k} c_kj below."""
    a = -nuq - 1j * nup
    xi = ga * abs(a)
    lam = math.sqrt(Om ** 2 + xi ** 2)
    e1 = math.cos(2 * lam * tau) - 1
    e2 = math.cos(lam * tau) - 1
    e3 = 1j * math.sin(2 * lam * tau)
    e4 = 1j * math.sin(lam * tau)
    l4 = lam ** 4
    c = {}
    c[11] = ((8 * Om ** 4 + 8 * Om ** 2 * xi ** 2 + xi ** 4) * e1 + 4 * xi ** 2 * (2 * Om ** 2 + xi ** 2) * e2
             - 4 * Om * lam * (2 * Om ** 2 + xi ** 2) * e3 - 8 * Om * lam * xi ** 2 * e4 + 8 * l4) / (8 * l4)
    c[12] = ga / (4 * l4) * (-Om * (4 * Om ** 2 + 3 * xi ** 2) * e1 + 4 * Om ** 3 * e2
                            + lam * (4 * Om ** 2 + xi ** 2) * e3 - 2 * lam * (2 * Om ** 2 - xi ** 2) * e4)
    c[13] = math.sqrt(6) * ga ** 2 / (4 * l4) * ((2 * Om ** 2 + xi ** 2) * e2 - 2 * Om * lam * e4 + 2 * lam ** 2) * e2
    c[14] = ga ** 3 / (2 * l4) * (-Om * e2 + lam * e4) * e2
    c[15] = ga ** 4 / (8 * l4) * (e1 - 4 * e2)
    c[22] = 1 / (2 * l4) * (2 * xi ** 2 * e2 + lam ** 2) * ((2 * Om ** 2 + xi ** 2) * e2 - 2 * Om * lam * e4 + 2 * lam ** 2)
    c[23] = math.sqrt(6) * ga / (2 * l4) * (xi ** 2 * e2 + lam ** 2) * (-Om * e2 + lam * e4)
    c[24] = ga ** 2 / (2 * l4) * (2 * xi ** 2 * e2 + 3 * lam ** 2) * e2
    c[25] = c[14] + Om * ga ** 3 / l4 * e2 ** 2
    c[33] = 3 * xi ** 2 / (4 * l4) * (xi ** 2 * e1 + 4 * Om ** 2 * e2) + 1
    c[34] = c[23] + math.sqrt(6) * Om * ga / l4 * (xi ** 2 * e2 + lam ** 2) * e2
    c[35] = c[13] + math.sqrt(6) * Om * ga ** 2 / lam ** 3 * e2 * e4
    c[44] = c[22] + 2 * Om / lam ** 3 * (2 * xi ** 2 * e2 + lam ** 2) * e4
    c[45] = c[12] + Om * ga / (2 * l4) * ((4 * Om ** 2 + 3 * xi ** 2) * e1 - 4 * Om ** 2 * e2)
    c[55] = c[11] + Om / lam ** 3 * ((2 * Om ** 2 + xi ** 2) * e3 + 2 * xi ** 2 * e4)
    E = np.zeros((5, 5), dtype=complex)
    for j in range(1, 6):
        for k in range(1, 6):
            if j == k:
                E[j - 1, k - 1] = c[11 * j]
            elif j < k:
                E[j - 1, k - 1] = a ** (k - j) * c[10 * j + k]
            else:
                E[j - 1, k - 1] = np.conj(a) ** (j - k) * c[10 * k + j]
    return E


@pytest.mark.parametrize("seed", range(6))
def test_mode_matrix_equals_printed_closed_form(seed):
    rng = np.random.default_rng(seed)
    nup, nuq = rng.uniform(-6, 6, size=2)
    Om = rng.uniform(-1.5, 1.5)
    ga = rng.uniform(-2, 2)
    tau = rng.uniform(-0.3, 0.3)
    Q = O.q_matrix(nup, nuq, Om, ga)
    E = O.expm_hermitian(Q, tau)
    assert np.abs(E - printed_expm_iTQ(nup, nuq, Om, ga, tau)).max() < 1e-12


def test_mode_matrix_spectrum_and_unitarity():
    rng = np.random.default_rng(11)
    for _ in range(10):
        nup, nuq, Om, ga = rng.normal(size=4) * 3
        Q = O.q_matrix(nup, nuq, Om, ga)
        lam = math.sqrt(Om ** 2 + ga ** 2 * (nup ** 2 + nuq ** 2))
        w = np.linalg.eigvalsh(Q)
        assert np.allclose(np.sort(w), lam * np.array([-2, -1, 0, 1, 2]), atol=1e-12)
        E = O.expm_hermitian(Q, 0.37)
        assert np.abs(E.conj().T @ E - np.eye(5)).max() < 1e-13
        E2 = O.expm_hermitian(Q, 0.2) @ O.expm_hermitian(Q, 0.17)
        assert np.abs(E2 - E).max() < 1e-13


def test_mode_matrix_gamma0_is_nonsoc_diagonal():
    """gamma = 0 gives diag(e^{-2i tau Om}, e^{-i tau Om}, 1, e^{i tau Om}, e^{2i tau Om}) (NonSOCMat)."""
    tau, Om = 0.3, 0.7
    E = O.expm_hermitian(O.q_matrix(2.0, -1.0, Om, 0.0), tau)
    ref = np.diag(np.exp(1j * tau * Om * np.array([-2, -1, 0, 1, 2])))
    assert np.abs(E - ref).max() < 1e-15


def test_free_gaussian_linear_flow_is_exact():
    """V = 0, c = 0, gamma = 0: phi_l(t) = e^{-i l Omega t} psi_free(t) with the
    free Schroedinger Gaussian (1+it)^{-1} exp(-|x|^2 / (2(1+it)))."""
    g = O.Grid((96, 96), 16.0)
    p = O.Params(omega=0.6, gamma=0.0, gx=0.0, gy=0.0)
    X, Y = g.coords()
    G = np.exp(-0.5 * (X ** 2 + Y ** 2))
    phi0 = np.stack([G] * 5).astype(complex)
    pr = O.Propagator(g, p)
    T = 1.0
    out, t = pr.run(phi0, 0.0, 0.25, 4, "ts2")
    free = np.exp(-(X ** 2 + Y ** 2) / (2 * (1 + 1j * T))) / (1 + 1j * T)
    ref = np.stack([np.exp(-1j * l * 0.6 * T) * free for l in (2, 1, 0, -1, -2)])
    assert abs(t - T) < 1e-15
    assert np.abs(out - ref).max() < 1e-11


def test_linear_only_scheme_is_step_independent():
    """With c = 0 and V = 0 the splitting is exact: one step of size T equals
    n steps of T/n (SOC and rotation on)."""
    g = O.Grid((32, 32), 8.0)
    p = O.Params(omega=0.4, gamma=0.8, gx=0.0, gy=0.0)
    phi0 = inputs.gaussian_random_phase((32, 32), 8.0, seed=5, amp=0.5)
    pr = O.Propagator(g, p)
    a, _ = pr.run(phi0, 0.0, 0.6, 1, "ts4")
    b, _ = pr.run(phi0, 0.0, 0.05, 12, "ts2")
    assert O.rel_l2(a, b) < 1e-12


# ----------------------------------------------------------------------------
# nonlinear subflow (Sec. 3.2)
# ----------------------------------------------------------------------------
def test_spin_polynomial_equals_matrix_exponential():
    rng = np.random.default_rng(2)
    for _ in range(8):
        F = rng.normal(size=3) * 2
        c1d = rng.uniform(-1, 1)
        U = O.spin2_exp_poly(np.array(F[0]), np.array(F[1]), np.array(F[2]), c1d)
        Ff = F[0] * O.FX + F[1] * O.FY + F[2] * O.FZ
        assert np.abs(U - O.expm_hermitian(Ff, -c1d)).max() < 1e-13


def _rk4_nonlinear_point(psi, V, p, T, n):
    """RK4 of Eq. (nonlEQ1) with rho, F, A00 recomputed from Psi each stage."""
    def f(v):
        rho = np.sum(abs(v) ** 2)
        Fz = 2 * abs(v[0]) ** 2 + abs(v[1]) ** 2 - abs(v[3]) ** 2 - 2 * abs(v[4]) ** 2
        Fp = 2 * (np.conj(v[0]) * v[1] + np.conj(v[3]) * v[4]) + math.sqrt(6) * (
            np.conj(v[1]) * v[2] + np.conj(v[2]) * v[3])
        Fm = np.conj(Fp)
        Ff = np.array([[2 * Fz, Fm, 0, 0, 0],
                       [Fp, Fz, S6H * Fm, 0, 0],
                       [0, S6H * Fp, 0, S6H * Fm, 0],
                       [0, 0, S6H * Fp, -Fz, Fm],
                       [0, 0, 0, Fp, -2 * Fz]])
        A00 = (2 * v[0] * v[4] - 2 * v[1] * v[3] + v[2] ** 2) / math.sqrt(5)
        Ac = np.array([np.conj(v[4]), -np.conj(v[3]), np.conj(v[2]), -np.conj(v[1]),
                       np.conj(v[0])]) / math.sqrt(5)
        return -1j * ((V + p.c0 * rho) * v + p.c1 * Ff @ v + p.c2 * A00 * Ac)
    dt = T / n
    for _ in range(n):
        k1 = f(psi)
        k2 = f(psi + 0.5 * dt * k1)
        k3 = f(psi + 0.5 * dt * k2)
        k4 = f(psi + dt * k3)
        psi = psi + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return psi


@pytest.mark.parametrize("seed", range(4))
def test_nonlinear_flow_equals_rk4_of_the_ode(seed):
    rng = np.random.default_rng(100 + seed)
    p = O.Params(omega=0.0, gamma=0.0, c0=rng.uniform(-3, 3), c1=rng.uniform(-3, 3),
                 c2=rng.uniform(-3, 3), gx=0.0, gy=0.0)
    g = O.Grid((2, 2), 1.0)
    psi = (rng.normal(size=(5, 2, 2)) + 1j * rng.normal(size=(5, 2, 2))) * 0.6
    delta = rng.uniform(-0.4, 0.4)
    out = O.nonlinear_substep(psi, g, p, delta, 0.0)
    for j in range(2):
        for k in range(2):
            ref = _rk4_nonlinear_point(psi[:, j, k], 0.0, p, delta, 4000)
            assert np.abs(out[:, j, k] - ref).max() < 1e-11 * np.abs(ref).max()


def test_nonlinear_invariants_and_group_property():
    rng = np.random.default_rng(9)
    g = O.Grid((8, 8), 3.0)
    p = O.Params(omega=0.7, c0=4.0, c1=-2.0, c2=3.0, gx=1.3, gy=0.8)
    psi = rng.normal(size=(5, 8, 8)) + 1j * rng.normal(size=(5, 8, 8))
    d, t = 0.31, 0.9
    out = O.nonlinear_substep(psi, g, p, d, t)
    r0 = O.local_densities(psi)
    r1 = O.local_densities(out)
    for a, b in zip(r0[:4], r1[:4]):            # rho, F_x, F_y, F_z frozen
        assert np.abs(a - b).max() < 1e-12
    V = O.trap_rotated(g, p, t)                 # A00(t) of Sec. 3.2
    A_ref = np.exp(-2j * d * (V + (p.c0 + p.c2 / 5) * r0[0])) * r0[5]
    assert np.abs(r1[5] - A_ref).max() < 1e-12
    two = O.nonlinear_substep(O.nonlinear_substep(psi, g, p, 0.2, t), g, p, 0.11, t)
    assert np.abs(two - out).max() < 1e-12
    back = O.nonlinear_substep(out, g, p, -d, t)
    assert np.abs(back - psi).max() < 1e-12


# ----------------------------------------------------------------------------
# conservation lemmas (Sec. 3.4)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
def test_mass_is_conserved_exactly(scheme):
    g = O.Grid((32, 48), (8.0, 9.0))
    p = O.Params(omega=0.5, gamma=0.9, c0=80, c1=-3, c2=4, gx=1.2, gy=0.9)
    phi = inputs.gaussian_random_phase((32, 48), (8.0, 9.0), seed=3, amp=0.3)
    pr = O.Propagator(g, p)
    out, _ = pr.run(phi, 0.0, 0.01, 20, scheme)
    m0 = O.observables(phi, g, p, 0.0)["mass"]
    m1 = O.observables(out, g, p, 0.2)["mass"]
    assert abs(m1 - m0) < 1e-13


def test_magnetization_conserved_when_gamma_zero():
    g = O.Grid((32, 32), 8.0)
    p = O.Params(omega=0.5, gamma=0.0, c0=50, c1=2, c2=-3, gx=1.3, gy=1.0)
    phi = inputs.gaussian_random_phase((32, 32), 8.0, seed=4, amp=0.5)
    phi[0] *= 1.5
    pr = O.Propagator(g, p)
    out, _ = pr.run(phi, 0.0, 0.02, 15, "ts4")
    m0 = O.observables(phi, g, p, 0.0)["magnetization"]
    m1 = O.observables(out, g, p, 0.3)["magnetization"]
    assert abs(m0) > 0.1
    assert abs(m1 - m0) < 1e-13


# ----------------------------------------------------------------------------
# temporal order and the printed Table 1
# ----------------------------------------------------------------------------
def test_temporal_orders_two_and_four():
    n, L = (48, 48), 8.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.3, gamma=0.4, c0=30, c1=-1, c2=1)
    phi = inputs.gaussian_random_phase(n, L, seed=1, amp=0.2)
    pr = O.Propagator(g, p)
    T = 0.2
    ref, _ = pr.run(phi, 0.0, T / 160, 160, "ts4")
    e = {}
    for sch in ("ts2", "ts4"):
        e[sch] = [O.rel_l2(pr.run(phi, 0.0, T / k, k, sch)[0], ref) for k in (10, 20)]
    r2 = math.log2(e["ts2"][0] / e["ts2"][1])
    r4 = math.log2(e["ts4"][0] / e["ts4"][1])
    assert 1.9 < r2 < 2.1, r2
    assert 3.8 < r4 < 4.2, r4


@pytest.mark.parametrize("sch,order", [("ts2_lnl", 2), ("ts4_l", 4)])
def test_linear_outer_compositions_orders(sch, order):
    """The compositions with the flows' roles exchanged reach the same
    solution (a TS4 reference) at their own orders, and differ from the
    default compositions at finite tau (they are different schemes)."""
    n, L = (48, 48), 8.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.3, gamma=0.4, c0=30, c1=-1, c2=1)
    phi = inputs.gaussian_random_phase(n, L, seed=1, amp=0.2)
    pr = O.Propagator(g, p)
    T = 0.2
    ref, _ = pr.run(phi, 0.0, T / 160, 160, "ts4")
    e = [O.rel_l2(pr.run(phi, 0.0, T / k, k, sch)[0], ref) for k in (10, 20)]
    r = math.log2(e[0] / e[1])
    assert abs(r - order) < 0.15, r
    other = "ts2" if order == 2 else "ts4"
    assert O.rel_l2(pr.run(phi, 0.0, T / 10, 10, sch)[0], pr.run(phi, 0.0, T / 10, 10, other)[0]) > 1e-9


def _golden_table1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_2d_temporal.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[(f[0], int(f[1]))] = [float(v) for v in f[2:]]
    return rows


@pytest.mark.slow
def test_table1_temporal_errors_reproduced():
    """Table 1 (Sec. 4.1), TS2 and TS4 at tau = 1/80: E_l for all five
    components within 0.3% of the printed values.  Run at h = 1/8 (N = 192)
    with a TS4 reference at tau = 1/640 (the paper: h = 1/32, tau0 = 1e-4);
    the temporal error is resolved at this h to the shown digits."""
    n, L = (192, 192), 12.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.2, gamma=0.3, c0=100, c1=-1, c2=1)
    psi0 = inputs.ini_example1(n, L)
    pr = O.Propagator(g, p)
    ref, _ = pr.run(psi0, 0.0, 1.0 / 640, 320, "ts4")
    gold = _golden_table1()
    for sch in ("ts2", "ts4"):
        out, _ = pr.run(psi0, 0.0, 1.0 / 80, 40, sch)
        err = O.component_errors(out, ref)
        for e, pe in zip(err, gold[(sch, 80)]):
            assert abs(e / pe - 1) < 3e-3, (sch, err, gold[(sch, 80)])


# ----------------------------------------------------------------------------
# observables (Sec. 2)
# ----------------------------------------------------------------------------
def test_observables_gaussian_and_vortex_closed_forms():
    n, L = (64, 64), 8.0
    g = O.Grid(n, L)
    X, Y = g.coords()
    G = np.exp(-0.5 * (X ** 2 + Y ** 2)) / math.sqrt(math.pi)   # unit mass in 2D
    phi = np.zeros((5,) + G.shape, complex)
    phi[2] = G
    p = O.Params(omega=0.0, c0=7.0, gx=1.0, gy=1.0)
    ob = O.observables(phi, g, p, 0.0)
    assert abs(ob["mass"] - 1) < 1e-12
    assert abs(ob["e_kin"] - 0.5) < 1e-12          # d/4
    assert abs(ob["e_pot"] - 0.5) < 1e-12          # d/4
    assert abs(ob["e_int"] - 7.0 / 2 / (2 * math.pi)) < 1e-12
    assert abs(ob["width2"][0] - 0.5) < 1e-12
    assert abs(ob["lz"]) < 1e-14
    v = inputs.vortex_state(n, L)                   # (x+iy) G in l = 2
    p2 = O.Params(omega=0.3, c1=2.0, gx=1.0, gy=1.0)
    ob = O.observables(v, g, p2, 0.4)
    assert abs(ob["lz"] - 1.0) < 1e-12
    assert abs(ob["e_kin"] - 1.0) < 1e-12
    assert abs(ob["e_pot"] - 1.0) < 1e-12
    assert abs(ob["e_rot"] + 0.3) < 1e-12
    assert abs(ob["magnetization"] - 2.0) < 1e-12
    # F_z = 2 rho: c1/2 * 4 int rho^2, int rho^2 = 1/(4 pi) for |x+iy|^2 e^{-r^2}/pi
    assert abs(ob["e_int"] - 2.0 * 2.0 / (4 * math.pi)) < 1e-12


def test_soc_energy_equals_physical_space_operator_form():
    """e_soc (Parseval in the oracle) against the printed operator expression
    -gamma [psi2* L- psi1 + psi1*(L+ psi2 + s L- psi0) + ...] in physical space."""
    n, L = (32, 40), (6.0, 7.0)
    g = O.Grid(n, L)
    p = O.Params(gamma=0.7)
    phi = inputs.gaussian_random_phase(n, L, seed=8, amp=2.0)
    ob = O.observables(phi, g, p, 0.0)
    dx, dy = lab_rk4.grad(phi, L[0], L[1])
    Lp = 1j * dy + dx
    Lm = 1j * dy - dx
    c = np.conj(phi)
    dens = (c[0] * Lm[1] + c[1] * (Lp[0] + S6H * Lm[2]) + S6H * c[2] * (Lp[1] + Lm[3])
            + c[3] * (Lm[4] + S6H * Lp[2]) + c[4] * Lp[3])
    ref = -0.7 * g.cell * np.sum(dens)
    assert abs(ref.imag) < 1e-12
    assert abs(ob["e_soc"] - ref.real) < 1e-12 * max(1, abs(ref.real))


@pytest.mark.parametrize("scheme,expect", [("ts2", 4.0), ("ts4", 16.0)])
def test_energy_drift_scales_with_order(scheme, expect):
    n, L = (48, 48), 8.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.4, gamma=0.5, c0=40, c1=-1, c2=2, gx=1.1, gy=0.9)
    phi = inputs.gaussian_random_phase(n, L, seed=6, amp=0.3)
    pr = O.Propagator(g, p)
    T = 0.4
    e0 = O.observables(phi, g, p, 0.0)["energy"]
    drift = []
    for k in (10, 20):
        out, t = pr.run(phi, 0.0, T / k, k, scheme)
        drift.append(abs(O.observables(out, g, p, t)["energy"] - e0))
    ratio = drift[0] / drift[1]
    assert 0.75 * expect < ratio < 1.3 * expect, (drift, ratio)


def test_width_closed_form_lemma2():
    """gamma = 0, isotropic trap, real radially symmetric data: delta_r(t) of
    Eq. (delta_r), with delta_r'(0) = 0."""
    n, L = (128, 128), 16.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.2, gamma=0.0, c0=120.0, c1=1.0, c2=1.0, gx=1.0, gy=1.0)
    psi0 = inputs.ini_example3(n, L)
    ob0 = O.observables(psi0, g, p, 0.0)
    E0, lz0 = ob0["energy"], ob0["lz"]
    d0 = ob0["width2"][0] + ob0["width2"][1]
    pr = O.Propagator(g, p)
    phi, t = psi0, 0.0
    for T in (0.25, 0.5):
        phi, t = pr.run(phi, t, 1.0 / 200, 50, "ts4")
        ob = O.observables(phi, g, p, t)
        dr = ob["width2"][0] + ob["width2"][1]
        ref = (E0 + p.omega * lz0) * (1 - math.cos(2 * t)) + d0 * math.cos(2 * t)
        assert abs(dr - ref) < 1e-6 * abs(ref), (t, dr, ref)
        assert abs(ob["width2"][0] - ob["width2"][1]) < 1e-8 * dr


def _central_rate(pr, phi, t0, eps, fn):
    a, _ = pr.run(phi, t0, -eps / 4, 4, "ts4")
    b, _ = pr.run(phi, t0, eps / 4, 4, "ts4")
    return (fn(b, t0 + eps) - fn(a, t0 - eps)) / (2 * eps)


def test_magnetization_law_with_soc():
    """dM/dt = 2 gamma Re int i (psi2* L- psi1 - psi_-2 L- conj(psi_-1)
    + s psi1* L- psi0 - s psi_-1 L- conj(psi0)) (Sec. 2, Magnetization)."""
    n, L = (48, 48), 8.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.3, gamma=0.6, c0=20, c1=-1, c2=1, gx=1.1, gy=0.9)
    phi = inputs.gaussian_random_phase(n, L, seed=12, amp=1.0)
    phi[0] *= 1.4
    pr = O.Propagator(g, p)
    phi, t0 = pr.run(phi, 0.0, 0.01, 10, "ts4")
    rate = _central_rate(pr, phi, t0, 2e-3,
                         lambda f, t: O.observables(f, g, p, t)["magnetization"])

    def Lminus(f):
        dx, dy = lab_rk4.grad(f, L, L)
        return 1j * dy - dx
    c = np.conj
    dens = (c(phi[0]) * Lminus(phi[1]) - phi[4] * Lminus(c(phi[3]))
            + S6H * c(phi[1]) * Lminus(phi[2]) - S6H * phi[3] * Lminus(c(phi[2])))
    law = 2 * p.gamma * np.real(1j * g.cell * np.sum(dens))
    assert abs(law) > 1e-3
    assert abs(rate - law) < 1e-5 * abs(law) + 1e-9, (rate, law)


def test_angular_momentum_law_anisotropic_trap():
    """d<L_z>/dt = (gx^2 - gy^2) int x y rho (gamma = 0, lab coordinates x, y)."""
    n, L = (64, 64), 8.0
    g = O.Grid(n, L)
    p = O.Params(omega=0.35, gamma=0.0, c0=20, c1=-1, c2=1, gx=1.3, gy=1.0)
    phi = inputs.gaussian_random_phase(n, L, seed=13, amp=1.0)
    X, Y = g.coords()
    phi = phi * np.exp(-0.2 * (X - 0.5 * Y) ** 2)
    pr = O.Propagator(g, p)
    phi, t0 = pr.run(phi, 0.0, 0.02, 10, "ts4")
    rate = _central_rate(pr, phi, t0, 1e-3, lambda f, t: O.observables(f, g, p, t)["lz"])
    co, si = math.cos(p.omega * t0), math.sin(p.omega * t0)
    xl, yl = co * X + si * Y, -si * X + co * Y
    rho = np.sum(np.abs(phi) ** 2, axis=0)
    law = (p.gx ** 2 - p.gy ** 2) * g.cell * np.sum(xl * yl * rho)
    assert abs(law) > 1e-3
    assert abs(rate - law) < 2e-6 * abs(law), (rate, law)


# ----------------------------------------------------------------------------
# the whole scheme against an independent lab-frame integrator
# ----------------------------------------------------------------------------
def test_splitting_converges_to_lab_frame_rk4():
    """TS4 in the rotating frame, mapped back by psi_l(x) = e^{i l Omega T}
    phi_l(R(T)^{-1} x), against RK4 of the lab-frame Eq. (CGPEs) with the
    rotation term in physical space (anisotropic trap, SOC on)."""
    n, L = (48, 48), 6.0
    g = O.Grid(n, L)
    pd = dict(omega=0.5, gamma=0.4, c0=5.0, c1=-1.0, c2=2.0, gx=1.2, gy=0.9)
    p = O.Params(**pd)
    psi0 = inputs.gaussian_random_phase(n, L, seed=21, amp=0.3)
    X, Y = g.coords()
    T = 0.2
    lab = lab_rk4.integrate(psi0, X, Y, L, L, pd, T, 2e-4)
    pr = O.Propagator(g, p)
    phi, t = pr.run(psi0, 0.0, T / 40, 40, "ts4")
    co, si = math.cos(p.omega * T), math.sin(p.omega * T)
    xq, yq = co * X - si * Y, si * X + co * Y        # R(T)^{-1} x
    mapped = np.stack([np.exp(1j * l * p.omega * T) * lab_rk4.trig_interp(phi[c], L, L, xq, yq)
                       for c, l in enumerate((2, 1, 0, -1, -2))])
    err = O.rel_l2(mapped, lab)
    assert err < 2e-7, err
