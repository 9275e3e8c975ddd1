"""GPU parity of the adjoint (sgp_record / sgp_backward and the autograd
Function) against the two FP64 oracle gradients (the tangent-linear one of
oracle/sgp_tangent.py and the central differences of oracle/sgp_grad.py)
and GPU central finite differences.

Objective: the terminal density misfit J of oracle/sgp_grad.py.  Gradient
convention dJ/dRe + i dJ/dIm; parameter slots (Omega, gamma, c0, c1, c2).
Tolerances:
  * FP64 GPU adjoint vs the tangent-linear oracle gradient: 1e-8 relative
    (both exact up to FP64 rounding);
  * FP64 GPU adjoint vs oracle central FD: 1e-6 relative (the FD truncation
    error of the pinned oracle gradient is about 1e-8 relative at these
    steps; the adjoint itself is exact up to rounding);
  * FP64 GPU adjoint vs GPU central FD at the 256^2, 2000-step workload:
    1e-6 relative;
  * FP32 GPU adjoint vs the FP64 ones: 1e-4 relative, the accuracy the
    gradients are specified to.
"""
import dataclasses
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import sgp_grad as G
from oracle import sgp_oracle as O
from oracle import sgp_tangent as TL
from paper_2603_25282_gb300 import inputs, sgp
from paper_2603_25282_gb300.autograd import density_misfit, propagate

NAMES = ("omega", "gamma", "c0", "c1", "c2")


def _gT(phiT, n, L, omega, T, c, w):
    """dJ/dRe + i dJ/dIm of the misfit at phiT (closed form, host)."""
    grid = O.Grid(n, L)
    tgt = G.target_density(grid, omega, T, c, w)
    return 4.0 * grid.cell * (np.abs(phiT) ** 2 - tgt) * phiT


def _frame_term(phiT, n, L, omega, T, c, w):
    """dJ/dOmega through R(T) only (the target), closed form."""
    grid = O.Grid(n, L)
    X = grid.coords()
    co, si = math.cos(omega * T), math.sin(omega * T)
    Y = G.rotated_coords(grid, omega, T)
    dY = [T * (-si * X[0] + co * X[1]), T * (-co * X[0] - si * X[1])]
    tgt = G.target_density(grid, omega, T, c, w)
    dtgt = np.stack([tgt[m] * sum(-2.0 * (Y[a] - c[m][a]) * dY[a] for a in range(2))
                     for m in range(5)])
    return grid.cell * float(np.sum(-2.0 * (np.abs(phiT) ** 2 - tgt) * dtgt))


def _run_adjoint(n, L, prm, psi0, dt, nsteps, scheme, prec, c, w, interval=0):
    ctx = sgp.Context(n, L, batch=1, prec=prec)
    ctx.set_params(**dataclasses.asdict(prm))
    dtype = np.complex64 if prec == "f32" else np.complex128
    ctx.set_state(psi0.astype(dtype)[None].copy(), 0.0)
    ctx.record(nsteps, dt, scheme, interval)
    phiT = ctx.get_state()[0].astype(np.complex128)
    T = nsteps * dt
    gT = _gT(phiT, n, L, prm.omega, T, c, w).astype(dtype)[None].copy()
    g0, dp = ctx.backward(gT)
    dp = dp[0].copy()
    dp[0] += _frame_term(phiT, n, L, prm.omega, T, c, w)
    ctx.close()
    return g0[0].astype(np.complex128), dp


PRM_SMALL = O.Params(omega=0.6, gamma=1.0, c0=400.0, c1=-3.0, c2=5.0, gx=1.0, gy=1.3)


@pytest.mark.parametrize("scheme,nsteps,interval", [("ts2", 6, 0), ("ts4", 4, 3), ("ts2", 5, 1),
                                                     ("ts2_lnl", 5, 2), ("ts4_l", 4, 3)])
def test_adjoint_fp64_matches_oracle_fd(scheme, nsteps, interval):
    n, L, dt = (16, 16), 8.0, 2e-3
    psi0 = inputs.gaussian_random_phase(n, L, seed=11, amp=0.3)
    c, w = inputs.density_target(n, L, seed=12)
    g0, dp = _run_adjoint(n, L, PRM_SMALL, psi0, dt, nsteps, scheme, "f64", c, w, interval)
    grid = O.Grid(n, L)
    rng = np.random.default_rng(13)
    dirs = [rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape) for _ in range(3)]
    fd_dirs, fd_par = G.gradient_fd(psi0, grid, PRM_SMALL, dt, nsteps, scheme, c, w,
                                    directions=dirs, params=NAMES)
    for V, ref in zip(dirs, fd_dirs):
        got = float(np.real(np.vdot(g0, V)))
        assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)
    scale = max(abs(v) for v in fd_par.values())
    for k, name in enumerate(NAMES):
        assert abs(dp[k] - fd_par[name]) <= 1e-6 * scale, (name, dp[k], fd_par[name])


@pytest.mark.parametrize("scheme,nsteps,interval", [("ts2", 6, 0), ("ts4", 4, 3), ("ts2_lnl", 5, 2),
                                                     ("ts4_l", 4, 1)])
def test_adjoint_fp64_matches_tangent_oracle(scheme, nsteps, interval):
    """The adjoint (reverse sweep over the checkpointed run) against the
    forward-mode dual-number gradient of the oracle: three state directions
    and all five parameters to 1e-8."""
    n, L, dt = (16, 16), 8.0, 2e-3
    psi0 = inputs.gaussian_random_phase(n, L, seed=14, amp=0.3)
    c, w = inputs.density_target(n, L, seed=15)
    g0, dp = _run_adjoint(n, L, PRM_SMALL, psi0, dt, nsteps, scheme, "f64", c, w, interval)
    grid = O.Grid(n, L)
    rng = np.random.default_rng(16)
    dirs = [rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape) for _ in range(3)]
    tl_dirs, tl_par = TL.gradient_tangent(psi0, grid, PRM_SMALL, dt, nsteps, scheme, c, w,
                                          directions=dirs, params=NAMES)
    for V, ref in zip(dirs, tl_dirs):
        got = float(np.real(np.vdot(g0, V)))
        assert abs(got - ref) <= 1e-8 * abs(ref), (got, ref)
    scale = max(abs(v) for v in tl_par.values())
    for k, name in enumerate(NAMES):
        assert abs(dp[k] - tl_par[name]) <= 1e-8 * scale, (name, dp[k], tl_par[name])


def test_adjoint_fp64_3d_matches_tangent_oracle():
    n, L, dt, nsteps = (16, 16, 16), 6.0, 2e-3, 3
    prm = dataclasses.replace(PRM_SMALL, gz=1.7)
    psi0 = inputs.gaussian_random_phase(n, L, seed=24, amp=0.3)
    c, w = inputs.density_target(n, L, seed=25)
    g0, dp = _run_adjoint(n, L, prm, psi0, dt, nsteps, "ts4", "f64", c, w)
    V = np.random.default_rng(26).standard_normal(psi0.shape) * (1 + 1j)
    tl_dirs, tl_par = TL.gradient_tangent(psi0, O.Grid(n, L), prm, dt, nsteps, "ts4", c, w,
                                          directions=[V], params=NAMES)
    got = float(np.real(np.vdot(g0, V)))
    assert abs(got - tl_dirs[0]) <= 1e-8 * abs(tl_dirs[0])
    scale = max(abs(v) for v in tl_par.values())
    for k, name in enumerate(NAMES):
        assert abs(dp[k] - tl_par[name]) <= 1e-8 * scale, name


def test_adjoint_fp64_3d_matches_oracle_fd():
    n, L, dt, nsteps = (16, 16, 16), 6.0, 2e-3, 3
    prm = dataclasses.replace(PRM_SMALL, gz=1.7)
    psi0 = inputs.gaussian_random_phase(n, L, seed=21, amp=0.3)
    c, w = inputs.density_target(n, L, seed=22)
    # 3D: the frame acts on (x, y) only, as in _frame_term
    g0, dp = _run_adjoint(n, L, prm, psi0, dt, nsteps, "ts2", "f64", c, w)
    grid = O.Grid(n, L)
    rng = np.random.default_rng(23)
    V = rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)
    fd_dirs, fd_par = G.gradient_fd(psi0, grid, prm, dt, nsteps, "ts2", c, w,
                                    directions=[V], params=NAMES)
    got = float(np.real(np.vdot(g0, V)))
    assert abs(got - fd_dirs[0]) <= 1e-6 * abs(fd_dirs[0])
    scale = max(abs(v) for v in fd_par.values())
    for k, name in enumerate(NAMES):
        assert abs(dp[k] - fd_par[name]) <= 1e-6 * scale, name


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_backward_graph_replay_equals_eager(prec):
    n, L, dt, nsteps = (32, 32), 8.0, 1e-3, 30
    psi0 = inputs.gaussian_random_phase(n, L, seed=51, amp=0.3)
    dtype = np.complex64 if prec == "f32" else np.complex128
    rng = np.random.default_rng(52)
    gT = (rng.standard_normal((1, 5) + n) + 1j * rng.standard_normal((1, 5) + n)).astype(dtype)
    out = []
    for graphs in (True, False):
        ctx = sgp.Context(n, L, prec=prec)
        ctx.set_graphs(graphs)
        ctx.set_params(**dataclasses.asdict(PRM_SMALL))
        ctx.set_state(psi0.astype(dtype)[None].copy(), 0.0)
        ctx.record(nsteps, dt, "ts2", 4)          # 8 segments, the first one ragged
        out.append(ctx.backward(gT))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_adjoint_global_phase_invariance():
    n, L = (32, 32), 8.0
    psi0 = inputs.gaussian_random_phase(n, L, seed=31, amp=0.3)
    c, w = inputs.density_target(n, L, seed=32)
    g0, _ = _run_adjoint(n, L, PRM_SMALL, psi0, 1e-3, 20, "ts2", "f64", c, w)
    lhs = float(np.real(np.vdot(g0, 1j * psi0)))
    assert abs(lhs) <= 1e-10 * float(np.linalg.norm(g0) * np.linalg.norm(psi0))


def test_backward_without_record_is_an_error():
    ctx = sgp.Context((16, 16), 8.0, prec="f64")
    ctx.set_params(omega=0.5)
    ctx.set_state(np.zeros((1, 5, 16, 16), np.complex128))
    with pytest.raises(sgp.SgpError):
        ctx.backward(np.zeros((1, 5, 16, 16), np.complex128))
    ctx.record(3, 1e-3)
    ctx.step(1, 1e-3)                      # invalidates the record
    with pytest.raises(sgp.SgpError):
        ctx.backward(np.zeros((1, 5, 16, 16), np.complex128))
    ctx.close()


def test_autograd_gradcheck_fp64():
    n, L = (16, 16), 6.0
    ctx = sgp.Context(n, L, prec="f64")
    psi0 = torch.from_numpy(inputs.gaussian_random_phase(n, L, seed=41, amp=0.3)[None].copy()).cuda()
    prm = torch.tensor([[0.6, 1.0, 40.0, -3.0, 5.0]], dtype=torch.float64, device="cuda")
    psi0.requires_grad_(True)
    prm.requires_grad_(True)
    f = lambda p0, pr: propagate(ctx, p0, pr, 3, 2e-3, "ts2", trap=(1.0, 1.3, 1.0))
    assert torch.autograd.gradcheck(f, (psi0, prm), eps=1e-6, atol=1e-7, rtol=1e-5,
                                    fast_mode=True)
    ctx.close()


def _c5_setup(prec):
    n, L = (256, 256), 8.0
    prm = O.Params(omega=0.6, gamma=1.0, c0=400.0, c1=-1.0, c2=2.0)
    psi0 = inputs.gaussian_random_phase(n, L, seed=5, amp=0.01)
    c, w = inputs.density_target(n, L, seed=6)
    return n, L, prm, psi0, c, w


def _c5_objective(ctx, n, L, prm, psi0, c, w, nsteps, dt):
    ctx.set_params(**dataclasses.asdict(prm))
    ctx.set_state(psi0.astype(ctx.dtype)[None].copy(), 0.0)
    ctx.step(nsteps, dt, "ts2")
    phiT = ctx.get_state()[0].astype(np.complex128)
    return G.misfit(phiT, O.Grid(n, L), prm.omega, nsteps * dt, c, w)


@pytest.fixture(scope="module")
def c5_results():
    """Adjoint gradients of the 256^2, 2000-step workload in FP64 and FP32
    and FP64 GPU central differences for a state direction and Omega,
    gamma, c1."""
    n, L, prm, psi0, c, w = _c5_setup("f64")
    nsteps, dt = 2000, 1e-3
    res = {}
    for prec in ("f64", "f32"):
        res[prec] = _run_adjoint(n, L, prm, psi0, dt, nsteps, "ts2", prec, c, w)
    rng = np.random.default_rng(7)
    V = (rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)) * np.abs(psi0)
    ctx = sgp.Context(n, L, prec="f64")
    J = lambda P, p: _c5_objective(ctx, n, L, p, P, c, w, nsteps, dt)
    hs = 1e-4
    fd = {"dir": (J(psi0 + hs * V, prm) - J(psi0 - hs * V, prm)) / (2 * hs)}
    for name, h in (("omega", 1e-5), ("gamma", 1e-5), ("c1", 1e-4)):
        v = getattr(prm, name)
        fd[name] = (J(psi0, dataclasses.replace(prm, **{name: v + h}))
                    - J(psi0, dataclasses.replace(prm, **{name: v - h}))) / (2 * h)
    ctx.close()
    return dict(res=res, fd=fd, V=V)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c5_adjoint_matches_central_fd(c5_results, prec):
    g0, dp = c5_results["res"][prec]
    fd = c5_results["fd"]
    tol = 1e-6 if prec == "f64" else 1e-4
    got = float(np.real(np.vdot(g0, c5_results["V"])))
    assert abs(got - fd["dir"]) <= tol * abs(fd["dir"]), (got, fd["dir"])
    for k, name in ((0, "omega"), (1, "gamma"), (3, "c1")):
        assert abs(dp[k] - fd[name]) <= tol * abs(fd[name]), (name, dp[k], fd[name])


def test_c5_fp32_gradient_field_close_to_fp64(c5_results):
    g64, dp64 = c5_results["res"]["f64"]
    g32, dp32 = c5_results["res"]["f32"]
    assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64)
    for k in range(5):
        assert abs(dp32[k] - dp64[k]) <= 1e-4 * max(abs(dp64[k]), 1e-12 * np.abs(dp64).max())
