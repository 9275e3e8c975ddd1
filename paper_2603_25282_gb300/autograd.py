"""Differentiable propagation: torch.autograd.Function over the C ABI.

``propagate(ctx, psi0, prm, nsteps, dt, scheme)`` advances psi0 (a complex
CUDA tensor in the context's layout and precision) by nsteps of the
composition with the per-member parameters prm = (Omega, gamma, c0, c1, c2)
(a float64 tensor of shape (batch, 5)), returning the final rotating-frame
field.  Its backward calls ``sgp_backward``: the hand-written adjoint of the
recorded run, with sqrt(nsteps) checkpoints by default.  Both directions run
in the CUDA library; this module only moves pointers and orders streams.

Gradient convention (torch's): for a real objective J, the gradient of a
complex tensor is dJ/dRe + i dJ/dIm, which is what sgp_backward takes and
returns.  The trap frequencies come from ``trap`` and are not differentiated.
"""
from __future__ import annotations

import torch

from . import sgp

PRM_NAMES = ("omega", "gamma", "c0", "c1", "c2")


def _record(ctx, run):
    plist, psi0c, t0, nsteps, dt, scheme, interval = run
    ctx.set_params_batch(plist)
    ctx.set_state(psi0c, t0)
    ctx.record(nsteps, dt, scheme, interval)
    ctx._adj_run = run


class Propagate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, psi0, prm, ctx, nsteps, dt, scheme, interval, t0, trap):
        if not psi0.is_cuda:
            raise ValueError("psi0 must be a CUDA tensor")
        vals = prm.detach().to("cpu", torch.float64).reshape(ctx.batch, 5).tolist()
        plist = [dict(zip(PRM_NAMES, row), gx=trap[0], gy=trap[1], gz=trap[2]) for row in vals]
        psi0c = psi0.detach().contiguous()
        torch.cuda.current_stream(psi0.device).synchronize()
        run = (plist, psi0c, t0, nsteps, dt, scheme, interval)
        _record(ctx, run)
        out = torch.empty_like(psi0c)
        ctx.get_state(out)
        ctx.synchronize()
        fctx.sgp = ctx
        fctx.run = run
        fctx.prm_shape = prm.shape
        fctx.prm_device = prm.device
        return out

    @staticmethod
    def backward(fctx, g_out):
        ctx = fctx.sgp
        g = g_out.contiguous()
        torch.cuda.current_stream(g.device).synchronize()
        if getattr(ctx, "_adj_run", None) is not fctx.run:
            _record(ctx, fctx.run)     # the context recorded another run since
        g0 = torch.empty_like(g)
        _, dp = ctx.backward(g, g0)
        dprm = torch.as_tensor(dp, dtype=torch.float64).reshape(fctx.prm_shape).to(fctx.prm_device)
        return g0, dprm, None, None, None, None, None, None, None


def propagate(ctx, psi0, prm, nsteps, dt, scheme="ts2", interval=0, t0=0.0,
              trap=(1.0, 1.0, 1.0)):
    """Differentiable nsteps of the composition on the sgp context ``ctx``."""
    return Propagate.apply(psi0, prm, ctx, int(nsteps), float(dt), scheme, int(interval),
                           float(t0), tuple(float(v) for v in trap))


def density_misfit(phiT, n, L, omega, T, centres, weights):
    """J = h^d sum_{l,j} (|phi_l(x_j, T)|^2 - rho_l(R(T) x_j))^2 in torch.

    rho_l(y) = w_l exp(-|y - c_l|^2) (centres and weights from
    ``inputs.density_target``); R(T) x = (x cos + y sin, -x sin + y cos[, z])
    with the angle omega*T, so J is differentiable in omega (a tensor) through
    the frame.  phiT: (5, [nz,] ny, nx) or (batch, 5, ...) complex tensor.
    """
    dev = phiT.device
    d = len(n)
    Ls = (float(L),) * d if not hasattr(L, "__len__") else tuple(float(v) for v in L)
    axes = [torch.arange(N, device=dev, dtype=torch.float64) * (2.0 * Lk / N) - Lk
            for N, Lk in zip(n, Ls)]
    grids = torch.meshgrid(*axes[::-1], indexing="ij")[::-1]     # X, Y[, Z] in array order
    cell = 1.0
    for N, Lk in zip(n, Ls):
        cell *= 2.0 * Lk / N
    ang = omega * T
    co, si = torch.cos(ang), torch.sin(ang)
    Y = [co * grids[0] + si * grids[1], -si * grids[0] + co * grids[1]] + list(grids[2:])
    c = torch.as_tensor(centres, dtype=torch.float64, device=dev)
    w = torch.as_tensor(weights, dtype=torch.float64, device=dev)
    tgt = torch.stack([w[m] * torch.exp(-sum((Y[a] - c[m, a]) ** 2 for a in range(d)))
                       for m in range(5)])
    dens = (phiT.real.double() ** 2 + phiT.imag.double() ** 2)
    return cell * ((dens - tgt) ** 2).sum()
