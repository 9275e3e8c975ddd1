"""The persistent work-queue kernel of 2D ensembles (sgp_ensemble_* with the
persistent kernel in use), through the C ABI.

  * It gives the same fields, bit for bit, as the per-group launches of the
    same passes (the graph of parallel branches), over a run that uses a
    captured 64-step launch and a directly launched rest.
  * It matches the FP64 oracle (1e-10 FP64, 1e-5 FP32) on a mixed-size
    ensemble with per-member parameters.
  * Its bounded waits: a test-only hook withholds one completion signal on
    the device; the dependent wait gives up after the configured limit, the
    call returns SGP_ETIMEOUT, nothing traps or hangs, and the ensemble runs
    normally once its states are set again.
"""
import time

import numpy as np
import pytest

from oracle import sgp_oracle as O
from paper_2603_25282_gb300 import inputs, sgp

pytestmark = pytest.mark.gpu

KEYS = ("omega", "gamma", "c0", "c1", "c2", "gx", "gy", "gz")


def _members(sides, per_side, seed):
    pool = inputs.ensemble_members(200, seed=seed, sides=sides)
    out = []
    for s in sides:
        out += [m for m in pool if m["n"] == s][:per_side]
    return out


def _ensemble(members, prec, persistent):
    ens = sgp.Ensemble([((m["n"], m["n"]), m["L"]) for m in members], prec=prec)
    ens.set_params([{k: m[k] for k in KEYS} for m in members])
    if not persistent:
        ens.set_persistent(False)
    assert ens.persistent == persistent
    return ens


def _init(ens, members, amp=0.3):
    psis = [inputs.gaussian_random_phase((m["n"], m["n"]), m["L"], seed=m["seed"], amp=amp)
            for m in members]
    for i, p in enumerate(psis):
        ens.set_member_state(i, p.astype(ens.dtype))
    return psis


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("scheme", ["ts2", "ts4"])
def test_persistent_equals_group_launches_bitwise(prec, scheme):
    members = _members((64, 96, 128, 192, 256), 2, seed=7)
    out = []
    for persistent in (True, False):
        ens = _ensemble(members, prec, persistent)
        _init(ens, members)
        ens.step(70, 1e-3, scheme)          # one captured 64-step launch + 6 steps launched directly
        out.append([ens.get_member_state(i) for i in range(len(members))])
        ens.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_persistent_matches_oracle(prec, tol):
    members = _members((64, 96, 128), 2, seed=8)
    ens = _ensemble(members, prec, True)
    psis = _init(ens, members)
    ens.step(12, 1e-3, "ts4")
    for i, m in enumerate(members):
        ref = O.Propagator(O.Grid((m["n"], m["n"]), m["L"]),
                           O.Params(**{k: m[k] for k in KEYS})).run(psis[i], 0.0, 1e-3, 12, "ts4")[0]
        got = ens.get_member_state(i).astype(np.complex128)
        assert O.rel_l2(got, ref) < tol, (m["n"], O.rel_l2(got, ref))
    ens.close()


def test_bounded_wait_gives_up_with_etimeout():
    members = _members((64, 128, 256), 2, seed=9)
    ens = _ensemble(members, "f32", True)
    psis = _init(ens, members)
    ens.set_wait_limit(0.05)
    ens.inject_stall(3)
    t0 = time.perf_counter()
    with pytest.raises(sgp.SgpError, match="SGP_ETIMEOUT"):
        ens.step(8, 1e-3, "ts2")
    assert time.perf_counter() - t0 < 30.0
    # the ensemble is usable again once its states are set
    for i, p in enumerate(psis):
        ens.set_member_state(i, p.astype(np.complex64), 0.0)
    ens.step(8, 1e-3, "ts2")
    got = [ens.get_member_state(i) for i in range(len(members))]
    ens.close()
    ref_ens = _ensemble(members, "f32", False)
    _init(ref_ens, members)
    ref_ens.step(8, 1e-3, "ts2")
    for i in range(len(members)):
        assert np.array_equal(got[i], ref_ens.get_member_state(i))
    ref_ens.close()


def test_ensembles_outside_the_persistent_kernel():
    """3D ensembles and line lengths the kernel is not compiled for use the
    per-group launches; asking for the persistent kernel is refused."""
    for grids in ([((32, 32), 8.0), ((64, 64), 8.0)], [((16, 16, 16), 6.0)]):
        ens = sgp.Ensemble(grids, prec="f32")
        assert not ens.persistent
        with pytest.raises(sgp.SgpError, match="SGP_EUNSUPPORTED"):
            ens.set_persistent(True)
        with pytest.raises(sgp.SgpError, match="SGP_EUNSUPPORTED"):
            ens.inject_stall(0)
        ens.close()
    ens = sgp.Ensemble([((64, 64), 8.0)], prec="f32")
    with pytest.raises(sgp.SgpError, match="SGP_EINVAL"):
        ens.set_wait_limit(0.0)
    ens.close()
