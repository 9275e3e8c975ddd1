"""Thin Python binding of the C ABI in ``include/sgp.h`` (libsgp.so).

Argument marshalling only: every step of the propagator runs in the CUDA
library.  The functions keep the C names (create_grid, set_params,
set_state, get_state, step, substep, observables, synchronize, destroy);
``Context`` bundles them for convenience.  Fields are numpy arrays (host) or
torch tensors (host or CUDA) of complex64 (F32 contexts) or complex128 (F64),
shaped (batch, 5, [nz,] ny, nx) or, for batch 1, (5, [nz,] ny, nx).

There is no fallback: if libsgp.so is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgp.so")

SGP_F32, SGP_F64 = 32, 64
SGP_TS2, SGP_TS4, SGP_TS2_LNL, SGP_TS4_LOUTER = 0, 1, 2, 3
SGP_SUB_NONLINEAR, SGP_SUB_LINEAR = 0, 1
SCHEMES = {"ts2": SGP_TS2, "ts4": SGP_TS4, "ts2_lnl": SGP_TS2_LNL, "ts4_l": SGP_TS4_LOUTER}
PRECS = {"f32": SGP_F32, "f64": SGP_F64}


class SgpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("omega", "gamma", "c0", "c1", "c2", "gx", "gy", "gz")]


class Obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("mass", ctypes.c_double),
                ("energy", ctypes.c_double), ("magnetization", ctypes.c_double),
                ("lz", ctypes.c_double), ("comp_mass", ctypes.c_double * 5),
                ("width2", ctypes.c_double * 3), ("e_kin", ctypes.c_double),
                ("e_pot", ctypes.c_double), ("e_rot", ctypes.c_double),
                ("e_int", ctypes.c_double), ("e_soc", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["comp_mass"] = list(self.comp_mass)
        d["width2"] = list(self.width2)
        return d


_lib = None

# caller allocator callbacks (sgp_set_allocator)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                            ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_allocator_keep = None      # the registered callbacks must outlive their use


def lib():
    """Load libsgp.so once (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsgp.so is not built (run __graft_entry__.build() or "
                           "python paper_2603_25282_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "sgp_version": (I, []),
        "sgp_status_string": (ctypes.c_char_p, [I]),
        "sgp_last_error": (ctypes.c_char_p, [P]),
        "sgp_create_grid": (I, [I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                I, I, I, P, ctypes.POINTER(P)]),
        "sgp_set_params": (I, [P, ctypes.POINTER(Params)]),
        "sgp_set_params_batch": (I, [P, ctypes.POINTER(Params), I]),
        "sgp_set_graphs": (I, [P, I]),
        "sgp_ensemble_create": (I, [I, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                    I, I, P, ctypes.POINTER(P)]),
        "sgp_ensemble_groups": (I, [P]),
        "sgp_ensemble_set_params": (I, [P, ctypes.POINTER(Params)]),
        "sgp_ensemble_set_member_state": (I, [P, I, P, I, D]),
        "sgp_ensemble_get_member_state": (I, [P, I, P, I]),
        "sgp_ensemble_step": (I, [P, LL, D, I]),
        "sgp_ensemble_step_host": (I, [P, ctypes.POINTER(P), D, ctypes.POINTER(P), LL, D, I]),
        "sgp_ensemble_observables": (I, [P, ctypes.POINTER(Obs)]),
        "sgp_ensemble_synchronize": (I, [P]),
        "sgp_ensemble_launch_count": (LL, [P]),
        "sgp_ensemble_last_error": (ctypes.c_char_p, [P]),
        "sgp_ensemble_destroy": (I, [P]),
        "sgp_set_state": (I, [P, P, I, D]),
        "sgp_get_state": (I, [P, P, I]),
        "sgp_get_time": (I, [P, ctypes.POINTER(ctypes.c_double)]),
        "sgp_get_state_lab": (I, [P, P, I]),
        "sgp_step": (I, [P, LL, D, I]),
        "sgp_step_host": (I, [P, P, D, P, LL, D, I, I]),
        "sgp_substep_plan": (I, [I, LL, D, LL, ctypes.c_char_p, ctypes.POINTER(D),
                                 ctypes.POINTER(D), ctypes.POINTER(LL)]),
        "sgp_substep": (I, [P, I, D]),
        "sgp_observables": (I, [P, ctypes.POINTER(Obs)]),
        "sgp_synchronize": (I, [P]),
        "sgp_launch_count": (LL, [P]),
        "sgp_destroy": (I, [P]),
        "sgp_observables_static": (I, [I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                       I, I, ctypes.POINTER(Params), D, P, I, P, ctypes.POINTER(Obs)]),
        "sgp_set_allocator": (I, [ALLOC_FN, FREE_FN, P]),
        "sgp_set_health_check": (I, [P, LL, D]),
        "sgp_variant_exists": (I, [I, I, I]),
        "sgp_set_plan": (I, [P, ctypes.POINTER(ctypes.c_int)]),
        "sgp_get_plan": (I, [P, ctypes.POINTER(ctypes.c_int)]),
        "sgp_autotune": (I, [P, I, I, ctypes.POINTER(ctypes.c_double)]),
        "sgp_ensemble_autotune": (I, [P, I, I]),
        "sgp_ensemble_set_persistent": (I, [P, I]),
        "sgp_ensemble_persistent": (I, [P]),
        "sgp_ensemble_set_wait_limit": (I, [P, D]),
        "sgp_ensemble_inject_stall": (I, [P, I]),
        "sgp_record": (I, [P, LL, D, I, LL]),
        "sgp_backward": (I, [P, P, I, P, I, ctypes.POINTER(ctypes.c_double)]),
        "sgp_set_profiling": (I, [P, I]),
        "sgp_get_profile": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status, ctx=None):
    if status != 0:
        L = lib()
        msg = L.sgp_last_error(ctx).decode()
        raise SgpError(L.sgp_status_string(status).decode(), msg)


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != dtype:
            raise TypeError("field dtype %s, expected %s" % (x.dtype, np.dtype(dtype)))
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("field must be C-contiguous")
        return x.ctypes.data, 0, x
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        want = torch.complex64 if np.dtype(dtype) == np.complex64 else torch.complex128
        if x.dtype != want:
            raise TypeError("field dtype %s, expected %s" % (x.dtype, want))
        if not x.is_contiguous():
            raise ValueError("field must be contiguous")
        return x.data_ptr(), int(x.is_cuda), x
    raise TypeError("field must be a numpy array or a torch tensor")


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------
def create_grid(n, L, batch=1, prec="f32", device=0, stream=None):
    """sgp_create_grid; n and L in (x, y[, z]) order.  Returns the handle."""
    dim = len(n)
    if np.isscalar(L):
        L = [float(L)] * dim
    m = max(3, dim)
    na = (ctypes.c_int * m)(*(list(n) + [1] * (m - dim)))
    La = (ctypes.c_double * m)(*(list(L) + [1.0] * (m - len(L))))
    out = ctypes.c_void_p()
    st = lib().sgp_create_grid(dim, na, La, int(batch), PRECS[prec] if isinstance(prec, str) else prec,
                               int(device), ctypes.c_void_p(stream or 0), ctypes.byref(out))
    _check(st, None)
    return out


def _params(kw):
    return Params(**{k: float(kw.get(k, 1.0 if k in ("gx", "gy", "gz") else 0.0))
                     for k, _ in Params._fields_})


def use_torch_allocator(enable=True):
    """sgp_set_allocator with PyTorch's caching allocator (contexts created
    afterwards take their device memory from torch's pool; it shows in
    torch.cuda.memory_allocated).  enable=False restores cudaMalloc."""
    global _allocator_keep
    if not enable:
        _check(lib().sgp_set_allocator(ALLOC_FN(), FREE_FN(), None), None)
        _allocator_keep = None
        return
    import torch

    def _alloc(size, device, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), int(device), int(stream or 0))
        except Exception:
            return None

    def _free(ptr, device, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    keep = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().sgp_set_allocator(keep[0], keep[1], None), None)
    _allocator_keep = keep


def set_params(ctx, **kw):
    p = _params(kw)
    _check(lib().sgp_set_params(ctx, ctypes.byref(p)), ctx)


def set_params_batch(ctx, plist):
    """Per-member parameters: plist is a list of dicts (one per member)."""
    arr = (Params * len(plist))(*[_params(d) for d in plist])
    _check(lib().sgp_set_params_batch(ctx, arr, len(plist)), ctx)


def set_health_check(ctx, every, drift_tol):
    """sgp_set_health_check: mass checked every `every` steps of sgp_step."""
    _check(lib().sgp_set_health_check(ctx, int(every), float(drift_tol)), ctx)


def set_graphs(ctx, enable):
    _check(lib().sgp_set_graphs(ctx, int(bool(enable))), ctx)


def set_state(ctx, src, dtype, t0=0.0):
    ptr, dev, _keep = _ptr(src, dtype)
    _check(lib().sgp_set_state(ctx, ctypes.c_void_p(ptr), dev, float(t0)), ctx)


def get_state(ctx, dst, dtype):
    ptr, dev, _keep = _ptr(dst, dtype)
    _check(lib().sgp_get_state(ctx, ctypes.c_void_p(ptr), dev), ctx)
    return dst


def get_state_lab(ctx, dst, dtype):
    ptr, dev, _keep = _ptr(dst, dtype)
    _check(lib().sgp_get_state_lab(ctx, ctypes.c_void_p(ptr), dev), ctx)
    return dst


def get_time(ctx):
    t = ctypes.c_double()
    _check(lib().sgp_get_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def step(ctx, nsteps, dt, scheme="ts2"):
    s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
    _check(lib().sgp_step(ctx, int(nsteps), float(dt), s), ctx)


def substep_plan(scheme, nsteps, dt):
    """sgp_substep_plan: [(kind, delta, time offset), ...] of a run (host only)."""
    s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
    n = ctypes.c_longlong()
    _check(lib().sgp_substep_plan(s, int(nsteps), float(dt), 0, None, None, None, ctypes.byref(n)))
    cap = n.value
    kinds = ctypes.create_string_buffer(max(cap, 1))
    deltas = (ctypes.c_double * max(cap, 1))()
    toffs = (ctypes.c_double * max(cap, 1))()
    _check(lib().sgp_substep_plan(s, int(nsteps), float(dt), cap, kinds, deltas, toffs,
                                  ctypes.byref(n)))
    return [(kinds.raw[k:k + 1].decode(), deltas[k], toffs[k]) for k in range(n.value)]


def step_host(ctx, src, t0, dst, nsteps, dt, scheme, chunks, dtype):
    """sgp_step_host: host buffers in and out, copies overlapped with the steps."""
    pi, di, _ki = _ptr(src, dtype)
    po, do, _ko = _ptr(dst, dtype)
    if di or do:
        raise ValueError("sgp_step_host takes host buffers")
    s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
    _check(lib().sgp_step_host(ctx, ctypes.c_void_p(pi), float(t0), ctypes.c_void_p(po),
                               int(nsteps), float(dt), s, int(chunks)), ctx)
    return dst


SGP_TUNE_FORCE = 1
N_VARIANTS = 7


def variant_exists(prec, n, variant):
    return bool(lib().sgp_variant_exists(PRECS[prec] if isinstance(prec, str) else prec,
                                         int(n), int(variant)))


def set_plan(ctx, variants):
    """Kernel variant per axis (x-pass, y lines, z lines)."""
    v = list(variants) + [0] * (3 - len(variants))
    _check(lib().sgp_set_plan(ctx, (ctypes.c_int * 3)(*v)), ctx)


def get_plan(ctx):
    v = (ctypes.c_int * 3)()
    _check(lib().sgp_get_plan(ctx, v), ctx)
    return list(v)


def autotune(ctx, reps=20, force=False, timings=False):
    """sgp_autotune; returns the plan, and with timings=True also the
    [axis][variant] ms per launch (None where absent)."""
    ms = (ctypes.c_double * (3 * N_VARIANTS))() if timings else None
    _check(lib().sgp_autotune(ctx, int(reps), SGP_TUNE_FORCE if force else 0, ms), ctx)
    plan = get_plan(ctx)
    if not timings:
        return plan
    tab = [[(ms[a * N_VARIANTS + v] if ms[a * N_VARIANTS + v] >= 0 else None)
            for v in range(N_VARIANTS)] for a in range(3)]
    return plan, tab


def record(ctx, nsteps, dt, scheme="ts2", interval=0):
    """sgp_record: step with checkpoints every `interval` steps (0: sqrt)."""
    s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
    _check(lib().sgp_record(ctx, int(nsteps), float(dt), s, int(interval)), ctx)


def backward(ctx, g_T, g_0, dtype, batch=1):
    """sgp_backward: g_0 <- VJP of the recorded run applied to g_T; returns
    dJ/d(Omega, gamma, c0, c1, c2) per member as a (batch, 5) float64 array."""
    pi, di, _k1 = _ptr(g_T, dtype)
    po, do, _k2 = _ptr(g_0, dtype)
    dp = (ctypes.c_double * (5 * batch))()
    _check(lib().sgp_backward(ctx, ctypes.c_void_p(pi), di, ctypes.c_void_p(po), do, dp), ctx)
    return np.array(dp[:], dtype=np.float64).reshape(batch, 5)


def substep(ctx, kind, delta):
    k = {"nonlinear": SGP_SUB_NONLINEAR, "linear": SGP_SUB_LINEAR}.get(kind, kind)
    _check(lib().sgp_substep(ctx, k, float(delta)), ctx)


def observables(ctx, batch=1):
    arr = (Obs * batch)()
    _check(lib().sgp_observables(ctx, arr), ctx)
    return [o.as_dict() for o in arr]


def observables_static(n, L, field_dev_ptr, batch=1, prec="f32", t=0.0, device=0,
                       stream=None, **params):
    """sgp_observables_static: observables of a device field the caller holds
    (pointer as an int), computed without any allocation by the library."""
    dim = len(n)
    if np.isscalar(L):
        L = [float(L)] * dim
    m = max(3, dim)
    na = (ctypes.c_int * m)(*(list(n) + [1] * (m - dim)))
    La = (ctypes.c_double * m)(*(list(L) + [1.0] * (m - len(L))))
    p = Params(**{k: float(params.get(k, 1.0 if k in ("gx", "gy", "gz") else 0.0))
                  for k, _ in Params._fields_})
    arr = (Obs * batch)()
    st = lib().sgp_observables_static(dim, na, La, int(batch), PRECS[prec] if isinstance(prec, str) else prec,
                                      ctypes.byref(p), float(t), ctypes.c_void_p(int(field_dev_ptr)),
                                      int(device), ctypes.c_void_p(stream or 0), arr)
    _check(st, None)
    return [o.as_dict() for o in arr]


def synchronize(ctx):
    _check(lib().sgp_synchronize(ctx), ctx)


def launch_count(ctx):
    return int(lib().sgp_launch_count(ctx))


PROFILE_KINDS = ("xpass", "linepass_y", "linepass_z", "tables", "observables", "other")


def set_profiling(ctx, enable):
    _check(lib().sgp_set_profiling(ctx, int(bool(enable))), ctx)


def get_profile(ctx):
    """{kind: (launches, device ms)} since profiling was enabled."""
    n = (ctypes.c_longlong * 6)()
    ms = (ctypes.c_double * 6)()
    _check(lib().sgp_get_profile(ctx, n, ms), ctx)
    return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(PROFILE_KINDS)}


def destroy(ctx):
    if ctx:
        _check(lib().sgp_destroy(ctx), None)


# ---------------------------------------------------------------------------
# convenience object
# ---------------------------------------------------------------------------
class Context:
    """One sgp context: grid, precision, batch, device and stream."""

    def __init__(self, n, L, batch=1, prec="f32", device=0, stream=None):
        self.n = tuple(int(v) for v in n)
        self.L = (float(L),) * len(n) if np.isscalar(L) else tuple(float(v) for v in L)
        self.batch = int(batch)
        self.prec = prec
        self.dtype = np.complex64 if prec == "f32" else np.complex128
        self.handle = create_grid(self.n, self.L, batch, prec, device, stream)

    @property
    def shape(self):
        return (self.batch, 5) + self.n[::-1]

    def set_params(self, **kw):
        set_params(self.handle, **kw)

    def set_params_batch(self, plist):
        set_params_batch(self.handle, plist)

    def set_graphs(self, enable):
        set_graphs(self.handle, enable)

    def set_health_check(self, every, drift_tol):
        set_health_check(self.handle, every, drift_tol)

    def set_state(self, src, t0=0.0):
        set_state(self.handle, src, self.dtype, t0)

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        get_state(self.handle, out, self.dtype)
        return out

    def get_state_lab(self, out=None):
        """Lab-frame field at the current time (sgp_get_state_lab)."""
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        get_state_lab(self.handle, out, self.dtype)
        return out

    @property
    def t(self):
        return get_time(self.handle)

    def step(self, nsteps, dt, scheme="ts2"):
        step(self.handle, nsteps, dt, scheme)

    def step_host(self, src, t0, nsteps, dt, scheme="ts2", chunks=1, out=None):
        """State from host memory, nsteps steps, state back to host memory
        (sgp_step_host); `out` defaults to a new array."""
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        return step_host(self.handle, src, t0, out, nsteps, dt, scheme, chunks, self.dtype)

    def substep(self, kind, delta):
        substep(self.handle, kind, delta)

    def set_plan(self, variants):
        set_plan(self.handle, variants)

    def get_plan(self):
        return get_plan(self.handle)

    def autotune(self, reps=20, force=False, timings=False):
        return autotune(self.handle, reps, force, timings)

    def record(self, nsteps, dt, scheme="ts2", interval=0):
        record(self.handle, nsteps, dt, scheme, interval)

    def backward(self, g_T, out=None):
        """(g_0, dparams) for the recorded run; g_T and out as in set_state /
        get_state (numpy or torch, host or CUDA)."""
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        dp = backward(self.handle, g_T, out, self.dtype, self.batch)
        return out, dp

    def observables(self):
        return observables(self.handle, self.batch)

    def synchronize(self):
        synchronize(self.handle)

    def launch_count(self):
        return launch_count(self.handle)

    def set_profiling(self, enable):
        set_profiling(self.handle, enable)

    def get_profile(self):
        return get_profile(self.handle)

    def close(self):
        if self.handle:
            destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------
# ensembles of runs on different grids
# ---------------------------------------------------------------------------
def _echeck(status, ens):
    if status != 0:
        L = lib()
        raise SgpError(L.sgp_status_string(status).decode(), L.sgp_ensemble_last_error(ens).decode())


class Ensemble:
    """sgp_ensemble_*: members on different grids, advanced together."""

    def __init__(self, grids, prec="f32", device=0, stream=None):
        """grids: list of (n, L) with n and L in (x, y[, z]) order."""
        dim = len(grids[0][0])
        self.count = len(grids)
        self.dim = dim
        self.prec = prec
        self.dtype = np.complex64 if prec == "f32" else np.complex128
        self.grids = []
        na, La = [], []
        for n, L in grids:
            n = tuple(int(v) for v in n)
            L = (float(L),) * dim if np.isscalar(L) else tuple(float(v) for v in L)
            self.grids.append((n, L))
            na += list(n)
            La += list(L)
        out = ctypes.c_void_p()
        st = lib().sgp_ensemble_create(dim, self.count, (ctypes.c_int * len(na))(*na),
                                       (ctypes.c_double * len(La))(*La), PRECS[prec],
                                       int(device), ctypes.c_void_p(stream or 0), ctypes.byref(out))
        _echeck(st, None)
        self.handle = out

    @property
    def groups(self):
        return lib().sgp_ensemble_groups(self.handle)

    def set_params(self, plist):
        arr = (Params * self.count)(*[_params(d) for d in plist])
        _echeck(lib().sgp_ensemble_set_params(self.handle, arr), self.handle)

    def set_member_state(self, m, src, t0=0.0):
        ptr, dev, _keep = _ptr(src, self.dtype)
        _echeck(lib().sgp_ensemble_set_member_state(self.handle, int(m), ctypes.c_void_p(ptr), dev,
                                                    float(t0)), self.handle)

    def get_member_state(self, m, out=None):
        n, _ = self.grids[m]
        if out is None:
            out = np.empty((5,) + n[::-1], dtype=self.dtype)
        ptr, dev, _keep = _ptr(out, self.dtype)
        _echeck(lib().sgp_ensemble_get_member_state(self.handle, int(m), ctypes.c_void_p(ptr), dev),
                self.handle)
        return out

    def step(self, nsteps, dt, scheme="ts2"):
        s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        _echeck(lib().sgp_ensemble_step(self.handle, int(nsteps), float(dt), s), self.handle)

    def step_host(self, srcs, t0, nsteps, dt, scheme="ts2", outs=None):
        """Every member's state from host buffers srcs[m], nsteps steps, the
        states to host buffers outs[m] (new arrays by default) in one call
        (sgp_ensemble_step_host)."""
        if len(srcs) != len(self.grids):
            raise ValueError("one source buffer per member")
        if outs is None:
            outs = [np.empty((5,) + n[::-1], dtype=self.dtype) for n, _ in self.grids]
        keep = []
        pin = (ctypes.c_void_p * len(srcs))()
        pout = (ctypes.c_void_p * len(srcs))()
        for m, (a, b) in enumerate(zip(srcs, outs)):
            pa, da, ka = _ptr(a, self.dtype)
            pb, db, kb = _ptr(b, self.dtype)
            if da or db:
                raise ValueError("sgp_ensemble_step_host takes host buffers")
            pin[m], pout[m] = pa, pb
            keep += [ka, kb]
        s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        _echeck(lib().sgp_ensemble_step_host(self.handle, pin, float(t0), pout, int(nsteps),
                                             float(dt), s), self.handle)
        return outs

    def autotune(self, reps=20, force=False):
        _echeck(lib().sgp_ensemble_autotune(self.handle, int(reps), SGP_TUNE_FORCE if force else 0),
                self.handle)

    def set_persistent(self, enable):
        """sgp_ensemble_set_persistent: run the steps in the persistent
        work-queue kernel (default when the ensemble qualifies) or not."""
        _echeck(lib().sgp_ensemble_set_persistent(self.handle, int(bool(enable))), self.handle)

    @property
    def persistent(self):
        return bool(lib().sgp_ensemble_persistent(self.handle))

    def set_wait_limit(self, seconds):
        _echeck(lib().sgp_ensemble_set_wait_limit(self.handle, float(seconds)), self.handle)

    def inject_stall(self, member):
        """Test hook: the next step's first work item of `member` does not
        signal its completion (sgp_ensemble_inject_stall)."""
        _echeck(lib().sgp_ensemble_inject_stall(self.handle, int(member)), self.handle)

    def observables(self):
        arr = (Obs * self.count)()
        _echeck(lib().sgp_ensemble_observables(self.handle, arr), self.handle)
        return [o.as_dict() for o in arr]

    def synchronize(self):
        _echeck(lib().sgp_ensemble_synchronize(self.handle), self.handle)

    def launch_count(self):
        return int(lib().sgp_ensemble_launch_count(self.handle))

    def close(self):
        if self.handle:
            lib().sgp_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
