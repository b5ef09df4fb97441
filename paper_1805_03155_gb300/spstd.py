"""Thin ctypes binding of the SPSTD C ABI (include/spstd.h).

Argument marshalling only: every step of the time integration, the
reductions and the spectra run in the CUDA kernels of libspstd.so.  PyTorch
supplies the device workspace (one uint8 tensor) and the CUDA stream.  There is
no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspstd.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
HEADER = os.path.join(INCLUDE, "spstd.h")

SPSTD_OK, SPSTD_EINVAL, SPSTD_ENOMEM, SPSTD_ECUDA, SPSTD_EUNSTABLE = 0, 1, 2, 3, 4
SPSTD_EDIVERGED, SPSTD_ETIMEOUT, SPSTD_ENOTREADY, SPSTD_EUNSUPPORTED = 5, 6, 7, 8
PRESETS = {"CUSTOM": -1, "LEAPFROG": 0, "STRANG": 1, "PAPER3": 2, "FR4": 3, "SUZUKI6": 4, "RK4": 5}
PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2
MAX_STAGES = 8
MAX_PROBES = 16
SCHEDULES = 7


class SpstdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"spstd status {status}: {msg}")
        self.status = status


class spstd_config(C.Structure):
    _fields_ = [
        ("dims", C.c_int),
        ("n", C.c_int64 * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("hbar", C.c_double),
        ("mass", C.c_double),
        ("precision", C.c_int),
        ("preset", C.c_int),
        ("m", C.c_int),
        ("c", C.c_double * MAX_STAGES),
        ("d", C.c_double * MAX_STAGES),
        ("dt", C.c_double),
        ("n_probe", C.c_int),
        ("probe_idx", C.c_int64 * MAX_PROBES),
        ("probe_capacity", C.c_int64),
        ("max_nfft", C.c_int64),
        ("nyquist_zero", C.c_int),
        ("device", C.c_int),
        ("stream", C.c_void_p),
        ("bc", C.c_int * 3),
        ("max_eigenstates", C.c_int),
        ("unmerged_steps", C.c_int),
        ("no_graph", C.c_int),
        ("norm_drift_limit", C.c_double),
        ("v_field_only", C.c_int),
    ]


_lib = None


def declared_functions():
    """Names of the entry points the headers in include/ declare (the API in
    spstd.h, the test hooks in spstd_testing.h)."""
    txt = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spstd_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """Loads libspstd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1805_03155_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
    cfgp = C.POINTER(spstd_config)
    sig = {
        "spstd_config_init": (None, [cfgp]),
        "spstd_workspace_size": (C.c_int, [cfgp, C.POINTER(C.c_size_t)]),
        "spstd_stability_limit": (C.c_int, [cfgp, C.c_double, dp, dp]),
        "spstd_create": (C.c_int, [cfgp, vp, C.c_size_t, C.POINTER(vp)]),
        "spstd_destroy": (C.c_int, [vp]),
        "spstd_set_potential": (C.c_int, [vp, dp]),
        "spstd_set_state": (C.c_int, [vp, dp, dp]),
        "spstd_get_state": (C.c_int, [vp, dp, dp]),
        "spstd_step": (C.c_int, [vp, C.c_int64]),
        "spstd_probe": (C.c_int, [vp, C.c_int, dp, dp, C.c_int64, ip]),
        "spstd_spectrum": (C.c_int, [vp, C.c_int, C.c_int64, C.c_int, C.c_double, C.c_int, dp, dp,
                                     C.POINTER(C.c_int)]),
        "spstd_energy_norm": (C.c_int, [vp, dp, dp]),
        "spstd_check_workspace": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "spstd_apply_hamiltonian": (C.c_int, [vp, C.c_int, dp]),
        "spstd_get_dt": (C.c_int, [vp, dp]),
        "spstd_steps_taken": (C.c_int, [vp, ip]),
        "spstd_potential_separable": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "spstd_separable_split": (C.c_int, [dp, C.c_int64, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                            C.POINTER(C.c_int)]),
        "spstd_get_coefficients": (C.c_int, [vp, C.POINTER(C.c_int), dp, dp]),
        "spstd_launch_count": (C.c_int, [vp, C.c_int64, ip]),
        "spstd_profile_steps": (C.c_int, [vp, C.c_int64, dp, ip]),
        "spstd_norm_noalloc": (C.c_int, [vp, vp, C.c_int64, C.c_int, C.c_double, vp, vp]),
        "spstd_eigenstates_begin": (C.c_int, [vp, C.c_int, dp, C.c_int64]),
        "spstd_eigenstate_get": (C.c_int, [vp, C.c_int, C.c_int, dp, dp, ip]),
        "spstd_eigenstates_end": (C.c_int, [vp]),
        "spstd_batch_workspace_size": (C.c_int, [C.c_int, C.POINTER(C.c_size_t)]),
        "spstd_batch_create": (C.c_int, [C.c_int, C.c_size_t, C.c_int, vp, vp, C.c_size_t, C.POINTER(vp)]),
        "spstd_batch_footprint": (C.c_int, [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
        "spstd_batch_destroy": (C.c_int, [vp]),
        "spstd_batch_add": (C.c_int, [vp, vp, C.POINTER(C.c_int)]),
        "spstd_batch_remove": (C.c_int, [vp, C.c_int]),
        "spstd_batch_size": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "spstd_batch_step": (C.c_int, [vp, C.c_int64]),
        "spstd_batch_sync": (C.c_int, [vp]),
        "spstd_batch_launch_count": (C.c_int, [vp, C.c_int64, ip]),
        "spstd_batch_last_error": (C.c_char_p, [vp]),
        "spstd_schedule_candidates": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "spstd_get_schedule": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int)]),
        "spstd_set_schedule": (C.c_int, [vp, C.c_int, C.c_int]),
        "spstd_tune": (C.c_int, [vp, C.c_int, dp]),
        "spstd_set_xy_fusion": (C.c_int, [vp, C.c_int]),
        "spstd_get_xy_fusion": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "spstd_inject_wait_timeout": (C.c_int, [vp]),
        "spstd_batch_tune": (C.c_int, [vp, C.c_int]),
        "spstd_batch_get_schedule": (C.c_int, [vp, C.c_int, C.c_int, ip, C.POINTER(C.c_int)]),
        "spstd_batch_set_schedule": (C.c_int, [vp, C.c_int, C.c_int, ip, C.POINTER(C.c_int)]),
        "spstd_last_error": (C.c_char_p, [vp]),
        "spstd_status_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(dims, n, lo, hi, precision=64, integrator="FR4", dt=0.0, probes=(), probe_capacity=1024,
                max_nfft=0, hbar=1.0, mass=1.0, nyquist_zero=False, c=None, d=None, device=0, stream=None,
                bc=(0, 0, 0), merge=True, max_eigenstates=0, no_graph=False, norm_drift_limit=1e-3,
                v_field_only=False):
    cfg = spstd_config()
    lib().spstd_config_init(C.byref(cfg))
    cfg.dims = int(dims)
    nn = list(n) + [1] * (3 - len(n))
    ll = list(lo) + [0.0] * (3 - len(lo))
    hh = list(hi) + [1.0] * (3 - len(hi))
    for a in range(3):
        cfg.n[a] = int(nn[a])
        cfg.lo[a] = float(ll[a])
        cfg.hi[a] = float(hh[a])
    cfg.hbar = float(hbar)
    cfg.mass = float(mass)
    cfg.precision = int(precision)
    if c is not None:
        cfg.preset = PRESETS["CUSTOM"]
        cfg.m = len(c)
        for i, (ci, di) in enumerate(zip(c, d)):
            cfg.c[i] = float(ci)
            cfg.d[i] = float(di)
    else:
        cfg.preset = PRESETS[integrator]
    cfg.dt = float(dt)
    cfg.n_probe = len(probes)
    for i, p in enumerate(probes):
        cfg.probe_idx[i] = int(p)
    cfg.probe_capacity = int(probe_capacity)
    cfg.max_nfft = int(max_nfft)
    cfg.nyquist_zero = int(bool(nyquist_zero))
    cfg.device = int(device)
    cfg.stream = stream
    bb = list(bc) + [0] * (3 - len(bc))
    for a in range(3):
        cfg.bc[a] = int(bb[a])
    cfg.unmerged_steps = 0 if merge else 1
    cfg.max_eigenstates = int(max_eigenstates)
    cfg.no_graph = int(bool(no_graph))
    cfg.norm_drift_limit = float(norm_drift_limit)
    cfg.v_field_only = int(bool(v_field_only))
    return cfg


class Solver:
    """One SPSTD context on one CUDA device, workspace owned by a torch tensor."""

    def __init__(self, cfg: spstd_config, stream=None):
        import torch

        self.L = lib()
        self.cfg = cfg
        dev = torch.device("cuda", cfg.device)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.torch_stream = stream
        cfg.stream = C.c_void_p(stream.cuda_stream)
        nbytes = C.c_size_t(0)
        self._check(self.L.spstd_workspace_size(C.byref(cfg), C.byref(nbytes)), None)
        self.workspace_bytes = nbytes.value
        self._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.workspace_offset = aligned - base  # where the library's workspace starts in self._ws
        self.ctx = C.c_void_p(0)
        self._check(self.L.spstd_create(C.byref(cfg), C.c_void_p(aligned), nbytes.value, C.byref(self.ctx)), None)
        self.n_total = int(cfg.n[0] * cfg.n[1] * cfg.n[2])

    def _check(self, st, ctx=None):
        if st != SPSTD_OK:
            msg = self.L.spstd_status_string(st).decode()
            c = ctx if ctx is not None else getattr(self, "ctx", None)
            if c is not None and c.value:
                msg += ": " + self.L.spstd_last_error(c).decode()
            raise SpstdError(st, msg)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.L.spstd_destroy(self.ctx)
            self.ctx = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C ABI calls, same names ------------------------------------------------
    def spstd_set_potential(self, V):
        V = np.ascontiguousarray(V, dtype=np.float64)
        assert V.size == self.n_total
        self._check(self.L.spstd_set_potential(self.ctx, _dp(V)))

    def spstd_set_state(self, psiR, psiI):
        pr = np.ascontiguousarray(psiR, dtype=np.float64)
        pi = np.ascontiguousarray(psiI, dtype=np.float64)
        assert pr.size == self.n_total and pi.size == self.n_total
        self._check(self.L.spstd_set_state(self.ctx, _dp(pr), _dp(pi)))

    def spstd_get_state(self, out_r=None, out_i=None):
        pr = out_r if out_r is not None else np.empty(self.n_total)
        pi = out_i if out_i is not None else np.empty(self.n_total)
        self._check(self.L.spstd_get_state(self.ctx, _dp(pr), _dp(pi)))
        return pr, pi

    def spstd_step(self, nsteps):
        self._check(self.L.spstd_step(self.ctx, int(nsteps)))

    def spstd_probe(self, p, cap=None):
        if cap is None:
            cap = self.cfg.probe_capacity
        re_ = np.empty(max(int(cap), 1))
        im_ = np.empty(max(int(cap), 1))
        n = C.c_int64(0)
        self._check(self.L.spstd_probe(self.ctx, int(p), _dp(re_), _dp(im_), int(cap), C.byref(n)))
        return re_[: n.value] + 1j * im_[: n.value]

    def spstd_spectrum(self, p=-1, nfft=0, max_peaks=32, thresh=1e-3, phase_correct=False):
        E = np.empty(max_peaks)
        A = np.empty(max_peaks)
        n = C.c_int(0)
        self._check(self.L.spstd_spectrum(self.ctx, int(p), int(nfft), int(max_peaks), float(thresh),
                                          int(bool(phase_correct)), _dp(E), _dp(A), C.byref(n)))
        return E[: n.value].copy(), A[: n.value].copy()

    def spstd_energy_norm(self):
        """(norm, energy).  On SPSTD_EDIVERGED the SpstdError carries both
        values as .norm and .energy (the C call writes them before it returns)."""
        nv = C.c_double(0)
        ev = C.c_double(0)
        st = self.L.spstd_energy_norm(self.ctx, C.byref(nv), C.byref(ev))
        try:
            self._check(st)
        except SpstdError as e:
            e.norm, e.energy = nv.value, ev.value
            raise
        return nv.value, ev.value

    def spstd_check_workspace(self):
        """True while every guard word of the workspace is intact."""
        v = C.c_int(0)
        self._check(self.L.spstd_check_workspace(self.ctx, C.byref(v)))
        return bool(v.value)

    def spstd_apply_hamiltonian(self, which):
        out = np.empty(self.n_total)
        self._check(self.L.spstd_apply_hamiltonian(self.ctx, int(which), _dp(out)))
        return out

    def spstd_get_dt(self):
        v = C.c_double(0)
        self._check(self.L.spstd_get_dt(self.ctx, C.byref(v)))
        return v.value

    def spstd_potential_separable(self):
        v = C.c_int(0)
        self._check(self.L.spstd_potential_separable(self.ctx, C.byref(v)))
        return bool(v.value)

    def spstd_steps_taken(self):
        v = C.c_int64(0)
        self._check(self.L.spstd_steps_taken(self.ctx, C.byref(v)))
        return v.value

    def spstd_get_coefficients(self):
        m = C.c_int(0)
        c = np.zeros(MAX_STAGES)
        d = np.zeros(MAX_STAGES)
        self._check(self.L.spstd_get_coefficients(self.ctx, C.byref(m), _dp(c), _dp(d)))
        return c[: m.value].copy(), d[: m.value].copy()

    def spstd_eigenstates_begin(self, E, window):
        E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
        self._check(self.L.spstd_eigenstates_begin(self.ctx, len(E), _dp(E), int(window)))

    def spstd_eigenstate_get(self, k, normalise=True):
        """Accumulator k as a complex array (normalised in the library when
        normalise: sum |phi|^2 = 1, largest entry real positive)."""
        re_ = np.empty(self.n_total)
        im_ = np.empty(self.n_total)
        n = C.c_int64(0)
        self._check(self.L.spstd_eigenstate_get(self.ctx, int(k), int(bool(normalise)), _dp(re_), _dp(im_),
                                                C.byref(n)))
        return re_ + 1j * im_

    def spstd_eigenstates_end(self):
        self._check(self.L.spstd_eigenstates_end(self.ctx))

    KERNEL_KINDS = ("x_pass", "y_pass", "z_pass", "probe", "resident_1d", "xy_pass")

    def spstd_profile_steps(self, nsteps):
        """Per kernel kind: (total device ms, launches) over nsteps real steps."""
        ms = np.zeros(len(self.KERNEL_KINDS))
        cnt = np.zeros(len(self.KERNEL_KINDS), dtype=np.int64)
        self._check(self.L.spstd_profile_steps(self.ctx, int(nsteps), _dp(ms),
                                               cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNEL_KINDS)}

    def spstd_launch_count(self, nsteps):
        v = C.c_int64(0)
        self._check(self.L.spstd_launch_count(self.ctx, int(nsteps), C.byref(v)))
        return v.value

    def spstd_schedule_candidates(self, axis):
        lst = (C.c_int * SCHEDULES)()
        n = C.c_int(0)
        self._check(self.L.spstd_schedule_candidates(self.ctx, int(axis), lst, C.byref(n)))
        return [lst[i] for i in range(n.value)]

    def spstd_get_schedule(self, axis):
        v = C.c_int(0)
        self._check(self.L.spstd_get_schedule(self.ctx, int(axis), C.byref(v)))
        return v.value

    def spstd_set_schedule(self, axis, schedule):
        self._check(self.L.spstd_set_schedule(self.ctx, int(axis), int(schedule)))

    def spstd_set_xy_fusion(self, on):
        self._check(self.L.spstd_set_xy_fusion(self.ctx, int(bool(on))))

    def spstd_inject_wait_timeout(self):
        self._check(self.L.spstd_inject_wait_timeout(self.ctx))

    def spstd_get_xy_fusion(self):
        v = C.c_int(0)
        self._check(self.L.spstd_get_xy_fusion(self.ctx, C.byref(v)))
        return bool(v.value)

    def spstd_tune(self, reps=20):
        """Times every candidate schedule per axis and keeps the fastest;
        returns ms[axis][schedule] (-1 where not a candidate)."""
        ms = np.zeros(3 * SCHEDULES)
        self._check(self.L.spstd_tune(self.ctx, int(reps), _dp(ms)))
        return ms.reshape(3, SCHEDULES)


def stability_limit(cfg: spstd_config, vmax=0.0):
    s = C.c_double(0)
    dtm = C.c_double(0)
    st = lib().spstd_stability_limit(C.byref(cfg), float(vmax), C.byref(s), C.byref(dtm))
    if st != SPSTD_OK:
        raise SpstdError(st, lib().spstd_status_string(st).decode())
    return s.value, dtm.value


def separable_split(V, nx):
    """(separable, vx, vyz): the host-side split of V (nx points along x,
    x fastest) that spstd_set_potential tries; see spstd_separable_split."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    rows = V.size // nx
    assert rows * nx == V.size
    vx = np.empty(nx, dtype=np.float32)
    vyz = np.empty(rows, dtype=np.float32)
    ok = C.c_int(0)
    st = lib().spstd_separable_split(_dp(V), int(nx), int(rows), vx.ctypes.data_as(C.POINTER(C.c_float)),
                                     vyz.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ok))
    if st != SPSTD_OK:
        raise SpstdError(st, lib().spstd_status_string(st).decode())
    return bool(ok.value), vx, vyz


class Batch:
    """Many independent solves advanced by one call (spstd_batch_*); the
    descriptor workspace is a torch uint8 tensor."""

    def __init__(self, max_members, device=0, stream=None, hbm_cap_bytes=0):
        import torch

        self.L = lib()
        dev = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.torch_stream = stream
        nbytes = C.c_size_t(0)
        self._check(self.L.spstd_batch_workspace_size(int(max_members), C.byref(nbytes)))
        self._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        aligned = (self._ws.data_ptr() + 255) // 256 * 256
        self.b = C.c_void_p(0)
        self._check(self.L.spstd_batch_create(int(max_members), int(hbm_cap_bytes), int(device),
                                              C.c_void_p(stream.cuda_stream), C.c_void_p(aligned), nbytes.value,
                                              C.byref(self.b)))
        self.members = {}

    def _check(self, st):
        if st != SPSTD_OK:
            msg = self.L.spstd_status_string(st).decode()
            if getattr(self, "b", None) is not None and self.b.value:
                msg += ": " + self.L.spstd_batch_last_error(self.b).decode()
            raise SpstdError(st, msg)

    def spstd_batch_add(self, solver):
        slot = C.c_int(-1)
        self._check(self.L.spstd_batch_add(self.b, solver.ctx, C.byref(slot)))
        self.members[slot.value] = solver
        return slot.value

    def spstd_batch_remove(self, slot):
        self._check(self.L.spstd_batch_remove(self.b, int(slot)))
        return self.members.pop(slot)

    def spstd_batch_footprint(self):
        """(bytes of member workspaces admitted, cap); cap 0 = none."""
        used = C.c_size_t(0)
        cap = C.c_size_t(0)
        self._check(self.L.spstd_batch_footprint(self.b, C.byref(used), C.byref(cap)))
        return int(used.value), int(cap.value)

    def spstd_batch_size(self):
        n = C.c_int(0)
        self._check(self.L.spstd_batch_size(self.b, C.byref(n)))
        return n.value

    def spstd_batch_step(self, nsteps):
        self._check(self.L.spstd_batch_step(self.b, int(nsteps)))

    def spstd_batch_sync(self):
        self._check(self.L.spstd_batch_sync(self.b))

    def spstd_batch_launch_count(self, nsteps):
        v = C.c_int64(0)
        self._check(self.L.spstd_batch_launch_count(self.b, int(nsteps), C.byref(v)))
        return v.value

    def spstd_batch_tune(self, reps=10):
        self._check(self.L.spstd_batch_tune(self.b, int(reps)))

    def spstd_batch_get_schedule(self, precision, dims, n):
        nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
        out = (C.c_int * 3)()
        self._check(self.L.spstd_batch_get_schedule(self.b, int(precision), int(dims), nn, out))
        return [out[i] for i in range(3)]

    def spstd_batch_set_schedule(self, precision, dims, n, schedule):
        nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
        sv = (C.c_int * 3)(*(list(schedule) + [0] * (3 - len(schedule))))
        self._check(self.L.spstd_batch_set_schedule(self.b, int(precision), int(dims), nn, sv))

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            self.L.spstd_batch_destroy(self.b)
            self.b = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_ELEMS = 65536 * 2048


def spstd_norm_noalloc(psiR_ptr, psiI_ptr, n, precision, cell_volume, out_ptr, stream_ptr=0):
    """Norm of two device arrays into a device double, with no device
    allocation (scratch in the library's static device array).  Pointers are
    integers (e.g. torch tensor data_ptr()); returns the status code."""
    return lib().spstd_norm_noalloc(C.c_void_p(psiR_ptr), C.c_void_p(psiI_ptr), int(n), int(precision),
                                    float(cell_volume), C.c_void_p(out_ptr), C.c_void_p(stream_ptr))


def solver_for(problem, precision=64, probe_capacity=None, stream=None, device=0, dt=None, merge=True,
               max_eigenstates=0, no_graph=False, norm_drift_limit=1e-3, v_field_only=False):
    """Creates a Solver for an inputs.Problem and uploads V and the state."""
    cap = probe_capacity if probe_capacity is not None else max(1, problem.steps)
    cfg = make_config(problem.dims, problem.n[: problem.dims], problem.lo[: problem.dims],
                      problem.hi[: problem.dims], precision=precision, integrator=problem.integrator,
                      dt=problem.dt if dt is None else dt, probes=problem.probes, probe_capacity=cap,
                      max_nfft=problem.nfft if problem.nfft else 0, hbar=problem.hbar, mass=problem.mass,
                      device=device, bc=getattr(problem, "bc", (0, 0, 0)), merge=merge,
                      max_eigenstates=max_eigenstates, no_graph=no_graph, norm_drift_limit=norm_drift_limit,
                      v_field_only=v_field_only)
    s = Solver(cfg, stream=stream)
    s.spstd_set_potential(problem.V)
    s.spstd_set_state(problem.psiR, problem.psiI)
    return s
