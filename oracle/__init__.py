"""FP64 CPU oracle for the SPSTD method (arXiv 1805.03155) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The product library in
``paper_1805_03155_gb300/`` never does: it shares no code with the oracle.

The numerics live in ``spstd_oracle.c`` (plain C, single threaded, FP64); this
module compiles it with gcc on first use and marshals numpy arrays to it.
Nothing here computes any step of the method itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spstd_oracle.c")
_HDR = os.path.join(_HERE, "spstd_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LEAPFROG, STRANG, PAPER3, FR4, SUZUKI6 = 0, 1, 2, 3, 4
PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2
PRESETS = {"LEAPFROG": LEAPFROG, "STRANG": STRANG, "PAPER3": PAPER3, "FR4": FR4, "SUZUKI6": SUZUKI6}


class Grid(C.Structure):
    _fields_ = [
        ("dims", C.c_int),
        ("n", C.c_int64 * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("hbar", C.c_double),
        ("mass", C.c_double),
        ("nyquist_zero", C.c_int),
        ("bc", C.c_int * 3),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so from spstd_oracle.c (gcc -O2, no -march flags)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR)
    )
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int64)
            gp = C.POINTER(Grid)
            L.orc_preset.argtypes = [C.c_int, dp, dp, C.POINTER(C.c_int)]
            L.orc_fft.argtypes = [dp, dp, C.c_int64, C.c_int]
            L.orc_laplacian_axis.argtypes = [dp, dp, gp, C.c_int]
            L.orc_apply_K.argtypes = [dp, dp, dp, gp]
            L.orc_run.argtypes = [dp, dp, dp, gp, dp, dp, C.c_int, C.c_double, C.c_int64,
                                  C.c_int, ip, dp, dp]
            L.orc_trace.argtypes = [dp, dp, C.c_int, C.c_double]
            L.orc_trace.restype = C.c_double
            L.orc_evolution_matrix.argtypes = [dp, dp, C.c_int, C.c_double, dp]
            L.orc_evolution_matrix.restype = None
            L.orc_stability_limit.argtypes = [dp, dp, C.c_int]
            L.orc_stability_limit.restype = C.c_double
            L.orc_spectrum.argtypes = [dp, dp, C.c_int64, C.c_int64, C.c_int, C.c_double,
                                       C.c_double, C.c_double, dp, dp, dp]
            L.orc_phase_correct.argtypes = [C.c_double, dp, dp, C.c_int]
            L.orc_phase_correct.restype = C.c_double
            L.orc_norm_energy.argtypes = [dp, dp, dp, gp, dp, dp]
            L.orc_run_rk4.argtypes = [dp, dp, dp, gp, C.c_double, C.c_int64, C.c_int, ip, dp, dp]
            L.orc_run_eigen.argtypes = [dp, dp, dp, gp, dp, dp, C.c_int, C.c_double, C.c_int64, C.c_int,
                                        dp, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_grid(dims, n, lo, hi, hbar=1.0, mass=1.0, nyquist_zero=False, bc=(0, 0, 0)) -> Grid:
    g = Grid()
    g.dims = int(dims)
    nn = list(n) + [1] * (3 - len(n))
    ll = list(lo) + [0.0] * (3 - len(lo))
    hh = list(hi) + [1.0] * (3 - len(hi))
    for i in range(3):
        g.n[i] = int(nn[i])
        g.lo[i] = float(ll[i])
        g.hi[i] = float(hh[i])
    g.hbar = float(hbar)
    g.mass = float(mass)
    g.nyquist_zero = int(bool(nyquist_zero))
    bb = list(bc) + [0] * (3 - len(bc))
    for i in range(3):
        g.bc[i] = int(bb[i])
    return g


def preset(name):
    c = np.zeros(8)
    d = np.zeros(8)
    m = C.c_int(0)
    if lib().orc_preset(PRESETS[name] if isinstance(name, str) else int(name), _dp(c), _dp(d), C.byref(m)):
        raise ValueError(f"unknown preset {name}")
    return c[: m.value].copy(), d[: m.value].copy()


def fft(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    re = _f64(x.real).copy()
    im = _f64(x.imag).copy()
    if lib().orc_fft(_dp(re), _dp(im), len(re), int(sign)):
        raise ValueError("orc_fft failed")
    return re + 1j * im


def laplacian_axis(f, g: Grid, axis):
    f = _f64(f)
    out = np.empty_like(f)
    if lib().orc_laplacian_axis(_dp(f), _dp(out), C.byref(g), int(axis)):
        raise ValueError("orc_laplacian_axis failed")
    return out


def apply_K(src, V, g: Grid):
    src = _f64(src)
    V = _f64(V) if V is not None else np.zeros_like(src)
    out = np.empty_like(src)
    if lib().orc_apply_K(_dp(src), _dp(V), _dp(out), C.byref(g)):
        raise ValueError("orc_apply_K failed")
    return out


def run(psiR, psiI, V, g: Grid, c, d, dt, nsteps, probe_idx=()):
    """Advance copies of (psiR, psiI) by nsteps; returns (psiR, psiI, probes)
    with probes complex of shape [n_probe, nsteps]."""
    pr = _f64(psiR).copy()
    pi = _f64(psiI).copy()
    V = _f64(V) if V is not None else np.zeros_like(pr)
    c = _f64(c)
    d = _f64(d)
    assert len(c) == len(d)
    idx = np.ascontiguousarray(probe_idx, dtype=np.int64)
    npb = len(idx)
    bre = np.zeros(max(npb * int(nsteps), 1))
    bim = np.zeros(max(npb * int(nsteps), 1))
    rc = lib().orc_run(_dp(pr), _dp(pi), _dp(V), C.byref(g), _dp(c), _dp(d), len(c), float(dt),
                       int(nsteps), npb, idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(bre), _dp(bim))
    if rc:
        raise ValueError("orc_run failed")
    probes = (bre[: npb * nsteps] + 1j * bim[: npb * nsteps]).reshape(npb, int(nsteps))
    return pr, pi, probes


def trace(c, d, s):
    c = _f64(c)
    d = _f64(d)
    return lib().orc_trace(_dp(c), _dp(d), len(c), float(s))


def evolution_matrix(c, d, s):
    c = _f64(c)
    d = _f64(d)
    M = np.zeros(4)
    lib().orc_evolution_matrix(_dp(c), _dp(d), len(c), float(s), _dp(M))
    return M.reshape(2, 2)


def stability_limit(c, d):
    c = _f64(c)
    d = _f64(d)
    return lib().orc_stability_limit(_dp(c), _dp(d), len(c))


def spectrum(z, dt, hbar=1.0, nfft=0, max_peaks=32, thresh=1e-3):
    """Peaks of the windowed spectrum of a complex series: (theta, E, amp)."""
    z = np.asarray(z, dtype=np.complex128)
    M = len(z)
    if nfft <= 0:
        nfft = 1
        while nfft < 4 * M:
            nfft *= 2
    re = _f64(z.real).copy()
    im = _f64(z.imag).copy()
    th = np.zeros(max_peaks)
    E = np.zeros(max_peaks)
    A = np.zeros(max_peaks)
    n = lib().orc_spectrum(_dp(re), _dp(im), M, int(nfft), int(max_peaks), float(thresh),
                           float(dt), float(hbar), _dp(th), _dp(E), _dp(A))
    if n < 0:
        raise ValueError("orc_spectrum failed")
    return th[:n].copy(), E[:n].copy(), A[:n].copy()


def phase_correct(theta, c, d):
    c = _f64(c)
    d = _f64(d)
    return lib().orc_phase_correct(float(theta), _dp(c), _dp(d), len(c))


def norm_energy(psiR, psiI, V, g: Grid):
    pr = _f64(psiR)
    pi = _f64(psiI)
    V = _f64(V) if V is not None else np.zeros_like(pr)
    nv = C.c_double(0)
    ev = C.c_double(0)
    if lib().orc_norm_energy(_dp(pr), _dp(pi), _dp(V), C.byref(g), C.byref(nv), C.byref(ev)):
        raise ValueError("orc_norm_energy failed")
    return nv.value, ev.value


def run_eigen(psiR, psiI, V, g: Grid, c, d, dt, nsteps, E):
    """Advance copies by nsteps and return (psiR, psiI, acc) with acc complex
    [len(E), n_total]: the Hann-windowed Fourier components at energies E."""
    pr = _f64(psiR).copy()
    pi = _f64(psiI).copy()
    V = _f64(V) if V is not None else np.zeros_like(pr)
    c = _f64(c)
    d = _f64(d)
    E = _f64(np.atleast_1d(E))
    n = len(pr)
    ar = np.zeros(len(E) * n)
    ai = np.zeros(len(E) * n)
    if lib().orc_run_eigen(_dp(pr), _dp(pi), _dp(V), C.byref(g), _dp(c), _dp(d), len(c), float(dt), int(nsteps),
                           len(E), _dp(E), _dp(ar), _dp(ai)):
        raise ValueError("orc_run_eigen failed")
    return pr, pi, (ar + 1j * ai).reshape(len(E), n)


def run_rk4(psiR, psiI, V, g: Grid, dt, nsteps, probe_idx=()):
    """Classical RK4 (the non-symplectic comparison of Fig. 3); as run()."""
    pr = _f64(psiR).copy()
    pi = _f64(psiI).copy()
    V = _f64(V) if V is not None else np.zeros_like(pr)
    idx = np.ascontiguousarray(probe_idx, dtype=np.int64)
    npb = len(idx)
    bre = np.zeros(max(npb * int(nsteps), 1))
    bim = np.zeros(max(npb * int(nsteps), 1))
    if lib().orc_run_rk4(_dp(pr), _dp(pi), _dp(V), C.byref(g), float(dt), int(nsteps), npb,
                         idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(bre), _dp(bim)):
        raise ValueError("orc_run_rk4 failed")
    probes = (bre[: npb * nsteps] + 1j * bim[: npb * nsteps]).reshape(npb, int(nsteps))
    return pr, pi, probes
