"""Seeded synthetic inputs for SPSTD solves (initial states, potentials, probes).

This module serves both the CUDA library's callers and the FP64 oracle, and
holds none of the method's arithmetic: it only samples the potential V(r) and
the initial wave function on the grid of Eq. 5/6 and draws probe points.  All
randomness comes from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) with
53-bit uniforms and Box-Muller normals, so the same seed gives the same input
on every machine.

Workloads (atomic units, hbar = m* = 1; periodic boxes, x fastest):

* ``well_1d``  -- finite quantum well: N = 256 on [-20, 20], V = 0 for |x| < 2
  and V0 = 5 outside; psi_R a Gaussian (centre U(-1, 1), width 0.5) plus 1e-3
  N(0, 1) noise per point, psi_I = 0, normalised; 4 probes with |x| <= 3;
  FR4 integrator, 20000 steps.
* ``ho_3d``    -- isotropic harmonic oscillator: 64^3 on [-8, 8]^3, V =
  omega^2 r^2 / 2 with omega = 1; a Gaussian of width 0.7 displaced by
  U(-0.5, 0.5) per axis; 8 probes with |r_d| <= 2; FR4, 10000 steps.
* ``aniso_ho_3d`` -- anisotropic oscillator at scale: 256^3 on [-12, 12]^3,
  omegas (1.0, 1.3, 1.7); five Gaussians (centres U(-2, 2)^3, widths
  U(0.5, 1.0), amplitudes +-U(0.5, 1)); SUZUKI6, 50000 steps, 8 probes,
  2^16-point probe spectrum.
* ``gaussian_problem`` -- the same recipe on any small grid, for tests.

The time steps are half of the spectral stability limit, dt = 0.5 s*/w_max
with w_max = (hbar/2m*) sum_d (pi/dx_d)^2 + max V / hbar, rounded down to
three significant digits and written out as decimals.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# Half the spectral stability limit, 0.5 s*/w_max, rounded down to three
# significant digits (s* of the named integrator, w_max as in the module doc).
TIME_STEPS = {
    "well_1d_N256": 3.79e-3,     # FR4, w_max = (pi/dx)^2/2 + 5 = 207.13
    "ho_3d_64": 2.36e-3,         # FR4, w_max = 1.5 (pi/0.25)^2 + 96 = 332.87
    "aniso_ho_3d_256": 6.52e-4,  # SUZUKI6, w_max = 1.5 (pi/0.09375)^2 + 401.76
}


class SplitMix64:
    """SplitMix64 stream (counter-based: state_k = seed + k * golden gamma)."""

    GAMMA = np.uint64(0x9E3779B97F4A7C15)

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, count: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, count + 1, dtype=np.uint64)
            z = self.state + k * self.GAMMA
            self.state = np.uint64(self.state + np.uint64(count) * self.GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, count: int) -> np.ndarray:
        m = (count + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:count]

    def integers(self, count: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi)."""
        u = self.uniform(count)
        return (lo + np.floor(u * (hi - lo))).astype(np.int64)


@dataclass
class Problem:
    name: str
    dims: int
    n: Tuple[int, int, int]          # points per axis, x first; unused axes are 1
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    V: np.ndarray                    # float64, flat, x fastest
    psiR: np.ndarray                 # float64, flat
    psiI: np.ndarray                 # float64, flat
    probes: List[int] = field(default_factory=list)
    integrator: str = "FR4"
    dt: float = 1e-3
    steps: int = 100
    nfft: int = 0
    hbar: float = 1.0
    mass: float = 1.0
    bc: Tuple[int, int, int] = (0, 0, 0)   # per axis: 0 periodic, 1 Dirichlet, 2 Neumann

    @property
    def n_total(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def coords(self):
        """Per-axis coordinate vectors (Eq. 5/6): periodic x_j = lo + j L/n,
        Dirichlet x_j = lo + (j+1) L/(n+1), Neumann x_j = lo + j L/(n-1)."""
        return [_axis_coords(self.n[a], self.lo[a], self.hi[a], self.bc[a]) for a in range(3)]


def _axis_coords(n, lo, hi, bc=0):
    L = hi - lo
    if bc == 1:
        return lo + np.arange(1, n + 1) * L / (n + 1)
    if bc == 2:
        return lo + np.arange(n) * L / max(n - 1, 1)
    return lo + np.arange(n) * L / n


def _mesh(n, lo, hi, bc=(0, 0, 0)):
    xs = [_axis_coords(n[a], lo[a], hi[a], bc[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _spacing(n, lo, hi, bc):
    cells = n + 1 if bc == 1 else (n - 1 if bc == 2 else n)
    return (hi - lo) / cells


def _normalise(psiR, psiI, n, lo, hi, dims, bc=(0, 0, 0)):
    cell = 1.0
    for a in range(dims):
        cell *= _spacing(n[a], lo[a], hi[a], bc[a])
    s = np.sqrt(cell * np.sum(psiR * psiR + psiI * psiI))
    return psiR / s, psiI / s


def _central_probes(rng, n, lo, hi, dims, half_width, count):
    """Flat indices of grid points drawn uniformly with |x_d| <= half_width
    (the grid points at +-half_width included)."""
    ranges = []
    for a in range(3):
        if a >= dims:
            ranges.append((0, 1))
            continue
        dx = (hi[a] - lo[a]) / n[a]
        j0 = int(np.ceil((-half_width - lo[a]) / dx))
        j1 = int(np.floor((half_width - lo[a]) / dx))
        j0 = max(j0, 0)
        j1 = min(j1, n[a] - 1)
        ranges.append((j0, j1 + 1))
    idx = []
    for _ in range(count):
        j = [int(rng.integers(1, r0, r1)[0]) for (r0, r1) in ranges]
        idx.append(j[0] + n[0] * (j[1] + n[1] * j[2]))
    return idx


def well_1d(seed: int = 1, N: int = 256, steps: int = 20000, V0: float = 5.0,
            halfwidth: float = 2.0) -> Problem:
    n = (N, 1, 1)
    lo = (-20.0, 0.0, 0.0)
    hi = (20.0, 1.0, 1.0)
    rng = SplitMix64(seed)
    x0 = rng.uniform(1, -1.0, 1.0)[0]
    X, _, _ = _mesh(n, lo, hi)
    V = np.where(np.abs(X) < halfwidth, 0.0, V0)
    psiR = np.exp(-((X - x0) ** 2) / (2 * 0.5 ** 2)) + 1e-3 * rng.normal(N)
    psiI = np.zeros(N)
    psiR, psiI = _normalise(psiR, psiI, n, lo, hi, 1)
    probes = _central_probes(rng, n, lo, hi, 1, 3.0, 4)
    if N != 256 or V0 != 5.0:
        raise ValueError("well_1d: dt is tabulated for N = 256, V0 = 5 only; use gaussian_problem")
    return Problem("well_1d_N256", 1, n, lo, hi, V, psiR, psiI, probes, "FR4",
                   TIME_STEPS["well_1d_N256"], steps, 0)


def ho_3d(seed: int = 2, N: int = 64, steps: int = 10000, sigma: float = 0.7) -> Problem:
    n = (N, N, N)
    lo = (-8.0, -8.0, -8.0)
    hi = (8.0, 8.0, 8.0)
    rng = SplitMix64(seed)
    c = rng.uniform(3, -0.5, 0.5)
    X, Y, Z = _mesh(n, lo, hi)
    V = 0.5 * (X * X + Y * Y + Z * Z)
    psiR = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * sigma ** 2))
    psiI = np.zeros_like(psiR)
    psiR, psiI = _normalise(psiR, psiI, n, lo, hi, 3)
    probes = _central_probes(rng, n, lo, hi, 3, 2.0, 8)
    if N != 64:
        raise ValueError("ho_3d: dt is tabulated for N = 64; use gaussian_problem")
    return Problem("ho_3d_64", 3, n, lo, hi, V, psiR, psiI, probes, "FR4",
                   TIME_STEPS["ho_3d_64"], steps, 0)


def aniso_ho_3d(seed: int = 3, N: int = 256, steps: int = 50000,
                omegas=(1.0, 1.3, 1.7)) -> Problem:
    n = (N, N, N)
    L = 12.0
    lo = (-L, -L, -L)
    hi = (L, L, L)
    rng = SplitMix64(seed)
    X, Y, Z = _mesh(n, lo, hi)
    V = 0.5 * (omegas[0] ** 2 * X * X + omegas[1] ** 2 * Y * Y + omegas[2] ** 2 * Z * Z)
    psiR = np.zeros_like(X)
    for _ in range(5):
        cen = rng.uniform(3, -2.0, 2.0)
        sig = rng.uniform(1, 0.5, 1.0)[0]
        amp = rng.uniform(1, 0.5, 1.0)[0] * (1.0 if rng.uniform(1)[0] < 0.5 else -1.0)
        psiR += amp * np.exp(-((X - cen[0]) ** 2 + (Y - cen[1]) ** 2 + (Z - cen[2]) ** 2)
                             / (2 * sig ** 2))
    psiI = np.zeros_like(psiR)
    psiR, psiI = _normalise(psiR, psiI, n, lo, hi, 3)
    probes = _central_probes(rng, n, lo, hi, 3, 2.0, 8)
    if N != 256:
        raise ValueError("aniso_ho_3d: dt is tabulated for N = 256; use gaussian_problem")
    return Problem("aniso_ho_3d_256", 3, n, lo, hi, V, psiR, psiI, probes, "SUZUKI6",
                   TIME_STEPS["aniso_ho_3d_256"], steps, 1 << 16)


def gaussian_problem(n, lo=None, hi=None, seed: int = 7, omega=None, integrator="FR4",
                     dt=1e-3, steps=10, n_probe=4, noise=0.0, well=None, bc=(0, 0, 0)) -> Problem:
    """A seeded test problem on an arbitrary grid.

    n: points per axis (x first), 1 to 3 entries.  Potential: harmonic with the
    given omegas (default 1 per axis), or a square well (V0, halfwidth) if
    ``well`` is given.  Initial psi_R: a displaced Gaussian of width 0.15 of the
    box plus optional N(0, 1) noise, psi_I a second, smaller displaced Gaussian
    (so both fields start nonzero).  Normalised."""
    dims = len(n)
    nn = tuple(list(n) + [1] * (3 - dims))
    lo = tuple(list(lo if lo is not None else [-4.0] * dims) + [0.0] * (3 - dims))
    hi = tuple(list(hi if hi is not None else [4.0] * dims) + [1.0] * (3 - dims))
    rng = SplitMix64(seed)
    bcc = tuple(list(bc) + [0] * (3 - len(bc)))
    X, Y, Z = _mesh(nn, lo, hi, bcc)
    R = [X, Y, Z]
    if well is not None:
        V0, hw = well
        inside = np.ones_like(X, dtype=bool)
        for a in range(dims):
            inside &= np.abs(R[a]) < hw
        V = np.where(inside, 0.0, V0)
    else:
        om = omega if omega is not None else [1.0] * dims
        V = np.zeros_like(X)
        for a in range(dims):
            V += 0.5 * om[a] ** 2 * R[a] ** 2
    e1 = np.zeros_like(X)
    e2 = np.zeros_like(X)
    for a in range(dims):
        w = 0.15 * (hi[a] - lo[a])
        c1, c2 = rng.uniform(2, -0.1 * w * 4, 0.1 * w * 4)
        mid = 0.5 * (lo[a] + hi[a])
        e1 += (R[a] - mid - c1) ** 2 / (2 * w * w)
        e2 += (R[a] - mid - c2) ** 2 / (2 * (0.7 * w) ** 2)
    psiR = np.exp(-e1)
    psiI = 0.3 * np.exp(-e2)
    if noise:
        psiR = psiR + noise * rng.normal(len(psiR))
    psiR, psiI = _normalise(psiR, psiI, nn, lo, hi, dims, bcc)
    probes = [int(i) for i in rng.integers(n_probe, 0, len(psiR))] if n_probe else []
    return Problem(f"gauss_{'x'.join(map(str, n))}", dims, nn, lo, hi, V, psiR, psiI, probes,
                   integrator, dt, steps, 0, bc=bcc)


def batch_mix(count: int = 512, seed: int = 4, steps: int = 5000, sizes3d=(32, 48, 64, 96)) -> List[Problem]:
    """Seeded mix of uneven solves, one third each of:

    * 1D finite wells: N a uniform power of two in 128..8192 on [-20, 20],
      half-width 2, V0 ~ U(1, 10);
    * 2D isotropic oscillators: n^2 with n uniform in {64, 128, 256, 512} on
      [-8, 8]^2, omega = 1;
    * 3D isotropic oscillators: n^3 with n uniform in ``sizes3d`` on
      [-8, 8]^3, omega = 1 (32^3..96^3 read as the FFT-friendly sizes
      32, 48, 64 and 96).

    Each gets the gaussian_problem start (psi_R and psi_I displaced Gaussians,
    seeded per member), 2 probes, FR4, dt = 0 (half the stability limit, chosen
    by the solver) and `steps` steps; kinds are interleaved."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        kind = i % 3
        sub = seed * 1000003 + i
        if kind == 0:
            N = int(2 ** rng.integers(1, 7, 14)[0])
            V0 = float(rng.uniform(1, 1.0, 10.0)[0])
            p = gaussian_problem((N,), (-20.0,), (20.0,), seed=sub, integrator="FR4", dt=0.0, steps=steps,
                                 n_probe=2, well=(V0, 2.0))
        elif kind == 1:
            n = int(2 ** rng.integers(1, 6, 10)[0])
            p = gaussian_problem((n, n), (-8.0, -8.0), (8.0, 8.0), seed=sub, integrator="FR4", dt=0.0,
                                 steps=steps, n_probe=2)
        else:
            n = int(sizes3d[int(rng.integers(1, 0, len(sizes3d))[0])])
            p = gaussian_problem((n, n, n), (-8.0,) * 3, (8.0,) * 3, seed=sub, integrator="FR4", dt=0.0,
                                 steps=steps, n_probe=2)
        p.name = f"mix{i}_{p.name}"
        out.append(p)
    return out
