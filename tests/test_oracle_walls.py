"""Pins of the oracle's wall boundary conditions (Section 2.2: DST for
Dirichlet walls, DCT for Neumann walls) against closed forms and against the
numbers the paper prints for its infinite wells (Tables 2 and 3)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# CODATA constants in nm, fs, eV: hbar [eV fs], electron rest energy [eV], c [nm/fs]
HBAR = 0.6582119569
M_E = 0.51099895e6 / 299.792458 ** 2


def golden(name):
    return np.array([[float(x) for x in l.split()] for l in open(os.path.join(GOLDEN, name))
                     if l.strip() and not l.startswith("#")])


def test_dirichlet_sine_modes():
    """DST: sin(pi n x/L) on the interior points is an eigenvector with k^2 = (pi n/L)^2."""
    n, L = 11, 2.5
    g = oracle.make_grid(1, (n,), (0.0,), (L,), bc=(oracle.DIRICHLET,))
    x = np.arange(1, n + 1) * L / (n + 1)
    for m in range(1, n + 1):
        f = np.sin(np.pi * m * x / L)
        assert np.max(np.abs(oracle.laplacian_axis(f, g, 0) - (np.pi * m / L) ** 2 * f)) < 1e-10 * m * m


def test_neumann_cosine_modes():
    """DCT: cos(pi n x/L) on the points including both walls, k^2 = (pi n/L)^2."""
    n, L = 10, 3.0
    g = oracle.make_grid(1, (n,), (0.0,), (L,), bc=(oracle.NEUMANN,))
    x = np.arange(n) * L / (n - 1)
    for m in range(0, n):
        f = np.cos(np.pi * m * x / L)
        assert np.max(np.abs(oracle.laplacian_axis(f, g, 0) - (np.pi * m / L) ** 2 * f)) < 1e-10 * max(1, m * m)


def test_mixed_walls_3d():
    n = (7, 6, 5)
    lo, hi = (0.0, -1.0, 0.5), (1.0, 2.0, 3.0)
    bc = (oracle.DIRICHLET, oracle.NEUMANN, oracle.PERIODIC)
    g = oracle.make_grid(3, n, lo, hi, bc=bc)
    L = [hi[a] - lo[a] for a in range(3)]
    x = lo[0] + np.arange(1, n[0] + 1) * L[0] / (n[0] + 1)
    y = lo[1] + np.arange(n[1]) * L[1] / (n[1] - 1)
    z = lo[2] + np.arange(n[2]) * L[2] / n[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = (np.sin(np.pi * 2 * (X - lo[0]) / L[0]) * np.cos(np.pi * 3 * (Y - lo[1]) / L[1])
         * np.cos(2 * np.pi * (Z - lo[2]) / L[2])).ravel()
    k2 = (2 * np.pi / L[0]) ** 2 + (3 * np.pi / L[1]) ** 2 + (2 * np.pi / L[2]) ** 2
    K = oracle.apply_K(f, np.zeros_like(f), g)
    assert np.max(np.abs(K - 0.5 * k2 * f)) < 1e-10 * k2


def well_dense_K(n, L, dims=1):
    g = oracle.make_grid(dims, (n,) * dims, (0.0,) * dims, (L,) * dims, hbar=HBAR, mass=M_E,
                         bc=(oracle.DIRICHLET,) * dims)
    N = n ** dims
    K = np.zeros((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        K[:, j] = oracle.apply_K(e, np.zeros(N), g)
    return g, K


def test_infinite_well_levels_are_exact():
    """With the DST the discrete levels of a 9-point well are the continuum
    ones, hbar pi^2 n^2 / (2 m* L^2) in rad/fs (the analytic column of Table 2)."""
    _, K = well_dense_K(9, 1.0)
    w = np.sort(np.linalg.eigvalsh(K))
    exact = HBAR * np.pi ** 2 * np.arange(1, 10) ** 2 / (2 * M_E)
    assert np.max(np.abs(w - exact) / exact) < 1e-12
    tab = golden("table2_1d_infinite_well.txt")
    assert np.allclose(exact[:8], tab[:, 3], atol=5.1e-5)


def scheme_frequency(name, w, dt):
    c, d = oracle.preset(name)
    return np.arccos(np.trace(oracle.evolution_matrix(c, d, w * dt)) / 2) / dt


def test_table2_columns_within_one_bin():
    """Table 2: every numeric entry is an FFT bin 2 pi/(1024 dt).  The scheme's
    discrete frequencies (leapfrog for PSTD, the paper's coefficients for
    SPSTD) on the DST levels land within one bin of every printed value, and a
    delta-source run read off the raw FFT finds its peaks in the same bins."""
    tab = golden("table2_1d_infinite_well.txt")
    dt = M_E * 0.1 ** 2 / (4 * HBAR)
    b = 2 * np.pi / (1024 * dt)
    _, K = well_dense_K(9, 1.0)
    w = np.sort(np.linalg.eigvalsh(K))[:8]
    # SPSTD: every printed bin is the nearest bin to the discrete frequency
    # but one (omega_7 sits at 98.52 bins, printed 98); PSTD: omega_5 and omega_7
    # are printed 0.53 and 1.09 bins below the leapfrog's discrete frequency.
    for col, name, tol in ((1, "LEAPFROG", 1.1), (2, "PAPER3", 0.6)):
        pred = np.array([scheme_frequency(name, wi, dt) for wi in w]) / b
        assert np.max(np.abs(pred - tab[:, col] / b)) <= tol, (name, pred, tab[:, col] / b)
        # the printed values are integer bins
        assert np.max(np.abs(tab[:, col] / b - np.round(tab[:, col] / b))) < 2e-3
    # simulation: delta two cells off the centre, 1024 steps, raw FFT bins
    g, _ = well_dense_K(9, 1.0)
    for col, name in ((1, "LEAPFROG"), (2, "PAPER3")):
        c, d = oracle.preset(name)
        R = np.zeros(9)
        R[6] = 1.0
        _, _, pr = oracle.run(R, np.zeros(9), np.zeros(9), g, c, d, dt, 1024, [6])
        S = np.abs(oracle.fft(pr[0], +1))
        peaks = [k for k in range(1, 511) if S[k] > S[k - 1] and S[k] >= S[k + 1]]
        top = np.sort(sorted(peaks, key=lambda k: -S[k])[:9])[:8]
        assert np.max(np.abs(top - np.round(tab[:, col] / b))) <= 1, (name, top)


def test_table3_spstd_column():
    """Table 3 (2D well): the paper's SPSTD frequencies are within 0.15 bin of
    the scheme's discrete frequencies on the DST levels (n_x, n_y); the analytic
    column is hbar pi^2 (n_x^2 + n_y^2) / (2 m* L^2)."""
    tab = golden("table3_2d_infinite_well.txt")
    dt = M_E * 0.1 ** 2 / (8 * HBAR)
    b = 2 * np.pi / (2048 * dt)
    _, K1 = well_dense_K(9, 1.0)
    lev = np.sort(np.linalg.eigvalsh(K1))
    for nx, ny, spstd, analytic in tab:
        w = lev[int(nx) - 1] + lev[int(ny) - 1]
        assert abs(w - analytic) / analytic < 1e-4
        assert abs(scheme_frequency("PAPER3", w, dt) - spstd) / b < 0.15, (nx, ny)
