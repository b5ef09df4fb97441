"""Pins of the oracle's eigenstate reconstruction (the eigenstates of Figs. 1,
2 and 4 belong to spectral peaks): the windowed Fourier component of the
evolving field at a level's energy is that level's eigenvector of the discrete
Hamiltonian (dense eigensolver)."""
import numpy as np

import oracle
from paper_1805_03155_gb300 import inputs


def test_well_eigenstates_match_dense_eigenvectors():
    n, L = 128, 40.0
    g = oracle.make_grid(1, (n,), (-20.0,), (20.0,))
    x = -20 + np.arange(n) * L / n
    V = np.where(np.abs(x) < 2, 0.0, 5.0)
    K = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        K[:, j] = oracle.apply_K(e, V, g)
    w, U = np.linalg.eigh(K)
    # start from a mix of the three lowest levels plus a little of the rest
    rng = np.random.default_rng(2)
    coef = np.zeros(n)
    coef[:3] = [1.0, 0.7, 0.5]
    coef[3:] = 0.01 * rng.standard_normal(n - 3)
    psi0 = U @ coef
    c, d = oracle.preset("FR4")
    dt = 0.4 / (0.5 * (np.pi * n / L) ** 2 + 5.0)
    steps = 4000
    # the map's own frequencies: theta(w dt)/dt for each level
    th = [np.arccos(np.trace(oracle.evolution_matrix(c, d, wi * dt)) / 2) / dt for wi in w[:3]]
    _, _, acc = oracle.run_eigen(psi0, np.zeros(n), V, g, c, d, dt, steps, th)
    for k in range(3):
        v = acc[k] / np.linalg.norm(acc[k])
        overlap = abs(np.vdot(U[:, k], v))
        assert overlap > 1 - 1e-4, (k, overlap)


def test_eigen_accumulator_definition():
    """One sample: acc = w_0 psi^1 exp(+i E dt/hbar) with w = 1."""
    p = inputs.gaussian_problem((16,), (-3.0,), (3.0,), seed=3, dt=1e-3, steps=1)
    g = oracle.make_grid(1, (16,), (-3.0,), (3.0,), hbar=1.7)
    c, d = oracle.preset("FR4")
    R, I, acc = oracle.run_eigen(p.psiR, p.psiI, p.V, g, c, d, 1e-3, 1, [2.5])
    expect = (R + 1j * I) * np.exp(1j * 2.5 * 1e-3 / 1.7)
    assert np.max(np.abs(acc[0] - expect)) < 1e-15
