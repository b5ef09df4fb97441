"""Eigenstate reconstruction on the device (the eigenstates of Figs. 1, 2, 4):
the FP64 accumulators equal the oracle's windowed Fourier components, and the
normalised result is the dense-eigensolver eigenvector."""
import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs
from helpers import gpu_solver, oracle_grid

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,bc", [((64,), (0,)), ((32, 16), (0, 0)), ((8, 16, 8), (0, 0, 0)), ((21,), (1,)),
                                      ((12, 10), (2, 1))], ids=str)
@pytest.mark.parametrize("precision", [64, 32])
def test_accumulators_match_oracle(shape, bc, precision):
    dims = len(shape)
    lo, hi = [-4.0] * dims, [4.0] * dims
    dx = min(8.0 / n for n in shape)
    dt = 0.25 / (0.5 * dims * (np.pi / dx) ** 2 + 0.5 * 16 * dims)
    p = inputs.gaussian_problem(shape, lo, hi, seed=41, dt=dt, steps=30, n_probe=2, bc=bc)
    E = [0.9, 2.3, 5.0]
    s = gpu_solver(p, precision, cap=40, max_eigenstates=3)
    s.spstd_eigenstates_begin(E, 25)
    s.spstd_step(30)  # 25 samples, then the window is closed
    got = np.array([s.spstd_eigenstate_get(k, normalise=False) for k in range(3)])
    s.close()
    c, d = oracle.preset(p.integrator)
    _, _, acc = oracle.run_eigen(p.psiR, p.psiI, p.V, oracle_grid(p), c, d, p.dt, 25, E)
    tol = 1e-10 if precision == 64 else 1e-4
    assert np.max(np.abs(got - acc)) <= tol * np.max(np.abs(acc))


def test_well_eigenstates_on_device():
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
    coef = np.zeros(n)
    coef[:3] = [1.0, 0.7, 0.5]
    coef[3:] = 0.01 * np.random.default_rng(2).standard_normal(n - 3)
    psi0 = U @ coef
    c, d = oracle.preset("FR4")
    dt = 0.4 / (0.5 * (np.pi * n / L) ** 2 + 5.0)
    steps = 4000
    th = [np.arccos(np.trace(oracle.evolution_matrix(c, d, wi * dt)) / 2) / dt for wi in w[:3]]
    p = inputs.Problem("well_eig", 1, (n, 1, 1), (-20.0, 0, 0), (20.0, 1, 1), V, psi0, np.zeros(n), [],
                       "FR4", dt, steps)
    s = gpu_solver(p, 64, cap=1, max_eigenstates=3)
    s.spstd_eigenstates_begin(th, steps)
    s.spstd_step(steps)
    for k in range(3):
        v = s.spstd_eigenstate_get(k)
        assert abs(np.vdot(U[:, k], v)) > 1 - 1e-4, k
    s.close()
