"""Pins of the oracle's Runge-Kutta comparison scheme (Fig. 3) and of the
norm behaviour the paper claims: the symplectic scheme holds the normalisation,
RK does not."""
import numpy as np

import oracle
from paper_1805_03155_gb300 import inputs


def test_rk4_per_mode_amplification():
    """V = 0: each Fourier mode z = psi_R + i psi_I with rate w is multiplied per
    step by the RK4 polynomial of -i s, s = w dt: 1 - i s - s^2/2 + i s^3/6 + s^4/24."""
    n, L = 32, 5.0
    g = oracle.make_grid(1, (n,), (0.0,), (L,), hbar=1.1, mass=0.8)
    rng = np.random.default_rng(7)
    pR, pI = rng.standard_normal(n), rng.standard_normal(n)
    dt, steps = 3e-3, 9
    R, I, _ = oracle.run_rk4(pR, pI, np.zeros(n), g, dt, steps)
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    s = 1.1 * k * k / (2 * 0.8) * dt
    amp = (1 - 1j * s - s ** 2 / 2 + 1j * s ** 3 / 6 + s ** 4 / 24) ** steps
    # K acts on psi_R and psi_I separately, so transform each real field
    ZR, ZI = np.fft.fft(pR), np.fft.fft(pI)
    z = ZR + 1j * ZI  # transform of psi_R + i psi_I, mode by mode
    expect = np.fft.ifft(amp * z)
    assert np.max(np.abs(expect.real - R)) < 1e-12 and np.max(np.abs(expect.imag - I)) < 1e-12


def test_rk4_is_fourth_order():
    n = 24
    g = oracle.make_grid(1, (n,), (-5.0,), (5.0,))
    x = -5 + np.arange(n) * 10 / n
    V = 0.5 * x * x
    K = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        K[:, j] = oracle.apply_K(e, V, g)
    w, U = np.linalg.eigh(K)
    pR, pI = np.exp(-(x - 0.5) ** 2), 0.2 * np.exp(-(x + 0.3) ** 2)
    T = 0.4
    ex = U @ (np.exp(-1j * w * T) * (U.T @ (pR + 1j * pI)))
    errs = []
    for steps in (40, 80, 160):
        R, I, _ = oracle.run_rk4(pR, pI, V, g, T / steps, steps)
        errs.append(np.sqrt(np.sum((R - ex.real) ** 2 + (I - ex.imag) ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 4) < 0.25), slopes


def test_fig3_symplectic_holds_the_norm_rk_does_not():
    """Fig. 3 (qualitative, Section 3.1): over a long run the RK norm decays
    steadily (|amplification|^2 = 1 - s^6/72 + s^8/576 < 1 per mode), while the
    paper's SPSTD keeps its norm error bounded and much smaller at the same dt."""
    p = inputs.well_1d(steps=0)
    n = 256
    g = oracle.make_grid(1, (n,), (-20.0,), (20.0,))
    dt = 2.5e-3
    c, d = oracle.preset("PAPER3")
    R1, I1, R2, I2 = p.psiR.copy(), p.psiI.copy(), p.psiR.copy(), p.psiI.copy()
    n0, _ = oracle.norm_energy(R1, I1, p.V, g)
    dev_sym, dev_rk = [], []
    for _ in range(10):
        R1, I1, _ = oracle.run(R1, I1, p.V, g, c, d, dt, 200)
        R2, I2, _ = oracle.run_rk4(R2, I2, p.V, g, dt, 200)
        dev_sym.append(oracle.norm_energy(R1, I1, p.V, g)[0] - n0)
        dev_rk.append(oracle.norm_energy(R2, I2, p.V, g)[0] - n0)
    dev_rk = np.array(dev_rk)
    assert np.all(np.diff(dev_rk) < 0)                 # RK: monotone loss of norm
    assert max(abs(x) for x in dev_sym) < 0.1 * abs(dev_rk[-1])
