"""The non-symplectic comparison scheme of Fig. 3 (classical Runge-Kutta) on the
device: element-wise parity with the oracle's RK4 on FFT, tiled and wall axes,
the norm behaviour of Fig. 3, and its stability limit and phase correction."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs

pytestmark = pytest.mark.gpu

RK4_S_STAR = 2.0 * np.sqrt(2.0)  # |R(-is)| <= 1 iff s^2 <= 8


def rk4_case(p, precision, steps):
    from helpers import gpu_solver, oracle_grid

    s = gpu_solver(p, precision, cap=steps)
    s.spstd_step(steps)
    R, Im = s.spstd_get_state()
    z = np.array([s.spstd_probe(q) for q in range(len(p.probes))])
    s.close()
    oR, oI, oz = oracle.run_rk4(p.psiR, p.psiI, p.V, oracle_grid(p), p.dt, steps, p.probes)
    return R, Im, z, oR, oI, oz


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
@pytest.mark.parametrize("n,bc", [
    ((64,), (0,)),                 # 1D FFT line
    ((100,), (1,)),                # 1D Dirichlet wall (dense line operator)
    ((32, 16), (0, 0)),            # 2D FFT
    ((48, 20, 6), (0, 2, 1)),      # mixed: FFT x, Neumann y, Dirichlet z
    ((64, 64, 64), (0, 0, 0)),     # 3D FFT, several tiles per pass
])
def test_rk4_matches_oracle(n, bc, precision, tol):
    from helpers import rel_l2

    p = inputs.gaussian_problem(n, integrator="RK4", dt=2e-3, steps=7, bc=bc)
    R, Im, z, oR, oI, oz = rk4_case(p, precision, 7)
    assert rel_l2(R, Im, oR, oI) <= tol
    assert np.max(np.abs(z - oz)) <= tol * np.max(np.abs(oz))


def test_rk4_norm_decays_symplectic_holds_fig3():
    """Fig. 3 on the device: the 1D finite well, same dt for both schemes; RK4's
    norm falls every interval (|R|^2 = 1 - s^6/72 + s^8/576 per mode), the
    paper's three-stage SPSTD scheme keeps it to a far smaller bounded error."""
    from helpers import gpu_solver

    p = inputs.well_1d(steps=0)
    dt = 2.5e-3
    sym = gpu_solver(dataclasses.replace(p, integrator="PAPER3", dt=dt), 64, cap=1)
    # RK4 loses norm by design (Fig. 3): the divergence rule is off for it
    rk = gpu_solver(dataclasses.replace(p, integrator="RK4", dt=dt), 64, cap=1, norm_drift_limit=0.0)
    n0 = sym.spstd_energy_norm()[0]
    dev_sym, dev_rk = [], []
    for _ in range(10):
        sym.spstd_step(200)
        rk.spstd_step(200)
        dev_sym.append(sym.spstd_energy_norm()[0] - n0)
        dev_rk.append(rk.spstd_energy_norm()[0] - n0)
    sym.close()
    rk.close()
    assert np.all(np.diff(dev_rk) < 0)
    assert max(abs(x) for x in dev_sym) < 0.1 * abs(dev_rk[-1])
    # the oracle's RK4 at the same dt loses the same norm
    g = oracle.make_grid(1, (256,), (-20.0,), (20.0,))
    R, Im, _ = oracle.run_rk4(p.psiR, p.psiI, p.V, g, dt, 2000)
    on = oracle.norm_energy(R, Im, p.V, g)[0] - n0
    assert abs(on - dev_rk[-1]) <= 1e-9 * abs(n0)


def test_rk4_stability_limit_and_dt():
    from paper_1805_03155_gb300 import spstd

    p = inputs.gaussian_problem((64,), integrator="RK4", dt=0.0, steps=1)
    cfg = spstd.make_config(1, p.n[:1], p.lo[:1], p.hi[:1], integrator="RK4")
    s_star, dt_max = spstd.stability_limit(cfg)
    assert abs(s_star - RK4_S_STAR) < 1e-14
    # automatic dt: half of s*/w_max
    s = spstd.Solver(cfg)
    s.spstd_set_potential(p.V)
    vmax = float(np.max(p.V))
    L = p.hi[0] - p.lo[0]
    w_max = (np.pi * 64 / L) ** 2 / 2 + vmax
    assert abs(s.spstd_get_dt() - 0.5 * RK4_S_STAR / w_max) <= 1e-12 * s.spstd_get_dt()
    assert s.spstd_get_coefficients()[0].size == 0
    s.close()
    bad = spstd.make_config(1, p.n[:1], p.lo[:1], p.hi[:1], integrator="RK4", dt=1.01 * RK4_S_STAR / w_max)
    with pytest.raises(spstd.SpstdError) as ei:
        b = spstd.Solver(bad)
        b.spstd_set_potential(p.V)
    assert ei.value.status == spstd.SPSTD_EUNSTABLE


def test_rk4_plane_wave_phase_correction():
    """V = 0, psi = exp(i k x): the probe turns by -arg R(-is) per step (s = w dt,
    w = hbar k^2/2m); the phase-corrected spectrum recovers E = hbar^2 k^2/2m
    while the raw peak sits at hbar theta/dt."""
    from paper_1805_03155_gb300 import spstd

    n, L = 16, 10.0  # w_max = (pi n/L)^2/2 = 12.6: dt = 0.122 is inside s*/w_max = 0.224
    x = np.arange(n) * L / n
    k = 2 * np.pi * 5 / L
    dt = 0.6 / (k * k / 2)
    M = 2048
    cfg = spstd.make_config(1, (n,), (0.0,), (L,), integrator="RK4", dt=dt, probes=(3,), probe_capacity=M)
    s = spstd.Solver(cfg)
    s.spstd_set_potential(np.zeros(n))
    s.spstd_set_state(np.cos(k * x), np.sin(k * x))
    s.spstd_step(M)
    E_raw, A_raw = s.spstd_spectrum(0, max_peaks=4)
    E_cor, A_cor = s.spstd_spectrum(0, max_peaks=4, phase_correct=True)
    s.close()
    sv = 0.6
    R = 1 - 1j * sv - sv ** 2 / 2 + 1j * sv ** 3 / 6 + sv ** 4 / 24
    theta = -np.angle(R)
    # the probe rotates as exp(+i k x0) R^t: the spectrum is of exp(-i theta t)
    # (the window times the real decay |R|^t is real, so the peak sits at theta)
    e_raw, e_cor = E_raw[np.argmax(A_raw)], E_cor[np.argmax(A_cor)]
    assert abs(e_raw - theta / dt) <= 1e-6 * theta / dt
    assert abs(e_cor - k * k / 2) <= 1e-6 * k * k / 2


def test_rk4_not_batched():
    from helpers import gpu_solver
    from paper_1805_03155_gb300 import spstd

    p = inputs.gaussian_problem((32, 32), integrator="RK4", dt=1e-3, steps=1)
    s = gpu_solver(p, 32)
    b = spstd.Batch(4)
    with pytest.raises(spstd.SpstdError) as ei:
        b.spstd_batch_add(s)
    assert ei.value.status == spstd.SPSTD_EUNSUPPORTED
    b.close()
    s.close()
