"""x lines longer than one block transforms on chip (four-step FFT through a
scratch array): element-wise parity with the oracle, whose FFT has no length
limit, on 1D lines past the single-block limit up to the 2^22-point maximum,
and on 2D/3D grids with long x lines (even and odd line counts)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs

pytestmark = pytest.mark.gpu


def long_problem(n, integrator="FR4", steps=5, noise=1e-2, seed=7):
    """Grid spacing 0.025 along x (a box of 0.025 n), [-4, 4] on the other
    axes, a weak x oscillator (omega 0.01) so that dt is set by the kinetic
    term; dt = half the stability limit."""
    from paper_1805_03155_gb300 import spstd

    Lx = 0.025 * n[0]
    lo = [-Lx / 2] + [-4.0] * (len(n) - 1)
    hi = [Lx / 2] + [4.0] * (len(n) - 1)
    om = [0.01] + [1.0] * (len(n) - 1)
    p = inputs.gaussian_problem(n, lo, hi, seed=seed, omega=om, integrator=integrator, dt=0.0, steps=steps,
                                noise=noise)
    cfg = spstd.make_config(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], integrator=integrator)
    _, dt_max = spstd.stability_limit(cfg, float(np.max(p.V)))
    return dataclasses.replace(p, dt=0.5 * dt_max)


@pytest.mark.parametrize("n,precision", [
    ((16384,), 32), ((16384,), 64), ((8192,), 64), ((32768,), 32), ((65536,), 64),
    ((2048, 6), 32),        # 2D, x long, dense y (6 points), 3 line pairs
    ((2048, 3), 64),        # odd line count: the last line travels alone
    ((4096, 4, 2), 32),     # 3D, FFT y and z
    ((2048, 8, 3), 64),
])
def test_long_x_matches_oracle(n, precision):
    from helpers import gpu_run, oracle_run, rel_l2

    p = long_problem(n)
    R, Im, pr = gpu_run(p, precision)
    oR, oI, opr = oracle_run(p)
    tol = 1e-10 if precision == 64 else 1e-4
    assert rel_l2(R, Im, oR, oI) <= tol
    assert np.max(np.abs(pr - opr)) <= tol * np.max(np.abs(opr))


@pytest.mark.parametrize("precision,tol", [(32, 2e-6), (64, 1e-12)])
def test_max_length_halfstage(precision, tol):
    """The longest line taken (2^22 points, 1024 x 4096 split): one half-stage
    psi_R += 0.7 dt K psi_I, every element against the oracle."""
    from paper_1805_03155_gb300 import spstd

    n = 1 << 22
    p = long_problem((n,), steps=1, noise=0.3)
    cfg = spstd.make_config(1, (n,), p.lo[:1], p.hi[:1], precision=precision, c=[0.7], d=[0.0], dt=p.dt,
                            probes=p.probes, probe_capacity=2)
    s = spstd.Solver(cfg)
    s.spstd_set_potential(p.V)
    s.spstd_set_state(p.psiR, p.psiI)
    s.spstd_step(1)
    R, Im = s.spstd_get_state()
    s.close()
    g = oracle.make_grid(1, (n,), p.lo[:1], p.hi[:1])
    oR, oI, _ = oracle.run(p.psiR, p.psiI, p.V, g, [0.7], [0.0], p.dt, 1)
    assert np.array_equal(Im, p.psiI.astype(np.float32).astype(np.float64)) if precision == 32 else \
        np.array_equal(Im, p.psiI)
    scale = max(np.max(np.abs(p.psiR)), np.max(np.abs(p.psiI)))
    assert np.max(np.abs(R - oR)) <= tol * scale


def test_long_x_nyquist_zero():
    from helpers import oracle_grid, rel_l2
    from paper_1805_03155_gb300 import spstd

    p = long_problem((16384,), steps=4, noise=0.3)
    cfg = spstd.make_config(1, p.n[:1], p.lo[:1], p.hi[:1], precision=64, integrator="FR4", dt=p.dt,
                            nyquist_zero=True)
    s = spstd.Solver(cfg)
    s.spstd_set_potential(p.V)
    s.spstd_set_state(p.psiR, p.psiI)
    s.spstd_step(4)
    R, Im = s.spstd_get_state()
    s.close()
    c, d = oracle.preset("FR4")
    g = oracle.make_grid(1, p.n[:1], p.lo[:1], p.hi[:1], nyquist_zero=True)
    oR, oI, _ = oracle.run(p.psiR, p.psiI, p.V, g, c, d, p.dt, 4)
    assert rel_l2(R, Im, oR, oI) <= 1e-10
    # and it differs from the kept-Nyquist run by far more than that
    oR2, oI2, _ = oracle.run(p.psiR, p.psiI, p.V, oracle_grid(p), c, d, p.dt, 4)
    assert rel_l2(oR2, oI2, oR, oI) > 1e-8


def test_long_x_energy_and_launches():
    """H-apply (energy) through the four-step pass, graph replay over many
    steps, and the launch count (three launches per x application)."""
    from helpers import gpu_solver

    p = long_problem((32768,), steps=0)
    s = gpu_solver(p, 64, cap=64)
    n0, e0 = s.spstd_energy_norm()
    g = oracle.make_grid(1, p.n[:1], p.lo[:1], p.hi[:1])
    on, oe = oracle.norm_energy(p.psiR, p.psiI, p.V, g)
    assert abs(n0 - on) <= 1e-12 and abs(e0 - oe) <= 1e-10 * abs(oe)
    s.spstd_step(40)
    n1, e1 = s.spstd_energy_norm()
    c, d = oracle.preset("FR4")
    oR, oI, _ = oracle.run(p.psiR, p.psiI, p.V, g, c, d, p.dt, 40)
    on1, oe1 = oracle.norm_energy(oR, oI, p.V, g)
    assert abs(n1 - on1) <= 1e-12 and abs(e1 - oe1) <= 1e-10 * abs(oe1)
    prof = s.spstd_profile_steps(3)
    total = sum(c for _, c in prof.values())
    assert total == s.spstd_launch_count(3)
    nh = 7  # FR4: 4 c's + 3 nonzero d's; boundaries merged: 3 (7 - 1) + 1 applies
    assert prof["x_pass"][1] == 3 * (3 * (nh - 1) + 1)
    s.close()


def test_long_x_not_batched():
    from helpers import gpu_solver
    from paper_1805_03155_gb300 import spstd

    p = long_problem((16384,), steps=1)
    s = gpu_solver(p, 32)
    b = spstd.Batch(2)
    with pytest.raises(spstd.SpstdError) as ei:
        b.spstd_batch_add(s)
    assert ei.value.status == spstd.SPSTD_EUNSUPPORTED
    b.close()
    s.close()
