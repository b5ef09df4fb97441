"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (FP32, pipelined passes at 256^3), on outputs the oracle can compute one
by one: a single half-stage psi_R += c dt K psi_I evaluated at sampled grid
points from the three grid lines through each point (oracle line transforms),
plus properties that hold at any size (norm conservation, psi_I untouched)."""
import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs

pytestmark = pytest.mark.gpu


def line_laplacian(f3, axis, idx, n, lo, hi):
    """Oracle L_axis f at grid index idx = (i, j, k) from the line through it."""
    i, j, k = idx
    if axis == 0:
        line = f3[k, j, :]
    elif axis == 1:
        line = f3[k, :, i]
    else:
        line = f3[:, j, i]
    g = oracle.make_grid(1, (n[axis],), (lo[axis],), (hi[axis],))
    out = oracle.laplacian_axis(np.ascontiguousarray(line), g, 0)
    return out[(i, j, k)[axis]]


@pytest.fixture(scope="module")
def aniso():
    return inputs.aniso_ho_3d(steps=4)


def test_halfstage_256cubed_sampled(aniso):
    from paper_1805_03155_gb300 import spstd

    p = aniso
    # give psi_I structure: 3 SUZUKI6 steps on the device
    a = spstd.solver_for(p, precision=32, probe_capacity=4)
    a.spstd_step(3)
    R, Im = a.spstd_get_state()
    a.close()
    # one custom half-stage: m = 1, c = 0.7, d = 0  ->  psi_R += 0.7 dt K psi_I
    c1 = 0.7
    cfg = spstd.make_config(3, p.n, p.lo, p.hi, precision=32, c=[c1], d=[0.0], dt=p.dt,
                            probes=p.probes, probe_capacity=4)
    b = spstd.Solver(cfg)
    b.spstd_set_potential(p.V)
    b.spstd_set_state(R, Im)
    b.spstd_step(1)
    R2, I2 = b.spstd_get_state()
    b.close()
    assert np.array_equal(I2, Im)
    n = p.n
    R3 = R.reshape(n[2], n[1], n[0])
    I3 = Im.reshape(n[2], n[1], n[0])
    V3 = p.V.reshape(n[2], n[1], n[0])
    rng = np.random.default_rng(4)
    pts = [tuple(int(rng.integers(0, n[a])) for a in range(3)) for _ in range(150)]
    pts += [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (31, 32, 255), (32, 255, 0)]
    err = 0.0
    for (i, j, k) in pts:
        lap = sum(line_laplacian(I3, ax, (i, j, k), n, p.lo, p.hi) for ax in range(3))
        K = p.hbar / (2 * p.mass) * lap + V3[k, j, i] / p.hbar * I3[k, j, i]
        ref = R3[k, j, i] + c1 * p.dt * K
        got = R2.reshape(n[2], n[1], n[0])[k, j, i]
        err = max(err, abs(got - ref))
    scale = max(np.max(np.abs(R)), np.max(np.abs(Im)))
    # FP32 arithmetic of one half-stage: a few epsilons of (|psi| + dt ||K|| |psi|)
    assert err <= 2e-6 * scale, (err, scale)


def test_norm_conserved_256cubed(aniso):
    from paper_1805_03155_gb300 import spstd

    p = aniso
    s = spstd.solver_for(p, precision=32, probe_capacity=64)
    n0, e0 = s.spstd_energy_norm()
    s.spstd_step(40)
    n1, e1 = s.spstd_energy_norm()
    z = s.spstd_probe(0)
    s.close()
    assert abs(n0 - 1.0) < 1e-6
    assert abs(n1 - n0) < 2e-5, (n0, n1)
    assert abs(e1 - e0) < 2e-4 * abs(e0), (e0, e1)
    assert len(z) == 40 and np.all(np.isfinite(z))


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_ho_64cubed_steps_match_oracle(precision, tol):
    """64^3 isotropic oscillator (FR4), 6 full steps, every element."""
    from helpers import gpu_run, oracle_run, rel_l2

    p = inputs.ho_3d(steps=6)
    R, Im, pr = gpu_run(p, precision)
    oR, oI, opr = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= tol
    assert np.max(np.abs(pr - opr)) <= tol * np.max(np.abs(opr))


@pytest.mark.slow
def test_well_1d_full_run_fp64():
    """The 1D finite well at its full length (256 points, FR4, 20000 steps,
    FP64): state and probe series to 1e-10 of the oracle, the device spectrum
    to the oracle's, and the four bound levels within 5 % of the continuum well
    (k tan(ka) = kappa, -k cot(ka) = kappa; the grid puts the wall between two
    points, so the discrete levels differ by 1-4 %)."""
    from helpers import gpu_solver, oracle_run, rel_l2

    p = inputs.well_1d()
    s = gpu_solver(p, 64, cap=p.steps)
    s.spstd_step(p.steps)
    R, Im = s.spstd_get_state()
    z = np.array([s.spstd_probe(q) for q in range(len(p.probes))])
    E, A = s.spstd_spectrum(-1, max_peaks=8, thresh=1e-3, phase_correct=True)
    s.close()
    oR, oI, opr = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-10
    assert np.max(np.abs(z - opr)) <= 1e-10 * np.max(np.abs(opr))
    c, d = oracle.preset(p.integrator)
    th, _, oA = oracle.spectrum(opr.sum(axis=0), p.dt, max_peaks=8, thresh=1e-3)
    oE = np.array([oracle.phase_correct(t, c, d) / p.dt for t in th])
    assert len(E) == len(oE) and np.max(np.abs(E - oE) / oE) <= 1e-6
    cont = np.array([0.229468, 0.911550, 2.023038, 3.500540])
    for e in cont:
        assert np.min(np.abs(E - e)) / e < 0.05


@pytest.mark.parametrize("precision", [32, 64])
def test_ho_3d_levels_vs_closed_form(precision):
    """64^3 isotropic oscillator, FR4, the full 10000 steps on the device: the
    spectral peaks (dispersion-corrected) sit on omega (n + 3/2), n = 0, 1, 2, ...
    (hbar = m = omega = 1), within what a Hann-windowed series of T = 23.6
    resolves: the bin is 2 pi/T = 0.266, adjacent levels are 3.8 bins apart, and
    a strong neighbour's leakage biases a weak refined peak by up to ~0.1 bin;
    the strongest (ground) peak to 5e-3 of a bin."""
    from paper_1805_03155_gb300 import spstd

    p = inputs.ho_3d()
    s = spstd.solver_for(p, precision=precision, probe_capacity=p.steps)
    s.spstd_step(p.steps)
    n0, e0 = s.spstd_energy_norm()
    E, A = s.spstd_spectrum(-1, max_peaks=8, thresh=1e-3, phase_correct=True)
    s.close()
    T = p.steps * p.dt
    bin_e = 2 * np.pi / T
    strong = E[A > 0.05 * A.max()]
    assert len(strong) >= 3
    for e in strong:
        n = np.round(e - 1.5)
        assert abs(e - (n + 1.5)) < 0.1 * bin_e, (e, E, A)
    e0 = E[np.argmax(A)]
    assert abs(e0 - 1.5) < 5e-3 * bin_e, (e0, E, A)
    assert abs(n0 - 1.0) < 1e-5
