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
