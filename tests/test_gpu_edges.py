"""Edge cases against the oracle: the smallest axes (2 points), the largest
lengths each pass takes directly, no probes and the most probes, and the full
512-solve batch of the benchmark (tuned, as timed there) checked member by
member on one sampled solve of every shape."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs
from helpers import gpu_run, gpu_solver, oracle_grid, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def stable(p, frac=0.3):
    from paper_1805_03155_gb300 import spstd

    cfg = spstd.make_config(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], integrator=p.integrator,
                            bc=p.bc[: p.dims])
    _, dt_max = spstd.stability_limit(cfg, float(np.max(p.V)))
    return dataclasses.replace(p, dt=frac * dt_max)


@pytest.mark.parametrize("shape", [(2,), (2, 2), (2, 2, 2), (4, 2, 2), (2, 8), (8, 2, 4)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_two_point_axes(shape, precision, tol):
    """n = 2: k = 0 and the Nyquist mode only (k^2 = (pi/dx)^2 kept)."""
    p = stable(inputs.gaussian_problem(shape, steps=9, noise=0.1))
    R, Im, z = gpu_run(p, precision)
    oR, oI, oz = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= tol
    assert np.max(np.abs(z - oz)) <= tol * np.max(np.abs(oz))


@pytest.mark.parametrize("shape,precision", [((8192,), 32), ((4096,), 64), ((2, 1024), 32), ((1024, 2), 64),
                                             ((4, 2, 1024), 32), ((1024, 4, 2), 32)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_largest_direct_lengths(shape, precision):
    p = stable(inputs.gaussian_problem(shape, [-30.0] * len(shape), [30.0] * len(shape), steps=5, noise=1e-2))
    R, Im, z = gpu_run(p, precision)
    oR, oI, oz = oracle_run(p)
    tol = 1e-10 if precision == 64 else 1e-4
    assert rel_l2(R, Im, oR, oI) <= tol


@pytest.mark.parametrize("n_probe", [0, 16])
def test_probe_counts(n_probe):
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem((32, 16, 8), steps=6, n_probe=n_probe))
    s = gpu_solver(p, 64, cap=6)
    s.spstd_step(6)
    R, Im = s.spstd_get_state()
    zs = [s.spstd_probe(q) for q in range(n_probe)]
    with pytest.raises(spstd.SpstdError):
        s.spstd_probe(n_probe)  # one past the last probe
    s.close()
    oR, oI, oz = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-10
    for q in range(n_probe):
        assert np.max(np.abs(zs[q] - oz[q])) <= 1e-10 * np.max(np.abs(oz))


def test_full_benchmark_batch_sampled():
    """The 512-solve mix as bench.py times it (FP32, tuned schedules): after 4
    batched steps, one member of every shape matches the oracle run with the
    dt its solver chose."""
    from paper_1805_03155_gb300 import spstd

    steps = 4
    probs = inputs.batch_mix(512, steps=steps)
    solvers = [spstd.solver_for(p, precision=32, probe_capacity=8, merge=False) for p in probs]
    b = spstd.Batch(513)
    for s in solvers:
        b.spstd_batch_add(s)
    b.spstd_batch_tune(reps=2)
    b.spstd_batch_step(steps)
    b.spstd_batch_sync()
    seen = set()
    checked = 0
    for p, s in zip(probs, solvers):
        key = (p.dims, tuple(p.n))
        if key in seen:
            continue
        seen.add(key)
        R, Im = s.spstd_get_state()
        q = dataclasses.replace(p, dt=s.spstd_get_dt())
        oR, oI, _ = oracle_run(q, steps=steps)
        assert rel_l2(R, Im, oR, oI) <= 1e-4, key
        checked += 1
    b.close()
    for s in solvers:
        s.close()
    assert checked == len(seen) >= 12
