"""Batched solves: every member of a batch ends in the same state (and probe
series) as the same solve stepped alone -- bitwise in FP64 (same kernels, same
arithmetic), within the FP32 tolerance in FP32 (the lone FP32 path may take
the pipelined passes, whose V-term rounding order differs)."""
import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs
from helpers import gpu_solver

pytestmark = pytest.mark.gpu


def members():
    out = []
    for k, (shape, integ) in enumerate([((64,), "FR4"), ((64,), "FR4"), ((256,), "SUZUKI6"),
                                         ((32, 64), "FR4"), ((32, 64), "FR4"), ((16, 32, 8), "FR4"),
                                         ((16, 32, 8), "FR4"), ((8, 16, 32), "PAPER3"), ((64, 64), "FR4")]):
        dims = len(shape)
        lo = [-4.0 - 0.3 * k] * dims
        hi = [4.0 + 0.2 * k] * dims
        dx = min((hi[a] - lo[a]) / shape[a] for a in range(dims))
        dt = (0.2 + 0.01 * k) / (0.5 * dims * (np.pi / dx) ** 2 + 0.5 * 5.0 ** 2 * dims)
        out.append(inputs.gaussian_problem(shape, lo, hi, seed=100 + k, integrator=integ, dt=dt, steps=0,
                                           n_probe=3))
    return out


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_members_equal_lone_solves(precision):
    from paper_1805_03155_gb300 import spstd

    probs = members()
    steps = 27  # two graph chunks of 10 + 7 direct steps
    alone = []
    for p in probs:
        s = gpu_solver(p, precision, cap=steps, merge=False)  # batches run every half-stage
        s.spstd_step(steps)
        R, Im = s.spstd_get_state()
        alone.append((R, Im, np.array([s.spstd_probe(q) for q in range(3)])))
        s.close()
    batch = spstd.Batch(16)
    solvers = [gpu_solver(p, precision, cap=steps) for p in probs]
    for s in solvers:
        batch.spstd_batch_add(s)
    assert batch.spstd_batch_size() == len(probs)
    batch.spstd_batch_step(steps)
    batch.spstd_batch_sync()
    for s, (R, Im, pr) in zip(solvers, alone):
        bR, bI = s.spstd_get_state()
        bp = np.array([s.spstd_probe(q) for q in range(3)])
        if precision == 64:
            assert np.array_equal(bR, R) and np.array_equal(bI, Im)
            assert np.array_equal(bp, pr)
        else:
            scale = max(np.abs(R).max(), np.abs(Im).max())
            assert np.max(np.abs(bR - R)) <= 1e-5 * scale and np.max(np.abs(bI - Im)) <= 1e-5 * scale
            assert np.max(np.abs(bp - pr)) <= 1e-5 * scale
    assert batch.spstd_batch_launch_count(steps) > 0
    batch.close()
    for s in solvers:
        s.close()


def test_batch_membership_changes():
    """Members leave and join between batch steps; the others are unaffected."""
    from paper_1805_03155_gb300 import spstd

    probs = members()[:6]
    ref = []
    for p in probs:
        s = gpu_solver(p, 64, cap=40, merge=False)
        s.spstd_step(30)
        ref.append(s.spstd_get_state())
        s.close()
    batch = spstd.Batch(4)
    solvers = [gpu_solver(p, 64, cap=40, merge=False) for p in probs]
    slots = [batch.spstd_batch_add(s) for s in solvers[:4]]
    with pytest.raises(spstd.SpstdError) as ei:
        batch.spstd_batch_add(solvers[4])
    assert ei.value.status == spstd.SPSTD_ENOTREADY
    batch.spstd_batch_step(12)
    batch.spstd_batch_remove(slots[1])          # member 1 leaves after 12 steps
    solvers[1].spstd_step(18)                   # and finishes alone
    solvers[4].spstd_step(12)                   # member 4 runs 12 steps alone,
    batch.spstd_batch_add(solvers[4])           # then joins for the last 18
    batch.spstd_batch_step(18)
    batch.spstd_batch_sync()
    for i in (0, 1, 2, 3, 4):
        R, Im = solvers[i].spstd_get_state()
        assert np.array_equal(R, ref[i][0]) and np.array_equal(Im, ref[i][1]), i
    batch.close()
    for s in solvers:
        s.close()


def test_tma_batch_members_equal_lone_solves_bitwise():
    """FP32 members whose axes have 32..512 points run the batched
    pipelined passes (every member's tiles in one launch, its own tensor maps
    and dt-scaled multipliers); they reach bit for bit the state and probes
    of the same solve stepped alone on the single-grid pipelined passes,
    which do the same per-tile arithmetic."""
    from paper_1805_03155_gb300 import spstd

    shapes = [((64, 64), "FR4"), ((64, 64), "FR4"), ((128, 64), "SUZUKI6"), ((64, 64, 64), "FR4"),
              ((64, 64, 64), "FR4"), ((64, 128, 64), "FR4"), ((256, 64), "FR4"), ((512, 512), "FR4"),
              ((512, 512), "FR4"), ((32, 64, 128), "FR4"), ((32, 32, 32), "FR4"), ((32, 32, 32), "FR4"),
              ((32, 64), "FR4")]
    probs = []
    for k, (shape, integ) in enumerate(shapes):
        dims = len(shape)
        lo = [-5.0 - 0.4 * k] * dims
        hi = [5.0 + 0.3 * k] * dims
        probs.append(inputs.gaussian_problem(shape, lo, hi, seed=300 + k, integrator=integ, dt=0.0, steps=0,
                                             n_probe=2))
    steps = 23  # two graph chunks of 10 + 3 direct steps
    alone = []
    for p in probs:
        s = gpu_solver(p, 32, cap=steps, merge=False)
        # harmonic potentials: the lone x pass rebuilds V from separable tables,
        # the batched one reads the V field, which holds the same FP32 sums
        assert s.spstd_potential_separable()
        s.spstd_step(steps)
        R, Im = s.spstd_get_state()
        alone.append((R, Im, np.array([s.spstd_probe(q) for q in range(2)])))
        s.close()
    batch = spstd.Batch(len(probs))
    solvers = [gpu_solver(p, 32, cap=steps) for p in probs]
    for s in solvers:
        batch.spstd_batch_add(s)
    batch.spstd_batch_step(steps)
    batch.spstd_batch_sync()
    for i, (s, (R, Im, pr)) in enumerate(zip(solvers, alone)):
        bR, bI = s.spstd_get_state()
        bp = np.array([s.spstd_probe(q) for q in range(2)])
        assert np.array_equal(bR, R) and np.array_equal(bI, Im), i
        assert np.array_equal(bp, pr), i
    for (shape, _) in shapes:
        assert batch.spstd_batch_get_schedule(32, len(shape), shape) == [0, 0, 0]
    assert batch.spstd_batch_launch_count(steps) > 0
    batch.close()
    for s in solvers:
        s.close()
