"""The fused x-y passes.  The stored-tile form (3D FP32 grids with nx = ny in
{64, 128, 256}): the same half-stages as the separate passes to FP32 rounding,
the oracle to the FP32 tolerance, deterministic across chunkings and graph
replays (its counters reset themselves between launches), and a bounded wait
that runs out reports SPSTD_ETIMEOUT and leaves the context usable.  The
reduce-add form (nx = ny in {32, 64}, on by default): the oracle to the FP32
tolerance, the plain passes to FP32 rounding, one launch fewer per
half-stage, partial plane units."""
import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs
from helpers import gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def stable(p, frac=0.4):
    import dataclasses

    from paper_1805_03155_gb300 import spstd

    cfg = spstd.make_config(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], integrator=p.integrator)
    _, dt_max = spstd.stability_limit(cfg, float(np.max(p.V)))
    return dataclasses.replace(p, dt=frac * dt_max)


@pytest.mark.parametrize("n", [(64, 64, 64), (128, 128, 8), (256, 256, 4), (64, 64, 2), (128, 128, 33)])
def test_fused_matches_separate_and_oracle(n):
    p = stable(inputs.gaussian_problem(n, steps=6, noise=1e-2, integrator="SUZUKI6"))
    out = {}
    for fused in (True, False):
        s = gpu_solver(p, 32, cap=8)
        assert not s.spstd_get_xy_fusion()  # off until selected
        s.spstd_set_xy_fusion(fused)
        assert s.spstd_get_xy_fusion() == fused
        s.spstd_step(p.steps)
        out[fused] = (*s.spstd_get_state(), s.spstd_probe(0))
        per_step = s.spstd_launch_count(p.steps)
        s.close()
        out[(fused, "launches")] = per_step
    oR, oI, oz = oracle_run(p)
    for fused in (True, False):
        R, Im, z = out[fused]
        assert rel_l2(R, Im, oR, oI) <= 1e-4, fused
        assert np.max(np.abs(z - oz[0])) <= 1e-4 * np.max(np.abs(oz))
    (R1, I1, _), (R0, I0, _) = out[True], out[False]
    assert rel_l2(R1, I1, R0, I0) <= 2e-6
    # one launch fewer per half-stage: 6 steps of SUZUKI6 with fused boundaries apply 6 * 10 + 1;
    # without the stored-tile form, 64-point x-y planes still run the reduce-add fused pass
    fewer = 0 if n[0] == 64 else 6 * 10 + 1
    assert out[(False, "launches")] - out[(True, "launches")] == fewer


def test_fused_deterministic_over_chunks_and_replays():
    """80 steps as one call (graph replays of 16-step chunks) and as uneven
    calls end bit for bit alike: the fused pass's tile counters and tickets
    reset themselves after every launch."""
    p = stable(inputs.gaussian_problem((128, 128, 16), steps=80, noise=1e-2))
    s1 = gpu_solver(p, 32, cap=80, merge=False)
    s1.spstd_set_xy_fusion(True)
    s1.spstd_step(80)
    a = s1.spstd_get_state()
    z1 = s1.spstd_probe(1)
    s1.close()
    s2 = gpu_solver(p, 32, cap=80, merge=False)
    s2.spstd_set_xy_fusion(True)
    for ch in (1, 17, 3, 40, 19):
        s2.spstd_step(ch)
    b = s2.spstd_get_state()
    z2 = s2.spstd_probe(1)
    s2.close()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(z1, z2)


def test_fusion_unavailable_elsewhere():
    from paper_1805_03155_gb300 import spstd

    for n, prec in [((64, 128, 32), 32), ((64, 64, 64), 64), ((64, 64), 32), ((32, 32, 32), 32)]:
        p = stable(inputs.gaussian_problem(n, steps=1))
        s = gpu_solver(p, prec)
        assert not s.spstd_get_xy_fusion()
        with pytest.raises(spstd.SpstdError) as ei:
            s.spstd_set_xy_fusion(True)
        assert ei.value.status == spstd.SPSTD_EUNSUPPORTED
        s.spstd_set_xy_fusion(False)
        s.close()


def test_tune_decides_fusion():
    p = stable(inputs.gaussian_problem((128, 128, 32), steps=4))
    s = gpu_solver(p, 32, cap=8)
    s.spstd_tune(reps=5)
    if s.spstd_get_xy_fusion():
        assert s.spstd_get_schedule(0) == 0 and s.spstd_get_schedule(1) == 0
    s.spstd_step(4)
    R, Im = s.spstd_get_state()
    s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-4


def test_wait_timeout_is_reported_and_recoverable():
    """The x tiles of a fused pass whose plane misses a y tile wait about a
    second, give up and set the status word: the next synchronising call reports
    SPSTD_ETIMEOUT; after a fresh state the context steps correctly again."""
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem((64, 64, 64), steps=3))
    s = gpu_solver(p, 32, cap=8, merge=False)
    s.spstd_set_xy_fusion(True)
    s.spstd_inject_wait_timeout()
    s.spstd_step(1)
    with pytest.raises(spstd.SpstdError) as ei:
        s.spstd_get_state()
    assert ei.value.status == spstd.SPSTD_ETIMEOUT
    s.spstd_set_state(p.psiR, p.psiI)
    s.spstd_step(3)
    R, Im = s.spstd_get_state()
    s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-4


def test_default_pass_wait_timeout_is_reported_and_recoverable():
    """The default pipelined x pass whose first tile is never loaded: the wait
    on that tile's barrier runs out, the block drains its other loads and
    returns with the status word set; the next synchronising call reports
    SPSTD_ETIMEOUT, and after a fresh state the context steps correctly again."""
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem((64, 64, 64), steps=3))
    s = gpu_solver(p, 32, cap=8, merge=False)
    s.spstd_set_xy_fusion(False)
    assert s.spstd_get_schedule(0) == 0
    s.spstd_inject_wait_timeout()
    s.spstd_step(1)
    with pytest.raises(spstd.SpstdError) as ei:
        s.spstd_get_state()
    assert ei.value.status == spstd.SPSTD_ETIMEOUT
    s.spstd_set_state(p.psiR, p.psiI)
    s.spstd_step(3)
    R, Im = s.spstd_get_state()
    s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-4


@pytest.mark.parametrize("n", [(64, 64, 64), (32, 32, 32), (32, 32, 18), (64, 64), (32, 32, 2), (64, 64, 3)])
def test_reduce_fused_xy_matches_oracle_and_plain(n):
    p = stable(inputs.gaussian_problem(n, steps=5, noise=1e-2))
    runs = {}
    for plain in (False, True):
        s = gpu_solver(p, 32, cap=8)
        if plain:  # plain passes on x and y: no fused pass
            s.spstd_set_schedule(0, 4)
            s.spstd_set_schedule(1, 4)
        s.spstd_step(p.steps)
        runs[plain] = (*s.spstd_get_state(), s.spstd_probe(0), s.spstd_launch_count(p.steps))
        s.close()
    oR, oI, oz = oracle_run(p)
    R, Im, z, launches = runs[False]
    assert rel_l2(R, Im, oR, oI) <= 1e-4
    assert np.max(np.abs(z - oz[0])) <= 1e-4 * np.max(np.abs(oz))
    R0, I0, _, launches0 = runs[True]
    assert rel_l2(R, Im, R0, I0) <= 2e-6
    # FR4 (7 half-stages) with fused step boundaries applies 5 * 6 + 1 half-stages
    assert launches0 - launches == 5 * 6 + 1


def test_warp_tile_x_pass_wait_timeout_is_reported_and_recoverable():
    """The same failure path on the per-warp-tile x pass (schedule 6): the
    first tile of the grid's first warp is never loaded, that warp's bounded
    wait runs out and it drains its own loads and returns while the other warps
    finish; SPSTD_ETIMEOUT is reported and the context steps correctly again."""
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem((64, 64, 64), steps=3))
    s = gpu_solver(p, 32, cap=8, merge=False)
    s.spstd_set_schedule(0, 6)
    s.spstd_inject_wait_timeout()
    s.spstd_step(1)
    with pytest.raises(spstd.SpstdError) as ei:
        s.spstd_get_state()
    assert ei.value.status == spstd.SPSTD_ETIMEOUT
    s.spstd_set_state(p.psiR, p.psiI)
    s.spstd_step(3)
    R, Im = s.spstd_get_state()
    s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-4
