"""Schedules and the autotuner: every candidate schedule of every axis computes
the same step (bitwise where only the tile plan changes, to rounding where the
radix sequence changes), matches the oracle, and tuning leaves the state alone;
a tuned batch still equals its members' lone solves."""
import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs
from helpers import gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def stable(p, frac=0.4):
    """The problem with dt at frac of its stability limit."""
    import dataclasses

    from paper_1805_03155_gb300 import spstd

    cfg = spstd.make_config(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], integrator=p.integrator)
    _, dt_max = spstd.stability_limit(cfg, float(np.max(p.V)))
    return dataclasses.replace(p, dt=frac * dt_max)


def schedule_runs(p, precision, steps):
    """{(axis, schedule): (psiR, psiI)} for every candidate, other axes default."""
    out = {}
    s0 = gpu_solver(p, precision, cap=steps, merge=False)
    cands = {ax: s0.spstd_schedule_candidates(ax) for ax in range(p.dims)}
    s0.close()
    for ax, lst in cands.items():
        for v in lst:
            s = gpu_solver(p, precision, cap=steps, merge=False)
            s.spstd_set_schedule(ax, v)
            assert s.spstd_get_schedule(ax) == v
            s.spstd_step(steps)
            out[(ax, v)] = s.spstd_get_state()
            s.close()
    return cands, out


@pytest.mark.parametrize("n,precision", [((128, 64), 32), ((128, 64), 64), ((64, 64, 64), 32),
                                         ((32, 256, 16), 64), ((512, 32), 32), ((64, 512), 32),
                                         ((16, 32, 512), 32), ((16, 128, 64), 32), ((32, 32, 32), 32),
                                         ((32, 64), 32), ((96, 48, 16), 32), ((48, 32), 32)])
def test_every_schedule_same_step(n, precision):
    p = stable(inputs.gaussian_problem(n, steps=12, noise=1e-2))
    cands, runs = schedule_runs(p, precision, p.steps)
    oR, oI, _ = oracle_run(p)
    tol = 1e-10 if precision == 64 else 1e-4
    plain_exact = {0, 1, 2, 4}
    for ax, lst in cands.items():
        if 32 <= n[ax] <= 512 and n[ax] & (n[ax] - 1) == 0:
            assert 3 in lst and len(lst) >= 3, (ax, lst)   # a radix variant and a tile variant at least
        # plain schedules with the default radix plan agree bit for bit
        ref_v = 4 if 4 in lst else 0
        R0, I0 = runs[(ax, ref_v)]
        for v in lst:
            R, Im = runs[(ax, v)]
            assert rel_l2(R, Im, oR, oI) <= tol, (ax, v)
            if v in plain_exact and not (v == 0 and ref_v == 4):
                assert np.array_equal(R, R0) and np.array_equal(Im, I0), (ax, v)
            else:
                assert rel_l2(R, Im, R0, I0) <= (1e-13 if precision == 64 else 1e-5), (ax, v)
        # per-warp x tiles run the default TMA x pass's arithmetic: the same bits,
        # except where schedule 0 means the fused reduce-add x-y pass (nx = ny in
        # {32, 64}), which sums the x and y terms in another order
        if 6 in lst:
            assert ax == 0 and 0 in lst
            Rw, Iw = runs[(ax, 6)]
            Rd, Id = runs[(ax, 0)]
            if len(n) >= 2 and n[0] == n[1] and n[0] in (32, 64):
                assert rel_l2(Rw, Iw, Rd, Id) <= 1e-5
            else:
                assert np.array_equal(Rw, Rd) and np.array_equal(Iw, Id)


def test_set_schedule_rejects_unknown():
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem((16, 1024), steps=1))   # 16 and 1024 points: not tunable
    s = gpu_solver(p, 32)
    assert s.spstd_schedule_candidates(0) == [0] and s.spstd_schedule_candidates(1) == [0]
    for bad in (1, 3, 7, -1):
        with pytest.raises(spstd.SpstdError) as ei:
            s.spstd_set_schedule(0, bad)
        assert ei.value.status == spstd.SPSTD_EINVAL
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_tune_keeps_state_and_picks_a_candidate(precision):
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem((64, 128, 32), steps=6))
    s = gpu_solver(p, precision, cap=16)
    s.spstd_step(3)
    R0, I0 = s.spstd_get_state()
    ms = s.spstd_tune(reps=5)
    R1, I1 = s.spstd_get_state()
    assert np.array_equal(R0, R1) and np.array_equal(I0, I1)
    assert s.spstd_steps_taken() == 3
    for ax in range(3):
        cand = s.spstd_schedule_candidates(ax)
        chosen = s.spstd_get_schedule(ax)
        assert chosen in cand
        for v in range(spstd.SCHEDULES):
            assert (ms[ax, v] > 0) == (v in cand)
        assert ms[ax, chosen] == min(ms[ax, v] for v in cand)
    s.spstd_step(3)
    R, Im = s.spstd_get_state()
    z = s.spstd_probe(0)
    s.close()
    oR, oI, oz = oracle_run(p)
    tol = 1e-10 if precision == 64 else 1e-4
    assert rel_l2(R, Im, oR, oI) <= tol
    assert len(z) == 6 and np.max(np.abs(z - oz[0])) <= tol * np.max(np.abs(oz))


def test_tuned_batch_equals_lone_solves():
    from paper_1805_03155_gb300 import spstd

    shapes = [(64, 64), (64, 64), (128, 32), (32, 32, 32), (32, 32, 32), (256,)]
    probs = [stable(inputs.gaussian_problem(sh, seed=40 + k, steps=0, n_probe=2)) for k, sh in enumerate(shapes)]
    steps = 14
    alone = []
    for p in probs:
        s = gpu_solver(p, 32, cap=steps, merge=False)
        s.spstd_step(steps)
        alone.append(s.spstd_get_state())
        s.close()
    batch = spstd.Batch(8)
    solvers = [gpu_solver(p, 32, cap=steps) for p in probs]
    for s in solvers:
        batch.spstd_batch_add(s)
    batch.spstd_batch_tune(reps=3)
    for sh in set(shapes):
        sched = batch.spstd_batch_get_schedule(32, len(sh), sh)
        assert all(v in (0, 1, 2, 3, 4, 6) for v in sched)
        assert all(v != 6 for v in sched[1:])
    # tuning touched no state
    for s, p in zip(solvers, probs):
        R, Im = s.spstd_get_state()
        assert np.array_equal(R, p.psiR.astype(np.float32)) and np.array_equal(Im, p.psiI.astype(np.float32))
    batch.spstd_batch_step(steps)
    batch.spstd_batch_sync()
    for s, (R, Im) in zip(solvers, alone):
        bR, bI = s.spstd_get_state()
        scale = max(np.abs(R).max(), np.abs(Im).max())
        assert np.max(np.abs(bR - R)) <= 1e-5 * scale and np.max(np.abs(bI - Im)) <= 1e-5 * scale
    batch.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("n", [(256, 48), (64, 32, 24), (128, 96), (96, 32, 8), (48, 64)])
def test_warp_x_tiles_with_a_potential_field(n):
    """Schedule 6 with a potential that does not separate (a square well in
    2D/3D is a box, not a sum), so the per-warp x pass reads the V field: the
    same bits as schedule 0, and the oracle's step to the FP32 tolerance."""
    from paper_1805_03155_gb300 import spstd

    p = stable(inputs.gaussian_problem(n, steps=8, noise=1e-2, well=(6.0, 1.5)))
    out = []
    for v in (0, 6):
        s = gpu_solver(p, 32, cap=8, merge=False)
        assert not s.spstd_potential_separable()
        assert 6 in s.spstd_schedule_candidates(0)
        s.spstd_set_schedule(0, v)
        s.spstd_step(p.steps)
        out.append(s.spstd_get_state())
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    oR, oI, _ = oracle_run(p)
    assert rel_l2(out[1][0], out[1][1], oR, oI) <= 1e-4


def test_batch_warp_x_tiles_equal_lone_solves():
    """Batch schedule 6 (per-warp x tiles) on x lines of 32, 48, 96, 128 and 256
    points, in groups whose members all have separable tables and in groups
    that read V fields (a square well, or a member that asks for the field):
    every member ends bit for bit where its lone solve (block x tiles) ends."""
    from paper_1805_03155_gb300 import spstd

    shapes = [((32, 64), "ho"), ((32, 64), "ho"), ((48, 32, 8), "ho"), ((48, 32, 8), "well"),
              ((96, 48, 16), "ho"), ((96, 48, 16), "ho"), ((128, 32, 8), "ho"), ((128, 32, 8), "field"),
              ((256, 64), "ho"), ((256, 64), "well")]
    probs = []
    for k, (sh, kind) in enumerate(shapes):
        kw = dict(well=(5.0, 1.5)) if kind == "well" else {}
        probs.append(stable(inputs.gaussian_problem(sh, seed=900 + k, steps=0, n_probe=2, **kw)))
    steps = 9
    alone = []
    for p, (_, kind) in zip(probs, shapes):
        s = gpu_solver(p, 32, cap=steps, merge=False, v_field_only=kind == "field")
        assert s.spstd_get_schedule(0) == 0
        s.spstd_step(steps)
        alone.append(s.spstd_get_state())
        s.close()
    batch = spstd.Batch(len(probs))
    solvers = [gpu_solver(p, 32, cap=steps, v_field_only=kind == "field") for p, (_, kind) in zip(probs, shapes)]
    for s in solvers:
        batch.spstd_batch_add(s)
    for sh in {sh for sh, _ in shapes}:
        batch.spstd_batch_set_schedule(32, len(sh), sh, [6] + [0] * (len(sh) - 1))
        assert batch.spstd_batch_get_schedule(32, len(sh), sh)[0] == 6
    batch.spstd_batch_step(steps)
    batch.spstd_batch_sync()
    for i, (s, (R, Im)) in enumerate(zip(solvers, alone)):
        bR, bI = s.spstd_get_state()
        assert np.array_equal(bR, R) and np.array_equal(bI, Im), i
    batch.close()
    for s in solvers:
        s.close()


def test_batch_set_schedule_rejects_unknown():
    from paper_1805_03155_gb300 import spstd

    batch = spstd.Batch(2)
    for prec, sh, sched in [(32, (96, 48, 16), [0, 6, 0]),     # per-warp tiles are an x schedule
                            (64, (128, 32), [6, 0]),            # FP32 only
                            (32, (96, 48, 16), [3, 0, 0]),      # no plain variants for 3 * 2^k lines
                            (32, (512, 64), [6, 0]),            # 512-point x lines: block tiles only
                            (32, (128, 32), [7, 0])]:
        with pytest.raises(spstd.SpstdError) as ei:
            batch.spstd_batch_set_schedule(prec, len(sh), sh, sched)
        assert ei.value.status == spstd.SPSTD_EINVAL
    batch.spstd_batch_set_schedule(32, 2, (128, 32), [6, 3])
    assert batch.spstd_batch_get_schedule(32, 2, (128, 32))[:2] == [6, 3]
    batch.close()
