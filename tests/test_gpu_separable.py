"""Separable potentials (FP32, x axis of 32..512, 48 or 96 points): detection,
the x pass that rebuilds Eq. 16's V term from the tables vx(x) + vyz(y, z)
against the oracle, the general form for potentials that do not separate (and
for any potential when the config asks for the V field), a context whose
potential is replaced (the tables must not go stale), and batches whose x
passes take the table form or read the V field."""
import dataclasses

import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs, spstd
from helpers import gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def stable(p, frac=0.4):
    cfg = spstd.make_config(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], integrator=p.integrator)
    _, dt_max = spstd.stability_limit(cfg, float(np.max(p.V)))
    return dataclasses.replace(p, dt=frac * dt_max)


def coupled(p, eps=0.05):
    """The problem's potential plus eps x y: not a sum of an x part and a (y, z) part."""
    xs = p.coords()
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return dataclasses.replace(p, V=p.V + eps * (X * Y).ravel())


def separable(p, precision=32, **kw):
    s = gpu_solver(p, precision, cap=1, **kw)
    f = s.spstd_potential_separable()
    s.close()
    return f


def test_detection():
    ho3 = stable(inputs.gaussian_problem((64, 32, 16), omega=[1.0, 1.3, 1.7], steps=1))
    assert separable(ho3)
    assert not separable(ho3, 64)                     # FP64 fields read the V field
    assert separable(stable(inputs.gaussian_problem((128, 64), steps=1)))
    assert separable(stable(inputs.gaussian_problem((512, 32), omega=[0.0, 0.0], steps=1)))   # V = 0
    assert not separable(stable(coupled(ho3)))
    assert not separable(stable(inputs.gaussian_problem((64, 32, 16), well=(5.0, 1.5), steps=1)))
    assert not separable(stable(inputs.gaussian_problem((16, 64, 32), steps=1)))   # no pipelined x pass
    assert separable(stable(inputs.gaussian_problem((96, 48, 16), steps=1)))       # radix-3 x lines
    assert separable(stable(inputs.gaussian_problem((48, 32), steps=1)))
    assert not separable(ho3, v_field_only=True)      # the config asks for the V field


@pytest.mark.parametrize("n", [(64, 32, 16), (256, 64), (512, 32), (32, 64, 8), (128, 16, 4), (96, 48, 16),
                               (48, 32, 8)])
def test_separable_matches_oracle(n):
    p = stable(inputs.gaussian_problem(n, omega=[1.0, 1.3, 1.7][: len(n)], steps=12, noise=1e-2))
    s = gpu_solver(p, 32, cap=p.steps, merge=False)
    assert s.spstd_potential_separable()
    s.spstd_step(p.steps)
    R, Im = s.spstd_get_state()
    nv, ev = s.spstd_energy_norm()
    s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-4


@pytest.mark.parametrize("n,kind", [((64, 32, 16), "well"), ((64, 32, 16), "coupled"), ((128, 64), "coupled"),
                                    ((256, 16, 8), "well")])
def test_nonseparable_matches_oracle(n, kind):
    if kind == "well":
        p = inputs.gaussian_problem(n, well=(5.0, 1.5), steps=12, noise=1e-2)
    else:
        p = coupled(inputs.gaussian_problem(n, steps=12, noise=1e-2))
    p = stable(p)
    s = gpu_solver(p, 32, cap=p.steps, merge=False)
    assert not s.spstd_potential_separable()
    s.spstd_step(p.steps)
    R, Im = s.spstd_get_state()
    s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(R, Im, oR, oI) <= 1e-4


@pytest.mark.parametrize("n", [(64, 32, 16), (96, 48, 16)])
def test_v_field_only_matches_oracle_and_tables(n):
    """The same separable problem with the V field forced: it matches the
    oracle, and the table form to FP32 rounding (the field is V rounded once,
    the tables' sum rounds vx and vyz first)."""
    p = stable(inputs.gaussian_problem(n, omega=[1.0, 1.3, 1.7], steps=10, noise=1e-2))
    out = []
    for vfo in (False, True):
        s = gpu_solver(p, 32, cap=p.steps, merge=False, v_field_only=vfo)
        assert s.spstd_potential_separable() == (not vfo)
        s.spstd_step(p.steps)
        out.append(s.spstd_get_state())
        s.close()
    oR, oI, _ = oracle_run(p)
    assert rel_l2(*out[1], oR, oI) <= 1e-4
    assert rel_l2(*out[1], *out[0]) <= 1e-5


@pytest.mark.parametrize("order", ["sep_then_not", "not_then_sep"])
def test_replaced_potential(order):
    """set_potential on a context that has already stepped: the new potential's
    form (tables or field) is the one used from then on."""
    base = stable(inputs.gaussian_problem((64, 32, 16), steps=8, noise=1e-2), frac=0.3)
    first, second = (base, coupled(base)) if order == "sep_then_not" else (coupled(base), base)
    s = gpu_solver(first, 32, cap=16, merge=False, dt=base.dt)
    s.spstd_step(4)
    R4, I4 = s.spstd_get_state()
    s.spstd_set_potential(second.V)
    assert s.spstd_potential_separable() == (order == "not_then_sep")
    s.spstd_step(4)
    R, Im = s.spstd_get_state()
    s.close()
    aR, aI, _ = oracle_run(first, steps=4)
    assert rel_l2(R4, I4, aR, aI) <= 1e-4
    bR, bI, _ = oracle_run(second, steps=4, psiR=aR, psiI=aI)
    assert rel_l2(R, Im, bR, bI) <= 1e-4


def test_field_form_wait_timeout_is_reported_and_recoverable():
    """The x pass that reads the V field (a potential that does not separate),
    with its first tile never loaded: the wait runs out, the status is
    reported, and a fresh state steps correctly again."""
    p = stable(coupled(inputs.gaussian_problem((64, 64, 64), steps=3)))
    s = gpu_solver(p, 32, cap=8, merge=False)
    s.spstd_set_xy_fusion(False)
    assert s.spstd_get_schedule(0) == 0 and not s.spstd_potential_separable()
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


def test_batch_mixed_separability_equals_lone():
    """A batched x pass takes the table form when every member of its group
    has tables and reads the V fields otherwise; for a member with a separable
    potential the V field holds the FP32 sums of its tables.  Groups with
    table members only (x lines of 128, 512 and 96 points), groups that mix
    them with potentials that do not separate or with a member that asks for
    the V field, and the fused x-y groups (which read V fields) end bit for bit
    where the lone solves do."""
    shapes = [((64, 64, 64), "ho"), ((64, 64, 64), "ho"), ((32, 32, 32), "ho"), ((32, 32, 32), "coupled"),
              ((256, 64), "ho"), ((256, 64), "well"), ((128, 32, 16), "ho"), ((128, 32, 16), "ho"),
              ((512, 64), "ho"), ((96, 48, 16), "ho"), ((96, 48, 16), "ho"), ((48, 32, 8), "ho"),
              ((48, 32, 8), "coupled"), ((128, 64, 8), "ho"), ((128, 64, 8), "field")]
    probs = []
    for k, (shape, kind) in enumerate(shapes):
        dims = len(shape)
        lo, hi = [-5.0 - 0.3 * k] * dims, [5.0 + 0.2 * k] * dims
        if kind == "well":
            p = inputs.gaussian_problem(shape, lo, hi, seed=400 + k, well=(5.0, 1.5), dt=0.0, steps=0, n_probe=2)
        else:
            p = inputs.gaussian_problem(shape, lo, hi, seed=400 + k, dt=0.0, steps=0, n_probe=2)
            if kind == "coupled":
                p = coupled(p)
        probs.append(p)
    steps = 13
    alone = []
    for p, (_, kind) in zip(probs, shapes):
        s = gpu_solver(p, 32, cap=steps, merge=False, v_field_only=kind == "field")
        assert s.spstd_potential_separable() == (kind == "ho")
        s.spstd_step(steps)
        alone.append(s.spstd_get_state())
        s.close()
    batch = spstd.Batch(len(probs))
    solvers = [gpu_solver(p, 32, cap=steps, v_field_only=kind == "field") for p, (_, kind) in zip(probs, shapes)]
    for s in solvers:
        batch.spstd_batch_add(s)
    batch.spstd_batch_step(steps)
    batch.spstd_batch_sync()
    for i, (s, (R, Im)) in enumerate(zip(solvers, alone)):
        bR, bI = s.spstd_get_state()
        assert np.array_equal(bR, R) and np.array_equal(bI, Im), i
    batch.close()
    for s in solvers:
        s.close()


def test_batch_member_potential_replaced():
    """A batch member whose potential is replaced between batch steps (tables
    to V field, and the dt that follows the new potential): the batch rebuilds
    its descriptors, and every member ends bit for bit where a lone solve that
    does the same ends."""
    probs = [inputs.gaussian_problem((128, 32, 16), [-5.0 - k, -5.0, -5.0], [5.0, 5.0, 5.0 + k], seed=700 + k,
                                     dt=0.0, steps=0, n_probe=2) for k in range(3)]
    newV = coupled(probs[0]).V
    alone = []
    for k, p in enumerate(probs):
        s = gpu_solver(p, 32, cap=16, merge=False)
        s.spstd_step(4)
        if k == 0:
            s.spstd_set_potential(newV)
            assert not s.spstd_potential_separable()
        s.spstd_step(4)
        alone.append(s.spstd_get_state())
        s.close()
    solvers = [gpu_solver(p, 32, cap=16) for p in probs]
    batch = spstd.Batch(len(probs))
    for s in solvers:
        batch.spstd_batch_add(s)
    batch.spstd_batch_step(4)
    batch.spstd_batch_sync()
    solvers[0].spstd_set_potential(newV)
    batch.spstd_batch_step(4)
    batch.spstd_batch_sync()
    for i, (s, (R, Im)) in enumerate(zip(solvers, alone)):
        bR, bI = s.spstd_get_state()
        assert np.array_equal(bR, R) and np.array_equal(bI, Im), i
    batch.close()
    for s in solvers:
        s.close()
