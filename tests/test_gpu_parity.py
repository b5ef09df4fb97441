"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 fields to 1e-10 relative (L2 over the grid; element-wise
1e-10 of the field's max), FP32 fields to 1e-4 relative L2 (the FP32 target),
eigen-energies to 1e-5 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs
from helpers import gpu_run, gpu_solver, oracle_grid, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

SHAPES = [
    (8,), (64,), (256,), (1024,), (4096,),
    (32, 64), (128, 16), (4, 8), (256, 64),
    (16, 32, 8), (32, 32, 32), (8, 4, 64), (64, 16, 16),
    # radix-3 line lengths (3 * 2^k) on every axis
    (96, 48), (384, 24), (48, 24, 96), (24, 192, 8),
]


_ORACLE_CACHE = {}


def cached_oracle_run(p, key):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle_run(p)
    return _ORACLE_CACHE[key]


def small_problem(shape, integrator="FR4", steps=12, seed=11):
    dims = len(shape)
    lo = [-4.0 - 0.5 * a for a in range(dims)]
    hi = [4.0 + 0.25 * a for a in range(dims)]
    # dt at ~0.3 of the stability limit of the finest axis
    dx = min((hi[a] - lo[a]) / shape[a] for a in range(dims))
    dt = 0.3 / (0.5 * dims * (np.pi / dx) ** 2 + 0.5 * 4.5 ** 2 * dims)
    return inputs.gaussian_problem(shape, lo, hi, seed=seed + len(shape), integrator=integrator,
                                   dt=dt, steps=steps, n_probe=4)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("precision", [64, 32])
def test_hamiltonian_apply_matches_oracle(shape, precision):
    """H psi_R and H psi_I (the kernels of one half-stage with coefficient 1)."""
    p = small_problem(shape)
    s = gpu_solver(p, precision)
    g = oracle_grid(p)
    # error scale of a spectral second derivative: the operator norm of H times
    # the field's size (a rounding of the input at the highest wave number is
    # amplified by (pi/dx)^2), ||H|| <= (hbar^2/2m) sum (pi/dx_d)^2 + max V
    hnorm = p.hbar ** 2 / (2 * p.mass) * sum((np.pi * p.n[a] / (p.hi[a] - p.lo[a])) ** 2
                                             for a in range(p.dims)) + np.max(np.abs(p.V))
    for which, f in ((0, p.psiR), (1, p.psiI)):
        got = s.spstd_apply_hamiltonian(which)
        ref = p.hbar * oracle.apply_K(f, p.V, g)
        err = np.max(np.abs(got - ref))
        if precision == 64:
            assert err <= 1e-11 * np.max(np.abs(ref)), (which, err)
        else:  # ~8 FP32 epsilons of ||H|| max|psi|
            assert err <= 1e-6 * hnorm * np.max(np.abs(f)), (which, err, hnorm)
    s.close()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("integrator", ["FR4", "SUZUKI6", "PAPER3"])
def test_steps_match_oracle(shape, precision, integrator):
    p = small_problem(shape, integrator=integrator, steps=20)
    R, Im, pr = gpu_run(p, precision)
    oR, oI, opr = cached_oracle_run(p, (shape, integrator, 20))
    err = rel_l2(R, Im, oR, oI)
    tol = 1e-10 if precision == 64 else 1e-4
    assert err <= tol, err
    if precision == 64:
        scale = max(np.max(np.abs(oR)), np.max(np.abs(oI)))
        assert np.max(np.abs(R - oR)) <= 1e-10 * scale
        assert np.max(np.abs(Im - oI)) <= 1e-10 * scale
    assert np.max(np.abs(pr - opr)) <= (1e-10 if precision == 64 else 1e-4) * np.max(np.abs(opr))


@pytest.mark.parametrize("shape", [(64,), (16, 32), (8, 16, 32)], ids=lambda s: "x".join(map(str, s)))
def test_graph_replay_equals_single_steps(shape):
    """Chunks replayed from the captured graph give bitwise the same result as
    single-step calls (and the probes line up)."""
    p = small_problem(shape, steps=40)
    a = gpu_run(p, 64, chunks=[40], merge=False)
    b = gpu_run(p, 64, chunks=[1] * 40, merge=False)
    c = gpu_run(p, 64, chunks=[17, 3, 16, 4], merge=False)
    # a short first call captures the graph without replaying it; the next,
    # longer call replays it
    d = gpu_run(p, 64, chunks=[5, 20, 15], merge=False)
    for x, y in ((a, b), (a, c), (a, d)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])


@pytest.mark.parametrize("shape", [(16, 32), (8, 16, 32)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("precision", [64, 32])
def test_graph_captured_by_a_short_first_call(shape, precision):
    """With merged step boundaries, a short first call (which captures the
    step graph) and a longer second call (which replays it) give the same bits
    as the same calls with every kernel launched directly."""
    p = small_problem(shape, integrator="SUZUKI6", steps=23)
    out = []
    for no_graph in (False, True):
        s = gpu_solver(p, precision, cap=23, no_graph=no_graph)
        s.spstd_step(3)
        s.spstd_step(20)
        R, Im = s.spstd_get_state()
        z = np.array([s.spstd_probe(q) for q in range(len(p.probes))])
        s.close()
        out.append((R, Im, z))
    for k in range(3):
        assert np.array_equal(out[0][k], out[1][k])


@pytest.mark.parametrize("shape,integrator", [((16, 32), "FR4"), ((8, 16, 32), "SUZUKI6"), ((32, 16), "STRANG"),
                                              ((16, 8, 8), "PAPER3")], ids=str)
def test_merged_step_boundaries_equal_unmerged(shape, integrator):
    """Fusing the last half-stage of a step with the first of the next (same
    field, summed coefficient) is exact: merged and unmerged runs agree to FP64
    rounding, probes included (the boundary probe is interpolated from a
    snapshot), for any chunking of the steps."""
    p = small_problem(shape, integrator=integrator, steps=41)
    ref = gpu_run(p, 64, chunks=[41], merge=False)
    for chunks in ([41], [1] * 41, [17, 3, 21]):
        got = gpu_run(p, 64, chunks=chunks, merge=True)
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        assert np.max(np.abs(got[0] - ref[0])) <= 1e-12 * scale
        assert np.max(np.abs(got[1] - ref[1])) <= 1e-12 * scale
        assert np.max(np.abs(got[2] - ref[2])) <= 1e-12 * np.abs(ref[2]).max()


@pytest.mark.parametrize("shape", [(256,), (32, 64), (16, 16, 32)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("precision", [64, 32])
def test_energy_norm_match_oracle(shape, precision):
    p = small_problem(shape)
    s = gpu_solver(p, precision)
    s.spstd_step(5)
    R, Im = s.spstd_get_state()
    nv, ev = s.spstd_energy_norm()
    on, oe = oracle.norm_energy(R, Im, p.V, oracle_grid(p))
    tol = 1e-12 if precision == 64 else 1e-6
    assert abs(nv - on) <= tol * abs(on)
    assert abs(ev - oe) <= tol * 10 * abs(oe)
    s.close()


def test_checkpoint_resume_is_bitwise():
    p = small_problem((16, 8, 32), steps=30)
    full = gpu_run(p, 64, merge=False)
    s = gpu_solver(p, 64, cap=30, merge=False)
    s.spstd_step(13)
    R, Im = s.spstd_get_state()
    s.close()
    s2 = gpu_solver(p, 64, cap=30, merge=False)
    s2.spstd_set_state(R, Im)
    s2.spstd_step(17)
    R2, I2 = s2.spstd_get_state()
    assert np.array_equal(R2, full[0]) and np.array_equal(I2, full[1])


def test_zero_steps_and_probe_before_steps():
    from paper_1805_03155_gb300 import spstd

    p = small_problem((32, 16))
    s = gpu_solver(p, 64)
    s.spstd_step(0)
    R, Im = s.spstd_get_state()
    assert np.array_equal(R, p.psiR) and np.array_equal(Im, p.psiI)
    with pytest.raises(spstd.SpstdError) as ei:
        s.spstd_probe(0)
    assert ei.value.status == spstd.SPSTD_ENOTREADY
    with pytest.raises(spstd.SpstdError):
        s.spstd_step(-1)
    s.close()


def test_probe_ring_keeps_latest_samples():
    p = small_problem((64,), steps=50)
    s = gpu_solver(p, 64, cap=16)
    s.spstd_step(50)
    z = s.spstd_probe(1)
    _, _, opr = oracle_run(p, steps=50)
    assert len(z) == 16
    assert np.max(np.abs(z - opr[1, -16:])) < 1e-12
    # shorter reads return the latest samples: across the ring's wrap (50 steps
    # in a 16-slot ring: samples 45..49 sit in slots 13, 14, 15, 0, 1) and not
    for cap in (5, 3, 2, 1):
        z = s.spstd_probe(1, cap=cap)
        assert len(z) == cap
        assert np.max(np.abs(z - opr[1, -cap:])) < 1e-12


@pytest.mark.parametrize("precision", [64, 32])
def test_spectrum_matches_oracle_on_well(precision):
    """1D finite well, 3000 steps: the device spectrum of the device series vs
    the oracle spectrum of the oracle series, peak by peak."""
    p = inputs.well_1d(steps=3000)
    s = gpu_solver(p, precision, cap=p.steps)
    s.spstd_step(p.steps)
    E, A = s.spstd_spectrum(-1, max_peaks=8, thresh=1e-3)
    Ec, _ = s.spstd_spectrum(-1, max_peaks=8, thresh=1e-3, phase_correct=True)
    _, _, opr = oracle_run(p)
    th, oE, oA = oracle.spectrum(opr.sum(axis=0), p.dt, max_peaks=8, thresh=1e-3)
    c, d = oracle.preset(p.integrator)
    oEc = np.array([oracle.phase_correct(t, c, d) / p.dt for t in th])
    big = oA > 1e-2 * oA.max()
    assert len(E) == len(oE)
    # FP64: both sides maximise the same flat peak |S(theta)| = f0 (1 - a d^2),
    # a ~ (M/2)^2; rounding-level differences of f move the argmax by
    # ~sqrt(eps/a), 1e-7 relative at M = 3000.  FP32: the 1e-5 energy target.
    tol = 1e-6 if precision == 64 else 1e-5
    assert np.max(np.abs(E[big] - oE[big]) / oE[big]) <= tol
    assert np.max(np.abs(Ec[big] - oEc[big]) / oEc[big]) <= tol
    assert np.allclose(A[big], oA[big], rtol=1e-4)
    s.close()
