"""Host logic of separable potentials (no GPU): the split V(x_i, row r) =
vx[i] + vyz[r] that spstd_set_potential tries before the x pass may rebuild
Eq. 16's V term from two tables.  Pinned against closed forms of the harmonic
well, against potentials that do not separate, and against the acceptance
rule itself (every FP32 sum within 4 units in the last place of V)."""
import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs, spstd


def within_4ulp(V, vx, vyz):
    s = (vyz[:, None] + vx[None, :]).astype(np.float64).ravel()   # IEEE single sums
    return bool(np.all(np.abs(s - V) <= 2.0 ** -22 * np.abs(V)))


def test_harmonic_well_splits_into_its_closed_form():
    om = (1.0, 1.3, 1.7)
    p = inputs.gaussian_problem((64, 32, 16), omega=list(om), steps=1)
    ok, vx, vyz = spstd.separable_split(p.V, 64)
    assert ok and within_4ulp(p.V, vx, vyz)
    # the split is taken at the smallest |V|: the x table is the x term relative
    # to its value there, and vanishes at that column
    x, y, z = p.coords()
    i0 = int(np.argmin(np.abs(x)))
    want_x = 0.5 * om[0] ** 2 * (x * x - x[i0] ** 2)
    assert vx[i0] == 0.0
    np.testing.assert_allclose(vx, want_x, rtol=2e-7, atol=1e-12)
    Z, Y = np.meshgrid(z, y, indexing="ij")
    want_yz = (0.5 * om[0] ** 2 * x[i0] ** 2 + 0.5 * om[1] ** 2 * Y * Y + 0.5 * om[2] ** 2 * Z * Z).ravel()
    np.testing.assert_allclose(vyz, want_yz, rtol=2e-7)
    assert np.all(vx >= 0) and np.all(vyz >= 0)   # one sign: the FP32 sum cannot cancel


@pytest.mark.parametrize("n", [(128, 64), (32, 8, 4), (512, 2)])
def test_two_dimensional_and_thin_grids(n):
    p = inputs.gaussian_problem(n, omega=[0.7, 1.9, 1.1][: len(n)], steps=1)
    ok, vx, vyz = spstd.separable_split(p.V, n[0])
    assert ok and within_4ulp(p.V, vx, vyz)


def test_zero_potential():
    ok, vx, vyz = spstd.separable_split(np.zeros(64 * 12), 64)
    assert ok and not vx.any() and not vyz.any()


def test_potentials_that_do_not_separate():
    p = inputs.gaussian_problem((64, 32, 16), steps=1)
    x, y, z = p.coords()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    assert not spstd.separable_split(p.V + 0.05 * (X * Y).ravel(), 64)[0]        # an x y coupling
    well = inputs.gaussian_problem((64, 32, 16), well=(5.0, 1.5), steps=1)       # a box well: a product
    assert not spstd.separable_split(well.V, 64)[0]
    r = np.sqrt(X * X + Y * Y + Z * Z).ravel()
    assert not spstd.separable_split(-1.0 / (1.0 + r), 64)[0]                    # a radial well


def test_acceptance_is_four_units_in_the_last_place():
    p = inputs.gaussian_problem((64, 32, 16), steps=1)
    k = 64 * 32 * 7 + 13
    for rel, want in ((1e-5, False), (1e-6, False), (1e-8, True)):
        V = p.V.copy()
        V[k] *= 1.0 + rel
        ok, vx, vyz = spstd.separable_split(V, 64)
        assert ok == want, rel
        assert ok == within_4ulp(V, vx, vyz)


def test_random_separable_potentials_accepted_only_when_the_sums_hold():
    rng = inputs.SplitMix64(11)
    for trial in range(20):
        nx, rows = 32, 24
        f = rng.normal(nx)
        g = rng.normal(rows) * (0.1 if trial % 2 else 10.0)
        V = (g[:, None] + f[None, :]).ravel()
        ok, vx, vyz = spstd.separable_split(V, nx)
        assert ok == within_4ulp(V, vx, vyz)
        # potentials of one sign always pass
        ok2, vx2, vyz2 = spstd.separable_split(V - V.min() + 1.0, nx)
        assert ok2 and within_4ulp(V - V.min() + 1.0, vx2, vyz2)


def test_rejects_bad_arguments():
    with pytest.raises(spstd.SpstdError) as ei:
        spstd.separable_split(np.zeros(0), 1)
    assert ei.value.status == spstd.SPSTD_EINVAL
