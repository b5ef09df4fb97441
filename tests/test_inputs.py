"""The seeded input recipes: the generator against its published definition,
and each workload against the shapes, potentials, normalisation, probe
regions and time steps it is documented to have.  CPU only."""
import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs

M64 = (1 << 64) - 1


def splitmix64_reference(seed, count):
    """SplitMix64 written out from its published definition (Steele, Lea and
    Flood 2014), one value at a time in Python integers."""
    s, out = seed, []
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_its_definition():
    # the stream's first output for seed 0 is the generator's well-known first value
    assert int(inputs.SplitMix64(0).next_u64(1)[0]) == 0xE220A8397B1DCDAF
    for seed in (0, 1, 12345, 2 ** 63 + 7):
        g = inputs.SplitMix64(seed)
        got = [int(x) for x in g.next_u64(5)] + [int(x) for x in g.next_u64(3)]  # state carries over
        assert got == splitmix64_reference(seed, 8)


def test_uniform_normal_and_integer_draws():
    g = inputs.SplitMix64(9)
    u = g.uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3
    z = inputs.SplitMix64(10).normal(200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    k = inputs.SplitMix64(11).integers(100000, 7, 14)
    assert set(np.unique(k)) == set(range(7, 14))


def _cell(p):
    return np.prod([(p.hi[a] - p.lo[a]) / p.n[a] for a in range(p.dims)])


def _coords_of(p, idx):
    x = p.coords()
    i = idx % p.n[0]
    j = (idx // p.n[0]) % p.n[1]
    k = idx // (p.n[0] * p.n[1])
    return [x[0][i], x[1][j], x[2][k]][: p.dims]


def test_well_1d_recipe():
    p = inputs.well_1d()
    assert p.dims == 1 and p.n == (256, 1, 1) and p.lo[0] == -20.0 and p.hi[0] == 20.0
    x = p.coords()[0]
    assert np.all(p.V[np.abs(x) < 2] == 0.0) and np.all(p.V[np.abs(x) >= 2] == 5.0)
    assert np.all(p.psiI == 0.0)
    assert abs(_cell(p) * np.sum(p.psiR ** 2 + p.psiI ** 2) - 1.0) < 1e-12
    assert len(p.probes) == 4 and all(abs(_coords_of(p, q)[0]) <= 3 for q in p.probes)
    assert p.integrator == "FR4" and p.dt == 3.79e-3 and p.steps == 20000
    # the Gaussian's centre lies in (-1, 1): the largest value sits near it
    assert abs(x[np.argmax(p.psiR)]) < 1.1


def test_ho_3d_recipe():
    p = inputs.ho_3d()
    assert p.dims == 3 and p.n == (64, 64, 64)
    X, Y, Z = np.meshgrid(*p.coords(), indexing="ij")
    r2 = (X * X + Y * Y + Z * Z).transpose(2, 1, 0).ravel()  # x fastest
    assert np.allclose(p.V, 0.5 * r2, rtol=0, atol=1e-12)
    assert abs(_cell(p) * np.sum(p.psiR ** 2) - 1.0) < 1e-12 and np.all(p.psiI == 0.0)
    assert len(p.probes) == 8 and all(max(abs(c) for c in _coords_of(p, q)) <= 2 for q in p.probes)
    assert p.integrator == "FR4" and p.dt == 2.36e-3 and p.steps == 10000


@pytest.mark.parametrize("count", [48])
def test_batch_mix_composition(count):
    mix = inputs.batch_mix(count=count, steps=7)
    assert len(mix) == count
    for i, p in enumerate(mix):
        assert p.dims == i % 3 + 1 and p.steps == 7 and p.integrator == "FR4" and p.dt == 0.0
        assert len(p.probes) == 2
        assert abs(_cell(p) * np.sum(p.psiR ** 2 + p.psiI ** 2) - 1.0) < 1e-10
        n = p.n[0]
        if p.dims == 1:
            assert n in [2 ** k for k in range(7, 14)] and (p.lo[0], p.hi[0]) == (-20.0, 20.0)
            V0 = p.V.max()
            assert 1.0 <= V0 < 10.0 and p.V.min() == 0.0
        elif p.dims == 2:
            assert p.n == (n, n, 1) and n in (64, 128, 256, 512)
        else:
            assert p.n == (n, n, n) and n in (32, 48, 64, 96)
    # every 3D size of the mix is drawn
    assert {p.n[0] for p in mix if p.dims == 3} == {32, 48, 64, 96}
    # the same seed gives the same mix
    again = inputs.batch_mix(count=count, steps=7)
    assert all(np.array_equal(a.psiR, b.psiR) and np.array_equal(a.V, b.V) for a, b in zip(mix, again))


def test_aniso_ho_3d_recipe():
    p = inputs.aniso_ho_3d()
    assert p.dims == 3 and p.n == (256, 256, 256) and p.lo == (-12.0,) * 3 and p.hi == (12.0,) * 3
    x = p.coords()
    idx = inputs.SplitMix64(5).integers(2000, 0, p.n_total)
    i, j, k = idx % 256, (idx // 256) % 256, idx // 65536
    want = 0.5 * (x[0][i] ** 2 + 1.3 ** 2 * x[1][j] ** 2 + 1.7 ** 2 * x[2][k] ** 2)
    assert np.allclose(p.V[idx], want, rtol=1e-15, atol=0)
    assert abs(_cell(p) * np.sum(p.psiR ** 2) - 1.0) < 1e-12 and not np.any(p.psiI)
    assert len(p.probes) == 8 and all(max(abs(c) for c in _coords_of(p, q)) <= 2 for q in p.probes)
    assert p.integrator == "SUZUKI6" and p.dt == 6.52e-4 and p.steps == 50000 and p.nfft == 1 << 16
