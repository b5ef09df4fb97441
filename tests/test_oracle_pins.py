"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each reference value is a brute
force sum, a closed form, a textbook result, a library routine (numpy / scipy)
used as one step, or a number the paper prints (tests/golden/).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_dft(x, sign=-1):
    n = len(x)
    j = np.arange(n)
    return np.array([np.sum(x * np.exp(sign * 2j * np.pi * j * k / n)) for k in range(n)])


# ---------------------------------------------------------------- FFT --------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 18, 24, 27, 32, 36, 48, 64, 7, 11, 20])
def test_fft_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, +1):
        ref = brute_dft(x, sign)
        got = oracle.fft(x, sign)
        assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_fft_roundtrip_large():
    rng = np.random.default_rng(5)
    for n in (256, 1536, 4096):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        back = oracle.fft(oracle.fft(x, -1), +1) / n
        assert np.max(np.abs(back - x)) < 1e-13


# ------------------------------------------------- spectral derivative -------

@pytest.mark.parametrize("dims,n", [(1, (32,)), (2, (16, 12)), (3, (8, 6, 16))])
def test_laplacian_of_trig_modes_is_k2(dims, n):
    """Eq. 9/10: d^2/dx^2 exp(i K_n x) = -K_n^2 exp(i K_n x), so L = F^-1 k^2 F
    maps sin/cos of a grid mode to k^2 times itself."""
    lo = [-1.0, -2.0, -3.0][:dims]
    hi = [2.0, 1.5, 5.0][:dims]
    g = oracle.make_grid(dims, n, lo, hi)
    nn = list(n) + [1] * (3 - dims)
    xs = [lo[a] + np.arange(nn[a]) * (hi[a] - lo[a]) / nn[a] if a < dims else np.zeros(1)
          for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    R = [X.ravel(), Y.ravel(), Z.ravel()]
    for ax in range(dims):
        L = hi[ax] - lo[ax]
        for m in range(0, nn[ax] // 2):
            k = 2 * np.pi * m / L
            for f in (np.sin(k * R[ax] + 0.3), np.cos(k * R[ax] - 1.1) * (1 + 0 * R[0])):
                got = oracle.laplacian_axis(f, g, ax)
                assert np.max(np.abs(got - k * k * f)) < 1e-11 * max(1, k * k)
            # the other axes see a constant along their lines: zero
            for other in range(dims):
                if other != ax:
                    f = np.cos(k * R[ax])
                    assert np.max(np.abs(oracle.laplacian_axis(f, g, other))) < 1e-11


def test_nyquist_mode_kept_or_zeroed():
    """At the Nyquist index the reading multiplies by (pi/dx)^2; the literal
    Eq. 10 (iK twice, real part after each inverse) zeroes it."""
    n = 16
    g_keep = oracle.make_grid(1, (n,), (0.0,), (4.0,))
    g_zero = oracle.make_grid(1, (n,), (0.0,), (4.0,), nyquist_zero=True)
    dx = 4.0 / n
    x = np.arange(n) * dx
    f = np.cos(np.pi * x / dx)  # (-1)^j
    assert np.allclose(oracle.laplacian_axis(f, g_keep, 0), (np.pi / dx) ** 2 * f, atol=1e-10)
    assert np.allclose(oracle.laplacian_axis(f, g_zero, 0), 0.0, atol=1e-10)


def dense_K(g, V, n_total):
    """Dense matrix of the oracle's K, one column per unit vector."""
    K = np.zeros((n_total, n_total))
    e = np.zeros(n_total)
    for j in range(n_total):
        e[:] = 0
        e[j] = 1
        K[:, j] = oracle.apply_K(e, V, g)
    return K


def test_harmonic_oscillator_levels_1d():
    """Spectral K on a 64-point grid on [-8, 8] with V = x^2/2: the low
    eigenvalues are the textbook n + 1/2 (hbar = m = omega = 1)."""
    n = 64
    g = oracle.make_grid(1, (n,), (-8.0,), (8.0,))
    x = -8 + np.arange(n) * 16 / n
    K = dense_K(g, 0.5 * x * x, n)
    assert np.allclose(K, K.T, atol=1e-12)  # K symmetric (real symmetric H)
    w = np.linalg.eigvalsh(K)
    assert np.max(np.abs(w[:12] - (np.arange(12) + 0.5))) < 1e-9


def test_separable_levels_3d_are_sums():
    """A separable V: eigenvalues of the 3D K are sums of 1D ones.  Checked on
    K applied to a product of 1D eigenvectors."""
    n = (8, 6, 10)
    lo, hi = (-3.0, -2.0, -4.0), (3.0, 2.0, 4.0)
    om = (1.0, 1.7, 0.6)
    vecs, vals = [], []
    for a in range(3):
        g1 = oracle.make_grid(1, (n[a],), (lo[a],), (hi[a],))
        x = lo[a] + np.arange(n[a]) * (hi[a] - lo[a]) / n[a]
        w, U = np.linalg.eigh(dense_K(g1, 0.5 * om[a] ** 2 * x * x, n[a]))
        vecs.append(U[:, 1])
        vals.append(w[1])
    g3 = oracle.make_grid(3, n, lo, hi)
    p = inputs.gaussian_problem(n, lo, hi, omega=om)
    psi = np.einsum("k,j,i->kji", vecs[2], vecs[1], vecs[0]).ravel()
    Kpsi = oracle.apply_K(psi, p.V, g3)
    assert np.max(np.abs(Kpsi - sum(vals) * psi)) < 1e-11


def test_nyquist_choice_changes_well_ground_level():
    """cfg1 well (N = 256 on [-20, 20], V0 = 5, half-width 2): the ground level
    of the discrete H with the Nyquist mode kept vs zeroed."""
    n = 256
    x = -20 + np.arange(n) * 40 / n
    V = np.where(np.abs(x) < 2, 0.0, 5.0)
    e_keep = np.linalg.eigvalsh(dense_K(oracle.make_grid(1, (n,), (-20.0,), (20.0,)), V, n))[0]
    e_zero = np.linalg.eigvalsh(dense_K(oracle.make_grid(1, (n,), (-20.0,), (20.0,), nyquist_zero=True), V, n))[0]
    assert abs(e_keep - 0.237760) < 2e-6
    assert abs(e_zero - 0.237685) < 2e-6


# ---------------------------------------------------------- integrator -------

def per_mode_matrix(c, d, s):
    """Eq. 23 for one Fourier mode with s = w dt, factors in stage order:
    each stage applies [[1, c s], [0, 1]] then [[1, 0], [-d s, 1]]."""
    M = np.eye(2)
    for cl, dl in zip(c, d):
        M = np.array([[1.0, 0.0], [-dl * s, 1.0]]) @ np.array([[1.0, cl * s], [0.0, 1.0]]) @ M
    return M


@pytest.mark.parametrize("name", ["LEAPFROG", "STRANG", "PAPER3", "FR4", "SUZUKI6"])
def test_free_particle_matches_per_mode_propagator(name):
    """V = 0: every Fourier mode of K has rate w = hbar k^2/2m* and evolves by
    the 2x2 matrix of Eq. 23, so the oracle's FFT stage loop must agree with the
    closed-form per-mode product (computed here with numpy's FFT)."""
    c, d = oracle.preset(name)
    n = 32
    L = 6.0
    g = oracle.make_grid(1, (n,), (0.0,), (L,), hbar=1.3, mass=0.7)
    rng = np.random.default_rng(3)
    pR = rng.standard_normal(n)
    pI = rng.standard_normal(n)
    dt, steps = 2e-3, 7
    R, Im, _ = oracle.run(pR, pI, np.zeros(n), g, c, d, dt, steps)
    kk = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    w = 1.3 * kk ** 2 / (2 * 0.7)
    FR, FI = np.fft.fft(pR), np.fft.fft(pI)
    outR, outI = np.zeros(n, complex), np.zeros(n, complex)
    for j in range(n):
        M = np.linalg.matrix_power(per_mode_matrix(c, d, w[j] * dt), steps)
        outR[j] = M[0, 0] * FR[j] + M[0, 1] * FI[j]
        outI[j] = M[1, 0] * FR[j] + M[1, 1] * FI[j]
    assert np.max(np.abs(np.fft.ifft(outR).real - R)) < 1e-12
    assert np.max(np.abs(np.fft.ifft(outI).real - Im)) < 1e-12


def test_paper3_coefficients_golden():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "paper3_coefficients.txt"))
                if l.strip() and not l.startswith("#"))
    c, d = oracle.preset("PAPER3")
    assert np.allclose(c, [float(vals["c1"]), float(vals["c2"]), float(vals["c3"])], rtol=0, atol=0)
    assert np.allclose(d, c[::-1], rtol=0, atol=0)


@pytest.mark.parametrize("name", ["LEAPFROG", "STRANG", "PAPER3", "FR4", "SUZUKI6"])
def test_consistency_and_unit_determinant(name):
    """Sum c = sum d = 1 (first-order consistency) and det M = 1 (Eq. 25)."""
    c, d = oracle.preset(name)
    assert abs(sum(c) - 1) < 1e-7 and abs(sum(d) - 1) < 1e-7
    for s in (0.1, 0.7, 1.3):
        assert abs(np.linalg.det(oracle.evolution_matrix(c, d, s)) - 1) < 1e-12


def test_table1_cfl_numbers():
    """Table 1: PSTD (leapfrog, textbook s* = 2) and SPSTD (the paper's
    coefficients) stability, as multiples of 2/(sqrt(D) pi).  With the fastest
    mode w = D (hbar/2m*) (pi/dx)^2 the bound w dt <= s* gives
    sqrt(hbar dt/(m* dx^2)) <= sqrt(s*/2) * 2/(sqrt(D) pi)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_cfl.txt"))
            if l.strip() and not l.startswith("#")]
    got = {"PSTD": oracle.stability_limit(*oracle.preset("LEAPFROG")),
           "SPSTD": oracle.stability_limit(*oracle.preset("PAPER3"))}
    assert abs(got["PSTD"] - 2.0) < 1e-12
    for name, factor, digits in rows:
        ratio = np.sqrt(got[name] / 2.0)
        assert round(ratio, int(digits)) == float(factor), (name, ratio)


def exact_propagate(K, pR, pI, T):
    """exp(-i K T) applied to psi_R + i psi_I (K symmetric, dense eigh)."""
    w, U = np.linalg.eigh(K)
    z = U @ (np.exp(-1j * w * T) * (U.T @ (pR + 1j * pI)))
    return z.real, z.imag


@pytest.mark.parametrize("name,order", [("LEAPFROG", 1), ("STRANG", 2), ("PAPER3", 3),
                                        ("FR4", 4), ("SUZUKI6", 4)])
def test_order_of_convergence(name, order):
    """Global error at fixed T against the exact propagator exp(-iKT): halving
    dt divides it by 2^p, p the order the integrator claims (the paper's set:
    3 in the state).  This also pins the stage ordering of Eq. 17."""
    n = 24
    g = oracle.make_grid(1, (n,), (-5.0,), (5.0,))
    x = -5 + np.arange(n) * 10 / n
    V = 0.5 * x * x
    K = dense_K(g, V, n)
    pR = np.exp(-(x - 0.5) ** 2)
    pI = 0.2 * np.exp(-(x + 0.3) ** 2)
    c, d = oracle.preset(name)
    T = 0.4
    errs = []
    for steps in (40, 80, 160):
        R, Im, _ = oracle.run(pR, pI, V, g, c, d, T / steps, steps)
        eR, eI = exact_propagate(K, pR, pI, T)
        errs.append(np.sqrt(np.sum((R - eR) ** 2 + (Im - eI) ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - order) < 0.25), (errs, slopes)


# ------------------------------------------------------------ spectrum -------

def test_spectrum_recovers_synthetic_frequencies():
    """A series of known complex exponentials z_n = sum a_j exp(-i th_j n):
    the refined peaks sit at th_j (to the golden-section resolution)."""
    M = 3000
    th = np.array([0.031, 0.2, 0.45, 1.1])
    a = np.array([1.0, 0.5, 0.25, 0.8])
    n = np.arange(M)
    z = sum(aj * np.exp(-1j * t * n + 1j * 0.3 * j) for j, (aj, t) in enumerate(zip(a, th)))
    th_got, E, amp = oracle.spectrum(z, dt=0.01, hbar=2.0)
    assert len(th_got) == 4
    assert np.max(np.abs(th_got - th)) < 1e-7
    assert np.allclose(E, 2.0 * th / 0.01, rtol=1e-6)
    assert np.allclose(amp, a, rtol=2e-3)


def test_phase_correct_inverts_dispersion():
    c, d = oracle.preset("FR4")
    for s in (0.01, 0.2, 0.5, 0.78):
        theta = np.arccos(np.trace(per_mode_matrix(c, d, s)) / 2)
        assert abs(oracle.phase_correct(theta, c, d) - s) < 1e-10


@pytest.mark.slow
def test_well_levels_dense_eig_and_transcendental():
    """cfg1 finite well: peaks of the probe spectrum, phase corrected, equal the
    dense-eig levels of the discrete H; and lie within 5 % of the levels of the
    continuum well (k tan(ka) = kappa, -k cot(ka) = kappa, a = 2, V0 = 5)."""
    from scipy.optimize import brentq

    p = inputs.well_1d()  # full run: 20000 steps
    g = oracle.make_grid(1, (256,), (-20.0,), (20.0,))
    c, d = oracle.preset("FR4")
    _, _, probes = oracle.run(p.psiR, p.psiI, p.V, g, c, d, p.dt, p.steps, p.probes)
    th, E, amp = oracle.spectrum(probes.sum(axis=0), p.dt, max_peaks=8, thresh=1e-3)
    Ec = np.array([oracle.phase_correct(t, c, d) / p.dt for t in th])
    levels = np.linalg.eigvalsh(dense_K(g, p.V, 256))
    bound = levels[levels < 5.0]
    assert len(bound) == 4
    # each bound level is found, to 1/500 of a frequency bin 2 pi hbar/T: the
    # Hann window's leakage from the other levels biases a refined peak by a
    # small fraction of a bin
    tol = 2e-3 * 2 * np.pi / (p.steps * p.dt)
    for e in bound:
        assert np.min(np.abs(Ec - e)) < tol, (e, Ec)
    # continuum levels from the transcendental equations
    a, V0 = 2.0, 5.0
    f_even = lambda E: np.sqrt(E) * np.tan(np.sqrt(E) * a) - np.sqrt(V0 - E)
    f_odd = lambda E: -np.sqrt(E) / np.tan(np.sqrt(E) * a) - np.sqrt(V0 - E)
    # hbar = m = 1: k = sqrt(2E); rewrite with k directly
    def roots():
        out = []
        ks = np.linspace(1e-6, np.sqrt(2 * V0) - 1e-9, 20001)
        for par in (0, 1):
            def f(k):
                kap = np.sqrt(2 * V0 - k * k)
                return (k * np.tan(k * a) - kap) if par == 0 else (-k / np.tan(k * a) - kap)
            vals = f(ks)
            for i in range(len(ks) - 1):
                if np.sign(vals[i]) != np.sign(vals[i + 1]) and abs(vals[i]) < 50 and abs(vals[i + 1]) < 50:
                    out.append(brentq(f, ks[i], ks[i + 1]) ** 2 / 2)
        return np.sort(out)
    cont = roots()
    assert np.allclose(cont[:4], [0.229468, 0.911550, 2.023038, 3.500540], atol=2e-6)
    for e_grid, e_cont in zip(bound[:4], cont[:4]):
        assert abs(e_grid - e_cont) / e_cont < 0.05


# ---------------------------------------------------------- norm/energy ------

def test_norm_energy_of_oscillator_ground_states():
    """pi^(-D/4) exp(-r^2/2) has norm 1 and energy D/2 (hbar = m = omega = 1)."""
    for n, dims in (((64,), 1), ((32, 32, 32), 3)):
        lo = [-8.0] * dims
        hi = [8.0] * dims
        p = inputs.gaussian_problem(n, lo, hi)
        xs = p.coords()
        Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        r2 = (X ** 2 + (Y ** 2 if dims > 1 else 0) + (Z ** 2 if dims > 2 else 0)).ravel()
        psi = np.pi ** (-dims / 4) * np.exp(-r2 / 2)
        g = oracle.make_grid(dims, n, lo, hi)
        nv, ev = oracle.norm_energy(psi, np.zeros_like(psi), p.V, g)
        assert abs(nv - 1) < 1e-10
        assert abs(ev - dims / 2) < 1e-8


@pytest.mark.slow
def test_norm_and_energy_do_not_drift():
    """Symplectic map: norm and energy oscillate boundedly (the conservation
    claim of Fig. 3): the largest deviation in the second half of the run is no
    larger than in the first half (+10 %), and small."""
    p = inputs.well_1d(steps=0)
    g = oracle.make_grid(1, (256,), (-20.0,), (20.0,))
    c, d = oracle.preset("FR4")
    R, Im = p.psiR.copy(), p.psiI.copy()
    n0, e0 = oracle.norm_energy(R, Im, p.V, g)
    dn, de = [], []
    for _ in range(20):
        R, Im, _ = oracle.run(R, Im, p.V, g, c, d, p.dt, 400)
        nv, ev = oracle.norm_energy(R, Im, p.V, g)
        dn.append(abs(nv - n0))
        de.append(abs(ev - e0))
    assert max(dn[10:]) <= 1.1 * max(dn[:10]) + 1e-14
    assert max(de[10:]) <= 1.1 * max(de[:10]) + 1e-14
    assert max(dn) < 1e-5 and max(de) / abs(e0) < 1e-4


def test_tabulated_time_steps_are_half_the_limit():
    """The dt written out in the input recipes is 0.5 s*/w_max rounded down to
    three significant digits."""
    cases = [("well_1d_N256", "FR4", [np.pi / (40 / 256)], 5.0),
             ("ho_3d_64", "FR4", [np.pi / 0.25] * 3, 96.0),
             ("aniso_ho_3d_256", "SUZUKI6", [np.pi / (24 / 256)] * 3,
              0.5 * 144 * (1 + 1.3 ** 2 + 1.7 ** 2))]
    for name, integ, kmax, vmax in cases:
        s = oracle.stability_limit(*oracle.preset(integ))
        wmax = 0.5 * sum(k * k for k in kmax) + vmax
        ideal = 0.5 * s / wmax
        e = np.floor(np.log10(ideal)) - 2
        expect = np.floor(ideal / 10 ** e) * 10 ** e
        assert abs(inputs.TIME_STEPS[name] - expect) < 1e-12 * expect, (name, ideal, expect)
