"""Integrity of the stored oracle run (tests/golden/ho_3d_64_fr4_oracle.npz,
written by tests/golden/make_ho_3d_64_golden.py from the oracle alone): the
inputs it was made from, the probe series against the stored states at the
snapshot steps, and the norm and energy the symplectic scheme conserves."""
import os

import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ho_3d_64_fr4_oracle.npz")


@pytest.fixture(scope="module")
def golden():
    return np.load(GOLDEN)


def test_golden_inputs_and_snapshots(golden):
    p = inputs.ho_3d(steps=1)
    assert list(golden["steps"]) == [2000, 10000]
    assert float(golden["dt"]) == p.dt and list(golden["probe_idx"]) == list(p.probes)
    z = golden["probes"]
    assert z.shape == (len(p.probes), 10000)
    for n in (2000, 10000):
        R, Im = golden[f"psiR_{n}"], golden[f"psiI_{n}"]
        assert R.shape == (64 ** 3,) and np.all(np.isfinite(R)) and np.all(np.isfinite(Im))
        # the probe sample recorded after step n is the stored state at the probe points
        assert np.array_equal(z[:, n - 1], R[p.probes] + 1j * Im[p.probes])


def test_golden_conserves_norm_and_energy(golden):
    p = inputs.ho_3d(steps=1)
    g = oracle.make_grid(3, p.n, p.lo, p.hi)
    n0, e0 = oracle.norm_energy(p.psiR, p.psiI, p.V, g)
    for n in (2000, 10000):
        nv, ev = oracle.norm_energy(golden[f"psiR_{n}"], golden[f"psiI_{n}"], p.V, g)
        assert abs(nv - n0) < 1e-10 and abs(ev - e0) < 1e-6 * abs(e0), (n, nv, n0, ev, e0)
