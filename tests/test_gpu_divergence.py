"""The divergence rule and the batch's HBM cap, on the device.

spstd_energy_norm reports SPSTD_EDIVERGED when the norm or energy is not
finite, or when the norm has drifted from that of the last state set by more
than cfg.norm_drift_limit (1e-3 by default): the symplectic schemes keep the
norm to a bounded rounding-level oscillation, so a larger drift means a bad
dt or corrupted fields.  The failures are made on the host: a state with a
NaN, and the RK4 comparison scheme, whose norm decays by design (Fig. 3)."""
import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs, spstd
from helpers import gpu_solver

pytestmark = pytest.mark.gpu


def test_nan_state_is_reported_diverged():
    p = inputs.gaussian_problem((64, 32), dt=1e-3, steps=2)
    s = gpu_solver(p, 32, cap=4)
    R = p.psiR.copy()
    R[17] = np.nan
    s.spstd_set_state(R, p.psiI)
    s.spstd_step(2)
    with pytest.raises(spstd.SpstdError) as ei:
        s.spstd_energy_norm()
    assert ei.value.status == spstd.SPSTD_EDIVERGED and not np.isfinite(ei.value.norm)
    # the context stays usable: a good state steps and reports normally
    s.spstd_set_state(p.psiR, p.psiI)
    s.spstd_step(2)
    nv, _ = s.spstd_energy_norm()
    assert abs(nv - 1.0) < 1e-5
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_norm_drift_past_the_limit_is_reported(precision):
    # a noisy start puts weight in the high modes, which RK4 damps (|R|^2 =
    # 1 - s^6/72 + s^8/576 per step at s = w dt): the norm falls by ~2e-4 a step
    p = inputs.gaussian_problem((64,), integrator="RK4", dt=0.0, steps=1, noise=0.1, seed=9)
    s = gpu_solver(p, precision, cap=1)
    loss = 0.0
    raised = None
    for _ in range(200):
        s.spstd_step(1)
        try:
            nv, _ = s.spstd_energy_norm()
            loss = 1.0 - nv
        except spstd.SpstdError as e:
            raised = e
            break
    s.close()
    assert raised is not None and raised.status == spstd.SPSTD_EDIVERGED
    assert 1.0 - raised.norm > 1e-3 and loss <= 1e-3
    # with the rule off the same run only reports the values
    s = gpu_solver(p, precision, cap=1, norm_drift_limit=0.0)
    s.spstd_step(200)
    nv, _ = s.spstd_energy_norm()
    s.close()
    assert 1.0 - nv > 1e-3


def test_symplectic_long_run_stays_under_the_limit():
    p = inputs.well_1d(steps=0)
    s = gpu_solver(p, 32, cap=1)
    s.spstd_step(20000)
    nv, _ = s.spstd_energy_norm()
    s.close()
    assert abs(nv - 1.0) < 1e-4


def test_batch_hbm_cap_admission():
    probs = [inputs.gaussian_problem((64, 64), (-8.0,) * 2, (8.0,) * 2, seed=50 + i, dt=0.0, steps=4, n_probe=2)
             for i in range(3)]
    solvers = [gpu_solver(q, 32, cap=8) for q in probs]
    need = solvers[0].workspace_bytes
    b = spstd.Batch(8, hbm_cap_bytes=2 * need)
    assert b.spstd_batch_footprint() == (0, 2 * need)
    s0 = b.spstd_batch_add(solvers[0])
    b.spstd_batch_add(solvers[1])
    assert b.spstd_batch_footprint()[0] == 2 * need
    with pytest.raises(spstd.SpstdError) as ei:
        b.spstd_batch_add(solvers[2])
    assert ei.value.status == spstd.SPSTD_ENOTREADY
    b.spstd_batch_step(4)
    b.spstd_batch_sync()
    b.spstd_batch_remove(s0)
    assert b.spstd_batch_footprint()[0] == need
    b.spstd_batch_add(solvers[2])
    b.spstd_batch_step(4)
    b.spstd_batch_sync()
    b.close()
    # a member larger than the cap by itself is refused outright
    small = spstd.Batch(2, hbm_cap_bytes=need // 2)
    with pytest.raises(spstd.SpstdError) as ei:
        small.spstd_batch_add(solvers[0])
    assert ei.value.status == spstd.SPSTD_EINVAL
    small.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("n,precision,x_schedule", [((64, 64, 64), 32, 0), ((64, 64, 64), 32, 6),
                                                    ((96, 48), 32, 0), ((48, 24, 96), 64, 0), ((2048,), 32, 0),
                                                    ((256,), 64, 0), ((4096, 16), 32, 0)])
def test_workspace_guards_intact_after_steps(n, precision, x_schedule):
    """No pass writes past its workspace region: the guard words after every
    region keep their pattern through steps, H applies, spectra and norms."""
    p = inputs.gaussian_problem(n, dt=0.0, steps=20, n_probe=3)
    s = gpu_solver(p, precision, cap=32)
    if x_schedule:
        s.spstd_set_schedule(0, x_schedule)
    assert s.spstd_check_workspace()
    s.spstd_step(20)
    s.spstd_apply_hamiltonian(1)
    s.spstd_spectrum(-1)
    s.spstd_energy_norm()
    assert s.spstd_check_workspace()
    s.close()


def test_workspace_guard_damage_is_reported():
    """A byte of the guard after psi_R, overwritten from the host side through
    the caller-owned workspace tensor, is reported (a made fault, no kernel
    involved)."""
    p = inputs.gaussian_problem((32, 32), dt=0.0, steps=2)
    s = gpu_solver(p, 32, cap=4)
    assert s.spstd_check_workspace()
    psi_bytes = (4 * p.n_total + 255) // 256 * 256   # psi_R's region, then its guard
    s._ws[s.workspace_offset + psi_bytes + 7] = 0
    assert not s.spstd_check_workspace()
    s.close()


def test_workspace_guards_intact_rk4():
    """The RK4 comparison scheme's stage fields (reduce-add TMA passes on
    fields of their own) stay inside their regions too."""
    p = inputs.gaussian_problem((64, 64, 64), integrator="RK4", dt=0.0, steps=6, n_probe=2)
    s = gpu_solver(p, 32, cap=8, norm_drift_limit=0.0)
    s.spstd_step(6)
    assert s.spstd_check_workspace()
    s.close()
