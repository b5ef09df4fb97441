"""Continuous batching: requests arriving while others run are admitted
between chunks, their work overlaps on the device, and every result equals the
same solve run alone (bitwise in FP64; FP32 within 1e-5 of the field scale)."""
import time

import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs

pytestmark = pytest.mark.gpu


def requests():
    probs = []
    for k, shape in enumerate([(128,), (512,), (32, 64), (64, 64), (16, 32, 8), (32, 32, 32), (256,), (64, 32)]):
        dims = len(shape)
        p = inputs.gaussian_problem(shape, [-6.0] * dims, [6.0] * dims, seed=300 + k, integrator="FR4",
                                    dt=0.0, steps=0, n_probe=2)
        probs.append((p, 20 + 7 * k))
    return probs


@pytest.mark.parametrize("precision,tune", [(64, False), (64, True), (32, True)])
def test_served_results_equal_lone_solves(precision, tune):
    """Bitwise in FP64 with the default schedules (the same kernels); with
    autotuned schedules the radix plan may differ from the lone solve's, so
    FP64 agrees to rounding and FP32 to its tolerance."""
    from paper_1805_03155_gb300 import serve, spstd

    reqs = requests()
    srv = serve.Server(hbm_cap_bytes=2e9, max_slots=4, chunk_steps=9, precision=precision, keep_state=True,
                       tune=tune)
    t0 = time.perf_counter()
    for i, (p, steps) in enumerate(reqs):
        srv.submit(p, steps, arrival=t0 + 0.002 * i)
    done = srv.run()
    assert len(done) == len(reqs)
    assert srv.chunks > 3
    # overlap: some request was admitted while another was running
    spans = sorted((r.admitted, r.finished) for r in done)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    srv.close()
    for r in done:
        p, steps = reqs[r.rid]
        s = spstd.solver_for(p, precision=precision, probe_capacity=steps, merge=False)
        s.spstd_step(steps)
        R, Im = s.spstd_get_state()
        nv, ev = s.spstd_energy_norm()
        s.close()
        bR, bI = r.result["state"]
        if precision == 64 and not tune:
            assert np.array_equal(bR, R) and np.array_equal(bI, Im), r.rid
            assert r.result["energy"] == ev
        else:
            tol = 1e-12 if precision == 64 else 1e-5
            scale = max(np.abs(R).max(), np.abs(Im).max())
            assert np.max(np.abs(bR - R)) <= tol * scale and np.max(np.abs(bI - Im)) <= tol * scale
            assert abs(r.result["energy"] - ev) <= tol * abs(ev)


def test_admission_respects_hbm_cap():
    """With the cap at the largest request's footprint every request still
    runs, but never more at once than fit: the server's total of set-up
    contexts and the batch's own total of members stay under the cap."""
    from paper_1805_03155_gb300 import serve

    reqs = requests()[:4]
    probe = serve.Server(hbm_cap_bytes=1 << 50)
    cap = max(probe.footprint_of(p, steps) for p, steps in reqs)
    srv = serve.Server(hbm_cap_bytes=cap, max_slots=8, chunk_steps=5, precision=32)
    for p, steps in reqs:
        srv.submit(p, steps)
    most = 0
    while srv.step() or srv.queue or srv.ready:
        used, bcap = srv.batch.spstd_batch_footprint()
        assert bcap == cap and used <= cap and srv.footprint <= cap
        most = max(most, len(srv.running))
    srv.run()
    assert len(srv.done) == 4 and most >= 1
    assert all(r.result["status"] == "ok" for r in srv.done)
    srv.close()


def test_cancelled_request_leaves_at_a_chunk_boundary():
    """Cancelling a running request takes its member out of the batch between
    chunks and frees its context; the other requests still equal their lone
    solves bit for bit (FP64, default schedules)."""
    from paper_1805_03155_gb300 import serve, spstd

    reqs = requests()[:4]
    srv = serve.Server(hbm_cap_bytes=2e9, max_slots=8, chunk_steps=5, precision=64, keep_state=True, tune=False)
    for p, steps in reqs:
        srv.submit(p, steps)
    assert srv.step()
    victim = sorted(srv.running)[1]
    assert srv.cancel(victim)
    srv.run()
    assert [r.rid for r in srv.cancelled] == [victim] and srv.cancelled[0].result["status"] == "cancelled"
    assert sorted(r.rid for r in srv.done) == sorted(set(range(4)) - {victim})
    assert srv.batch.spstd_batch_footprint()[0] == 0 and srv.footprint == 0
    assert not srv.cancel(victim) and not srv.cancel(99)
    srv.close()
    for r in srv.done:
        p, steps = reqs[r.rid]
        s = spstd.solver_for(p, precision=64, probe_capacity=steps, merge=False)
        s.spstd_step(steps)
        R, Im = s.spstd_get_state()
        s.close()
        bR, bI = r.result["state"]
        assert np.array_equal(bR, R) and np.array_equal(bI, Im), r.rid
