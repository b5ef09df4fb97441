"""Host-side checks of admission and of the divergence rule's configuration,
without a GPU: the request server refuses a request whose device footprint
alone exceeds its HBM cap (it could never be admitted, so queueing it would
keep the request loop waiting for good), and config validation refuses a NaN
norm-drift limit."""
import ctypes as C

import pytest

from paper_1805_03155_gb300 import build, inputs, serve, spstd


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    spstd.lib()


def test_oversized_request_is_refused_and_loop_returns():
    p = inputs.gaussian_problem((64, 64, 64), (-8.0,) * 3, (8.0,) * 3, seed=3, dt=0.0, steps=10, n_probe=2)
    srv = serve.Server(hbm_cap_bytes=1 << 20, max_slots=4, chunk_steps=5)
    need = srv.footprint_of(p)
    assert need > (1 << 20)
    with pytest.raises(spstd.SpstdError) as ei:
        srv.submit(p, 10)
    assert ei.value.status == spstd.SPSTD_EINVAL
    assert not srv.queue
    # nothing is queued, so the loop ends at once (and never touches a device)
    assert srv.run() == []
    assert srv.batch is None
    srv.close()


def test_request_at_the_cap_is_queued():
    p = inputs.gaussian_problem((32, 32), (-8.0,) * 2, (8.0,) * 2, seed=4, dt=0.0, steps=10, n_probe=2)
    probe = serve.Server(hbm_cap_bytes=1 << 40)
    need = probe.footprint_of(p)
    srv = serve.Server(hbm_cap_bytes=need, max_slots=4)
    rid = srv.submit(p, 10, arrival=1e30)
    assert rid == 0 and len(srv.queue) == 1 and srv.queue[0].need == need
    srv.queue.clear()
    srv.close()


def test_nan_drift_limit_is_refused():
    cfg = spstd.make_config(1, (64,), (-4.0,), (4.0,), norm_drift_limit=float("nan"))
    n = C.c_size_t(0)
    assert spstd.lib().spstd_workspace_size(C.byref(cfg), C.byref(n)) == spstd.SPSTD_EINVAL
    cfg = spstd.make_config(1, (64,), (-4.0,), (4.0,), norm_drift_limit=0.0)
    assert spstd.lib().spstd_workspace_size(C.byref(cfg), C.byref(n)) == spstd.SPSTD_OK


def test_config_init_sets_the_drift_limit():
    cfg = spstd.spstd_config()
    spstd.lib().spstd_config_init(C.byref(cfg))
    assert cfg.norm_drift_limit == 1e-3 and cfg.no_graph == 0
