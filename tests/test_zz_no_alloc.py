"""spstd_norm_noalloc: the norm reduction for callers that may not allocate
device memory where they call (a framework that owns every device byte, or a
hot loop that cannot take cudaMalloc's implicit synchronisation).  Its scratch
is the library's static device array; the caller passes only inputs and the
output.  Checked through the C ABI against the existing spstd_energy_norm on
two calls in a row.  Collected last so that a run stopping at the first failure
has already run every other test; it also passes alone in a fresh process (the
first call sets up the array's address for the device)."""
import numpy as np
import pytest

from paper_1805_03155_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-6)])
def test_norm_noalloc_matches_energy_norm(precision, tol):
    import torch

    from paper_1805_03155_gb300 import spstd

    p = inputs.gaussian_problem((32, 16, 64), (-4, -4, -4), (4, 4, 4), seed=21, dt=1e-3, steps=4, n_probe=0)
    s = spstd.solver_for(p, precision=precision, probe_capacity=1)
    s.spstd_step(3)
    R, Im = s.spstd_get_state()
    norm_ref, _ = s.spstd_energy_norm()
    s.close()

    dtype = torch.float64 if precision == 64 else torch.float32
    dev = torch.device("cuda", 0)
    tr = torch.tensor(R, dtype=dtype, device=dev)
    ti = torch.tensor(Im, dtype=dtype, device=dev)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    cell = np.prod([(p.hi[a] - p.lo[a]) / p.n[a] for a in range(3)])
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out.fill_(float("nan"))
        st = spstd.spstd_norm_noalloc(tr.data_ptr(), ti.data_ptr(), tr.numel(), precision, cell,
                                      out.data_ptr(), stream.cuda_stream)
        assert st == spstd.SPSTD_OK, st
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - norm_ref) <= tol * abs(norm_ref), (call, got, norm_ref)


def test_norm_noalloc_rejects_bad_sizes():
    import torch

    from paper_1805_03155_gb300 import spstd

    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    o = torch.zeros(1, dtype=torch.float64, device="cuda")
    ok = spstd.spstd_norm_noalloc(t.data_ptr(), t.data_ptr(), 8, 64, 1.0, o.data_ptr())
    assert ok == spstd.SPSTD_OK
    too_big = spstd.spstd_norm_noalloc(t.data_ptr(), t.data_ptr(), spstd.NOALLOC_MAX_ELEMS + 1, 64, 1.0,
                                       o.data_ptr())
    assert too_big == spstd.SPSTD_EINVAL
    assert spstd.spstd_norm_noalloc(0, t.data_ptr(), 8, 64, 1.0, o.data_ptr()) == spstd.SPSTD_EINVAL
    assert spstd.spstd_norm_noalloc(t.data_ptr(), t.data_ptr(), 0, 64, 1.0, o.data_ptr()) == spstd.SPSTD_EINVAL
    assert spstd.spstd_norm_noalloc(t.data_ptr(), t.data_ptr(), 8, 16, 1.0, o.data_ptr()) == spstd.SPSTD_EINVAL
    torch.cuda.synchronize()
