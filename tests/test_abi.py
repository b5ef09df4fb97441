"""The C ABI without a GPU: the library loads, exports every entry point the
header declares, its config struct matches the binding byte for byte, and the
host-only calls (validation, workspace sizing, stability limit) behave."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1805_03155_gb300 import build, spstd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return spstd.lib()


def test_exports_every_declared_symbol(L):
    names = spstd.declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_config_layout_matches_c(tmp_path):
    """sizeof/offsetof of spstd_config from a C compiler vs the ctypes mirror."""
    fields = [f[0] for f in spstd.spstd_config._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'printf("{f} %zu\\n", offsetof(spstd_config, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "spstd.h"\nint main(void){\n'
                   f'printf("size %zu\\n", sizeof(spstd_config));\n{body}\nreturn 0;}}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(out["size"]) == C.sizeof(spstd.spstd_config)
    for f in fields:
        assert int(out[f]) == getattr(spstd.spstd_config, f).offset, f


@pytest.mark.parametrize("name", ["LEAPFROG", "STRANG", "PAPER3", "FR4", "SUZUKI6"])
def test_stability_limit_matches_oracle(L, name):
    cfg = spstd.make_config(3, (64, 64, 64), (-8,) * 3, (8,) * 3, integrator=name)
    s, dtm = spstd.stability_limit(cfg, vmax=96.0)
    so = oracle.stability_limit(*oracle.preset(name))
    assert abs(s - so) <= 1e-12 * so
    wmax = 1.5 * (np.pi / 0.25) ** 2 + 96.0
    assert abs(dtm - so / wmax) <= 1e-12 * dtm


def _status(cfg):
    n = C.c_size_t(0)
    return spstd.lib().spstd_workspace_size(C.byref(cfg), C.byref(n)), n.value


def test_validation_codes(L):
    ok = spstd.make_config(3, (16, 32, 8), (-1,) * 3, (1,) * 3, precision=32, probes=[0, 5], probe_capacity=100)
    st, nbytes = _status(ok)
    assert st == spstd.SPSTD_OK and nbytes > 16 * 32 * 8 * 4 * 4
    bad = [
        spstd.make_config(4, (16,), (0,), (1,)),                       # dims
        spstd.make_config(1, (1,), (0,), (1,)),                        # n < 2
        spstd.make_config(1, (16,), (0,), (1,), bc=(7,)),              # unknown boundary
        spstd.make_config(1, (16,), (1,), (0,)),                       # hi < lo
        spstd.make_config(1, (16,), (0,), (1,), precision=16),         # precision
        spstd.make_config(1, (16,), (0,), (1,), probes=[16]),          # probe outside
        spstd.make_config(1, (16,), (0,), (1,), probe_capacity=0),
        spstd.make_config(1, (16,), (0,), (1,), c=[0.0], d=[0.0]),     # no nonzero coefficient
        spstd.make_config(1, (16,), (0,), (1,), max_nfft=100),
    ]
    for cfg in bad:
        assert _status(cfg)[0] == spstd.SPSTD_EINVAL
    long_x = spstd.make_config(2, (2048, 16), (0, 0), (1, 1))      # x beyond one block: four-step pass
    assert _status(long_x)[0] == spstd.SPSTD_OK
    for n in [(4096, 2048), (1 << 23,)]:                          # long y; x beyond 2^22
        assert _status(spstd.make_config(len(n), n, (0,) * len(n), (1,) * len(n)))[0] == spstd.SPSTD_EUNSUPPORTED
    odd_long = spstd.make_config(1, (300,), (0,), (1,))          # not a power of two, > 256
    assert _status(odd_long)[0] == spstd.SPSTD_EUNSUPPORTED
    walls = spstd.make_config(3, (9, 12, 100), (0,) * 3, (1,) * 3, bc=(1, 2, 0))
    assert _status(walls)[0] == spstd.SPSTD_OK
    unstable = spstd.make_config(1, (256,), (-20,), (20,), dt=1.0)
    assert _status(unstable)[0] == spstd.SPSTD_EUNSTABLE


def test_null_arguments_are_rejected(L):
    assert L.spstd_step(None, 1) == spstd.SPSTD_EINVAL
    assert L.spstd_destroy(None) == spstd.SPSTD_OK
    assert L.spstd_last_error(None) == b"no context"
    ws = C.c_void_p(0)
    cfg = spstd.make_config(1, (16,), (0,), (1,))
    out = C.c_void_p(0)
    assert L.spstd_create(C.byref(cfg), None, 0, C.byref(out)) == spstd.SPSTD_EINVAL
    assert L.spstd_create(C.byref(cfg), C.c_void_p(256 * 1024), 16, C.byref(out)) == spstd.SPSTD_ENOMEM
    assert L.spstd_create(C.byref(cfg), C.c_void_p(257), 1 << 30, C.byref(out)) == spstd.SPSTD_EINVAL
    assert not out.value
