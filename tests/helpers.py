"""Shared test helpers: run a seeded problem through the CUDA library (C ABI) or
through the FP64 oracle, with identical inputs."""
import numpy as np

import oracle
from paper_1805_03155_gb300 import inputs


def oracle_grid(p: inputs.Problem, nyquist_zero=False):
    return oracle.make_grid(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], p.hbar, p.mass,
                            nyquist_zero, bc=p.bc[: p.dims])


def oracle_run(p: inputs.Problem, steps=None, psiR=None, psiI=None, c=None, d=None, dt=None):
    steps = p.steps if steps is None else steps
    if c is None:
        c, d = oracle.preset(p.integrator)
    R = p.psiR if psiR is None else psiR
    Im = p.psiI if psiI is None else psiI
    return oracle.run(R, Im, p.V, oracle_grid(p), c, d, p.dt if dt is None else dt, steps, p.probes)


def gpu_solver(p: inputs.Problem, precision=64, cap=None, **kw):
    from paper_1805_03155_gb300 import spstd
    return spstd.solver_for(p, precision=precision, probe_capacity=cap, **kw)


def gpu_run(p: inputs.Problem, precision=64, steps=None, chunks=None, merge=True):
    """Runs steps (default p.steps) on the GPU; returns (psiR, psiI, probes)."""
    steps = p.steps if steps is None else steps
    s = gpu_solver(p, precision, cap=max(1, steps), merge=merge)
    if chunks is None:
        s.spstd_step(steps)
    else:
        for ch in chunks:
            s.spstd_step(ch)
    R, Im = s.spstd_get_state()
    probes = np.array([s.spstd_probe(q) for q in range(len(p.probes))]) if p.probes and steps else None
    s.close()
    return R, Im, probes


def rel_l2(aR, aI, bR, bI):
    num = np.sqrt(np.sum((aR - bR) ** 2 + (aI - bI) ** 2))
    den = np.sqrt(np.sum(bR ** 2 + bI ** 2))
    return num / den
