"""Writes tests/golden/ho_3d_64_fr4_oracle.npz: the FP64 oracle's run of the
64^3 isotropic oscillator (FR4, dt = 2.36e-3, seed 2), i.e. Eq. 17 stepped
10000 times with Eq. 16's operator, the state after 2000 and after 10000
steps and the eight probe series over all 10000 steps.

Only the oracle (oracle/) and the seeded input generator compute anything here;
no value comes from the CUDA library.  The run takes about two hours on one
x86 core (0.65 s per step), which is why its result is stored rather than
recomputed by the tests.

    python tests/golden/make_ho_3d_64_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1805_03155_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ho_3d_64_fr4_oracle.npz")
SNAP = (2000, 10000)


def main():
    p = inputs.ho_3d()
    g = oracle.make_grid(3, p.n, p.lo, p.hi, p.hbar, p.mass)
    c, d = oracle.preset(p.integrator)
    R, Im = p.psiR, p.psiI
    done = 0
    snaps = {}
    series = []
    t0 = time.time()
    for target in SNAP:
        R, Im, pr = oracle.run(R, Im, p.V, g, c, d, p.dt, target - done, p.probes)
        series.append(pr)
        done = target
        snaps[target] = (R.copy(), Im.copy())
        print(f"{done} steps, {time.time() - t0:.0f} s", flush=True)
    probes = np.concatenate(series, axis=1)
    np.savez_compressed(
        OUT,
        steps=np.array(SNAP, dtype=np.int64),
        dt=np.float64(p.dt),
        probe_idx=np.array(p.probes, dtype=np.int64),
        psiR_2000=snaps[2000][0], psiI_2000=snaps[2000][1],
        psiR_10000=snaps[10000][0], psiI_10000=snaps[10000][1],
        probes=probes,
        source=np.array("oracle.run on inputs.ho_3d(seed=2): FR4, 64^3 on [-8,8)^3, dt 2.36e-3"),
    )
    print("wrote", OUT)


if __name__ == "__main__":
    main()
