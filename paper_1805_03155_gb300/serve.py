"""Continuous-batching request loop on top of the batch C ABI.

Requests (an inputs.Problem plus a step count) arrive over time.  A request
is admitted as soon as a batch slot is free and its device footprint (the
context workspace) fits under the HBM cap; its state then stays on the device
while the batch advances every member in chunks of `chunk_steps`.  A member
whose steps are done is retired at the next chunk boundary: its energy, norm
and probe spectrum are read back, its slot and memory are freed, and its
latency (retire time minus arrival time) is recorded.  A request whose
footprint alone exceeds the cap is refused at submit().  The batch itself
enforces the cap on its members (spstd_batch_add refuses a member that would
take it over); the server checks the same sum, plus the contexts it has set up
but not yet admitted, before it allocates a context.  Requests that arrive
while others run are admitted between chunks, so their work overlaps on the
device with the running ones.  Setting up a request's context and reading a
retired member's results happen on a stream of their own while the batch's
next chunk runs.  When a 2D/3D shape joins the batch for the
first time, the batch's pass schedules are autotuned (spstd_batch_tune, a few
milliseconds) before the next chunk; the choice stays for later members.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import spstd


@dataclass
class Request:
    rid: int
    problem: object
    steps: int
    arrival: float
    admitted: Optional[float] = None
    finished: Optional[float] = None
    done_steps: int = 0
    slot: int = -1
    solver: object = None
    result: Dict = field(default_factory=dict)
    cancelled: bool = False


class Server:
    def __init__(self, hbm_cap_bytes: float = 150e9, max_slots: int = 1024, chunk_steps: int = 500,
                 precision: int = 32, device: int = 0, keep_state: bool = False, spectrum: bool = True,
                 tune: bool = True, keep_series: bool = False):
        # the batch and the setup stream are made on first use (the device is
        # touched only once there is work)
        self.batch = None
        self.setup_stream = None
        self.max_slots = int(max_slots)
        self.cap = int(hbm_cap_bytes)
        self.chunk = int(chunk_steps)
        self.precision = precision
        self.device = device
        self.keep_state = keep_state
        self.keep_series = keep_series
        self.spectrum = spectrum
        self.queue: List[Request] = []
        self.ready: List[Request] = []      # set up, waiting for a batch slot
        self.running: Dict[int, Request] = {}
        self.retiring: List[Request] = []   # out of the batch, results not read yet
        self.done: List[Request] = []
        self.cancelled: List[Request] = []
        self.footprint = 0
        self._next = 0
        self.chunks = 0
        self.tune = tune
        self.tuned_shapes = set()
        self._untuned = False

    def _device(self):
        if self.batch is None:
            import torch

            self.batch = spstd.Batch(self.max_slots, device=self.device, hbm_cap_bytes=self.cap)
            # contexts are set up, and their results read, on a stream of their
            # own, so that this host and device work overlaps the batch's chunks
            self.setup_stream = torch.cuda.Stream(device=torch.device("cuda", self.device))

    def footprint_of(self, problem, steps=None) -> int:
        """Device bytes of the context a request of `steps` steps (default:
        problem.steps) needs: its workspace, with a probe ring of one sample
        per step."""
        steps = problem.steps if steps is None else steps
        cfg = spstd.make_config(problem.dims, problem.n[: problem.dims], problem.lo[: problem.dims],
                                problem.hi[: problem.dims], precision=self.precision,
                                integrator=problem.integrator, dt=problem.dt, probes=problem.probes,
                                probe_capacity=max(1, int(steps)))
        import ctypes as C
        n = C.c_size_t(0)
        st = spstd.lib().spstd_workspace_size(C.byref(cfg), C.byref(n))
        if st != spstd.SPSTD_OK:
            raise spstd.SpstdError(st, "workspace size")
        return int(n.value)

    def submit(self, problem, steps: int, arrival: Optional[float] = None) -> int:
        need = self.footprint_of(problem, steps)
        if need > self.cap:
            # it could never be admitted: refuse it now rather than queue it for good
            raise spstd.SpstdError(spstd.SPSTD_EINVAL, f"request needs {need} bytes of device memory, more than "
                                                       f"the HBM cap of {self.cap} bytes")
        r = Request(self._next, problem, int(steps), time.perf_counter() if arrival is None else arrival)
        r.need = need
        self._next += 1
        self.queue.append(r)
        return r.rid

    def _prepare(self, now: float):
        """Sets up the contexts of arrived requests that fit under the cap."""
        still = []
        for r in self.queue:
            if r.arrival > now or self.footprint + r.need > self.cap:
                still.append(r)
                continue
            self._device()
            r.solver = spstd.solver_for(r.problem, precision=self.precision, probe_capacity=max(1, r.steps),
                                        device=self.device, stream=self.setup_stream)
            self.footprint += r.need
            self.ready.append(r)
        self.queue = still

    def _admit(self):
        """Adds set-up requests to the batch (between chunks)."""
        still = []
        for r in self.ready:
            try:
                r.slot = self.batch.spstd_batch_add(r.solver)
            except spstd.SpstdError as e:
                if e.status == spstd.SPSTD_ENOTREADY:  # batch full: wait for a slot
                    still.append(r)
                    continue
                raise
            r.admitted = time.perf_counter()
            self.running[r.rid] = r
            shape = (r.problem.dims, tuple(r.problem.n))
            if r.problem.dims > 1 and shape not in self.tuned_shapes:
                self.tuned_shapes.add(shape)
                self._untuned = True
        self.ready = still
        if self.tune and self._untuned:
            self.batch.spstd_batch_tune(reps=2)
            self._untuned = False

    def cancel(self, rid: int) -> bool:
        """Withdraws request rid: at once if it is queued or set up but not yet
        admitted; if it is running, its member leaves the batch at the next
        chunk boundary (never while a chunk is on the device) and its context
        is freed.  Its result then carries status "cancelled".  False if rid
        is unknown or already finished."""
        for lst in (self.queue, self.ready):
            for r in lst:
                if r.rid == rid:
                    lst.remove(r)
                    self._drop(r)
                    return True
        r = self.running.get(rid)
        if r is not None:
            r.cancelled = True
            return True
        return False

    def _drop(self, r):
        if r.solver is not None:
            r.solver.close()
            r.solver = None
            self.footprint -= r.need
        r.result["status"] = "cancelled"
        r.finished = time.perf_counter()
        self.cancelled.append(r)

    def _remove_cancelled(self):
        """Takes cancelled members out of the batch (after a chunk)."""
        for rid in [rid for rid, r in self.running.items() if r.cancelled]:
            r = self.running.pop(rid)
            self.batch.spstd_batch_remove(r.slot)
            self._drop(r)

    def _remove_finished(self):
        """Takes members whose steps are done out of the batch (after a chunk)."""
        for rid in [rid for rid, r in self.running.items() if r.done_steps >= r.steps]:
            r = self.running.pop(rid)
            self.batch.spstd_batch_remove(r.slot)
            self.retiring.append(r)

    def _collect(self):
        """Reads the results of retired members (energy, norm, spectrum) and
        frees them; their work runs on the setup stream."""
        for r in self.retiring:
            s = r.solver
            try:
                r.result["norm"], r.result["energy"] = s.spstd_energy_norm()
                r.result["status"] = "ok"
            except spstd.SpstdError as e:
                if e.status != spstd.SPSTD_EDIVERGED:
                    raise
                # the divergence rule: a non-finite or drifted norm marks the request failed
                r.result["norm"], r.result["energy"] = e.norm, e.energy
                r.result["status"] = "diverged"
            r.result["dt"] = s.spstd_get_dt()
            if self.spectrum and r.problem.probes and r.steps >= 2:
                # the strongest 16 peaks above 1e-3 of the largest, dispersion-corrected energies
                r.result["E"], r.result["amp"] = s.spstd_spectrum(-1, max_peaks=16, thresh=1e-3, phase_correct=True)
            if self.keep_series and r.problem.probes:
                r.result["series"] = np.array([s.spstd_probe(q) for q in range(len(r.problem.probes))])
            if self.keep_state:
                r.result["state"] = s.spstd_get_state()
            s.close()
            r.solver = None
            r.finished = time.perf_counter()
            self.footprint -= r.need
            self.done.append(r)
        self.retiring = []

    def step(self):
        """One scheduling round: admit, start one chunk for every member (or
        up to the nearest finish), and while it runs read the results of the
        members retired last round and set up newly arrived requests; then
        take the finished members out of the batch."""
        self._prepare(time.perf_counter())
        self._admit()
        if not self.running:
            self._collect()
            return False
        n = min(self.chunk, min(r.steps - r.done_steps for r in self.running.values()))
        self.batch.spstd_batch_step(n)
        self._collect()
        self._prepare(time.perf_counter())
        self.batch.spstd_batch_sync()
        self.chunks += 1
        for r in self.running.values():
            r.done_steps += n
        self._remove_cancelled()
        self._remove_finished()
        return True

    def run(self, until_empty=True, idle_sleep=1e-3):
        while self.queue or self.ready or self.running or self.retiring:
            if not self.step():
                if not self.queue and not self.ready:
                    break
                if self.queue:
                    nxt = min(r.arrival for r in self.queue)
                    time.sleep(max(0.0, min(idle_sleep, nxt - time.perf_counter())))
        self._collect()
        return self.done

    def latencies(self):
        lat = np.array([r.finished - r.arrival for r in self.done])
        return lat

    def close(self):
        for r in list(self.running.values()) + self.ready + self.retiring:
            if r.solver is not None:
                r.solver.close()
                r.solver = None
        if self.batch is not None:
            self.batch.close()
