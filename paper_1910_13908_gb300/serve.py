"""Continuous-batching calibration server on one GPU.

Calibration jobs (one sub-band x time chunk each, of any station, cluster,
timeslot and channel count) arrive over time.  A job waits in a FIFO queue
until it can be admitted: admission needs a free slot and room for the job's
device footprint (its workspace, visibilities, coherency cache and Jones
state) inside the memory budget.  An admitted job is copied to the device
once, stays resident there while it is calibrated on its own CUDA stream,
and releases its slot and memory when its completion event fires.  Admitted
jobs overlap on the GPU: every kernel of a job runs on that job's stream
and the persistent factorisation kernel of each job is capped to a share of
the SMs, so one job's latency-bound critical path leaves room for the
others.  The results of a job do not depend on what else is running (the
kernels use no atomics in their sums and no data-dependent scheduling of
arithmetic).

Enqueuing a job (thousands of kernel launches) happens on a small pool of
host threads; ctypes releases the GIL during the library call, so the
scheduler keeps admitting and retiring jobs meanwhile.

The policy (Scheduler) is separate from the device (CudaBackend), so that it
can be exercised on the host alone.  A job fails alone: one that cannot be
launched (a library error), fails on the way, is larger than the whole
budget, or is refused memory while nothing else runs gets a "failed" result
with the reason, and its slot and memory go to the next job.  Queued and
running jobs can be cancelled.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import time

import numpy as np

from . import sagecal as sc


@dataclasses.dataclass
class HostJob:
    """A job as it arrives: host arrays (numpy) and its shape."""
    job_id: int
    shape: sc.Shape
    uvw: np.ndarray          # float64 [T][N][3]
    freqs: np.ndarray        # float64 [F]
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray
    alpha: np.ndarray
    offsets: list            # cluster offsets [K+1]
    V: np.ndarray            # complex [T][B][F][2][2]
    jones0: np.ndarray       # complex128 [K][N][2][2]
    f0: float = 150e6
    arrival: float = 0.0     # seconds after the server start


@dataclasses.dataclass
class Result:
    job_id: int
    jones: np.ndarray | None       # None unless outcome == "done"
    costs: np.ndarray | None
    arrival: float
    admitted: float | None         # None if the job was never admitted
    finished: float
    status: int                    # device status word (sc_device_status)
    outcome: str = "done"          # "done", "failed" or "cancelled"
    error: str | None = None       # why the job failed

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint(shape: sc.Shape, prec: int) -> int:
    """Device bytes a job holds while admitted."""
    cb = 8 if prec == sc.SC_MIXED else 16
    B = shape.B
    vis = shape.T * B * shape.F * 4 * cb
    rest = shape.T * shape.N * 3 * 8 + shape.F * 8 + 4 * 8 * shape.S_max * shape.K + \
        2 * shape.K * shape.N * 4 * 16 + shape.K * 8
    return sc.workspace_size(shape, prec) + vis + rest


def job_shape(job: HostJob) -> sc.Shape:
    K = len(job.offsets) - 1
    S_max = int(np.max(np.diff(job.offsets))) if K > 0 else 0
    return sc.Shape(job.shape.N, job.shape.T, job.shape.F, K, S_max)


class AllocationRefused(RuntimeError):
    """The backend cannot reserve a job's device memory at this moment."""


@dataclasses.dataclass
class _Running:
    job: HostJob
    handle: object
    bytes: int
    admitted: float


class Scheduler:
    """Admission and retirement of calibration jobs, independent of the
    device.  A backend provides footprint(job) -> bytes, launch(job) ->
    handle (copies the job in and enqueues its calibration; may raise
    AllocationRefused), done(handle) -> bool, collect(handle) -> (jones,
    costs, device status) (raises if the job failed on the way) and
    release(handle).

    Policy: FIFO; a job is admitted when a slot is free and its footprint
    fits in what the budget has left.  A job larger than the whole budget
    can never run and fails at once (it does not block the queue).  A job
    whose memory the backend refuses waits at the head of the queue while
    other jobs run (their retirement frees memory) and fails if nothing is
    running.  A job that fails to launch or to complete fails alone: its
    slot and memory are released and the other jobs go on.  A queued job
    can be cancelled; a running one finishes on the device (kernels are not
    interrupted) and its result is discarded."""

    def __init__(self, backend, mem_budget: int, max_slots: int, clock=time.perf_counter):
        self.backend = backend
        self.mem_budget = int(mem_budget)
        self.max_slots = int(max_slots)
        self.clock = clock
        self.pending = collections.deque()
        self.running = {}
        self.results = {}
        self.cancel_requested = set()
        self.used = 0
        self.max_used = 0
        self.t0 = None

    # -- submission --------------------------------------------------------------------------
    def start(self):
        self.t0 = self.clock()

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, job: HostJob):
        job.arrival = self.now()
        self.pending.append(job)

    def cancel(self, job_id) -> bool:
        """Cancels a queued or running job; False if it is neither."""
        for job in self.pending:
            if job.job_id == job_id:
                self.pending.remove(job)
                self._finish(job, None, "cancelled")
                return True
        if job_id in self.running:
            self.cancel_requested.add(job_id)
            return True
        return False

    def _finish(self, job, admitted, outcome, jones=None, costs=None, status=0, error=None):
        self.results[job.job_id] = Result(job.job_id, jones, costs, job.arrival, admitted, self.now(), status,
                                          outcome, error)

    # -- one scheduling round ------------------------------------------------------------------
    def _retire(self, jid):
        e = self.running.pop(jid)
        self.used -= e.bytes
        try:
            jones, costs, status = self.backend.collect(e.handle)
            if jid in self.cancel_requested:
                self._finish(e.job, e.admitted, "cancelled", status=status)
            else:
                self._finish(e.job, e.admitted, "done", jones, costs, status)
        except Exception as ex:  # the job alone fails
            self._finish(e.job, e.admitted, "failed", error="%s: %s" % (type(ex).__name__, ex))
        finally:
            self.cancel_requested.discard(jid)
            self.backend.release(e.handle)

    def _admit_next(self) -> bool:
        """Admits (or fails) the job at the head of the queue; False when
        it has to wait."""
        job = self.pending[0]
        try:
            need = int(self.backend.footprint(job))
        except Exception as ex:
            self.pending.popleft()
            self._finish(job, None, "failed", error="%s: %s" % (type(ex).__name__, ex))
            return True
        if need > self.mem_budget:
            self.pending.popleft()
            self._finish(job, None, "failed",
                         error="footprint of %d bytes exceeds the budget of %d" % (need, self.mem_budget))
            return True
        if self.used + need > self.mem_budget:
            return False
        self.pending.popleft()
        admitted = self.now()
        try:
            handle = self.backend.launch(job)
        except AllocationRefused as ex:
            if self.running:
                self.pending.appendleft(job)
                return False
            self._finish(job, admitted, "failed", error="AllocationRefused: %s" % ex)
            return True
        except Exception as ex:
            self._finish(job, admitted, "failed", error="%s: %s" % (type(ex).__name__, ex))
            return True
        self.running[job.job_id] = _Running(job, handle, need, admitted)
        self.used += need
        self.max_used = max(self.max_used, self.used)
        return True

    def step(self) -> int:
        """Retire finished jobs, then admit queued jobs while they fit.
        Returns the number of jobs still queued or running."""
        for jid in list(self.running):
            if self.backend.done(self.running[jid].handle):
                self._retire(jid)
        while self.pending and len(self.running) < self.max_slots:
            if not self._admit_next():
                break
        return len(self.pending) + len(self.running)

    def drain(self, poll_s=0.0005):
        while self.step():
            time.sleep(poll_s)

    def stats(self):
        done = [r for r in self.results.values() if r.outcome == "done"]
        lat = np.array([r.latency for r in done])
        if lat.size == 0:
            return {}
        span = max(r.finished for r in done) - min(r.arrival for r in done)
        return {"jobs": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "jobs_per_s": float(lat.size / span) if span > 0 else 0.0, "span_s": float(span),
                "failed": sum(r.outcome == "failed" for r in self.results.values()),
                "cancelled": sum(r.outcome == "cancelled" for r in self.results.values())}


class CudaBackend:
    """Runs each admitted job on its own CUDA stream: its inputs are copied
    to the device once, its sc_calibrate_sage launch sequence is enqueued on
    a small host thread pool (ctypes releases the GIL during the library
    call), and a CUDA event marks its completion."""

    def __init__(self, prec, device, n_em, n_lm, refine_sweeps, max_ctas, enqueue_threads):
        import torch
        self.torch = torch
        self.prec = prec
        self.dev = torch.device(device)
        self.opts = dict(n_em=n_em, n_lm=n_lm, refine_sweeps=refine_sweeps)
        self.max_ctas = max_ctas
        self.pool = cf.ThreadPoolExecutor(max_workers=enqueue_threads)

    def footprint(self, job: HostJob) -> int:
        return footprint(job_shape(job), self.prec)

    def launch(self, job: HostJob):
        torch = self.torch
        shp = job_shape(job)
        stream = torch.cuda.Stream(self.dev)
        cdt = torch.complex64 if self.prec == sc.SC_MIXED else torch.complex128
        try:
            with torch.cuda.stream(stream):
                t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).pin_memory().to(
                    self.dev, dtype=dt, non_blocking=True)
                d = dict(
                    uvw=t(job.uvw, torch.float64), freqs=t(job.freqs, torch.float64),
                    sky=sc.DeviceSky(t(job.l, torch.float64), t(job.m, torch.float64),
                                     t(job.flux, torch.float64), t(job.alpha, torch.float64), list(job.offsets),
                                     job.f0),
                    V=t(job.V, cdt), jones=t(job.jones0, torch.complex128),
                    costs=torch.zeros(shp.K, dtype=torch.float64, device=self.dev),
                    ws=torch.empty(sc.workspace_size(shp, self.prec), dtype=torch.uint8, device=self.dev))
        except torch.cuda.OutOfMemoryError as ex:
            raise AllocationRefused(str(ex)) from ex
        h = dict(shape=shp, stream=stream, dev=d, event=None)

        def enqueue():
            with torch.cuda.stream(stream):
                sc.calibrate_sage(shp, d["uvw"], d["freqs"], d["sky"], d["V"], d["jones"], self.prec, d["ws"],
                                  costs=d["costs"], max_ctas=self.max_ctas, **self.opts)
                ev = torch.cuda.Event()
                ev.record(stream)
            return ev
        h["future"] = self.pool.submit(enqueue)
        return h

    def done(self, h) -> bool:
        f = h["future"]
        if not f.done():
            return False
        if f.exception() is not None:
            return True
        if h["event"] is None:
            h["event"] = f.result()
        return h["event"].query()

    def collect(self, h):
        h["future"].result()  # re-raises an enqueue error
        d = h["dev"]
        return d["jones"].cpu().numpy(), d["costs"].cpu().numpy(), sc.device_status(d["ws"])

    def release(self, h):
        if h.get("future") is not None and not h["future"].done():
            h["future"].result()
        h.clear()

    def close(self):
        self.pool.shutdown(wait=True)


class Server(Scheduler):
    """The scheduler on the CUDA backend, with a memory budget of 80% of the
    device's free memory unless given."""

    def __init__(self, prec=sc.SC_MIXED, mem_budget=None, max_slots=8, n_em=3, n_lm=10,
                 refine_sweeps=1, device="cuda", enqueue_threads=4):
        import torch
        dev = torch.device(device)
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(dev)
            mem_budget = int(0.8 * free)
        max_ctas = max(8, 2 * torch.cuda.get_device_properties(dev).multi_processor_count // max_slots)
        super().__init__(CudaBackend(prec, device, n_em, n_lm, refine_sweeps, max_ctas, enqueue_threads),
                         mem_budget, max_slots)
        self.prec = prec
        self.max_ctas = max_ctas

    def close(self):
        self.backend.close()


def run_poisson(server: Server, jobs, rate_hz, seed=0):
    """Submit `jobs` with Poisson arrivals (mean rate rate_hz), scheduling
    continuously, and return when every job has finished."""
    from . import synth
    u = synth.uniform(seed, synth.TAG_JOBS + 1, len(jobs))
    gaps = -np.log(u) / rate_hz
    arrivals = np.cumsum(gaps) - gaps[0]
    server.start()
    i = 0
    while i < len(jobs) or server.step():
        while i < len(jobs) and server.now() >= arrivals[i]:
            server.submit(jobs[i])
            i += 1
        server.step()
        time.sleep(0.0005)
    return server.stats()
