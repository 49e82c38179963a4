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
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
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
    jones: np.ndarray
    costs: np.ndarray
    arrival: float
    admitted: float
    finished: float
    status: int

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


class Server:
    def __init__(self, prec=sc.SC_MIXED, mem_budget=None, max_slots=8, n_em=3, n_lm=10,
                 refine_sweeps=1, device="cuda", enqueue_threads=4):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.prec = prec
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            mem_budget = int(0.8 * free)
        self.mem_budget = mem_budget
        self.max_slots = max_slots
        self.opts = dict(n_em=n_em, n_lm=n_lm, refine_sweeps=refine_sweeps)
        self.pending = collections.deque()
        self.running = {}
        self.results = {}
        self.used = 0
        self.max_used = 0
        self.t0 = None
        self.pool = cf.ThreadPoolExecutor(max_workers=enqueue_threads)
        self.lock = threading.Lock()
        self.max_ctas = max(8, 2 * torch.cuda.get_device_properties(self.dev).multi_processor_count // max_slots)

    # -- submission --------------------------------------------------------------------------
    def start(self):
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, job: HostJob):
        job.arrival = self.now()
        self.pending.append(job)

    # -- one scheduling round ------------------------------------------------------------------
    def _admit(self, job: HostJob):
        torch = self.torch
        shp = sc.Shape(job.shape.N, job.shape.T, job.shape.F, len(job.offsets) - 1,
                       int(np.max(np.diff(job.offsets))) if len(job.offsets) > 1 else 0)
        fp = footprint(shp, self.prec)
        stream = torch.cuda.Stream(self.dev)
        cdt = torch.complex64 if self.prec == sc.SC_MIXED else torch.complex128
        with torch.cuda.stream(stream):
            t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).pin_memory().to(
                self.dev, dtype=dt, non_blocking=True)
            d = dict(
                uvw=t(job.uvw, torch.float64), freqs=t(job.freqs, torch.float64),
                sky=sc.DeviceSky(t(job.l, torch.float64), t(job.m, torch.float64), t(job.flux, torch.float64),
                                 t(job.alpha, torch.float64), list(job.offsets), job.f0),
                V=t(job.V, cdt), jones=t(job.jones0, torch.complex128),
                costs=torch.zeros(shp.K, dtype=torch.float64, device=self.dev),
                ws=torch.empty(sc.workspace_size(shp, self.prec), dtype=torch.uint8, device=self.dev))
        entry = dict(job=job, shape=shp, stream=stream, dev=d, bytes=fp, admitted=self.now(),
                     event=None, future=None)

        def enqueue():
            with torch.cuda.stream(stream):
                sc.calibrate_sage(shp, d["uvw"], d["freqs"], d["sky"], d["V"], d["jones"], self.prec, d["ws"],
                                  costs=d["costs"], max_ctas=self.max_ctas, **self.opts)
                ev = torch.cuda.Event()
                ev.record(stream)
            return ev
        entry["future"] = self.pool.submit(enqueue)
        self.used += fp
        self.max_used = max(self.max_used, self.used)
        self.running[job.job_id] = entry

    def _retire(self, jid):
        e = self.running.pop(jid)
        d = e["dev"]
        jones = d["jones"].cpu().numpy()
        costs = d["costs"].cpu().numpy()
        st = sc.device_status(d["ws"])
        self.results[jid] = Result(jid, jones, costs, e["job"].arrival, e["admitted"], self.now(), st)
        self.used -= e["bytes"]
        del e

    def step(self) -> int:
        """Retire finished jobs, then admit queued jobs while they fit.
        Returns the number of jobs still queued or running."""
        for jid in list(self.running):
            e = self.running[jid]
            f = e["future"]
            if f.done():
                if e["event"] is None:
                    e["event"] = f.result()
                if e["event"].query():
                    self._retire(jid)
        while self.pending and len(self.running) < self.max_slots:
            job = self.pending[0]
            shp = sc.Shape(job.shape.N, job.shape.T, job.shape.F, len(job.offsets) - 1,
                           int(np.max(np.diff(job.offsets))))
            need = footprint(shp, self.prec)
            if self.running and self.used + need > self.mem_budget:
                break
            self.pending.popleft()
            self._admit(job)
        return len(self.pending) + len(self.running)

    def drain(self, poll_s=0.0005):
        while self.step():
            time.sleep(poll_s)

    def stats(self):
        lat = np.array([r.latency for r in self.results.values()])
        if lat.size == 0:
            return {}
        span = max(r.finished for r in self.results.values()) - min(r.arrival for r in self.results.values())
        return {"jobs": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "jobs_per_s": float(lat.size / span), "span_s": float(span)}

    def close(self):
        self.pool.shutdown(wait=True)


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
