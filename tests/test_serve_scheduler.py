"""The serving scheduler's policy on the host, with a fake backend whose
jobs complete after a set number of scheduling rounds and whose failures
are injected on the host (no GPU is involved or faulted): admission never
exceeds the memory budget or the slots, the queue is served in order, and a
job that fails to launch, fails on the way, is refused memory, is too large
or is cancelled fails alone while every other job completes."""
import numpy as np
import pytest

from paper_1910_13908_gb300 import serve


class FakeJob:
    def __init__(self, job_id, nbytes, rounds=2, fail_launch=False, fail_collect=False, refuse=0):
        self.job_id = job_id
        self.nbytes = nbytes
        self.rounds = rounds               # scheduling rounds until complete
        self.fail_launch = fail_launch
        self.fail_collect = fail_collect
        self.refuse = refuse               # how many launch attempts are refused memory
        self.arrival = 0.0


class FakeBackend:
    def __init__(self):
        self.live = {}
        self.launched = []
        self.released = []

    def footprint(self, job):
        return job.nbytes

    def launch(self, job):
        if job.refuse > 0:
            job.refuse -= 1
            raise serve.AllocationRefused("no room for %d bytes" % job.nbytes)
        if job.fail_launch:
            raise RuntimeError("sagecal_gb error -1: bad shape")
        h = {"job": job, "left": job.rounds}
        self.live[job.job_id] = h
        self.launched.append(job.job_id)
        return h

    def done(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def collect(self, h):
        if h["job"].fail_collect:
            raise RuntimeError("sagecal_gb error -5: a CUDA runtime call failed")
        return np.full(2, h["job"].job_id), np.zeros(1), 0

    def release(self, h):
        self.released.append(h["job"].job_id)
        self.live.pop(h["job"].job_id, None)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def run(jobs, budget, slots, cancel=None):
    be = FakeBackend()
    s = serve.Scheduler(be, budget, slots, clock=Clock())
    s.start()
    for j in jobs:
        s.submit(j)
    rounds = 0
    peak_slots = 0
    while True:
        if cancel:
            for at, jid in cancel:
                if at == rounds:
                    assert s.cancel(jid)
        n = s.step()
        peak_slots = max(peak_slots, len(s.running))
        assert s.used <= budget and len(s.running) <= slots
        assert s.used == sum(e.bytes for e in s.running.values())
        rounds += 1
        if n == 0:
            break
        assert rounds < 1000
    return s, be, peak_slots


def test_admission_respects_budget_slots_and_order():
    jobs = [FakeJob(i, nb, rounds=r) for i, (nb, r) in
            enumerate([(40, 3), (30, 1), (50, 2), (20, 4), (60, 1), (10, 2)])]
    s, be, peak = run(jobs, budget=100, slots=3)
    assert sorted(s.results) == list(range(6))
    assert all(r.outcome == "done" for r in s.results.values())
    assert be.launched == list(range(6))            # FIFO
    assert s.max_used <= 100 and peak == 3
    assert sorted(be.released) == list(range(6)) and not be.live
    st = s.stats()
    assert st["jobs"] == 6 and st["failed"] == 0 and st["p99_s"] >= st["p50_s"] > 0


def test_a_job_that_fails_to_launch_fails_alone():
    jobs = [FakeJob(0, 30), FakeJob(1, 30, fail_launch=True), FakeJob(2, 30)]
    s, be, _ = run(jobs, budget=100, slots=2)
    assert s.results[1].outcome == "failed" and "bad shape" in s.results[1].error
    assert s.results[1].jones is None
    assert s.results[0].outcome == s.results[2].outcome == "done"
    assert s.used == 0


def test_a_job_that_fails_on_the_way_releases_its_slot_and_memory():
    jobs = [FakeJob(0, 60, fail_collect=True), FakeJob(1, 60), FakeJob(2, 60)]
    s, be, _ = run(jobs, budget=100, slots=2)
    assert s.results[0].outcome == "failed" and "CUDA runtime" in s.results[0].error
    assert s.results[1].outcome == s.results[2].outcome == "done"
    assert sorted(be.released) == [0, 1, 2] and s.used == 0


def test_refused_memory_waits_for_running_jobs_then_fails_when_idle():
    # job 1 is refused twice while job 0 runs: it waits at the head of the queue
    jobs = [FakeJob(0, 50, rounds=4), FakeJob(1, 20, refuse=2), FakeJob(2, 20)]
    s, be, _ = run(jobs, budget=100, slots=3)
    assert all(s.results[i].outcome == "done" for i in range(3))
    assert be.launched.index(1) < be.launched.index(2)   # order kept
    # refused with nothing running: no one can free memory, so it fails
    s2, _, _ = run([FakeJob(0, 20, refuse=5), FakeJob(1, 20)], budget=100, slots=1)
    assert s2.results[0].outcome == "failed" and "AllocationRefused" in s2.results[0].error
    assert s2.results[1].outcome == "done"


def test_a_job_larger_than_the_budget_is_rejected_without_blocking_the_queue():
    jobs = [FakeJob(0, 30), FakeJob(1, 500), FakeJob(2, 30)]
    s, be, _ = run(jobs, budget=100, slots=1)
    assert s.results[1].outcome == "failed" and "exceeds the budget" in s.results[1].error
    assert s.results[1].admitted is None
    assert s.results[0].outcome == s.results[2].outcome == "done"
    assert 1 not in be.launched


def test_cancelling_queued_and_running_jobs():
    jobs = [FakeJob(0, 40, rounds=5), FakeJob(1, 40, rounds=5), FakeJob(2, 40), FakeJob(3, 40)]
    # round 0: job 2 is still queued (one slot); round 2: job 0 is running
    s, be, _ = run(jobs, budget=100, slots=1, cancel=[(0, 2), (2, 0)])
    assert s.results[2].outcome == "cancelled" and s.results[2].admitted is None
    assert 2 not in be.launched
    assert s.results[0].outcome == "cancelled" and s.results[0].jones is None
    assert 0 in be.released                        # it ran to the end on the device, then was dropped
    assert s.results[1].outcome == s.results[3].outcome == "done"
    assert not s.cancel(99)
