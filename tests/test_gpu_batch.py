"""Batched calibration: uneven jobs overlapping on one GPU give, job by job,
exactly the result of calibrating each job alone."""
import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402


def build_job(N, T, F, K, S, seed, prec):
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=S, f_lo=140e6, f_hi=160e6, seed=seed)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Jt = synth.jones_true(spec)
    Cs = O.predict_sky(uvw, f, sky)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(K)) + synth.noise(spec)
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    shp = sc.Shape(N, T, F, K, S)
    return sc.Job(shape=shp, uvw=torch.as_tensor(uvw).cuda(), freqs=torch.as_tensor(f).cuda(),
                  sky=sc.DeviceSky.from_synth(sky), V=torch.as_tensor(V).to("cuda", cdt).contiguous(),
                  jones=torch.as_tensor(synth.identity_jones(K, N)).cuda(),
                  costs=torch.zeros(K, dtype=torch.float64, device="cuda"),
                  ws=sc.workspace(shp, prec), stream=torch.cuda.Stream())


@pytest.mark.parametrize("prec", [sc.SC_MIXED, sc.SC_FP64])
def test_batch_equals_jobs_alone(prec):
    shapes = [(37, 3, 2, 2, 5, 1), (70, 5, 1, 3, 4, 2), (20, 7, 3, 1, 6, 3), (64, 2, 2, 2, 3, 4)]
    batch = [build_job(*s, prec) for s in shapes]
    alone = [build_job(*s, prec) for s in shapes]
    sc.calibrate_batch(batch, prec, n_em=2, n_lm=5)
    torch.cuda.synchronize()
    for j in alone:
        sc.calibrate_sage(j.shape, j.uvw, j.freqs, j.sky, j.V, j.jones, prec, j.ws, n_em=2, n_lm=5,
                          costs=j.costs)
    torch.cuda.synchronize()
    for a, b in zip(batch, alone):
        assert torch.equal(a.jones, b.jones)
        assert torch.equal(a.costs, b.costs)
        assert sc.device_status(a.ws) & 2 == 0


def test_batch_rejects_a_bad_job_and_still_runs_the_rest():
    good = build_job(20, 2, 1, 1, 3, 5, sc.SC_MIXED)
    bad = build_job(20, 2, 1, 1, 3, 6, sc.SC_MIXED)
    bad.ws = bad.ws[:1024]                       # workspace far too small
    ref = build_job(20, 2, 1, 1, 3, 5, sc.SC_MIXED)
    with pytest.raises(sc.ScError) as e:
        sc.calibrate_batch([bad, good], sc.SC_MIXED, n_em=1, n_lm=3)
    assert e.value.code == -2 and "job 0" in str(e.value)
    torch.cuda.synchronize()
    sc.calibrate_sage(ref.shape, ref.uvw, ref.freqs, ref.sky, ref.V, ref.jones, sc.SC_MIXED, ref.ws, n_em=1,
                      n_lm=3, costs=ref.costs)
    torch.cuda.synchronize()
    assert torch.equal(good.jones, ref.jones)


# Lock-step batches (sc_calibrate_batched): equal N and K, anything else
# uneven.  70 stations give 9 tile rows with a ragged last one; the jobs
# differ in timeslots, channels and sources, so their statistics passes and
# chunk counts differ while their LM stages share every launch.
LOCKSTEP = [(70, 3, 2, 2, 5, 11), (70, 5, 1, 2, 4, 12), (70, 7, 3, 2, 6, 13), (70, 2, 2, 2, 3, 14),
            (70, 1, 1, 2, 2, 15)]


@pytest.mark.parametrize("prec", [sc.SC_MIXED, sc.SC_FP64])
def test_lockstep_batch_equals_jobs_alone(prec):
    batch = [build_job(*s, prec) for s in LOCKSTEP]
    alone = [build_job(*s, prec) for s in LOCKSTEP]
    ws = sc.batched_workspace(batch, prec)
    sc.calibrate_batched(batch, prec, ws, n_em=2, n_lm=5)
    torch.cuda.synchronize()
    for j in alone:
        sc.calibrate_sage(j.shape, j.uvw, j.freqs, j.sky, j.V, j.jones, prec, j.ws, n_em=2, n_lm=5,
                          costs=j.costs)
    torch.cuda.synchronize()
    for a, b in zip(batch, alone):
        assert torch.equal(a.jones, b.jones)
        assert torch.equal(a.costs, b.costs)
        assert sc.device_status(a.ws) == 0


def test_lockstep_batch_of_one_and_of_many_factor_rows():
    """One job alone in a batch, and 4 jobs of 130 stations (17 tile rows,
    every kind of factorisation task many times over), bit for bit."""
    for shapes in ([(70, 4, 2, 3, 5, 21)], [(130, 3, 1, 2, 4, 22 + i) for i in range(4)]):
        batch = [build_job(*s, sc.SC_MIXED) for s in shapes]
        alone = [build_job(*s, sc.SC_MIXED) for s in shapes]
        ws = sc.batched_workspace(batch, sc.SC_MIXED)
        sc.calibrate_batched(batch, sc.SC_MIXED, ws, n_em=1, n_lm=4)
        for j in alone:
            sc.calibrate_sage(j.shape, j.uvw, j.freqs, j.sky, j.V, j.jones, sc.SC_MIXED, j.ws, n_em=1, n_lm=4,
                              costs=j.costs)
        torch.cuda.synchronize()
        for a, b in zip(batch, alone):
            assert torch.equal(a.jones, b.jones)
            assert torch.equal(a.costs, b.costs)


def test_lockstep_batch_refuses_unequal_station_or_cluster_counts():
    a = build_job(40, 2, 1, 2, 3, 31, sc.SC_MIXED)
    for other in (build_job(41, 2, 1, 2, 3, 32, sc.SC_MIXED), build_job(40, 2, 1, 3, 3, 33, sc.SC_MIXED)):
        with pytest.raises(sc.ScError) as e:
            sc.batched_workspace([a, other], sc.SC_MIXED)
        assert e.value.code == -1 and "job 1" in str(e.value)


@pytest.mark.parametrize("window", [1, 2, 3, 8])
def test_lockstep_batch_result_does_not_depend_on_the_window(window):
    """The staggered factorisation order changes only when each tile is
    computed, not how: every window gives each job its alone result."""
    shapes = [(130, 2, 1, 2, 4, 40 + i) for i in range(4)]
    batch = [build_job(*s, sc.SC_MIXED) for s in shapes]
    alone = [build_job(*s, sc.SC_MIXED) for s in shapes]
    ws = sc.batched_workspace(batch, sc.SC_MIXED)
    sc.calibrate_batched(batch, sc.SC_MIXED, ws, n_em=1, n_lm=3, window=window)
    for j in alone:
        sc.calibrate_sage(j.shape, j.uvw, j.freqs, j.sky, j.V, j.jones, sc.SC_MIXED, j.ws, n_em=1, n_lm=3,
                          costs=j.costs)
    torch.cuda.synchronize()
    for a, b in zip(batch, alone):
        assert torch.equal(a.jones, b.jones)
        assert torch.equal(a.costs, b.costs)
        assert sc.device_status(a.ws) == 0


def test_tuner_times_every_window_and_returns_the_fastest():
    jobs = [build_job(130, 2, 1, 2, 4, 50 + i, sc.SC_MIXED) for i in range(3)]
    ws = sc.batched_workspace(jobs, sc.SC_MIXED)
    best, ms = sc.tune_batched(jobs, sc.SC_MIXED, ws, windows=(1, 2, 3, 16), reps=2)
    assert set(ms) == {1, 2, 3, 16}
    assert all(v > 0 for v in ms.values())
    assert best == min(ms, key=ms.get)
    # the tuner leaves nothing behind that a calibration would see
    alone = build_job(130, 2, 1, 2, 4, 50, sc.SC_MIXED)
    sc.calibrate_batched(jobs, sc.SC_MIXED, ws, n_em=1, n_lm=3, window=best)
    sc.calibrate_sage(alone.shape, alone.uvw, alone.freqs, alone.sky, alone.V, alone.jones, sc.SC_MIXED, alone.ws,
                      n_em=1, n_lm=3, costs=alone.costs)
    torch.cuda.synchronize()
    assert torch.equal(jobs[0].jones, alone.jones)
