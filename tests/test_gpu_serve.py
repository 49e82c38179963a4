"""Serving: jobs arriving while others run are admitted as slots and memory
free up, overlap on the GPU, and each result equals the job calibrated
alone."""
import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc, serve  # noqa: E402


def host_job(i, N, T, F, K, S):
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=S, f_lo=140e6, f_hi=160e6, seed=100 + i)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Jt = synth.jones_true(spec)
    Cs = O.predict_sky(uvw, f, sky)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(K)) + synth.noise(spec)
    return serve.HostJob(i, sc.Shape(N, T, F, K, S), uvw, f, sky.l, sky.m, sky.flux, sky.alpha,
                         list(sky.offsets), V.astype(np.complex64), synth.identity_jones(K, N))


SHAPES = [(40, 3, 2, 2, 4), (64, 2, 1, 3, 3), (24, 5, 2, 1, 5), (70, 2, 2, 2, 3), (33, 4, 1, 3, 2),
          (50, 3, 3, 1, 4)]


def test_each_result_is_the_same_alone_and_in_the_mix():
    jobs = [host_job(i, *s) for i, s in enumerate(SHAPES)]
    # alone: one server slot, jobs one after the other
    alone = serve.Server(max_slots=1, n_em=2, n_lm=5)
    alone.start()
    for j in jobs:
        alone.submit(j)
        alone.drain()
    # the mix: Poisson arrivals into 3 slots under a budget that forces queueing
    fps = [serve.footprint(sc.Shape(j.shape.N, j.shape.T, j.shape.F, j.shape.K, j.shape.S_max), sc.SC_MIXED)
           for j in jobs]
    mix = serve.Server(max_slots=3, n_em=2, n_lm=5, mem_budget=2 * max(fps))
    stats = serve.run_poisson(mix, [host_job(i, *s) for i, s in enumerate(SHAPES)], rate_hz=200.0)
    assert stats["jobs"] == len(jobs)
    assert mix.max_used <= 2 * max(fps)
    for i in range(len(jobs)):
        a, b = alone.results[i], mix.results[i]
        assert a.status & 2 == 0 and b.status & 2 == 0
        np.testing.assert_array_equal(a.jones, b.jones)
        np.testing.assert_array_equal(a.costs, b.costs)
    assert stats["p99_s"] >= stats["p50_s"] > 0
    alone.close()
    mix.close()


def test_served_result_matches_the_oracle():
    j = host_job(7, 30, 3, 2, 2, 4)
    srv = serve.Server(max_slots=2, n_em=2, n_lm=6)
    srv.start()
    srv.submit(j)
    srv.drain()
    r = srv.results[7]
    spec = synth.JobSpec(N=30, T=3, F=2, K=2, S=4, f_lo=140e6, f_hi=160e6, seed=107)
    Cs = O.predict_sky(synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec))
    J_ref, c_ref = O.sage_calibrate(j.V.astype(np.complex128), Cs, j.jones0, n_em=2, n_lm=6)
    np.testing.assert_allclose(r.costs, c_ref, rtol=1e-4)
    for k in range(2):
        assert O.aligned_error(r.jones[k], J_ref[k]) <= 1e-4
    srv.close()
