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
