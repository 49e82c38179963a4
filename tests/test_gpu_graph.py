"""A SAGE calibration captured once as a CUDA graph (sc_graph_capture_sage)
and replayed: every replay computes exactly what sc_calibrate_sage computes
on the buffers' current contents.

The kernels are deterministic and a replay runs the same kernels in the same
order, so replays are compared with direct calls bit for bit, on two
replays in a row with different data written into the captured buffers in
between (a replay that reused stale state from the capture or from the
previous replay would differ).  A capture that fails on a bad argument must
leave nothing behind: the stream is usable and the next capture works."""
import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402


def data(N, T, F, K, S, seed, prec):
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=S, f_lo=140e6, f_hi=160e6, seed=seed)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Jt = synth.jones_true(spec)
    Cs = O.predict_sky(uvw, f, sky)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(K)) + synth.noise(spec)
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    return (sc.Shape(N, T, F, K, S), torch.as_tensor(uvw).cuda(), torch.as_tensor(f).cuda(),
            sc.DeviceSky.from_synth(sky), torch.as_tensor(V).to("cuda", cdt).contiguous())


def direct(shp, uvw, f, sky, V, prec, n_em, n_lm):
    J = torch.as_tensor(synth.identity_jones(shp.K, shp.N)).cuda()
    costs = torch.zeros(shp.K, dtype=torch.float64, device="cuda")
    ws = sc.workspace(shp, prec)
    sc.calibrate_sage(shp, uvw, f, sky, V, J, prec, ws, n_em=n_em, n_lm=n_lm, costs=costs)
    torch.cuda.synchronize()
    assert sc.device_status(ws) == 0
    return J, costs


@pytest.mark.parametrize("prec", [sc.SC_MIXED, sc.SC_FP64])
def test_graph_replays_equal_direct_calls(prec):
    n_em, n_lm = 2, 5
    # two data sets of one shape and sky layout (the sky values differ too)
    a = data(37, 3, 2, 3, 4, 11, prec)
    b = data(37, 3, 2, 3, 4, 12, prec)
    shp, uvw, f, sky, V = a
    J0 = torch.as_tensor(synth.identity_jones(shp.K, shp.N)).cuda()
    J = J0.clone()
    costs = torch.zeros(shp.K, dtype=torch.float64, device="cuda")
    ws = sc.workspace(shp, prec)
    n0 = sc.launch_count()
    g = sc.capture_sage(shp, uvw, f, sky, V, J, prec, ws, costs, n_em=n_em, n_lm=n_lm)
    torch.cuda.synchronize()
    assert torch.equal(J, J0)                        # the capture itself runs nothing
    kernels = sc.launch_count() - n0
    for src in (a, b):
        _, uvw_s, f_s, sky_s, V_s = src
        uvw.copy_(uvw_s)
        f.copy_(f_s)
        for t in ("l", "m", "flux", "alpha"):
            getattr(sky, t).copy_(getattr(sky_s, t))
        V.copy_(V_s)
        J.copy_(J0)
        m0 = sc.launch_count()
        g.launch()
        torch.cuda.synchronize()
        assert sc.launch_count() - m0 == kernels
        assert sc.device_status(ws) == 0
        J_ref, c_ref = direct(*src, prec, n_em, n_lm)
        assert torch.equal(J, J_ref)
        assert torch.equal(costs, c_ref)
    g.close()


def test_failed_capture_leaves_the_stream_usable():
    prec = sc.SC_MIXED
    shp, uvw, f, sky, V = data(20, 2, 1, 2, 3, 21, prec)
    J = torch.as_tensor(synth.identity_jones(shp.K, shp.N)).cuda()
    costs = torch.zeros(shp.K, dtype=torch.float64, device="cuda")
    ws = sc.workspace(shp, prec)
    with pytest.raises(sc.ScError) as e:               # n_lm < 0 is refused inside the capture
        sc.capture_sage(shp, uvw, f, sky, V, J, prec, ws, costs, n_lm=-1)
    assert e.value.code == -1
    with pytest.raises(sc.ScError) as e:               # workspace too small
        sc.capture_sage(shp, uvw, f, sky, V, J, prec, ws[:4096], costs)
    assert e.value.code == -2
    g = sc.capture_sage(shp, uvw, f, sky, V, J, prec, ws, costs, n_em=1, n_lm=3)
    g.launch()
    torch.cuda.synchronize()
    J_ref, c_ref = direct(shp, uvw, f, sky, V, prec, 1, 3)
    assert torch.equal(J, J_ref) and torch.equal(costs, c_ref)
    assert np.isfinite(costs.cpu().numpy()).all()
    g.close()
    with pytest.raises(RuntimeError):
        g.launch()
