"""Polarised and Gaussian-extended source prediction
(sc_predict_coherencies_full) against the oracle, through the C ABI.

Tolerances: the plain FP64 path to 1e-12 of the scale of the sum and the
mixed path to 1e-5 of it, element by element, where the scale of a channel
is sum_s (f/f0)^alpha_s (|I_s| + |Q_s| + |U_s| + |V_s|), the largest any
entry of a 2x2 coherency can reach.  Shapes: N = 37 and 70 (ragged 32-station
tiles), a cluster of 40 sources (two staged batches of 32, the second
ragged), an empty cluster, N = 2, and a point-only unpolarised sky that
must reproduce sc_predict_coherencies times the identity.  The full-size case
runs the 512-station launch configuration on sampled entries recomputed by
the oracle one baseline at a time.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402

PRECS = [sc.SC_FP64, sc.SC_MIXED]


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def scale(sky, a, b, f):
    amp = np.abs(sky.I[a:b]) + np.abs(sky.Q[a:b]) + np.abs(sky.U[a:b]) + np.abs(sky.V[a:b])
    return (amp[:, None] * (np.asarray(f)[None, :] / sky.f0) ** sky.alpha[a:b, None]).sum(0)


def run(prec, spec, sky):
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    shp = sc.Shape(spec.N, spec.T, spec.F, sky.K, max(1, max(np.diff(sky.offsets))))
    ws = sc.workspace(shp, prec)
    C = sc.predict_coherencies_full(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                                    sc.DeviceSkyFull.from_synth(sky), prec, ws)
    got = C.cpu().numpy().astype(np.complex128)
    assert sc.device_status(ws) == 0
    return uvw, f, got


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,T,F,counts", [(37, 3, 2, [5, 0, 40]), (70, 2, 3, [9, 3]), (2, 1, 1, [4])])
def test_predict_full_matches_oracle(prec, N, T, F, counts):
    spec = synth.JobSpec(N=N, T=T, F=F, K=len(counts), S=max(counts), f_lo=140e6, f_hi=160e6, seed=N,
                         alpha=-0.7)
    sky = synth.sky_pol(spec, sources_per_cluster=counts, frac_extended=0.5, max_circ_pol=0.1)
    uvw, f, got = run(prec, spec, sky)
    ref = O.predict_sky_full(uvw, f, sky)
    assert got.shape == ref.shape
    for k in range(sky.K):
        a, b = int(sky.offsets[k]), int(sky.offsets[k + 1])
        if a == b:
            assert np.all(got[k] == 0)
            continue
        tol = (1e-12 if prec == sc.SC_FP64 else 1e-5) * scale(sky, a, b, f)
        err = np.abs(got[k] - ref[k])
        assert np.all(err <= tol[None, None, :, None, None]), (k, err.max(), tol)


@pytest.mark.parametrize("prec", PRECS)
def test_unpolarised_points_equal_the_scalar_prediction(prec):
    spec = synth.JobSpec(N=37, T=2, F=2, K=2, S=6, f_lo=140e6, f_hi=160e6, seed=4)
    sky = synth.sky_pol(spec, frac_extended=0.0, max_lin_pol=0.0, max_circ_pol=0.0)
    uvw, f, got = run(prec, spec, sky)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.workspace(shp, prec)
    Cs = sc.predict_coherencies(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                                sc.DeviceSky.from_synth(synth.sky(spec)), prec, ws).cpu().numpy()
    assert np.all(got[..., 0, 1] == 0) and np.all(got[..., 1, 0] == 0)
    np.testing.assert_array_equal(got[..., 0, 0], got[..., 1, 1])
    # both paths multiply the same station phasors; the order of the float
    # products differs, so agree to rounding
    tol = (1e-13 if prec == sc.SC_FP64 else 1e-6) * scale(sky, 0, spec.S, f).max()
    assert np.abs(got[..., 0, 0] - Cs).max() <= tol


def test_full_size_predict_full_sampled_against_oracle():
    """512 stations x 10 timeslots x 4 channels, 2 clusters x 100 polarised
    sources, 30% of them Gaussian: 300 sampled (k, t, b, f) entries."""
    spec = synth.config("c4")
    spec.K = 2
    sky = synth.sky_pol(spec)
    uvw, f, got_all = None, None, None
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.workspace(shp, sc.SC_MIXED)
    C = sc.predict_coherencies_full(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                                    sc.DeviceSkyFull.from_synth(sky), sc.SC_MIXED, ws)
    rng = np.random.default_rng(1)
    n = 300
    p = rng.integers(0, spec.N - 1, n)
    q = p + 1 + rng.integers(0, 1 << 30, n) % (spec.N - 1 - p)
    t = rng.integers(0, spec.T, n)
    fi = rng.integers(0, spec.F, n)
    k = rng.integers(0, spec.K, n)
    b = p * spec.N - p * (p + 1) // 2 + (q - p - 1)
    got = C[torch.as_tensor(k), torch.as_tensor(t), torch.as_tensor(b), torch.as_tensor(fi)].cpu().numpy()
    for i in range(n):
        a, e = int(sky.offsets[k[i]]), int(sky.offsets[k[i] + 1])
        c = sky.cluster(k[i])
        ref = O.predict_coherencies_full(uvw[t[i]:t[i] + 1][:, [p[i], q[i]], :], f[fi[i]:fi[i] + 1], c.l, c.m,
                                         c.I, c.Q, c.U, c.V, c.alpha, c.maj, c.mnr, c.pa, c.f0)[0, 0, 0]
        tol = 1e-5 * scale(sky, a, e, f[fi[i]:fi[i] + 1])[0]
        assert np.abs(got[i] - ref).max() <= tol
    assert sc.device_status(ws) == 0
