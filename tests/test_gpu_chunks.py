"""Consecutive time chunks warm-started from the previous chunk's solution
(sc_calibrate_chunks) against the oracle's chain, through the C ABI.

Each chunk is a full SAGE calibration, so the tolerances are those of the
calibration itself: final costs within 1e-4 relative and Jones within 1e-4
after removing the unitary ambiguity, chunk by chunk.  Resuming from a
checkpoint must reproduce the uninterrupted run bit for bit: the kernels are
deterministic, and the solution of a chunk is the whole solver state."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402

DEV = "cuda"


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype).contiguous()


def chunked(n, Tc, N=12, F=2, K=2, S=3, seed=51, drift=0.05, sigma=0.01):
    """n chunks of Tc timeslots; the gains drift by a per-station phase of
    up to `drift` radians per chunk; thermal noise of sigma."""
    spec = synth.JobSpec(N=N, T=Tc, F=F, K=K, S=S, f_lo=140e6, f_hi=160e6, seed=seed, sigma=sigma)
    full = dataclasses.replace(spec, T=n * Tc)
    uvw, f, sky = synth.station_uvw(full), synth.freqs(full), synth.sky(full)
    Jt = synth.jones_true(full)
    ph = np.linspace(0.0, 1.0, N)[None, :, None, None]
    noise = synth.noise(full)
    Vs, Css = [], []
    for i in range(n):
        Cs = O.predict_sky(uvw[i * Tc:(i + 1) * Tc], f, sky)
        Ji = Jt * np.exp(1j * drift * i * ph)
        Vs.append(sum(O.model_vis(Cs[k], Ji[k]) for k in range(K)) + noise[i * Tc:(i + 1) * Tc])
        Css.append(Cs)
    return spec, uvw, f, sky, Vs, Css, Jt


def run_chunks(prec, spec, uvw, f, sky, Vs, J0, n_em, n_lm, ws=None):
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.workspace(shp, prec) if ws is None else ws
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    J = tdev(J0, torch.complex128)
    _, hist, costs = sc.calibrate_chunks(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                                         sc.DeviceSky.from_synth(sky), tdev(np.stack(Vs), cdt), J, prec,
                                         ws, n_em=n_em, n_lm=n_lm)
    assert sc.device_status(ws) == 0
    return J, hist, costs, ws


@pytest.mark.parametrize("prec", [sc.SC_FP64, sc.SC_MIXED])
def test_chunks_match_oracle_chain(prec):
    # compared at converged minima (every chunk ends at the noise floor, about
    # 0.21 here), where the 1e-4 tolerance of a calibration applies: start 5%
    # from the truth, as from an earlier solve, with 3 sweeps x 10 LM steps
    n, Tc = 3, 2
    spec, uvw, f, sky, Vs, Css, Jt = chunked(n, Tc)
    J0 = Jt * (1 + 0.05j)
    J_ref, c_ref = O.calibrate_chunks(Vs, Css, J0, n_em=3, n_lm=10)
    assert np.all(c_ref < 0.25)
    J, hist, costs, _ = run_chunks(prec, spec, uvw, f, sky, Vs, J0, n_em=3, n_lm=10)
    h = hist.cpu().numpy()
    np.testing.assert_allclose(costs.cpu().numpy(), c_ref, rtol=1e-4)
    for i in range(n):
        for k in range(spec.K):
            assert O.aligned_error(h[i, k], J_ref[i, k]) <= 1e-4, (i, k)
    assert np.array_equal(J.cpu().numpy(), h[-1])


@pytest.mark.parametrize("prec", [sc.SC_FP64, sc.SC_MIXED])
def test_chunks_resume_from_checkpoint_is_bit_exact(prec):
    n, Tc = 4, 2
    spec, uvw, f, sky, Vs, _, _ = chunked(n, Tc, seed=52)
    J0 = synth.identity_jones(spec.K, spec.N)
    _, h_all, c_all, ws = run_chunks(prec, spec, uvw, f, sky, Vs, J0, n_em=1, n_lm=4)
    _, h_a, c_a, _ = run_chunks(prec, spec, uvw[:2 * Tc], f, sky, Vs[:2], J0, n_em=1, n_lm=4, ws=ws)
    _, h_b, c_b, _ = run_chunks(prec, spec, uvw[2 * Tc:], f, sky, Vs[2:], h_a[-1].cpu().numpy(), n_em=1,
                                n_lm=4, ws=ws)
    assert torch.equal(torch.cat([h_a, h_b]), h_all)
    assert torch.equal(torch.cat([c_a, c_b]), c_all)


def test_warm_start_lowers_the_cost_on_the_gpu():
    # with the same iteration budget a warm-started chunk ends far below a
    # cold start from the identity (slowly drifting, noiseless gains)
    n, Tc = 3, 2
    spec, uvw, f, sky, Vs, _, _ = chunked(n, Tc, seed=53, drift=0.02, sigma=0.0)
    J0 = synth.identity_jones(spec.K, spec.N)
    _, _, c_warm, ws = run_chunks(sc.SC_MIXED, spec, uvw, f, sky, Vs, J0, n_em=1, n_lm=3)
    for i in range(1, n):
        _, _, c_cold, _ = run_chunks(sc.SC_MIXED, spec, uvw[i * Tc:(i + 1) * Tc], f, sky, Vs[i:i + 1], J0,
                                     n_em=1, n_lm=3, ws=ws)
        assert c_warm[i].sum().item() < 0.1 * c_cold[0].sum().item()
