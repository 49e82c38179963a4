"""Consensus across sub-bands (sc_calibrate_consensus) against the oracle's
consensus ADMM, through the C ABI.

Each J-step is a full SAGE calibration with a penalty, so the tolerances are
those of the calibration: Jones within 1e-4 after removing the unitary
ambiguity and each band's data cost within 1e-4 relative, in both
precisions; for the FP64 path also the final LM costs (penalty included)
within 1e-4 relative and the frequency model and the duals within 1e-4 of
the Jones' scale.  The mixed path's penalised quantities depend on the
bands' relative gauges, which its float32 solves leave free to order
eps32 |g| / mu, so they are not compared.
Sizes: 4 bands of N = 12 and 20 stations (8N = 96 and 160, a ragged last
256-wide block of the consensus kernels), 2 clusters, 2 basis terms; rho = 0
must give independent SAGE per band exactly as sc_calibrate_sage does, and
a basis with too few distinct bands must raise SC_STATUS_BASIS."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def bands(N, n_bands=4, T=2, F=2, K=2, S=3, sigma=0.05, seed=7):
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=S, seed=seed, sigma=sigma)
    fr, centres = synth.sub_bands(spec, n_bands)
    uvw, sky = synth.station_uvw(spec), synth.sky(spec)
    Jt = synth.jones_true_bands(spec, centres)
    Vs, Css = [], []
    for f in range(n_bands):
        Cs = O.predict_sky(uvw, fr[f], sky)
        V = sum(O.model_vis(Cs[k], Jt[f, k]) for k in range(K))
        Vs.append(V + synth.noise(dataclasses.replace(spec, seed=seed * 100 + f)))
        Css.append(Cs)
    return spec, uvw, fr, centres, sky, Vs, Css, Jt


def run_gpu(prec, spec, uvw, fr, sky, Vs, basis, J0, rho, n_admm, n_em, n_lm, concurrent=1):
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.consensus_workspace(shp, prec, concurrent)
    J = tdev(J0, torch.complex128)
    _, U, Z, costs = sc.calibrate_consensus(shp, tdev(uvw, torch.float64), tdev(fr, torch.float64),
                                            sc.DeviceSky.from_synth(sky), tdev(np.stack(Vs), cdt),
                                            tdev(basis, torch.float64), J, prec, ws, rho, n_admm=n_admm,
                                            n_em=n_em, n_lm=n_lm)
    status = sc.device_status(ws)
    return J.cpu().numpy(), U.cpu().numpy(), Z.cpu().numpy(), costs.cpu().numpy(), status


@pytest.mark.parametrize("prec", [sc.SC_FP64, sc.SC_MIXED])
@pytest.mark.parametrize("N", [12, 20])
def test_consensus_matches_oracle(prec, N):
    spec, uvw, fr, centres, sky, Vs, Css, Jt = bands(N)
    basis = synth.frequency_basis(centres, 2)
    J0 = np.stack([synth.identity_jones(spec.K, spec.N)] * len(Vs))
    rho, n_admm, n_em, n_lm = 30.0, 3, 1, 6
    J_ref, Z_ref, U_ref, c_ref = O.consensus_calibrate(Vs, Css, J0, basis, rho, n_admm, n_em, n_lm)
    J, U, Z, costs, status = run_gpu(prec, spec, uvw, fr, sky, Vs, basis, J0, rho, n_admm, n_em, n_lm)
    assert status == 0
    for f in range(len(Vs)):
        for k in range(spec.K):
            assert O.aligned_error(J[f, k], J_ref[f, k]) <= 1e-4
        # the data cost of each band is invariant to the unitary gauge
        _, c_gpu, _ = O.residual_all(Vs[f], Css[f], J[f])
        _, c_orc, _ = O.residual_all(Vs[f], Css[f], J_ref[f])
        assert abs(c_gpu - c_orc) <= 1e-4 * c_orc
    # the duals stay orthogonal to the model, as in the oracle
    assert np.abs(np.einsum("fp,fknij->pknij", basis, U)).max() <= 1e-10 * np.abs(J).max()
    if prec == sc.SC_MIXED:
        # The float32 solves leave a component along the gauge directions
        # (the null space of the data term, where the gradient has none) of
        # order eps32 |g| / mu, which the first, unpenalised iteration keeps.
        # The penalty, the frequency model and the duals depend on the bands'
        # relative gauges, so only gauge-invariant quantities are compared
        # for this path.
        return
    np.testing.assert_allclose(costs, c_ref, rtol=1e-4)
    M, M_ref = O.consensus_model(Z, basis), O.consensus_model(Z_ref, basis)
    np.testing.assert_allclose(M, M_ref, rtol=0, atol=1e-4 * np.abs(M_ref).max())
    np.testing.assert_allclose(U, U_ref, rtol=0, atol=1e-4 * np.abs(J_ref).max())


def test_zero_rho_is_sage_per_band():
    prec = sc.SC_MIXED
    spec, uvw, fr, centres, sky, Vs, Css, Jt = bands(12, n_bands=3)
    basis = synth.frequency_basis(centres, 2)
    J0 = np.stack([synth.identity_jones(spec.K, spec.N)] * len(Vs))
    J, U, Z, costs, status = run_gpu(prec, spec, uvw, fr, sky, Vs, basis, J0, 0.0, 2, 1, 5)
    assert status == 0
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    for f in range(len(Vs)):
        ws = sc.workspace(shp, prec)
        Jf = tdev(J0[f], torch.complex128)
        _, cf = sc.calibrate_sage(shp, tdev(uvw, torch.float64), tdev(fr[f], torch.float64),
                                  sc.DeviceSky.from_synth(sky), tdev(Vs[f], torch.complex64), Jf, prec, ws,
                                  n_em=1, n_lm=5)
        # two independent sweeps, as two ADMM iterations with no penalty
        sc.calibrate_sage(shp, tdev(uvw, torch.float64), tdev(fr[f], torch.float64),
                          sc.DeviceSky.from_synth(sky), tdev(Vs[f], torch.complex64), Jf, prec, ws,
                          n_em=1, n_lm=5, costs=cf)
        np.testing.assert_array_equal(J[f], Jf.cpu().numpy())
        np.testing.assert_array_equal(costs[f], cf.cpu().numpy())


def test_singular_basis_is_flagged():
    spec, uvw, fr, centres, sky, Vs, Css, Jt = bands(12, n_bands=3)
    basis = np.ones((3, 2))                          # two identical columns
    J0 = np.stack([synth.identity_jones(spec.K, spec.N)] * len(Vs))
    J, U, Z, costs, status = run_gpu(sc.SC_MIXED, spec, uvw, fr, sky, Vs, basis, J0, 10.0, 2, 1, 3)
    assert status & sc.SC_STATUS_BASIS
    assert np.all(Z == 0)


@pytest.mark.parametrize("prec", [sc.SC_FP64, sc.SC_MIXED])
def test_concurrent_bands_equal_sequential_bands(prec):
    """A workspace for four bands runs the four J-steps at once on internal
    streams; every output equals the sequential run's bit for bit (each
    band's kernels are deterministic and see the same inputs)."""
    spec, uvw, fr, centres, sky, Vs, Css, Jt = bands(20)
    basis = synth.frequency_basis(centres, 2)
    J0 = np.broadcast_to(np.eye(2, dtype=complex), (4, spec.K, spec.N, 2, 2)).copy()
    seq = run_gpu(prec, spec, uvw, fr, sky, Vs, basis, J0, 5.0, 2, 1, 4, concurrent=1)
    par = run_gpu(prec, spec, uvw, fr, sky, Vs, basis, J0, 5.0, 2, 1, 4, concurrent=4)
    for a, b in zip(seq[:4], par[:4]):
        assert np.array_equal(a, b)
    assert seq[4] == par[4] == 0
