"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (from the arithmetic of each path):
* coherencies: FP64 path 1e-12 relative; mixed path 1e-5 relative, measured
  element-wise against the cluster's flux scale sum_s S_s(f) (the bound on
  |C|) and norm-wise against |C|;
* residual, J^T J: FP64 1e-11; mixed 1e-5 of the array's largest
  magnitude (float32 data, float32 accumulation over T*F terms);
* J^T r: FP64 1e-11 of its largest magnitude; mixed 1e-5 of the magnitudes
  it sums per station (its float32 per-baseline sums round relative to
  those; the sum over stations can cancel far below them);
* final LM/SAGE cost within 1e-4 relative and Jones within 1e-4 after
  removing the unitary ambiguity (Procrustes), for both paths.
Sizes span several 64-wide tiles with ragged tails (N = 37, 70: 8N = 296,
560), odd T and F, a cluster without sources and N = 2; the LM solve is also
compared at the 512-station workload's factorisation order (8N = 4096) and
at a ragged 8N = 2408.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402

PRECS = [sc.SC_FP64, sc.SC_MIXED]
DEV = "cuda"


def cdt(prec):
    return torch.complex64 if prec == sc.SC_MIXED else torch.complex128


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype).contiguous()


def make_job(N=37, T=3, F=2, K=3, S=7, seed=21, sigma=0.01, counts=None, alpha=-0.7):
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=S, f_lo=140e6, f_hi=160e6, alpha=alpha,
                         seed=seed, sigma=sigma)
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    sky = synth.sky(spec, counts)
    Jt = synth.jones_true(spec)
    Cs = O.predict_sky(uvw, f, sky)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(K))
    if sigma > 0:
        V = V + synth.noise(spec)
    return spec, uvw, f, sky, Jt, Cs, V


def shape_of(spec, sky):
    return sc.Shape(spec.N, spec.T, spec.F, spec.K, int(np.max(np.diff(sky.offsets))))


# --- (a) coherencies ----------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,T,F", [(37, 3, 2), (70, 2, 3), (2, 1, 1)])
def test_predict_matches_oracle(prec, N, T, F):
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=N, T=T, F=F, K=3, S=7, counts=[7, 0, 1])
    # the 1-source cluster sits at the phase centre: C = its flux exactly
    sky.l[7] = 0.0
    sky.m[7] = 0.0
    Cs = O.predict_sky(uvw, f, sky)
    shp = shape_of(spec, sky)
    ws = sc.workspace(shp, prec)
    C = sc.predict_coherencies(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                               sc.DeviceSky.from_synth(sky), prec, ws)
    got = C.cpu().numpy().astype(np.complex128)
    assert got.shape == Cs.shape
    assert np.all(got[1] == 0)
    scale0 = (sky.flux[:7][:, None] * (f[None, :] / sky.f0) ** sky.alpha[:7][:, None]).sum(0)
    if prec == sc.SC_FP64:
        np.testing.assert_allclose(got, Cs, rtol=0, atol=1e-12 * scale0.max())
        np.testing.assert_allclose(got[2], Cs[2], rtol=1e-14)
    else:
        err = np.abs(got[0] - Cs[0])
        assert np.all(err <= 1e-5 * scale0[None, None, :])
        assert np.linalg.norm(got[0] - Cs[0]) <= 1e-5 * np.linalg.norm(Cs[0])
        np.testing.assert_allclose(got[2], Cs[2], rtol=2e-7)
    assert sc.device_status(ws) == 0


# --- (b) residual -----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_residual_matches_oracle(prec):
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=37, T=3, F=2, K=2)
    J = Jt[0] * (1 + 0.01j)
    R_ref, cost_ref = O.residual(V, Cs[0], J)
    shp = sc.Shape(spec.N, spec.T, spec.F, 1, 7)
    ws = sc.workspace(shp, prec)
    X = tdev(V, cdt(prec))
    R, cost = sc.residual(shp, X, tdev(Cs[0], cdt(prec)), tdev(J, torch.complex128), prec, ws)
    got = R.cpu().numpy()
    tol = 1e-11 if prec == sc.SC_FP64 else 1e-5
    assert np.max(np.abs(got - R_ref)) <= tol * np.max(np.abs(V))
    assert abs(cost.item() - cost_ref) <= (1e-11 if prec == sc.SC_FP64 else 1e-5) * cost_ref
    # in place
    R2, _ = sc.residual(shp, X, tdev(Cs[0], cdt(prec)), tdev(J, torch.complex128), prec, ws, out=X,
                        want_cost=False)
    assert torch.equal(R2, R)


# --- (c) normal equations ---------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [37, 9])
def test_normal_equations_match_oracle(prec, N):
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=N, T=3, F=2, K=1)
    J = Jt[0] + 0.05
    R_ref, _ = O.residual(V, Cs[0], J)
    A_ref, g_ref = O.normal_equations(R_ref, Cs[0], J)
    shp = sc.Shape(spec.N, spec.T, spec.F, 1, 7)
    ws = sc.workspace(shp, prec)
    A, g = sc.lm_normal_eqs(shp, tdev(R_ref, cdt(prec)), tdev(Cs[0], cdt(prec)),
                            tdev(J, torch.complex128), prec, ws)
    A, g = A.cpu().numpy().astype(np.float64), g.cpu().numpy()
    tol = 1e-11 if prec == sc.SC_FP64 else 1e-5
    assert np.max(np.abs(A - A_ref)) <= tol * np.max(np.abs(A_ref))
    if prec == sc.SC_FP64:
        assert np.max(np.abs(g - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))
    else:
        # Each entry of g_s sums, over the other stations o, float32 sums over
        # (t, f) of conj(c) r multiplied by J_o.  Their rounding error is
        # relative to the magnitudes summed, bounded per station by
        # S_s = sum_o sum_tf |c| |r|_F |J_o|_F (about (T F + 2) eps_32 S_s);
        # cancellation between stations can leave |g| itself far below S_s.
        p, q = O.baselines(N)
        mag = (np.abs(Cs[0]) * np.linalg.norm(R_ref, axis=(-2, -1))).sum(axis=(0, 2))    # [B]
        jn = np.linalg.norm(J, axis=(1, 2))                                                # [N]
        S = np.zeros(N)
        np.add.at(S, p, mag * jn[q])
        np.add.at(S, q, mag * jn[p])
        assert np.all(np.abs(g - g_ref) <= 1e-5 * np.repeat(S, 8))


# --- (c) LM solve of one cluster ----------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [37, 70])
def test_solve_cluster_matches_oracle(prec, N):
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=N, T=3, F=2, K=1, S=9, seed=5)
    J0 = np.tile(np.eye(2, dtype=complex), (spec.N, 1, 1))
    shp = sc.Shape(spec.N, spec.T, spec.F, 1, 9)
    ws = sc.workspace(shp, prec)
    # the early gradient stop is an integer decided by rounding-level values
    # near the minimum, so it is compared only as a bound; with the stop
    # disabled both sides take exactly n_lm steps
    for eps in (1e-12, 0.0):
        J_ref, cost_ref, it_ref = O.lm_cluster(V, Cs[0], J0, 10, eps_grad=eps)
        Jg = tdev(J0, torch.complex128)
        _, cost, iters = sc.solve_cluster(shp, tdev(V, cdt(prec)), tdev(Cs[0], cdt(prec)), Jg, prec, ws,
                                          n_lm=10, refine_sweeps=2, eps_grad=eps)
        Jn = Jg.cpu().numpy()
        if eps == 0.0:
            assert iters.item() == it_ref == 10
        else:
            assert 1 <= iters.item() <= 10
        assert abs(cost.item() - cost_ref) <= 1e-4 * cost_ref
        assert O.aligned_error(Jn, J_ref) <= 1e-4
        assert sc.device_status(ws) & 2 == 0


@functools.lru_cache(maxsize=None)
def _full_order_case(N, n_lm):
    """One cluster of 100 sources on N stations, one timeslot and one channel
    (the oracle's cost grows with the data, the factorisation's order 8N does
    not), solved by the oracle from identity Jones with the gradient stop off."""
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=N, T=1, F=1, K=1, S=100, seed=5)
    J0 = np.tile(np.eye(2, dtype=complex), (N, 1, 1))
    J_ref, cost_ref, it_ref = O.lm_cluster(V, Cs[0], J0, n_lm, eps_grad=0.0)
    return spec, Cs, V, J0, J_ref, cost_ref, it_ref


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,n_lm", [(512, 3), (301, 2)])
def test_solve_cluster_full_order_matches_oracle(prec, N, n_lm):
    """The LM solve at the factorisation order of the 512-station workload
    (8N = 4096: 64 tile rows, the walker on the diagonal chain, the two-deep
    bulk prefetch and the tagged-word solves across 64 block rows) and at a
    ragged order (8N = 2408, padded to 2432 = 38 tile rows), against the
    oracle: final cost within 1e-4 relative, Jones within 1e-4 after the
    unitary alignment, the same number of LM steps.  With n_lm = 2 the
    solution is still 1% above the minimum's cost, so both steps count."""
    spec, Cs, V, J0, J_ref, cost_ref, it_ref = _full_order_case(N, n_lm)
    shp = sc.Shape(N, 1, 1, 1, 100)
    ws = sc.workspace(shp, prec)
    Jg = tdev(J0, torch.complex128)
    _, cost, iters = sc.solve_cluster(shp, tdev(V, cdt(prec)), tdev(Cs[0], cdt(prec)), Jg, prec, ws,
                                      n_lm=n_lm, refine_sweeps=2, eps_grad=0.0)
    assert iters.item() == it_ref == n_lm
    assert abs(cost.item() - cost_ref) <= 1e-4 * cost_ref
    assert O.aligned_error(Jg.cpu().numpy(), J_ref) <= 1e-4
    assert sc.device_status(ws) == 0


def test_solve_cluster_full_order_tensor_core_factorisation_matches_oracle():
    """The mixed-precision LM solve at order 4096 with the tensor-core
    factorisation kernel (three TF32 passes per tile product, then one more
    float64 refinement sweep than the float32 kernel needs): the same
    oracle tolerances as above."""
    spec, Cs, V, J0, J_ref, cost_ref, it_ref = _full_order_case(512, 3)
    shp = sc.Shape(512, 1, 1, 1, 100)
    ws = sc.workspace(shp, sc.SC_MIXED)
    Jg = tdev(J0, torch.complex128)
    _, cost, iters = sc.solve_cluster(shp, tdev(V, torch.complex64), tdev(Cs[0], torch.complex64), Jg, sc.SC_MIXED,
                                      ws, n_lm=3, refine_sweeps=2, eps_grad=0.0, chol_kernel=sc.SC_CHOL_TENSOR)
    assert iters.item() == it_ref == 3
    assert abs(cost.item() - cost_ref) <= 1e-4 * cost_ref
    assert O.aligned_error(Jg.cpu().numpy(), J_ref) <= 1e-4
    assert sc.device_status(ws) == 0


# --- the whole path ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_sage_matches_oracle(prec):
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=37, T=3, F=2, K=3, S=7, seed=8)
    J0 = synth.identity_jones(spec.K, spec.N)
    J_ref, costs_ref = O.sage_calibrate(V, Cs, J0, n_em=2, n_lm=6)
    shp = shape_of(spec, sky)
    ws = sc.workspace(shp, prec)
    Jg = tdev(J0, torch.complex128)
    _, costs = sc.calibrate_sage(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                                 sc.DeviceSky.from_synth(sky), tdev(V, cdt(prec)), Jg, prec, ws,
                                 n_em=2, n_lm=6)
    Jn = Jg.cpu().numpy()
    np.testing.assert_allclose(costs.cpu().numpy(), costs_ref, rtol=1e-4)
    for k in range(spec.K):
        assert O.aligned_error(Jn[k], J_ref[k]) <= 1e-4
    assert sc.device_status(ws) & 2 == 0


def test_mixed_noiseless_recovers_truth():
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=37, T=4, F=2, K=1, S=6, seed=31, sigma=0.0)
    shp = sc.Shape(spec.N, spec.T, spec.F, 1, 6)
    ws = sc.workspace(shp, sc.SC_MIXED)
    Jg = tdev(np.tile(np.eye(2, dtype=complex), (spec.N, 1, 1)), torch.complex128)
    _, cost, _ = sc.solve_cluster(shp, tdev(V, torch.complex64), tdev(Cs[0], torch.complex64), Jg,
                                  sc.SC_MIXED, ws, n_lm=20)
    assert O.aligned_error(Jg.cpu().numpy(), Jt[0]) <= 1e-4
    assert cost.item() <= 1e-9 * float(np.sum(np.abs(V) ** 2))


def test_two_stations_and_zero_source_cluster():
    """N = 2 (one baseline, 16 parameters padded to one tile) and a cluster
    with no sources (its J^T J and gradient vanish: the solve stops at once,
    as in the oracle)."""
    spec, uvw, f, sky, Jt, Cs, V = make_job(N=2, T=2, F=1, K=2, S=3, counts=[3, 0], seed=2)
    J0 = synth.identity_jones(2, 2)
    J_ref, costs_ref = O.sage_calibrate(V, Cs, J0, n_em=1, n_lm=4)
    for prec in PRECS:
        shp = shape_of(spec, sky)
        ws = sc.workspace(shp, prec)
        Jg = tdev(J0, torch.complex128)
        _, costs = sc.calibrate_sage(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                                     sc.DeviceSky.from_synth(sky), tdev(V, cdt(prec)), Jg, prec, ws,
                                     n_em=1, n_lm=4)
        np.testing.assert_allclose(costs.cpu().numpy(), costs_ref, rtol=1e-4)
        assert np.array_equal(Jg.cpu().numpy()[1], J0[1])


# --- full-size workloads, sampled against the oracle -----------------------------------------------

def test_full_size_predict_sampled_against_oracle():
    """512 stations x 10 timeslots x 4 channels, 100 sources: the launch
    configuration of the benchmark; 300 random (t, b, f) entries recomputed by
    the oracle one baseline at a time."""
    spec = synth.config("c4")
    spec.K = 2
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.workspace(shp, sc.SC_MIXED)
    C = sc.predict_coherencies(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                               sc.DeviceSky.from_synth(sky), sc.SC_MIXED, ws)
    rng = np.random.default_rng(0)
    p = rng.integers(0, spec.N - 1, 300)
    q = p + 1 + rng.integers(0, 1 << 30, 300) % (spec.N - 1 - p)
    t = rng.integers(0, spec.T, 300)
    fi = rng.integers(0, spec.F, 300)
    k = rng.integers(0, spec.K, 300)
    b = p * spec.N - p * (p + 1) // 2 + (q - p - 1)
    got = C[torch.as_tensor(k), torch.as_tensor(t), torch.as_tensor(b), torch.as_tensor(fi)].cpu().numpy()
    for n in range(300):
        a, e = sky.offsets[k[n]], sky.offsets[k[n] + 1]
        ref = O.predict_coherencies(uvw[t[n]:t[n] + 1][:, [p[n], q[n]], :], f[fi[n]:fi[n] + 1],
                                    sky.l[a:e], sky.m[a:e], sky.flux[a:e], sky.alpha[a:e])[0, 0, 0]
        scale = sky.flux[a:e].sum()
        assert abs(got[n] - ref) <= 1e-5 * scale


def test_full_size_precision_path_matches_fp64_path():
    """128 stations, 20 timeslots, 8 channels, 10 clusters x 25 sources
    (the precision-path workload): the mixed path's final costs and Jones agree
    with the plain FP64 GPU path (itself pinned to the oracle above)."""
    spec = synth.config("c2")
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Jt = synth.jones_true(spec)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    dsky = sc.DeviceSky.from_synth(sky)
    u, fr = tdev(uvw, torch.float64), tdev(f, torch.float64)
    ws64 = sc.workspace(shp, sc.SC_FP64)
    C = sc.predict_coherencies(shp, u, fr, dsky, sc.SC_FP64, ws64)
    Jtd = tdev(Jt, torch.complex128)
    p, q = np.triu_indices(spec.N, 1)
    G = Jtd[:, p] @ Jtd[:, q].conj().transpose(-1, -2)                     # [K][B][2][2]
    V = torch.einsum("ktbf,kbij->tbfij", C, G)
    V = V + tdev(synth.noise(spec), torch.complex128)
    res = {}
    for prec in PRECS:
        ws = ws64 if prec == sc.SC_FP64 else sc.workspace(shp, prec)
        Jg = tdev(synth.identity_jones(spec.K, spec.N), torch.complex128)
        _, costs = sc.calibrate_sage(shp, u, fr, dsky, V.to(cdt(prec)).contiguous(), Jg, prec, ws,
                                     n_em=3, n_lm=10)
        res[prec] = (costs.cpu().numpy(), Jg.cpu().numpy())
    c64, J64 = res[sc.SC_FP64]
    c32, J32 = res[sc.SC_MIXED]
    np.testing.assert_allclose(c32, c64, rtol=1e-4)
    for k in range(spec.K):
        assert O.aligned_error(J32[k], J64[k]) <= 1e-4


def test_full_size_512_station_cluster_mixed_matches_fp64():
    """One cluster of the 512-station workload (130816 baselines, 10
    timeslots, 4 channels, 100 sources): the mixed path factorises and solves
    at order 4096, as the bench does, and its final cost and Jones after 10 LM
    steps agree with the plain FP64 GPU path (itself pinned to the oracle
    above); the cost falls well below its starting value."""
    import dataclasses
    spec = dataclasses.replace(synth.config("c4"), K=1)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Jt = synth.jones_true(spec)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    dsky = sc.DeviceSky.from_synth(sky)
    u, fr = tdev(uvw, torch.float64), tdev(f, torch.float64)
    ws64 = sc.workspace(shp, sc.SC_FP64)
    C = sc.predict_coherencies(shp, u, fr, dsky, sc.SC_FP64, ws64)
    Jtd = tdev(Jt, torch.complex128)
    p, q = np.triu_indices(spec.N, 1)
    G = Jtd[:, p] @ Jtd[:, q].conj().transpose(-1, -2)                     # [1][B][2][2]
    V = torch.einsum("ktbf,kbij->tbfij", C, G) + tdev(synth.noise(spec), torch.complex128)
    del C, G
    res = {}
    for prec in PRECS:
        ws = ws64 if prec == sc.SC_FP64 else sc.workspace(shp, prec)
        Jg = tdev(synth.identity_jones(spec.K, spec.N), torch.complex128)
        Cp = sc.predict_coherencies(shp, u, fr, dsky, prec, ws)
        _, cost0 = sc.residual(shp, V.to(cdt(prec)).contiguous(), Cp[0].contiguous(), Jg[0], prec, ws)
        _, cost, iters = sc.solve_cluster(shp, V.to(cdt(prec)).contiguous(), Cp[0].contiguous(), Jg[0], prec, ws,
                                          n_lm=10, refine_sweeps=1, eps_grad=0.0)
        assert sc.device_status(ws) == 0
        res[prec] = (float(cost0), cost.item(), Jg[0].cpu().numpy(), iters.item())
        del Cp
    c0, c64, J64, it64 = res[sc.SC_FP64]
    _, c32, J32, it32 = res[sc.SC_MIXED]
    assert it64 == it32 == 10
    assert c64 < 0.5 * c0
    assert abs(c32 - c64) <= 1e-4 * c64
    assert O.aligned_error(J32, J64) <= 1e-4
