"""Residual of all clusters and its correction (sc_residual_all) against the
FP64 oracle, element by element, through the C ABI.

Both sides take the same inputs: the oracle's coherencies and data rounded to
the path's complex type, and those rounded values, widened back, given to the
oracle.  What differs is the arithmetic alone:
* FP64 path: 1e-12 of the visibility scale s = max|V| + sum_k max|C_k| max|G_k|
  (G_k = J_kp J_kq^H);
* mixed path: float32 sums of K + 1 terms, 2e-6 of s; after the correction
  also scaled by max|J^-1|_F^2 (the inverses are formed in float64 and
  rounded);
* the cost (before correction): |sum|R'|^2 - sum|R|^2| <= 2 |R| e + e^2 with
  e = |R' - R|_F bounded by the element tolerance (Cauchy-Schwarz), plus the
  float32 rounding of each |R|^2.
Sizes: N = 37 and 70 (666 and 2415 baselines, several 256-thread blocks and a
ragged last one), T*F = 6 and 5 (a ragged last slab of 4 visibilities), a
cluster without sources, N = 2, T = F = K = 1, and K = 4, 8, 9 (the
complex64 path streams the coherencies through its 4-stage shared-memory
ring once K reaches the stage count; K = 1 and 3 take the register kernel).  The full-size case runs the
512-station, 40-cluster launch configuration the benchmark times.
"""
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


def npc(prec):
    return np.complex64 if prec == sc.SC_MIXED else np.complex128


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype).contiguous()


def job(N, T, F, K, counts=None, seed=31):
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=5, f_lo=140e6, f_hi=160e6, alpha=-0.7,
                         seed=seed, sigma=0.05, jones_var=0.2)
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    sky = synth.sky(spec, counts)
    Jt = synth.jones_true(spec)
    Cs = O.predict_sky(uvw, f, sky)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(K)) + synth.noise(spec)
    # the solution differs a little from the truth, as after calibration
    J = Jt * (1.0 + 0.02j)
    return spec, Cs, V, J


def g_max(J):
    """max over baselines of |J_p J_q^H|_F, per cluster."""
    n = np.linalg.norm(J, axis=(-2, -1))
    return n.max(axis=1) ** 2


def inv_max(Jc):
    return max(np.linalg.norm(np.linalg.inv(j)) for j in Jc)


def run(prec, spec, Cs, V, J, corr, out_in_place=False):
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, 1)
    ws = sc.workspace(shp, prec)
    Vd = tdev(V, cdt(prec))
    R, cost = sc.residual_all(shp, Vd, tdev(Cs, cdt(prec)), tdev(J, torch.complex128), prec, ws,
                              corr=corr, out=Vd if out_in_place else None)
    return R.cpu().numpy().astype(np.complex128), cost.item(), sc.device_status(ws)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,T,F,K,counts", [(37, 3, 2, 3, [5, 0, 2]), (70, 2, 3, 4, None),
                                            (2, 1, 1, 1, None), (37, 3, 2, 9, None),
                                            (70, 1, 5, 8, None)])
def test_residual_all_matches_oracle(prec, N, T, F, K, counts):
    spec, Cs, V, J = job(N, T, F, K, counts)
    # both sides see the same rounded inputs
    Cs = Cs.astype(npc(prec)).astype(np.complex128)
    V = V.astype(npc(prec)).astype(np.complex128)
    s = np.abs(V).max() + sum(np.abs(Cs[k]).max() * g_max(J)[k] for k in range(K))
    rel = 1e-12 if prec == sc.SC_FP64 else 2e-6
    for corr in sorted({-1, 0, K - 1}):
        R_ref, cost_ref, sing = O.residual_all(V, Cs, J, corr)
        assert not sing.any()
        got, cost, status = run(prec, spec, Cs, V, J, corr)
        tol = rel * s * (inv_max(J[corr]) ** 2 if corr >= 0 else 1.0)
        assert np.max(np.abs(got - R_ref)) <= tol, (corr, np.max(np.abs(got - R_ref)), tol)
        e = rel * s * np.sqrt(V.size)
        ctol = 2 * np.sqrt(cost_ref) * e + e * e + (1e-12 if prec == sc.SC_FP64 else 1e-6) * cost_ref
        assert abs(cost - cost_ref) <= ctol
        assert status == 0
        # in place: bit for bit the out-of-place result
        got2, cost2, _ = run(prec, spec, Cs, V, J, corr, out_in_place=True)
        assert np.array_equal(got2, got) and cost2 == cost


@pytest.mark.parametrize("prec", PRECS)
def test_residual_all_singular_station_is_zeroed(prec):
    spec, Cs, V, J = job(37, 3, 2, 3)
    Cs = Cs.astype(npc(prec)).astype(np.complex128)
    V = V.astype(npc(prec)).astype(np.complex128)
    J[1, 5] = [[1.0, 2.0j], [0.5, 1.0j]]         # rank one: det = 0 exactly
    J[1, 30] = 0.0
    R_ref, _, sing = O.residual_all(V, Cs, J, corr=1)
    assert np.flatnonzero(sing).tolist() == [5, 30]
    got, _, status = run(prec, spec, Cs, V, J, corr=1)
    assert status & sc.SC_STATUS_SINGULAR
    p, q = synth.baseline_pairs(spec.N)
    hit = sing[p] | sing[q]
    assert np.all(got[:, hit] == 0)
    good = np.delete(np.arange(spec.N), [5, 30])
    s = np.abs(V).max() + sum(np.abs(Cs[k]).max() * g_max(J)[k] for k in range(3))
    rel = 1e-12 if prec == sc.SC_FP64 else 2e-6
    tol = rel * s * inv_max(J[1][good]) ** 2
    assert np.max(np.abs(got[:, ~hit] - R_ref[:, ~hit])) <= tol
    # without the correction nothing is flagged
    _, _, status = run(prec, spec, Cs, V, J, corr=-1)
    assert status == 0


def test_full_size_residual_all_sampled_against_oracle():
    """512 stations x 10 timeslots x 4 channels, 40 clusters x 100 sources,
    mixed path, corrected towards cluster 0: the launch configuration of the
    benchmark.  The coherencies come from the library's own prediction; the
    oracle predicts each sampled (t, b, f) itself, so the tolerance adds the
    prediction's 1e-5 (of each cluster's flux sum) times |G_k|.  The cost
    equals sum |R|^2 of the uncorrected output."""
    spec = synth.config("c4")
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    J = synth.jones_true(spec)
    V = synth.noise(spec) * 100.0            # a Jy-scale stand-in for the data
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    prec = sc.SC_MIXED
    ws = sc.workspace(shp, prec)
    C = sc.predict_coherencies(shp, tdev(uvw, torch.float64), tdev(f, torch.float64),
                               sc.DeviceSky.from_synth(sky), prec, ws)
    Vd = tdev(V, torch.complex64)
    Jd = tdev(J, torch.complex128)
    R0, cost0 = sc.residual_all(shp, Vd, C, Jd, prec, ws, corr=-1)
    direct = torch.sum(R0.real.double() ** 2 + R0.imag.double() ** 2).item()
    assert abs(cost0.item() - direct) <= 1e-6 * direct
    R1, _ = sc.residual_all(shp, Vd, C, Jd, prec, ws, corr=0)
    assert sc.device_status(ws) == 0
    del C
    rng = np.random.default_rng(1)
    n = 200
    p = rng.integers(0, spec.N - 1, n)
    q = p + 1 + rng.integers(0, 1 << 30, n) % (spec.N - 1 - p)
    t = rng.integers(0, spec.T, n)
    fi = rng.integers(0, spec.F, n)
    b = p * spec.N - p * (p + 1) // 2 + (q - p - 1)
    idx = (torch.as_tensor(t), torch.as_tensor(b), torch.as_tensor(fi))
    g0 = R0[idx].cpu().numpy().astype(np.complex128)
    g1 = R1[idx].cpu().numpy().astype(np.complex128)
    Vs = V.astype(np.complex64).astype(np.complex128)
    flux = [sky.flux[a:e].sum() for a, e in zip(sky.offsets[:-1], sky.offsets[1:])]
    for m in range(n):
        pq = [p[m], q[m]]
        Cs = np.stack([O.predict_coherencies(uvw[t[m]:t[m] + 1][:, pq, :], f[fi[m]:fi[m] + 1],
                                             sky.l[a:e], sky.m[a:e], sky.flux[a:e], sky.alpha[a:e])
                       for a, e in zip(sky.offsets[:-1], sky.offsets[1:])])   # [K][1][1][1]
        Vm = Vs[t[m]:t[m] + 1, b[m]:b[m] + 1, fi[m]:fi[m] + 1]
        Jm = J[:, pq]
        r0, _, _ = O.residual_all(Vm, Cs, Jm)
        r1, _, _ = O.residual_all(Vm, Cs, Jm, corr=0)
        gk = [np.linalg.norm(Jm[k, 0] @ Jm[k, 1].conj().T) for k in range(spec.K)]
        s = np.abs(Vm).max() + sum(abs(Cs[k]).max() * gk[k] for k in range(spec.K))
        tol = 1e-5 * sum(flux[k] * gk[k] for k in range(spec.K)) + 2e-6 * s
        amp = np.linalg.norm(np.linalg.inv(Jm[0, 0])) * np.linalg.norm(np.linalg.inv(Jm[0, 1]))
        assert np.max(np.abs(g0[m] - r0[0, 0, 0])) <= tol
        assert np.max(np.abs(g1[m] - r1[0, 0, 0])) <= tol * amp
