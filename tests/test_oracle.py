"""Pins of the FP64 oracle against facts the mathematics fixes.

Each test checks the oracle against something other than itself: closed
forms, an independent geometric construction, finite differences, known
minimisers, symmetries and a noise statistic.  A dropped term, a wrong sign,
a swapped index or a transposed operand in the oracle fails at least one.
"""
import math

import numpy as np
import pytest
import scipy.optimize

import oracle as O
from paper_1910_13908_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def small_spec(**kw):
    base = dict(N=6, T=3, F=2, K=1, S=4, f_lo=140e6, f_hi=160e6, seed=3)
    base.update(kw)
    return synth.JobSpec(**base)


# --- prediction -----------------------------------------------------------------

def test_unit_source_at_phase_centre_is_exactly_one():
    spec = small_spec()
    uvw = synth.station_uvw(spec)
    C = O.predict_coherencies(uvw, synth.freqs(spec), [0.0], [0.0], [1.0], [0.0])
    assert C.shape == (spec.T, spec.B, spec.F)
    assert np.array_equal(C, np.ones_like(C))


def test_phase_is_the_geometric_delay():
    """A source given by hour angle and declination: the phase of C_pq must be
    -2 pi f/c (x_p - x_q).(s - s0) with x the equatorial station positions and
    s, s0 unit vectors to the source and the phase centre.  This never uses
    (u, v, w) nor the (l, m) projection."""
    spec = small_spec(N=7, T=4, F=3)
    lat, dec0 = math.radians(spec.lat_deg), math.radians(spec.dec_deg)
    xyz = synth.enu_to_xyz(synth.stations_enu(spec), lat)
    dra, dec_s = math.radians(2.1), math.radians(53.3)
    l = math.cos(dec_s) * math.sin(dra)
    m = math.sin(dec_s) * math.cos(dec0) - math.cos(dec_s) * math.sin(dec0) * math.cos(dra)
    flux = 2.5
    f = synth.freqs(spec)
    C = O.predict_coherencies(synth.station_uvw(spec), f, [l], [m], [flux], [0.0])
    p, q = O.baselines(spec.N)
    for t, H in enumerate(synth.hour_angles(spec)):
        Hs = H - dra
        s = np.array([math.cos(dec_s) * math.cos(Hs), -math.cos(dec_s) * math.sin(Hs), math.sin(dec_s)])
        s0 = np.array([math.cos(dec0) * math.cos(H), -math.cos(dec0) * math.sin(H), math.sin(dec0)])
        delay_m = (xyz[p] - xyz[q]) @ (s - s0)
        for fi, fr in enumerate(f):
            ref = flux * np.exp(-2j * np.pi * fr / O.C_LIGHT * delay_m)
            np.testing.assert_allclose(C[t, :, fi], ref, rtol=0, atol=1e-9)


def test_conjugate_baseline_is_hermitian():
    """Swapping the stations of a baseline negates its uvw: C_qp = conj(C_pq),
    and J_q C_qp J_p^H = (J_p C_pq J_q^H)^H."""
    spec = small_spec()
    uvw = synth.station_uvw(spec)
    sky = synth.sky(spec)
    f = synth.freqs(spec)
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    Cr = O.predict_coherencies(uvw[:, ::-1, :], f, sky.l, sky.m, sky.flux, sky.alpha)
    N = spec.N
    p, q = O.baselines(N)
    rb = {(a, b): i for i, (a, b) in enumerate(zip(*O.baselines(N)))}
    # reversed station order: station a of the reversed array is N-1-a
    idx = [rb[(N - 1 - q[i], N - 1 - p[i])] for i in range(len(p))]
    np.testing.assert_allclose(Cr[:, idx, :], np.conj(C), atol=1e-12)
    J = synth.jones_true(spec)[0]
    M = O.model_vis(C, J)
    Mr = O.model_vis(Cr, J[::-1])
    np.testing.assert_allclose(Mr[:, idx], np.conj(np.swapaxes(M, -1, -2)), atol=1e-12)


def test_linear_in_sources():
    spec = small_spec(S=6)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    a = O.predict_coherencies(uvw, f, sky.l[:2], sky.m[:2], sky.flux[:2], sky.alpha[:2])
    b = O.predict_coherencies(uvw, f, sky.l[2:], sky.m[2:], sky.flux[2:], sky.alpha[2:])
    c = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    np.testing.assert_allclose(a + b, c, atol=1e-12)


def test_spectral_law_at_phase_centre():
    """At l = m = 0 every baseline sees the source flux density at f."""
    spec = small_spec(F=1, f_lo=300e6, f_hi=300e6)
    C = O.predict_coherencies(synth.station_uvw(spec), [300e6], [0.0], [0.0], [4.0], [-0.7])
    np.testing.assert_allclose(C, 4.0 * 2.0 ** -0.7, rtol=1e-15)


# --- Jacobian and normal equations ----------------------------------------------

def _residual_vec(X, C, theta):
    R, _ = O.residual(X, C, O.theta_to_jones(theta))
    R = R.reshape(-1, 4)
    return np.concatenate([R.real, R.imag], axis=1).ravel()


def test_normal_equations_match_finite_differences():
    spec = small_spec(N=4, T=2, F=2, S=3)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    Jt = synth.jones_true(spec)[0]
    X = O.model_vis(C, Jt) + synth.noise(spec)
    J = Jt + 0.05 * (synth.normal(9, 9, 32)[:16] + 1j * synth.normal(9, 9, 32)[16:]).reshape(4, 2, 2)
    theta = O.jones_to_theta(J)
    h = 1e-6
    r0 = _residual_vec(X, C, theta)
    Jr = np.empty((r0.size, theta.size))
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        Jr[:, k] = (_residual_vec(X, C, theta + e) - _residual_vec(X, C, theta - e)) / (2 * h)
    R, cost = O.residual(X, C, J)
    A, g = O.normal_equations(R, C, J)
    # model Jacobian = -d r / d theta
    np.testing.assert_allclose(A, Jr.T @ Jr, rtol=1e-7, atol=1e-7 * np.abs(A).max())
    np.testing.assert_allclose(g, -Jr.T @ r0, rtol=1e-7, atol=1e-7 * np.abs(g).max())
    # and the cost gradient is -2 g
    dc = np.empty(theta.size)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        dc[k] = (O.residual(X, C, O.theta_to_jones(theta + e))[1]
                 - O.residual(X, C, O.theta_to_jones(theta - e))[1]) / (2 * h)
    np.testing.assert_allclose(dc, -2 * g, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_gauge_directions_are_in_the_null_space():
    """J_p -> J_p exp(i eps H) (H Hermitian, same for all p) leaves every
    J_p C J_q^H unchanged, so those 4 directions annihilate J^T J and g."""
    spec = small_spec(N=5)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    J = synth.jones_true(spec)[0]
    X = O.model_vis(C, J * 1.1) + synth.noise(spec)
    R, _ = O.residual(X, C, J)
    A, g = O.normal_equations(R, C, J)
    gens = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
    for H in gens:
        xi = O.jones_to_theta(J @ (1j * np.asarray(H, dtype=complex)))
        assert np.linalg.norm(A @ xi) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(xi)
        assert abs(g @ xi) <= 1e-12 * np.linalg.norm(g) * np.linalg.norm(xi)
    # and J^T J is symmetric positive semidefinite with exactly 4 null directions
    w = np.linalg.eigvalsh(A)
    assert np.allclose(A, A.T)
    assert np.sum(w < 1e-10 * w.max()) == 4 and w.min() > -1e-10 * w.max()


# --- linear algebra -------------------------------------------------------------

def test_cholesky_solve_exact_integer_system():
    rng = np.random.default_rng(1)
    n = 12
    L = np.tril(rng.integers(-3, 4, size=(n, n)), -1) + np.diag(rng.integers(1, 4, size=n))
    A = (L @ L.T).astype(np.float64)
    x = rng.integers(-5, 6, size=n).astype(np.float64)
    np.testing.assert_allclose(O.cholesky_solve(A, A @ x), x, rtol=0, atol=1e-9)
    M = rng.standard_normal((40, 40))
    S = M @ M.T + 40 * np.eye(40)
    Lc = np.linalg.cholesky(S)
    assert np.linalg.norm(Lc @ Lc.T - S) <= 1e-13 * np.linalg.norm(S)
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky_solve(-S, np.ones(40))


# --- Levenberg-Marquardt ----------------------------------------------------------

def test_lm_on_a_linear_problem():
    """For a linear model the gain ratio is exactly 1, so every step is taken
    and mu shrinks by 3 per step; the iterates reach the least-squares
    solution."""
    rng = np.random.default_rng(2)
    M = rng.standard_normal((30, 5))
    y = rng.standard_normal(30)

    def ev(th):
        r = y - M @ th
        return float(r @ r), M.T @ M, M.T @ r

    trace = []
    # heavy initial damping (tau = 10) keeps the first steps short, so the
    # decrease of each is well above rounding
    th, cost, done = O.levenberg_marquardt(ev, np.zeros(5), 200, tau=10.0, eps_grad=1e-14, trace=trace)
    ref = np.linalg.lstsq(M, y, rcond=None)[0]
    # the cost-based acceptance stalls once the remaining cost excess is below
    # the rounding of the cost (|theta - ref| ~ 1e-8 here)
    np.testing.assert_allclose(th, ref, atol=1e-7)
    mu0 = 10.0 * np.max(np.diag(M.T @ M))
    assert trace[0]["mu"] == pytest.approx(mu0, rel=1e-15)
    for a, b in zip(trace[:3], trace[1:4]):
        assert a["rho"] == pytest.approx(1.0, abs=1e-6)
        assert b["mu"] == pytest.approx(a["mu"] / 3.0, rel=1e-12)


def test_lm_rosenbrock():
    def ev(th):
        x, yv = th
        r = np.array([10.0 * (yv - x * x), 1.0 - x])
        Jm = -np.array([[-20.0 * x, 10.0], [-1.0, 0.0]])   # d model / d theta = -dr/dtheta
        return float(r @ r), Jm.T @ Jm, Jm.T @ r

    th, cost, _ = O.levenberg_marquardt(ev, np.array([-1.2, 1.0]), 200, eps_grad=1e-15)
    np.testing.assert_allclose(th, [1.0, 1.0], atol=1e-8)
    assert cost < 1e-16


def test_noiseless_lm_recovers_true_jones_up_to_unitary():
    spec = small_spec(N=8, T=4, F=2, S=5, seed=11)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    Jt = synth.jones_true(spec)[0]
    V = O.model_vis(C, Jt)
    J, cost, _ = O.lm_cluster(V, C, np.tile(np.eye(2, dtype=complex), (spec.N, 1, 1)), 40, eps_grad=0.0)
    assert cost <= 1e-20 * float(np.sum(np.abs(V) ** 2))
    assert O.aligned_error(J, Jt) < 1e-8


def test_noisy_minimum_has_the_chi2_cost():
    """At the least-squares minimum E[cost] = sigma^2 (n_data - rank J), with
    n_data = 8 B T F reals and rank 8N - 4 (the U(2) gauge); the standard
    deviation is sigma^2 sqrt(2 (n_data - rank))."""
    spec = small_spec(N=16, T=10, F=2, S=6, seed=5, sigma=0.05)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    Jt = synth.jones_true(spec)[0]
    V = O.model_vis(C, Jt) + synth.noise(spec)
    J, cost, _ = O.lm_cluster(V, C, np.tile(np.eye(2, dtype=complex), (spec.N, 1, 1)), 30)
    dof = 8 * spec.B * spec.T * spec.F - (8 * spec.N - 4)
    mean, sd = spec.sigma ** 2 * dof, spec.sigma ** 2 * math.sqrt(2 * dof)
    assert abs(cost - mean) < 4 * sd


def test_multistart_finds_no_lower_minimum_on_three_stations():
    spec = small_spec(N=3, T=3, F=1, S=2, seed=7, sigma=0.02)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    Jt = synth.jones_true(spec)[0]
    V = O.model_vis(C, Jt) + synth.noise(spec)
    J, cost, _ = O.lm_cluster(V, C, np.tile(np.eye(2, dtype=complex), (3, 1, 1)), 50, eps_grad=0.0)
    best = np.inf
    for s in range(20):
        x0 = O.jones_to_theta(np.eye(2)[None].repeat(3, 0)) + 0.5 * synth.normal(100 + s, 1, 24)
        res = scipy.optimize.least_squares(lambda th: _residual_vec(V, C, th), x0, method="lm",
                                           xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
        best = min(best, 2 * res.cost)
    assert cost <= best * (1 + 1e-9)


# --- SAGE ---------------------------------------------------------------------------

def _multi(spec):
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Cs = O.predict_sky(uvw, f, sky)
    return Cs, synth.jones_true(spec)


def test_sage_with_one_cluster_is_lm():
    spec = small_spec(N=6, K=1, seed=4)
    Cs, Jt = _multi(spec)
    V = O.model_vis(Cs[0], Jt[0]) + synth.noise(spec)
    J0 = synth.identity_jones(1, spec.N)
    Js, cs = O.sage_calibrate(V, Cs, J0, n_em=1, n_lm=7)
    Jl, cl, _ = O.lm_cluster(V, Cs[0], J0[0], 7)
    assert np.array_equal(Js[0], Jl) and cs[0] == cl


def test_sage_noiseless_two_clusters_recovers_both():
    spec = small_spec(N=8, T=4, F=2, K=2, S=4, seed=12)
    Cs, Jt = _multi(spec)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(2))
    sweeps = []
    J, costs = O.sage_calibrate(V, Cs, synth.identity_jones(2, spec.N), n_em=40, n_lm=10,
                                eps_grad=0.0, sweep_costs=sweeps)
    for k in range(2):
        assert O.aligned_error(J[k], Jt[k]) < 1e-6
    assert sweeps[-1] < 1e-10 * float(np.sum(np.abs(V) ** 2))


def test_sage_total_cost_never_increases():
    spec = small_spec(N=7, T=3, F=2, K=3, S=3, seed=13, sigma=0.02)
    Cs, Jt = _multi(spec)
    V = sum(O.model_vis(Cs[k], Jt[k]) for k in range(3)) + synth.noise(spec)
    sweeps = []
    O.sage_calibrate(V, Cs, synth.identity_jones(3, spec.N), n_em=6, n_lm=5, sweep_costs=sweeps)
    R0 = V - sum(O.model_vis(Cs[k], np.tile(np.eye(2), (spec.N, 1, 1))) for k in range(3))
    prev = float(np.sum(np.abs(R0) ** 2))
    for c in sweeps:
        assert c <= prev * (1 + 1e-12)
        prev = c


def test_procrustes_recovers_a_known_rotation():
    spec = small_spec(N=9)
    Jt = synth.jones_true(spec)[0]
    H = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])
    w, v = np.linalg.eigh(H)
    U = v @ np.diag(np.exp(1j * w)) @ v.conj().T
    J = Jt @ U.conj().T
    np.testing.assert_allclose(O.align_unitary(J, Jt), U, atol=1e-12)
    assert O.aligned_error(J, Jt) < 1e-12


# --- residual of all clusters and its correction ---------------------------------

def _brute_vis(Cs, J, A=None, c=None):
    """V_pq = sum_k J_kp (C_kpq Id) J_kq^H (+ J_cp A_pq J_cq^H), one visibility
    at a time, with explicit 2x2 products."""
    K, T, B, F = Cs.shape
    N = J.shape[1]
    pq = [(a, b) for a in range(N) for b in range(a + 1, N)]
    V = np.zeros((T, B, F, 2, 2), dtype=np.complex128)
    for t in range(T):
        for b, (p, q) in enumerate(pq):
            for f in range(F):
                for k in range(K):
                    V[t, b, f] += J[k, p] @ (Cs[k, t, b, f] * np.eye(2)) @ J[k, q].conj().T
                if A is not None:
                    V[t, b, f] += J[c, p] @ A[t, b, f] @ J[c, q].conj().T
    return V


def test_residual_all_removes_every_cluster():
    spec = small_spec(N=5, T=2, F=2, K=3, S=3, seed=21, sigma=0.3)
    Cs, Jt = _multi(spec)
    A = synth.noise(spec)
    V = _brute_vis(Cs, Jt) + A
    R, cost, sing = O.residual_all(V, Cs, Jt)
    np.testing.assert_allclose(R, A, rtol=0, atol=1e-12 * np.abs(V).max())
    assert math.isclose(cost, float(np.sum(np.abs(A) ** 2)), rel_tol=1e-9)
    assert not sing.any()
    # leaving one cluster in the data leaves exactly its model behind
    R2, _, _ = O.residual_all(V, Cs[:2], Jt[:2])
    np.testing.assert_allclose(R2 - A, _brute_vis(Cs[2:], Jt[2:]), rtol=0,
                               atol=1e-12 * np.abs(V).max())


def test_residual_all_correction_recovers_the_planted_signal():
    # the unmodelled signal A seen through direction c's gains comes back as A
    spec = small_spec(N=6, T=2, F=3, K=3, S=2, seed=22, sigma=0.5, jones_var=0.3)
    Cs, Jt = _multi(spec)
    A = synth.noise(spec)
    for c in range(3):
        V = _brute_vis(Cs, Jt, A, c)
        R, cost, sing = O.residual_all(V, Cs, Jt, corr=c)
        np.testing.assert_allclose(R, A, rtol=0, atol=1e-11 * np.abs(A).max())
        seen = _brute_vis(np.zeros_like(Cs[:1]), Jt[c:c + 1], A, 0)
        assert math.isclose(cost, float(np.sum(np.abs(seen) ** 2)), rel_tol=1e-9)
        assert not sing.any()


def test_residual_all_identity_gains_correct_nothing():
    spec = small_spec(N=5, T=2, F=2, K=2, S=2, seed=23)
    Cs, Jt = _multi(spec)
    V = _brute_vis(Cs, Jt) + synth.noise(spec)
    J = Jt.copy()
    J[1] = np.eye(2)
    R0, c0, _ = O.residual_all(V, Cs, J)
    R1, c1, _ = O.residual_all(V, Cs, J, corr=1)
    assert np.array_equal(R0, R1) and c0 == c1


def test_residual_all_singular_stations_are_zeroed():
    spec = small_spec(N=6, T=2, F=2, K=2, S=2, seed=24, sigma=0.5)
    Cs, Jt = _multi(spec)
    J = Jt.copy()
    J[0, 1] = [[1.0, 2.0j], [0.5, 1.0j]]          # rank one: det = 0
    J[0, 4] = 0.0
    A = synth.noise(spec)
    V = _brute_vis(Cs, J, A, 0)
    R, _, sing = O.residual_all(V, Cs, J, corr=0)
    assert sing.tolist() == [False, True, False, False, True, False]
    p, q = synth.baseline_pairs(spec.N)
    hit = sing[p] | sing[q]
    assert np.all(R[:, hit] == 0)
    np.testing.assert_allclose(R[:, ~hit], A[:, ~hit], rtol=0, atol=1e-11 * np.abs(A).max())


def test_residual_all_is_invariant_to_the_unitary_ambiguity():
    # J_k -> J_k U_k leaves every model unchanged; the corrected residual turns
    # into U_c^H R U_c, so its per-visibility Frobenius norms stay the same
    spec = small_spec(N=5, T=2, F=2, K=2, S=2, seed=25, sigma=0.2)
    Cs, Jt = _multi(spec)
    V = _brute_vis(Cs, Jt) + synth.noise(spec)
    H = np.array([[0.7, 0.1 + 0.4j], [0.1 - 0.4j, -0.2]])
    w, v = np.linalg.eigh(H)
    U = v @ np.diag(np.exp(1j * w)) @ v.conj().T
    R0, c0, _ = O.residual_all(V, Cs, Jt, corr=1)
    R1, c1, _ = O.residual_all(V, Cs, Jt @ U, corr=1)
    assert math.isclose(c0, c1, rel_tol=1e-12)
    np.testing.assert_allclose(R1, U.conj().T @ R0 @ U, rtol=0, atol=1e-12 * np.abs(R0).max())
    np.testing.assert_allclose(np.linalg.norm(R1, axis=(-2, -1)), np.linalg.norm(R0, axis=(-2, -1)),
                               rtol=1e-12, atol=1e-14)


# --- consecutive time chunks, warm-started -------------------------------------------

def _chunked(spec, n, Tc, drift=0.0):
    """n chunks of Tc timeslots of one observation, noiseless.  The true gains
    of chunk i are J_true times a phase exp(i drift i x_s), x_s in [0, 1]
    per station: they drift slowly from chunk to chunk."""
    import dataclasses
    full = dataclasses.replace(spec, T=n * Tc)
    uvw, f, sky = synth.station_uvw(full), synth.freqs(full), synth.sky(full)
    Jt = synth.jones_true(full)
    ph = np.linspace(0.0, 1.0, spec.N)[None, :, None, None]
    Vs, Css, Jts = [], [], []
    for i in range(n):
        u = uvw[i * Tc:(i + 1) * Tc]
        Cs = O.predict_sky(u, f, sky)
        Ji = Jt * np.exp(1j * drift * i * ph)
        Vs.append(sum(O.model_vis(Cs[k], Ji[k]) for k in range(spec.K)))
        Css.append(Cs)
        Jts.append(Ji)
    return Vs, Css, Jts


def test_chunks_single_chunk_is_sage():
    spec = small_spec(N=6, T=2, F=2, K=2, S=3, seed=41)
    Vs, Css, _ = _chunked(spec, 1, 2)
    J0 = synth.identity_jones(2, spec.N)
    Jc, cc = O.calibrate_chunks(Vs, Css, J0, n_em=2, n_lm=4)
    Js, cs = O.sage_calibrate(Vs[0], Css[0], J0, n_em=2, n_lm=4)
    assert np.array_equal(Jc[0], Js) and np.array_equal(cc[0], cs)


def test_chunks_resume_from_a_checkpoint_continues_exactly():
    # the solution of chunk 1 is the whole solver state: restarting there
    # reproduces chunks 2 and 3 of the uninterrupted run bit for bit
    spec = small_spec(N=6, T=2, F=2, K=2, S=3, seed=42)
    Vs, Css, _ = _chunked(spec, 4, 2, drift=0.05)
    J0 = synth.identity_jones(2, spec.N)
    J_all, c_all = O.calibrate_chunks(Vs, Css, J0, n_em=1, n_lm=3)
    J_a, c_a = O.calibrate_chunks(Vs[:2], Css[:2], J0, n_em=1, n_lm=3)
    J_b, c_b = O.calibrate_chunks(Vs[2:], Css[2:], J_a[-1], n_em=1, n_lm=3)
    assert np.array_equal(np.concatenate([J_a, J_b]), J_all)
    assert np.array_equal(np.concatenate([c_a, c_b]), c_all)
    # and the chunks are not independent: a cold restart at chunk 2 differs
    J_c, _ = O.calibrate_chunks(Vs[2:], Css[2:], J0, n_em=1, n_lm=3)
    assert not np.array_equal(J_c, J_b)


def test_warm_start_beats_cold_start_on_slowly_drifting_gains():
    # noiseless data whose gains drift slowly: each warm-started chunk begins
    # near its answer, a cold start (identity) does not; same iteration budget
    spec = small_spec(N=7, T=2, F=2, K=2, S=3, seed=43)
    n = 4
    Vs, Css, Jts = _chunked(spec, n, 2, drift=0.02)
    J0 = synth.identity_jones(2, spec.N)
    _, c_warm = O.calibrate_chunks(Vs, Css, J0, n_em=1, n_lm=3)
    for i in range(1, n):
        _, c_cold = O.sage_calibrate(Vs[i], Css[i], J0, n_em=1, n_lm=3)
        assert c_warm[i].sum() < 0.1 * c_cold.sum(), (i, c_warm[i], c_cold)
