"""FP64 CPU oracle of the calibration hot path (test infrastructure only).

The paper (Spreeuw et al., "GPU acceleration of the SAGECal calibration
package for the SKA") times SAGECal's CPU and GPU builds calibrating clustered
sky models (§2: "a single calibration solution will be derived for each
cluster") on arrays whose data size grows as the N(N-1)/2 baselines (§3).  It
prints no equation; the method it times is SAGECal's:

* the radio-interferometric measurement equation (Hamaker, Bregman & Sault
  1996): per cluster k, V_pq = J_kp C_kpq J_kq^H with 2x2 complex Jones
  matrices J and the point-source coherency
  C_pq(t, f) = sum_s S_s(f) exp(-2 pi i f/c (u l_s + v m_s + w (n_s - 1))) Id;
* Levenberg-Marquardt on the Gauss-Newton normal equations J^T J, J^T r
  (Madsen, Nielsen & Tingleff 2004, Alg. 3.16: damping mu I with
  mu0 = tau max diag(J^T J)), each damped system solved by a Cholesky
  factorisation;
* SAGE/EM (Fessler & Hero 1994; Kazemi et al. 2011, SAGECal's solver): the
  clusters are solved one at a time, cluster k against the data minus the
  current models of all other clusters.

Everything is float64 / complex128.  Plain and slow by design: the Jacobian is
built row by row from its definition (product rule on J_p C J_q^H), J^T J is
summed from those rows, and the LM loop follows the textbook order.  Library
steps: numpy.linalg.cholesky and scipy's triangular solves; numpy.linalg.svd
for the Procrustes alignment.

Conventions
-----------
* baselines b = (p, q), p < q, ordered b = p*N - p(p+1)/2 + (q-p-1)
* station (u, v, w) in metres, [T][N][3]; baseline uvw_pq = uvw_p - uvw_q
* visibilities [T][B][F][2][2] complex, coherencies [T][B][F] complex (the
  unpolarised brightness matrix is a multiple of the identity)
* parameters of station s: theta[8s + 4i + 2j + 0/1] = Re/Im J_s[i, j]
* "Jhr" = J^T r with r = X - model (so the LM step solves (A + mu I) d = Jhr)

What pins each function (tests/test_oracle.py):
* predict_coherencies: a unit source at the phase centre gives exactly 1;
  a source given by (hour angle, declination) gives the phase of its
  geometric delay (x_p - x_q).(s - s0) f/c computed in the equatorial frame;
  Hermitian swap of p and q; linearity in sources; spectral law at l=m=0.
* normal_equations: central finite differences of the residual on 4 stations;
  gradient of the cost; gauge generators in the null space of J^T J.
* cholesky_solve: reconstruction and exact integer systems.
* levenberg_marquardt: a linear least-squares problem (rho = 1, mu/3 per
  step, exact solution); Rosenbrock's function; noiseless recovery of the
  true Jones up to the unitary ambiguity; the chi^2 statistic of the noisy
  minimum; a multistart search on 3 stations finds no lower cost.
* sage_calibrate: K = 1 is the single-cluster LM bit for bit; noiseless
  multi-cluster recovery; the total cost never increases over EM sweeps.
* predict_coherencies_full (polarised, extended sources): an unpolarised
  point-source sky reduces it to predict_coherencies x Id; the Gaussian
  visibility equals a brute-force quadrature of the Fourier integral of the
  Gaussian brightness laid out with the stated axes and position angle
  (elongated and rotated); a zero-size Gaussian is a point; rotating the
  feeds by chi mixes (Q, U) by 2 chi and leaves I and V alone; the brightness
  matrix is Hermitian with det I^2 - |p|^2 and trace 2I; swapping p and q
  gives the conjugate transpose; linear in sources; the spectral law scales
  all four Stokes parameters.
* penalised / lm_cluster(penalty=...): on a linear least-squares problem
  the penalised LM reaches the closed form (A^T A + w I)^-1 (A^T b + w a).
* consensus_fit: np.linalg.lstsq per parameter; exact on data that is a
  polynomial of the basis.
* consensus_calibrate: rho = 0 is independent SAGE per band; noiseless data
  whose Jones vary along the basis is recovered with every penalty ~0;
  consensus lowers the error of noisy sub-band solutions; a larger rho
  shrinks the disagreement |J_f - basis[f] Z|.
* residual_all: against visibilities built one at a time with explicit 2x2
  products, removing every cluster leaves exactly the planted unmodelled
  signal A, and one cluster left in leaves its model; A seen through the gains
  of direction c comes back as A after correcting for c (each c); identity
  gains correct nothing; rank-one and zero Jones are flagged and zeroed;
  the unitary ambiguity turns the corrected residual into U^H R U.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

C_LIGHT = 299792458.0


# --- layout -------------------------------------------------------------------

def baselines(N: int):
    """(p, q) of every baseline, p < q, in baseline-index order."""
    p, q = [], []
    for a in range(N):
        for b in range(a + 1, N):
            p.append(a)
            q.append(b)
    return np.array(p, dtype=np.int64), np.array(q, dtype=np.int64)


def jones_to_theta(J: np.ndarray) -> np.ndarray:
    """[N][2][2] complex -> [8N] real, theta[8s+4i+2j] = Re, +1 = Im."""
    N = J.shape[0]
    th = np.empty((N, 2, 2, 2))
    th[..., 0] = J.real
    th[..., 1] = J.imag
    return th.reshape(8 * N)


def theta_to_jones(theta: np.ndarray) -> np.ndarray:
    th = theta.reshape(-1, 2, 2, 2)
    return th[..., 0] + 1j * th[..., 1]


# --- prediction ---------------------------------------------------------------

def predict_coherencies(uvw, freqs, l, m, flux, alpha, f0=150e6):
    """Point-source coherencies of one cluster, [T][B][F] complex128.

    C_pq(t,f) = sum_s S_s(f) exp(-2 pi i (f/c)(u l_s + v m_s + w (n_s - 1)))
    with S_s(f) = S_s (f/f0)^alpha_s, n_s = sqrt(1 - l_s^2 - m_s^2) and
    (u, v, w) the baseline coordinates uvw_p - uvw_q at timeslot t.
    """
    uvw = np.asarray(uvw, dtype=np.float64)
    T, N, _ = uvw.shape
    p, q = baselines(N)
    l = np.asarray(l, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    n = np.sqrt(1.0 - l * l - m * m)
    F = len(freqs)
    out = np.zeros((T, len(p), F), dtype=np.complex128)
    for t in range(T):
        b = uvw[t, p, :] - uvw[t, q, :]                       # [B][3]
        path = (np.outer(b[:, 0], l) + np.outer(b[:, 1], m)
                + np.outer(b[:, 2], n - 1.0))                 # [B][S] metres
        for fi, f in enumerate(freqs):
            S = np.asarray(flux) * (f / f0) ** np.asarray(alpha)
            out[t, :, fi] = np.exp(-2j * np.pi * (f / C_LIGHT) * path) @ S
    return out


def predict_sky(uvw, freqs, sky):
    """Coherencies of every cluster of a `synth.Sky`: [K][T][B][F]."""
    return np.stack([
        predict_coherencies(uvw, freqs, sky.l[a:b], sky.m[a:b], sky.flux[a:b],
                            sky.alpha[a:b], sky.f0)
        for a, b in zip(sky.offsets[:-1], sky.offsets[1:])])


# --- polarised and extended sources ------------------------------------------

FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


def brightness_matrix(I, Q, U, V):
    """Source brightness (coherency) matrix in the linear-feed basis,
    [S][2][2] complex:  [[I + Q, U + iV], [U - iV, I - Q]].

    Unnormalised, so that an unpolarised source of flux I gives I * Id, the
    coherency the point-source path uses; tr/2 = I, det = I^2 - Q^2 - U^2 - V^2.
    """
    I, Q, U, V = (np.asarray(a, dtype=np.float64) for a in (I, Q, U, V))
    out = np.empty(I.shape + (2, 2), dtype=np.complex128)
    out[..., 0, 0] = I + Q
    out[..., 0, 1] = U + 1j * V
    out[..., 1, 0] = U - 1j * V
    out[..., 1, 1] = I - Q
    return out


def gaussian_visibility(u_lam, v_lam, maj, mnr, pa):
    """Visibility of a unit-flux elliptical Gaussian at (u, v) in wavelengths:
    the Fourier transform of exp(-(x_a^2 / sigma_a^2 + x_b^2 / sigma_b^2) / 2)
    normalised to 1 at the origin,

        exp(-2 pi^2 (sigma_a^2 u_a^2 + sigma_b^2 u_b^2)),

    where sigma = FWHM / (2 sqrt(2 ln 2)), the major axis points along
    (l, m) = (sin pa, cos pa) (position angle from +m towards +l), the minor
    along (cos pa, -sin pa), and (u_a, u_b) are (u, v) projected on the same
    two unit vectors.  Broadcasts; maj = mnr = 0 gives 1 (a point source).
    """
    sa = np.asarray(maj, dtype=np.float64) / FWHM_PER_SIGMA
    sb = np.asarray(mnr, dtype=np.float64) / FWHM_PER_SIGMA
    sp, cp = np.sin(pa), np.cos(pa)
    ua = u_lam * sp + v_lam * cp
    ub = u_lam * cp - v_lam * sp
    return np.exp(-2.0 * np.pi ** 2 * (sa ** 2 * ua ** 2 + sb ** 2 * ub ** 2))


def predict_coherencies_full(uvw, freqs, l, m, I, Q, U, V, alpha, maj, mnr, pa, f0=150e6):
    """Full 2x2 coherencies of one cluster of polarised, possibly extended
    sources, [T][B][F][2][2] complex128:

        C_pq(t,f) = sum_s (f/f0)^alpha_s  G_s(u f/c, v f/c)
                    exp(-2 pi i (f/c)(u l_s + v m_s + w (n_s - 1)))  B_s

    with B_s = brightness_matrix(I_s, Q_s, U_s, V_s), G_s the Gaussian
    visibility (gaussian_visibility; 1 for a point source) and (u, v, w) the
    baseline uvw_p - uvw_q.  The shape is taken on the tangent plane at the
    source (its visibility depends on u, v only).
    """
    uvw = np.asarray(uvw, dtype=np.float64)
    T, N, _ = uvw.shape
    p, q = baselines(N)
    l = np.asarray(l, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    n = np.sqrt(1.0 - l * l - m * m)
    Bs = brightness_matrix(I, Q, U, V)                         # [S][2][2]
    F = len(freqs)
    out = np.zeros((T, len(p), F, 2, 2), dtype=np.complex128)
    for t in range(T):
        b = uvw[t, p, :] - uvw[t, q, :]                       # [B][3]
        path = (np.outer(b[:, 0], l) + np.outer(b[:, 1], m)
                + np.outer(b[:, 2], n - 1.0))                 # [B][S] metres
        for fi, f in enumerate(freqs):
            spec = (f / f0) ** np.asarray(alpha, dtype=np.float64)          # [S]
            G = gaussian_visibility(b[:, 0:1] * (f / C_LIGHT), b[:, 1:2] * (f / C_LIGHT),
                                    maj, mnr, pa)              # [B][S]
            w = np.exp(-2j * np.pi * (f / C_LIGHT) * path) * G * spec       # [B][S]
            out[t, :, fi] = np.einsum("bs,sij->bij", w, Bs)
    return out


def predict_sky_full(uvw, freqs, sky):
    """Full coherencies of every cluster of a `synth.PolSky`: [K][T][B][F][2][2]."""
    return np.stack([
        predict_coherencies_full(uvw, freqs, sky.l[a:b], sky.m[a:b], sky.I[a:b], sky.Q[a:b],
                                 sky.U[a:b], sky.V[a:b], sky.alpha[a:b], sky.maj[a:b],
                                 sky.mnr[a:b], sky.pa[a:b], sky.f0)
        for a, b in zip(sky.offsets[:-1], sky.offsets[1:])])


# --- measurement equation -----------------------------------------------------

def model_vis(C, J):
    """J_p (C_pq Id) J_q^H for every vis: [T][B][F][2][2]."""
    N = J.shape[0]
    p, q = baselines(N)
    G = J[p] @ np.conj(np.swapaxes(J[q], -1, -2))             # [B][2][2]
    return C[..., None, None] * G[None, :, None, :, :]


def residual(X, C, J):
    """R = X - J_p C J_q^H and cost = sum |R|^2 (squared Frobenius norms)."""
    R = X - model_vis(C, J)
    return R, float(np.sum(R.real ** 2 + R.imag ** 2))


# Threshold of the singular-Jones test of residual_all: a station's Jones J
# counts as singular when |det J| <= SINGULAR_RTOL * |J|_F^2 (|det J| is at
# most |J|_F^2 / 2, with equality for a multiple of a unitary matrix).
SINGULAR_RTOL = 1e-12


def residual_all(V, Cs, J, corr=-1):
    """Residual of the whole sky model after calibration, optionally corrected
    for the gains of one direction (the output that follows the solve: data
    with every calibrated cluster removed, left for imaging).

        R_pq = V_pq - sum_k J_kp (C_kpq Id) J_kq^H
        cost = sum |R|^2                      (before any correction)
        if corr >= 0:  R_pq <- J_cp^{-1} R_pq J_cq^{-H},  c = corr

    Inputs: V [T][B][F][2][2], Cs [K][T][B][F], J [K][N][2][2].  A station
    whose J_c is singular (SINGULAR_RTOL) cannot be corrected: every
    visibility of its baselines is set to zero.  The 2x2 inverse is the
    adjugate over the determinant.  Returns (R, cost, singular [N] bool).
    """
    K, N = J.shape[0], J.shape[1]
    p, q = baselines(N)
    R = np.array(V, dtype=np.complex128)
    for k in range(K):
        R = R - model_vis(Cs[k], J[k])
    cost = float(np.sum(R.real ** 2 + R.imag ** 2))
    singular = np.zeros(N, dtype=bool)
    if corr < 0:
        return R, cost, singular
    Jinv = np.zeros((N, 2, 2), dtype=np.complex128)
    for s in range(N):
        a, b = J[corr, s, 0, 0], J[corr, s, 0, 1]
        c, d = J[corr, s, 1, 0], J[corr, s, 1, 1]
        det = a * d - b * c
        fro2 = abs(a) ** 2 + abs(b) ** 2 + abs(c) ** 2 + abs(d) ** 2
        if abs(det) <= SINGULAR_RTOL * fro2:
            singular[s] = True
            continue
        Jinv[s] = np.array([[d, -b], [-c, a]]) / det
    # J_cp^{-1} R J_cq^{-H}; a singular station has Jinv = 0, so its
    # baselines come out zero
    Lp = Jinv[p][None, :, None, :, :]
    Rq = np.conj(np.swapaxes(Jinv[q], -1, -2))[None, :, None, :, :]
    R = Lp @ R @ Rq
    return R, cost, singular


def simulate(uvw, freqs, sky, J_true, noise=None):
    """V = sum_k model_k + noise, and the coherencies [K][T][B][F]."""
    Cs = predict_sky(uvw, freqs, sky)
    V = sum(model_vis(Cs[k], J_true[k]) for k in range(len(Cs)))
    if noise is not None:
        V = V + noise
    return V, Cs


# --- Jacobian and normal equations ---------------------------------------------

def _unit(i, j, imag):
    E = np.zeros((2, 2), dtype=np.complex128)
    E[i, j] = 1j if imag else 1.0
    return E


def model_jacobian(C, J):
    """Real Jacobian of the model per vis, [T][B][F][8][16].

    Rows: Re of the 4 entries of M = C J_p J_q^H, then Im of the 4 entries.
    Columns: the 8 parameters of J_p, then the 8 of J_q (theta order).  By
    the product rule, dM = C (dJ_p J_q^H + J_p dJ_q^H), with dJ the unit
    change of one real parameter.
    """
    N = J.shape[0]
    p, q = baselines(N)
    Jp, Jq = J[p], J[q]
    JqH = np.conj(np.swapaxes(Jq, -1, -2))
    cols = []
    for side in (0, 1):
        for i in range(2):
            for j in range(2):
                for imag in (0, 1):
                    dJ = _unit(i, j, imag)
                    if side == 0:
                        d = dJ[None] @ JqH                     # dJ_p J_q^H
                    else:
                        d = Jp @ np.conj(dJ.T)[None]           # J_p dJ_q^H
                    cols.append(d.reshape(-1, 4))              # [B][4]
    D = np.stack(cols, axis=-1)                                # [B][4][16]
    dM = C[..., None, None] * D[None, :, None, :, :]           # [T][B][F][4][16]
    return np.concatenate([dM.real, dM.imag], axis=-2)         # [T][B][F][8][16]


def normal_equations(R, C, J, t_chunk=4):
    """Gauss-Newton normal equations A = J^T J ([8N][8N]) and g = J^T r ([8N])
    of the cost sum |X - C J_p J_q^H|^2 at residual R = X - model."""
    N = J.shape[0]
    p, q = baselines(N)
    T = C.shape[0]
    P = 8 * N
    blocks = np.zeros((len(p), 16, 16))
    grads = np.zeros((len(p), 16))
    for t0 in range(0, T, t_chunk):
        Jv = model_jacobian(C[t0:t0 + t_chunk], J)             # [t][B][F][8][16]
        Rt = R[t0:t0 + t_chunk].reshape(*R[t0:t0 + t_chunk].shape[:3], 4)
        r = np.concatenate([Rt.real, Rt.imag], axis=-1)        # [t][B][F][8]
        blocks += np.einsum("tbfrk,tbfrl->bkl", Jv, Jv)
        grads += np.einsum("tbfrk,tbfr->bk", Jv, r)
    A = np.zeros((N, 8, N, 8))
    g = np.zeros((N, 8))
    for b in range(len(p)):
        s = (p[b], q[b])
        for x in range(2):
            g[s[x]] += grads[b, 8 * x:8 * x + 8]
            for y in range(2):
                A[s[x], :, s[y], :] += blocks[b, 8 * x:8 * x + 8, 8 * y:8 * y + 8]
    return A.reshape(P, P), g.reshape(P)


# --- linear algebra -----------------------------------------------------------

def cholesky_solve(A, b):
    """Solve A x = b for symmetric positive definite A: A = L L^T, then
    L y = b and L^T x = y.  Raises numpy.linalg.LinAlgError if A is not PD."""
    L = np.linalg.cholesky(A)
    y = scipy.linalg.solve_triangular(L, b, lower=True)
    return scipy.linalg.solve_triangular(L.T, y, lower=False)


# --- Levenberg-Marquardt ------------------------------------------------------

def levenberg_marquardt(evaluate, theta0, n_iter, tau=1e-3, eps_grad=1e-12,
                        trace=None):
    """Levenberg-Marquardt (Madsen, Nielsen & Tingleff 2004, Alg. 3.16): the
    step d solves (A + mu I) d = g.

    evaluate(theta) -> (cost, A, g): cost = |r|^2, A = J^T J, g = J^T r with
    r = data - model (g is minus half the gradient of the cost).

    mu starts at tau * max diag(A), nu at 2.  Each of the n_iter iterations
    tries one step; the gain ratio rho = (cost - cost_trial) / (d^T (mu d
    + g)) (actual over predicted decrease of the cost |r|^2) accepts it when
    rho > 0 (then mu *= max(1/3, 1 - (2 rho - 1)^3), nu = 2), else mu *= nu,
    nu *= 2.  Iterations stop early once max|g| <= eps_grad * (1 + cost).  A
    damped matrix that is not positive definite (or not finite) counts as a
    rejected step.
    Returns (theta, cost, iterations done).
    """
    theta = np.array(theta0, dtype=np.float64)
    cost, A, g = evaluate(theta)
    mu = tau * float(np.max(np.diag(A)))
    nu = 2.0
    done = 0
    for _ in range(n_iter):
        if float(np.max(np.abs(g))) <= eps_grad * (1.0 + cost):
            break
        done += 1
        try:
            d = cholesky_solve(A + mu * np.eye(len(g)), g)
        except (np.linalg.LinAlgError, ValueError):  # not PD, or mu overflowed
            mu *= nu
            nu *= 2.0
            continue
        trial = theta + d
        cost_t, A_t, g_t = evaluate(trial)
        pred = float(d @ (mu * d + g))
        rho = (cost - cost_t) / pred if pred > 0.0 else -1.0
        if trace is not None:
            trace.append(dict(mu=mu, nu=nu, rho=rho, cost=cost, cost_trial=cost_t))
        if rho > 0.0:
            theta, cost, A, g = trial, cost_t, A_t, g_t
            mu *= max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
            nu = 2.0
        else:
            mu *= nu
            nu *= 2.0
    return theta, cost, done


def penalised(evaluate, a, w):
    """The least-squares problem of `evaluate` with the quadratic penalty
    w |theta - a|^2 added, written as extra residual rows sqrt(w) (a - theta)
    with unit Jacobian: cost + w |theta - a|^2, A + w I, g + w (a - theta)."""
    a = np.asarray(a, dtype=np.float64)

    def ev(theta):
        cost, A, g = evaluate(theta)
        d = theta - a
        return cost + w * float(d @ d), A + w * np.eye(len(theta)), g - w * d
    return ev


def lm_cluster(X, C, J0, n_lm, tau=1e-3, eps_grad=1e-12, trace=None, penalty=None):
    """Solve one cluster: minimise sum |X - C J_p J_q^H|^2 over the Jones,
    plus w |J - A|_F^2 when penalty = (A [N][2][2], w) is given.
    Returns (J, final cost (with the penalty), iterations done)."""
    def evaluate(theta):
        J = theta_to_jones(theta)
        R, cost = residual(X, C, J)
        A, g = normal_equations(R, C, J)
        return cost, A, g
    if penalty is not None:
        evaluate = penalised(evaluate, jones_to_theta(penalty[0]), penalty[1])
    theta, cost, done = levenberg_marquardt(evaluate, jones_to_theta(J0), n_lm,
                                            tau, eps_grad, trace)
    return theta_to_jones(theta), cost, done


# --- SAGE / EM ----------------------------------------------------------------

def sage_calibrate(V, Cs, J0, n_em, n_lm, tau=1e-3, eps_grad=1e-12,
                   sweep_costs=None, penalties=None):
    """SAGE: for each EM iteration and each cluster k in ascending order, the
    E-step forms the data of cluster k, X_k = V - sum_{j != k} model_j, from
    the current solutions of the other clusters; the M-step solves cluster k
    on X_k by LM, warm-started from its current Jones.  penalties[k] =
    (A_k, w), if given, adds w |J_k - A_k|_F^2 to cluster k's LM cost.
    Returns (J [K][N][2][2], final LM cost of each cluster)."""
    K = len(Cs)
    J = np.array(J0, dtype=np.complex128)
    costs = np.zeros(K)
    for _ in range(n_em):
        for k in range(K):
            X = V.copy()
            for j in range(K):
                if j != k:
                    X = X - model_vis(Cs[j], J[j])
            pen = None if penalties is None else penalties[k]
            J[k], costs[k], _ = lm_cluster(X, Cs[k], J[k], n_lm, tau, eps_grad, penalty=pen)
        if sweep_costs is not None:
            R = V - sum(model_vis(Cs[j], J[j]) for j in range(K))
            sweep_costs.append(float(np.sum(R.real ** 2 + R.imag ** 2)))
    return J, costs


def calibrate_chunks(Vs, Css, J0, n_em, n_lm, tau=1e-3, eps_grad=1e-12):
    """Consecutive time chunks of one observation, calibrated in order: chunk
    i runs sage_calibrate on its own data Vs[i] and coherencies Css[i],
    starting from the solution of chunk i-1 (chunk 0 from J0).  The solution
    of each chunk is the solver state carried forward, so restarting at
    chunk i from the solution of chunk i-1 continues the run exactly.
    Returns (J [n][K][N][2][2] per chunk, final LM costs [n][K])."""
    J = np.array(J0, dtype=np.complex128)
    Js, costs = [], []
    for V, Cs in zip(Vs, Css):
        J, c = sage_calibrate(V, Cs, J, n_em, n_lm, tau, eps_grad)
        Js.append(J.copy())
        costs.append(c)
    return np.stack(Js), np.stack(costs)


# --- consensus across sub-bands ------------------------------------------------

def consensus_fit(Y, basis):
    """The consensus step: the smooth frequency model that fits Y best, per
    cluster and real parameter, in the least-squares sense over the bands.
    Y [n_bands][K][N][2][2], basis [n_bands][n_poly]; returns Z
    [K][n_poly][N][2][2] with sum_f |basis[f] Z - Y[f]|^2 minimal, from the
    normal equations (B^T B) Z = B^T Y."""
    B = np.asarray(basis, dtype=np.float64)
    n_bands, n_poly = B.shape
    rhs = np.einsum("fp,fknij->pknij", B, Y)
    Z = np.linalg.solve(B.T @ B, rhs.reshape(n_poly, -1)).reshape(rhs.shape)
    return np.ascontiguousarray(np.moveaxis(Z, 0, 1))


def consensus_model(Z, basis):
    """basis[f] Z for every band: [n_bands][K][N][2][2]."""
    return np.einsum("fp,kpnij->fknij", np.asarray(basis, dtype=np.float64), Z)


def consensus_calibrate(Vs, Css, J0s, basis, rho, n_admm, n_em, n_lm, tau=1e-3, eps_grad=1e-12,
                        U0=None):
    """Sub-band calibrations coupled by a smooth frequency model of the
    Jones: consensus ADMM in scaled form (Boyd et al. 2011, §7.1) on
    sum_f f_f(J_f) subject to J_f = basis[f] Z, with f_f the SAGE cost of
    band f (sum |R|^2 over its data).  Each iteration:

      J-step  every band runs SAGE (n_em sweeps, n_lm LM steps per cluster)
              from its current Jones on f_f(J) + (rho/2) |J - (basis[f] Z - U_f)|^2;
              in the first iteration the bands are calibrated alone (no
              penalty: there is no Z yet);
      Z-step  Z = consensus_fit(J + U, basis);
      U-step  U_f += J_f - basis[f] Z.

    Vs [n_bands] data, Css [n_bands][K][T][B][F] coherencies, J0s
    [n_bands][K][N][2][2] initial Jones, U0 the initial scaled duals (zero
    if None).  Returns (J, Z [K][n_poly][N][2][2], U, costs [n_bands][K]):
    the final LM costs, penalty included."""
    n_bands = len(Vs)
    J = np.array(J0s, dtype=np.complex128)
    U = np.zeros_like(J) if U0 is None else np.array(U0, dtype=np.complex128)
    K, N = J.shape[1], J.shape[2]
    n_poly = np.asarray(basis).shape[1]
    Z = np.zeros((K, n_poly, N, 2, 2), dtype=np.complex128)
    costs = np.zeros((n_bands, K))
    for it in range(n_admm):
        target = consensus_model(Z, basis) - U
        for f in range(n_bands):
            pens = None if it == 0 else [(target[f, k], 0.5 * rho) for k in range(K)]
            J[f], costs[f] = sage_calibrate(Vs[f], Css[f], J[f], n_em, n_lm, tau, eps_grad,
                                            penalties=pens)
        Z = consensus_fit(J + U, basis)
        U = U + J - consensus_model(Z, basis)
    return J, Z, U, costs


# --- comparison up to the unitary ambiguity -----------------------------------

def align_unitary(J, J_ref):
    """Unitary U minimising sum_p |J_p U - J_ref,p|_F^2 (orthogonal
    Procrustes): U = W Z^H from the SVD W S Z^H of sum_p J_p^H J_ref,p.
    J_p -> J_p U leaves every J_p C J_q^H unchanged."""
    M = np.einsum("pji,pjk->ik", np.conj(J), J_ref)
    W, _, Zh = np.linalg.svd(M)
    return W @ Zh


def aligned_error(J, J_ref):
    """max_p |J_p U - J_ref,p|_F / |J_ref,p|_F after Procrustes alignment."""
    U = align_unitary(J, J_ref)
    d = np.linalg.norm(J @ U - J_ref, axis=(1, 2))
    return float(np.max(d / np.linalg.norm(J_ref, axis=(1, 2))))
