"""Pins of the oracle's consensus calibration across sub-bands
(penalised LM, consensus_fit, consensus_calibrate) against facts fixed
from outside the code: the closed form of a penalised linear least-squares
problem and the finite-difference derivatives of its cost, numpy's
least-squares solver, the invariant that scaled-form ADMM keeps the duals
orthogonal to the frequency model after every Z-step, the optimality
condition of a converged J-step written with the updated duals, the fixed
point at the true solution, and two statistical consequences.

Planted mistakes each of these catches (checked by substituting each into
the oracle): the penalty gradient with the wrong sign, the penalty left out
of the damped matrix, the penalty weight rho instead of rho/2 in the
J-step, the target basis[f] Z + U instead of basis[f] Z - U, the dual update
with the wrong sign, the fit without the normal matrix (B^T Y alone), the
basis rows taken in reverse band order in the model.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def bands(N=12, T=2, F=1, K=1, S=4, n_bands=4, sigma=0.0, drift=0.02, seed=3):
    """n_bands sub-bands of one observation: same stations, timeslots and
    sky; true Jones linear in the normalised frequency; independent noise."""
    spec = synth.JobSpec(N=N, T=T, F=F, K=K, S=S, seed=seed, sigma=sigma)
    fr, centres = synth.sub_bands(spec, n_bands)
    uvw, sky = synth.station_uvw(spec), synth.sky(spec)
    Jt = synth.jones_true_bands(spec, centres, drift_var=drift)
    Vs, Css = [], []
    for f in range(n_bands):
        Cs = O.predict_sky(uvw, fr[f], sky)
        V = sum(O.model_vis(Cs[k], Jt[f, k]) for k in range(K))
        if sigma > 0:
            V = V + synth.noise(dataclasses.replace(spec, seed=seed * 100 + f))
        Vs.append(V)
        Css.append(Cs)
    return spec, centres, Vs, Css, Jt


def identity(spec, n):
    return np.stack([synth.identity_jones(spec.K, spec.N)] * n)


def test_penalised_lm_reaches_the_closed_form_of_a_linear_problem():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(30, 6))
    b = rng.normal(size=30)
    a = rng.normal(size=6)
    w = 3.7

    def evaluate(th):
        r = b - A @ th
        return float(r @ r), A.T @ A, A.T @ r
    th, cost, _ = O.levenberg_marquardt(O.penalised(evaluate, a, w), np.zeros(6), 60, eps_grad=0.0)
    ref = np.linalg.solve(A.T @ A + w * np.eye(6), A.T @ b + w * a)
    np.testing.assert_allclose(th, ref, rtol=0, atol=1e-10)
    r = b - A @ ref
    assert abs(cost - (r @ r + w * np.sum((ref - a) ** 2))) < 1e-10


def test_a_heavy_penalty_holds_the_jones_at_its_target():
    spec, centres, Vs, Css, Jt = bands(n_bands=1, sigma=0.01)
    target = Jt[0, 0] * np.exp(0.3j)                 # a target the data disagree with
    J, cost, _ = O.lm_cluster(Vs[0], Css[0][0], synth.identity_jones(1, spec.N)[0], 15,
                              penalty=(target, 1e9))
    assert np.abs(J - target).max() < 1e-4


def test_consensus_fit_is_least_squares_per_parameter():
    rng = np.random.default_rng(4)
    n_bands, n_poly, K, N = 7, 3, 2, 5
    B = synth.frequency_basis(np.linspace(120e6, 180e6, n_bands), n_poly)
    Y = rng.normal(size=(n_bands, K, N, 2, 2)) + 1j * rng.normal(size=(n_bands, K, N, 2, 2))
    Z = O.consensus_fit(Y, B)
    assert Z.shape == (K, n_poly, N, 2, 2)
    flat = Y.reshape(n_bands, -1)
    ref = np.linalg.lstsq(B, flat.real, rcond=None)[0] + 1j * np.linalg.lstsq(B, flat.imag, rcond=None)[0]
    np.testing.assert_allclose(np.moveaxis(Z, 1, 0).reshape(n_poly, -1), ref, atol=1e-12)
    # data that is exactly a polynomial of the basis is reproduced
    Zt = rng.normal(size=(K, n_poly, N, 2, 2)) + 0j
    np.testing.assert_allclose(O.consensus_fit(O.consensus_model(Zt, B), B), Zt, atol=1e-12)


def test_duals_stay_orthogonal_to_the_frequency_model():
    """After each Z-step the scaled duals satisfy sum_f basis[f] U_f = 0
    (the optimality condition of the Z-step rewritten with the new duals)."""
    spec, centres, Vs, Css, Jt = bands(n_bands=5, sigma=0.3, seed=5)
    B = synth.frequency_basis(centres, 2)
    for n_admm in (1, 3):
        J, Z, U, _ = O.consensus_calibrate(Vs, Css, identity(spec, 5), B, 30.0, n_admm, 1, 6)
        assert np.abs(np.einsum("fp,fknij->pknij", B, U)).max() < 1e-12
        assert np.abs(U).max() > 1e-3                 # the duals themselves are not zero


def test_zero_rho_is_independent_sage_per_band():
    spec, centres, Vs, Css, Jt = bands(n_bands=3, sigma=0.05, K=2, S=3)
    B = synth.frequency_basis(centres, 2)
    J0 = identity(spec, 3)
    J, Z, U, costs = O.consensus_calibrate(Vs, Css, J0, B, 0.0, 2, 1, 5)
    for f in range(3):
        Jf, cf = O.sage_calibrate(Vs[f], Css[f], J0[f], 2, 5)
        np.testing.assert_array_equal(J[f], Jf)
        np.testing.assert_array_equal(costs[f], cf)


def test_the_true_solution_is_a_fixed_point():
    """Noiseless data whose Jones are linear in the basis: started at the
    truth with zero duals, every penalty and gradient vanishes, so nothing
    moves, and Z is the true frequency model."""
    spec, centres, Vs, Css, Jt = bands(n_bands=4)
    B = synth.frequency_basis(centres, 2)
    J, Z, U, costs = O.consensus_calibrate(Vs, Css, Jt, B, 10.0, 3, 1, 5)
    np.testing.assert_allclose(J, Jt, atol=1e-12)
    np.testing.assert_allclose(O.consensus_model(Z, B), Jt, atol=1e-12)
    assert np.abs(U).max() < 1e-12
    assert costs.max() < 1e-20


def test_consensus_lowers_the_error_of_noisy_sub_band_solutions():
    spec, centres, Vs, Css, Jt = bands(n_bands=6, sigma=1.0, seed=5)
    B = synth.frequency_basis(centres, 2)
    J0 = identity(spec, 6)

    def err(J):
        return np.mean([O.aligned_error(J[f, 0], Jt[f, 0]) for f in range(6)])
    J_ind, Z0, _, _ = O.consensus_calibrate(Vs, Css, J0, B, 0.0, 6, 1, 10)
    J_con, Z1, _, _ = O.consensus_calibrate(Vs, Css, J0, B, 300.0, 6, 1, 10)
    assert err(J_con) < 0.85 * err(J_ind)
    # and the bands agree with one smooth model more closely
    assert np.linalg.norm(J_con - O.consensus_model(Z1, B)) < 0.8 * np.linalg.norm(J_ind - O.consensus_model(Z0, B))


def test_penalised_problem_has_the_derivatives_of_its_cost():
    """For linear residuals, g is minus half the gradient and A half the
    Hessian of the penalised cost: checked by central differences."""
    rng = np.random.default_rng(8)
    A = rng.normal(size=(20, 5))
    b = rng.normal(size=20)
    a = rng.normal(size=5)
    w = 2.5

    def evaluate(th):
        r = b - A @ th
        return float(r @ r), A.T @ A, A.T @ r
    ev = O.penalised(evaluate, a, w)
    th = rng.normal(size=5)
    cost, H, g = ev(th)
    h = 1e-5
    E = np.eye(5)
    grad = np.array([(ev(th + h * e)[0] - ev(th - h * e)[0]) / (2 * h) for e in E])
    np.testing.assert_allclose(-0.5 * grad, g, rtol=0, atol=1e-7)
    hess = np.array([[(ev(th + h * (ei + ej))[0] - ev(th + h * (ei - ej))[0] - ev(th - h * (ei - ej))[0]
                       + ev(th - h * (ei + ej))[0]) / (4 * h * h) for ej in E] for ei in E])
    np.testing.assert_allclose(0.5 * hess, H, rtol=0, atol=1e-4)


def test_j_step_optimality_links_the_gradient_to_the_duals():
    """When each J-step's LM has converged, its optimality condition
    g_data(J_f) = (rho/2) (J_f - basis[f] Z_old + U_old) becomes, with the
    updated duals, g_data(J_f) = (rho/2) (U_f + basis[f] (Z_new - Z_old)):
    this fixes the penalty weight rho/2, the target basis[f] Z - U and the
    sign of the dual update."""
    spec, centres, Vs, Css, Jt = bands(n_bands=4, sigma=0.05, seed=6)
    B = synth.frequency_basis(centres, 2)
    rho = 40.0
    J0 = identity(spec, 4)
    _, Z1, _, _ = O.consensus_calibrate(Vs, Css, J0, B, rho, 1, 1, 40, eps_grad=0.0)
    J2, Z2, U2, _ = O.consensus_calibrate(Vs, Css, J0, B, rho, 2, 1, 40, eps_grad=0.0)
    dZ = O.consensus_model(Z2 - Z1, B)
    for f in range(4):
        R, _ = O.residual(Vs[f], Css[f][0], J2[f, 0])
        _, g = O.normal_equations(R, Css[f][0], J2[f, 0])
        rhs = 0.5 * rho * O.jones_to_theta(U2[f, 0] + dZ[f, 0])
        np.testing.assert_allclose(g, rhs, rtol=0, atol=1e-7 * max(1.0, np.abs(rhs).max()))
