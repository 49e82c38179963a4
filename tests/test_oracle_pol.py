"""Pins of the oracle's polarised and extended-source prediction
(predict_coherencies_full, brightness_matrix, gaussian_visibility) against
facts fixed from outside the formulas: the already pinned point-source
prediction, a brute-force quadrature of the Fourier integral of a Gaussian
brightness, the transformation of Stokes parameters under a rotation of the
feeds, and the symmetries of a Hermitian coherency.

Planted mistakes each of these catches: sigma taken as the FWHM or as the
half width, 2 pi^2 written pi^2, the position angle measured from +l instead
of +m, the axes swapped, Q placed off the diagonal, V placed on the diagonal,
a missing spectral factor on Q/U/V, B transposed (U - iV above the diagonal
with the layout of Hermitian swap), the Gaussian evaluated in metres.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def spec_(**kw):
    base = dict(N=7, T=3, F=3, K=1, S=6, f_lo=120e6, f_hi=180e6, seed=5, alpha=-0.7)
    base.update(kw)
    return synth.JobSpec(**base)


def full(uvw, f, s, f0=150e6):
    return O.predict_coherencies_full(uvw, f, s.l, s.m, s.I, s.Q, s.U, s.V, s.alpha, s.maj, s.mnr,
                                      s.pa, f0)


def test_unpolarised_point_sky_is_the_scalar_prediction_times_identity():
    spec = spec_()
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    sk = synth.sky(spec)
    z = np.zeros_like(sk.flux)
    C = O.predict_coherencies(uvw, f, sk.l, sk.m, sk.flux, sk.alpha)
    Cf = O.predict_coherencies_full(uvw, f, sk.l, sk.m, sk.flux, z, z, z, sk.alpha, z, z, z)
    assert Cf.shape == C.shape + (2, 2)
    np.testing.assert_allclose(Cf, C[..., None, None] * np.eye(2), rtol=0, atol=1e-12)


@pytest.mark.parametrize("maj_arcmin,mnr_arcmin,pa_deg", [(1.5, 0.6, 30.0), (2.0, 2.0, 0.0),
                                                          (1.0, 0.3, 115.0)])
def test_gaussian_visibility_equals_the_fourier_integral(maj_arcmin, mnr_arcmin, pa_deg):
    """Lay the brightness exp(-(x_a^2/sigma_a^2 + x_b^2/sigma_b^2)/2) out on a
    fine (l, m) grid, with x_a the coordinate along (sin pa, cos pa) and
    sigma the FWHM over 2 sqrt(2 ln 2) read from the Gaussian's own
    half-maximum, and sum its Fourier integral directly."""
    maj, mnr, pa = math.radians(maj_arcmin / 60), math.radians(mnr_arcmin / 60), math.radians(pa_deg)
    # sigma from the half-maximum condition exp(-x^2 / (2 s^2)) = 1/2 at x = FWHM / 2
    sa = (maj / 2) / math.sqrt(2 * math.log(2))
    sb = (mnr / 2) / math.sqrt(2 * math.log(2))
    n = 801
    x = np.linspace(-9 * sa, 9 * sa, n)
    h = x[1] - x[0]
    L, M = np.meshgrid(x, x, indexing="ij")
    xa = L * math.sin(pa) + M * math.cos(pa)
    xb = L * math.cos(pa) - M * math.sin(pa)
    img = np.exp(-0.5 * (xa ** 2 / sa ** 2 + xb ** 2 / sb ** 2))
    img /= img.sum() * h * h                                  # unit flux
    rng = np.random.default_rng(7)
    for _ in range(6):
        # baselines where the visibility is between ~1e-3 and ~1
        r = rng.uniform(0.05, 0.45) / sa
        th = rng.uniform(0, 2 * np.pi)
        u, v = r * math.cos(th), r * math.sin(th)
        ref = np.sum(img * np.exp(-2j * np.pi * (u * L + v * M))) * h * h
        got = O.gaussian_visibility(u, v, maj, mnr, pa)
        assert abs(ref.imag) < 1e-12
        assert abs(got - ref.real) < 1e-10 * max(1.0, abs(ref.real)), (u, v, got, ref)


def test_zero_size_gaussian_is_a_point_and_a_gaussian_only_attenuates():
    spec = spec_()
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    s = synth.sky_pol(spec, frac_extended=0.0)
    assert np.all(s.maj == 0)
    C_pt = full(uvw, f, s)
    s_ext = synth.sky_pol(spec, frac_extended=1.0)
    # same sources, every one extended: each term shrinks by its G in (0, 1]
    one = dict(I=[1.0], Q=[0.0], U=[0.0], V=[0.0], alpha=[0.0])
    for k in range(len(s.l)):
        a = O.predict_coherencies_full(uvw, f, [s.l[k]], [s.m[k]], **one, maj=[0.0], mnr=[0.0], pa=[0.0])
        b = O.predict_coherencies_full(uvw, f, [s.l[k]], [s.m[k]], **one, maj=[s_ext.maj[k]],
                                       mnr=[s_ext.mnr[k]], pa=[s_ext.pa[k]])
        ratio = b[..., 0, 0] / a[..., 0, 0]
        assert np.all(np.abs(ratio.imag) < 1e-12)
        assert np.all((ratio.real > 0) & (ratio.real <= 1 + 1e-15))
        # longer baselines are attenuated more: compare within one timeslot and channel
        bl = np.linalg.norm(uvw[0][O.baselines(spec.N)[0]] - uvw[0][O.baselines(spec.N)[1]], axis=1)
        order = np.argsort(bl)
        if s_ext.maj[k] == s_ext.mnr[k]:
            assert np.all(np.diff(ratio[0, order, 0].real) <= 1e-15)
    assert np.isfinite(C_pt).all()


def test_feed_rotation_mixes_q_and_u_by_twice_the_angle():
    """Feeds turned by chi see E' = R E with R = [[c, s], [-s, c]]: the
    coherency becomes R B R^T, and in the turned frame the polarisation angle
    is chi_pol - chi: I and V stay, (Q, U) rotate by -2 chi."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        I = rng.uniform(1, 3)
        Q, U, V = rng.uniform(-0.5, 0.5, 3)
        chi = rng.uniform(-np.pi, np.pi)
        c, s = math.cos(chi), math.sin(chi)
        R = np.array([[c, s], [-s, c]])
        B = O.brightness_matrix(I, Q, U, V)
        Q2 = Q * math.cos(2 * chi) + U * math.sin(2 * chi)
        U2 = U * math.cos(2 * chi) - Q * math.sin(2 * chi)
        np.testing.assert_allclose(R @ B @ R.T, O.brightness_matrix(I, Q2, U2, V), atol=1e-14)


def test_brightness_matrix_invariants():
    """Hermitian; trace 2I; det I^2 - Q^2 - U^2 - V^2; positive semidefinite
    exactly when the polarised flux does not exceed I; a fully circular
    source (V = I) is rank one with the circular feed vector as its range."""
    rng = np.random.default_rng(11)
    I = rng.uniform(0.5, 2, 50)
    Q, U, V = rng.uniform(-1, 1, (3, 50))
    B = O.brightness_matrix(I, Q, U, V)
    np.testing.assert_allclose(B, np.conj(np.swapaxes(B, -1, -2)), atol=0)
    np.testing.assert_allclose(np.trace(B, axis1=-2, axis2=-1), 2 * I, atol=1e-15)
    np.testing.assert_allclose(np.linalg.det(B), I ** 2 - Q ** 2 - U ** 2 - V ** 2, atol=1e-12)
    ev = np.linalg.eigvalsh(B)
    pol = np.sqrt(Q ** 2 + U ** 2 + V ** 2)
    np.testing.assert_allclose(np.sort(ev, axis=-1), np.stack([I - pol, I + pol], -1), atol=1e-12)
    Bc = O.brightness_matrix(1.0, 0.0, 0.0, 1.0)
    e = np.array([1.0, -1j]) / math.sqrt(2)                   # B e = 2 e
    np.testing.assert_allclose(Bc @ e, 2 * e, atol=1e-15)


def test_swapping_stations_gives_the_conjugate_transpose():
    spec = spec_()
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    s = synth.sky_pol(spec, frac_extended=0.5, max_circ_pol=0.3)
    C = full(uvw, f, s)
    Cr = full(uvw[:, ::-1, :], f, s)
    N = spec.N
    p, q = O.baselines(N)
    rb = {(a, b): i for i, (a, b) in enumerate(zip(p, q))}
    idx = [rb[(N - 1 - q[i], N - 1 - p[i])] for i in range(len(p))]
    np.testing.assert_allclose(Cr[:, idx], np.conj(np.swapaxes(C, -1, -2)), atol=1e-12)


def test_linear_in_sources_and_spectral_law_on_every_stokes_parameter():
    spec = spec_(S=5)
    uvw, f = synth.station_uvw(spec), synth.freqs(spec)
    s = synth.sky_pol(spec, frac_extended=0.5, max_circ_pol=0.2)
    C = full(uvw, f, s)
    parts = sum(O.predict_coherencies_full(uvw, f, *[[getattr(s, a)[k]] for a in
                                                     ("l", "m", "I", "Q", "U", "V", "alpha", "maj", "mnr",
                                                      "pa")]) for k in range(len(s.l)))
    np.testing.assert_allclose(C, parts, atol=1e-12)
    # at the phase centre, zero size: C(f) = (f/f0)^alpha B exactly, for each channel
    B = O.brightness_matrix(2.0, 0.3, -0.4, 0.1)
    C0 = O.predict_coherencies_full(uvw, f, [0.0], [0.0], [2.0], [0.3], [-0.4], [0.1], [-0.7], [0.0],
                                    [0.0], [0.0])
    for fi, fr in enumerate(f):
        np.testing.assert_allclose(C0[:, :, fi], np.broadcast_to((fr / 150e6) ** -0.7 * B, C0[:, :, fi].shape),
                                   rtol=1e-14)


def test_extended_source_depends_on_baseline_length_in_wavelengths():
    """The same source seen at twice the frequency on a baseline of half the
    length has the same Gaussian attenuation (u f / c is all that matters)."""
    maj, mnr, pa = math.radians(1.2 / 60), math.radians(0.5 / 60), 0.7
    uvw = np.zeros((1, 3, 3))
    uvw[0, 1] = [800.0, -300.0, 5.0]
    uvw[0, 2] = [400.0, -150.0, 2.5]                         # baseline (0, 2) is half of (0, 1)
    C = O.predict_coherencies_full(uvw, [100e6, 200e6], [0.0], [0.0], [1.0], [0.0], [0.0], [0.0], [0.0],
                                   [maj], [mnr], [pa])
    # baseline order: (0,1), (0,2), (1,2)
    np.testing.assert_allclose(C[0, 0, 0, 0, 0], C[0, 1, 1, 0, 0], rtol=1e-14)
