"""The seeded input generator: published PRNG vector, determinism, geometry."""
import math
import os

import numpy as np

from paper_1910_13908_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    want = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    i = np.arange(1, 6, dtype=np.uint64)
    with np.errstate(over="ignore"):
        got = synth._mix64(np.uint64(1234567) + i * synth._GAMMA)
    assert [int(v) for v in got] == want


def test_streams_are_deterministic_and_drawable_in_pieces():
    spec = synth.JobSpec(N=9, T=6, F=3, seed=42)
    a = synth.noise(spec)
    assert np.array_equal(a[2:5], synth.noise(spec, 2, 5))
    assert np.array_equal(synth.jones_true(spec), synth.jones_true(spec))
    u = synth.uniform(1, 2, 100000)
    assert 0.0 < u.min() and u.max() <= 1.0 and abs(u.mean() - 0.5) < 0.005
    z = synth.normal(1, 3, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_layout_and_sky_ranges():
    spec = synth.config("c2")
    enu = synth.stations_enu(spec)
    assert np.all(np.hypot(enu[:, 0], enu[:, 1]) <= spec.radius_m)
    sky = synth.sky(spec)
    assert sky.K == 10 and sky.offsets[-1] == 250
    assert sky.flux.min() >= 0.1 and sky.flux.max() <= 10.0
    assert np.all(np.hypot(sky.l, sky.m) < math.sin(math.radians(5.5)))
    f = synth.freqs(spec)
    assert len(f) == 8 and f[0] > 140e6 and f[-1] < 160e6


def test_uvw_is_a_rotation_of_the_station_positions():
    spec = synth.JobSpec(N=12, T=5)
    xyz = synth.enu_to_xyz(synth.stations_enu(spec), math.radians(spec.lat_deg))
    uvw = synth.station_uvw(spec)
    for t in range(spec.T):
        np.testing.assert_allclose(np.linalg.norm(uvw[t], axis=1),
                                   np.linalg.norm(xyz, axis=1), rtol=1e-12)


def test_uneven_time_chunks_span_the_range():
    T = synth.uneven_time_chunks(2000, 5, 40)
    assert T.min() == 5 and T.max() == 40


def test_polarised_sky_recipe():
    spec = synth.JobSpec(N=8, T=2, F=2, K=4, S=250, seed=9)
    base, s = synth.sky(spec), synth.sky_pol(spec)
    # same directions, Stokes I and spectral indices as the point-source sky
    for a, b in (("l", "l"), ("m", "m"), ("flux", "I"), ("alpha", "alpha")):
        assert np.array_equal(getattr(base, a), getattr(s, b))
    p_lin = np.hypot(s.Q, s.U) / s.I
    assert p_lin.max() <= 0.2 + 1e-12 and p_lin.mean() > 0.05
    assert np.abs(s.V / s.I).max() <= 0.02 + 1e-12
    ext = (s.maj > 0)
    assert abs(ext.mean() - 0.3) < 0.05                      # 1000 sources, 30% extended
    arcmin = math.radians(1 / 60)
    assert s.maj[ext].min() >= 0.2 * arcmin - 1e-15 and s.maj.max() <= 2.0 * arcmin + 1e-15
    assert np.all(s.mnr <= s.maj) and np.all(s.mnr[ext] >= 0.3 * s.maj[ext] - 1e-18)
    assert np.all(s.mnr[~ext] == 0) and np.all(s.pa[~ext] == 0)
    assert np.all((s.pa >= 0) & (s.pa <= np.pi))
    c = s.cluster(2)
    assert np.array_equal(c.I, s.I[500:750]) and list(c.offsets) == [0, 250]
    assert np.array_equal(synth.sky_pol(spec).Q, s.Q)       # deterministic


def test_sub_bands_basis_and_drifting_jones():
    spec = synth.JobSpec(N=6, T=2, F=3, K=2, S=3, seed=4)
    fr, centres = synth.sub_bands(spec, 5)
    assert fr.shape == (5, 3) and np.all(np.diff(fr.ravel()) > 0)      # tiles the band in order
    assert fr.min() > 115e6 and fr.max() < 185e6
    np.testing.assert_allclose(fr.mean(axis=1), centres)
    B = synth.frequency_basis(centres, 3)
    x = (centres - 150e6) / 35e6
    np.testing.assert_allclose(B, np.stack([np.ones(5), x, x * x], 1))
    assert np.all(np.abs(B[:, 1]) < 1)
    J = synth.jones_true_bands(spec, centres)
    assert J.shape == (5, spec.K, spec.N, 2, 2)
    # linear in x: second differences vanish on the equally spaced centres
    np.testing.assert_allclose(J[2:] - 2 * J[1:-1] + J[:-2], 0, atol=1e-12)
    # at the band centre (x = 0) it is the single-band truth
    np.testing.assert_allclose(synth.jones_true_bands(spec, [150e6])[0], synth.jones_true(spec), atol=0)
