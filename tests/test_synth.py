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
