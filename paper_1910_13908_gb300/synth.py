"""Seeded synthetic inputs for direction-dependent calibration runs.

This module only *draws inputs*: station layouts, the projected station
coordinates (u, v, w) of each timeslot, clustered point-source sky models,
"true" Jones matrices and thermal noise.  It holds none of the calibration
arithmetic (no coherency prediction, no residuals, no solver): both the FP64
CPU oracle and the CUDA path receive exactly the same arrays from here.

The paper benchmarks SAGECal on five artificial datasets of 64, 128, 256, 384
and 512 stations with several cluster counts (paper §2, §3); the datasets
themselves are not published, so the recipe below stands in for them:

* stations uniform in a 3 km radius disc, local ENU frame, zero height;
* Earth-rotation synthesis at array latitude 52.9 deg, phase centre at
  declination +52 deg, timeslots 10 s apart centred on transit;
* sky: point sources, flux log-uniform in [0.1, 10] Jy at 150 MHz,
  unpolarised; one cluster: (l, m) uniform in a 3 deg disc; several
  clusters: centres uniform in a 5 deg disc, sources within 0.5 deg;
* true Jones J = I + CN(0, 0.1) per station, per cluster;
* noise: N(0, sigma^2) on the real and imaginary part of each correlation.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea &
Flood 2014: state_i = seed + i * 0x9E3779B97F4A7C15, output = mix(state_i))
with Box-Muller for normals, so every array is bit-identical on x86 and Arm
and independent of numpy's own generators.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# --- counter-based SplitMix64 -------------------------------------------------

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags, one per kind of quantity
TAG_STATIONS = 1
TAG_SKY = 2
TAG_JONES = 3
TAG_NOISE = 4
TAG_CENTRES = 5
TAG_JOBS = 6
TAG_POL = 7
TAG_BANDS = 8


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def raw_u64(seed: int, tag: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 for stream (seed, tag), starting at `offset`."""
    base = np.uint64(((seed & 0xFFFFFFFF) << 32) ^ (tag & 0xFFFFFFFF))
    base = _mix64(np.array([base], dtype=np.uint64))[0]
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(base + i * _GAMMA)


def uniform(seed: int, tag: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1]: (top 53 bits + 1) * 2^-53."""
    u = raw_u64(seed, tag, n, offset)
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, tag: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller, two per pair of uniforms.

    `offset` is the index of the first normal of the stream (even), so that
    a stream can be drawn in pieces.
    """
    assert offset % 2 == 0
    m = (n + 1) // 2
    u = uniform(seed, tag, 2 * m, offset)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[:n]


# --- configuration ------------------------------------------------------------

C_LIGHT = 299792458.0          # m/s
OMEGA_EARTH = 7.2921159e-5     # rad/s, sidereal rotation rate
F0 = 150e6                     # reference frequency of the fluxes, Hz


@dataclasses.dataclass
class JobSpec:
    """Shape of one calibration job (one sub-band x time chunk)."""
    N: int = 64                 # stations
    T: int = 10                 # timeslots
    F: int = 1                  # channels
    K: int = 1                  # clusters (calibration directions)
    S: int = 20                 # sources per cluster
    f_lo: float = 150e6         # band edges, Hz; channel centres between them
    f_hi: float = 150e6
    alpha: float = 0.0          # spectral index of every source
    radius_m: float = 3000.0    # array radius
    lat_deg: float = 52.9
    dec_deg: float = 52.0
    dt_s: float = 10.0
    sigma: float = 0.01         # noise per real/imag component, Jy
    jones_var: float = 0.1      # variance of the complex perturbation of J
    seed: int = 0

    @property
    def B(self) -> int:
        return self.N * (self.N - 1) // 2


# The five workloads of the study, sized like the paper's datasets (§2, §3).
def config(name: str, seed: int = 0) -> JobSpec:
    if name == "c1":   # plain FP64, LOFAR-like 64 stations, one direction
        return JobSpec(N=64, T=10, F=1, K=1, S=20, seed=seed)
    if name == "c2":   # precision path, 128 stations, 10 directions, 8 channels
        return JobSpec(N=128, T=20, F=8, K=10, S=25, f_lo=140e6, f_hi=160e6,
                       alpha=-0.7, seed=seed)
    if name == "c3":   # one sub-band job of the batched workload (T set per job)
        return JobSpec(N=256, T=20, F=1, K=20, S=50, seed=seed)
    if name == "c4":   # SKA1-LOW scale, 512 stations, 40 directions
        return JobSpec(N=512, T=10, F=4, K=40, S=100, f_lo=140e6, f_hi=160e6,
                       seed=seed)
    raise KeyError(name)


def freqs(spec: JobSpec) -> np.ndarray:
    """Channel centres: F equal channels spanning [f_lo, f_hi]."""
    if spec.F == 1 or spec.f_hi == spec.f_lo:
        return np.full(spec.F, 0.5 * (spec.f_lo + spec.f_hi))
    width = (spec.f_hi - spec.f_lo) / spec.F
    return spec.f_lo + width * (np.arange(spec.F) + 0.5)


def stations_enu(spec: JobSpec) -> np.ndarray:
    """[N][3] east, north, up (m): uniform in a disc of radius radius_m."""
    u = uniform(spec.seed, TAG_STATIONS, 2 * spec.N)
    r = spec.radius_m * np.sqrt(u[0::2])
    th = 2.0 * np.pi * u[1::2]
    enu = np.zeros((spec.N, 3))
    enu[:, 0] = r * np.cos(th)
    enu[:, 1] = r * np.sin(th)
    return enu


def enu_to_xyz(enu: np.ndarray, lat_rad: float) -> np.ndarray:
    """Local ENU -> equatorial (X towards H=0, Y towards H=-6h, Z to the pole)."""
    e, n, up = enu[:, 0], enu[:, 1], enu[:, 2]
    sl, cl = math.sin(lat_rad), math.cos(lat_rad)
    return np.stack([-sl * n + cl * up, e, cl * n + sl * up], axis=1)


def hour_angles(spec: JobSpec) -> np.ndarray:
    return (np.arange(spec.T) - 0.5 * (spec.T - 1)) * spec.dt_s * OMEGA_EARTH


def station_uvw(spec: JobSpec) -> np.ndarray:
    """[T][N][3] station (u, v, w) in metres (Thompson, Moran & Swenson 4.1).

    The (u, v, w) of baseline pq is uvw[t, p] - uvw[t, q].
    """
    xyz = enu_to_xyz(stations_enu(spec), math.radians(spec.lat_deg))
    d = math.radians(spec.dec_deg)
    sd, cd = math.sin(d), math.cos(d)
    out = np.empty((spec.T, spec.N, 3))
    for t, h in enumerate(hour_angles(spec)):
        sh, ch = math.sin(h), math.cos(h)
        X, Y, Z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        out[t, :, 0] = sh * X + ch * Y
        out[t, :, 1] = -sd * ch * X + sd * sh * Y + cd * Z
        out[t, :, 2] = cd * ch * X - cd * sh * Y + sd * Z
    return out


@dataclasses.dataclass
class Sky:
    """Point sources sorted by cluster: sources of cluster k are
    [offsets[k], offsets[k+1])."""
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray      # Jy at f0
    alpha: np.ndarray     # spectral index
    offsets: np.ndarray   # int32 [K+1]
    f0: float = F0

    @property
    def K(self) -> int:
        return len(self.offsets) - 1

    def cluster(self, k: int) -> "Sky":
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        return Sky(self.l[a:b], self.m[a:b], self.flux[a:b], self.alpha[a:b],
                   np.array([0, b - a], dtype=np.int32), self.f0)


def sky(spec: JobSpec, sources_per_cluster=None) -> Sky:
    K = spec.K
    counts = (np.full(K, spec.S, dtype=np.int64) if sources_per_cluster is None
              else np.asarray(sources_per_cluster, dtype=np.int64))
    offsets = np.zeros(K + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(counts)
    S = int(offsets[-1])
    u = uniform(spec.seed, TAG_SKY, 3 * S).reshape(S, 3)
    if K == 1:
        r = math.sin(math.radians(3.0)) * np.sqrt(u[:, 0])
        th = 2.0 * np.pi * u[:, 1]
        l, m = r * np.cos(th), r * np.sin(th)
    else:
        uc = uniform(spec.seed, TAG_CENTRES, 2 * K).reshape(K, 2)
        rc = math.sin(math.radians(5.0)) * np.sqrt(uc[:, 0])
        lc, mc = rc * np.cos(2 * np.pi * uc[:, 1]), rc * np.sin(2 * np.pi * uc[:, 1])
        cl = np.repeat(np.arange(K), counts)
        r = math.sin(math.radians(0.5)) * np.sqrt(u[:, 0])
        th = 2.0 * np.pi * u[:, 1]
        l, m = lc[cl] + r * np.cos(th), mc[cl] + r * np.sin(th)
    flux = 10.0 ** (-1.0 + 2.0 * u[:, 2])
    alpha = np.full(S, spec.alpha)
    return Sky(l, m, flux, alpha, offsets)


@dataclasses.dataclass
class PolSky:
    """Polarised and extended sources sorted by cluster (offsets as in Sky).

    Per source: direction (l, m); Stokes I, Q, U, V in Jy at f0, all scaled
    by (f/f0)^alpha; an elliptical Gaussian shape with full widths at half
    maximum maj >= mnr (radians) and the position angle pa (radians, of the
    major axis, from +m towards +l); maj = mnr = 0 is a point source."""
    l: np.ndarray
    m: np.ndarray
    I: np.ndarray
    Q: np.ndarray
    U: np.ndarray
    V: np.ndarray
    alpha: np.ndarray
    maj: np.ndarray
    mnr: np.ndarray
    pa: np.ndarray
    offsets: np.ndarray
    f0: float = F0

    @property
    def K(self) -> int:
        return len(self.offsets) - 1

    def cluster(self, k: int) -> "PolSky":
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        cut = {f.name: getattr(self, f.name)[a:b] for f in dataclasses.fields(self)
               if f.name not in ("offsets", "f0")}
        return PolSky(**cut, offsets=np.array([0, b - a], dtype=np.int32), f0=self.f0)


def sky_pol(spec: JobSpec, sources_per_cluster=None, frac_extended=0.3, max_lin_pol=0.2,
            max_circ_pol=0.02, fwhm_arcmin=(0.2, 2.0)) -> PolSky:
    """The sky of sky(spec) (same directions, I = flux, alpha), with
    polarisation and shapes added: linear polarisation fraction uniform in
    [0, max_lin_pol] at a uniform angle chi (Q = p I cos 2chi, U = p I sin
    2chi), circular fraction uniform in [-max_circ_pol, max_circ_pol]; each
    source extended with probability frac_extended, its major FWHM uniform
    in fwhm_arcmin, minor = major x U(0.3, 1), position angle U(0, pi)."""
    base = sky(spec, sources_per_cluster)
    S = len(base.l)
    u = uniform(spec.seed, TAG_POL, 7 * S).reshape(S, 7)
    I = base.flux
    p_lin = max_lin_pol * u[:, 0]
    chi = np.pi * u[:, 1]
    Q, U = p_lin * I * np.cos(2 * chi), p_lin * I * np.sin(2 * chi)
    V = max_circ_pol * (2 * u[:, 2] - 1) * I
    ext = u[:, 3] < frac_extended
    lo, hi = (math.radians(a / 60.0) for a in fwhm_arcmin)
    maj = np.where(ext, lo + (hi - lo) * u[:, 4], 0.0)
    mnr = maj * (0.3 + 0.7 * u[:, 5])
    pa = np.where(ext, np.pi * u[:, 6], 0.0)
    return PolSky(base.l, base.m, I, Q, U, V, base.alpha, maj, mnr, pa, base.offsets, base.f0)


def jones_true(spec: JobSpec) -> np.ndarray:
    """[K][N][2][2] complex128: I + CN(0, jones_var) per entry."""
    z = normal(spec.seed, TAG_JONES, 2 * 4 * spec.K * spec.N)
    s = math.sqrt(0.5 * spec.jones_var)
    pert = (z[0::2] + 1j * z[1::2]).reshape(spec.K, spec.N, 2, 2) * s
    return pert + np.eye(2)[None, None]


def sub_bands(spec: JobSpec, n_bands: int, f_lo: float = 115e6, f_hi: float = 185e6):
    """n_bands equal sub-bands tiling [f_lo, f_hi], each with spec.F equal
    channels: ([n_bands][F] channel centres, [n_bands] band centres)."""
    edges = np.linspace(f_lo, f_hi, n_bands + 1)
    width = (edges[1:] - edges[:-1]) / spec.F
    fr = edges[:-1, None] + width[:, None] * (np.arange(spec.F)[None, :] + 0.5)
    return fr, 0.5 * (edges[:-1] + edges[1:])


def frequency_basis(centres, n_poly: int, f_lo: float = 115e6, f_hi: float = 185e6) -> np.ndarray:
    """[n_bands][n_poly] values of the powers x^0 .. x^(n_poly-1) of the
    normalised frequency x = (f - f_mid) / (f_hi - f_mid) in [-1, 1] at each
    band centre: the smooth frequency model the sub-band solutions share."""
    x = (np.asarray(centres, dtype=np.float64) - 0.5 * (f_lo + f_hi)) / (0.5 * (f_hi - f_lo))
    return x[:, None] ** np.arange(n_poly)[None, :]


def jones_true_bands(spec: JobSpec, centres, drift_var: float = 0.02, f_lo: float = 115e6,
                     f_hi: float = 185e6) -> np.ndarray:
    """[n_bands][K][N][2][2] true Jones varying linearly across the band:
    J(f) = jones_true(spec) + x(f) D, D = CN(0, drift_var) per entry, x the
    normalised frequency of frequency_basis."""
    z = normal(spec.seed, TAG_BANDS, 2 * 4 * spec.K * spec.N)
    D = (z[0::2] + 1j * z[1::2]).reshape(spec.K, spec.N, 2, 2) * math.sqrt(0.5 * drift_var)
    x = (np.asarray(centres, dtype=np.float64) - 0.5 * (f_lo + f_hi)) / (0.5 * (f_hi - f_lo))
    return jones_true(spec)[None] + x[:, None, None, None, None] * D[None]


def noise(spec: JobSpec, t0: int = 0, t1: int | None = None) -> np.ndarray:
    """Noise for timeslots [t0, t1): [t1-t0][B][F][2][2] complex128."""
    t1 = spec.T if t1 is None else t1
    per_t = spec.B * spec.F * 8
    z = normal(spec.seed, TAG_NOISE, (t1 - t0) * per_t, offset=t0 * per_t)
    v = (z[0::2] + 1j * z[1::2]) * spec.sigma
    return v.reshape(t1 - t0, spec.B, spec.F, 2, 2)


def identity_jones(K: int, N: int) -> np.ndarray:
    return np.broadcast_to(np.eye(2, dtype=np.complex128), (K, N, 2, 2)).copy()


def baseline_pairs(N: int):
    """Stations (p, q), p < q, in baseline order b = p*N - p(p+1)/2 + (q-p-1)."""
    p, q = np.triu_indices(N, k=1)
    return p.astype(np.int64), q.astype(np.int64)


def uneven_time_chunks(n_jobs: int, lo: int = 5, hi: int = 40, seed: int = 0):
    """Timeslot counts of a batch of jobs, uniform integers in [lo, hi]."""
    u = uniform(seed, TAG_JOBS, n_jobs)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64).clip(lo, hi)
