"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws inputs: grids, models, sources, receivers and observed times. It
holds none of the solver's arithmetic, and both the CUDA path and the CPU oracle take its
arrays as plain data. Every generator is driven by numpy's PCG64 with an explicit seed.

The paper's real data sets (NCEDC/SCEDC picks, TSAR waveforms, AK135) are not available;
the workloads below stand in for them with the shapes and spacings of its experiments
(Sec. 4.1 synthetic test: 5 -> 8 km/s background, staggered anomalies; Sec. 4.2: 1-5 km
spacing, hundreds of sources with uneven pick counts).
"""
from dataclasses import dataclass, field, asdict

import numpy as np

EARTH_RADIUS_KM = 6371.0


@dataclass
class GridSpec:
    n_r: int
    n_t: int
    n_p: int
    depth_min_km: float
    depth_max_km: float
    lat_min_deg: float
    lat_max_deg: float
    lon_min_deg: float
    lon_max_deg: float
    earth_radius_km: float = EARTH_RADIUS_KM
    flat: int = 0

    @property
    def shape(self):
        return (self.n_r, self.n_t, self.n_p)

    @property
    def n_nodes(self):
        return self.n_r * self.n_t * self.n_p

    def axes(self):
        """Depth (km) of each radial index (i = 0 deepest), latitude and longitude (deg)."""
        depth = np.linspace(self.depth_max_km, self.depth_min_km, self.n_r)
        lat = np.linspace(self.lat_min_deg, self.lat_max_deg, self.n_t)
        lon = np.linspace(self.lon_min_deg, self.lon_max_deg, self.n_p)
        return depth, lat, lon

    def as_dict(self):
        return asdict(self)


@dataclass
class Workload:
    grid: GridSpec
    s: np.ndarray          # slowness s/km, (n_r, n_t, n_p) float64
    xi: np.ndarray
    eta: np.ndarray
    src: np.ndarray        # (n_src, 3) depth_km, lat_deg, lon_deg
    rec: np.ndarray        # (n_rec, 3) global receiver list
    abs_off: np.ndarray    # (n_src+1,) CSR offsets into the absolute-time records
    abs_rec: np.ndarray    # receiver index of each record
    abs_tobs: np.ndarray
    abs_w: np.ndarray
    cs_off: np.ndarray     # (n_src+1,) CSR offsets into the common-source pairs
    cs_m: np.ndarray
    cs_i: np.ndarray
    cs_dtobs: np.ndarray
    cs_w: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_src(self):
        return len(self.src)

    def source_data(self, n):
        """Per-source slices (receiver indices refer to the global receiver list)."""
        a0, a1 = self.abs_off[n], self.abs_off[n + 1]
        c0, c1 = self.cs_off[n], self.cs_off[n + 1]
        return dict(abs_rec=self.abs_rec[a0:a1], abs_tobs=self.abs_tobs[a0:a1],
                    abs_w=self.abs_w[a0:a1], cs_m=self.cs_m[c0:c1], cs_i=self.cs_i[c0:c1],
                    cs_dtobs=self.cs_dtobs[c0:c1], cs_w=self.cs_w[c0:c1])

    def subset(self, idx):
        """Workload restricted to the sources idx (receiver list unchanged)."""
        idx = list(idx)
        parts = [self.source_data(n) for n in idx]
        def cat(key, dt):
            return np.concatenate([p[key] for p in parts]).astype(dt) if parts else np.zeros(0, dt)
        abs_off = np.concatenate([[0], np.cumsum([len(p["abs_rec"]) for p in parts])]).astype(np.int32)
        cs_off = np.concatenate([[0], np.cumsum([len(p["cs_m"]) for p in parts])]).astype(np.int32)
        return Workload(self.grid, self.s, self.xi, self.eta, self.src[idx], self.rec, abs_off,
                        cat("abs_rec", np.int32), cat("abs_tobs", np.float64),
                        cat("abs_w", np.float64), cs_off, cat("cs_m", np.int32),
                        cat("cs_i", np.int32), cat("cs_dtobs", np.float64),
                        cat("cs_w", np.float64), self.name + "-subset", dict(self.meta))


# --------------------------------------------------------------------------- models

def background_velocity(grid, v_top=5.0, v_bottom=8.0):
    """1-D velocity rising linearly with depth over the whole grid depth (Sec. 4.1 style)."""
    depth, _, _ = grid.axes()
    d = (depth - grid.depth_min_km) / (grid.depth_max_km - grid.depth_min_km)
    v = v_top + (v_bottom - v_top) * d
    return np.broadcast_to(v[:, None, None], grid.shape).astype(np.float64)


def checker(grid, n_d=1.5, n_t=2.0, n_p=2.0, phase_cos_phi=False):
    """Sinusoidal checkerboard in [-1, 1]: sin(2 pi n x) along each axis, x the coordinate
    normalised to [0, 1] and n_* the number of periods across the grid."""
    depth, lat, lon = grid.axes()
    d = (depth - grid.depth_min_km) / (grid.depth_max_km - grid.depth_min_km)
    t = (lat - grid.lat_min_deg) / (grid.lat_max_deg - grid.lat_min_deg)
    p = (lon - grid.lon_min_deg) / (grid.lon_max_deg - grid.lon_min_deg)
    fp = np.cos if phase_cos_phi else np.sin
    return (np.sin(2 * np.pi * n_d * d)[:, None, None] * np.sin(2 * np.pi * n_t * t)[None, :, None]
            * fp(2 * np.pi * n_p * p)[None, None, :])


def gaussian_random_field(grid, corr_km, sigma, rng):
    """Smooth random field (Gaussian covariance of length corr_km) by spectral filtering of
    white noise on the index grid, scaled to standard deviation sigma."""
    depth, lat, lon = grid.axes()
    h = [abs(depth[1] - depth[0]),
         np.deg2rad(lat[1] - lat[0]) * grid.earth_radius_km,
         np.deg2rad(lon[1] - lon[0]) * grid.earth_radius_km * np.cos(np.deg2rad(lat.mean()))]
    w = rng.standard_normal(grid.shape)
    F = np.fft.fftn(w)
    ks = np.meshgrid(*[np.fft.fftfreq(n, d=hh) * 2 * np.pi for n, hh in zip(grid.shape, h)],
                     indexing="ij")
    k2 = sum(k * k for k in ks)
    F *= np.exp(-0.25 * k2 * corr_km ** 2)
    f = np.real(np.fft.ifftn(F))
    f = f - f.mean()
    return f * (sigma / (f.std() + 1e-30))


# --------------------------------------------------------------------------- geometry

def chord_km(grid, a, b):
    """Straight-line distance between points given as (depth, lat, lon) rows."""
    def xyz(p):
        p = np.atleast_2d(p)
        r = grid.earth_radius_km - p[:, 0]
        if grid.flat:
            return np.stack([r, grid.earth_radius_km * np.deg2rad(p[:, 1]),
                             grid.earth_radius_km * np.deg2rad(p[:, 2])], 1)
        th, ph = np.deg2rad(p[:, 1]), np.deg2rad(p[:, 2])
        return np.stack([r * np.cos(th) * np.cos(ph), r * np.cos(th) * np.sin(ph),
                         r * np.sin(th)], 1)
    return np.linalg.norm(xyz(a)[:, None, :] - xyz(b)[None, :, :], axis=2)


def lateral_margin_deg(grid, cells=2):
    dt = (grid.lat_max_deg - grid.lat_min_deg) / (grid.n_t - 1)
    dp = (grid.lon_max_deg - grid.lon_min_deg) / (grid.n_p - 1)
    return cells * dt, cells * dp


def random_sources(grid, n, depth_range, rng, cells=2):
    mt, mp = lateral_margin_deg(grid, cells)
    return np.stack([rng.uniform(*depth_range, n),
                     rng.uniform(grid.lat_min_deg + mt, grid.lat_max_deg - mt, n),
                     rng.uniform(grid.lon_min_deg + mp, grid.lon_max_deg - mp, n)], 1)


def surface_receivers(grid, n, rng, cells=2):
    mt, mp = lateral_margin_deg(grid, cells)
    return np.stack([np.full(n, grid.depth_min_km),
                     rng.uniform(grid.lat_min_deg + mt, grid.lat_max_deg - mt, n),
                     rng.uniform(grid.lon_min_deg + mp, grid.lon_max_deg - mp, n)], 1)


def synthetic_observations(grid, src, rec, v_ref, noise_s, rng, ratio=1.0):
    """Observed times: straight-ray distance over a reference speed, scaled, plus Gaussian
    noise. A stand-in for picks; only the residual sizes matter for the solver."""
    return chord_km(grid, src, rec) / v_ref * ratio + noise_s * rng.standard_normal((len(src), len(rec)))


def build_data(grid, src, rec, tobs, rng, counts=None, cs_max_deg=1.0, weight=1.0):
    """Per-source receiver subsets (all receivers, or a seeded subset of the given sizes),
    absolute records and all common-source pairs of the subset closer than cs_max_deg."""
    n_src = len(src)
    abs_off, abs_rec, abs_tobs = [0], [], []
    cs_off, cs_m, cs_i, cs_dt = [0], [], [], []
    for n in range(n_src):
        if counts is None:
            sub = np.arange(len(rec))
        else:
            sub = np.sort(rng.choice(len(rec), size=int(counts[n]), replace=False))
        abs_rec.extend(sub.tolist())
        abs_tobs.extend(tobs[n, sub].tolist())
        abs_off.append(len(abs_rec))
        lat, lon = rec[sub, 1], rec[sub, 2]
        a, b = np.triu_indices(len(sub), k=1)
        keep = np.hypot(lat[a] - lat[b], lon[a] - lon[b]) <= cs_max_deg
        m, i = sub[a[keep]], sub[b[keep]]
        cs_m.extend(m.tolist()); cs_i.extend(i.tolist())
        cs_dt.extend((tobs[n, m] - tobs[n, i]).tolist())
        cs_off.append(len(cs_m))
    f64 = lambda x: np.asarray(x, dtype=np.float64)
    i32 = lambda x: np.asarray(x, dtype=np.int32)
    return dict(abs_off=i32(abs_off), abs_rec=i32(abs_rec), abs_tobs=f64(abs_tobs),
                abs_w=np.full(len(abs_rec), weight), cs_off=i32(cs_off), cs_m=i32(cs_m),
                cs_i=i32(cs_i), cs_dtobs=f64(cs_dt), cs_w=np.full(len(cs_m), weight))


# --------------------------------------------------------------------------- workloads

SEED_BASE = 20241200


def homogeneous_41(seed=SEED_BASE + 0):
    """41^3 grid, depth 0-40 km, 1 x 1 deg, Vp = 6 km/s, xi = eta = 0, one source at the
    surface centre (a grid node), 16 seeded surface receivers, T_obs = chord / 6.06."""
    rng = np.random.default_rng(seed)
    g = GridSpec(41, 41, 41, 0.0, 40.0, 0.0, 1.0, 0.0, 1.0)
    s = np.full(g.shape, 1.0 / 6.0)
    z = np.zeros(g.shape)
    src = np.array([[0.0, 0.5, 0.5]])
    rec = surface_receivers(g, 16, rng)
    tobs = chord_km(g, src, rec) / 6.06
    d = build_data(g, src, rec, tobs, rng, cs_max_deg=0.5)
    return Workload(g, s, z, z.copy(), src, rec, name="homogeneous-41^3", **d)


def checkerboard_81(seed=SEED_BASE + 1, n_src=64, n_rec=100, shape=(81, 81, 81)):
    """81^3 grid, depth 0-60 km, 2 x 2 deg; Vp 5 -> 8 km/s with depth times a +-5 %
    checkerboard; isotropic; n_src sources at 5-40 km; n_rec surface receivers; absolute
    times and common-source pairs closer than 1 deg."""
    rng = np.random.default_rng(seed)
    g = GridSpec(shape[0], shape[1], shape[2], 0.0, 60.0, 0.0, 2.0, 0.0, 2.0)
    v = background_velocity(g) * (1.0 + 0.05 * checker(g))
    s = 1.0 / v
    z = np.zeros(g.shape)
    src = random_sources(g, n_src, (5.0, 40.0), rng)
    rec = surface_receivers(g, n_rec, rng)
    tobs = synthetic_observations(g, src, rec, 6.0, 0.05, rng)
    d = build_data(g, src, rec, tobs, rng)
    return Workload(g, s, z, z.copy(), src, rec, name="checkerboard-81^3", **d)


def anisotropic_batch(seed=SEED_BASE + 2, n_src=256, n_pool=200, shape=(121, 161, 161),
                      count_range=(20, 200)):
    """121 x 161 x 161 grid (r x lat x lon), depth 0-100 km, 3 x 4 deg; Vp 5 -> 8 km/s with
    depth times a +-4 % checkerboard; xi and eta checkerboards of amplitude 0.04; n_src
    sources at 5-90 km; each source sees a seeded subset of U{20..200} receivers out of a
    pool of 200 surface stations; absolute times and common-source pairs within 1 deg."""
    rng = np.random.default_rng(seed)
    g = GridSpec(shape[0], shape[1], shape[2], 0.0, 100.0, 0.0, 3.0, 0.0, 4.0)
    v = background_velocity(g) * (1.0 + 0.04 * checker(g))
    s = 1.0 / v
    xi = 0.04 * checker(g)
    eta = 0.04 * checker(g, phase_cos_phi=True)
    src = random_sources(g, n_src, (5.0, 90.0), rng)
    rec = surface_receivers(g, n_pool, rng)
    tobs = synthetic_observations(g, src, rec, 6.2, 0.05, rng)
    lo, hi = count_range
    counts = rng.integers(lo, min(hi, n_pool) + 1, n_src)
    d = build_data(g, src, rec, tobs, rng, counts=counts)
    return Workload(g, s, xi, eta, src, rec, name="anisotropic-121x161x161", **d)


def inversion_201(seed=SEED_BASE + 4, n_src=1024, n_pool=400, shape=(101, 201, 201),
                  count_range=(20, 200), cs_max_deg=0.5, cr_max_deg=0.3):
    """201 (lat) x 201 (lon) x 101 (depth) grid, depth 0-200 km, 5 x 5 deg (2 km, 0.025 deg).
    Start model: Vp 5 -> 8 km/s with depth, isotropic. True model (meta["true"] = (s, xi,
    eta)): the start times a +-5 % checkerboard, with xi and eta checkerboards of amplitude
    0.02. n_src sources at 5-180 km; each sees a seeded subset of U{20..200} of n_pool surface
    stations; common-source pairs of a subset closer than cs_max_deg. meta["cr_deg"] is the
    largest epicentral distance of a common-receiver source pair. The times here are
    straight-ray placeholders; a caller that needs consistent data replaces them by solves
    in the true model (meta["noise_s"] = 0.05 s of Gaussian noise)."""
    rng = np.random.default_rng(seed)
    g = GridSpec(shape[0], shape[1], shape[2], 0.0, 200.0, 0.0, 5.0, 0.0, 5.0)
    v0 = background_velocity(g)
    s = 1.0 / v0
    z = np.zeros(g.shape)
    s_true = 1.0 / (v0 * (1.0 + 0.05 * checker(g, 1.5, 2.5, 2.5)))
    xi_true = 0.02 * checker(g, 1.5, 2.5, 2.5)
    eta_true = 0.02 * checker(g, 1.5, 2.5, 2.5, phase_cos_phi=True)
    src = random_sources(g, n_src, (5.0, 180.0), rng)
    rec = surface_receivers(g, n_pool, rng)
    tobs = synthetic_observations(g, src, rec, 6.5, 0.05, rng)
    lo, hi = count_range
    counts = rng.integers(lo, min(hi, n_pool) + 1, n_src)
    d = build_data(g, src, rec, tobs, rng, counts=counts, cs_max_deg=cs_max_deg)
    meta = dict(true=(s_true, xi_true, eta_true), cr_deg=cr_max_deg, noise_s=0.05,
                noise_seed=seed + 1000)
    return Workload(g, s, z, z.copy(), src, rec, name="inversion-201x201x101", meta=meta, **d)


def random_field_models(seed=SEED_BASE + 3, n_models=250, shape=(81, 81, 81),
                        depth_km=60.0, extent_deg=2.0, corr_km=10.0, sigma_v=0.03,
                        sigma_aniso=0.02, clip_aniso=0.04, n_src=8, depth_range=(5.0, 40.0)):
    """Training models of the warm-start network: on an n_r x n_t x n_p grid (depth 0 to
    depth_km, extent_deg square, or (lat, lon) extents), Vp = (5 -> 8 km/s with depth) x
    (1 + GRF), the GRF of correlation length corr_km and standard deviation sigma_v; xi, eta
    independent GRFs of standard deviation sigma_aniso clipped to +-clip_aniso; n_src sources
    per model uniform in depth_range. Returns the grid and a list of (s, xi, eta, src) per
    model."""
    rng = np.random.default_rng(seed)
    ext_t, ext_p = (extent_deg, extent_deg) if np.isscalar(extent_deg) else extent_deg
    g = GridSpec(shape[0], shape[1], shape[2], 0.0, depth_km, 0.0, ext_t, 0.0, ext_p)
    vb = background_velocity(g)
    out = []
    for _ in range(n_models):
        v = vb * (1.0 + gaussian_random_field(g, corr_km, sigma_v, rng))
        xi = np.clip(gaussian_random_field(g, corr_km, sigma_aniso, rng), -clip_aniso, clip_aniso)
        eta = np.clip(gaussian_random_field(g, corr_km, sigma_aniso, rng), -clip_aniso, clip_aniso)
        out.append((1.0 / v, xi, eta, random_sources(g, n_src, depth_range, rng)))
    return g, out


def small_case(seed, shape=(13, 15, 17), n_src=3, n_rec=6, aniso=0.03, flat=0,
               depth_max=12.0, extent_deg=0.12):
    """Small heterogeneous anisotropic case with ragged dimensions for parity tests."""
    rng = np.random.default_rng(seed)
    g = GridSpec(shape[0], shape[1], shape[2], 0.0, depth_max, 0.0, extent_deg, 0.0,
                 extent_deg * 1.1, flat=flat)
    v = background_velocity(g) * (1.0 + 0.04 * checker(g, 1.0, 1.0, 1.0))
    s = 1.0 / v
    xi = aniso * checker(g, 1.0, 1.0, 1.0)
    eta = aniso * checker(g, 1.0, 1.0, 1.0, phase_cos_phi=True)
    src = random_sources(g, n_src, (0.3 * depth_max, 0.8 * depth_max), rng)
    rec = surface_receivers(g, n_rec, rng)
    tobs = synthetic_observations(g, src, rec, 6.0, 0.05, rng)
    d = build_data(g, src, rec, tobs, rng, cs_max_deg=extent_deg)
    return Workload(g, s, xi, eta, src, rec, name="small-%dx%dx%d" % shape, **d)
