"""Seeded synthetic inputs for the elastic staggered-grid solver.

Everything here is *input generation*: media, wavelets, source tensors and
receiver layouts.  None of the scheme's arithmetic (finite differences, medium
averaging at staggered points, injection or sampling weights, boundary
profiles) lives in this module, so that the CUDA path and the FP64 oracle can
both be fed from it without sharing any of the method.

Conventions (shared by both sides through the arrays they receive):
  * arrays are C-ordered ``[nz][ny][nx]`` (x fastest), float32;
  * positions are metres measured from the normal-stress point of cell
    (0, 0, 0), z positive downwards;
  * the medium is returned as (vp, vs, rho) in m/s, m/s and kg/m^3.

The paper's own case study (Sec. 3) uses real IRIS waveforms that are not
available here; these seeded models stand in for it (layered crust plus a
Gaussian-correlated random perturbation, Gardner density).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 15071

# Stability constant printed with the time-step rule (Sec. 2.1.3, Eq. 5).
PAPER_CFL = 0.495


def ricker(nt: int, dt: float, f0: float, t0: float | None = None,
           shift: float = 0.0) -> np.ndarray:
    """Ricker wavelet sampled at t = (n + shift) * dt, n = 0..nt-1 (float32).

    The paper does not state its source time function; a Ricker with
    t0 = 1.5 / f0 starts at ~1e-8 of its peak, so there is no step at t = 0.
    ``shift = 0.5`` gives the half-step samples a moment-rate source needs,
    ``shift = 0`` the integer-step samples of a force source.
    """
    if t0 is None:
        t0 = 1.5 / f0
    t = (np.arange(nt, dtype=np.float64) + shift) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def ricker_fp64(t: np.ndarray, f0: float, t0: float) -> np.ndarray:
    a = (math.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def double_couple(strike_deg: float, dip_deg: float, rake_deg: float,
                  m0: float = 1e15) -> np.ndarray:
    """Moment tensor (Mxx, Myy, Mzz, Mxy, Mxz, Myz) of a shear dislocation.

    Aki & Richards (Box 4.4) with x = north, y = east, z = down.  Input
    generation only: the solver receives the six components.
    """
    p, d, l = (math.radians(strike_deg), math.radians(dip_deg),
               math.radians(rake_deg))
    sd, cd, s2d, c2d = math.sin(d), math.cos(d), math.sin(2 * d), math.cos(2 * d)
    sl, cl = math.sin(l), math.cos(l)
    sp, cp, s2p, c2p = math.sin(p), math.cos(p), math.sin(2 * p), math.cos(2 * p)
    mxx = -m0 * (sd * cl * s2p + s2d * sl * sp * sp)
    myy = m0 * (sd * cl * s2p - s2d * sl * cp * cp)
    mzz = m0 * s2d * sl
    mxy = m0 * (sd * cl * c2p + 0.5 * s2d * sl * s2p)
    mxz = -m0 * (cd * cl * cp + c2d * sl * sp)
    myz = -m0 * (cd * cl * sp - c2d * sl * cp)
    return np.array([mxx, myy, mzz, mxy, mxz, myz], dtype=np.float64)


def explosion(m0: float = 1e15) -> np.ndarray:
    return np.array([m0, m0, m0, 0.0, 0.0, 0.0], dtype=np.float64)


# Moment tensor printed for the 2016-01-17 Cuba event (Sec. 3.1.1, Eq. 7),
# rows/columns in the paper's (x, y, z) order; units read as N*m.
PAPER_MOMENT_TENSOR = np.array([
    [-2.37e14, -3.39e15, -7.79e14],
    [-3.39e15, -4.31e16, 4.60e15],
    [-7.79e14, 4.60e15, 4.33e16],
])

# 1D crustal model of the case study (Sec. 3.1.2, table "Medium parameters"):
# top of layer (km), vp (km/s), vs (km/s), rho (g/cm^3).
PAPER_LAYERS = np.array([
    [0.0, 4.90, 2.816, 2.50],
    [3.0, 5.40, 3.103, 2.60],
    [5.0, 6.00, 3.448, 2.70],
    [7.0, 6.90, 3.966, 2.80],
    [20.0, 7.60, 4.368, 3.10],
    [26.0, 7.80, 4.483, 3.26],
    [34.0, 8.00, 4.598, 3.30],
])

# Level-of-detail grids of the case study (Sec. 3.2.1, table "Simulation
# details"): (nx, ny, nz, steps).
PAPER_LEVELS = [
    (64, 64, 32, 1700), (64, 64, 64, 1700), (128, 64, 64, 1700),
    (128, 128, 64, 1700), (128, 128, 128, 3400), (256, 128, 128, 3400),
    (256, 256, 128, 3400), (256, 256, 256, 17000), (512, 256, 256, 17000),
    (512, 512, 256, 17000), (512, 512, 512, 17000),
]


def gardner(vp: np.ndarray) -> np.ndarray:
    """Gardner density rho = 310 * vp^0.25 (kg/m^3, vp in m/s)."""
    return (310.0 * np.power(vp.astype(np.float64), 0.25)).astype(np.float32)


def homogeneous(nx: int, ny: int, nz: int, vp: float = 3000.0,
                vs: float = 1730.0, rho: float = 2500.0):
    shp = (nz, ny, nx)
    return (np.full(shp, vp, np.float32), np.full(shp, vs, np.float32),
            np.full(shp, rho, np.float32))


def _gauss_filter_axis(a: np.ndarray, axis: int, sigma_cells: float) -> np.ndarray:
    """Circular convolution along one axis with exp(-x^2 / L^2), via rFFT."""
    import scipy.fft as sfft
    n = a.shape[axis]
    x = np.arange(n, dtype=np.float64)
    x = np.minimum(x, n - x)
    ker = np.exp(-(x / sigma_cells) ** 2)
    kf = sfft.rfft(ker)
    shape = [1] * a.ndim
    shape[axis] = kf.shape[0]
    af = sfft.rfft(a, axis=axis, workers=-1)
    af *= kf.reshape(shape).astype(af.dtype)
    return sfft.irfft(af, n=n, axis=axis, workers=-1).astype(a.dtype)


def correlated_noise(nx: int, ny: int, nz: int, spacing, corr_len: float,
                     seed: int) -> np.ndarray:
    """Seeded white noise convolved with exp(-r^2 / corr_len^2), max|p| = 1.

    The Gaussian kernel is separable, so the 3D convolution is three 1D ones.
    """
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((nz, ny, nx), dtype=np.float32)
    dx, dy, dz = spacing
    p = _gauss_filter_axis(p, 2, corr_len / dx)
    p = _gauss_filter_axis(p, 1, corr_len / dy)
    p = _gauss_filter_axis(p, 0, corr_len / dz)
    p /= np.max(np.abs(p))
    return p


def layered_random(nx: int, ny: int, nz: int, spacing,
                   layer_vp=(2000.0, 3000.0, 4000.0, 5000.0, 6000.0),
                   vpvs: float = 1.73, corr_len: float = 200.0,
                   amp: float = 0.05, seed: int = SEED):
    """Horizontal equal-thickness layers (vp increasing with depth), vs = vp /
    vpvs, perturbed by (1 + p) with Gaussian-correlated p (max|p| = amp);
    density from Gardner on the perturbed vp."""
    nl = len(layer_vp)
    k = np.arange(nz)
    layer = np.minimum((k * nl) // nz, nl - 1)
    vp1 = np.asarray(layer_vp, np.float64)[layer]
    vp = np.broadcast_to(vp1[:, None, None], (nz, ny, nx)).astype(np.float32)
    if amp > 0:
        p = correlated_noise(nx, ny, nz, spacing, corr_len, seed) * np.float32(amp)
        vp = vp * (1.0 + p)
    vp = vp.astype(np.float32)
    vs = (vp / np.float32(vpvs)).astype(np.float32)
    return vp, vs, gardner(vp)


def layered_random_device(nx: int, ny: int, nz: int, spacing, device,
                          layer_vp=(2000.0, 3000.0, 4000.0, 5000.0, 6000.0),
                          vpvs: float = 1.73, corr_len: float = 200.0,
                          amp: float = 0.05, seed: int = SEED):
    """The layered_random recipe generated directly in device memory with
    torch (for grids whose host generation would take minutes): the same
    layers, circular Gaussian filtering and Gardner density, drawn from
    torch's seeded generator instead of numpy's.  Returns CUDA tensors."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    p = torch.randn((nz, ny, nx), generator=gen, device=device, dtype=torch.float32)
    for axis, h in ((2, spacing[0]), (1, spacing[1]), (0, spacing[2])):
        n = p.shape[axis]
        x = torch.arange(n, device=device, dtype=torch.float64)
        x = torch.minimum(x, n - x)
        kf = torch.fft.rfft(torch.exp(-(x / (corr_len / h)) ** 2))
        shape = [1, 1, 1]
        shape[axis] = kf.shape[0]
        pf = torch.fft.rfft(p, dim=axis)
        pf *= kf.reshape(shape).to(pf.dtype)
        p = torch.fft.irfft(pf, n=n, dim=axis).float()
        del pf
    p *= amp / p.abs().max()
    nl = len(layer_vp)
    layer = torch.clamp((torch.arange(nz, device=device) * nl) // nz, max=nl - 1)
    vp1 = torch.tensor(layer_vp, device=device, dtype=torch.float32)[layer]
    vp = (vp1[:, None, None] * (1.0 + p)).contiguous()
    del p
    vs = vp / vpvs
    rho = (310.0 * vp.double() ** 0.25).float()
    return vp, vs, rho


def add_sphere(vp, vs, spacing, centre, radius: float, frac: float):
    """Multiply vp and vs by (1 + frac) inside a sphere; Gardner rho."""
    nz, ny, nx = vp.shape
    dx, dy, dz = spacing
    z, y, x = np.meshgrid(np.arange(nz) * dz, np.arange(ny) * dy,
                          np.arange(nx) * dx, indexing="ij")
    inside = ((x - centre[0]) ** 2 + (y - centre[1]) ** 2
              + (z - centre[2]) ** 2) <= radius ** 2
    vp = np.where(inside, vp * np.float32(1 + frac), vp).astype(np.float32)
    vs = np.where(inside, vs * np.float32(1 + frac), vs).astype(np.float32)
    return vp, vs, gardner(vp)


def smooth(a: np.ndarray, spacing, sigma_m: float) -> np.ndarray:
    """Gaussian smoothing exp(-r^2 / (2 sigma^2)) with edge replication."""
    from scipy.ndimage import gaussian_filter
    s = (sigma_m / spacing[2], sigma_m / spacing[1], sigma_m / spacing[0])
    return gaussian_filter(a.astype(np.float64), s, mode="nearest").astype(np.float32)


def max_stable_dt(spacing, vp_max: float, cfl: float = PAPER_CFL) -> float:
    return cfl * min(spacing) / vp_max


@dataclass
class Problem:
    """One seeded forward (or gradient) problem, ready for either side."""
    name: str
    nx: int
    ny: int
    nz: int
    spacing: tuple
    dt: float
    nt: int
    vp: np.ndarray
    vs: np.ndarray
    rho: np.ndarray
    src_kind: str               # "moment" or "force"
    src_pos: np.ndarray         # (3,) metres
    src_comp: np.ndarray        # (6,) moment or (3,) force
    wavelet: np.ndarray         # (nt,) float32, value injected at step n
    rec_pos: np.ndarray         # (nrec, 3) metres
    boundary: str = "sponge"    # "none", "sponge", "cpml"
    width: int = 16
    f0: float = 10.0
    extra: dict = field(default_factory=dict)
    free_surface: tuple | None = None   # (ks, eps): vacuum above plane ks
    coarse_medium: tuple | None = None  # (lambda, mu, rho) on a medium grid [mz][my][mx]

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def lame(self):
        """(lambda, mu, rho) in float32 from (vp, vs, rho); convenience for
        callers that want the Lame form of the inputs."""
        vp = self.vp.astype(np.float64)
        vs = self.vs.astype(np.float64)
        rho = self.rho.astype(np.float64)
        mu = rho * vs * vs
        lam = rho * vp * vp - 2.0 * mu
        return lam.astype(np.float32), mu.astype(np.float32), self.rho.copy()


def _wavelet_for(kind: str, nt: int, dt: float, f0: float) -> np.ndarray:
    # Moment-rate sources are injected into the stress update centred on
    # t_{n+1/2}; forces into the velocity update centred on t_n.
    return ricker(nt, dt, f0, shift=0.5 if kind == "moment" else 0.0)


def line_receivers(src, n=8, dxs=20.0, perp=(141.42, 141.42)) -> np.ndarray:
    off = (np.arange(n) - (n - 1) / 2.0) * dxs
    r = np.zeros((n, 3))
    r[:, 0] = src[0] + off
    r[:, 1] = src[1] + perp[0]
    r[:, 2] = src[2] + perp[1]
    return r


def grid_receivers(nx, ny, spacing, width, k, na, nb) -> np.ndarray:
    """na x nb receivers evenly spread over the interior (x, y) at depth
    index k (off-grid in x and y)."""
    dx, dy, dz = spacing
    xs = (width + (np.arange(na) + 0.5) * (nx - 2 * width) / na) * dx
    ys = (width + (np.arange(nb) + 0.5) * (ny - 2 * width) / nb) * dy
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    r = np.zeros((na * nb, 3))
    r[:, 0] = X.ravel()
    r[:, 1] = Y.ravel()
    r[:, 2] = k * dz
    return r


def config1(nt: int = 500) -> Problem:
    """Plain forward parity case: 64^3, dx = 10 m, homogeneous, sponge 16,
    centred explosion, 15 Hz Ricker, 8 receivers on a line ~200 m away."""
    n, h = 64, 10.0
    vp, vs, rho = homogeneous(n, n, n)
    dt = 0.5 * PAPER_CFL * h / 3000.0
    src = np.array([32 * h, 32 * h, 32 * h])
    return Problem("config1_64cube", n, n, n, (h, h, h), dt, nt, vp, vs, rho,
                   "moment", src, explosion(), _wavelet_for("moment", nt, dt, 15.0),
                   line_receivers(src), "sponge", 16, 15.0)


def config2(n: int = 256, nt: int = 2000, h: float = 20.0, width: int = 20,
            seed: int = SEED) -> Problem:
    """Forward throughput case: n^3 (256), dx = 20 m, 5 layers plus a
    Gaussian-correlated +-5 % perturbation, C-PML 20, double couple
    (30, 60, 90) at 2 km depth with a 5 Hz Ricker, 16 x 16 receivers."""
    sp = (h, h, h)
    vp, vs, rho = layered_random(n, n, n, sp, seed=seed)
    vmax = 6000.0 * 1.05
    dt = 0.5 * PAPER_CFL * h / vmax
    ksrc = min(int(round(2000.0 / h)), n - 3)
    src = np.array([(n // 2) * h, (n // 2) * h, ksrc * h])
    f0 = 5.0
    rec = grid_receivers(n, n, sp, width, width, 16, 16)
    return Problem(f"config2_{n}cube_cpml", n, n, n, sp, dt, nt, vp, vs, rho,
                   "moment", src, double_couple(30, 60, 90),
                   _wavelet_for("moment", nt, dt, f0), rec, "cpml", width, f0)


def config3(nx: int = 1024, ny: int = 1024, nz: int = 512, nt: int = 3000,
            h: float = 50.0, width: int = 20, seed: int = SEED, device=None) -> Problem:
    """Large forward case: 1024 x 1024 x 512, dx = 50 m, layered + random,
    sponge 20, vertical point force at 10 km depth (2 Hz), 32 x 32 receivers.
    With `device`, the model is generated in device memory (torch tensors)."""
    sp = (h, h, h)
    if device is not None:
        vp, vs, rho = layered_random_device(nx, ny, nz, sp, device, seed=seed)
    else:
        vp, vs, rho = layered_random(nx, ny, nz, sp, seed=seed)
    dt = 0.5 * PAPER_CFL * h / (6000.0 * 1.05)
    ksrc = min(int(round(10000.0 / h)), nz - 3)
    src = np.array([(nx // 2) * h, (ny // 2) * h, ksrc * h])
    f0 = 2.0
    rec = grid_receivers(nx, ny, sp, width, width, 32, 32)
    return Problem(f"config3_{nx}x{ny}x{nz}", nx, ny, nz, sp, dt, nt, vp, vs, rho,
                   "force", src, np.array([0.0, 0.0, 1e10]),
                   _wavelet_for("force", nt, dt, f0), rec, "sponge", width, f0)


# Grid spacings (km) and time steps (s) of the level-of-detail table (Sec.
# 3.2.1, "Simulation details"), level by level.
PAPER_LEVEL_SPACING = [
    (6.67, 10.61, 3.75, 0.1), (6.67, 10.61, 1.87, 0.1), (3.33, 10.61, 1.87, 0.1),
    (3.33, 5.30, 1.87, 0.1), (3.33, 5.30, 0.93, 0.05), (1.66, 5.30, 0.93, 0.05),
    (1.66, 2.65, 0.93, 0.05), (1.66, 2.65, 0.46, 0.01), (0.83, 2.65, 0.46, 0.01),
    (0.83, 1.32, 0.46, 0.01), (0.83, 1.32, 0.23, 0.01),
]


def paper_level(level: int, nt: int | None = None) -> Problem:
    """Level `level` of the paper's level-of-detail table as a synthetic
    input: the grid, spacing and time step of the table, the 1D crustal
    model of Sec. 3.1.2 (layer tops measured from 30 km below the top of the
    grid, whose depth range is -30..90 km; cells above depth 0 take the top
    layer), the moment tensor of Eq. 7 at the centroid depth (7 km) in the
    centre of (x, y), a Ricker at the table's maximum frequency, a sponge of a quarter of the thinnest axis (at most
    16 cells) and 8 receivers on a line at the top of the interior.  Timing
    workload only (the real seismograms are not available)."""
    nx, ny, nz, steps = PAPER_LEVELS[level]
    dxk, dyk, dzk, dt = PAPER_LEVEL_SPACING[level]
    sp = (dxk * 1e3, dyk * 1e3, dzk * 1e3)
    nt = steps if nt is None else nt
    depth = (np.arange(nz) * sp[2]) / 1e3 - 30.0            # km, cell tops
    li = np.clip(np.searchsorted(PAPER_LAYERS[:, 0], depth, side="right") - 1, 0, None)
    vp1, vs1, rho1 = (PAPER_LAYERS[li, c] * 1e3 for c in (1, 2, 3))
    shp = (nz, ny, nx)
    vp = np.broadcast_to(vp1[:, None, None], shp).astype(np.float32)
    vs = np.broadcast_to(vs1[:, None, None], shp).astype(np.float32)
    rho = np.broadcast_to(rho1[:, None, None], shp).astype(np.float32)
    width = max(4, min(16, min(nx, ny, nz) // 4))
    M = PAPER_MOMENT_TENSOR
    comp = np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])
    ks = min(int(round((30.0 + 7.0) * 1e3 / sp[2])), nz - width - 2)
    src = np.array([(nx // 2) * sp[0], (ny // 2) * sp[1], ks * sp[2]])
    fmax = 0.037 if level < 3 else 0.075 if level < 6 else 0.15 if level < 9 else 0.30
    rec = grid_receivers(nx, ny, sp, width, width, 8, 1)
    return Problem(f"paper_level{level}_{nx}x{ny}x{nz}", nx, ny, nz, sp, dt, nt, vp, vs, rho,
                   "moment", src, comp, _wavelet_for("moment", nt, dt, fmax), rec, "sponge",
                   width, fmax)


def sphere_anomaly_device(vp, vs, spacing, frac: float = 0.05):
    """+frac on vp and vs inside a centred sphere of a quarter of the cube
    side (device tensors); Gardner density.  The 'observed' variant of a
    batched shot."""
    import torch
    nz, ny, nx = vp.shape
    dev = vp.device
    z = torch.arange(nz, device=dev, dtype=torch.float32)[:, None, None] - nz // 2
    y = torch.arange(ny, device=dev, dtype=torch.float32)[None, :, None] - ny // 2
    x = torch.arange(nx, device=dev, dtype=torch.float32)[None, None, :] - nx // 2
    inside = (x * x + y * y + z * z) <= (min(nx, ny, nz) / 4.0) ** 2
    f = torch.where(inside, torch.tensor(1.0 + frac, device=dev), torch.tensor(1.0, device=dev))
    vp2 = (vp * f).contiguous()
    vs2 = (vs * f).contiguous()
    return vp2, vs2, (310.0 * vp2.double() ** 0.25).float()


def config3_crop(n: int = 128, nt: int = 1000, h: float = 50.0, width: int = 20,
                 seed: int = SEED) -> Problem:
    """The large forward recipe re-instantiated on an n^3 crop (128^3) for the
    storage-error comparison against the oracle: same spacing, model recipe,
    sponge and receiver layout; the point force sits at the same fraction of
    the depth (10 km of 25.6 km)."""
    sp = (h, h, h)
    vp, vs, rho = layered_random(n, n, n, sp, seed=seed)
    dt = 0.5 * PAPER_CFL * h / (6000.0 * 1.05)
    ksrc = int(round(n * 10000.0 / (512 * 50.0)))
    src = np.array([(n // 2) * h, (n // 2) * h, ksrc * h])
    f0 = 2.0
    rec = grid_receivers(n, n, sp, width, width, 32, 32)
    return Problem(f"config3_crop_{n}cube", n, n, n, sp, dt, nt, vp, vs, rho,
                   "force", src, np.array([0.0, 0.0, 1e10]),
                   _wavelet_for("force", nt, dt, f0), rec, "sponge", width, f0)


def config4(n: int = 192, nt: int = 1500, h: float = 15.0, width: int = 20,
            seed: int = SEED):
    """Adjoint case: returns (true, start) problems on n^3 (192), dx = 15 m.
    True = layers + random + 10 % sphere of radius 300 m at the centre;
    start = the layers smoothed by a Gaussian of sigma = 150 m."""
    sp = (h, h, h)
    vp, vs, rho = layered_random(n, n, n, sp, seed=seed)
    c = ((n // 2) * h,) * 3
    scale = n * h / (192 * 15.0)        # physical size relative to the 192^3, 15 m case
    vpt, vst, rhot = add_sphere(vp, vs, sp, c, 300.0 * scale, 0.10)
    vp0, vs0, _ = layered_random(n, n, n, sp, amp=0.0)
    vp0 = smooth(vp0, sp, 150.0 * scale)
    vs0 = smooth(vs0, sp, 150.0 * scale)
    rho0 = gardner(vp0)
    vmax = float(max(vpt.max(), vp0.max()))
    dt = 0.5 * PAPER_CFL * h / vmax
    src = np.array([(n // 2) * h, (n // 2) * h, (width + 10) * h])
    f0 = 6.0
    nr = 20 if n >= 96 else max(4, n // 8)
    rec = grid_receivers(n, n, sp, width, width, nr, nr)
    wav = _wavelet_for("moment", nt, dt, f0)
    true = Problem(f"config4_{n}cube_true", n, n, n, sp, dt, nt, vpt, vst, rhot,
                   "moment", src, explosion(), wav, rec, "sponge", width, f0)
    start = Problem(f"config4_{n}cube_start", n, n, n, sp, dt, nt, vp0, vs0, rho0,
                    "moment", src, explosion(), wav, rec, "sponge", width, f0)
    return true, start


def config5_shots(nshots: int = 48, seed: int = SEED, device=None):
    """Batched case: seeded cube sizes in {96, 104, ..., 224}, nt in
    [800, 1600], f0 in [5, 15] Hz, dx = vs_min / (12.5 f0) rounded down to
    0.5 m; each shot has its own layered + random model (seed + shot).
    With `device`, the models are generated in device memory (torch)."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.arange(96, 225, 8), size=nshots)
    nts = rng.integers(800, 1601, size=nshots)
    f0s = rng.uniform(5.0, 15.0, size=nshots)
    shots = []
    for s in range(nshots):
        n, nt, f0 = int(sizes[s]), int(nts[s]), float(f0s[s])
        vs_min = 2000.0 * 0.95 / 1.73
        h = math.floor(vs_min / (12.5 * f0) * 2.0) / 2.0
        sp = (h, h, h)
        if device is not None:
            vp, vs, rho = layered_random_device(n, n, n, sp, device,
                                                corr_len=max(200.0, 4 * h), seed=seed + s)
        else:
            vp, vs, rho = layered_random(n, n, n, sp, corr_len=max(200.0, 4 * h),
                                         seed=seed + s)
        dt = 0.5 * PAPER_CFL * h / (6000.0 * 1.05)
        src = np.array([(n // 2) * h, (n // 2) * h, (n // 3) * h])
        rec = grid_receivers(n, n, sp, 16, 16, 8, 8)
        shots.append(Problem(f"shot{s}_{n}cube", n, n, n, sp, dt, nt, vp, vs, rho,
                             "moment", src, explosion(),
                             _wavelet_for("moment", nt, dt, f0), rec, "sponge",
                             16, f0))
    return shots


def small_problem(nx=40, ny=36, nz=28, nt=60, h=10.0, boundary="sponge",
                  width=6, kind="moment", seed=SEED, layered=True,
                  nrec=5, spacing=None) -> Problem:
    """Small ragged seeded problem for parity tests (non-multiple-of-tile
    sizes, heterogeneous medium, off-grid source and receivers).

    spacing: (dx, dy, dz) in metres for a grid whose spacing differs per axis
    (the paper's level table has such grids); then h is unused, the time step
    is 0.9 x Eq. 5's rule on the smallest spacing and the wavelet keeps 8
    cells per shortest S wavelength on the largest spacing.  Without it the
    grid is cubic with spacing h and dt is half Eq. 5's rule."""
    sp = (h, h, h) if spacing is None else tuple(float(a) for a in spacing)
    rng = np.random.default_rng(seed)
    if layered:
        vp, vs, rho = layered_random(nx, ny, nz, sp, layer_vp=(2500.0, 3000.0, 3600.0),
                                     corr_len=4 * max(sp), seed=seed)
    else:
        vp, vs, rho = homogeneous(nx, ny, nz)
    vmax = float(vp.max())
    if spacing is None:
        dt = 0.5 * PAPER_CFL * h / vmax
    else:
        dt = 0.9 * PAPER_CFL * min(sp) / vmax
    lo = np.array([width + 1.0, width + 1.0, width + 1.0])
    hi = np.array([nx, ny, nz], float) - width - 2.0
    src = (lo + (hi - lo) * rng.uniform(0.3, 0.7, 3)) * np.array(sp)
    rec = (lo + (hi - lo) * rng.uniform(0.0, 1.0, (nrec, 3))) * np.array(sp)
    f0 = vs.min() / (8.0 * max(sp))
    if kind == "moment":
        comp = double_couple(*rng.uniform(0, 90, 3))
    else:
        comp = rng.standard_normal(3) * 1e10
    return Problem(f"small_{nx}x{ny}x{nz}_{boundary}_{kind}", nx, ny, nz, sp, dt, nt,
                   vp, vs, rho, kind, src, comp, _wavelet_for(kind, nt, dt, f0), rec,
                   boundary, width, float(f0))


def with_coarse_medium(prob: Problem, m, seed: int = SEED, layer_vp=None) -> Problem:
    """The problem with its medium given on a grid of m = (mx, my, mz) cells
    over the same box (the paper's coarse medium textures, Sec. 2.2.1): the
    layered-plus-random recipe drawn at that resolution (cell size n h / m
    per axis), as Lame parameters and density.  The problem's own vp / vs /
    rho stay as they were (the CFL step is kept: the coarse speeds come from
    the same layer table)."""
    mx, my, mz = (int(a) for a in m)
    sp = tuple(prob.spacing[a] * (prob.nx, prob.ny, prob.nz)[a] / (mx, my, mz)[a] for a in range(3))
    kw = {} if layer_vp is None else {"layer_vp": layer_vp}
    vp, vs, rho = layered_random(mx, my, mz, sp, corr_len=4 * max(sp), seed=seed, **kw)
    vp64, vs64, rho64 = (a.astype(np.float64) for a in (vp, vs, rho))
    mu = rho64 * vs64 * vs64
    lam = rho64 * vp64 * vp64 - 2.0 * mu
    prob.coarse_medium = (lam.astype(np.float32), mu.astype(np.float32), rho.astype(np.float32))
    return prob


def random_state(nx: int, ny: int, nz: int, seed: int = SEED,
                 scale: float = 1.0) -> np.ndarray:
    """Seeded random wavefield state [9][nz][ny][nx] (vx, vy, vz, sxx, syy,
    szz, sxy, sxz, syz), float32."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((9, nz, ny, nx), dtype=np.float32)
            * np.float32(scale))
