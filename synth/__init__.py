"""Seeded synthetic inputs for the tiled Hogbom CLEAN workloads.

This module builds inputs only: point spread functions, point-source skies,
dirty images and small adversarial test images.  It holds none of the CLEAN
arithmetic (no peak search, no subtraction, no feedback), so both the CPU
oracle and the CUDA path can take their inputs from here without sharing any
part of the method.

The paper deconvolves a simulated VLA configuration-D point-source image
(Section 1) that is not distributed with it.  The generator below stands in
for it: a Y-shaped array of 27 antennas, earth-rotation synthesis over eight
hours at declination +45 deg, natural weighting, and a sky of point sources
with one bright 2.1 Jy source (the brightest flux quoted in Section 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "y_array_enu", "uv_tracks", "make_psf", "make_sky", "make_dirty",
    "fit_beam", "Workload", "workload", "WORKLOADS",
    "random_psf", "random_image", "tie_image", "batch_jobs", "serving_stream",
]

# ---------------------------------------------------------------------------
# Array and uv coverage
# ---------------------------------------------------------------------------

def y_array_enu(n_per_arm: int = 9, r_max: float = 600.0,
                alpha: float = 1.716) -> np.ndarray:
    """East/North/Up positions (metres) of a Y-shaped array.

    Three arms at azimuths 0, 120 and 240 degrees, ``n_per_arm`` antennas per
    arm at radii r_k = r_max * (k / n_per_arm) ** alpha, k = 1..n_per_arm
    (the VLA's power-law arm spacing).  Returns shape (3 * n_per_arm, 3).
    """
    pos = []
    for az_deg in (0.0, 120.0, 240.0):
        az = math.radians(az_deg)
        for k in range(1, n_per_arm + 1):
            r = r_max * (k / n_per_arm) ** alpha
            pos.append((r * math.sin(az), r * math.cos(az), 0.0))
    return np.asarray(pos, dtype=np.float64)


def uv_tracks(lat_deg: float = 34.08, dec_deg: float = 45.0,
              n_ha: int = 64, ha_half_span_h: float = 4.0,
              enu: np.ndarray | None = None) -> np.ndarray:
    """(u, v) samples in metres for every baseline and hour angle.

    Antenna positions are rotated from the local horizon frame to equatorial
    XYZ at latitude ``lat_deg``; each baseline is projected for ``n_ha`` hour
    angles evenly spaced over +-``ha_half_span_h`` hours at declination
    ``dec_deg``.  Returns shape (n_baselines * n_ha, 2).
    """
    if enu is None:
        enu = y_array_enu()
    lat = math.radians(lat_deg)
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    X = -n * math.sin(lat) + u * math.cos(lat)
    Y = e
    Z = n * math.cos(lat) + u * math.sin(lat)
    xyz = np.stack([X, Y, Z], axis=1)
    i, j = np.triu_indices(len(enu), k=1)
    b = xyz[j] - xyz[i]                                   # (nb, 3)
    ha = np.linspace(-ha_half_span_h, ha_half_span_h, n_ha) * (math.pi / 12.0)
    dec = math.radians(dec_deg)
    sh, ch = np.sin(ha)[None, :], np.cos(ha)[None, :]
    bx, by, bz = b[:, 0:1], b[:, 1:2], b[:, 2:3]
    uu = sh * bx + ch * by
    vv = -math.sin(dec) * ch * bx + math.sin(dec) * sh * by + math.cos(dec) * bz
    return np.stack([uu.ravel(), vv.ravel()], axis=1)


def make_psf(py: int, px: int, freq_scale: float = 1.0,
             longest_frac: float = 0.1) -> np.ndarray:
    """Point spread function of the Y array on a ``py`` x ``px`` grid, float32.

    (u, v) and (-u, -v) are gridded to the nearest cell with natural
    weighting (sample counts); the longest projected baseline lands at
    ``longest_frac * px * freq_scale`` cells from the grid centre.  The PSF is
    the real part of the inverse FFT (float64), centred at (py // 2, px // 2)
    and normalised to 1 there.  Every off-centre value is strictly below 1 in
    magnitude (asserted).
    """
    uv = uv_tracks()
    scale = longest_frac * px * freq_scale / np.max(np.hypot(uv[:, 0], uv[:, 1]))
    iu = np.rint(uv[:, 0] * scale).astype(np.int64)
    iv = np.rint(uv[:, 1] * scale).astype(np.int64)
    iu = np.concatenate([iu, -iu]) + px // 2
    iv = np.concatenate([iv, -iv]) + py // 2
    ok = (iu >= 0) & (iu < px) & (iv >= 0) & (iv < py)
    grid = np.zeros((py, px), dtype=np.float64)
    np.add.at(grid, (iv[ok], iu[ok]), 1.0)
    import scipy.fft as sfft
    img = np.fft.fftshift(sfft.ifft2(np.fft.ifftshift(grid), workers=-1).real)
    cy, cx = py // 2, px // 2
    img /= img[cy, cx]
    psf = img.astype(np.float32)
    psf[cy, cx] = np.float32(1.0)
    off = np.abs(psf).copy()
    off[cy, cx] = 0.0
    assert off.max() < 1.0, "PSF has an off-centre value of magnitude >= 1"
    return psf


# ---------------------------------------------------------------------------
# Sky and dirty image
# ---------------------------------------------------------------------------

def make_sky(n: int, n_sources: int, lo: float, hi: float = 2.1,
             rng: np.random.Generator | int = 0,
             margin: int = 0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Point sources at distinct pixels of an n x n image.

    One source has flux exactly ``hi``; the others are log-uniform in
    [lo, hi].  Positions are uniform over pixels at least ``margin`` from the
    image edge.  Returns (ys, xs, flux) as int64, int64, float64 arrays.
    """
    rng = np.random.default_rng(rng) if not isinstance(rng, np.random.Generator) else rng
    side = n - 2 * margin
    flat = rng.choice(side * side, size=n_sources, replace=False)
    ys = flat // side + margin
    xs = flat % side + margin
    flux = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_sources))
    flux[0] = hi
    return ys.astype(np.int64), xs.astype(np.int64), flux


def make_dirty(psf: np.ndarray, n: int, ys: np.ndarray, xs: np.ndarray,
               flux: np.ndarray, sigma: float,
               rng: np.random.Generator | int = 0) -> np.ndarray:
    """Dirty image = sum of flux * PSF shifted to each source + noise, float32.

    The PSF centre (py // 2, px // 2) lands on the source pixel; PSF values
    outside the PSF array contribute nothing.  Accumulated in float64 (a
    direct gather for small images, an exact-size FFT convolution for large
    ones), plus white Gaussian noise of standard deviation ``sigma``.
    """
    rng = np.random.default_rng(rng) if not isinstance(rng, np.random.Generator) else rng
    py, px = psf.shape
    cy, cx = py // 2, px // 2
    p64 = psf.astype(np.float64)
    full = py >= 2 * n - 1 and px >= 2 * n - 1 and cy >= n - 1 and cx >= n - 1
    if len(flux) * n * n <= 2e8 or not full:
        d = np.zeros((n, n), dtype=np.float64)
        for y, x, s in zip(ys, xs, flux):
            # rows q with 0 <= q - y + cy < py, likewise for columns
            q0y, q1y = max(0, y - cy), min(n, y - cy + py)
            q0x, q1x = max(0, x - cx), min(n, x - cx + px)
            if q0y >= q1y or q0x >= q1x:
                continue
            d[q0y:q1y, q0x:q1x] += s * p64[q0y - y + cy:q1y - y + cy,
                                            q0x - x + cx:q1x - x + cx]
    else:
        import scipy.fft as sfft
        sky = np.zeros((py, px), dtype=np.float64)
        np.add.at(sky, (ys, xs), flux)
        conv = sfft.irfft2(sfft.rfft2(sky, workers=-1) * sfft.rfft2(p64, workers=-1),
                           s=(py, px), workers=-1)
        # circular index (q + c - s) mod P never wraps for q, s in [0, n)
        d = conv[cy:cy + n, cx:cx + n].copy()
    d += rng.normal(0.0, sigma, size=(n, n))
    return d.astype(np.float32)


def fit_beam(psf: np.ndarray, level: float = 0.5) -> tuple[float, float, float]:
    """Gaussian clean beam (FWHM major px, FWHM minor px, position angle rad).

    Fits log P over the PSF main lobe (the 4-connected pixels >= ``level``
    around the centre) by least squares with the quadratic form
    -(a dx^2 + 2 b dx dy + c dy^2) / 2 (peak fixed at 1), which is exact for
    a sampled Gaussian.  The angle of the major axis is measured from +x
    (columns) toward +y (rows).
    """
    py, px = psf.shape
    cy, cx = py // 2, px // 2
    seen = {(cy, cx)}
    stack = [(cy, cx)]
    while stack:
        y, x = stack.pop()
        for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            yy, xx = y + dy, x + dx
            if 0 <= yy < py and 0 <= xx < px and (yy, xx) not in seen \
                    and psf[yy, xx] >= level:
                seen.add((yy, xx))
                stack.append((yy, xx))
    pts = np.array(sorted(seen), dtype=np.int64)
    v = psf[pts[:, 0], pts[:, 1]].astype(np.float64) / float(psf[cy, cx])
    dy = (pts[:, 0] - cy).astype(np.float64)
    dx = (pts[:, 1] - cx).astype(np.float64)
    keep = (dy != 0) | (dx != 0)
    A = np.stack([dx * dx, 2 * dx * dy, dy * dy], axis=1)[keep]
    rhs = -2.0 * np.log(v[keep])
    (a, b, c), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    inv = np.array([[a, b], [b, c]])              # inverse covariance (x, y)
    evals, evecs = np.linalg.eigh(inv)            # ascending: major axis first
    evals = np.maximum(evals, 1e-12)
    smaj, smin = 1.0 / math.sqrt(evals[0]), 1.0 / math.sqrt(evals[1])
    vx, vy = evecs[0, 0], evecs[1, 0]
    pa = math.atan2(vy, vx)
    pa = (pa + math.pi / 2) % math.pi - math.pi / 2
    k = 2.0 * math.sqrt(2.0 * math.log(2.0))
    return k * smaj, k * smin, pa


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    psf_n: int
    n_sources: int
    lo: float
    sigma: float
    gain: float
    niter: int
    threshold: float
    tiles: tuple[int, int]
    feedback_interval: int
    seed: int
    extra: dict = field(default_factory=dict)

    def build(self, threshold: float | None = None):
        """Returns dict(psf, dirty, sky, params) for this workload."""
        psf = make_psf(self.psf_n, self.psf_n)
        rng = np.random.default_rng(self.seed)
        ys, xs, fl = make_sky(self.n, self.n_sources, self.lo, 2.1, rng)
        dirty = make_dirty(psf, self.n, ys, xs, fl, self.sigma, rng)
        return dict(psf=psf, dirty=dirty, sky=(ys, xs, fl),
                    gain=self.gain, niter=self.niter,
                    threshold=self.threshold if threshold is None else threshold,
                    tiles=self.tiles, K=self.feedback_interval)


WORKLOADS = {
    # plain untiled CLEAN: 256^2 image, 512^2 PSF, 20 sources
    "untiled-256": Workload("untiled-256", 256, 512, 20, 0.05, 1e-3, 0.1,
                            2000, 5e-3, (1, 1), 0, 1000),
    # tiled with feedback: 1024^2 image, 2048^2 PSF, 2x2 tiles, K = 50
    "tiled-1024": Workload("tiled-1024", 1024, 2048, 80, 0.05, 1e-3, 0.1,
                           10000, 5e-3, (2, 2), 50, 1001),
    # tiled with feedback: 4096^2 image, 8192^2 PSF, 4x4 tiles, K = 50
    "tiled-4096": Workload("tiled-4096", 4096, 8192, 500, 1e-3, 1e-3, 0.1,
                           50000, 0.0, (4, 4), 50, 1002),
}


def workload(name: str, **over) -> Workload:
    w = WORKLOADS[name]
    if over:
        w = Workload(**{**w.__dict__, **over})
    return w


# ---------------------------------------------------------------------------
# Small adversarial inputs for tests
# ---------------------------------------------------------------------------

def random_psf(py: int, px: int, rng, peak_margin: float = 0.05) -> np.ndarray:
    """Random signed float32 PSF, value 1 at (py//2, px//2), |P| < 1 elsewhere."""
    rng = np.random.default_rng(rng) if not isinstance(rng, np.random.Generator) else rng
    p = rng.uniform(-(1 - peak_margin), 1 - peak_margin, size=(py, px)).astype(np.float32)
    p[py // 2, px // 2] = 1.0
    return p


def random_image(ny: int, nx: int, rng, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(rng) if not isinstance(rng, np.random.Generator) else rng
    return (rng.standard_normal((ny, nx)) * scale).astype(np.float32)


def tie_image(ny: int, nx: int, rng, levels: int = 3) -> np.ndarray:
    """Integer-valued signed image with many equal |values| (tie-heavy)."""
    rng = np.random.default_rng(rng) if not isinstance(rng, np.random.Generator) else rng
    return rng.integers(-levels, levels + 1, size=(ny, nx)).astype(np.float32)


def batch_jobs(n_images: int = 64, seed: int = 1003, niter: int = 2000, n_sources: int = 40):
    """Uneven multi-channel batch: sides drawn uniformly from {512, 1024, 1536,
    2048}, per-channel PSFs from the same array with frequency scaling
    linspace(1, 2, n_images), 2 x 2 tiles up to 1024 and 4 x 4 above, K = 50,
    gain 0.1, threshold 0.  Returns a list of dicts (n, psf, dirty, tiles, K,
    niter, gain)."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([512, 1024, 1536, 2048], size=n_images)
    freqs = np.linspace(1.0, 2.0, n_images)
    jobs = []
    for i in range(n_images):
        n = int(sides[i])
        psf = make_psf(2 * n, 2 * n, freq_scale=float(freqs[i]))
        ys, xs, fl = make_sky(n, n_sources, 0.01, 2.1, rng)
        dirty = make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
        jobs.append(dict(n=n, psf=psf, dirty=dirty, tiles=(2, 2) if n <= 1024 else (4, 4),
                         K=50, niter=niter, gain=0.1))
    return jobs


def serving_stream(psf_full, n_jobs: int = 500, seed: int = 1004, lo: int = 256,
                   hi: int = 4096, step: int = 64, device: str = "cuda"):
    """Serving stream of independent jobs, built on the GPU (torch).

    Each job: side n log-uniform over [lo, hi] rounded to a multiple of
    ``step`` (so most sides are not powers of two), 10 - 500 point sources
    (log-uniform 10 mJy .. 2.1 Jy, one at 2.1 Jy), 1000 - 20000 iterations,
    gain 0.1, K 50, tiles 1x1 up to 256, 2x2 up to 1024, 4x4 above, its own
    dirty image = sum of flux * PSF shifted (float64) + white noise
    sigma = 1 mJy (a torch generator seeded 10000 + job).  The PSF of a side n
    is the central 2n x 2n crop of ``psf_full`` (the Y-array PSF on a grid of
    at least 2 hi: its main lobe and near sidelobes sit at the same pixel
    scale for every size); jobs of one side share it.  Returns a list of dicts
    (n, n_sources, niter, tiles, K, gain, psf, dirty) with CUDA float32
    tensors."""
    import torch
    rng = np.random.default_rng(seed)
    P = torch.as_tensor(psf_full, device=device)
    cy, cx = P.shape[0] // 2, P.shape[1] // 2
    sides = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_jobs))
    sides = np.clip(np.rint(sides / step) * step, lo, hi).astype(np.int64)
    crops, crops64 = {}, {}
    jobs = []
    for j in range(n_jobs):
        n = int(sides[j])
        if n not in crops:
            c = P[cy - n:cy + n, cx - n:cx + n].contiguous()
            crops[n], crops64[n] = c, c.double()
        ns = int(rng.integers(10, 501))
        niter = int(rng.integers(1000, 20001))
        ys, xs, fl = make_sky(n, ns, 0.01, 2.1, rng)
        p64 = crops64[n]
        d = torch.zeros((n, n), dtype=torch.float64, device=device)
        for y, x, f in zip(ys.tolist(), xs.tolist(), fl.tolist()):
            # pixel q takes P[q - source + centre]; the crop's centre is (n, n)
            d += f * p64[n - y:2 * n - y, n - x:2 * n - x]
        g = torch.Generator(device=device)
        g.manual_seed(10000 + j)
        d += 1e-3 * torch.randn((n, n), generator=g, dtype=torch.float64, device=device)
        tiles = (1, 1) if n <= 256 else (2, 2) if n <= 1024 else (4, 4)
        jobs.append(dict(n=n, n_sources=ns, niter=niter, tiles=tiles, K=50, gain=0.1,
                         psf=crops[n], dirty=d.float().contiguous()))
    return jobs
