"""Seeded synthetic CMOS-like frames for the L.A.Cosmic workloads.

This module only draws inputs; it contains none of the detection arithmetic,
and both the CUDA path's tests/benchmarks and the CPU oracle's tests feed on
it.  The paper measures on astroscrappy's mock data and an HST WFPC2 image,
neither of which ships here; these recipes stand in for them.

Recipe (per frame, in this order), with ``Generator(PCG64(SeedSequence(
[config_seed, frame_index])))``:

1. sky + Gaussian noise with sigma = sqrt(gain*sky + rn^2) / gain (ADU);
2. Gaussian-PSF stars, FWHM 2.5 px (sigma 1.0617 px), peak log-uniform in
   the given range, uniform sub-pixel positions, added noise-free;
3. cosmic-ray tracks: width 1 or 2 px, length U[1, 15] px, angle U[0, pi),
   amplitude U[200, 5000] ADU, rasterised as a constant-amplitude segment
   (a pixel is hit once per track; overlapping tracks add);
4. hot pixels SET to 3000 ADU; "salt-and-pepper" splits them half salt
   (3000 ADU) and half pepper (0 ADU);
5. uint16 frames: round half to even and clip to [0, 65535]; float32 frames
   are cast without rounding.

Densities scale with area from 20 stars and 200 tracks per 512 x 512.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FWHM_TO_SIGMA = 1.0 / 2.3548


@dataclass
class FrameSpec:
    ny: int
    nx: int
    dtype: str = "f32"  # "f32" or "u16"
    seed: tuple = (0, 0)
    sky: float = 100.0
    gain: float = 1.0
    readnoise: float = 1.5
    n_stars: int = 20
    n_tracks: int = 200
    hot_frac: float = 0.001
    salt_pepper: bool = False
    star_peak: tuple = (500.0, 20000.0)
    fwhm: float = 2.5
    satlevel: float = 65535.0
    niter: int = 4
    sigclip: float = 4.5
    sigfrac: float = 0.3
    objlim: float = 5.0
    extra: dict = field(default_factory=dict)

    @property
    def npix(self) -> int:
        return self.ny * self.nx


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(seed))))


def _add_stars(img: np.ndarray, rng, n, peak_lo, peak_hi, fwhm):
    if n <= 0:
        return
    ny, nx = img.shape
    sig = fwhm * FWHM_TO_SIGMA
    cy = rng.uniform(0, ny, n)
    cx = rng.uniform(0, nx, n)
    peak = np.exp(rng.uniform(math.log(peak_lo), math.log(peak_hi), n))
    h = int(math.ceil(6 * sig))
    off = np.arange(-h, h + 1)
    iy = np.floor(cy).astype(np.int64)[:, None, None] + off[None, :, None]
    ix = np.floor(cx).astype(np.int64)[:, None, None] + off[None, None, :]
    dy = (iy + 0.5) - cy[:, None, None]
    dx = (ix + 0.5) - cx[:, None, None]
    val = peak[:, None, None] * np.exp(-(dy * dy + dx * dx) / (2 * sig * sig))
    iy, ix = np.broadcast_arrays(iy, ix)
    ok = (iy >= 0) & (iy < ny) & (ix >= 0) & (ix < nx)
    np.add.at(img, (iy[ok], ix[ok]), val[ok].astype(img.dtype))


def _add_tracks(img: np.ndarray, rng, n, amp_lo=200.0, amp_hi=5000.0):
    if n <= 0:
        return
    ny, nx = img.shape
    width = rng.integers(1, 3, n)
    length = rng.uniform(1.0, 15.0, n)
    ang = rng.uniform(0.0, math.pi, n)
    amp = rng.uniform(amp_lo, amp_hi, n)
    y0 = rng.uniform(0, ny, n)
    x0 = rng.uniform(0, nx, n)
    npts = np.ceil(2 * length).astype(np.int64) + 1
    tid = np.repeat(np.arange(n), npts)
    start = np.repeat(np.cumsum(npts) - npts, npts)
    t = (np.arange(tid.size) - start) / (npts[tid] - 1).clip(min=1)
    s = t * length[tid]
    py = y0[tid] + s * np.sin(ang[tid])
    px = x0[tid] + s * np.cos(ang[tid])
    iy = np.floor(py).astype(np.int64)
    ix = np.floor(px).astype(np.int64)
    # Second pixel column for width-2 tracks: step perpendicular to the track
    # along the axis where the normal is larger.
    w2 = width[tid] == 2
    ny_n = np.cos(ang[tid])  # normal direction (-sin, cos) -> (dy=cos, dx=-sin)
    nx_n = -np.sin(ang[tid])
    step_y = np.where(np.abs(ny_n) >= np.abs(nx_n), 1, 0)
    step_x = 1 - step_y
    iy = np.concatenate([iy, (iy + step_y)[w2]])
    ix = np.concatenate([ix, (ix + step_x)[w2]])
    tid = np.concatenate([tid, tid[w2]])
    ok = (iy >= 0) & (iy < ny) & (ix >= 0) & (ix < nx)
    key = tid[ok] * (ny * nx) + iy[ok] * nx + ix[ok]
    key = np.unique(key)
    t_u = key // (ny * nx)
    pix = key % (ny * nx)
    np.add.at(img.reshape(-1), pix, amp[t_u].astype(img.dtype))


def _hot_pixels(img: np.ndarray, rng, frac, salt_pepper):
    npx = img.size
    k = int(round(frac * npx))
    if k <= 0:
        return
    pos = rng.choice(npx, size=k, replace=False)
    flat = img.reshape(-1)
    if salt_pepper:
        half = k // 2
        flat[pos[:k - half]] = 3000.0
        flat[pos[k - half:]] = 0.0
    else:
        flat[pos] = 3000.0


def make_frame(spec: FrameSpec) -> np.ndarray:
    """Draw one frame from ``spec`` (float32 or uint16, row-major ny x nx)."""
    rng = _rng(spec.seed)
    sigma = math.sqrt(spec.gain * spec.sky + spec.readnoise ** 2) / spec.gain
    img = rng.standard_normal((spec.ny, spec.nx), dtype=np.float32)
    img *= np.float32(sigma)
    img += np.float32(spec.sky)
    _add_stars(img, rng, spec.n_stars, spec.star_peak[0], spec.star_peak[1], spec.fwhm)
    _add_tracks(img, rng, spec.n_tracks)
    _hot_pixels(img, rng, spec.hot_frac, spec.salt_pepper)
    if spec.dtype == "u16":
        np.rint(img, out=img)
        np.clip(img, 0, 65535, out=img)
        return img.astype(np.uint16)
    return img


def scaled(n_per_512sq: float, ny: int, nx: int) -> int:
    return int(round(n_per_512sq * ny * nx / (512 * 512)))


def config_specs(index: int, count: int | None = None) -> list[FrameSpec]:
    """Frame specs for the five workloads (index 0..4), optionally truncated."""
    specs: list[FrameSpec] = []
    if index == 0:
        specs = [FrameSpec(512, 512, "f32", (0, 0))]
    elif index == 1:
        ny, nx = 6388, 9576
        specs = [FrameSpec(ny, nx, "u16", (1, 0), sky=300.0, gain=0.8, readnoise=1.2,
                           n_stars=4000, n_tracks=150000, hot_frac=0.005, salt_pepper=True)]
    elif index == 2:
        rng = _rng((2, 1 << 20))
        sizes = [(2048, 2048, "f32")] * 16 + [(3072, 4096, "u16")] * 16 + [(6388, 9576, "u16")] * 32
        for i, (ny, nx, dt) in enumerate(sizes):
            g = float(rng.uniform(0.5, 1.5))
            rn = float(rng.uniform(1.0, 3.0))
            specs.append(FrameSpec(ny, nx, dt, (2, i), sky=100.0, gain=g, readnoise=rn,
                                   n_stars=scaled(20, ny, nx), n_tracks=scaled(200, ny, nx)))
    elif index == 3:
        rng = _rng((3, 1 << 20))
        n = count if count is not None else 1000
        for i in range(n):
            if rng.uniform() < 0.1:
                ny, nx, dt = 2048, 2048, "f32"
            else:
                ny, nx, dt = 6388, 9576, "u16"
            specs.append(FrameSpec(ny, nx, dt, (3, i), sky=100.0, gain=1.0, readnoise=1.5,
                                   n_stars=scaled(20, ny, nx), n_tracks=scaled(200, ny, nx)))
    elif index == 4:
        ny, nx = 6388, 9576
        for i in range(256):
            specs.append(FrameSpec(ny, nx, "u16", (4, i), sky=300.0, gain=0.8, readnoise=1.2,
                                   n_stars=200, star_peak=(1e5, 1e6), n_tracks=750000,
                                   hot_frac=0.01, salt_pepper=True, niter=(1, 4, 6)[i % 3]))
    else:
        raise ValueError(index)
    if count is not None:
        specs = specs[:count]
    return specs


def poisson_arrivals(rate_hz: float, n: int, seed=(3, 1 << 21)) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with ``rate_hz`` requests per second."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


def make_frames_parallel(specs: list[FrameSpec], workers: int | None = None) -> list[np.ndarray]:
    """make_frame over many specs on a thread pool (the same frames, faster:
    numpy's heavy parts release the GIL; no child processes are involved)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    n = workers or min(len(specs), os.cpu_count() or 1)
    if n <= 1 or len(specs) <= 1:
        return [make_frame(s) for s in specs]
    with ThreadPoolExecutor(n) as ex:
        return list(ex.map(make_frame, specs))
