"""Seeded synthetic cubes shaped like the paper's datasets.

The paper's datasets (DynamicEarthNet, DeepExtremeCubes, SimpleS2, ERA5;
Sec. 2.2) are not available here, so these generators stand in for them with
the same shapes, value ranges and kinds of structure.  This module holds no
step of the compression method: it only draws inputs, and both the CUDA path
and the CPU oracle are fed from it.  Every draw comes from
``numpy.random.default_rng(seed)`` with ``seed = seed_base + cube`` (a seed
base per workload).

The DeepExtremeCubes-, DynamicEarthNet- and ERA5-shaped generators are
frame-addressable: ``T`` may be smaller than the workload's length to draw a
causal prefix (the first ``T`` frames are the same numbers a full draw would
give).  The tiny generator is not: its motion steps and noise come from one
stream whose use depends on ``T``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class EncoderConfig:
    """Encoder parameters of one workload (restates the paper's mapping_rules)."""
    name: str
    seed_base: int        # seeds of the workload's cubes: seed_base + cube
    bands: int
    T: int
    H: int
    W: int
    dtype: str            # "f32" or "u16"
    ctu: int
    R: int
    tu_sizes: tuple       # allowed TU sizes
    qps: tuple            # QPs the workload is run at
    sub_T: tuple = field(default=())  # uneven sub-cube lengths (ERA5-shaped batch)

    @property
    def tu_mask(self) -> int:
        m = 0
        for n in self.tu_sizes:
            m |= 1 << (int(n).bit_length() - 1)
        return m


# The workloads, by what they stand in for (in this order: the serving
# stream draws its kinds by position).
WORKLOADS = {
    "tiny": EncoderConfig("tiny-3x8x64x64", 0, 3, 8, 64, 64, "f32", 8, 16, (8,), (27,)),
    "deepextremecubes": EncoderConfig("deepextremecubes-10x256x128x128", 1000, 10, 256, 128, 128, "f32", 16, 32,
                                      (4, 8, 16), (22, 27, 32)),
    "dynamicearthnet": EncoderConfig("dynamicearthnet-4x300x1024x1024", 2000, 4, 300, 1024, 1024, "u16", 64, 64,
                                     (4, 8, 16, 32), (27,)),
    "era5": EncoderConfig("era5-6x721x1440-subcubes", 3000, 6, 168, 721, 1440, "f32", 32, 16,
                          (4, 8, 16, 32), (22,), sub_T=(24, 53, 82, 110, 139, 168)),
}


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(np.ceil(3 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def _blur_periodic(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian filter with wrap-around borders (FFT)."""
    H, W = a.shape
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    g = np.exp(-2.0 * (np.pi ** 2) * (sigma ** 2) * (kx ** 2 + ky ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(a) * g))


# ------------------------------------------------------------------ tiny
def tiny_cube(seed: int = 0, T: int = 8, H: int = 64, W: int = 64, bands: int = 3):
    """Gaussian blobs translated by seeded integer steps in [-4, 4]^2 plus N(0, 0.002).

    Returns (cube float32 [bands,T,H,W], cumulative shifts S [T,2] as (sx, sy)).
    Frame t is the frame-0 field evaluated at x - S_t, so content moves by S_t
    and the motion vector that predicts frame t from frame t-1 is -(S_t - S_{t-1}).
    """
    rng = np.random.default_rng(seed)
    n = 12
    cx = rng.uniform(0, W, (bands, n))
    cy = rng.uniform(0, H, (bands, n))
    sg = rng.uniform(4, 16, (bands, n))
    amp = rng.uniform(0.2, 1.0, (bands, n))
    steps = rng.integers(-4, 5, size=(T, 2))
    steps[0] = 0
    S = np.cumsum(steps, axis=0)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.empty((bands, T, H, W), np.float32)
    for b in range(bands):
        def field(ox, oy):
            f = np.zeros((H, W))
            for k in range(n):
                f += amp[b, k] * np.exp(-((xx - ox - cx[b, k]) ** 2 + (yy - oy - cy[b, k]) ** 2)
                                        / (2 * sg[b, k] ** 2))
            return f
        peak = field(0, 0).max()
        for t in range(T):
            f = field(S[t, 0], S[t, 1]) / peak
            f = f + rng.normal(0, 0.002, (H, W))
            out[b, t] = np.clip(f, 0, 1)
    return out, S


# ------------------------------------------------------------------ DeepExtremeCubes-shaped
def deepextremecubes_cube(seed: int = 1000, T: int = 256, H: int = 128, W: int = 128, bands: int = 10,
                          T_full: int | None = None):
    """Beta(2,5) reflectance via a Gaussian copula of smooth noise (sigma 6 px),
    0.7 shared + 0.3 per band, seasonal modulation 1 + 0.3 sin(2 pi t / 73 + phi_b),
    N(0, 0.005) noise, and 15% of frames carrying 1-5 cloud blobs (sigma 8-32 px)
    that blend every band towards a U(0.8, 1.0) brightness.  Clipped to [0, 1]."""
    from scipy.special import ndtr
    from scipy.stats import beta as beta_dist

    T_full = T_full or T
    rng = np.random.default_rng(seed)
    shared = _blur_periodic(rng.normal(size=(H, W)), 6.0)
    shared /= shared.std()
    phis = rng.uniform(0, 2 * np.pi, bands)
    base = np.empty((bands, H, W))
    for b in range(bands):
        own = _blur_periodic(rng.normal(size=(H, W)), 6.0)
        own /= own.std()
        z = 0.7 * shared + 0.3 * own
        z /= z.std()
        base[b] = beta_dist.ppf(ndtr(z), 2, 5)
    out = np.empty((bands, T, H, W), np.float32)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for t in range(T):
        frng = np.random.default_rng([seed, t])
        season = 1.0 + 0.3 * np.sin(2 * np.pi * t / 73.0 + phis)
        fr = base * season[:, None, None] + frng.normal(0, 0.005, (bands, H, W))
        if frng.random() < 0.15:
            alpha = np.zeros((H, W))
            for _ in range(int(frng.integers(1, 6))):
                s = frng.uniform(8, 32)
                cx, cy = frng.uniform(0, W), frng.uniform(0, H)
                alpha = np.maximum(alpha, np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s)))
            bright = frng.uniform(0.8, 1.0)
            fr = (1 - alpha) * fr + alpha * bright
        out[:, t] = np.clip(fr, 0, 1)
    return out


# ------------------------------------------------------------------ DynamicEarthNet-shaped
def dynamicearthnet_cube(seed: int = 2000, T: int = 300, H: int = 1024, W: int = 1024, bands: int = 4,
                         n_seeds: int = 200):
    """Piecewise-constant Voronoi land-cover patches (200 seeds) with per-patch
    lognormal(ln 1500, 0.6) reflectance, slow drift x(1 + 0.002 t d_p),
    d_p ~ N(0,1), plus N(0, 50) noise; rounded and clipped to uint16 [0, 10000]."""
    rng = np.random.default_rng(seed)
    sx = rng.uniform(0, W, n_seeds)
    sy = rng.uniform(0, H, n_seeds)
    level = rng.lognormal(np.log(1500.0), 0.6, (bands, n_seeds))
    drift = rng.normal(0, 1, n_seeds)
    # nearest seed per pixel, computed row block by row block
    label = np.empty((H, W), np.int32)
    xs = np.arange(W, dtype=np.float64)
    for y0 in range(0, H, 64):
        ys = np.arange(y0, min(H, y0 + 64), dtype=np.float64)
        d = (ys[:, None, None] - sy[None, None, :]) ** 2 + (xs[None, :, None] - sx[None, None, :]) ** 2
        label[y0:y0 + len(ys)] = np.argmin(d, axis=2)
    out = np.empty((bands, T, H, W), np.uint16)
    for t in range(T):
        frng = np.random.default_rng([seed, t])
        for b in range(bands):
            v = (level[b] * (1.0 + 0.002 * t * drift))[label]
            v = v + frng.normal(0, 50, (H, W))
            out[b, t] = np.clip(np.rint(v), 0, 10000).astype(np.uint16)
    return out


# ------------------------------------------------------------------ ERA5-shaped
def era5_cube(seed: int = 3000, T: int = 24, H: int = 721, W: int = 1440, bands: int = 6):
    """Smooth spectral random fields, P(k) ~ k^-3, advected zonally (periodic in
    longitude) by u ~ U(2, 6) px/frame, plus a diurnal term 0.2 sigma
    sin(2 pi (t/24 + x/1440)).  float32."""
    rng = np.random.default_rng(seed)
    ky = np.fft.fftfreq(H)[:, None] * H
    kx = np.fft.rfftfreq(W)[None, :] * W
    k = np.sqrt(kx ** 2 + ky ** 2)
    k[0, 0] = 1.0
    amp = k ** (-1.5)  # amplitude ~ sqrt(P(k)), P ~ k^-3
    amp[0, 0] = 0.0
    u = rng.uniform(2, 6, bands)
    spec = [amp * (rng.normal(size=amp.shape) + 1j * rng.normal(size=amp.shape)) for _ in range(bands)]
    offs = rng.uniform(-1, 1, bands)
    out = np.empty((bands, T, H, W), np.float32)
    xx = np.arange(W)[None, :]
    for b in range(bands):
        f0 = np.fft.irfft2(spec[b], s=(H, W))
        sd = f0.std()
        for t in range(T):
            phase = np.exp(-2j * np.pi * kx * (u[b] * t) / W)
            f = np.fft.irfft2(spec[b] * phase, s=(H, W)) / sd
            f = f + 0.2 * np.sin(2 * np.pi * (t / 24.0 + xx / 1440.0)) + offs[b]
            out[b, t] = f
    return out


def make_cube(workload: str, cube: int = 0, T: int | None = None):
    """The synthetic cube of a workload (float32 or uint16 [bands, T, H, W])."""
    c = WORKLOADS[workload]
    seed = c.seed_base + cube
    if workload == "tiny":
        return tiny_cube(seed, T=T or c.T)[0]
    if workload == "deepextremecubes":
        return deepextremecubes_cube(seed, T=T or c.T)
    if workload == "dynamicearthnet":
        return dynamicearthnet_cube(seed, T=T or c.T)
    if workload == "era5":
        return era5_cube(seed, T=T or c.sub_T[0])
    raise ValueError(workload)


def random_planes(seed: int, G: int, T: int, Hp: int, Wp: int, smooth: float = 0.0):
    """Random 10-bit planes [G,T,3,Hp,Wp] (optionally smoothed) for kernel tests."""
    rng = np.random.default_rng(seed)
    p = rng.integers(0, 1024, size=(G, T, 3, Hp, Wp)).astype(np.float64)
    if smooth > 0:
        for idx in np.ndindex(G, T, 3):
            p[idx] = _blur_periodic(p[idx], smooth)
        p = (p - p.min()) / max(1e-9, p.max() - p.min()) * 1023
    return np.clip(np.rint(p), 0, 1023).astype(np.uint16)


def serving_requests(seed: int = 4000, n: int = 2000, mean_interval_s: float = 0.005):
    """Poisson arrival times and uniformly drawn workload kinds for the serving run.

    Returns a list of dicts (arrival_s, workload, qp, T, cube)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(mean_interval_s, n))
    names = list(WORKLOADS)
    out = []
    for i in range(n):
        name = names[int(rng.integers(0, 4))]
        c = WORKLOADS[name]
        qp = int(rng.choice(c.qps))
        T = int(rng.choice(c.sub_T)) if c.sub_T else c.T
        out.append(dict(arrival_s=float(t[i]), workload=name, qp=qp, T=T, cube=int(rng.integers(0, 4))))
    return out
