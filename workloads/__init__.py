"""Seeded synthetic inputs for the SSA workloads.

This module only *draws data*: series, images, masks and request mixes with the
shapes, sizes and value distributions of the workloads the library is measured
on.  It holds none of the SSA arithmetic (no embedding, no SVD, no averaging),
so both the CUDA path and the CPU oracle may consume it.

Conventions
-----------
* A 2D image is a numpy array ``x`` of shape ``(Nx, Ny)``: ``x[m, n]`` with the
  x axis pointing down (rows) and the y axis pointing right (columns), the
  paper's orientation (Sec. 4.1.1).  Its vectorisation is column-major
  (``order='F'``), the paper's ``vec``.
* Missing pixels are NaN; an explicit observation mask (True = observed) may be
  given beside the image.
* Every generator takes an integer seed and uses ``numpy.random.default_rng``,
  whose streams are identical across platforms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "series_1d", "mssa_series", "harmonic_image", "disc_with_holes_mask",
    "shaped_image", "window_circle", "window_triangle", "serving_requests",
    "Request", "CONFIGS",
]


# ---------------------------------------------------------------- 1D series
def series_1d(n: int = 1000, seed: int = 1) -> np.ndarray:
    """Trend + two sines + white noise, t = 1..n, float64.

    ``0.01 t + sin(2 pi t/12) + 0.5 sin(2 pi t/37) + N(0, 0.1^2)``.
    """
    rng = np.random.default_rng(seed)
    t = np.arange(1, n + 1, dtype=np.float64)
    x = 0.01 * t + np.sin(2 * np.pi * t / 12) + 0.5 * np.sin(2 * np.pi * t / 37)
    return x + rng.normal(0.0, 0.1, size=n)


def mssa_series(s: int = 16, n_lo: int = 2000, n_hi: int = 8000, seed: int = 2,
                periods=(12, 50), amp=(0.5, 2.0), growth: float = 0.0002,
                noise: float = 0.2, dtype=np.float32) -> list[np.ndarray]:
    """``s`` series of uneven lengths ``N_p ~ U{n_lo..n_hi}``.

    Each series is ``sum_h A_{p,h} sin(2 pi t/P_h + phi_{p,h}) + exp(growth t)
    + N(0, noise^2)``, t = 1..N_p, with ``A ~ U[amp]`` and ``phi ~ U[0, 2 pi)``
    drawn per series and harmonic.
    """
    rng = np.random.default_rng(seed)
    lengths = rng.integers(n_lo, n_hi + 1, size=s)
    out = []
    for p in range(s):
        t = np.arange(1, lengths[p] + 1, dtype=np.float64)
        x = np.exp(growth * t)
        for P in periods:
            a = rng.uniform(*amp)
            ph = rng.uniform(0.0, 2 * np.pi)
            x = x + a * np.sin(2 * np.pi * t / P + ph)
        x = x + rng.normal(0.0, noise, size=lengths[p])
        out.append(x.astype(dtype))
    return out


# ------------------------------------------------------------------- images
def harmonic_image(nx: int = 1024, ny: int = 1024, n_harm: int = 4, seed: int = 3,
                   noise: float = 0.3, trend: bool = False,
                   dtype=np.float32) -> np.ndarray:
    """Sum of separable 2D harmonics plus white noise (plus a planar trend).

    ``x[m, n] = sum_k a_k cos(2 pi fx_k m + phi_k) cos(2 pi fy_k n + psi_k)``
    with ``f ~ U(0, 0.25)``, ``a ~ U[0.5, 1.5]``, phases ``U[0, 2 pi)``; noise
    ``N(0, noise^2)``.  With ``trend`` a plane ``c0 + c1 m/nx + c2 n/ny``,
    ``c ~ U[-1, 1]``, is added.
    """
    rng = np.random.default_rng(seed)
    m = np.arange(nx, dtype=np.float64)[:, None]
    n = np.arange(ny, dtype=np.float64)[None, :]
    x = np.zeros((nx, ny))
    for _ in range(n_harm):
        fx, fy = rng.uniform(0.0, 0.25, size=2)
        a = rng.uniform(0.5, 1.5)
        phi, psi = rng.uniform(0.0, 2 * np.pi, size=2)
        x += a * np.cos(2 * np.pi * fx * m + phi) * np.cos(2 * np.pi * fy * n + psi)
    if trend:
        c = rng.uniform(-1.0, 1.0, size=3)
        x += c[0] + c[1] * m / nx + c[2] * n / ny
    x += rng.normal(0.0, noise, size=(nx, ny))
    return x.astype(dtype)


def disc_with_holes_mask(nx: int = 2048, ny: int = 2048, n_holes: int = 40,
                         missing: float = 0.30, seed: int = 4,
                         tol: float = 0.005) -> tuple[np.ndarray, dict]:
    """Observation mask: a centred disc of radius ``min(nx, ny)/2`` minus
    ``n_holes`` circular holes of one common radius.

    Hole centres are uniform in the disc; the common radius is set by bisection
    so that the holes cover ``missing`` (+-tol) of the disc's pixels.  Returns
    the boolean mask (True = observed) and a dict with the realised numbers.
    """
    rng = np.random.default_rng(seed)
    R = min(nx, ny) / 2.0
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    m = np.arange(nx, dtype=np.float64)[:, None]
    n = np.arange(ny, dtype=np.float64)[None, :]
    disc = (m - cx) ** 2 + (n - cy) ** 2 <= R * R
    # centres uniform in the disc (polar draw with sqrt radius)
    rad = R * np.sqrt(rng.uniform(0.0, 1.0, size=n_holes))
    ang = rng.uniform(0.0, 2 * np.pi, size=n_holes)
    hx = cx + rad * np.cos(ang)
    hy = cy + rad * np.sin(ang)
    disc_px = int(disc.sum())

    def holes(r):
        h = np.zeros((nx, ny), dtype=bool)
        for i in range(n_holes):
            x0, x1 = max(0, int(hx[i] - r) - 1), min(nx, int(hx[i] + r) + 2)
            y0, y1 = max(0, int(hy[i] - r) - 1), min(ny, int(hy[i] + r) + 2)
            mm = m[x0:x1]
            nn = n[:, y0:y1]
            h[x0:x1, y0:y1] |= (mm - hx[i]) ** 2 + (nn - hy[i]) ** 2 <= r * r
        return h & disc

    lo, hi = 0.0, R
    r = R * math.sqrt(missing / n_holes)
    for _ in range(60):
        frac = holes(r).sum() / disc_px
        if abs(frac - missing) <= tol:
            break
        if frac < missing:
            lo = r
        else:
            hi = r
        r = 0.5 * (lo + hi)
    mask = disc & ~holes(r)
    info = {"hole_radius": r, "missing_fraction": float(1.0 - mask.sum() / disc_px),
            "observed_pixels": int(mask.sum()), "disc_pixels": disc_px}
    return mask, info


def shaped_image(nx: int = 2048, ny: int = 2048, seed: int = 4,
                 dtype=np.float32) -> tuple[np.ndarray, np.ndarray, dict]:
    """Harmonic image with a planar trend restricted to a disc with holes.

    Pixels outside the mask are set to NaN (missing).  Returns
    ``(image, mask, info)``.
    """
    x = harmonic_image(nx, ny, seed=seed, trend=True, dtype=dtype)
    mask, info = disc_with_holes_mask(nx, ny, seed=seed + 1000)
    x = x.copy()
    x[~mask] = np.nan
    return x, mask, info


# ----------------------------------------------------------- window shapes
def window_circle(R: int) -> np.ndarray:
    """Circular window of radius R: bounding box (2R+1)^2, pixel (i, j)
    (0-based) inside when (i-R)^2 + (j-R)^2 <= R^2."""
    i = np.arange(2 * R + 1)[:, None]
    j = np.arange(2 * R + 1)[None, :]
    return (i - R) ** 2 + (j - R) ** 2 <= R * R


def window_triangle(side: int) -> np.ndarray:
    """Isosceles right triangle with the right angle at the top-left corner of
    its side x side bounding box: pixel (i, j) inside when i + j <= side-1."""
    i = np.arange(side)[:, None]
    j = np.arange(side)[None, :]
    return i + j <= side - 1


# ----------------------------------------------------------------- serving
@dataclass
class Request:
    """One decomposition request of the serving mix."""
    rid: int
    arrival_s: float
    kind: str                 # "1d" | "mssa" | "2d"
    rank: int
    data: object              # ndarray (1d, 2d) or list of ndarrays (mssa)
    L: int = 0                # 1d / mssa window
    window: tuple = (0, 0)    # 2d window (Lx, Ly)
    mask: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


def serving_requests(n: int = 20000, rate_hz: float = 1000.0, seed: int = 5,
                     n_max: int = 200000, frac_series: float = 0.7,
                     side_lo: int = 64, side_hi: int = 512) -> list[Request]:
    """Poisson arrivals of a mixed request stream.

    70% series requests (half 1D, half MSSA with ``s ~ U{2..16}`` series of
    lengths ``U[N/2, N]``), ``N`` log-uniform in ``[500, n_max]``, ``L = N/2``
    (MSSA: ``floor(min N_p / 2)``), rank ``r ~ U{5..50}``; 30% square masked
    images of side ``U{side_lo..side_hi}`` with square windows ``U{16..48}``
    (clipped to a quarter of the side) and disc-with-holes masks scaled from
    the 2048^2 case.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    reqs = []
    for i in range(n):
        sub = int(rng.integers(0, 2**31 - 1))
        r = int(rng.integers(5, 51))
        if rng.uniform() < frac_series:
            N = int(round(math.exp(rng.uniform(math.log(500), math.log(n_max)))))
            if rng.uniform() < 0.5:
                x = series_1d(N, seed=sub)
                L = N // 2
                r = min(r, L - 1)
                reqs.append(Request(i, float(t[i]), "1d", r, x, L=L))
            else:
                s = int(rng.integers(2, 17))
                # the 16-series recipe's exp(0.0002 t) reaches e^1.6 at its
                # longest series (8000); longer series keep that end value
                # instead of growing to e^40 at 200,000 samples
                growth = 0.0002 * min(1.0, 8000.0 / max(N, 65))
                xs = mssa_series(s, max(N // 2, 64), max(N, 65), seed=sub, growth=growth)
                L = min(len(v) for v in xs) // 2
                r = min(r, L - 1)
                reqs.append(Request(i, float(t[i]), "mssa", r, xs, L=L))
        else:
            side = int(rng.integers(side_lo, side_hi + 1))
            w = int(min(rng.integers(16, 49), side // 4))
            img = harmonic_image(side, side, seed=sub, trend=True)
            holes = max(1, round(40 * (side / 2048) ** 2))
            mask, _ = disc_with_holes_mask(side, side, n_holes=holes, seed=sub + 1)
            img = img.copy()
            img[~mask] = np.nan
            # the rank is capped at 30 and at min(L, K): a large hole can leave
            # fewer admissible window positions than the drawn rank
            r = min(r, 30, w * w, _full_boxes(mask, w))
            reqs.append(Request(i, float(t[i]), "2d", r, img,
                                window=(w, w), mask=mask))
    return reqs


def _full_boxes(mask: np.ndarray, w: int) -> int:
    """Number of w x w boxes lying wholly inside ``mask`` (a request
    parameter of the generator: bounds the rank a masked image can take)."""
    c = np.zeros((mask.shape[0] + 1, mask.shape[1] + 1), dtype=np.int64)
    c[1:, 1:] = np.cumsum(np.cumsum(mask.astype(np.int64), axis=0), axis=1)
    box = c[w:, w:] - c[:-w, w:] - c[w:, :-w] + c[:-w, :-w]
    return int(np.count_nonzero(box == w * w))


# Workload catalogue: sizes only (the data comes from the generators above).
CONFIGS = {
    "series_1d_n1000": dict(kind="1d", n=1000, L=500, rank=10, seed=1,
                            groups=[[0, 1], [2, 3]], residual=True),
    "mssa_16x2000-8000_L1000": dict(kind="mssa", s=16, L=1000, rank=20, seed=2),
    "image_1024x1024_w64": dict(kind="2d", nx=1024, ny=1024, lx=64, ly=64,
                                rank=30, seed=3),
    "shaped_2048x2048_disc40holes_w32": dict(kind="shaped", nx=2048, ny=2048,
                                             lx=32, ly=32, rank=20, seed=4),
}
