"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds none of the solver's arithmetic: it only draws images and
cost volumes with the shapes and value ranges of the workloads the paper
evaluates on (Sec. 5.1 ROF, Sec. 5.2 truncated quadratic, Sec. 5.4 stereo),
since the paper's own images are not available.

Randomness comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated on a counter so that
every draw is reproducible on any machine and numpy version.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1512013830

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class Rng:
    """Counter-based SplitMix64 stream: output i is mix(seed + (i+1)*golden)."""

    def __init__(self, seed: int, stream: int = 0):
        self.key = np.uint64((int(seed) * 0x2545F4914F6CDD1D + int(stream) * 0x632BE59BD9B4E019)
                             & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def _bits(self, n: int) -> np.ndarray:
        c = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.key + c * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self._bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        """Box-Muller on two uniform streams."""
        u1 = 1.0 - self.uniform(n)          # in (0, 1]
        u2 = self.uniform(n)
        return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] inclusive."""
        return lo + np.minimum((self.uniform(n) * (hi - lo + 1)).astype(np.int64), hi - lo)

    def choice(self, n: int, options) -> np.ndarray:
        options = np.asarray(options)
        return options[self.integers(n, 0, len(options) - 1)]


def gaussian_blobs(H: int, W: int, seed: int, blobs: int = 8, noise: float = 0.1) -> np.ndarray:
    """Sum of isotropic Gaussian blobs, min-max normalised to [0,1], plus noise.

    Centres uniform over the image, widths U[3,12] px, amplitudes U[0.3,1];
    additive N(0, noise^2).  Stand-in for the ROF test image of Sec. 5.1.
    """
    r = Rng(seed, 1)
    cy, cx = r.uniform(blobs, 0, H), r.uniform(blobs, 0, W)
    sg, amp = r.uniform(blobs, 3, 12), r.uniform(blobs, 0.3, 1.0)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.zeros((H, W))
    for b in range(blobs):
        img += amp[b] * np.exp(-((yy - cy[b]) ** 2 + (xx - cx[b]) ** 2) / (2 * sg[b] ** 2))
    lo, hi = img.min(), img.max()
    img = (img - lo) / (hi - lo) if hi > lo else np.zeros_like(img)
    return img + r.normal(H * W, noise).reshape(H, W)


def voronoi_ramps(H: int, W: int, seed: int, cells: int = 24, noise: float = 0.05,
                  outliers: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """Piecewise-smooth image plus Gaussian and salt-and-pepper style noise.

    Voronoi cells on seeded sites, each cell a linear ramp a + b x + c y with
    a ~ U[0.1,0.9] and slopes U[-1,1]/512 per pixel, clipped to [0,1]; then
    N(0, noise^2) and a fraction ``outliers`` of pixels replaced by U[0,1]
    (stand-in for the degraded image of Sec. 5.2).  Returns (noisy, clean).
    """
    r = Rng(seed, 2)
    sy, sx = r.uniform(cells, 0, H), r.uniform(cells, 0, W)
    a = r.uniform(cells, 0.1, 0.9)
    b = r.uniform(cells, -1, 1) / 512.0
    c = r.uniform(cells, -1, 1) / 512.0
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    lab = np.zeros((H, W), dtype=np.int64)
    best = np.full((H, W), np.inf)
    for j in range(cells):
        d = (yy - sy[j]) ** 2 + (xx - sx[j]) ** 2
        m = d < best
        best[m] = d[m]
        lab[m] = j
    clean = np.clip(a[lab] + b[lab] * xx + c[lab] * yy, 0.0, 1.0)
    noisy = clean + r.normal(H * W, noise).reshape(H, W)
    sel = r.uniform(H * W) < outliers
    noisy = noisy.reshape(-1)
    noisy[sel] = r.uniform(int(sel.sum()))
    return noisy.reshape(H, W), clean


def voronoi_ramps_3d(D: int, H: int, W: int, seed: int, cells: int = 24, noise: float = 0.05,
                     outliers: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """The volume form of voronoi_ramps: Voronoi cells on seeded sites in a
    D x H x W box, each a linear ramp a + b x + c y + e z (a ~ U[0.1,0.9],
    slopes U[-1,1]/512 per voxel) clipped to [0,1]; then N(0, noise^2) and a
    fraction ``outliers`` of voxels replaced by U[0,1].  Stand-in for a
    volumetric denoising input (the d = 3 grid of Sec. 4).  Returns (noisy,
    clean)."""
    r = Rng(seed, 7)
    sz, sy, sx = r.uniform(cells, 0, D), r.uniform(cells, 0, H), r.uniform(cells, 0, W)
    a = r.uniform(cells, 0.1, 0.9)
    b, c, e = (r.uniform(cells, -1, 1) / 512.0 for _ in range(3))
    zz, yy, xx = np.mgrid[0:D, 0:H, 0:W].astype(np.float64)
    lab = np.zeros((D, H, W), dtype=np.int64)
    best = np.full((D, H, W), np.inf)
    for j in range(cells):
        d = (zz - sz[j]) ** 2 + (yy - sy[j]) ** 2 + (xx - sx[j]) ** 2
        m = d < best
        best[m] = d[m]
        lab[m] = j
    clean = np.clip(a[lab] + b[lab] * xx + c[lab] * yy + e[lab] * zz, 0.0, 1.0)
    noisy = (clean + r.normal(D * H * W, noise).reshape(D, H, W)).reshape(-1)
    sel = r.uniform(D * H * W) < outliers
    noisy[sel] = r.uniform(int(sel.sum()))
    return noisy.reshape(D, H, W), clean


def gradient_noise(H: int, W: int, seed: int, octaves: int = 4, base: float = 64.0) -> np.ndarray:
    """Multi-octave lattice noise with smoothstep interpolation, scaled to [0,1]."""
    r = Rng(seed, 3)
    out = np.zeros((H, W))
    amp = 1.0
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for o in range(octaves):
        s = base / (2 ** o)
        gh, gw = int(np.ceil(H / s)) + 2, int(np.ceil(W / s)) + 2
        lat = r.uniform(gh * gw).reshape(gh, gw)
        fy, fx = yy / s, xx / s
        iy, ix = np.floor(fy).astype(np.int64), np.floor(fx).astype(np.int64)
        ty, tx = fy - iy, fx - ix
        ty, tx = ty * ty * (3 - 2 * ty), tx * tx * (3 - 2 * tx)
        v00, v01 = lat[iy, ix], lat[iy, ix + 1]
        v10, v11 = lat[iy + 1, ix], lat[iy + 1, ix + 1]
        out += amp * ((1 - ty) * ((1 - tx) * v00 + tx * v01) + ty * ((1 - tx) * v10 + tx * v11))
        amp *= 0.5
    lo, hi = out.min(), out.max()
    return (out - lo) / (hi - lo) if hi > lo else np.zeros_like(out)


def stereo_cost(H: int, W: int, seed: int, ndisp: int = 65, tau: float = 0.2,
                cells: int = 16) -> tuple[np.ndarray, np.ndarray]:
    """Matching cost of a synthetic rectified pair (stand-in for Sec. 5.4).

    Disparity: Voronoi cells of planes a + b x + c y (a ~ U[4,60],
    |b|,|c| <= 0.02) clipped to [0, ndisp-1].  Albedo: gradient noise.  The
    reference image samples the albedo at x + D(x,y) (linear interpolation,
    clamped); the target image is the albedo itself.  Cost at integer
    disparity d: min(|I0(x,y) - I1(x+d,y)|, tau), x+d clamped.
    Returns (cost [H,W,ndisp], disparity [H,W]).
    """
    r = Rng(seed, 4)
    dmax = float(ndisp - 1)
    sy, sx = r.uniform(cells, 0, H), r.uniform(cells, 0, W)
    a = r.uniform(cells, 4, 60)
    b = r.uniform(cells, -0.02, 0.02)
    c = r.uniform(cells, -0.02, 0.02)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    lab = np.zeros((H, W), dtype=np.int64)
    best = np.full((H, W), np.inf)
    for j in range(cells):
        d = (yy - sy[j]) ** 2 + (xx - sx[j]) ** 2
        m = d < best
        best[m] = d[m]
        lab[m] = j
    disp = np.clip(a[lab] + b[lab] * xx + c[lab] * yy, 0.0, dmax)
    alb = gradient_noise(H, W, seed)

    def sample(img, xs):
        xs = np.clip(xs, 0.0, W - 1.0)
        x0 = np.minimum(np.floor(xs).astype(np.int64), W - 2)
        t = xs - x0
        rows = np.arange(H)[:, None]
        return (1 - t) * img[rows, x0] + t * img[rows, x0 + 1]

    i0 = sample(alb, xx + disp)
    cost = np.empty((H, W, ndisp))
    for d in range(ndisp):
        i1 = alb[:, np.minimum(np.arange(W) + d, W - 1)]
        cost[:, :, d] = np.minimum(np.abs(i0 - i1), tau)
    return cost, disp


def wrapped_phase(H: int, W: int, seed: int, lo: float = 1.0, hi: float = 11.0,
                  noise: float = 0.1, period: float = 2.0 * np.pi) -> tuple[np.ndarray, np.ndarray]:
    """Wrapped phase (stand-in for the SAR data of Sec. 5.5): a smooth
    surface of 6 Gaussian bumps plus a seeded linear ramp, scaled to
    [lo, hi], plus N(0, noise^2), wrapped into [0, period).
    Returns (wrapped, true unwrapped)."""
    r = Rng(seed, 6)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    gy, gx = r.uniform(2, -1, 1)
    field = gx * xx / max(W, 1) + gy * yy / max(H, 1)
    for _ in range(6):
        cy, cx = r.uniform(1, 0, H)[0], r.uniform(1, 0, W)[0]
        sg = r.uniform(1, 0.1, 0.3)[0] * max(H, W)
        field = field + r.uniform(1, -1, 1)[0] * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * sg * sg))
    a, b = field.min(), field.max()
    true = lo + (hi - lo) * ((field - a) / (b - a) if b > a else np.zeros_like(field))
    wrapped = np.mod(true + r.normal(H * W, noise).reshape(H, W), period)
    return wrapped, true


def batch_instances(n: int, seed: int, smin: int = 128, smax: int = 1024,
                    Ls=(4, 8, 16, 32)) -> list[tuple[int, int]]:
    """(side, L) for n serving-style instances: side ~ U{smin..smax}, L ~ U(Ls)."""
    r = Rng(seed, 5)
    sides = r.integers(n, smin, smax)
    Lc = r.choice(n, list(Ls))
    return [(int(s), int(L)) for s, L in zip(sides, Lc)]


def as_f32(a: np.ndarray) -> np.ndarray:
    """Round to float32 so both solvers see identical inputs."""
    return np.ascontiguousarray(a, dtype=np.float32)
