"""Seeded synthetic inputs shaped like the paper's segmentation workloads.

This module holds input generation only (numpy, no part of the method's
arithmetic); both the CUDA path's tests/benchmark and the oracle-side tests
draw their images from it.  The paper's own images (grid, cartoon, calendar
snippet, fish; Sec. 4) are not available, so seeded stand-ins with the same
structure are generated: piecewise-constant regions with curved boundaries,
oriented gratings as texture, additive white Gaussian noise.

Seeds: 1805000 + 1000 * workload_index + image_index.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "seed_for", "ellipse_image", "bezier_texture_image", "rgb_texture_image",
    "grid_image", "scale_weights", "make_workload_image", "batch_shapes",
]


def seed_for(workload: int, image: int = 0) -> int:
    return 1805000 + 1000 * workload + image


def scale_weights(lam: float, J: int) -> np.ndarray:
    """Per-scale weights Lambda = lam * (0, 0.1, 0.2, 0.4, ..., 0.1 * 2^(J-1)).

    The paper writes its shearlet weights as a scalar times the pattern
    (0, 0.1, 0.2, 0.4, 0.8) (Sec. 4, cartoon, stripes and fish examples): the
    low-pass is not penalised and the weight doubles per scale."""
    out = np.zeros(J + 1)
    for j in range(J):
        out[j + 1] = lam * 0.1 * 2.0 ** j
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    H: int
    W: int
    C: int
    K: int
    J: int
    iters: int
    lam: float
    gamma: float
    index: int

    @property
    def eta(self) -> int:
        return 2 ** (self.J + 2) - 3

    def codebook(self) -> np.ndarray:
        if self.C == 3:  # the 8 colours {0.2, 0.8}^3
            return np.array([[a, b, c] for a in (0.2, 0.8) for b in (0.2, 0.8) for c in (0.2, 0.8)])[: self.K]
        if self.K == 3 and self.index == 1:
            return np.array([[0.2], [0.5], [0.8]])
        return np.array([[0.2 + 0.6 * k / (self.K - 1)] for k in range(self.K)])

    def Lambda(self) -> np.ndarray:
        return scale_weights(self.lam, self.J)


WORKLOADS = {
    "ellipses64": Workload("ellipses64", 64, 64, 1, 3, 2, 200, 0.1, 1.0, 1),
    "bezier512": Workload("bezier512", 512, 512, 1, 4, 4, 500, 0.1, 1.0, 2),
    "unrolled256": Workload("unrolled256", 256, 256, 1, 4, 3, 50, 0.1, 1.0, 4),
    "rgb2048": Workload("rgb2048", 2048, 2048, 3, 8, 5, 1000, 0.1, 1.0, 5),
}


def ellipse_image(H: int, W: int, codebook, rng: np.random.Generator, sigma: float = 0.05, n_ellipses: int = 6):
    """Background label 0 plus seeded ellipses painted in order (centres
    uniform in the image, semi-axes U[6,16] scaled by size/64, angle U[0,pi),
    label uniform), value = codebook value + N(0, sigma^2).  Returns
    (image [C,H,W], labels [H,W])."""
    cb = np.asarray(codebook, dtype=np.float64).reshape(len(codebook), -1)
    K, C = cb.shape
    scale = min(H, W) / 64.0
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    lab = np.zeros((H, W), dtype=np.int32)
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        a, b = rng.uniform(6, 16, size=2) * scale
        th = rng.uniform(0, math.pi)
        k = int(rng.integers(0, K))
        dy, dx = yy - cy, xx - cx
        p = dx * math.cos(th) + dy * math.sin(th)
        q = -dx * math.sin(th) + dy * math.cos(th)
        lab[(p / a) ** 2 + (q / b) ** 2 <= 1.0] = k
    img = cb[lab].transpose(2, 0, 1).copy() + sigma * rng.standard_normal((C, H, W))
    return img, lab


def _closed_bezier(cy: float, cx: float, radii: np.ndarray, phase: float, samples: int = 64):
    """Closed C1 cubic Bezier spline through anchors at the given radii around
    (cy, cx); handles from Catmull-Rom tangents.  Returns polygon vertices."""
    n = len(radii)
    ang = phase + 2 * math.pi * np.arange(n) / n
    P = np.stack([cy + radii * np.sin(ang), cx + radii * np.cos(ang)], axis=1)
    pts = []
    t = np.linspace(0.0, 1.0, samples, endpoint=False)[:, None]
    for i in range(n):
        p0, p3 = P[i], P[(i + 1) % n]
        m0 = (P[(i + 1) % n] - P[(i - 1) % n]) / 6.0
        m1 = (P[(i + 2) % n] - P[i]) / 6.0
        p1, p2 = p0 + m0, p3 - m1
        seg = ((1 - t) ** 3) * p0 + 3 * ((1 - t) ** 2) * t * p1 + 3 * (1 - t) * t * t * p2 + (t ** 3) * p3
        pts.append(seg)
    return np.concatenate(pts, axis=0)


def _fill_polygon(poly: np.ndarray, H: int, W: int) -> np.ndarray:
    """Even-odd scanline fill of a closed polygon (vertices (y, x)) at pixel centres."""
    mask = np.zeros((H, W), dtype=bool)
    y0, x0 = poly[:, 0], poly[:, 1]
    y1, x1 = np.roll(y0, -1), np.roll(x0, -1)
    cols = np.arange(W, dtype=np.float64)
    for r in range(H):
        yc = float(r)
        hit = ((y0 <= yc) & (y1 > yc)) | ((y1 <= yc) & (y0 > yc))
        if not hit.any():
            continue
        xs = x0[hit] + (yc - y0[hit]) * (x1[hit] - x0[hit]) / (y1[hit] - y0[hit])
        xs.sort()
        for a, b in zip(xs[0::2], xs[1::2]):
            mask[r] |= (cols >= a) & (cols < b)
    return mask


def _bezier_labels(H: int, W: int, K: int, rng: np.random.Generator, n_regions: int = 5):
    scale = min(H, W) / 512.0
    lab = np.zeros((H, W), dtype=np.int32)
    for i in range(n_regions):
        cy, cx = rng.uniform(0.15 * H, 0.85 * H), rng.uniform(0.15 * W, 0.85 * W)
        radii = rng.uniform(60, 180, size=8) * scale
        poly = _closed_bezier(cy, cx, radii, rng.uniform(0, 2 * math.pi))
        lab[_fill_polygon(poly, H, W)] = 1 + (i % (K - 1)) if i < K - 1 else int(rng.integers(0, K))
    return lab


def _grating(H: int, W: int, K: int, rng: np.random.Generator, amplitude: float = 0.15):
    """Oriented sinusoid per label: amplitude * sin(2 pi <x, (cos t_k, sin t_k)> / P_k),
    t_k = k pi / K, P_k ~ U[8, 16]."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    periods = rng.uniform(8, 16, size=K)
    g = np.empty((K, H, W))
    for k in range(K):
        th = k * math.pi / K
        g[k] = amplitude * np.sin(2 * math.pi * (xx * math.cos(th) + yy * math.sin(th)) / periods[k])
    return g


def bezier_texture_image(H: int, W: int, codebook, rng: np.random.Generator, sigma: float = 0.05):
    """Regions bounded by seeded closed Bezier contours, each filled with its
    codebook value plus an oriented grating, plus N(0, sigma^2) noise.
    Returns (image [C,H,W], labels [H,W])."""
    cb = np.asarray(codebook, dtype=np.float64).reshape(len(codebook), -1)
    K, C = cb.shape
    lab = _bezier_labels(H, W, K, rng)
    gr = _grating(H, W, K, rng)
    tex = np.take_along_axis(gr, lab[None], axis=0)[0]
    img = cb[lab].transpose(2, 0, 1) + tex[None] + sigma * rng.standard_normal((C, H, W))
    return np.ascontiguousarray(img), lab


def rgb_texture_image(H: int, W: int, codebook, rng: np.random.Generator, sigma: float = 0.05):
    """RGB form: the same curved textured regions, per-channel noise."""
    return bezier_texture_image(H, W, codebook, rng, sigma)


def grid_image(H: int, W: int, rng: np.random.Generator, period: int = 16, bar: int = 6, sigma: float = 0.2):
    """0/1 grid (bars of width `bar` every `period` pixels) plus N(0, sigma^2):
    a stand-in for the noisy grid of the first example of Sec. 4."""
    yy, xx = np.mgrid[0:H, 0:W]
    lab = (((yy % period) < bar) | ((xx % period) < bar)).astype(np.int32)
    img = lab.astype(np.float64) + sigma * rng.standard_normal((H, W))
    return img[None], lab


def make_workload_image(name: str, image: int = 0):
    """(image [C,H,W] float64, labels [H,W], workload) for a named workload."""
    wl = WORKLOADS[name]
    rng = np.random.default_rng(seed_for(wl.index, image))
    cb = wl.codebook()
    if name in ("ellipses64", "unrolled256"):
        img, lab = ellipse_image(wl.H, wl.W, cb, rng)
    else:
        img, lab = bezier_texture_image(wl.H, wl.W, cb, rng)
    return img, lab, wl


_BATCH_SIDES = (128, 160, 192, 256, 320, 384, 512, 640, 768, 1024)


def batch_shapes(n: int = 64, seed: int = seed_for(3)):
    """Shapes of the uneven batch: image 0 is 384 x 640, the rest draw H and W
    from sizes 2^a 3^b 5^c in [128, 1024]; K ~ U{2..6}; J = floor(log2(min)/2)."""
    rng = np.random.default_rng(seed)
    out = [(384, 640, int(rng.integers(2, 7)))]
    for _ in range(n - 1):
        H, W = (int(x) for x in rng.choice(_BATCH_SIDES, size=2))
        out.append((H, W, int(rng.integers(2, 7))))
    return [(H, W, K, int(math.floor(0.5 * math.log2(min(H, W))))) for H, W, K in out]
