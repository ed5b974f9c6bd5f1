"""Polygon/gradient/sinusoid clean images and noise models (see package doc)."""
from __future__ import annotations

import numpy as np


def _child_rngs(seed: int, n: int):
    ss = np.random.SeedSequence(int(seed))
    return [np.random.default_rng(s) for s in ss.spawn(n)]


def _polygon_mask(vx, vy, x0, y0, w, h):
    """Even-odd fill of polygon (vx, vy) over the box [x0, x0+w) x [y0, y0+h).

    Pixel centres are at integer coordinates.  Row-wise crossing parity: for
    every row the x-intersections with each edge are sorted and spans between
    consecutive pairs are filled through a difference array.
    """
    ys = y0 + np.arange(h, dtype=np.float64)[:, None]          # [h,1]
    ax, ay = vx[None, :], vy[None, :]
    bx, by = np.roll(vx, -1)[None, :], np.roll(vy, -1)[None, :]
    crosses = (ay <= ys) != (by <= ys)                            # [h,E]
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (ys - ay) / (by - ay)
    xi = np.where(crosses, ax + t * (bx - ax), np.inf)           # [h,E]
    xi.sort(axis=1)
    ncross = crosses.sum(axis=1)
    diff = np.zeros((h, w + 1), dtype=np.int32)
    for p in range(0, xi.shape[1] - 1, 2):
        valid = ncross > p + 1
        if not valid.any():
            break
        rows = np.nonzero(valid)[0]
        xa = np.clip(np.ceil(xi[rows, p] - x0), 0, w).astype(np.int64)
        xb = np.clip(np.floor(xi[rows, p + 1] - x0) + 1, 0, w).astype(np.int64)
        ok = xb > xa
        np.add.at(diff, (rows[ok], xa[ok]), 1)
        np.add.at(diff, (rows[ok], xb[ok]), -1)
    return np.cumsum(diff[:, :w], axis=1) > 0


def clean_image(h: int, w: int, seed: int) -> np.ndarray:
    """Clean RGB image, planar float32 [3][h][w] in [0, 1]."""
    rng = _child_rngs(seed, 1)[0]
    yy = np.arange(h, dtype=np.float32)[:, None] / max(h - 1, 1)
    xx = np.arange(w, dtype=np.float32)[None, :] / max(w - 1, 1)
    img = np.empty((3, h, w), dtype=np.float32)
    for c in range(3):
        a, b, d = rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(0.2, 0.8)
        img[c] = d + a * (xx - 0.5) + b * (yy - 0.5)
    mp = h * w / 1e6
    npoly = max(3, int(round(rng.uniform(20, 60) * max(mp, 0.05))))
    scale = max(h, w)
    for _ in range(npoly):
        nv = int(rng.integers(3, 9))
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        rad = scale * rng.uniform(0.03, 0.25)
        ang = np.sort(rng.uniform(0, 2 * np.pi, nv))
        rr = rad * rng.uniform(0.4, 1.0, nv)
        vx = cx + rr * np.cos(ang)
        vy = cy + rr * np.sin(ang)
        # even-odd fill of a possibly self-intersecting polygon: shuffle a few
        if rng.uniform() < 0.2:
            perm = rng.permutation(nv)
            vx, vy = vx[perm], vy[perm]
        x0 = int(max(0, np.floor(vx.min())))
        x1 = int(min(w, np.ceil(vx.max()) + 1))
        y0 = int(max(0, np.floor(vy.min())))
        y1 = int(min(h, np.ceil(vy.max()) + 1))
        if x1 <= x0 or y1 <= y0:
            continue
        m = _polygon_mask(vx, vy, x0, y0, x1 - x0, y1 - y0)
        if not m.any():
            continue
        py = np.arange(y0, y1, dtype=np.float32)[:, None]
        px = np.arange(x0, x1, dtype=np.float32)[None, :]
        if rng.uniform() < 0.3:
            period = rng.uniform(4.0, 32.0)
            th = rng.uniform(0, np.pi)
            phase = rng.uniform(0, 2 * np.pi)
            s = np.sin(2 * np.pi * (px * np.cos(th) + py * np.sin(th)) / period + phase)
            base = rng.uniform(0.2, 0.8, 3)
            amp = rng.uniform(0.05, 0.35, 3)
            for c in range(3):
                region = img[c, y0:y1, x0:x1]
                region[m] = (base[c] + amp[c] * s)[m]
        else:
            col = rng.uniform(0.0, 1.0, 3)
            gx, gy = rng.uniform(-0.4, 0.4, 3) / scale, rng.uniform(-0.4, 0.4, 3) / scale
            for c in range(3):
                region = img[c, y0:y1, x0:x1]
                val = col[c] + gx[c] * (px - cx) + gy[c] * (py - cy)
                region[m] = np.broadcast_to(val, m.shape)[m]
    np.clip(img, 0.0, 1.0, out=img)
    return img


def awgn(clean: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Additive white Gaussian noise, float, no clamp (Section 4: AWGN model)."""
    rng = _child_rngs(seed, 2)[1]
    n = rng.standard_normal(clean.shape, dtype=np.float32)
    return (clean + np.float32(sigma) * n).astype(np.float32)


def gain_field(h: int, w: int, seed: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Smooth log-uniform gain field in [lo, hi], shape [h][w] float32.

    Bilinear upsampling of a coarse 6x8 random grid in log space.
    """
    rng = _child_rngs(seed, 3)[2]
    gh, gw = 6, 8
    g = rng.uniform(np.log(lo), np.log(hi), (gh, gw))
    yi = np.linspace(0, gh - 1, h)
    xi = np.linspace(0, gw - 1, w)
    y0 = np.clip(np.floor(yi).astype(int), 0, gh - 2)
    x0 = np.clip(np.floor(xi).astype(int), 0, gw - 2)
    fy = (yi - y0)[:, None]
    fx = (xi - x0)[None, :]
    a = g[y0][:, x0]
    b = g[y0][:, x0 + 1]
    c = g[y0 + 1][:, x0]
    d = g[y0 + 1][:, x0 + 1]
    v = (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy
    return np.exp(v).astype(np.float32)


def signal_dependent_noise(clean: np.ndarray, a: float, b: float, seed: int,
                           gain: np.ndarray | None = None) -> np.ndarray:
    """z = u + G(x) * sqrt(a*u + b) * n  (camera-like heteroscedastic noise)."""
    rng = _child_rngs(seed, 2)[1]
    n = rng.standard_normal(clean.shape, dtype=np.float32)
    sd = np.sqrt(np.maximum(a * clean + b, 0.0)).astype(np.float32)
    if gain is not None:
        sd = sd * gain[None]
    return (clean + sd * n).astype(np.float32)


def quantize8(img: np.ndarray) -> np.ndarray:
    """8-bit storage of an image in [0, 1]: clamp, round to the nearest
    multiple of 1/255 (ties to even), float32."""
    return (np.rint(np.clip(img, 0.0, 1.0) * 255.0) / 255.0).astype(np.float32)


def noisy_pair(h: int, w: int, seed: int, sigma: float = 25.0 / 255.0,
               model: str = "awgn"):
    """(noisy, clean) float32 [3][h][w] pair from one seed.  Models: "awgn"
    (float, no clamp), "awgn8" (8-bit clean image, AWGN, then 8-bit
    quantisation with clamping, like noisy 8-bit photographs), "camera"
    (signal-dependent noise with a smooth gain field)."""
    u = clean_image(h, w, seed)
    if model == "awgn":
        z = awgn(u, sigma, seed)
    elif model == "awgn8":
        u = quantize8(u)
        z = quantize8(awgn(u, sigma, seed))
    elif model == "camera":
        z = signal_dependent_noise(u, 0.01, (10.0 / 255.0) ** 2, seed,
                                   gain_field(h, w, seed))
    else:
        raise ValueError(model)
    return z, u


def batch_pairs(n: int, h: int, w: int, seed0: int, sigma: float = 25.0 / 255.0,
                model: str = "awgn"):
    """Stacked (noisy, clean) float32 [n][3][h][w] from seeds seed0..seed0+n-1."""
    zs, us = zip(*(noisy_pair(h, w, seed0 + i, sigma, model) for i in range(n)))
    return np.stack(zs), np.stack(us)
