"""Helpers for GPU-vs-oracle comparisons (no arithmetic of the method)."""
import numpy as np


def dilate(mask, r):
    """Binary dilation by a (2r+1)^2 square (clamped at the border)."""
    if r <= 0:
        return mask.copy()
    h, w = mask.shape
    out = np.zeros_like(mask)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            ys, xs = slice(max(dy, 0), h + min(dy, 0)), slice(max(dx, 0), w + min(dx, 0))
            yd, xd = slice(max(-dy, 0), h + min(-dy, 0)), slice(max(-dx, 0), w + min(-dx, 0))
            out[yd, xd] |= mask[ys, xs]
    return out


def affected_mask(mismatch_per_level, r_coarse, shapes):
    """Finest-level pixels whose output depends on a mismatched bucket.

    mismatch_per_level[l]: bool [h_l][w_l] for filtered levels l = 0..nb-1.
    A level-l pixel depends on its own bucket and on the level-(l+1) output
    at floor(i/2) + [-r_coarse, r_coarse]."""
    nb = len(mismatch_per_level)
    aff = mismatch_per_level[nb - 1].copy()
    for l in range(nb - 2, -1, -1):
        h, w = shapes[l]
        up = np.repeat(np.repeat(dilate(aff, max(r_coarse, 0)), 2, 0), 2, 1)[:h, :w]
        aff = mismatch_per_level[l] | up
    return aff


def max_abs(a, b, mask=None):
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))
    if d.ndim == 3:
        d = d.max(axis=0)
    if mask is not None:
        d = d[mask]
    return float(d.max()) if d.size else 0.0
