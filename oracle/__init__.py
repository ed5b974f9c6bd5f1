"""FP64 CPU oracle for trainable multiscale denoising (arXiv 1802.06130).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product package.  It is a
thin ctypes layer over ``mdn_oracle.c`` (plain C, FP64) plus the level cascade
written as plain Python loops in the paper's order:

* ``pyramid``            -- Section 4 "Multiscale filtering": 2x downsampling
* ``select``             -- Section 3 "Filter selection": colour structure
                            tensor, eigen-features, bucket s(i)
* ``filter_level``       -- Eq. 1 and the multiscale equation of Section 4
* ``denoise_multiscale`` -- Section 4: base case u^L = z^L, levels L-1 .. 0
* ``gram_accumulate`` / ``solve_bank`` -- Eqs. 5-6: per-bucket least squares
* ``train_cascade``      -- Section 4: train level L-1 first, apply it, feed
                            its output to the next finer level
* ``estimate_noise``     -- noise level for choosing the bank set (the paper
                            assumes it known, Section 6): Donoho-Johnstone's
                            median(|HH|) / 0.6745
* ``dihedral`` / ``gram_accumulate_dihedral`` -- Section 5's training-set
                            augmentation by flips and 90-degree rotations,
                            by materialising the 8 transformed pairs

Precision: FP64 throughout, except ``mirror32=True`` which evaluates the
pyramid and the structure tensor/features in the documented FP32 order (for
bit-exact bucket comparison), and ``storage`` which rounds every stored
plane (pyramid levels, level outputs) to FP32 or FP16 (RN-even).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")

STORAGE = {"f64": 0, "f32": 1, "f16": 2}
MAX_THR = 16


def build(force: bool = False) -> str:
    """Compile mdn_oracle.c into oracle/_build/liborc.so (gcc, OpenMP)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _BParams(C.Structure):
    _fields_ = [("n_angle", C.c_int32), ("n_strength", C.c_int32), ("n_coherence", C.c_int32),
                ("strength_thr", C.c_float * MAX_THR), ("coherence_thr", C.c_float * MAX_THR),
                ("coh_eps", C.c_float)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp, u8p, i64p = C.POINTER(C.c_double), C.POINTER(C.c_uint8), C.POINTER(C.c_int64)
        i32p = C.POINTER(C.c_int32)
        L.orc_round_f16.restype = C.c_double
        L.orc_round_f16.argtypes = [C.c_double]
        L.orc_round_storage.argtypes = [dp, C.c_long, C.c_int]
        L.orc_pyramid_down.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_int]
        L.orc_structure_tensor.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp]
        L.orc_features.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_float, dp]
        L.orc_buckets.argtypes = [dp, C.c_int, C.c_int, C.POINTER(_BParams), C.c_double, i32p, u8p]
        L.orc_buckets_fp32.argtypes = [dp, C.c_int, C.c_int, C.POINTER(_BParams), i32p]
        L.orc_to_work.argtypes = [dp, C.c_long, C.c_int, dp]
        L.orc_from_work.argtypes = [dp, C.c_long, C.c_int, dp]
        L.orc_regressor_len.restype = C.c_int
        L.orc_regressor_len.argtypes = [C.c_int, C.c_int, C.c_int]
        L.orc_filter_level.argtypes = [dp, C.c_int, C.c_int, dp, C.c_int, C.c_int, i32p, dp, C.c_int,
                                       C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp]
        L.orc_gram_accumulate.argtypes = [dp, C.c_int, C.c_int, dp, C.c_int, C.c_int, dp, i32p, C.c_int,
                                          C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp, i64p]
        L.orc_cholesky_solve.restype = C.c_int
        L.orc_cholesky_solve.argtypes = [dp, C.c_int, dp, C.c_int]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_max_threads.restype = C.c_int
        L.orc_solve_bank.restype = C.c_int
        L.orc_solve_bank.argtypes = [dp, i64p, C.c_int, C.c_int, C.c_int, C.c_double, dp]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


# ---------------------------------------------------------------- parameters

@dataclass
class Geometry:
    """Filter footprint: fine radius, coarse radius (-1 = single level),
    cross-channel regressors, colour space (0 = YCbCr BT.601, 1 = RGB), and
    the coarse sampling: align = 0 takes the coarse patch at floor(i/2) (the
    reading of the paper's i/2), align = 1 samples it bilinearly at i/2 (the
    half-pixel-aligned variant of the multiscale equation of Section 4)."""
    r_fine: int = 3
    r_coarse: int = 3
    cross: int = 0
    color: int = 0
    align: int = 0

    def D(self) -> int:
        return lib().orc_regressor_len(self.r_fine, self.r_coarse, self.cross)


@dataclass
class BucketParams:
    """Bucket grid and thresholds for one level (Section 3; thresholds are
    this implementation's reading, the paper gives none)."""
    n_angle: int = 24
    strength_thr: tuple = (0.135, 0.16)
    coherence_thr: tuple = (0.10, 0.15)
    coh_eps: float = 1e-8

    @property
    def K(self) -> int:
        return self.n_angle * (len(self.strength_thr) + 1) * (len(self.coherence_thr) + 1)

    def c(self) -> _BParams:
        b = _BParams()
        b.n_angle = self.n_angle
        b.n_strength = len(self.strength_thr) + 1
        b.n_coherence = len(self.coherence_thr) + 1
        for i, t in enumerate(self.strength_thr):
            b.strength_thr[i] = t
        for i, t in enumerate(self.coherence_thr):
            b.coherence_thr[i] = t
        b.coh_eps = self.coh_eps
        return b


def default_bparams(level: int) -> BucketParams:
    """Level-l defaults: strength thresholds halve per coarser level.

    Level-0 values were fixed once from the feature histogram of the
    256x256, sigma = 25/255 training set (seeds 1000-1007) so that none of
    the 216 buckets is empty, then frozen."""
    s = 0.5 ** level
    return BucketParams(strength_thr=(0.135 * s, 0.16 * s), coherence_thr=(0.10, 0.15))


# The paper's own grid, 16 x 16 x 16 = 4096 buckets (Section 5).  Reading
# (the paper gives no thresholds): equal-population strength and coherence
# bins, the 15 quantiles k/16 of each feature over the 256x256, sigma =
# 25/255 training set (seeds 1000-1007) at levels 0 and 1, rounded to 4
# digits and frozen; coarser levels halve the level-1 strength thresholds
# per level and keep its coherence thresholds.
PAPER_GRID_STRENGTH = (
    (0.1101, 0.1145, 0.1176, 0.1202, 0.1225, 0.1247, 0.1268, 0.129, 0.1311, 0.1334, 0.1359, 0.1387,
     0.1422, 0.1469, 0.1556),
    (0.0297, 0.031, 0.032, 0.0329, 0.0336, 0.0343, 0.035, 0.0357, 0.0364, 0.0372, 0.038, 0.0391,
     0.0403, 0.0423, 0.0497))
PAPER_GRID_COHERENCE = (
    (0.0232, 0.0335, 0.042, 0.0496, 0.0569, 0.0641, 0.0713, 0.0789, 0.0869, 0.0955, 0.105, 0.1163,
     0.1299, 0.1484, 0.1801),
    (0.0278, 0.0402, 0.0504, 0.0598, 0.0687, 0.0774, 0.0861, 0.095, 0.1047, 0.1153, 0.1273, 0.1412,
     0.1588, 0.1844, 0.242))


def paper_grid_bparams(level: int) -> BucketParams:
    """16 angle x 16 strength x 16 coherence bins for level l."""
    if level <= 1:
        return BucketParams(n_angle=16, strength_thr=PAPER_GRID_STRENGTH[level],
                            coherence_thr=PAPER_GRID_COHERENCE[level])
    s = 0.5 ** (level - 1)
    return BucketParams(n_angle=16, strength_thr=tuple(t * s for t in PAPER_GRID_STRENGTH[1]),
                        coherence_thr=PAPER_GRID_COHERENCE[1])


def bucket_dtype(K: int):
    """Element type of a bucket map: u8 up to 256 buckets, else u16."""
    return np.uint8 if K <= 256 else np.uint16


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (OpenMP)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------- primitives

def round_storage(x, storage: str):
    x = _d(x).copy()
    lib().orc_round_storage(_p(x), x.size, STORAGE[storage])
    return x


def pyramid_down(img, mirror32: bool = False):
    img = _d(img)
    Cn, H, W = img.shape
    out = np.empty((Cn, (H + 1) // 2, (W + 1) // 2))
    lib().orc_pyramid_down(_p(img), Cn, H, W, _p(out), int(mirror32))
    return out


def pyramid(img, levels: int, storage: str = "f64", mirror32: bool = False):
    """[z^0, ..., z^{L-1}]; z^0 is the input rounded to storage."""
    z = [round_storage(img, storage)]
    for _ in range(1, levels):
        z.append(round_storage(pyramid_down(z[-1], mirror32), storage))
    return z


def structure_tensor(z, mirror32: bool = False):
    z = _d(z)
    _, H, W = z.shape
    T = np.empty((3, H, W))
    lib().orc_structure_tensor(_p(z), H, W, int(mirror32), _p(T))
    return T


def features(T, coh_eps: float = 1e-8, mirror32: bool = False):
    T = _d(T)
    _, H, W = T.shape
    f = np.empty((3, H, W))
    lib().orc_features(_p(T), H, W, int(mirror32), coh_eps, _p(f))
    return f


def buckets(feat, bp: BucketParams, band_eps: float = 1e-5):
    feat = _d(feat)
    _, H, W = feat.shape
    b = np.empty((H, W), dtype=np.int32)
    band = np.empty((H, W), dtype=np.uint8)
    cb = bp.c()
    lib().orc_buckets(_p(feat), H, W, C.byref(cb), band_eps, _p(b, C.c_int32), _p(band, C.c_uint8))
    return b.astype(bucket_dtype(bp.K)), band.astype(bool)


def buckets_fp32(T, bp: BucketParams):
    """Bucket map decided in FP32 on the tensor by the squared-domain
    comparisons of orc_buckets_fp32 (equivalent to thresholding the features
    in exact arithmetic)."""
    T = _d(T)
    _, H, W = T.shape
    b = np.empty((H, W), dtype=np.int32)
    cb = bp.c()
    lib().orc_buckets_fp32(_p(T), H, W, C.byref(cb), _p(b, C.c_int32))
    return b.astype(bucket_dtype(bp.K))


def select(z, bp: BucketParams, mirror32: bool = False, band_eps: float = 1e-5):
    """s(i) for one level: (bucket map [H][W], u8 up to 256 buckets else u16,
    band mask, features).  mirror32: the tensor in the documented FP32 order
    and the FP32 bucket decisions of buckets_fp32 (the band mask and the
    returned features stay those of the FP32-order tensor's features)."""
    T = structure_tensor(z, mirror32)
    f = features(T, bp.coh_eps, mirror32)
    b, band = buckets(f, bp, band_eps)
    if mirror32:
        b = buckets_fp32(T, bp)
    return b, band, f


def to_work(rgb, color: int = 0):
    rgb = _d(rgb)
    out = np.empty_like(rgb)
    lib().orc_to_work(_p(rgb), rgb.shape[1] * rgb.shape[2], color, _p(out))
    return out


def from_work(w, color: int = 0):
    w = _d(w)
    out = np.empty_like(w)
    lib().orc_from_work(_p(w), w.shape[1] * w.shape[2], color, _p(out))
    return out


def filter_level(z, uc, bucket, bank, geom: Geometry):
    """Level output (RGB, FP64) of the multiscale equation (Eq. 1 if uc is None)."""
    z = _d(z)
    _, H, W = z.shape
    bank = _d(bank)
    K = bank.shape[0]
    assert bank.shape == (K, 3, geom.D()), (bank.shape, geom.D())
    bucket = np.ascontiguousarray(bucket, dtype=np.int32)
    out = np.empty_like(z)
    if geom.r_coarse >= 0:
        uc = _d(uc)
        Hc, Wc = uc.shape[1:]
        ucp = _p(uc)
    else:
        Hc = Wc = 0
        ucp = None
    lib().orc_filter_level(_p(z), H, W, ucp, Hc, Wc, _p(bucket, C.c_int32), _p(bank), K,
                           geom.r_fine, geom.r_coarse, geom.cross, geom.color, geom.align, _p(out))
    return out


@dataclass
class DenoiseResult:
    out: np.ndarray
    buckets: list = field(default_factory=list)   # per filtered level
    bands: list = field(default_factory=list)
    pyramid: list = field(default_factory=list)
    levels_out: list = field(default_factory=list)  # u-hat^l, l = 0..L-1


def denoise_multiscale(noisy, banks, geom: Geometry, bparams=None, storage: str = "f64",
                       mirror32: bool = False, bank_storage: str | None = None):
    """Section 4 inference: pyramid, base u^{L-1} = z^{L-1}, then levels
    L-2 .. 0 each filtered with its bank.  len(banks) = max(L-1, 1); L = 1 is
    single-scale filtering (Eq. 1) and needs geom.r_coarse = -1."""
    nb = len(banks)
    L = 1 if geom.r_coarse < 0 else nb + 1
    if bparams is None:
        bparams = [default_bparams(l) for l in range(nb)]
    if bank_storage is not None:
        banks = [round_storage(b, bank_storage) for b in banks]
    # the selector always sees the pyramid evaluated in the same precision as
    # its own features (mirror32) -- a mirror32 pyramid differs from the FP64
    # one only in FP32 rounding
    zs = pyramid(noisy, L, storage, mirror32)
    res = DenoiseResult(out=None, pyramid=zs)
    u = [None] * L
    u[L - 1] = zs[L - 1]
    first = L - 2 if L > 1 else 0
    bks, bds = [None] * nb, [None] * nb
    for l in range(first, -1, -1):
        b, band, _ = select(zs[l], bparams[l], mirror32)
        uc = u[l + 1] if geom.r_coarse >= 0 else None
        u[l] = round_storage(filter_level(zs[l], uc, b, banks[l], geom), storage)
        bks[l], bds[l] = b, band
    res.out = u[0]
    res.buckets, res.bands, res.levels_out = bks, bds, u
    return res


# ---------------------------------------------------------------- training

def gram_accumulate(z, uc, target, bucket, K: int, geom: Geometry, gram=None, counts=None):
    """Adds one image's per-bucket Gram matrices of [x; y] (Eqs. 5-6)."""
    z, target = _d(z), _d(target)
    _, H, W = z.shape
    D = geom.D()
    G, T = (1, 3) if geom.cross else (3, 1)
    if gram is None:
        gram = np.zeros((K, G, D + T, D + T))
        counts = np.zeros(K, dtype=np.int64)
    bucket = np.ascontiguousarray(bucket, dtype=np.int32)
    if geom.r_coarse >= 0:
        uc = _d(uc)
        Hc, Wc = uc.shape[1:]
        ucp = _p(uc)
    else:
        Hc = Wc = 0
        ucp = None
    lib().orc_gram_accumulate(_p(z), H, W, ucp, Hc, Wc, _p(target), _p(bucket, C.c_int32), K,
                              geom.r_fine, geom.r_coarse, geom.cross, geom.color, geom.align,
                              _p(gram), _p(counts, C.c_int64))
    return gram, counts


def solve_bank(gram, counts, geom: Geometry, lam: float = 1e-3):
    """Ridge least squares per bucket, FP64 Cholesky; empty -> pooled."""
    K = gram.shape[0]
    D = geom.D()
    gram = _d(gram)
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    bank = np.zeros((K, 3, D))
    fails = lib().orc_solve_bank(_p(gram), _p(counts, C.c_int64), K, D, geom.cross, lam, _p(bank))
    if fails:
        raise RuntimeError(f"{fails} Cholesky solves failed")
    return bank


def cholesky_solve(A, B):
    A = _d(A).copy()
    B = _d(B).copy()
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None].copy()
    rc = lib().orc_cholesky_solve(_p(A), A.shape[0], _p(B), B.shape[1])
    if rc:
        raise np.linalg.LinAlgError("not positive definite")
    return B[:, 0] if squeeze else B


def train_cascade(noisy_list, clean_list, geom: Geometry, levels: int, bparams=None,
                  lam: float = 1e-3, mirror32: bool = False, storage: str = "f64", level_targets=None):
    """Section 4 training: level L-2 first (its coarse input is z^{L-1}), then
    every finer level using the trained coarser levels' outputs.

    The target of level l is level l of the clean image's pyramid, unless
    level_targets (one list [u^0 .. u^{L-1}] per pair) gives it directly: a
    hook for tests that plant a different target at every level."""
    nb = max(levels - 1, 1)
    L = 1 if geom.r_coarse < 0 else levels
    if bparams is None:
        bparams = [default_bparams(l) for l in range(nb)]
    zp = [pyramid(z, L, storage, mirror32) for z in noisy_list]
    if level_targets is not None:
        up = [[_d(t) for t in ts] for ts in level_targets]
    else:
        up = [pyramid(u, L, storage, mirror32) for u in clean_list]
    cur = [p[L - 1] for p in zp]           # u-hat at level l+1, per pair
    banks = [None] * nb
    stats = [None] * nb
    first = L - 2 if L > 1 else 0
    for l in range(first, -1, -1):
        K = bparams[l].K
        gram = counts = None
        sel = []
        for i in range(len(noisy_list)):
            b, _, _ = select(zp[i][l], bparams[l], mirror32)
            sel.append(b)
            uc = cur[i] if geom.r_coarse >= 0 else None
            gram, counts = gram_accumulate(zp[i][l], uc, up[i][l], b, K, geom, gram, counts)
        banks[l] = solve_bank(gram, counts, geom, lam)
        stats[l] = counts
        cur = [round_storage(filter_level(zp[i][l], cur[i] if geom.r_coarse >= 0 else None,
                                          sel[i], banks[l], geom), storage)
               for i in range(len(noisy_list))]
    return banks, stats


# ---------------------------------------------------------------- augmentation

def dihedral(img, t: int):
    """Transform t = rot + 4 * flip (t in 0..7) of a [C][H][W] image, one of
    the 8 flips / 90-degree rotations the paper augments its training pairs
    with (Section 5): rotate by 90 degrees `rot` times (numpy's rot90 on the
    (row, column) axes), then, if flip, mirror the columns."""
    r = np.rot90(np.asarray(img), t % 4, axes=(1, 2))
    if t >= 4:
        r = r[:, :, ::-1]
    return np.ascontiguousarray(r)


def dihedral_bucket(bucket, t: int, bp: BucketParams):
    """The bucket map of transform t of an image, from the image's own map.
    The structure tensor turns with the image, so the minor eigenvector's
    orientation theta moves by pi/2 per 90-degree rotation (bin a -> a + n/2
    mod n) and to pi - theta under the mirror (a -> n - 1 - a); strength and
    coherence are eigenvalue functions and do not change.  (Exact away from
    bin boundaries and the undefined orientation of a zero tensor.)  The map
    itself is transformed like the image."""
    n = bp.n_angle
    m = (len(bp.strength_thr) + 1) * (len(bp.coherence_thr) + 1)
    b = np.asarray(bucket).astype(np.int64)
    a, rest = b // m, b % m
    a = (a + (t % 4) * (n // 2)) % n
    if t >= 4:
        a = n - 1 - a
    return dihedral((a * m + rest).astype(bucket_dtype(bp.K))[None], t)[0]


def gram_accumulate_dihedral(z, target, bucket, K: int, geom: Geometry, bp: BucketParams, gram=None, counts=None):
    """Gram sums of one single-level pair augmented by the 8 dihedral
    transforms: each transformed pair (z_t, target_t) accumulated with its
    bucket map (dihedral_bucket).  The plain definition of training on the
    flipped and rotated copies."""
    if geom.r_coarse >= 0:
        raise ValueError("gram_accumulate_dihedral: single-level geometry only")
    for t in range(8):
        gram, counts = gram_accumulate(dihedral(z, t), None, dihedral(target, t), dihedral_bucket(bucket, t, bp),
                                       K, geom, gram, counts)
    return gram, counts


# ---------------------------------------------------------------- noise level

def estimate_noise(img):
    """Noise level of one [3][H][W] image for choosing the bank set trained
    for the nearest level (the paper assumes the level known and points to
    estimating it, Section 6).  Donoho and Johnstone's robust estimate: the
    finest diagonal Haar detail d = (a - b - c + e) / 2 of every 2x2 block
    [a b; c e] (rows and columns 2i, 2i+1; an odd last row/column left out) of
    every channel has variance sigma^2 under i.i.d. Gaussian noise, so
    sigma = median(|d|) / 0.6745 (the median of |N(0, 1)|), in FP64."""
    z = _d(img)
    _, H, W = z.shape
    h2, w2 = H // 2 * 2, W // 2 * 2
    a, b = z[:, 0:h2:2, 0:w2:2], z[:, 0:h2:2, 1:w2:2]
    c, e = z[:, 1:h2:2, 0:w2:2], z[:, 1:h2:2, 1:w2:2]
    d = 0.5 * ((a - b) - (c - e))
    return float(np.median(np.abs(d)) / 0.6744897501960817)
