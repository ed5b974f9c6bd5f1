"""GB300-native trainable multiscale denoising (arXiv 1802.06130).

Thin ctypes binding over ``libmdn.so`` (include/mdn.h).  Every step of the
method runs in the library's CUDA kernels; this module only marshals torch
tensors (device memory, streams) into the C ABI.  There is no CPU fallback:
importing works without a GPU, but every call needs the built library and a
CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB as _LIB_PATH, build

__all__ = ["build", "lib", "Geometry", "BucketParams", "default_bparams", "MdnError",
           "build_pyramid", "select_buckets", "filter_level", "denoise_multiscale",
           "denoise_workspace_bytes", "train_level_filters", "solve_bank", "regressor_len",
           "gram_state_shape", "train_status", "train_cascade", "Server", "F32", "F16", "YCBCR601", "RGB", "GRAM_FP32", "GRAM_TF32",
           "GRAM_BF16", "GRAM_SPLIT_BF16", "augment_dihedral", "dihedral", "estimate_noise", "nearest_level",
           "save_banks", "load_banks", "save_gram_state", "load_gram_state", "paper_grid_bparams",
           "bucket_map_dtype", "MAX_K", "levels_for_sigma", "denoise_multiscale_pipelined", "use_checked_build",
           "PreparedBank", "prepare_bank", "F16_ROWS", "F32_ROWS", "LEVEL_VARIANTS", "autotune_level",
           "autotune_lookup", "autotune_save", "autotune_load", "autotune_clear", "Tensor", "as_tensor",
           "t_build_pyramid", "t_filter_level", "t_denoise_multiscale", "t_train_level_filters",
           "check_status", "pyramid_noise_factor", "set_gram_wait_limit",
           "gram_expire_next_wait"]

F32, F16 = 0, 1
F16_ROWS, F32_ROWS = 2, 3   # prepared banks (mdn_prepare_bank_rows)
YCBCR601, RGB = 0, 1
GRAM_FP32, GRAM_TF32, GRAM_BF16, GRAM_SPLIT_BF16 = 0, 1, 2, 3
MAX_THR = 16
MAX_K = 4096


class MdnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmdn error {code}: {msg}")
        self.code = code


class Geometry(C.Structure):
    """mdn_geometry: r_fine, r_coarse (-1 = single scale), cross_channel, color."""
    _fields_ = [("r_fine", C.c_int32), ("r_coarse", C.c_int32), ("cross_channel", C.c_int32),
                ("color", C.c_int32)]

    def __init__(self, r_fine=3, r_coarse=3, cross_channel=0, color=YCBCR601):
        super().__init__(r_fine, r_coarse, cross_channel, color)


class BucketParams(C.Structure):
    """mdn_bucket_params: angle bins and ascending strength/coherence thresholds."""
    _fields_ = [("n_angle", C.c_int32), ("n_strength", C.c_int32), ("n_coherence", C.c_int32),
                ("strength_thr", C.c_float * MAX_THR), ("coherence_thr", C.c_float * MAX_THR),
                ("coh_eps", C.c_float)]

    def __init__(self, n_angle=24, strength_thr=(0.135, 0.16), coherence_thr=(0.10, 0.15), coh_eps=1e-8):
        super().__init__()
        self.n_angle = n_angle
        self.n_strength = len(strength_thr) + 1
        self.n_coherence = len(coherence_thr) + 1
        for i, t in enumerate(strength_thr):
            self.strength_thr[i] = t
        for i, t in enumerate(coherence_thr):
            self.coherence_thr[i] = t
        self.coh_eps = coh_eps

    @property
    def K(self) -> int:
        return self.n_angle * self.n_strength * self.n_coherence


def default_bparams(level: int) -> BucketParams:
    """Level-l selector defaults: 24 x 3 x 3 buckets, strength thresholds
    (0.135, 0.16) halved per coarser level, coherence thresholds (0.10, 0.15)."""
    s = 0.5 ** level
    return BucketParams(24, (0.135 * s, 0.16 * s), (0.10, 0.15), 1e-8)


# Thresholds of the paper's own 16 x 16 x 16 grid (Section 5 gives the grid,
# not the thresholds): equal-population bins of strength and coherence, the
# quantiles k/16 (k = 1..15) of each feature over a 256x256, sigma = 25/255
# training set at levels 0 and 1; coarser levels halve the level-1 strength
# thresholds per level and keep its coherence thresholds.
_GRID16_STRENGTH = (
    (0.1101, 0.1145, 0.1176, 0.1202, 0.1225, 0.1247, 0.1268, 0.129, 0.1311, 0.1334, 0.1359, 0.1387,
     0.1422, 0.1469, 0.1556),
    (0.0297, 0.031, 0.032, 0.0329, 0.0336, 0.0343, 0.035, 0.0357, 0.0364, 0.0372, 0.038, 0.0391,
     0.0403, 0.0423, 0.0497))
_GRID16_COHERENCE = (
    (0.0232, 0.0335, 0.042, 0.0496, 0.0569, 0.0641, 0.0713, 0.0789, 0.0869, 0.0955, 0.105, 0.1163,
     0.1299, 0.1484, 0.1801),
    (0.0278, 0.0402, 0.0504, 0.0598, 0.0687, 0.0774, 0.0861, 0.095, 0.1047, 0.1153, 0.1273, 0.1412,
     0.1588, 0.1844, 0.242))


def paper_grid_bparams(level: int) -> BucketParams:
    """The paper's 16 x 16 x 16 = 4096-bucket selector for level l (bucket
    maps are then u16, stored as int16 tensors; the bank is read through L2)."""
    if level <= 1:
        return BucketParams(16, _GRID16_STRENGTH[level], _GRID16_COHERENCE[level], 1e-8)
    s = 0.5 ** (level - 1)
    return BucketParams(16, tuple(t * s for t in _GRID16_STRENGTH[1]), _GRID16_COHERENCE[1], 1e-8)


def bucket_map_dtype(K: int):
    """torch dtype of a bucket map for K buckets: uint8 up to 256, else int16
    (the library writes u16 values < 4096)."""
    torch = _torch()
    return torch.uint8 if K <= 256 else torch.int16


class Tensor(C.Structure):
    """mdn_tensor: dtype code, rank, shape, strides (elements), device data."""
    _fields_ = [("dtype", C.c_int32), ("ndim", C.c_int32), ("shape", C.c_int64 * 4), ("strides", C.c_int64 * 4),
                ("data", C.c_void_p)]


U8, U16, F64, I64 = 8, 9, 10, 11


class ServerCfg(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int32),
                ("autotune", C.c_int32), ("tile_variant", C.c_int32), ("geom", Geometry)]


class BankSet(C.Structure):
    _fields_ = [("levels", C.c_int32), ("banks", C.POINTER(C.c_void_p)), ("bparams", C.POINTER(BucketParams)),
                ("color", C.c_int32)]


class ServerResult(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("submit_ms", C.c_double), ("admit_ms", C.c_double),
                ("done_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cancelled", C.c_uint64),
                ("ticks", C.c_uint64), ("tick_items", C.c_uint64), ("active", C.c_int32), ("queued", C.c_int32),
                ("arena_bytes", C.c_size_t), ("arena_used", C.c_size_t), ("arena_peak", C.c_size_t),
                ("tile_variant", C.c_int32), ("variant_ms", C.c_float * 4), ("variant_threads", C.c_int32 * 4),
                ("variant_rows", C.c_int32 * 4), ("ticks_large", C.c_uint64)]


_lib = None
_lib_path = _LIB_PATH


def use_checked_build(enable: bool = True) -> str:
    """Switches this process's calls to the bounds-checked debug library
    (built on first use; see mdn_check_status) or back to the normal one;
    returns the library path now in use."""
    global _lib, _lib_path
    import importlib   # the module, not the function re-exported above under the same name
    bmod = importlib.import_module(__name__ + ".build")
    _lib_path = bmod.build(check=True) if enable else _LIB_PATH
    _lib = None
    return _lib_path


def check_status():
    """(site, index) of the first bounds violation recorded by the checked
    library since the last call ((0, 0): none; site -1: not the checked
    library)."""
    site, idx = C.c_int32(0), C.c_int64(0)
    _check(lib().mdn_check_status(C.byref(site), C.byref(idx)))
    return site.value, idx.value


def lib():
    """The loaded libmdn (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_lib_path):
            raise RuntimeError(f"libmdn is not built ({_lib_path}); call paper_1802_06130_gb300.build()")
        L = C.CDLL(_lib_path)
        vp, i64, i32, sz = C.c_void_p, C.c_int64, C.c_int32, C.c_size_t
        G, B = C.POINTER(Geometry), C.POINTER(BucketParams)
        sig = {
            "mdn_version": (C.c_int, []),
            "mdn_last_error": (C.c_char_p, []),
            "mdn_regressor_len": (C.c_int, [G]),
            "mdn_bucket_elem_bytes": (C.c_int, [i32]),
            "mdn_pyramid_bytes": (sz, [i64, i64, i64, i32, i32]),
            "mdn_build_pyramid": (C.c_int, [vp, i32, i64, i64, i64, i32, C.POINTER(vp), vp]),
            "mdn_select_buckets": (C.c_int, [vp, i32, i64, i64, i64, B, vp, vp]),
            "mdn_filter_level": (C.c_int, [vp, vp, i32, i64, i64, i64, vp, i32, G, B, vp, vp, vp]),
            "mdn_denoise_workspace_bytes": (sz, [i64, i64, i64, i32, i32]),
            "mdn_denoise_multiscale": (C.c_int, [vp, i32, i64, i64, i64, i32, C.POINTER(vp), i32, G, B, vp,
                                                 C.POINTER(vp), vp, sz, vp]),
            "mdn_denoise_multiscale_pipelined": (C.c_int, [vp, i32, i64, i64, i64, i32, C.POINTER(vp), i32, G, B,
                                                           vp, i64, vp, vp, vp, sz, C.POINTER(vp), i32]),
            "mdn_gram_state_bytes": (sz, [G, i32]),
            "mdn_bank_rows_bytes": (sz, [G, i32, i32]),
            "mdn_autotune_level": (C.c_int, [G, B, i32, i32, i64, i64, i64, i32, C.POINTER(i32),
                                             C.POINTER(C.c_float), vp]),
            "mdn_autotune_lookup": (C.c_int, [G, i32, i32, i32, i64, i64, i64]),
            "mdn_autotune_server_lookup": (C.c_int, [G, i32]),
            "mdn_autotune_save": (C.c_int, [C.c_char_p]),
            "mdn_autotune_load": (C.c_int, [C.c_char_p]),
            "mdn_autotune_clear": (None, []),
            "mdn_t_build_pyramid": (C.c_int, [C.POINTER(Tensor), i32, C.POINTER(Tensor), vp]),
            "mdn_t_filter_level": (C.c_int, [C.POINTER(Tensor), C.POINTER(Tensor), C.POINTER(Tensor), G, B,
                                             C.POINTER(Tensor), C.POINTER(Tensor), vp]),
            "mdn_t_denoise_multiscale": (C.c_int, [C.POINTER(Tensor), i32, C.POINTER(Tensor), G, B,
                                                   C.POINTER(Tensor), C.POINTER(Tensor), vp, sz, vp]),
            "mdn_t_train_level_filters": (C.c_int, [C.POINTER(Tensor), C.POINTER(Tensor), C.POINTER(Tensor), G, B,
                                                    i32, i32, C.POINTER(Tensor), C.POINTER(Tensor), C.c_double,
                                                    C.POINTER(Tensor), vp, sz, vp]),
            "mdn_prepare_bank_rows": (C.c_int, [vp, i32, G, i32, vp, sz, vp]),
            "mdn_train_workspace_bytes": (sz, [i64, i64, i64, G, i32, i32]),
            "mdn_train_level_filters": (C.c_int, [vp, vp, vp, i32, i64, i64, i64, G, B, i32, i32, vp, vp,
                                                  C.c_double, vp, vp, sz, vp]),
            "mdn_solve_workspace_bytes": (sz, [G, i32]),
            "mdn_train_status": (C.c_int, [C.POINTER(C.c_int32)]),
            "mdn_set_gram_wait_limit": (C.c_int, [C.c_uint64]),
            "mdn_check_status": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
            "mdn_gram_expire_next_wait": (C.c_int, [i32]),
            "mdn_pyramid_noise_factor": (C.c_double, [i32]),
            "mdn_levels_for_sigma": (i32, [C.c_double, C.c_double, i32, i32]),
            "mdn_solve_bank": (C.c_int, [vp, vp, G, i32, C.c_double, vp, vp, vp, sz, vp]),
            "mdn_augment_dihedral": (C.c_int, [vp, vp, G, B, vp, vp, vp]),
            "mdn_noise_workspace_bytes": (sz, [i64]),
            "mdn_dihedral_images": (C.c_int, [vp, i32, i64, i64, i64, i32, vp, vp]),
            "mdn_estimate_noise": (C.c_int, [vp, i32, i64, i64, i64, vp, vp, sz, vp]),
            "mdn_server_create": (C.c_int, [C.POINTER(ServerCfg), C.POINTER(BankSet), i32, C.POINTER(vp)]),
            "mdn_server_submit": (C.c_int, [vp, vp, vp, i64, i64, i32, C.POINTER(C.c_uint64)]),
            "mdn_server_cancel": (C.c_int, [vp, C.c_uint64]),
            "mdn_server_poll": (C.c_int, [vp, C.POINTER(ServerResult), i32, C.POINTER(i32), i32]),
            "mdn_server_get_stats": (C.c_int, [vp, C.POINTER(ServerStats)]),
            "mdn_server_destroy": (C.c_int, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers

def _torch():
    import torch
    return torch


def _check(rc: int):
    if rc != 0:
        raise MdnError(rc, lib().mdn_last_error().decode())


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float16:
        return F16
    raise TypeError(f"unsupported dtype {t.dtype} (float32 or float16)")


class PreparedBank:
    """A filter bank in the fused level kernel's row-slot layout
    (mdn_prepare_bank_rows); accepted wherever a bank tensor is."""

    def __init__(self, rows, code: int, K: int, geom: Geometry):
        self.rows, self.code, self.K = rows, code, K
        self.geom = (geom.r_fine, geom.r_coarse, int(geom.cross_channel != 0))

    def data_ptr(self):
        return self.rows.data_ptr()


def prepare_bank(bank, geom: Geometry, stream=None) -> PreparedBank:
    """Lays out a [K][3][D] FP16/FP32 CUDA bank once in the fused kernel's
    row slots (mdn_prepare_bank_rows): banks too large for shared memory are
    then read through L2 with 16-byte loads."""
    torch = _torch()
    K = bank.shape[0]
    code = _dtype_code(bank)
    nbytes = lib().mdn_bank_rows_bytes(C.byref(geom), K, code)
    if nbytes == 0:
        raise ValueError("prepare_bank: geometry not compiled or bad bank")
    rows = torch.empty(nbytes, dtype=torch.uint8, device=bank.device)
    _check(lib().mdn_prepare_bank_rows(_dev(bank, "bank"), code, C.byref(geom), K, _dev(rows, "rows"), nbytes,
                                       _stream(stream)))
    return PreparedBank(rows, F16_ROWS if code == F16 else F32_ROWS, K, geom)


def _check_banks(banks, geom: Geometry, bparams):
    """The C ABI takes one bank type for all levels, and a prepared bank's
    layout is fixed by the geometry and bucket count it was prepared for."""
    codes = {_bank_code(b) for b in banks}
    if len(codes) != 1:
        raise ValueError("all banks must have the same dtype / layout")
    g = (geom.r_fine, geom.r_coarse, int(geom.cross_channel != 0))
    for b, bp in zip(banks, bparams):
        if isinstance(b, PreparedBank) and (b.geom != g or b.K != bp.K):
            raise ValueError(f"prepared bank is for geometry {b.geom} with K={b.K}, "
                             f"call has {g} with K={bp.K}")


def as_tensor(t):
    """An mdn_tensor describing a CUDA torch tensor (its own shape and strides;
    the library checks them), or a PreparedBank (1-D row-slot bytes)."""
    torch = _torch()
    if t is None:
        return None
    if isinstance(t, PreparedBank):
        d = Tensor(t.code, 1)
        d.shape[0], d.strides[0], d.data = t.rows.numel(), 1, t.rows.data_ptr()
        return d
    codes = {torch.float32: F32, torch.float16: F16, torch.uint8: U8, torch.int16: U16, torch.float64: F64,
             torch.int64: I64}
    if t.dtype not in codes:
        raise ValueError(f"no mdn_tensor dtype for {t.dtype}")
    if t.dim() > 4:
        raise ValueError("mdn_tensor has at most 4 dimensions")
    d = Tensor(codes[t.dtype], t.dim())
    for i in range(t.dim()):
        d.shape[i], d.strides[i] = t.shape[i], t.stride(i)
    d.data = t.data_ptr()
    return d


def _tarr(ts):
    arr = (Tensor * max(len(ts), 1))()
    for i, t in enumerate(ts):
        if t is not None:
            arr[i] = as_tensor(t)
    return arr


def t_build_pyramid(img, levels: int, outs, stream=None):
    """mdn_t_build_pyramid: img [N][3][H][W], outs the levels-1 output tensors."""
    _check(lib().mdn_t_build_pyramid(C.byref(as_tensor(img)), levels, _tarr(outs), _stream(stream)))


def t_filter_level(z, coarse, bank, geom: Geometry, bp: BucketParams, out, buckets_out=None, stream=None):
    """mdn_t_filter_level with tensor descriptors (shapes and strides checked by the library)."""
    c = as_tensor(coarse)
    m = as_tensor(buckets_out)
    _check(lib().mdn_t_filter_level(C.byref(as_tensor(z)), C.byref(c) if c is not None else None,
                                    C.byref(as_tensor(bank)), C.byref(geom), C.byref(bp), C.byref(as_tensor(out)),
                                    C.byref(m) if m is not None else None, _stream(stream)))


def t_denoise_multiscale(noisy, banks, geom: Geometry, bparams, out, bucket_maps=None, ws=None, stream=None):
    """mdn_t_denoise_multiscale with tensor descriptors; ws a CUDA uint8 tensor
    of at least denoise_workspace_bytes (allocated here when None)."""
    torch = _torch()
    n, _, h, w = noisy.shape
    levels = 1 if geom.r_coarse < 0 else len(banks) + 1
    need = denoise_workspace_bytes(n, h, w, levels, _dtype_code(noisy))
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=noisy.device)
    parr = (BucketParams * len(bparams))(*bparams)
    _check(lib().mdn_t_denoise_multiscale(C.byref(as_tensor(noisy)), levels, _tarr(banks), C.byref(geom), parr,
                                          C.byref(as_tensor(out)), _tarr(bucket_maps) if bucket_maps else None,
                                          C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def t_train_level_filters(noisy, coarse, clean, geom: Geometry, bp: BucketParams, gram_precision: int, gram, counts,
                          lam: float = 1e-3, bank_out=None, accumulate: bool = False, ws=None, stream=None):
    """mdn_t_train_level_filters with tensor descriptors; gram [K][G][Dp][Dp]
    float64, counts [K] int64, bank_out [K][3][D] float32 or None."""
    torch = _torch()
    n, _, h, w = noisy.shape
    need = lib().mdn_train_workspace_bytes(n, h, w, C.byref(geom), bp.K, gram_precision)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=noisy.device)
    c = as_tensor(coarse)
    b = as_tensor(bank_out)
    _check(lib().mdn_t_train_level_filters(C.byref(as_tensor(noisy)), C.byref(c) if c is not None else None,
                                           C.byref(as_tensor(clean)), C.byref(geom), C.byref(bp), gram_precision,
                                           int(accumulate), C.byref(as_tensor(gram)), C.byref(as_tensor(counts)),
                                           lam, C.byref(b) if b is not None else None, C.c_void_p(ws.data_ptr()),
                                           ws.numel(), _stream(stream)))


LEVEL_VARIANTS = ("fused_smem", "fused_l2", "strip", "tile_smem", "tile_l2", "fused_cluster")


def autotune_level(geom: Geometry, bp: BucketParams, dtype: int, bank_dtype: int, n: int, h: int, w: int,
                   reps: int = 3, stream=None):
    """Times every level-kernel variant that applies to this configuration
    (mdn_autotune_level) and records the fastest in the autotune table, which
    the level calls then follow.  -> (best variant index, {name: ms or None})."""
    best = C.c_int32(-1)
    ms = (C.c_float * len(LEVEL_VARIANTS))()
    _check(lib().mdn_autotune_level(C.byref(geom), C.byref(bp), dtype, bank_dtype, n, h, w, reps, C.byref(best), ms,
                                    _stream(stream)))
    return best.value, {name: (round(ms[i], 5) if ms[i] >= 0 else None) for i, name in enumerate(LEVEL_VARIANTS)}


def autotune_lookup(geom: Geometry, K: int, dtype: int, bank_dtype: int, n: int, h: int, w: int) -> int:
    return lib().mdn_autotune_lookup(C.byref(geom), K, dtype, bank_dtype, n, h, w)


def autotune_save(path):
    _check(lib().mdn_autotune_save(str(path).encode()))


def autotune_load(path):
    _check(lib().mdn_autotune_load(str(path).encode()))


def autotune_clear():
    lib().mdn_autotune_clear()


def _bank_code(b) -> int:
    return b.code if isinstance(b, PreparedBank) else _dtype_code(b)


def _bank_dev(b, name="bank"):
    return _dev(b.rows if isinstance(b, PreparedBank) else b, name)


def _dev(t, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _img(t):
    if t.dim() == 3:
        t = t.unsqueeze(0)
    if t.dim() != 4 or t.shape[1] != 3:
        raise ValueError("images are [n][3][h][w] (or [3][h][w])")
    return t


def regressor_len(geom: Geometry) -> int:
    return lib().mdn_regressor_len(C.byref(geom))


def gram_state_shape(geom: Geometry, K: int):
    D = regressor_len(geom)
    G, T = (1, 3) if geom.cross_channel else (3, 1)
    return (K, G, D + T, D + T)


# ---------------------------------------------------------------- API

def build_pyramid(img, levels: int, stream=None):
    """[z^1 .. z^{L-1}] of an [n][3][h][w] image (mdn_build_pyramid)."""
    torch = _torch()
    img4 = _img(img)
    n, _, h, w = img4.shape
    outs, ptrs = [], []
    hh, ww = h, w
    for _ in range(1, levels):
        hh, ww = (hh + 1) // 2, (ww + 1) // 2
        o = torch.empty((n, 3, hh, ww), dtype=img4.dtype, device=img4.device)
        outs.append(o)
        ptrs.append(o.data_ptr())
    arr = (C.c_void_p * max(len(ptrs), 1))(*ptrs)
    _check(lib().mdn_build_pyramid(_dev(img4, "img"), _dtype_code(img4), n, h, w, levels, arr, _stream(stream)))
    return [o if img.dim() == 4 else o[0] for o in outs]


def _map(m, K: int, n: int, h: int, w: int, name: str):
    """Device pointer of a bucket map after checking its type and size (the
    library writes one u8 per pixel for K <= 256 and one u16 above)."""
    if m is None:
        return None
    if m.dtype != bucket_map_dtype(K) or m.numel() != n * h * w:
        raise ValueError(f"{name}: need {bucket_map_dtype(K)} with {n * h * w} elements for {K} buckets, "
                         f"got {m.dtype} with {m.numel()}")
    return _dev(m, name)


def select_buckets(z, bp: BucketParams, stream=None):
    """Bucket map s(i), [n][h][w] uint8 (K <= 256) or int16 (mdn_select_buckets)."""
    torch = _torch()
    z4 = _img(z)
    n, _, h, w = z4.shape
    out = torch.empty((n, h, w), dtype=bucket_map_dtype(bp.K), device=z4.device)
    _check(lib().mdn_select_buckets(_dev(z4, "z"), _dtype_code(z4), n, h, w, C.byref(bp), _dev(out), _stream(stream)))
    return out if z.dim() == 4 else out[0]


def filter_level(z, coarse, bank, geom: Geometry, bp: BucketParams, out=None, buckets_out=None, stream=None):
    """One fused level: selector + filter (mdn_filter_level).  Returns out."""
    torch = _torch()
    z4 = _img(z)
    n, _, h, w = z4.shape
    c4 = _img(coarse) if coarse is not None else None
    if out is None:
        out = torch.empty_like(z4)
    _check_banks([bank], geom, [bp])
    _check(lib().mdn_filter_level(_dev(z4, "z"), _dev(c4, "coarse"), _dtype_code(z4), n, h, w, _bank_dev(bank),
                                  _bank_code(bank), C.byref(geom), C.byref(bp), _dev(out, "out"),
                                  _map(buckets_out, bp.K, n, h, w, "buckets_out"), _stream(stream)))
    return out if z.dim() == 4 else out[0]


def denoise_workspace_bytes(n, h, w, levels, dtype_code) -> int:
    return lib().mdn_denoise_workspace_bytes(n, h, w, levels, dtype_code)


def denoise_multiscale(noisy, banks, geom: Geometry, bparams, out=None, bucket_maps=None, ws=None, stream=None):
    """Section 4 multiscale inference (mdn_denoise_multiscale).

    banks: list of max(L-1, 1) [K][3][D] tensors; bparams: list of the same
    length; levels = len(banks) + 1 (or 1 when geom.r_coarse < 0)."""
    torch = _torch()
    z4 = _img(noisy)
    n, _, h, w = z4.shape
    levels = 1 if geom.r_coarse < 0 else len(banks) + 1
    nb = len(banks)
    if len(bparams) != nb:
        raise ValueError("need one BucketParams per bank")
    if out is None:
        out = torch.empty_like(z4)
    need = denoise_workspace_bytes(n, h, w, levels, _dtype_code(z4))
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=z4.device)
    _check_banks(banks, geom, bparams)
    bank_dt = _bank_code(banks[0])
    barr = (C.c_void_p * nb)(*[b.data_ptr() for b in banks])
    parr = (BucketParams * nb)(*bparams)
    marr = None
    if bucket_maps is not None:
        if len(bucket_maps) != nb:
            raise ValueError("need one bucket map entry (or None) per bank")
        ptrs, hl, wl = [], h, w
        for l in range(nb):
            p = _map(bucket_maps[l], bparams[l].K, n, hl, wl, f"bucket_maps[{l}]")
            ptrs.append(p.value if p is not None else None)
            hl, wl = (hl + 1) // 2, (wl + 1) // 2
        marr = (C.c_void_p * nb)(*ptrs)
    _check(lib().mdn_denoise_multiscale(_dev(z4, "noisy"), _dtype_code(z4), n, h, w, levels, barr, bank_dt,
                                        C.byref(geom), parr, _dev(out, "out"), marr, _dev(ws, "ws"),
                                        ws.numel() * ws.element_size(), _stream(stream)))
    return out if noisy.dim() == 4 else out[0]


def denoise_multiscale_pipelined(host_noisy, banks, geom: Geometry, bparams, host_out, chunk: int = 1,
                                 dev_in=None, dev_out=None, ws=None, streams=None, two_compute: bool = True):
    """Multiscale denoise of a batch in (pinned) host memory with the copies and
    kernels of consecutive chunks overlapped (mdn_denoise_multiscale_pipelined).
    host_noisy, host_out: [n][3][h][w] CPU tensors; dev_in, dev_out: matching
    CUDA tensors (allocated if None); ws: workspace for `chunk` images per
    compute stream; streams: (upload, compute, download) or (upload, compute
    A, compute B, download) torch streams (the first compute stream defaults
    to the current stream; two_compute picks the default layout).
    Asynchronous: host_out is complete once the first compute stream is
    synchronised.  Returns (dev_in, dev_out, ws, streams) for reuse."""
    torch = _torch()
    x = _img(host_noisy)
    n, _, h, w = x.shape
    if x.is_cuda or host_out.is_cuda or host_out.shape != x.shape or host_out.dtype != x.dtype:
        raise ValueError("host_noisy/host_out: matching [n][3][h][w] CPU tensors")
    if not x.is_contiguous() or not host_out.is_contiguous():
        raise ValueError("host tensors must be contiguous")
    dev = torch.device("cuda", torch.cuda.current_device())
    levels = 1 if geom.r_coarse < 0 else len(banks) + 1
    nb = len(banks)
    if len(bparams) != nb:
        raise ValueError("need one BucketParams per bank")
    if dev_in is None:
        dev_in = torch.empty(x.shape, dtype=x.dtype, device=dev)
    if dev_out is None:
        dev_out = torch.empty(x.shape, dtype=x.dtype, device=dev)
    c = max(1, min(chunk, n))
    if streams is None:
        cur = torch.cuda.current_stream(dev)
        streams = ((torch.cuda.Stream(device=dev), cur, torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))
                   if two_compute else (torch.cuda.Stream(device=dev), cur, torch.cuda.Stream(device=dev)))
    per = denoise_workspace_bytes(c, h, w, levels, _dtype_code(x))
    need = per if len(streams) == 3 else 2 * ((per + 255) // 256 * 256)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    sarr = (C.c_void_p * len(streams))(*[st.cuda_stream for st in streams])
    _check_banks(banks, geom, bparams)
    barr = (C.c_void_p * nb)(*[b.data_ptr() for b in banks])
    parr = (BucketParams * nb)(*bparams)
    _check(lib().mdn_denoise_multiscale_pipelined(C.c_void_p(x.data_ptr()), _dtype_code(x), n, h, w, levels, barr,
                                                  _bank_code(banks[0]), C.byref(geom), parr,
                                                  C.c_void_p(host_out.data_ptr()), chunk, _dev(dev_in, "dev_in"),
                                                  _dev(dev_out, "dev_out"), _dev(ws, "ws"),
                                                  ws.numel() * ws.element_size(), sarr, len(streams)))
    return dev_in, dev_out, ws, streams


def train_level_filters(noisy_lvl, coarse_out, clean_lvl, geom: Geometry, bp: BucketParams,
                        gram_precision: int = GRAM_SPLIT_BF16, gram=None, counts=None, accumulate=False,
                        lam: float = 1e-3, solve: bool = True, ws=None, stream=None):
    """One level of training (mdn_train_level_filters).

    Returns (gram [K][G][Dp][Dp] f64, counts [K] i64, bank [K][3][D] f32 or None)."""
    torch = _torch()
    z4 = _img(noisy_lvl)
    u4 = _img(clean_lvl)
    c4 = _img(coarse_out) if coarse_out is not None else None
    n, _, h, w = z4.shape
    K = bp.K
    dev = z4.device
    if gram is None:
        gram = torch.zeros(gram_state_shape(geom, K), dtype=torch.float64, device=dev)
        counts = torch.zeros(K, dtype=torch.int64, device=dev)
    bank = torch.empty((K, 3, regressor_len(geom)), dtype=torch.float32, device=dev) if solve else None
    need = lib().mdn_train_workspace_bytes(n, h, w, C.byref(geom), K, gram_precision)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    _check(lib().mdn_train_level_filters(_dev(z4, "noisy"), _dev(c4, "coarse"), _dev(u4, "clean"), _dtype_code(z4),
                                         n, h, w, C.byref(geom), C.byref(bp), gram_precision, int(accumulate),
                                         _dev(gram, "gram"), _dev(counts, "counts"), lam,
                                         _dev(bank, "bank") if bank is not None else None, _dev(ws, "ws"),
                                         ws.numel(), _stream(stream)))
    return gram, counts, bank


def train_status() -> int:
    """Reads and clears the tensor-core Gram error flag (1 = a bounded wait expired)."""
    v = C.c_int32(0)
    _check(lib().mdn_train_status(C.byref(v)))
    return v.value


def set_gram_wait_limit(ns: int = 0):
    """Bound of every wait inside the tensor-core Gram kernel for later
    launches, in ns (0 = the default 2 s) (mdn_set_gram_wait_limit)."""
    _check(lib().mdn_set_gram_wait_limit(int(ns)))


def gram_expire_next_wait(enable: bool = True):
    """Makes the next tensor-core Gram launch wait on a barrier phase that
    nothing completes, so that its bounded wait runs out (failure-detection
    test; mdn_gram_expire_next_wait)."""
    _check(lib().mdn_gram_expire_next_wait(int(enable)))


class Server:
    """Continuous-batching denoise server (mdn_server_*).

    bank_sets: list of (banks, bparams) with banks a list of levels-1 FP16
    [K][3][D] CUDA tensors in the server's geometry (default 7x7 + 7x7 per
    channel, D = 98; Geometry(3, 2) for 7x7 + 5x5, D = 74), K up to 4096,
    and bparams the matching BucketParams list.  Inputs/outputs are host
    FP16 [3][h][w] tensors (pinned for asynchronous copies) kept alive until
    polled.  tile_variant (autotune off): 0-2 tile kernels, 3 fused kernel,
    -1 the autotune table's entry (else 3)."""

    def __init__(self, bank_sets, budget_bytes: int, max_active: int = 16, autotune: bool = True,
                 tile_variant: int = -1, device: int = 0, color: int = YCBCR601, geom: Geometry = None):
        self._keep = []
        n = len(bank_sets)
        arr = (BankSet * n)()
        for i, (banks, bparams) in enumerate(bank_sets):
            if len(banks) != len(bparams):
                raise ValueError("one BucketParams per bank")
            ptrs = (C.c_void_p * len(banks))(*[b.data_ptr() for b in banks])
            bps = (BucketParams * len(bparams))(*bparams)
            self._keep += [ptrs, bps, banks]
            arr[i].levels = len(banks) + 1
            arr[i].banks = C.cast(ptrs, C.POINTER(C.c_void_p))
            arr[i].bparams = C.cast(bps, C.POINTER(BucketParams))
            arr[i].color = color
        cfg = ServerCfg(device, budget_bytes, max_active, int(autotune), tile_variant,
                        geom if geom is not None else Geometry(3, 3))
        h = C.c_void_p()
        _check(lib().mdn_server_create(C.byref(cfg), arr, n, C.byref(h)))
        self._h = h
        self._io = {}

    def submit(self, host_in, host_out, bank_set: int) -> int:
        if host_in.dtype != host_out.dtype or host_in.shape != host_out.shape or host_in.dim() != 3:
            raise ValueError("host_in/host_out: matching [3][h][w] FP16 host tensors")
        if host_in.is_cuda or host_out.is_cuda or not host_in.is_contiguous() or not host_out.is_contiguous():
            raise ValueError("host_in/host_out must be contiguous host tensors")
        rid = C.c_uint64()
        _, h, w = host_in.shape
        _check(lib().mdn_server_submit(self._h, C.c_void_p(host_in.data_ptr()), C.c_void_p(host_out.data_ptr()),
                                       h, w, bank_set, C.byref(rid)))
        self._io[rid.value] = (host_in, host_out)
        return rid.value

    def cancel(self, rid: int):
        _check(lib().mdn_server_cancel(self._h, rid))

    def poll(self, max_results: int = 64, timeout_ms: int = 100):
        res = (ServerResult * max_results)()
        n = C.c_int32()
        _check(lib().mdn_server_poll(self._h, res, max_results, C.byref(n), timeout_ms))
        out = []
        for i in range(n.value):
            r = res[i]
            self._io.pop(r.id, None)
            out.append({"id": r.id, "status": r.status, "submit_ms": r.submit_ms, "admit_ms": r.admit_ms,
                        "done_ms": r.done_ms})
        return out

    def stats(self):
        st = ServerStats()
        _check(lib().mdn_server_get_stats(self._h, C.byref(st)))
        d = {f: getattr(st, f) for f, _ in ServerStats._fields_}
        for k in ("variant_ms", "variant_threads", "variant_rows"):
            d[k] = list(d[k])
        return d

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().mdn_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dihedral(img, t: int, stream=None):
    """Transform t = rot + 4 * flip of [n][3][h][w] (or [3][h][w]) images on the
    device (mdn_dihedral_images): rotate by 90 degrees rot times (numpy's rot90
    on the row/column axes), then mirror the columns if flip."""
    torch = _torch()
    x = _img(img)
    n, _, h, w = x.shape
    out = torch.empty((n, 3, w, h) if t & 1 else (n, 3, h, w), dtype=x.dtype, device=x.device)
    _check(lib().mdn_dihedral_images(_dev(x, "img"), _dtype_code(x), n, h, w, t, _dev(out, "out"), _stream(stream)))
    return out


def train_cascade(noisy, clean, geom: Geometry, levels: int, bparams=None, gram_precision: int = GRAM_SPLIT_BF16,
                  lam: float = 1e-3, chunk: int = 0, augment: bool = False, checkpoint: str = None, stream=None):
    """Section 4 training cascade on the GPU: pyramids of the noisy and clean
    images, then for l = L-2 .. 0 (single-scale: l = 0 only) the bucketed
    least-squares fit of level l (mdn_train_level_filters) with the trained
    coarser output as the coarse input, and that level's output on every
    training image (mdn_filter_level) for the next finer level.  Base case:
    the coarse input of level L-2 is z^{L-1}.

    noisy, clean: [n][3][h][w] CUDA tensors, or lists of such tensors (image
    sets of different shapes, trained together); chunk > 0 feeds the images to
    the Gram accumulation in groups of that many (same result up to FP64
    summation order).  augment: train on the 8 flips / 90-degree rotations of
    every pair (Section 5) -- single-level geometries by permuting the Gram
    sums (mdn_augment_dihedral), multiscale ones on the transformed pairs
    (mdn_dihedral_images), whose pyramids are their own.  checkpoint: path
    prefix; each trained level writes "<prefix>.level<l>.gram" (its Gram
    state) and "<prefix>.level<l>.bank", and a level whose files exist is
    loaded instead of trained (its outputs are recomputed for the finer
    levels), so an interrupted cascade resumes at the level it stopped in.
    Returns (banks [K][3][D] FP32 per level, counts per level)."""
    import os
    torch = _torch()
    single = geom.r_coarse < 0
    nsets = list(noisy) if isinstance(noisy, (list, tuple)) else [noisy]
    csets = list(clean) if isinstance(clean, (list, tuple)) else [clean]
    if augment and not single:
        # the 8 transformed copies of every set, grouped by shape
        by_shape = {}
        for z, u in zip(nsets, csets):
            for t in range(8):
                zt, ut = dihedral(z, t, stream), dihedral(u, t, stream)
                by_shape.setdefault(tuple(zt.shape[2:]), []).append((zt, ut))
        nsets = [torch.cat([a for a, _ in v]) for v in by_shape.values()]
        csets = [torch.cat([b for _, b in v]) for v in by_shape.values()]
    L = 1 if single else levels
    nb = max(levels - 1, 1)
    if bparams is None:
        bparams = [default_bparams(l) for l in range(nb)]
    zp = [[z] + (build_pyramid(z, L, stream) if L > 1 else []) for z in nsets]
    up = [[u] + (build_pyramid(u, L, stream) if L > 1 else []) for u in csets]
    cur = [p[L - 1] if not single else None for p in zp]
    banks, counts_out = [None] * nb, [None] * nb
    perm = augment and single
    for l in range(L - 2 if L > 1 else 0, -1, -1):
        gram = counts = bank = None
        ck = f"{checkpoint}.level{l}" if checkpoint else None
        if ck and os.path.exists(ck + ".bank") and os.path.exists(ck + ".gram"):
            dev = nsets[0].device
            bl, _, _, _ = load_banks(ck + ".bank", device=dev)
            _, counts, _, _, _ = load_gram_state(ck + ".gram", device=dev)
            banks[l], counts_out[l] = bl[0], counts
            if l > 0 or not single:
                for si in range(len(nsets)):
                    out = torch.empty_like(zp[si][l])
                    filter_level(zp[si][l], cur[si], banks[l], geom, bparams[l], out=out, stream=stream)
                    cur[si] = out
            continue
        nchunks = sum((z.shape[0] + (chunk if chunk > 0 else z.shape[0]) - 1) // (chunk if chunk > 0 else z.shape[0])
                      for z in nsets)
        done = 0
        for si in range(len(nsets)):
            n = nsets[si].shape[0]
            step = chunk if chunk > 0 else n
            for i0 in range(0, n, step):
                sl = slice(i0, min(n, i0 + step))
                done += 1
                last = done == nchunks
                c_in = cur[si][sl].contiguous() if cur[si] is not None else None
                gram, counts, bank = train_level_filters(
                    zp[si][l][sl].contiguous(), c_in, up[si][l][sl].contiguous(), geom, bparams[l], gram_precision,
                    gram=gram, counts=counts, accumulate=gram is not None, lam=lam, solve=last and not perm,
                    stream=stream)
        if perm:
            gram, counts = augment_dihedral(gram, counts, geom, bparams[l], stream=stream)
            bank, _ = solve_bank(gram, counts, geom, lam, stream=stream)
        banks[l], counts_out[l] = bank, counts
        if ck:
            save_gram_state(ck + ".gram", gram, counts, geom, bparams[l], l)
            save_banks(ck + ".bank", [bank], geom, [bparams[l]])
        if l > 0 or not single:
            for si in range(len(nsets)):
                out = torch.empty_like(zp[si][l])
                filter_level(zp[si][l], cur[si], bank, geom, bparams[l], out=out, stream=stream)
                cur[si] = out
    return banks, counts_out


# ---------------------------------------------------------------- checkpoints
#
# File format (banks and Gram state alike): one line of UTF-8 JSON (the
# header, ending in "\n"), then the arrays it lists, raw little-endian, in
# header order.  Banks are FP32 [K][3][D] per level; the Gram state is FP64
# [K][G][Dp][Dp] plus int64 counts [K].

_CKPT_FORMAT = "mdn-1"


def _geom_dict(g: Geometry) -> dict:
    return {"r_fine": g.r_fine, "r_coarse": g.r_coarse, "cross_channel": g.cross_channel, "color": g.color}


def _bp_dict(b: BucketParams) -> dict:
    return {"n_angle": b.n_angle, "n_strength": b.n_strength, "n_coherence": b.n_coherence,
            "strength_thr": [float(b.strength_thr[i]) for i in range(b.n_strength - 1)],
            "coherence_thr": [float(b.coherence_thr[i]) for i in range(b.n_coherence - 1)],
            "coh_eps": float(b.coh_eps)}


def _bp_from(d: dict) -> BucketParams:
    b = BucketParams(d["n_angle"])
    b.n_strength, b.n_coherence = d["n_strength"], d["n_coherence"]
    for i, t in enumerate(d["strength_thr"]):
        b.strength_thr[i] = t
    for i, t in enumerate(d["coherence_thr"]):
        b.coherence_thr[i] = t
    b.coh_eps = d["coh_eps"]
    return b


def _write(path, header: dict, arrays):
    import json
    import numpy as np
    with open(path, "wb") as f:
        f.write((json.dumps(header) + "\n").encode())
        for a in arrays:
            f.write(np.ascontiguousarray(a).tobytes())


def _read(path):
    import json
    with open(path, "rb") as f:
        header = json.loads(f.readline().decode())
        if header.get("format") != _CKPT_FORMAT:
            raise ValueError(f"{path}: not an {_CKPT_FORMAT} checkpoint")
        return header, f.read()


def _check_payload(path, raw, nbytes):
    if len(raw) != nbytes:
        raise ValueError(f"{path}: payload is {len(raw)} bytes, the header describes {nbytes}")


def save_banks(path, banks, geom: Geometry, bparams, sigma=None):
    """Writes a bank set (one [K][3][D] FP32 or FP16 bank per level) with its
    geometry, per-level bucket parameters and the noise level it was trained
    for; the payload keeps each bank's own precision."""
    import numpy as np
    torch = _torch()
    arr, dts = [], []
    for b in banks:
        if b.dtype not in (torch.float32, torch.float16):
            raise ValueError(f"save_banks: banks must be float32 or float16, got {b.dtype}")
        dt = "<f2" if b.dtype == torch.float16 else "<f4"
        arr.append(b.detach().cpu().numpy().astype(dt))
        dts.append(dt)
    header = {"format": _CKPT_FORMAT, "kind": "banks", "geometry": _geom_dict(geom),
              "bparams": [_bp_dict(b) for b in bparams], "sigma": sigma,
              "shapes": [list(a.shape) for a in arr], "dtypes": dts}
    _write(path, header, arr)


def load_banks(path, device="cuda"):
    """-> (banks, geometry, bparams, sigma) from save_banks."""
    import numpy as np
    torch = _torch()
    h, raw = _read(path)
    if h["kind"] != "banks":
        raise ValueError(f"{path}: not a bank checkpoint")
    dts = h.get("dtypes", [h.get("dtype", "<f4")] * len(h["shapes"]))   # older files: one FP32 dtype
    if len(dts) != len(h["shapes"]) or any(d not in ("<f4", "<f2") for d in dts):
        raise ValueError(f"{path}: bad bank dtypes {dts}")
    sizes = [int(np.prod(shp)) * (2 if d == "<f2" else 4) for shp, d in zip(h["shapes"], dts)]
    _check_payload(path, raw, sum(sizes))
    banks, off = [], 0
    for shp, d, nb in zip(h["shapes"], dts, sizes):
        a = np.frombuffer(raw, dtype=d, count=nb // (2 if d == "<f2" else 4), offset=off).reshape(shp)
        off += nb
        banks.append(torch.tensor(a, dtype=torch.float16 if d == "<f2" else torch.float32, device=device))
    g = h["geometry"]
    geom = Geometry(g["r_fine"], g["r_coarse"], g["cross_channel"], g["color"])
    return banks, geom, [_bp_from(d) for d in h["bparams"]], h["sigma"]


def save_gram_state(path, gram, counts, geom: Geometry, bp: BucketParams, level: int = 0):
    """Writes the accumulated Gram sums of one level (FP64 [K][G][Dp][Dp]) and
    its counts (int64 [K]), so that training can resume or add more pairs."""
    g = gram.detach().cpu().numpy().astype("<f8")
    c = counts.detach().cpu().numpy().astype("<i8")
    header = {"format": _CKPT_FORMAT, "kind": "gram", "geometry": _geom_dict(geom), "bparams": _bp_dict(bp),
              "level": level, "gram_shape": list(g.shape), "counts_shape": list(c.shape)}
    _write(path, header, [g, c])


def load_gram_state(path, device="cuda"):
    """-> (gram, counts, geometry, bparams, level) from save_gram_state."""
    import numpy as np
    torch = _torch()
    h, raw = _read(path)
    if h["kind"] != "gram":
        raise ValueError(f"{path}: not a Gram checkpoint")
    n = int(np.prod(h["gram_shape"]))
    _check_payload(path, raw, 8 * n + 8 * int(np.prod(h["counts_shape"])))
    g = np.frombuffer(raw, dtype="<f8", count=n).reshape(h["gram_shape"])
    c = np.frombuffer(raw, dtype="<i8", count=int(np.prod(h["counts_shape"])), offset=8 * n)
    gm = h["geometry"]
    geom = Geometry(gm["r_fine"], gm["r_coarse"], gm["cross_channel"], gm["color"])
    return (torch.tensor(g, device=device), torch.tensor(c, device=device), geom, _bp_from(h["bparams"]),
            h["level"])


def estimate_noise(img, stream=None):
    """Noise-level estimate per image (mdn_estimate_noise): robust wavelet
    estimate median(|d|) / 0.6745 of the finest diagonal Haar details of all
    channels.  img: [n][3][h][w] or [3][h][w] CUDA F32/F16 -> float32 [n]."""
    torch = _torch()
    x = _img(img)
    n, _, h, w = x.shape
    sig = torch.empty(n, dtype=torch.float32, device=x.device)
    need = lib().mdn_noise_workspace_bytes(n)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=x.device)
    _check(lib().mdn_estimate_noise(_dev(x, "img"), _dtype_code(x), n, h, w, _dev(sig, "sigma"), _dev(ws, "ws"),
                                    need, _stream(stream)))
    return sig


def nearest_level(sigma: float, levels) -> int:
    """Index of the trained noise level closest to an estimate (host helper
    for choosing a bank set)."""
    return min(range(len(levels)), key=lambda i: abs(levels[i] - sigma))


def pyramid_noise_factor(level: int) -> float:
    """White-noise standard deviation at pyramid level l relative to the input,
    for this library's binomial pyramid (mdn_pyramid_noise_factor)."""
    v = lib().mdn_pyramid_noise_factor(level)
    if v < 0:
        raise ValueError("level must be 0..7")
    return v


def levels_for_sigma(sigma: float, coarsest: float = 2.0 / 255.0, min_levels: int = 1,
                     max_levels: int = 8) -> int:
    """Section 5's depth rule (mdn_levels_for_sigma): the fewest levels whose
    coarsest level's noise is below `coarsest` (2/255), clamped to
    [min_levels, max_levels]; pass min_levels = 2 for multiscale bank sets."""
    L = lib().mdn_levels_for_sigma(sigma, coarsest, min_levels, max_levels)
    if L < 0:
        raise ValueError("bad arguments to levels_for_sigma")
    return L


def augment_dihedral(gram, counts, geom: Geometry, bp: BucketParams, stream=None):
    """Gram sums and counts of the 8 dihedral transforms of the training pairs
    (mdn_augment_dihedral; single-level geometry) -> (gram, counts), new tensors."""
    torch = _torch()
    gout = torch.empty_like(gram)
    cout = torch.empty_like(counts)
    _check(lib().mdn_augment_dihedral(_dev(gram, "gram"), _dev(counts, "counts"), C.byref(geom), C.byref(bp),
                                      _dev(gout, "gram_out"), _dev(cout, "counts_out"), _stream(stream)))
    return gout, cout


def solve_bank(gram, counts, geom: Geometry, lam: float = 1e-3, stream=None):
    """Ridge Cholesky solve on the GPU (mdn_solve_bank) -> (bank, status)."""
    torch = _torch()
    K = gram.shape[0]
    dev = gram.device
    bank = torch.empty((K, 3, regressor_len(geom)), dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    need = lib().mdn_solve_workspace_bytes(C.byref(geom), K)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    _check(lib().mdn_solve_bank(_dev(gram, "gram"), _dev(counts, "counts"), C.byref(geom), K, lam,
                                _dev(bank, "bank"), _dev(status, "status"), _dev(ws, "ws"), need, _stream(stream)))
    return bank, status
