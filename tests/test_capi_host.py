"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every symbol include/mdn.h declares, and rejects bad arguments with the
documented status codes before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1802_06130_gb300 as mdn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mdn.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mdn_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    mdn.build()
    return mdn.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 14
    raw = C.CDLL(mdn.build())
    for n in names:
        assert hasattr(raw, n), n


def test_regressor_lengths(L):
    assert mdn.regressor_len(mdn.Geometry(2, -1)) == 25
    assert mdn.regressor_len(mdn.Geometry(3, 3)) == 98
    assert mdn.regressor_len(mdn.Geometry(3, 2)) == 74
    assert mdn.regressor_len(mdn.Geometry(3, -1, 1)) == 147
    assert mdn.regressor_len(mdn.Geometry(2, 1)) == 34   # the paper's low-noise 5x5 + 3x3
    assert L.mdn_regressor_len(None) == -1


def test_workspace_queries(L):
    # 3 levels of 1080p FP16: z1 + z2 + u1
    b = L.mdn_denoise_workspace_bytes(1, 1080, 1920, 3, mdn.F16)
    assert b >= 3 * 2 * (540 * 960 * 2 + 270 * 480)
    assert L.mdn_pyramid_bytes(2, 7, 5, 1, mdn.F32) == 0
    assert L.mdn_gram_state_bytes(C.byref(mdn.Geometry(3, -1, 1)), 216) == 216 * 150 * 150 * 8
    assert L.mdn_gram_state_bytes(C.byref(mdn.Geometry(3, 3)), 216) == 216 * 3 * 99 * 99 * 8


def test_bad_arguments_rejected_without_device(L):
    g, bp = mdn.Geometry(3, 3), mdn.default_bparams(0)
    rc = L.mdn_filter_level(None, None, 0, 1, 8, 8, None, 0, C.byref(g), C.byref(bp), None, None, None)
    assert rc == 1 and b"null" in L.mdn_last_error()
    bad = mdn.BucketParams(23)
    rc = L.mdn_select_buckets(C.c_void_p(16), 0, 1, 8, 8, C.byref(bad), C.c_void_p(16), None)
    assert rc == 1 and b"n_angle" in L.mdn_last_error()
    rc = L.mdn_build_pyramid(C.c_void_p(16), 0, 1, 8, 8, 9, None, None)
    assert rc == 1
    g2 = mdn.Geometry(3, 3)
    arr = (C.c_void_p * 1)(16)
    parr = (mdn.BucketParams * 1)(bp)
    # levels = 1 requires single-scale geometry
    rc = L.mdn_denoise_multiscale(C.c_void_p(16), 0, 1, 8, 8, 1, arr, 0, C.byref(g2), parr, C.c_void_p(32),
                                  None, None, 0, None)
    assert rc == 2
    # workspace too small
    g1 = mdn.Geometry(3, 3)
    arr2 = (C.c_void_p * 2)(16, 16)
    parr2 = (mdn.BucketParams * 2)(bp, bp)
    rc = L.mdn_denoise_multiscale(C.c_void_p(16), 0, 1, 64, 64, 3, arr2, 0, C.byref(g1), parr2, C.c_void_p(32),
                                  None, C.c_void_p(64), 10, None)
    assert rc == 3 and b"workspace" in L.mdn_last_error()
    rc = L.mdn_filter_level(C.c_void_p(16), None, 0, 1, 8, 8, C.c_void_p(48), 0, C.byref(mdn.Geometry(3, 3)),
                            C.byref(bp), C.c_void_p(32), None, None)
    assert rc == 1 and b"coarse" in L.mdn_last_error()
    rc = L.mdn_filter_level(C.c_void_p(16), None, 0, 1, 8, 8, C.c_void_p(48), 0, C.byref(mdn.Geometry(4, -1)),
                            C.byref(bp), C.c_void_p(32), None, None)
    assert rc == 2
    rc = L.mdn_train_level_filters(C.c_void_p(16), None, C.c_void_p(16), 0, 1, 8, 8, C.byref(mdn.Geometry(2, -1)),
                                   C.byref(bp), 9, 0, C.c_void_p(8), C.c_void_p(8), 1e-3, None, None, 0, None)
    assert rc == 1 and b"precision" in L.mdn_last_error()
    # noise estimate: null, dtype, size, workspace
    rc = L.mdn_estimate_noise(None, 0, 1, 8, 8, C.c_void_p(16), C.c_void_p(32), 1 << 20, None)
    assert rc == 1 and b"null" in L.mdn_last_error()
    rc = L.mdn_estimate_noise(C.c_void_p(16), 7, 1, 8, 8, C.c_void_p(16), C.c_void_p(32), 1 << 20, None)
    assert rc == 1 and b"dtype" in L.mdn_last_error()
    rc = L.mdn_estimate_noise(C.c_void_p(16), 0, 1, 1, 8, C.c_void_p(16), C.c_void_p(32), 1 << 20, None)
    assert rc == 2
    rc = L.mdn_estimate_noise(C.c_void_p(16), 0, 2, 8, 8, C.c_void_p(16), C.c_void_p(32), 100, None)
    assert rc == 3 and b"workspace" in L.mdn_last_error()
    assert L.mdn_noise_workspace_bytes(3) == 3 * 16384 * 4
    # image transforms: null, aliasing, transform index
    rc = L.mdn_dihedral_images(None, 0, 1, 4, 4, 0, C.c_void_p(16), None)
    assert rc == 1 and b"null" in L.mdn_last_error()
    rc = L.mdn_dihedral_images(C.c_void_p(16), 0, 1, 4, 4, 0, C.c_void_p(16), None)
    assert rc == 1 and b"alias" in L.mdn_last_error()
    rc = L.mdn_dihedral_images(C.c_void_p(16), 0, 1, 4, 4, 8, C.c_void_p(32), None)
    assert rc == 1 and b"0..7" in L.mdn_last_error()
    # dihedral augmentation: null, aliasing, multiscale geometry, odd angle count
    g1, bp0 = mdn.Geometry(2, -1), mdn.default_bparams(0)
    rc = L.mdn_augment_dihedral(None, C.c_void_p(16), C.byref(g1), C.byref(bp0), C.c_void_p(32), C.c_void_p(48), None)
    assert rc == 1 and b"null" in L.mdn_last_error()
    rc = L.mdn_augment_dihedral(C.c_void_p(16), C.c_void_p(16), C.byref(g1), C.byref(bp0), C.c_void_p(16),
                                C.c_void_p(48), None)
    assert rc == 1 and b"alias" in L.mdn_last_error()
    rc = L.mdn_augment_dihedral(C.c_void_p(16), C.c_void_p(24), C.byref(mdn.Geometry(3, 3)), C.byref(bp0),
                                C.c_void_p(32), C.c_void_p(48), None)
    assert rc == 2 and b"single-level" in L.mdn_last_error()
    rc = L.mdn_augment_dihedral(C.c_void_p(16), C.c_void_p(24), C.byref(g1), C.byref(mdn.BucketParams(23)),
                                C.c_void_p(32), C.c_void_p(48), None)
    assert rc == 1 and b"n_angle" in L.mdn_last_error()


def test_wide_bucket_grids_host(L):
    """Grids up to 4096 buckets: map element size, limits, workspace."""
    assert [L.mdn_bucket_elem_bytes(k) for k in (0, 1, 216, 256, 257, 4096, 4097)] == [0, 1, 1, 1, 2, 2, 0]
    bp = mdn.paper_grid_bparams(0)
    assert (bp.n_angle, bp.n_strength, bp.n_coherence, bp.K) == (16, 16, 16, 4096)
    too_many = mdn.paper_grid_bparams(0)
    too_many.n_angle = 18                      # 18 x 16 x 16 = 4608 buckets
    rc = L.mdn_select_buckets(C.c_void_p(16), 0, 1, 8, 8, C.byref(too_many), C.c_void_p(16), None)
    assert rc == 1 and b"4096" in L.mdn_last_error()
    bad = mdn.paper_grid_bparams(0)
    bad.n_strength = 18                        # more thresholds than the struct holds
    rc = L.mdn_select_buckets(C.c_void_p(16), 0, 1, 8, 8, C.byref(bad), C.c_void_p(16), None)
    assert rc == 1 and b"1..17" in L.mdn_last_error()
    g = mdn.Geometry(3, 2)
    n, h, w = 2, 64, 48
    wide = L.mdn_train_workspace_bytes(n, h, w, C.byref(g), 4096, mdn.GRAM_TF32)
    narrow = L.mdn_train_workspace_bytes(n, h, w, C.byref(g), 216, mdn.GRAM_TF32)
    assert wide > narrow + n * h * w           # u16 map and 4096-entry sort tables
    assert L.mdn_gram_state_bytes(C.byref(g), 4096) == 4096 * 3 * 75 * 75 * 8
    assert L.mdn_solve_workspace_bytes(C.byref(g), 4096) > 0


def test_paper_grid_parameters_agree_with_the_oracle():
    """The binding's and the oracle's 16 x 16 x 16 thresholds are the same
    numbers (selector parameters, defined on each side)."""
    import oracle as O
    for level in range(4):
        a, b = mdn.paper_grid_bparams(level), O.paper_grid_bparams(level)
        assert a.K == b.K == 4096
        assert np.allclose(list(a.strength_thr)[:15], b.strength_thr, rtol=1e-6)
        assert np.allclose(list(a.coherence_thr)[:15], b.coherence_thr, rtol=1e-6)
        assert all(np.diff(b.strength_thr) > 0) and all(np.diff(b.coherence_thr) > 0)


def test_bucket_map_guard_rejects_wrong_type():
    """The binding checks a caller's bucket map before the library writes
    1 or 2 bytes per pixel into it."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        mdn._map(torch.empty((1, 4, 4), dtype=torch.uint8), 4096, 1, 4, 4, "m")
    with pytest.raises(ValueError):
        mdn._map(torch.empty((1, 4, 4), dtype=torch.int16), 216, 1, 4, 4, "m")
    with pytest.raises(ValueError):
        mdn._map(torch.empty((1, 4, 3), dtype=torch.int16), 4096, 1, 4, 4, "m")


def test_product_path_has_no_oracle_dependency():
    """The package must not import or load anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1802_06130_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower().replace("oracle-free", ""), f


def test_oversized_images_rejected_without_overflow(L):
    """Sizes are bounded factor by factor before any product is formed: an n
    whose n * 3 * h * w wraps a signed 64-bit product to 0 is still rejected
    (and the null-pointer check is not skipped by a wrapped product)."""
    SIZE_MAX = 2 ** 64 - 1
    big = 1 << 20
    n_wrap = 1 << 26                       # 3 * 2^26 * 2^40 wraps int64 to 0... times 3 does not, 2^66 does
    for n, h, w in [(n_wrap, big, big), (1 << 24, big, big), (1, big + 1, 8), (2, 32768, 32768), (-1, 8, 8)]:
        rc = L.mdn_filter_level(None, None, 0, n, h, w, C.c_void_p(48), 0, C.byref(mdn.Geometry(3, -1)),
                                C.byref(mdn.default_bparams(0)), C.c_void_p(32), None, None)
        assert rc == 2, (n, h, w, rc)
        if n >= 0:
            assert L.mdn_denoise_workspace_bytes(n, h, w, 3, mdn.F16) == SIZE_MAX
            assert L.mdn_pyramid_bytes(n, h, w, 3, mdn.F16) == SIZE_MAX
    # the largest accepted batch: n * 3 * h * w = 2^31 - 1 rounded down
    h = w = 1024
    n_max = (2 ** 31 - 1) // (3 * h * w)
    assert L.mdn_denoise_workspace_bytes(n_max, h, w, 3, mdn.F16) < SIZE_MAX
    assert L.mdn_denoise_workspace_bytes(n_max + 1, h, w, 3, mdn.F16) == SIZE_MAX


def test_static_entry_checks_sizes_before_scratch_arithmetic(L):
    """mdn_denoise_multiscale_static validates the image sizes before it
    computes the scratch it would need, so an overflowing size is a shape
    error, not a size that happens to fit the static array."""
    raw = C.CDLL(mdn.build())
    f = raw.mdn_denoise_multiscale_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.POINTER(C.c_void_p),
                  C.c_int32, C.POINTER(mdn.Geometry), C.POINTER(mdn.BucketParams), C.c_void_p,
                  C.POINTER(C.c_void_p), C.c_void_p]
    bp = mdn.default_bparams(0)
    barr = (C.c_void_p * 2)(16, 16)
    parr = (mdn.BucketParams * 2)(bp, bp)
    rc = f(C.c_void_p(16), mdn.F16, 1 << 26, 1 << 20, 1 << 20, 3, barr, mdn.F16, C.byref(mdn.Geometry(3, 3)), parr,
           C.c_void_p(32), None, None)
    assert rc == 2 and b"too large" in L.mdn_last_error()
    rc = f(None, mdn.F16, 1, 64, 64, 3, barr, mdn.F16, C.byref(mdn.Geometry(3, 3)), parr, C.c_void_p(32), None, None)
    assert rc == 1 and b"null" in L.mdn_last_error()


def test_depth_rule_behind_the_c_abi(L):
    """Section 5's depth rule and its noise factors are library calls: exact
    factors of the composed binomial kernels (70/256 at level 1), the level
    counts 1 (sigma already below 2/255), 2, 3, 4, 5 at sigma 1, 5, 15, 25,
    50 (0-255 scale), the clamps, and argument errors."""
    assert L.mdn_pyramid_noise_factor(0) == 1.0
    assert abs(L.mdn_pyramid_noise_factor(1) - 70 / 256) < 1e-15
    # level 2 by hand: c_2 = b * (b upsampled by 2), sum of squares
    b = np.array([1, 4, 6, 4, 1]) / 16
    b2 = np.zeros(9)
    b2[::2] = b
    c2 = np.convolve(b, b2)
    assert abs(L.mdn_pyramid_noise_factor(2) - (c2 ** 2).sum()) < 1e-15
    f = [L.mdn_pyramid_noise_factor(l) for l in range(8)]
    assert all(f[i + 1] < f[i] for i in range(7))
    assert L.mdn_pyramid_noise_factor(8) == -1.0 and L.mdn_pyramid_noise_factor(-1) == -1.0
    got = [L.mdn_levels_for_sigma(s / 255, 2 / 255, 1, 8) for s in (1, 5, 15, 25, 50)]
    assert got == [1, 2, 3, 4, 5]
    assert L.mdn_levels_for_sigma(1 / 255, 2 / 255, 2, 8) == 2
    assert L.mdn_levels_for_sigma(1e6, 2 / 255, 1, 5) == 5
    for bad in [(-1.0, 2 / 255, 1, 8), (0.1, 0.0, 1, 8), (0.1, 2 / 255, 0, 8), (0.1, 2 / 255, 1, 9),
                (0.1, 2 / 255, 5, 4)]:
        assert L.mdn_levels_for_sigma(*bad) == -1
    assert mdn.levels_for_sigma(15 / 255) == 3 and mdn.levels_for_sigma(1 / 255, min_levels=2) == 2
    with pytest.raises(ValueError):
        mdn.pyramid_noise_factor(9)


def test_pipelined_entry_checks_arguments(L):
    """mdn_denoise_multiscale_pipelined rejects a stream count other than 3 or
    4, a zero chunk and a missing stream array before any device work."""
    bp = mdn.default_bparams(0)
    barr = (C.c_void_p * 2)(16, 16)
    parr = (mdn.BucketParams * 2)(bp, bp)
    s3 = (C.c_void_p * 5)(8, 16, 24, 32, 40)
    g = C.byref(mdn.Geometry(3, 3))
    f = L.mdn_denoise_multiscale_pipelined
    rc = f(C.c_void_p(16), 1, 2, 64, 64, 3, barr, 1, g, parr, C.c_void_p(32), 1, C.c_void_p(48), C.c_void_p(64),
           C.c_void_p(80), 1 << 30, s3, 5)
    assert rc == 1 and b"nstreams" in L.mdn_last_error()
    rc = f(C.c_void_p(16), 1, 2, 64, 64, 3, barr, 1, g, parr, C.c_void_p(32), 0, C.c_void_p(48), C.c_void_p(64),
           C.c_void_p(80), 1 << 30, s3, 3)
    assert rc == 1 and b"chunk" in L.mdn_last_error()
    rc = f(C.c_void_p(16), 1, 2, 64, 64, 3, barr, 1, g, parr, C.c_void_p(32), 1, C.c_void_p(48), C.c_void_p(64),
           C.c_void_p(80), 1 << 30, None, 3)
    assert rc == 1 and b"streams" in L.mdn_last_error()
    rc = f(C.c_void_p(16), 1, 2, 64, 64, 3, barr, 1, g, parr, C.c_void_p(32), 1, C.c_void_p(48), C.c_void_p(64),
           C.c_void_p(80), 10, s3, 4)
    assert rc == 3 and b"workspace" in L.mdn_last_error()


def test_prepared_bank_layout_sizes_and_checks(L):
    """mdn_bank_rows_bytes: one 16-byte (FP16) or 32-byte (FP32) slot per
    bucket, output channel, tap block and filter row (2r+1 rows per block; a
    7x7x3 cross-channel filter has three fine blocks per output channel);
    mdn_prepare_bank_rows rejects bad arguments before any device work."""
    cases = [((2, -1), 3 * 5), ((3, 3), 3 * (7 + 7)), ((3, 2), 3 * (7 + 5)), ((3, -1, 1), 3 * 3 * 7),
             ((2, 1), 3 * (3 + 5))]
    for args, slots in cases:
        g = C.byref(mdn.Geometry(*args))
        assert L.mdn_bank_rows_bytes(g, 216, mdn.F16) == 216 * slots * 16
        assert L.mdn_bank_rows_bytes(g, 4096, mdn.F32) == 4096 * slots * 32
        assert L.mdn_bank_rows_bytes(g, 0, mdn.F16) == 0
        assert L.mdn_bank_rows_bytes(g, 4097, mdn.F16) == 0
        assert L.mdn_bank_rows_bytes(g, 216, mdn.F16_ROWS) == 0
    assert L.mdn_bank_rows_bytes(C.byref(mdn.Geometry(1, -1)), 216, mdn.F16) == 0
    assert L.mdn_bank_rows_bytes(None, 216, mdn.F16) == 0
    g = C.byref(mdn.Geometry(3, 3))
    f = L.mdn_prepare_bank_rows
    need = L.mdn_bank_rows_bytes(g, 216, mdn.F16)
    assert f(None, mdn.F16, g, 216, C.c_void_p(256), need, None) == 1
    assert f(C.c_void_p(256), mdn.F16_ROWS, g, 216, C.c_void_p(256), need, None) == 1
    assert f(C.c_void_p(256), mdn.F16, g, 0, C.c_void_p(256), need, None) == 1
    assert f(C.c_void_p(256), mdn.F16, C.byref(mdn.Geometry(1, -1)), 216, C.c_void_p(256), need, None) == 2
    assert f(C.c_void_p(256), mdn.F16, g, 216, C.c_void_p(256), need - 16, None) == 3
    assert f(C.c_void_p(256), mdn.F16, g, 216, C.c_void_p(264), need, None) == 1
    assert b"16-byte" in L.mdn_last_error()


def test_autotune_table_host(L, tmp_path):
    """The autotune table without a device: load, exact and nearest-size
    lookups, server entries, save / reload, malformed files, clear; the tuner
    rejects bad arguments before touching the device."""
    try:
        L.mdn_autotune_clear()
        g = mdn.Geometry(3, 3)
        # level r_fine r_coarse cross dtype bank_elem prepared K size_class variant ms
        p = tmp_path / "t.txt"
        p.write_text("# a comment\n"
                     "level 3 3 0 1 1 0 216 20 2 0.5\n"
                     "level 3 3 0 1 1 0 216 24 3 1.5\n"
                     "level 3 2 0 1 1 1 4096 23 1 0.9\n"
                     "server 3 3 0 1 0.2\n")
        assert L.mdn_autotune_load(str(p).encode()) == 0
        f = L.mdn_autotune_lookup
        assert f(C.byref(g), 216, mdn.F16, mdn.F16, 1, 1024, 1024) == 2      # 2^20 pixels: exact class
        assert f(C.byref(g), 216, mdn.F16, mdn.F16, 8, 3024, 4032) == 3      # 2^26.5: nearest class 24
        assert f(C.byref(g), 216, mdn.F16, mdn.F32, 1, 1024, 1024) == -1     # other bank type: no entry
        assert f(C.byref(mdn.Geometry(3, 2)), 4096, mdn.F16, mdn.F16_ROWS, 1, 3024, 4032) == 1
        assert L.mdn_autotune_server_lookup(C.byref(g), 0) == 1
        assert L.mdn_autotune_server_lookup(C.byref(g), 1) == -1
        q = tmp_path / "saved.txt"
        assert L.mdn_autotune_save(str(q).encode()) == 0
        L.mdn_autotune_clear()
        assert f(C.byref(g), 216, mdn.F16, mdn.F16, 1, 1024, 1024) == -1
        assert L.mdn_autotune_load(str(q).encode()) == 0
        assert f(C.byref(g), 216, mdn.F16, mdn.F16, 1, 1024, 1024) == 2
        assert L.mdn_autotune_server_lookup(C.byref(g), 0) == 1
        bad = tmp_path / "bad.txt"
        bad.write_text("level 3 3 0 1 1 0 216 20 9 0.5\nnonsense\n")     # variant 9 does not exist
        assert L.mdn_autotune_load(str(bad).encode()) == 1
        assert L.mdn_autotune_load(str(tmp_path / "missing.txt").encode()) == 1
        best = C.c_int32()
        ms = (C.c_float * 6)()
        bp = mdn.default_bparams(0)
        t = L.mdn_autotune_level
        assert t(None, C.byref(bp), mdn.F16, mdn.F16, 1, 64, 64, 3, C.byref(best), ms, None) == 1
        assert t(C.byref(g), C.byref(bp), 7, mdn.F16, 1, 64, 64, 3, C.byref(best), ms, None) == 1
        assert t(C.byref(g), C.byref(bp), mdn.F16, mdn.F16, 1, 64, 64, 0, C.byref(best), ms, None) == 1
        assert t(C.byref(g), C.byref(bp), mdn.F16, 9, 1, 64, 64, 3, C.byref(best), ms, None) == 1
        assert t(C.byref(g), C.byref(bp), mdn.F16, mdn.F16, 1, 0, 64, 3, C.byref(best), ms, None) == 2
        assert t(C.byref(mdn.Geometry(1, -1)), C.byref(bp), mdn.F16, mdn.F16, 1, 64, 64, 3, C.byref(best), ms,
                 None) == 2
    finally:
        L.mdn_autotune_clear()


def _desc(dtype, shape, strides=None, data=256):
    t = mdn.Tensor(dtype, len(shape))
    dense = []
    acc = 1
    for e in reversed(shape):
        dense.append(acc)
        acc *= e
    dense = list(reversed(dense))
    for i, e in enumerate(shape):
        t.shape[i] = e
        t.strides[i] = (strides or dense)[i]
    t.data = data
    return t


def test_tensor_descriptors_are_checked_without_device(L):
    """The mdn_t_* forms refuse a wrong dtype, rank, extent or stride with
    MDN_ESHAPE and name the argument, and a null tensor with MDN_EINVAL,
    before any device work."""
    def err():
        return L.mdn_last_error().decode()
    img = _desc(mdn.F16, [2, 3, 64, 48])
    lv = (mdn.Tensor * 2)(_desc(mdn.F16, [2, 3, 32, 24]), _desc(mdn.F16, [2, 3, 16, 12]))
    f = L.mdn_t_build_pyramid
    for bad, word in [(_desc(mdn.U8, [2, 3, 64, 48]), "dtype"), (_desc(mdn.F16, [2, 3, 64]), "rank"),
                      (_desc(mdn.F16, [2, 4, 64, 48]), "extent"),
                      (_desc(mdn.F16, [2, 3, 64, 48], [9216, 3072, 48, 2]), "stride")]:
        assert f(C.byref(bad), 3, lv, None) == 2 and "img" in err() and word in err(), err()
    bad_lv = (mdn.Tensor * 2)(_desc(mdn.F16, [2, 3, 32, 24]), _desc(mdn.F16, [2, 3, 16, 13]))
    assert f(C.byref(img), 3, bad_lv, None) == 2 and "out[1]" in err()
    assert f(C.byref(_desc(mdn.F16, [2, 3, 64, 48], data=None)), 3, lv, None) == 1
    assert f(None, 3, lv, None) == 1
    # a dimension of extent 1 may carry any stride
    one = _desc(mdn.F16, [1, 3, 64, 48], [12345, 3072, 48, 1])
    lv1 = (mdn.Tensor * 1)(_desc(mdn.F32, [1, 3, 32, 24]))
    assert f(C.byref(one), 2, lv1, None) == 2 and "out[0]" in err() and "dtype" in err()

    g, bp = mdn.Geometry(3, 3), mdn.default_bparams(0)
    z, c, out = _desc(mdn.F32, [1, 3, 33, 17]), _desc(mdn.F32, [1, 3, 17, 9]), _desc(mdn.F32, [1, 3, 33, 17])
    t = L.mdn_t_filter_level
    assert t(C.byref(z), C.byref(c), C.byref(_desc(mdn.F16, [216, 3, 74])), C.byref(g), C.byref(bp), C.byref(out),
             None, None) == 2 and "bank" in err()
    assert t(C.byref(z), C.byref(_desc(mdn.F32, [1, 3, 16, 9])), C.byref(_desc(mdn.F16, [216, 3, 98])), C.byref(g),
             C.byref(bp), C.byref(out), None, None) == 2 and "coarse" in err()
    assert t(C.byref(z), C.byref(c), C.byref(_desc(mdn.F16, [216, 3, 98])), C.byref(g), C.byref(bp), C.byref(out),
             C.byref(_desc(mdn.U16, [1, 33, 17])), None) == 2 and "buckets_out" in err()
    rows = L.mdn_bank_rows_bytes(C.byref(g), 216, mdn.F16)
    assert t(C.byref(z), C.byref(c), C.byref(_desc(mdn.F16_ROWS, [rows - 16])), C.byref(g), C.byref(bp),
             C.byref(out), None, None) == 2 and "bank" in err()

    gx = mdn.Geometry(3, -1, 1)   # cross-channel: gram [K][1][D+3][D+3]
    n, cl = _desc(mdn.F32, [1, 3, 33, 17]), _desc(mdn.F32, [1, 3, 33, 17])
    tr = L.mdn_t_train_level_filters
    good_g, good_c = _desc(mdn.F64, [216, 1, 150, 150]), _desc(mdn.I64, [216])
    assert tr(C.byref(n), None, C.byref(cl), C.byref(gx), C.byref(bp), 1, 0, C.byref(_desc(mdn.F64, [216, 3, 150, 150])),
              C.byref(good_c), 1e-3, None, None, 0, None) == 2 and "gram" in err()
    assert tr(C.byref(n), None, C.byref(cl), C.byref(gx), C.byref(bp), 1, 0, C.byref(good_g),
              C.byref(_desc(mdn.F64, [216])), 1e-3, None, None, 0, None) == 2 and "counts" in err()
    assert tr(C.byref(n), None, C.byref(_desc(mdn.F16, [1, 3, 33, 17])), C.byref(gx), C.byref(bp), 1, 0,
              C.byref(good_g), C.byref(good_c), 1e-3, None, None, 0, None) == 2 and "clean_lvl" in err()
