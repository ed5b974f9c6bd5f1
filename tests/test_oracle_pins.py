"""Pins the FP64 oracle to facts that do not come from the oracle itself:
closed forms, library routines (numpy float16, LAPACK eigh/solve/lstsq),
brute force through independently built matrices, invariants, and the
hand-computed fixtures in tests/golden/ (each cites the passage it follows).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _clamp_matrix(n_out, n_in, taps, step, offset):
    """Dense 1-D operator: out[i] = sum_t taps[t] * in[clamp(step*i + t - offset)]."""
    M = np.zeros((n_out, n_in))
    for i in range(n_out):
        for t, w in enumerate(taps):
            j = min(max(step * i + t - offset, 0), n_in - 1)
            M[i, j] += w
    return M


# ------------------------------------------------------------ storage rounding

def test_f16_rounding_matches_numpy():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 3, rng.uniform(-1e-4, 1e-4, 5000),
                        np.array([0.0, -0.0, 65504.0, 65519.0, 1 + 2**-11, 1 + 3 * 2**-11,
                                  2**-24, 2**-25, 3 * 2**-25, 6e-8, 1e-9])])
    got = O.round_storage(x, "f16")
    ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, ref)


def test_f32_rounding_matches_numpy():
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.array_equal(O.round_storage(x, "f32"), x.astype(np.float32).astype(np.float64))


# ------------------------------------------------------------ A1 pyramid

@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (7, 5), (33, 17), (16, 16)])
def test_pyramid_equals_kronecker_operator(H, W):
    """2x binomial downsampling with clamping == (Dy kron Dx) applied to the
    flattened image, both 1-D operators built independently."""
    rng = np.random.default_rng(H * 100 + W)
    img = rng.standard_normal((3, H, W))
    b = np.array([1, 4, 6, 4, 1]) / 16.0
    Dy = _clamp_matrix((H + 1) // 2, H, b, 2, 2)
    Dx = _clamp_matrix((W + 1) // 2, W, b, 2, 2)
    ref = np.stack([Dy @ img[c] @ Dx.T for c in range(3)])
    got = O.pyramid_down(img)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    got32 = O.pyramid_down(img, mirror32=True)
    np.testing.assert_allclose(got32, ref, rtol=0, atol=5e-6)


def test_pyramid_constant_and_ramp():
    img = np.full((3, 20, 31), 0.37)
    np.testing.assert_allclose(O.pyramid_down(img), 0.37, atol=1e-15)
    # interior of a linear ramp maps to the ramp sampled at (2x, 2y)
    yy, xx = np.mgrid[0:40, 0:40].astype(float)
    ramp = np.stack([0.01 * xx - 0.02 * yy + 0.3] * 3)
    d = O.pyramid_down(ramp)
    Y, X = np.mgrid[0:20, 0:20].astype(float)
    exp = 0.01 * 2 * X - 0.02 * 2 * Y + 0.3
    np.testing.assert_allclose(d[0, 1:19, 1:19], exp[1:19, 1:19], atol=1e-14)


def test_pyramid_storage_rounding_is_representable():
    img = np.random.default_rng(2).uniform(0, 1, (3, 15, 9))
    zs = O.pyramid(img, 3, storage="f16")
    assert [z.shape for z in zs] == [(3, 15, 9), (3, 8, 5), (3, 4, 3)]
    for z in zs:
        assert np.array_equal(z, z.astype(np.float16).astype(np.float64))


# ------------------------------------------------------------ A2/A3 selector

def _ramp_image(H, W, grads, offs=(0.2, 0.4, 0.6)):
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    return np.stack([gx * xx + gy * yy + d for (gx, gy), d in zip(grads, offs)])


@pytest.mark.parametrize("mirror32", [False, True])
def test_ramp_closed_form(mirror32):
    """Parallel colour gradients g_c = k_c (gx, gy): T = sum_c g_c g_c^T away
    from the border, l2 = 0, coherence 1, strength = sqrt(sum |g_c|^2),
    orientation = angle(g) + pi/2 (mod pi)."""
    with open(os.path.join(GOLDEN, "ramp_features.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        g = case["grads"]
        img = _ramp_image(24, 24, g)
        T = O.structure_tensor(img, mirror32)
        Txx = sum(a * a for a, _ in g)
        Txy = sum(a * b for a, b in g)
        Tyy = sum(b * b for _, b in g)
        tol = 1e-12 if not mirror32 else 1e-6
        np.testing.assert_allclose(T[0, 3:-3, 3:-3], Txx, atol=tol)
        np.testing.assert_allclose(T[1, 3:-3, 3:-3], Txy, atol=tol)
        np.testing.assert_allclose(T[2, 3:-3, 3:-3], Tyy, atol=tol)
        f = O.features(T, mirror32=mirror32)
        np.testing.assert_allclose(f[1, 3:-3, 3:-3], case["strength"], rtol=1e-6)
        np.testing.assert_allclose(f[2, 3:-3, 3:-3], 1.0, atol=2e-3 if mirror32 else 1e-6)
        np.testing.assert_allclose(f[0, 3:-3, 3:-3], case["theta_over_pi"], atol=1e-6)
        b, _ = O.buckets(f, O.default_bparams(0))
        assert np.all(b[3:-3, 3:-3] == case["bucket"]), (case, np.unique(b[3:-3, 3:-3]))


def test_orientation_rotates_with_image():
    for alpha in np.linspace(0.05, 3.0, 9):
        g = (math.cos(alpha) * 0.05, math.sin(alpha) * 0.05)
        img = _ramp_image(20, 20, [g, g, g])
        f = O.features(O.structure_tensor(img))
        th = ((alpha + math.pi / 2) % math.pi) / math.pi
        np.testing.assert_allclose(f[0, 3:-3, 3:-3], th, atol=1e-9)


def test_edges_and_constant_buckets():
    bp = O.default_bparams(0)
    H = W = 16
    vert = np.zeros((3, H, W)); vert[:, :, 8:] = 1.0      # vertical edge: gradient along x
    horz = np.zeros((3, H, W)); horz[:, 8:, :] = 1.0      # horizontal edge: gradient along y
    bv, _, fv = O.select(vert, bp)
    bh, _, fh = O.select(horz, bp)
    assert np.all(bv[:, 7:9] // 9 == 12)        # theta = pi/2 -> angle bin 12
    assert np.all(bh[7:9, :] // 9 == 0)          # theta = 0    -> angle bin 0
    const = np.full((3, H, W), 0.5)
    bc, _, fc = O.select(const, bp)
    assert np.all(fc[1] == 0) and np.all(fc[2] == 0)
    assert np.all(bc == (12 * 3 + 0) * 3 + 0)


def test_features_match_lapack_eigh():
    z, _ = synth.noisy_pair(40, 40, 7)
    T = O.structure_tensor(z)
    f = O.features(T)
    rng = np.random.default_rng(3)
    for _ in range(200):
        y, x = rng.integers(0, 40, 2)
        M = np.array([[T[0, y, x], T[1, y, x]], [T[1, y, x], T[2, y, x]]])
        w, V = np.linalg.eigh(M)
        l2, l1 = max(w[0], 0), w[1]
        assert abs(f[1, y, x] - math.sqrt(l1)) < 1e-12
        coh = (math.sqrt(l1) - math.sqrt(l2)) / (math.sqrt(l1) + math.sqrt(l2))
        assert abs(f[2, y, x] - coh) < 1e-9
        v = V[:, 0]                                 # minor eigenvector (x, y)
        th = math.atan2(v[1], v[0]) % math.pi
        d = abs(f[0, y, x] * math.pi - th)
        assert min(d, math.pi - d) < 1e-7


def test_tensor_symmetries():
    """Transposing the image swaps Txx/Tyy; mirroring x negates Txy;
    adding a constant leaves T unchanged; scaling by a multiplies T by a^2."""
    z = synth.noisy_pair(24, 30, 11)[0].astype(np.float64)
    T = O.structure_tensor(z)
    Tt = O.structure_tensor(np.ascontiguousarray(z.transpose(0, 2, 1)))
    np.testing.assert_allclose(Tt[0], T[2].T, atol=1e-14)
    np.testing.assert_allclose(Tt[2], T[0].T, atol=1e-14)
    np.testing.assert_allclose(Tt[1], T[1].T, atol=1e-14)
    Tm = O.structure_tensor(np.ascontiguousarray(z[:, :, ::-1]))
    np.testing.assert_allclose(Tm[1], -T[1][:, ::-1], atol=1e-14)
    np.testing.assert_allclose(O.structure_tensor(z + 0.25), T, atol=1e-13)
    np.testing.assert_allclose(O.structure_tensor(3 * z), 9 * T, rtol=1e-12, atol=1e-14)


def test_coherence_range_and_fp32_path_agrees_outside_band():
    z, _ = synth.noisy_pair(64, 64, 13)
    bp = O.default_bparams(0)
    b64, band64, f64 = O.select(z, bp, mirror32=False)
    b32, band32, f32 = O.select(z, bp, mirror32=True)
    assert f64[2].min() >= 0 and f64[2].max() <= 1
    assert f32[2].min() >= 0 and f32[2].max() <= 1 + 1e-7
    mism = (b64 != b32) & ~band64 & ~band32
    assert mism.sum() == 0


def test_fp32_squared_domain_decisions_equal_feature_thresholds():
    """The FP32 bucket decisions (no square roots or divisions: strength and
    coherence thresholds compared in the squared domain on disc^2, lambda1 <
    eps^2 for the zero tensor) equal thresholding the exact FP64 features at
    every tensor whose features are not within 1e-6 of a threshold: random
    PSD tensors spread over the strength and coherence ranges of the
    thresholds (including 24 x 3 x 3, 16 x 5 x 3 and 16 x 16 x 16 grids), the
    zero tensor, isotropic tensors and pure edges."""
    rng = np.random.default_rng(21)
    n = 200000
    ang = rng.uniform(0, np.pi, n)
    l1 = (rng.uniform(0, 0.35, n) * rng.choice([0.125, 0.25, 0.5, 1], n)) ** 2
    l2 = l1 * rng.uniform(0, 1, n) ** rng.choice([1, 3, 8], n)
    ca, sa = np.cos(ang), np.sin(ang)
    a = l1 * ca ** 2 + l2 * sa ** 2
    b = (l1 - l2) * ca * sa
    c = l1 * sa ** 2 + l2 * ca ** 2
    T = np.stack([a, b, c]).astype(np.float32).astype(np.float64)
    T[:, :5] = 0.0                                   # zero tensors
    T[:, 5:10] = np.array([[0.01], [0.0], [0.01]])   # isotropic
    T[:, 10:15] = np.array([[0.02], [0.0], [0.0]])   # pure edges
    T = T.reshape(3, 1, n)
    for bp in [O.default_bparams(0), O.default_bparams(2), O.BucketParams(16, (0.02, 0.05, 0.1, 0.2), (0.2, 0.5)),
               O.paper_grid_bparams(0)]:
        ref, band = O.buckets(O.features(T, bp.coh_eps), bp, band_eps=1e-6)
        got = O.buckets_fp32(T, bp)
        # the angle bin is atan2 on the FP32 pair in both; compare outside the band
        mism = (got != ref) & ~band
        assert mism.sum() == 0, (bp.K, int(mism.sum()))
        assert len(np.unique(ref)) > min(bp.K, 200) // 2


# ------------------------------------------------------------ colour transform

def test_ycbcr_golden_and_roundtrip():
    with open(os.path.join(GOLDEN, "ycbcr_bt601.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        rgb = np.array(case["rgb"], dtype=float).reshape(3, 1, 1)
        w = O.to_work(rgb, 0)[:, 0, 0]
        np.testing.assert_allclose(w, case["ycbcr"], atol=1e-12)
    x = np.random.default_rng(5).uniform(-1, 2, (3, 8, 9))
    np.testing.assert_allclose(O.from_work(O.to_work(x, 0), 0), x, atol=1e-13)
    np.testing.assert_array_equal(O.to_work(x, 1), x)


# ------------------------------------------------------------ A4 filtering

def _delta_bank(K, geom, coarse_center=0.0, fine_center=1.0):
    D = geom.D()
    bank = np.zeros((K, 3, D))
    pf = (2 * geom.r_fine + 1) ** 2
    pc = (2 * geom.r_coarse + 1) ** 2 if geom.r_coarse >= 0 else 0
    for c in range(3):
        cc = c if geom.cross else 0
        if pc:
            bank[:, c, cc * pc + pc // 2] = coarse_center
        off = (3 if geom.cross else 1) * pc
        bank[:, c, off + cc * pf + pf // 2] = fine_center
    return bank


@pytest.mark.parametrize("geom", [O.Geometry(2, -1), O.Geometry(3, 3), O.Geometry(3, 2, cross=1),
                                  O.Geometry(3, 3, color=1)])
def test_delta_filter_is_identity(geom):
    z, _ = synth.noisy_pair(21, 18, 3)
    uc = O.pyramid_down(z)
    bk = np.random.default_rng(0).integers(0, 216, (21, 18)).astype(np.uint8)
    out = O.filter_level(z, uc, bk, _delta_bank(216, geom), geom)
    np.testing.assert_allclose(out, z, atol=1e-13)


def test_coarse_delta_is_nearest_upsampling():
    """f = delta at the coarse centre, g = 0: out_i = u^{l+1}_{floor(i/2)}."""
    geom = O.Geometry(3, 3)
    z = np.zeros((3, 13, 10))
    uc = np.random.default_rng(1).uniform(0, 1, (3, 7, 5))
    bank = _delta_bank(216, geom, coarse_center=1.0, fine_center=0.0)
    out = O.filter_level(z, uc, np.zeros((13, 10), np.uint8), bank, geom)
    ref = uc[:, np.arange(13) // 2][:, :, np.arange(10) // 2]
    np.testing.assert_allclose(out, ref, atol=1e-13)


def test_normalised_bank_preserves_constant():
    geom = O.Geometry(3, 3)
    rng = np.random.default_rng(2)
    bank = rng.standard_normal((216, 3, geom.D()))
    bank /= bank.sum(axis=2, keepdims=True)
    z = np.empty((3, 11, 12)); z[0], z[1], z[2] = 0.2, 0.5, 0.9
    uc = O.pyramid_down(z)
    bk = rng.integers(0, 216, (11, 12)).astype(np.uint8)
    out = O.filter_level(z, uc, bk, bank, geom)
    np.testing.assert_allclose(out, z, atol=1e-10)


def test_one_pixel_image_by_hand():
    """1x1 image: every clamped tap reads the single pixel, so the output in
    working space is (sum of taps) x value."""
    geom = O.Geometry(2, 2)
    rgb = np.array([0.3, 0.6, 0.1]).reshape(3, 1, 1)
    bank = np.zeros((216, 3, geom.D()))
    bank[5, 0, :] = 0.01      # Y: 50 taps x 0.01 = 0.5
    bank[5, 1, :25] = 0.04    # Cb: coarse taps only, 25 x 0.04 = 1.0
    bank[5, 2, 25:] = -0.02   # Cr: fine taps only, 25 x -0.02 = -0.5
    out = O.filter_level(rgb, rgb, np.array([[5]], np.uint8), bank, geom)
    Y = 0.299 * 0.3 + 0.587 * 0.6 + 0.114 * 0.1
    Cb, Cr = (0.1 - Y) / 1.772, (0.3 - Y) / 1.402
    y, cb, cr = 0.5 * Y, 1.0 * Cb, -0.5 * Cr
    R, B = y + 1.402 * cr, y + 1.772 * cb
    G = (y - 0.299 * R - 0.114 * B) / 0.587
    np.testing.assert_allclose(out[:, 0, 0], [R, G, B], atol=1e-14)


def _patches_numpy(img, r):
    """[C][H][W] -> [H][W][C][(2r+1)^2] clamped patches via edge padding."""
    p = np.pad(img, ((0, 0), (r, r), (r, r)), mode="edge")
    H, W = img.shape[1:]
    out = np.empty((H, W, img.shape[0], (2 * r + 1) ** 2))
    k = 0
    for dy in range(2 * r + 1):
        for dx in range(2 * r + 1):
            out[..., k] = p[:, dy:dy + H, dx:dx + W].transpose(1, 2, 0)
            k += 1
    return out


def _ycc(rgb):
    M = np.array([[0.299, 0.587, 0.114],
                  [-0.299 / 1.772, -0.587 / 1.772, (1 - 0.114) / 1.772],
                  [(1 - 0.299) / 1.402, -0.587 / 1.402, -0.114 / 1.402]])
    return np.einsum("ij,jhw->ihw", M, rgb), np.linalg.inv(M)


def test_filter_brute_force_multiscale():
    """Brute force of the multiscale equation on a 9x8 image: explicit patch
    tensors from edge padding, YCbCr by the BT.601 matrix and its inverse."""
    rng = np.random.default_rng(4)
    geom = O.Geometry(3, 2)
    z = rng.uniform(0, 1, (3, 9, 8))
    uc = rng.uniform(0, 1, (3, 5, 4))
    bk = rng.integers(0, 216, (9, 8)).astype(np.uint8)
    bank = rng.standard_normal((216, 3, geom.D())) * 0.05
    zw, Minv = _ycc(z)
    uw, _ = _ycc(uc)
    Pz = _patches_numpy(zw, 3)                     # [9][8][3][49]
    Pu = _patches_numpy(uw, 2)                     # [5][4][3][25]
    ow = np.zeros((3, 9, 8))
    for y in range(9):
        for x in range(8):
            h = bank[bk[y, x]]
            for c in range(3):
                ow[c, y, x] = h[c, :25] @ Pu[y // 2, x // 2, c] + h[c, 25:] @ Pz[y, x, c]
    ref = np.einsum("ij,jhw->ihw", Minv, ow)
    out = O.filter_level(z, uc, bk, bank, geom)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_filter_brute_force_single_scale_cross_channel():
    rng = np.random.default_rng(6)
    geom = O.Geometry(2, -1, cross=1, color=1)
    z = rng.uniform(0, 1, (3, 8, 8))
    bk = rng.integers(0, 216, (8, 8)).astype(np.uint8)
    bank = rng.standard_normal((216, 3, geom.D()))
    Pz = _patches_numpy(z, 2).reshape(8, 8, 75)    # channel-major (c, dy, dx)
    ref = np.einsum("hwcd,hwd->chw", bank[bk], Pz)
    np.testing.assert_allclose(O.filter_level(z, None, bk, bank, geom), ref, atol=1e-12)


# ------------------------------------------------------------ A5/A6 training

def test_cholesky_matches_lapack():
    rng = np.random.default_rng(8)
    for n in (1, 5, 49, 147):
        A = rng.standard_normal((n, n + 3))
        A = A @ A.T + 1e-3 * np.eye(n)
        B = rng.standard_normal((n, 3))
        np.testing.assert_allclose(O.cholesky_solve(A, B), np.linalg.solve(A, B),
                                   rtol=1e-9, atol=1e-9 * np.abs(np.linalg.solve(A, B)).max())


def test_gram_path_equals_lstsq():
    """Per bucket, the ridge solution from the accumulated Gram equals the
    LAPACK least-squares solution of the stacked system [X; sqrt(n lam) I] h
    = [y; 0], X built from numpy patch tensors."""
    rng = np.random.default_rng(9)
    geom = O.Geometry(2, -1)
    z, u = synth.noisy_pair(32, 32, 21)
    bk = rng.integers(0, 4, (32, 32)).astype(np.uint8)
    lam = 1e-3
    gram, counts = O.gram_accumulate(z, None, u, bk, 4, geom)
    bank = O.solve_bank(gram, counts, geom, lam)
    zw, _ = _ycc(z)
    uw, _ = _ycc(u)
    P = _patches_numpy(zw, 2)
    for k in range(4):
        m = bk == k
        n = m.sum()
        assert counts[k] == n
        for c in range(3):
            X = P[m][:, c, :]
            y = uw[c][m]
            A = np.vstack([X, math.sqrt(n * lam) * np.eye(25)])
            rhs = np.concatenate([y, np.zeros(25)])
            h = np.linalg.lstsq(A, rhs, rcond=None)[0]
            np.testing.assert_allclose(bank[k, c], h, rtol=1e-8, atol=1e-10)


def _ridge_lstsq(X, Y, lam):
    """LAPACK least squares of the stacked ridge system [X; sqrt(n lam) I] h =
    [Y; 0] (n = rows of X), the normalised ridge of reading 12."""
    n, D = X.shape
    A = np.vstack([X, math.sqrt(n * lam) * np.eye(D)])
    rhs = np.concatenate([Y, np.zeros((D,) + Y.shape[1:])])
    return np.linalg.lstsq(A, rhs, rcond=None)[0]


@pytest.mark.parametrize("cross", [0, 1])
def test_empty_buckets_take_pooled_ridge_solution(cross):
    """Reading 13 (the paper is silent on empty buckets): a bucket with no
    pixels takes the pooled filter, the ridge solution over every pixel of the
    level, (sum_k G_k / N + lam I) h = sum_k b_k / N with N = sum_k n_k.  It
    equals LAPACK lstsq of all pixels' stacked patches, whichever buckets they
    fall in; buckets 0..2 of 6 are used, 3..5 are empty."""
    rng = np.random.default_rng(19)
    geom = O.Geometry(2, -1, cross=cross)
    z, u = synth.noisy_pair(30, 34, 23)
    bk = rng.integers(0, 3, (30, 34)).astype(np.uint8)
    lam = 2e-3
    gram, counts = O.gram_accumulate(z, None, u, bk, 6, geom)
    assert list(counts[3:]) == [0, 0, 0] and counts.sum() == 30 * 34
    bank = O.solve_bank(gram, counts, geom, lam)
    zw, _ = _ycc(z)
    uw, _ = _ycc(u)
    P = _patches_numpy(zw, 2).reshape(30 * 34, 3, 25)
    Y = uw.reshape(3, -1).T
    if cross:
        pooled = _ridge_lstsq(P.reshape(-1, 75), Y, lam).T        # [3][75]
    else:
        pooled = np.stack([_ridge_lstsq(P[:, c, :], Y[:, c], lam) for c in range(3)])
    for k in (3, 4, 5):
        np.testing.assert_allclose(bank[k], pooled, rtol=1e-8, atol=1e-10)
    # a used bucket keeps its own solution, not the pooled one
    assert np.abs(bank[0] - pooled).max() > 1e-3


def _filter_numpy(zw, uw, bk, bank, rf, rc):
    """Brute force of the multiscale equation in working space ([C][H][W]
    arrays, per-channel regressors: coarse patch at floor(i/2), then fine)."""
    H, W = zw.shape[1:]
    Pz = _patches_numpy(zw, rf)
    Pu = _patches_numpy(uw, rc)
    pc = (2 * rc + 1) ** 2
    out = np.zeros_like(zw)
    for y in range(H):
        for x in range(W):
            h = bank[bk[y, x]]
            for c in range(3):
                out[c, y, x] = h[c, :pc] @ Pu[y // 2, x // 2, c] + h[c, pc:] @ Pz[y, x, c]
    return out


def test_cascade_feeds_trained_coarser_output():
    """Section 4's training cascade: level l regresses on the output u-hat^{l+1}
    of the coarser level trained just before it, not on z^{l+1} or on the
    clean target of level l+1.  Planted construction, lambda = 0, 3 levels:
    level 1's target t1 is an arbitrary image, so its least-squares fit B1
    (computed here with LAPACK) leaves a residual and u-hat^1 = B1 applied to
    (z^2, z^1) differs from t1 and from z^1; level 0's target is a planted
    bank P0 applied to (u-hat^1, z^0), computed here by brute force.  The
    cascade must give B1 and recover P0; feeding z^1 or t1 to level 0 leaves
    P0 outside the span of the regressors."""
    rng = np.random.default_rng(77)
    geom = O.Geometry(1, 1)                                  # D = 9 + 9 per channel
    bps = [O.BucketParams(n_angle=2, strength_thr=(), coherence_thr=()) for _ in range(2)]
    z, _ = synth.noisy_pair(64, 60, 91)
    zs = O.pyramid(z, 3)
    t1 = rng.uniform(0, 1, zs[1].shape)
    b1, _, _ = O.select(zs[1], bps[1])
    b0, _, _ = O.select(zs[0], bps[0])
    assert set(np.unique(b1)) == {0, 1} and set(np.unique(b0)) == {0, 1}
    # level 1 by LAPACK: per bucket and working channel, [coarse z^2 ; fine z^1] -> t1
    zw1, Minv = _ycc(zs[1])
    zw2, _ = _ycc(zs[2])
    tw1, _ = _ycc(t1)
    Pz, Pu = _patches_numpy(zw1, 1), _patches_numpy(zw2, 1)
    H1, W1 = zs[1].shape[1:]
    yy, xx = np.mgrid[0:H1, 0:W1]
    Xall = np.concatenate([Pu[yy // 2, xx // 2], Pz], axis=3)   # [H1][W1][3][18]
    B1 = np.zeros((2, 3, 18))
    for k in range(2):
        m = b1 == k
        for c in range(3):
            B1[k, c] = np.linalg.lstsq(Xall[m][:, c, :], tw1[c][m], rcond=None)[0]
    uhat1_w = np.einsum("hwcd,hwcd->chw", B1[b1], Xall)
    uhat1 = np.einsum("ij,jhw->ihw", Minv, uhat1_w)
    assert np.abs(uhat1 - t1).max() > 0.1 and np.abs(uhat1 - zs[1]).max() > 0.1
    # level 0: planted bank on (u-hat^1, z^0)
    P0 = rng.standard_normal((2, 3, 18)) * 0.1
    zw0, _ = _ycc(zs[0])
    t0 = np.einsum("ij,jhw->ihw", Minv, _filter_numpy(zw0, uhat1_w, b0, P0, 1, 1))
    banks, counts = O.train_cascade([z], None, geom, 3, bparams=bps, lam=0.0,
                                    level_targets=[[t0, t1, zs[2]]])
    np.testing.assert_allclose(banks[1], B1, rtol=1e-8, atol=1e-10)
    err = np.linalg.norm(banks[0] - P0) / np.linalg.norm(P0)
    assert err < 1e-8, err
    assert list(counts[0]) == [int((b0 == k).sum()) for k in range(2)]


@pytest.mark.parametrize("geom", [O.Geometry(2, -1), O.Geometry(3, 3), O.Geometry(3, -1, cross=1)])
def test_planted_bank_recovered(geom):
    """Noise-free targets made by a planted bank (selector computed on z) are
    fitted exactly by least squares with lambda = 0 (Eqs. 5-6)."""
    rng = np.random.default_rng(10)
    z, _ = synth.noisy_pair(160, 160, 31)
    uc = O.pyramid_down(z) if geom.r_coarse >= 0 else None
    bp = O.default_bparams(0)
    bk, _, _ = O.select(z, bp)
    planted = rng.standard_normal((216, 3, geom.D())) * 0.05
    target = O.filter_level(z, uc, bk, planted, geom)
    gram, counts = O.gram_accumulate(z, uc, target, bk, 216, geom)
    D = geom.D()
    checked = 0
    Gn = gram.shape[1]
    for k in range(216):
        if counts[k] < 4 * D:
            continue
        for g in range(Gn):
            A = gram[k, g, :D, :D]
            if np.linalg.cond(A) > 1e8:
                continue
            B = gram[k, g, :D, D:]
            h = O.cholesky_solve(A, B)
            ref = planted[k].T[:, :] if geom.cross else planted[k, g][:, None]
            err = np.linalg.norm(h - ref) / np.linalg.norm(ref)
            assert err < 1e-10, (k, g, err)
            checked += 1
    assert checked >= 5


def test_wide_grid_bucket_decomposition():
    """The 16 x 16 x 16 map is (a * 16 + s) * 16 + c with a, s and c each taken
    from a grid that bins that feature alone; values above 255 survive (u16)."""
    z, _ = synth.noisy_pair(96, 80, 61)
    bp = O.paper_grid_bparams(0)
    full, _, _ = O.select(z, bp)
    assert full.dtype == np.uint16 and full.max() > 255
    a, _, _ = O.select(z, O.BucketParams(16, (), ()))
    s, _, _ = O.select(z, O.BucketParams(16, bp.strength_thr, ()))
    c, _, _ = O.select(z, O.BucketParams(16, (), bp.coherence_thr))
    a = a.astype(np.int64)
    s = s.astype(np.int64) - 16 * a
    c = c.astype(np.int64) - 16 * a
    assert s.min() >= 0 and s.max() <= 15 and c.min() >= 0 and c.max() <= 15
    assert np.array_equal(full.astype(np.int64), (a * 16 + s) * 16 + c)


def test_planted_bank_recovered_above_256_buckets():
    """Buckets numbered above 255 (4096-bucket bank, 7x7 + 5x5 taps): targets
    made by a planted bank are fitted exactly at those buckets, so the filter
    and the Gram sums index the same bank rows."""
    rng = np.random.default_rng(12)
    geom = O.Geometry(3, 2)
    z, _ = synth.noisy_pair(96, 96, 33)
    uc = O.pyramid_down(z)
    used = np.array([7, 300, 1000, 4095])
    bk = used[rng.integers(0, 4, (96, 96))].astype(np.uint16)
    planted = rng.standard_normal((4096, 3, geom.D())) * 0.05
    target = O.filter_level(z, uc, bk, planted, geom)
    gram, counts = O.gram_accumulate(z, uc, target, bk, 4096, geom)
    assert set(np.flatnonzero(counts)) == set(used)
    D = geom.D()
    for k in used:
        for g in range(3):
            h = O.cholesky_solve(gram[k, g, :D, :D], gram[k, g, :D, D:])
            err = np.linalg.norm(h[:, 0] - planted[k, g]) / np.linalg.norm(planted[k, g])
            assert err < 1e-8, (k, g, err)


def test_cascade_with_identity_banks_returns_input():
    geom = O.Geometry(3, 3)
    z, _ = synth.noisy_pair(30, 26, 41)
    banks = [_delta_bank(216, geom), _delta_bank(216, geom)]
    r = O.denoise_multiscale(z, banks, geom)
    np.testing.assert_allclose(r.out, z, atol=1e-13)
    assert len(r.pyramid) == 3 and r.pyramid[2].shape == (3, 8, 7)


def test_training_reduces_error_single_level():
    """Sanity: a bank trained on 4 pairs denoises a held-out image."""
    geom = O.Geometry(2, -1)
    pairs = [synth.noisy_pair(64, 64, 1000 + i) for i in range(4)]
    banks, _ = O.train_cascade([p[0] for p in pairs], [p[1] for p in pairs], geom, 1)
    z, u = synth.noisy_pair(64, 64, 2000)
    out = O.denoise_multiscale(z, banks, geom).out
    assert np.mean((out - u) ** 2) < 0.3 * np.mean((z - u) ** 2)


# ------------------------------------------------------------ dihedral augmentation

def test_dihedral_group_and_bucket_map():
    """Section 5 augments the training pairs by flips and 90-degree rotations.
    The 8 transforms are the dihedral group (distinct, rot^4 = id, mirror^2 =
    id), and the structure tensor turns with the image: the selector on a
    transformed image equals the transformed, angle-remapped map of the
    original (bin + n/2 per quarter turn, n - 1 - a under the mirror) at every
    pixel outside the threshold band of either image."""
    idx = np.arange(35).reshape(1, 5, 7)
    assert len({O.dihedral(idx, t).tobytes() for t in range(8)}) == 8
    r = idx
    for _ in range(4):
        r = O.dihedral(r, 1)
    assert np.array_equal(r, idx)
    assert np.array_equal(O.dihedral(O.dihedral(idx, 4), 4), idx)
    z, _ = synth.noisy_pair(64, 48, 11)
    bp = O.default_bparams(0)
    b, band, _ = O.select(z, bp, mirror32=True)
    for t in range(8):
        bt, bandt, _ = O.select(O.dihedral(z, t), bp, mirror32=True)
        keep = ~(bandt | O.dihedral(band.astype(np.uint8)[None], t)[0].astype(bool))
        assert keep.mean() > 0.98
        assert np.array_equal(bt[keep], O.dihedral_bucket(b, t, bp)[keep]), t


@pytest.mark.parametrize("geom", [O.Geometry(2, -1), O.Geometry(1, -1, cross=1)], ids=["5x5", "3x3x3"])
def test_dihedral_gram_is_permuted_gram(geom):
    """Materialising the 8 transformed pairs (with the selector map carried
    along) gives per-bucket Gram sums that are the original sums with taps
    permuted by the transform of the (2r+1)^2 index grid and buckets moved by
    the angle remap; targets (and the channel order) stay in place."""
    z, u = synth.noisy_pair(24, 20, 12)
    bp = O.default_bparams(0)
    b, _, _ = O.select(z, bp, mirror32=True)
    K = 216
    g_aug, c_aug = O.gram_accumulate_dihedral(z, u, b, K, geom, bp)
    g, c = O.gram_accumulate(z, None, u, b, K, geom)
    n = 2 * geom.r_fine + 1
    D = geom.D()
    nch = 3 if geom.cross else 1
    exp = np.zeros_like(g)
    cexp = np.zeros_like(c)
    for t in range(8):
        tap = O.dihedral(np.arange(n * n).reshape(1, n, n), t)[0].ravel()
        fmap = np.concatenate([np.concatenate([ch * n * n + tap for ch in range(nch)]),
                               np.arange(D, g.shape[-1])])
        for k in range(K):
            kp = int(O.dihedral_bucket(np.array([[k]], dtype=np.uint8), t, bp)[0, 0])
            exp[kp] += g[k][:, fmap][:, :, fmap]
            cexp[kp] += c[k]
    assert np.array_equal(c_aug, cexp)
    np.testing.assert_allclose(g_aug, exp, rtol=1e-12, atol=1e-10)


def test_awgn8_model_is_8bit():
    """Section 5's noisy 8-bit training images: AWGN on the 8-bit clean image,
    then 8-bit quantisation with clamping; the same noise draw as "awgn"."""
    z, u = synth.noisy_pair(32, 24, 5, model="awgn8")
    for a in (z, u):
        assert a.min() >= 0.0 and a.max() <= 1.0
        assert np.abs(a * 255.0 - np.rint(a * 255.0)).max() < 1e-4
    zf, _ = synth.noisy_pair(32, 24, 5)
    assert np.abs(z - np.clip(zf, 0.0, 1.0)).max() <= 1.0 / 255.0 + 1e-6
    assert (z == 0.0).any() or (z == 1.0).any()   # sigma 25/255 reaches the clamp


# ------------------------------------------------------------ noise level

def test_noise_estimate_on_pure_noise():
    """On a constant image plus AWGN the diagonal Haar details are N(0, sigma^2)
    samples, so the robust estimate recovers sigma (12,288 samples: the
    median's standard error is about 1.1 %); it scales exactly with the noise
    and ignores a constant offset and a linear ramp (their d is 0)."""
    rng = np.random.default_rng(3)
    noise = rng.standard_normal((3, 128, 128))
    for s in (15 / 255, 25 / 255, 50 / 255):
        est = O.estimate_noise(0.5 + s * noise)
        assert abs(est - s) < 0.035 * s, (est, s)
    base = O.estimate_noise(noise)
    assert abs(O.estimate_noise(3.0 * noise) - 3.0 * base) < 1e-12
    yy, xx = np.mgrid[0:128, 0:128]
    ramp = 0.002 * xx + 0.003 * yy
    assert abs(O.estimate_noise(noise + ramp[None]) - base) < 1e-9
    assert O.estimate_noise(np.ones((3, 9, 7))) == 0.0


def test_pyramid_noise_factor_and_level_count():
    """The noise of the oracle's pyramid of pure AWGN (measured away from the
    clamped border) falls by the composed-kernel factors the depth rule uses
    (70/256 at level 1, then about 0.45, 0.49, 0.5 per level: the noise is no
    longer white after the first level), and the rule of Section 5 (coarsest
    sigma below 2/255) gives 2 levels at sigma 5, 3 at 15, 4 at 25 and 5 at 50
    (on the 0-255 scale).  The factors and the rule are the library's
    (mdn_pyramid_noise_factor, mdn_levels_for_sigma; host arithmetic)."""
    import paper_1802_06130_gb300 as mdn
    mdn.build()
    assert mdn.pyramid_noise_factor(0) == 1.0
    assert abs(mdn.pyramid_noise_factor(1) - 70 / 256) < 1e-15
    n = np.random.default_rng(5).standard_normal((3, 1024, 1024)) * 0.1
    zs = O.pyramid(n, 4)
    s0 = n[:, 16:-16, 16:-16].std()
    for l in (1, 2, 3):
        e = 16 >> l
        ratio = zs[l][:, e:-e, e:-e].std() / s0
        assert abs(ratio / mdn.pyramid_noise_factor(l) - 1) < 0.02, (l, ratio)
    assert [mdn.levels_for_sigma(s / 255) for s in (1, 5, 15, 25, 50)] == [1, 2, 3, 4, 5]
    assert mdn.levels_for_sigma(1 / 255, min_levels=2) == 2 and mdn.levels_for_sigma(1e6, max_levels=5) == 5


# ------------------------------------------------------------ phase-aware coarse patch (next row f1)

def test_aligned_coarse_patch_upsamples_a_ramp_exactly():
    """The half-pixel-aligned coarse term (coarse patch sampled bilinearly at
    i/2; coarse pixel (Y, X) sits at fine (2Y, 2X)) with a coarse delta bank
    reproduces a linear ramp u(Y, X) = a + bX + cY at fine resolution,
    a + b x/2 + c y/2, away from the clamped right and bottom edges; the
    floor(i/2) coarse term gives the staircase a + b floor(x/2) + c floor(y/2)."""
    Hc, Wc, H, W = 9, 11, 17, 21
    Y, X = np.mgrid[0:Hc, 0:Wc].astype(np.float64)
    coef = [(0.1, 0.02, 0.03), (0.5, -0.01, 0.04), (0.3, 0.05, -0.02)]
    uc = np.stack([a + b * X + c * Y for a, b, c in coef])
    z = np.zeros((3, H, W))
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    for align, yy, xx in [(1, y / 2, x / 2), (0, np.floor(y / 2), np.floor(x / 2))]:
        geom = O.Geometry(1, 1, color=1, align=align)
        bank = _delta_bank(216, geom, coarse_center=1.0, fine_center=0.0)
        out = O.filter_level(z, uc, np.zeros((H, W), np.uint8), bank, geom)
        ref = np.stack([a + b * xx + c * yy for a, b, c in coef])
        np.testing.assert_allclose(out[:, :H - 1, :W - 1], ref[:, :H - 1, :W - 1], atol=1e-13)


def test_aligned_coarse_patch_brute_force():
    """Brute force of the aligned multiscale equation on a 9x8 image: coarse
    patches from the mean of edge-padded shifted copies (two rows or columns
    at odd fine coordinates), fine patches as before; and at even-even pixels
    the aligned and floor(i/2) terms coincide."""
    rng = np.random.default_rng(14)
    geom = O.Geometry(3, 2, align=1)
    z = rng.uniform(0, 1, (3, 9, 8))
    uc = rng.uniform(0, 1, (3, 5, 4))
    bk = rng.integers(0, 216, (9, 8)).astype(np.uint8)
    bank = rng.standard_normal((216, 3, geom.D())) * 0.05
    zw, Minv = _ycc(z)
    uw, _ = _ycc(uc)
    Pz = _patches_numpy(zw, 3)
    # patches at integer coarse positions 0..Hc (0..Wc): the image gains one
    # edge-replicated row and column, so that every sample is clamped on its own
    Pu = _patches_numpy(np.pad(uw, ((0, 0), (0, 1), (0, 1)), mode="edge"), 2)
    ow = np.zeros((3, 9, 8))
    for yy in range(9):
        for xx in range(8):
            ys = [yy // 2, yy // 2 + 1] if yy % 2 else [yy // 2]
            xs = [xx // 2, xx // 2 + 1] if xx % 2 else [xx // 2]
            pu = np.mean([Pu[a, b] for a in ys for b in xs], axis=0)
            h = bank[bk[yy, xx]]
            for c in range(3):
                ow[c, yy, xx] = h[c, :25] @ pu[c] + h[c, 25:] @ Pz[yy, xx, c]
    ref = np.einsum("ij,jhw->ihw", Minv, ow)
    out = O.filter_level(z, uc, bk, bank, geom)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    floor = O.filter_level(z, uc, bk, bank, O.Geometry(3, 2, align=0))
    np.testing.assert_array_equal(out[:, ::2, ::2], floor[:, ::2, ::2])
    assert np.abs(out[:, 1::2, 1::2] - floor[:, 1::2, 1::2]).max() > 1e-3


def test_aligned_planted_bank_recovered():
    """Least squares with the aligned coarse regressor (lambda = 0) recovers a
    planted bank exactly: the Gram sums and the filter use the same samples."""
    rng = np.random.default_rng(16)
    geom = O.Geometry(2, 2, align=1)
    z, _ = synth.noisy_pair(128, 120, 35)
    uc = O.pyramid_down(z)
    bk, _, _ = O.select(z, O.default_bparams(0))
    planted = rng.standard_normal((216, 3, geom.D())) * 0.05
    target = O.filter_level(z, uc, bk, planted, geom)
    gram, counts = O.gram_accumulate(z, uc, target, bk, 216, geom)
    D = geom.D()
    checked = 0
    for k in range(216):
        if counts[k] < 4 * D:
            continue
        for g in range(3):
            A = gram[k, g, :D, :D]
            if np.linalg.cond(A) > 1e8:
                continue
            h = O.cholesky_solve(A, gram[k, g, :D, D:])[:, 0]
            assert np.linalg.norm(h - planted[k, g]) / np.linalg.norm(planted[k, g]) < 1e-8, (k, g)
            checked += 1
    assert checked >= 5


def test_phase_study_aligned_vs_floor_coarse_term(capsys):
    """Measurement behind the decision on the phase-aware coarse term (the
    numbers are printed; run with -s): a 2-level 7x7 + 7x7 cascade trained by
    the oracle on 4 synthetic 192x192 pairs at sigma 25/255 with the floor(i/2)
    and the half-pixel-aligned coarse patch, PSNR on 2 held-out frames.  The
    assertions are sanity only (both denoise by more than 6 dB)."""
    pairs = [synth.noisy_pair(192, 192, 3000 + i) for i in range(4)]
    tests = [synth.noisy_pair(192, 192, 3100 + i) for i in range(2)]
    res = {}
    for align in (0, 1):
        geom = O.Geometry(3, 3, align=align)
        banks, _ = O.train_cascade([p[0] for p in pairs], [p[1] for p in pairs], geom, 2)
        ps = []
        for z, u in tests:
            out = O.denoise_multiscale(z, banks, geom).out
            ps.append((10 * np.log10(1 / np.mean((z - u) ** 2)), 10 * np.log10(1 / np.mean((out - u) ** 2))))
        res[align] = np.mean(ps, axis=0)
    with capsys.disabled():
        print(f"\nphase study: noisy {res[0][0]:.2f} dB, floor(i/2) {res[0][1]:.2f} dB, aligned {res[1][1]:.2f} dB "
              f"(delta {res[1][1] - res[0][1]:+.3f} dB)")
    assert res[0][1] > res[0][0] + 6 and res[1][1] > res[1][0] + 6
