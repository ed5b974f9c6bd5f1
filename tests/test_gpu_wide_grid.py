"""The paper's own selector grid (Section 5): 16 angle x 16 strength x 16
coherence = 4096 buckets, with 7x7 fine + 5x5 coarse taps, through the C ABI
vs the FP64 oracle.  Above 256 buckets the bucket maps are u16, the bank is
read through L2 instead of shared memory, and the sort and Gram reduction run
over 4096 bucket runs.  Bars as in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle as O
import synth
from parity_util import affected_mask, max_abs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f16": 2e-3}
GEOM = O.Geometry(3, 2)          # the paper's 7x7 fine + 5x5 coarse, D = 74
K = 4096


@pytest.fixture(scope="module")
def mdn():
    import paper_1802_06130_gb300 as m
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.build()
    m.lib()
    return m


def _tt(a, storage):
    dt = torch.float32 if storage == "f32" else torch.float16
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _geom(m, g):
    return m.Geometry(g.r_fine, g.r_coarse, g.cross, g.color)


def _gbp(m, bp):
    """The library's parameters with the oracle's thresholds."""
    return m.BucketParams(bp.n_angle, tuple(bp.strength_thr), tuple(bp.coherence_thr), bp.coh_eps)


def _map(t):
    return t.cpu().numpy().astype(np.int64)


def _bank(geom, seed, storage):
    """Random bank whose taps sum to ~1 per output channel."""
    rng = np.random.default_rng(seed)
    D = geom.D()
    b = rng.standard_normal((K, 3, D)) * 0.05
    b += (1.0 - b.sum(axis=2, keepdims=True)) / D
    return O.round_storage(b, storage)


# ------------------------------------------------------------ A2/A3

@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("hw", [(1, 1), (7, 5), (33, 17), (131, 97), (256, 256)])
def test_wide_buckets_bit_exact_outside_band(mdn, storage, hw):
    h, w = hw
    z, _ = synth.noisy_pair(h, w, 5200 + w)
    zs = O.round_storage(z, storage)
    for level in (0, 1, 3):
        bp = O.paper_grid_bparams(level)
        assert bp.K == K
        ref, band, _ = O.select(zs, bp, mirror32=True)
        got_t = mdn.select_buckets(_tt(zs, storage)[None], _gbp(mdn, bp))[0]
        assert got_t.dtype == torch.int16
        got = _map(got_t)
        mism = got != ref.astype(np.int64)
        assert not (mism & ~band).any(), f"{(mism & ~band).sum()} mismatches outside the band"
        if h * w >= 4096:
            assert band.mean() < 0.01
            assert got.max() > 255          # values above the u8 range are exercised


def test_wide_buckets_spread_over_the_grid(mdn):
    """Equal-population thresholds: on the set they were taken from, every
    strength and coherence bin is populated and most of the 4096 buckets
    are hit."""
    seen = []
    for i in range(8):
        z, _ = synth.noisy_pair(256, 256, 1000 + i)
        seen.append(_map(mdn.select_buckets(_tt(z, "f32")[None], mdn.paper_grid_bparams(0))).ravel())
    b = np.concatenate(seen)
    s_bins = np.bincount((b // 16) % 16, minlength=16)
    c_bins = np.bincount(b % 16, minlength=16)
    assert (s_bins > 0.03 * b.size).all(), s_bins
    assert (c_bins > 0.03 * b.size).all(), c_bins
    assert len(np.unique(b)) > 2000


# ------------------------------------------------------------ A4

@pytest.mark.parametrize("prepared", [False, True], ids=["plain_bank", "prepared_bank"])
@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("bank_storage", ["f32", "f16"])
@pytest.mark.parametrize("geom", [GEOM, O.Geometry(2, -1)], ids=["7x7+5x5", "5x5"])
@pytest.mark.parametrize("hw", [(1, 1), (33, 17), (97, 130), (200, 300)])
def test_wide_filter_level(mdn, storage, bank_storage, geom, hw, prepared):
    """Plain banks run the tile kernel (taps through L2); prepared banks
    (mdn_prepare_bank_rows) run the fused kernel reading row slots through L2."""
    h, w = hw
    z, _ = synth.noisy_pair(h, w, 5300 + h * w)
    zs = O.round_storage(z, storage)
    hc, wc = (h + 1) // 2, (w + 1) // 2
    uc = O.round_storage(synth.clean_image(hc, wc, 5400 + h), storage) if geom.r_coarse >= 0 else None
    bank = _bank(geom, 11, bank_storage)
    bp = O.paper_grid_bparams(0)
    ref_b, band, _ = O.select(zs, bp, mirror32=True)
    ref = O.round_storage(O.filter_level(zs, uc, ref_b, bank, geom), storage)
    bmap = torch.empty((1, h, w), dtype=torch.int16, device="cuda")
    dbank = _tt(bank, bank_storage).contiguous()
    if prepared:
        dbank = mdn.prepare_bank(dbank, _geom(mdn, geom))
    out = mdn.filter_level(_tt(zs, storage)[None], _tt(uc, storage)[None] if uc is not None else None,
                           dbank, _geom(mdn, geom), _gbp(mdn, bp), buckets_out=bmap)
    mism = _map(bmap[0]) != ref_b.astype(np.int64)
    assert not (mism & ~band).any()
    err = max_abs(_np(out[0]), ref, ~mism)
    assert err <= TOL[storage], err


def test_wide_bucket_map_type_is_checked(mdn):
    """A u8 map for a 4096-bucket grid would be overrun by the u16 writes:
    the binding refuses it before the call."""
    z = _tt(synth.noisy_pair(16, 16, 1)[0], "f32")[None]
    bank = _tt(_bank(O.Geometry(2, -1), 1, "f32"), "f32")
    with pytest.raises(ValueError):
        mdn.filter_level(z, None, bank, mdn.Geometry(2, -1), mdn.paper_grid_bparams(0),
                         buckets_out=torch.empty((1, 16, 16), dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("prepared", [False, True], ids=["plain_bank", "prepared_bank"])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_wide_denoise_multiscale(mdn, storage, prepared):
    h, w, levels = 101, 77, 3
    nb = levels - 1
    banks = [_bank(GEOM, 20 + l, storage) for l in range(nb)]
    bps = [O.paper_grid_bparams(l) for l in range(nb)]
    z, _ = synth.noisy_pair(h, w, 5500)
    zs = O.round_storage(z, storage)
    ref = O.denoise_multiscale(zs, banks, GEOM, bparams=bps, storage=storage, mirror32=True)
    shapes = [r.shape[1:] for r in ref.pyramid]
    maps = [torch.empty((1, *shapes[l]), dtype=torch.int16, device="cuda") for l in range(nb)]
    dbanks = [_tt(b, storage) for b in banks]
    if prepared:
        dbanks = [mdn.prepare_bank(b, _geom(mdn, GEOM)) for b in dbanks]
    out = mdn.denoise_multiscale(_tt(zs, storage)[None], dbanks, _geom(mdn, GEOM),
                                 [_gbp(mdn, b) for b in bps], bucket_maps=maps)
    mism = []
    for l in range(nb):
        m = _map(maps[l][0]) != ref.buckets[l].astype(np.int64)
        assert not (m & ~ref.bands[l]).any(), (l, (m & ~ref.bands[l]).sum())
        mism.append(m)
    aff = affected_mask(mism, GEOM.r_coarse, shapes)
    err = max_abs(_np(out[0]), ref.out, ~aff)
    assert err <= TOL[storage], err


# ------------------------------------------------------------ A5/A6

GRAM_TOL = {0: 1e-6, 1: 3e-5, 2: 2e-4}
BANK_TOL = {0: 1e-3, 1: 1e-3, 2: 1e-2}
_SET = {}


def _training_set():
    """Two 512x384 pairs with a clean coarse input, the oracle's Gram sums
    over the 4096 buckets and its solved bank."""
    if not _SET:
        bp = O.paper_grid_bparams(0)
        gram = counts = None
        zb, ub, cb = [], [], []
        for i in range(2):
            z, u = synth.noisy_pair(512, 384, 5600 + i)
            uc = synth.clean_image(256, 192, 5700 + i)
            b, _, _ = O.select(z, bp, mirror32=True)
            gram, counts = O.gram_accumulate(z, uc, u, b, K, GEOM, gram, counts)
            zb.append(z); ub.append(u); cb.append(uc)
        _SET["v"] = (gram, counts, O.solve_bank(gram, counts, GEOM, 1e-3), zb, ub, cb)
    return _SET["v"]


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp32", "tf32", "bf16"])
def test_wide_train_level_gram_and_bank(mdn, prec):
    """Counts exact (the u16 sort over 4096 buckets), Gram sums and the bank
    vs the oracle: every well-sampled bucket (n_k >= 10 D) and every empty
    bucket, which takes the pooled filter."""
    gram, counts, ref_bank, zb, ub, cb = _training_set()
    assert (counts == 0).any() and (counts >= 10 * GEOM.D()).any()
    g, c, bank = mdn.train_level_filters(_tt(np.stack(zb), "f32"), _tt(np.stack(cb), "f32"),
                                         _tt(np.stack(ub), "f32"), _geom(mdn, GEOM),
                                         _gbp(mdn, O.paper_grid_bparams(0)), prec, lam=1e-3)
    torch.cuda.synchronize()
    assert mdn.train_status() == 0
    g, c, bank = _np(g), c.cpu().numpy(), _np(bank)
    assert np.array_equal(c, counts)
    rel = np.linalg.norm(g - gram) / np.linalg.norm(gram)
    assert rel < GRAM_TOL[prec], rel
    for k in np.flatnonzero((counts >= 10 * GEOM.D()) | (counts == 0)):
        e = np.linalg.norm(bank[k] - ref_bank[k]) / np.linalg.norm(ref_bank[k])
        assert e < BANK_TOL[prec], (k, counts[k], e)


# ------------------------------------------------------------ A8

def test_server_serves_wide_bank_sets(mdn):
    """A 4096-bucket set of 7x7 + 7x7 banks is served by the fused kernel
    reading the server's prepared copy through L2 (the tile kernels, which
    hold banks of at most 256 buckets in shared memory, are skipped), with
    the per-image path's results for the same prepared banks."""
    geom = mdn.Geometry(3, 3)
    banks = [_tt(_bank(O.Geometry(3, 3), 80 + l, "f16"), "f16") for l in range(2)]
    bps = [mdn.paper_grid_bparams(0), mdn.paper_grid_bparams(1)]
    srv = mdn.Server([(banks, bps)], budget_bytes=64 << 20, autotune=False, tile_variant=0)
    try:
        assert srv.stats()["tile_variant"] == 3
        xs = [torch.tensor(synth.noisy_pair(h, w, 8100 + h)[0], dtype=torch.float16).pin_memory()
              for h, w in [(33, 17), (131, 97)]]
        ys = [torch.empty_like(x).pin_memory() for x in xs]
        ids = [srv.submit(x, y, 0) for x, y in zip(xs, ys)]
        got = set()
        while len(got) < len(ids):
            got |= {r["id"] for r in srv.poll(8, 200)}
        prepared = [mdn.prepare_bank(b, geom) for b in banks]
        for x, y in zip(xs, ys):
            assert torch.equal(y, mdn.denoise_multiscale(x.cuda()[None], prepared, geom, bps)[0].cpu())
    finally:
        srv.close()


# ------------------------------------------------------------ the u8 / u16 boundary

def _edge_grid(K_target):
    """16 x 4 x 4 = 256 buckets (the last u8 grid) or 2 x 12 x 11 = 264 (the
    first u16 one), thresholds from the 16-bin tables."""
    st, co = O.paper_grid_bparams(0).strength_thr, O.paper_grid_bparams(0).coherence_thr
    if K_target == 256:
        return O.BucketParams(16, st[3::4][:3], co[3::4][:3])
    return O.BucketParams(2, st[2:13], co[3:13])


@pytest.mark.parametrize("Kt", [256, 264])
def test_bucket_map_type_boundary(mdn, Kt):
    bp = _edge_grid(Kt)
    assert bp.K == Kt
    z, u = synth.noisy_pair(128, 96, 5800 + Kt)
    ref, band, _ = O.select(z, bp, mirror32=True)
    got_t = mdn.select_buckets(_tt(z, "f32")[None], _gbp(mdn, bp))[0]
    assert got_t.dtype == (torch.uint8 if Kt <= 256 else torch.int16)
    got = _map(got_t)
    mism = got != ref.astype(np.int64)
    assert not (mism & ~band).any()
    assert got.max() >= 200      # the top of the range is used
    # filter with a random bank of this K (shared-memory bank at 256, tile kernel above)
    geom = O.Geometry(2, -1)
    rng = np.random.default_rng(3)
    bank = rng.standard_normal((Kt, 3, geom.D())) * 0.05
    bank += (1.0 - bank.sum(axis=2, keepdims=True)) / geom.D()
    out = mdn.filter_level(_tt(z, "f32")[None], None, _tt(bank, "f32"), _geom(mdn, geom), _gbp(mdn, bp))
    refo = O.filter_level(z, None, ref, bank, geom)
    assert max_abs(_np(out[0]), refo, ~mism) <= TOL["f32"]
    # training: counts exact, Gram within the FP32 bar
    gram, counts = O.gram_accumulate(z, None, u, ref, Kt, geom)
    g, c, _ = mdn.train_level_filters(_tt(z, "f32")[None], None, _tt(u, "f32")[None], _geom(mdn, geom),
                                      _gbp(mdn, bp), 1, solve=False)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), counts)
    g = _np(g)
    assert np.linalg.norm(g - gram) / np.linalg.norm(gram) < GRAM_TOL[1]
