"""Tensor-descriptor forms (mdn_t_*) against the pointer forms on the same
inputs: identical results, and strided views refused with MDN_ESHAPE."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdn():
    import paper_1802_06130_gb300 as m
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.build()
    m.lib()
    return m


def _img(h, w, seed, dt, n=1):
    return torch.stack([torch.tensor(synth.noisy_pair(h, w, seed + i)[0], dtype=dt) for i in range(n)]).cuda()


def _bank(K, D, seed, dt):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((K, 3, D)).astype(np.float32) * 0.03
    b += (1.0 - b.sum(axis=2, keepdims=True)) / D
    return torch.tensor(b, dtype=dt, device="cuda")


@pytest.mark.parametrize("dt", [torch.float16, torch.float32])
def test_pyramid_and_filter_level(mdn, dt):
    x = _img(131, 200, 7000, dt, n=2)
    outs = [torch.empty((2, 3, 66, 100), dtype=dt, device="cuda"), torch.empty((2, 3, 33, 50), dtype=dt, device="cuda")]
    mdn.t_build_pyramid(x, 3, outs)
    ref = mdn.build_pyramid(x, 3)
    assert all(torch.equal(a, b) for a, b in zip(outs, ref))
    geom, bp = mdn.Geometry(3, 3), mdn.default_bparams(0)
    bank = _bank(216, 98, 1, torch.float16)
    for b in (bank, mdn.prepare_bank(bank, geom)):
        out = torch.empty_like(x)
        m = torch.empty((2, 131, 200), dtype=torch.uint8, device="cuda")
        mdn.t_filter_level(x, outs[0], b, geom, bp, out, m)
        m2 = torch.empty_like(m)
        assert torch.equal(out, mdn.filter_level(x, outs[0], b, geom, bp, buckets_out=m2)) and torch.equal(m, m2)


def test_denoise_multiscale_with_maps(mdn):
    geom = mdn.Geometry(3, 3)
    x = _img(97, 131, 7100, torch.float16)
    banks = [_bank(216, 98, 10 + l, torch.float16) for l in range(2)]
    bps = [mdn.default_bparams(l) for l in range(2)]
    out = torch.empty_like(x)
    maps = [torch.empty((1, 97, 131), dtype=torch.uint8, device="cuda"),
            torch.empty((1, 49, 66), dtype=torch.uint8, device="cuda")]
    mdn.t_denoise_multiscale(x, banks, geom, bps, out, bucket_maps=maps)
    maps2 = [torch.empty_like(m) for m in maps]
    ref = mdn.denoise_multiscale(x, banks, geom, bps, bucket_maps=maps2)
    assert torch.equal(out, ref) and all(torch.equal(a, b) for a, b in zip(maps, maps2))


def test_train_level_filters(mdn):
    geom, bp = mdn.Geometry(3, -1, 1), mdn.default_bparams(0)
    pairs = [synth.noisy_pair(67, 45, 7200 + i) for i in range(2)]
    Z = torch.tensor(np.stack([a for a, _ in pairs]), device="cuda")
    U = torch.tensor(np.stack([b for _, b in pairs]), device="cuda")
    gram = torch.empty((216, 1, 150, 150), dtype=torch.float64, device="cuda")
    counts = torch.empty(216, dtype=torch.int64, device="cuda")
    bank = torch.empty((216, 3, 147), dtype=torch.float32, device="cuda")
    mdn.t_train_level_filters(Z, None, U, geom, bp, mdn.GRAM_FP32, gram, counts, 1e-3, bank)
    g2, c2, b2 = mdn.train_level_filters(Z, None, U, geom, bp, mdn.GRAM_FP32, lam=1e-3)
    assert torch.equal(counts, c2)
    assert ((gram - g2.reshape(gram.shape)).norm() / g2.norm()).item() < 1e-12
    assert ((bank - b2.reshape(bank.shape)).norm() / b2.norm()).item() < 1e-6


def test_strided_views_are_refused(mdn):
    x = _img(64, 96, 7300, torch.float16)
    wide = torch.empty((1, 3, 64, 192), dtype=torch.float16, device="cuda")
    view = wide[..., ::2]                                     # a step in the last dimension
    with pytest.raises(mdn.MdnError) as ei:
        mdn.t_build_pyramid(view, 2, [torch.empty((1, 3, 32, 48), dtype=torch.float16, device="cuda")])
    assert ei.value.code == 2 and "stride" in str(ei.value)
    bank = _bank(216, 98, 2, torch.float16)
    with pytest.raises(mdn.MdnError) as ei:
        mdn.t_filter_level(x, _img(32, 48, 7301, torch.float16), bank.transpose(1, 2), mdn.Geometry(3, 3),
                           mdn.default_bparams(0), torch.empty_like(x))
    assert ei.value.code == 2 and "bank" in str(ei.value)
