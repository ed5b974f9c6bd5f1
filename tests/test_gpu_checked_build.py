"""Bounds-checked debug build (-DMDN_CHECK, the stand-in for a memory
sanitizer): the library's kernels run with every checked shared- and
global-memory index tested against its buffer.  Each case runs through the
normal and the checked library; the checked run must record no violation
(mdn_check_status) and give the normal run's results (bit for bit where the
arithmetic is written out as explicit FP32 operations: pyramid levels and
bucket maps; within one FP16 / FP32 rounding for filtered outputs, whose
colour conversion the compiler may contract differently).  Sizes are the
odd ones that exercise every clamp and ragged-tile path (1x1, 2x3, 7x5,
33x17, 131x97) plus frames large enough for interior tiles."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ODD = [(1, 1), (2, 3), (7, 5), (33, 17), (131, 97)]


@pytest.fixture(scope="module")
def mdn():
    import paper_1802_06130_gb300 as m
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.build()
    m.use_checked_build(True)      # builds the checked library once
    assert m.check_status() == (0, 0)
    m.use_checked_build(False)
    yield m
    m.use_checked_build(False)


def _both(m, fn):
    """fn() through the normal and the checked library -> (normal, checked)."""
    m.use_checked_build(False)
    ref = fn()
    torch.cuda.synchronize()
    m.use_checked_build(True)
    try:
        got = fn()
        torch.cuda.synchronize()
        site, idx = m.check_status()
    finally:
        m.use_checked_build(False)
    assert site == 0, f"bounds violation at check site {site}, index {idx}"
    return ref, got


def _img(h, w, seed, dt):
    return torch.tensor(synth.noisy_pair(h, w, seed)[0], dtype=dt, device="cuda")[None]


def _bank(K, D, seed, dt):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((K, 3, D)).astype(np.float32) * 0.03
    b += (1.0 - b.sum(axis=2, keepdims=True)) / D
    return torch.tensor(b, dtype=dt, device="cuda")


def _close(a, b, dt):
    tol = 1e-3 if dt == torch.float16 else 1e-5
    assert (a.float() - b.float()).abs().max().item() <= tol


@pytest.mark.parametrize("dt", [torch.float32, torch.float16])
def test_checked_pyramid_and_selection(mdn, dt):
    for i, (h, w) in enumerate(ODD + [(300, 200), (260, 640)]):
        x = _img(h, w, 900 + i, dt)
        ref, got = _both(mdn, lambda: mdn.build_pyramid(x, 4))
        assert all(torch.equal(a, b) for a, b in zip(ref, got))
        for bp in (mdn.default_bparams(0), mdn.paper_grid_bparams(0)):
            r, g = _both(mdn, lambda: mdn.select_buckets(x, bp))
            assert torch.equal(r, g)


@pytest.mark.parametrize("geom_args,D", [((2, -1), 25), ((3, 3), 98), ((3, 2), 74), ((3, -1, 1), 147)],
                         ids=["5x5", "7x7+7x7", "7x7+5x5", "7x7x3"])
@pytest.mark.parametrize("bank_dt", [torch.float16, torch.float32])
def test_checked_filter_level(mdn, geom_args, D, bank_dt):
    geom = mdn.Geometry(*geom_args)
    bp = mdn.default_bparams(0)
    bank = _bank(216, D, 7, bank_dt)
    for i, (h, w) in enumerate(ODD + [(200, 300)]):
        for dt in (torch.float16, torch.float32):
            z = _img(h, w, 950 + i, dt)
            c = _img((h + 1) // 2, (w + 1) // 2, 960 + i, dt) if geom.r_coarse >= 0 else None
            ref, got = _both(mdn, lambda: mdn.filter_level(z, c, bank, geom, bp))
            _close(ref, got, dt)
            ref, got = _both(mdn, lambda: mdn.filter_level(z, c, mdn.prepare_bank(bank, geom), geom, bp))
            _close(ref, got, dt)


def test_checked_denoise_multiscale_and_wide_grid(mdn):
    geom, geom_p = mdn.Geometry(3, 3), mdn.Geometry(3, 2)
    banks = [_bank(216, 98, 11 + l, torch.float16) for l in range(3)]
    wide = [_bank(4096, 74, 21 + l, torch.float16) for l in range(2)]
    for i, (h, w) in enumerate([(131, 97), (257, 385)]):
        x = _img(h, w, 970 + i, torch.float16)
        ref, got = _both(mdn, lambda: mdn.denoise_multiscale(x, banks, geom, [mdn.default_bparams(l) for l in range(3)]))
        _close(ref, got, torch.float16)
        ref, got = _both(mdn, lambda: mdn.denoise_multiscale(x, wide, geom_p, [mdn.paper_grid_bparams(l) for l in range(2)]))
        _close(ref, got, torch.float16)
        ref, got = _both(mdn, lambda: mdn.denoise_multiscale(x, [mdn.prepare_bank(b, geom_p) for b in wide], geom_p,
                                                             [mdn.paper_grid_bparams(l) for l in range(2)]))
        _close(ref, got, torch.float16)
    host = _img(97, 131, 980, torch.float16).cpu().repeat(3, 1, 1, 1).contiguous().pin_memory()

    def piped():
        out = torch.empty_like(host).pin_memory()
        mdn.denoise_multiscale_pipelined(host, banks[:2], geom, [mdn.default_bparams(l) for l in range(2)], out,
                                         chunk=2)
        return out
    ref, got = _both(mdn, piped)
    _close(ref, got, torch.float16)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "split"])
def test_checked_training(mdn, prec):
    p = {"fp32": mdn.GRAM_FP32, "tf32": mdn.GRAM_TF32, "bf16": mdn.GRAM_BF16, "split": mdn.GRAM_SPLIT_BF16}[prec]
    pairs = [synth.noisy_pair(67, 45, 990 + i) for i in range(2)]
    Z = torch.tensor(np.stack([a for a, _ in pairs]), device="cuda")
    U = torch.tensor(np.stack([b for _, b in pairs]), device="cuda")
    for geom in (mdn.Geometry(3, -1, 1), mdn.Geometry(2, -1)):
        ref, got = _both(mdn, lambda: mdn.train_level_filters(Z, None, U, geom, mdn.default_bparams(0), p))
        assert torch.equal(ref[1], got[1])                       # counts
        g0, g1 = ref[0], got[0]
        assert ((g0 - g1).norm() / g0.norm()).item() < 1e-6      # same sums up to FP64 summation order


def test_checked_server(mdn):
    sets = [([_bank(216, 98, 31 + l, torch.float16) for l in range(2)], [mdn.default_bparams(l) for l in range(2)])]
    frames = [torch.tensor(synth.noisy_pair(h, w, 995 + i)[0], dtype=torch.float16).pin_memory()
              for i, (h, w) in enumerate([(33, 17), (131, 97), (64, 80)])]

    def serve():
        srv = mdn.Server(sets, budget_bytes=64 << 20, max_active=4, autotune=False)
        try:
            outs = [torch.empty_like(f).pin_memory() for f in frames]
            ids = [srv.submit(f, o, 0) for f, o in zip(frames, outs)]
            got = set()
            while len(got) < len(ids):
                got |= {r["id"] for r in srv.poll(8, 200)}
        finally:
            srv.close()
        return outs
    ref, got = _both(mdn, serve)
    for a, b in zip(ref, got):
        _close(a, b, torch.float16)
