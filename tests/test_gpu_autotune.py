"""Level-kernel autotuner: mdn_autotune_level times the variants that apply
to a configuration and records the fastest; the level calls then follow the
table, every variant the table can name stays within the parity bars of the
FP64 oracle, and the server stores and reads its own entry.  The table is
process-wide, so every test leaves it empty."""
import numpy as np
import pytest

import oracle as O
import synth
from parity_util import max_abs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f16": 2e-3}


@pytest.fixture()
def mdn():
    import paper_1802_06130_gb300 as m
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.build()
    m.autotune_clear()
    yield m
    m.autotune_clear()


def _tt(a, storage):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32 if storage == "f32" else torch.float16,
                        device="cuda")


def _bank(K, geom, seed):
    rng = np.random.default_rng(seed)
    D = geom.D()
    b = rng.standard_normal((K, 3, D)) * 0.05
    b += (1.0 - b.sum(axis=2, keepdims=True)) / D
    return O.round_storage(b, "f16")


def _gbp(m, bp):
    return m.BucketParams(bp.n_angle, tuple(bp.strength_thr), tuple(bp.coherence_thr), bp.coh_eps)


def test_tuner_picks_an_applicable_variant_and_the_calls_follow_it(mdn):
    geom = mdn.Geometry(3, 3)
    bp = mdn.default_bparams(0)
    best, ms = mdn.autotune_level(geom, bp, mdn.F16, mdn.F16, 1, 768, 1024)
    assert ms["fused_l2"] is None                      # plain bank: the L2 variant reads prepared banks only
    assert all(ms[k] is not None and ms[k] > 0 for k in ("fused_smem", "strip", "tile_smem", "tile_l2"))
    assert mdn.LEVEL_VARIANTS[best] == min((v, k) for k, v in ms.items() if v is not None)[1]
    assert mdn.autotune_lookup(geom, 216, mdn.F16, mdn.F16, 1, 768, 1024) == best
    # prepared 4096-bucket bank, 7x7 + 5x5: only the L2 variant applies
    best2, ms2 = mdn.autotune_level(mdn.Geometry(3, 2), mdn.paper_grid_bparams(0), mdn.F16, mdn.F16_ROWS,
                                    1, 512, 512)
    assert best2 == 1 and [k for k, v in ms2.items() if v is not None] == ["fused_l2"]


@pytest.mark.parametrize("variant", [0, 2, 3, 4])
def test_every_variant_named_by_the_table_meets_the_parity_bar(mdn, variant, tmp_path):
    """A table entry forcing each variant: filter_level follows it and stays
    within the FP16 bar of the oracle (same FP16 bank on both sides)."""
    geom_o = O.Geometry(3, 3)
    geom = mdn.Geometry(3, 3)
    h, w = 131, 197
    size_class = int(np.floor(np.log2(h * w)))
    p = tmp_path / "table.txt"
    p.write_text(f"level 3 3 0 {mdn.F16} {mdn.F16} 0 216 {size_class} {variant} 0.1\n")
    mdn.autotune_load(p)
    assert mdn.autotune_lookup(geom, 216, mdn.F16, mdn.F16, 1, h, w) == variant
    bank = _bank(216, geom_o, 90 + variant)
    zs = O.round_storage(synth.noisy_pair(h, w, 9100)[0], "f16")
    uc = O.round_storage(synth.clean_image((h + 1) // 2, (w + 1) // 2, 9200), "f16")
    bpo = O.default_bparams(0)
    ref_b, band, _ = O.select(zs, bpo, mirror32=True)
    ref = O.round_storage(O.filter_level(zs, uc, ref_b, bank, geom_o), "f16")
    m = torch.empty((1, h, w), dtype=torch.uint8, device="cuda")
    out = mdn.filter_level(_tt(zs, "f16")[None], _tt(uc, "f16")[None], _tt(bank, "f16"), geom, _gbp(mdn, bpo),
                           buckets_out=m)
    mism = m[0].cpu().numpy() != ref_b
    assert not (mism & ~band).any()
    assert max_abs(out[0].float().cpu().numpy().astype(np.float64), ref, ~mism) <= TOL["f16"]


def test_server_stores_and_reads_its_entry(mdn, tmp_path):
    rng = np.random.default_rng(5)
    banks = []
    for _ in range(2):
        b = rng.standard_normal((216, 3, 98)).astype(np.float32) * 0.03
        b += (1.0 - b.sum(axis=2, keepdims=True)) / 98
        banks.append(torch.tensor(b, dtype=torch.float16, device="cuda"))
    sets = [(banks, [mdn.default_bparams(l) for l in range(2)])]
    srv = mdn.Server(sets, budget_bytes=64 << 20, autotune=True)
    chosen = srv.stats()["tile_variant"]
    srv.close()
    assert mdn.lib().mdn_autotune_server_lookup(mdn.C.byref(mdn.Geometry(3, 3)), 0) == chosen
    # a saved table with another server entry: a server created without tuning takes it
    other = 1 if chosen != 1 else 2
    p = tmp_path / "server.txt"
    p.write_text(f"server 3 3 0 {other} 0.3\n")
    mdn.autotune_clear()
    mdn.autotune_load(p)
    srv = mdn.Server(sets, budget_bytes=64 << 20, autotune=False)
    try:
        assert srv.stats()["tile_variant"] == other
        x = torch.tensor(synth.noisy_pair(97, 131, 9300)[0], dtype=torch.float16).pin_memory()
        y = torch.empty_like(x).pin_memory()
        rid = srv.submit(x, y, 0)
        got = []
        while not got:
            got = [r for r in srv.poll(8, 200) if r["id"] == rid]
        ref = mdn.denoise_multiscale(x.cuda()[None], banks, mdn.Geometry(3, 3), sets[0][1])[0].cpu()
        assert torch.equal(y, ref)
    finally:
        srv.close()


@pytest.mark.parametrize("geom_args", [(3, 3), (3, 2)], ids=["7x7+7x7", "7x7+5x5"])
def test_cluster_bank_equals_l2_bank(mdn, geom_args, tmp_path):
    """An FP32 bank too large for one CTA's shared memory: split over a
    cluster of two CTAs (variant 5) it gives, bit for bit, the results of
    the same prepared bank read through L2 (variant 1), and meets the FP32
    parity bar of the oracle."""
    geom_o = O.Geometry(*geom_args)
    geom = mdn.Geometry(*geom_args)
    h, w = 197, 131
    sc = int(np.floor(np.log2(h * w)))
    rng = np.random.default_rng(95)
    D = geom_o.D()
    bank = rng.standard_normal((216, 3, D)) * 0.05
    bank += (1.0 - bank.sum(axis=2, keepdims=True)) / D
    bank = bank.astype(np.float32).astype(np.float64)
    zs = O.round_storage(synth.noisy_pair(h, w, 9400)[0], "f32")
    uc = O.round_storage(synth.clean_image((h + 1) // 2, (w + 1) // 2, 9401), "f32")
    bpo = O.default_bparams(0)
    prepared = mdn.prepare_bank(_tt(bank, "f32"), geom)
    outs = {}
    for v in (1, 5):
        p = tmp_path / f"t{v}.txt"
        p.write_text(f"level {geom_args[0]} {geom_args[1]} 0 {mdn.F32} {mdn.F32} 1 216 {sc} {v} 0.1\n")
        mdn.autotune_clear()
        mdn.autotune_load(p)
        m = torch.empty((1, h, w), dtype=torch.uint8, device="cuda")
        outs[v] = (mdn.filter_level(_tt(zs, "f32")[None], _tt(uc, "f32")[None], prepared, geom, _gbp(mdn, bpo),
                                    buckets_out=m), m)
    assert torch.equal(outs[1][0], outs[5][0]) and torch.equal(outs[1][1], outs[5][1])
    ref_b, band, _ = O.select(zs, bpo, mirror32=True)
    ref = O.filter_level(zs, uc, ref_b, bank, geom_o)
    mism = outs[5][1][0].cpu().numpy() != ref_b
    assert not (mism & ~band).any()
    assert max_abs(outs[5][0][0].cpu().numpy().astype(np.float64), ref, ~mism) <= TOL["f32"]
