"""Bank and Gram-state checkpoints (host only): round trips, header contents
and rejection of the wrong kind of file."""
import json

import numpy as np
import pytest
import torch

import paper_1802_06130_gb300 as mdn


def test_bank_round_trip(tmp_path):
    geom = mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    rng = np.random.default_rng(0)
    banks = [torch.tensor(rng.standard_normal((216, 3, 98)), dtype=torch.float32) for _ in range(2)]
    p = tmp_path / "set.bank"
    mdn.save_banks(p, banks, geom, bps, sigma=25 / 255)
    with open(p, "rb") as f:
        head = json.loads(f.readline())
    assert head["kind"] == "banks" and head["shapes"] == [[216, 3, 98]] * 2 and head["dtypes"] == ["<f4"] * 2
    b2, g2, bp2, sig = mdn.load_banks(p, device="cpu")
    assert all(torch.equal(a, b) for a, b in zip(banks, b2))
    assert (g2.r_fine, g2.r_coarse, g2.cross_channel, g2.color) == (3, 3, 0, 0)
    assert sig == pytest.approx(25 / 255)
    for a, b in zip(bps, bp2):
        assert (a.n_angle, a.n_strength, a.n_coherence) == (b.n_angle, b.n_strength, b.n_coherence)
        assert [a.strength_thr[i] for i in range(2)] == [b.strength_thr[i] for i in range(2)]
        assert [a.coherence_thr[i] for i in range(2)] == [b.coherence_thr[i] for i in range(2)]
        assert a.coh_eps == b.coh_eps


def test_gram_round_trip_and_kind_check(tmp_path):
    geom = mdn.Geometry(3, -1, 1)
    rng = np.random.default_rng(1)
    g = torch.tensor(rng.standard_normal((216, 1, 150, 150)), dtype=torch.float64)
    c = torch.tensor(rng.integers(0, 1 << 40, 216), dtype=torch.int64)
    p = tmp_path / "l0.gram"
    mdn.save_gram_state(p, g, c, geom, mdn.default_bparams(0), level=0)
    g2, c2, geom2, bp2, lev = mdn.load_gram_state(p, device="cpu")
    assert torch.equal(g, g2) and torch.equal(c, c2) and lev == 0 and geom2.cross_channel == 1
    with pytest.raises(ValueError):
        mdn.load_banks(p, device="cpu")
    bad = tmp_path / "bad"
    bad.write_bytes(b'{"format": "other"}\n')
    with pytest.raises(ValueError):
        mdn.load_gram_state(bad, device="cpu")


def test_paper_grid_bank_round_trip(tmp_path):
    """A 4096-bucket bank set keeps its 15 + 15 thresholds per level."""
    geom = mdn.Geometry(3, 2)
    bps = [mdn.paper_grid_bparams(0), mdn.paper_grid_bparams(1)]
    banks = [torch.zeros((4096, 3, 74), dtype=torch.float32) + l for l in range(2)]
    p = tmp_path / "grid16.bank"
    mdn.save_banks(p, banks, geom, bps)
    b2, g2, bp2, _ = mdn.load_banks(p, device="cpu")
    assert all(torch.equal(a, b) for a, b in zip(banks, b2))
    assert (g2.r_fine, g2.r_coarse) == (3, 2)
    for a, b in zip(bps, bp2):
        assert b.K == 4096 and (b.n_strength, b.n_coherence) == (16, 16)
        assert list(a.strength_thr) == list(b.strength_thr)
        assert list(a.coherence_thr) == list(b.coherence_thr)


def test_fp16_banks_keep_their_precision(tmp_path):
    geom = mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    rng = np.random.default_rng(2)
    banks = [torch.tensor(rng.standard_normal((216, 3, 98)), dtype=torch.float16),
             torch.tensor(rng.standard_normal((216, 3, 98)), dtype=torch.float32)]
    p = tmp_path / "mixed.bank"
    mdn.save_banks(p, banks, geom, bps)
    b2, _, _, _ = mdn.load_banks(p, device="cpu")
    assert [b.dtype for b in b2] == [torch.float16, torch.float32]
    assert all(torch.equal(a, b) for a, b in zip(banks, b2))
    with pytest.raises(ValueError):
        mdn.save_banks(tmp_path / "x.bank", [banks[0].double()], geom, bps[:1])


def test_payload_length_is_checked(tmp_path):
    """A truncated file or one with trailing bytes is refused with ValueError,
    not read short or past its header's shapes."""
    geom = mdn.Geometry(2, -1)
    bank = torch.zeros((216, 3, 25), dtype=torch.float32)
    p = tmp_path / "one.bank"
    mdn.save_banks(p, [bank], geom, [mdn.default_bparams(0)])
    data = p.read_bytes()
    (tmp_path / "short.bank").write_bytes(data[:-4])
    (tmp_path / "long.bank").write_bytes(data + b"\0" * 8)
    for name in ("short.bank", "long.bank"):
        with pytest.raises(ValueError, match="payload"):
            mdn.load_banks(tmp_path / name, device="cpu")
    g = torch.zeros((216, 1, 26, 26), dtype=torch.float64)
    c = torch.zeros(216, dtype=torch.int64)
    q = tmp_path / "l.gram"
    mdn.save_gram_state(q, g, c, geom, mdn.default_bparams(0))
    (tmp_path / "short.gram").write_bytes(q.read_bytes()[:-8])
    with pytest.raises(ValueError, match="payload"):
        mdn.load_gram_state(tmp_path / "short.gram", device="cpu")
