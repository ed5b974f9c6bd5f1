"""Serving (continuous batching): results identical alone and in a mixed
stream, admission by memory budget, cancellation and bounded polling."""
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


def _bank_set(mdn, levels, seed):
    rng = np.random.default_rng(seed)
    banks = []
    for _ in range(levels - 1):
        b = rng.standard_normal((216, 3, 98)).astype(np.float32) * 0.03
        b += (1.0 - b.sum(axis=2, keepdims=True)) / 98
        banks.append(torch.tensor(b, dtype=torch.float16, device="cuda"))
    return banks, [mdn.default_bparams(l) for l in range(levels - 1)]


def _frame(h, w, seed):
    z = synth.noisy_pair(h, w, seed)[0]
    return torch.tensor(z, dtype=torch.float16).pin_memory()


def _drain(srv, want, timeout_s=60.0):
    import time
    got = {}
    t0 = time.time()
    while len(got) < want:
        for r in srv.poll(64, 200):
            got[r["id"]] = r
        assert time.time() - t0 < timeout_s, "server did not finish in time"
    return got


def test_mixed_stream_equals_single_image_path(mdn):
    sets = [_bank_set(mdn, 3, 1), _bank_set(mdn, 4, 2)]
    sizes = [(64, 80), (131, 97), (240, 320), (33, 17), (1, 1), (480, 640), (97, 131), (256, 256)]
    srv = mdn.Server(sets, budget_bytes=256 << 20, max_active=6, autotune=True)
    try:
        # frames made first so that the requests arrive in a burst and share ticks
        io = []
        for i in range(16):
            h, w = sizes[i % len(sizes)]
            x = _frame(h, w, 60000 + i)
            io.append((x, torch.empty_like(x).pin_memory(), i % 2))
        reqs = [(srv.submit(x, y, s), x, y, s) for x, y, s in io]
        got = _drain(srv, len(reqs))
        assert all(r["status"] == 0 for r in got.values())
        for rid, x, y, s in reqs:
            banks, bps = sets[s]
            ref = mdn.denoise_multiscale(x.cuda()[None], banks, mdn.Geometry(3, 3), bps)[0].cpu()
            assert torch.equal(y, ref), rid
        st = srv.stats()
        assert st["completed"] == len(reqs)
        assert st["tick_items"] > st["ticks"]          # stages of several requests shared ticks
        assert st["tile_variant"] in (0, 1, 2, 3) and min(st["variant_ms"]) > 0
    finally:
        srv.close()


def test_admission_respects_the_budget(mdn):
    sets = [_bank_set(mdn, 3, 3)]
    one = 2 * 3 * 480 * 640 * 2 + 3 * 240 * 320 * 2 * 2 + 3 * 120 * 160 * 2 + 4096
    budget = max(int(2.5 * one), 1 << 20)
    srv = mdn.Server(sets, budget_bytes=budget, max_active=16, autotune=False)
    try:
        reqs = []
        for i in range(6):
            x = _frame(480, 640, 61000 + i)
            y = torch.empty_like(x).pin_memory()
            reqs.append((srv.submit(x, y, 0), x, y))
        got = _drain(srv, len(reqs))
        assert all(r["status"] == 0 for r in got.values())
        st = srv.stats()
        assert st["arena_peak"] <= budget
        assert st["arena_peak"] <= 2 * one + 8192          # at most two requests fit at a time
        big = _frame(2000, 2000, 61999)
        with pytest.raises(mdn.MdnError) as ei:
            srv.submit(big, torch.empty_like(big), 0)
        assert ei.value.code == 4
        banks, bps = sets[0]
        for rid, x, y in reqs:
            ref = mdn.denoise_multiscale(x.cuda()[None], banks, mdn.Geometry(3, 3), bps)[0].cpu()
            assert torch.equal(y, ref)
    finally:
        srv.close()


def test_cancel_queued_request_and_poll_timeout(mdn):
    sets = [_bank_set(mdn, 3, 4)]
    srv = mdn.Server(sets, budget_bytes=64 << 20, max_active=1, autotune=False)
    try:
        assert srv.poll(8, 50) == []                        # nothing submitted: bounded wait, no result
        xs = [_frame(1080, 1920, 62000 + i) for i in range(10)]
        ys = [torch.empty_like(x).pin_memory() for x in xs]
        ids = [srv.submit(x, y, 0) for x, y in zip(xs, ys)]
        cancelled = None
        for rid in reversed(ids):
            try:
                srv.cancel(rid)
                cancelled = rid
                break
            except mdn.MdnError:
                continue
        assert cancelled is not None
        got = _drain(srv, len(ids))
        assert got[cancelled]["status"] == 5
        assert sum(r["status"] == 0 for r in got.values()) == len(ids) - 1
        with pytest.raises(mdn.MdnError):
            srv.cancel(ids[0])                              # already finished
    finally:
        srv.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_level_kernel_variant_equals_single_image_path(mdn, variant):
    """Tile kernels (0-2) and the fused warp-specialised kernel reading
    prepared banks through L2 (3) give the per-image path's results bit for
    bit, on sizes with ragged tiles."""
    sets = [_bank_set(mdn, 3, 11), _bank_set(mdn, 4, 12)]
    sizes = [(1, 1), (33, 17), (131, 97), (240, 320), (517, 389)]
    srv = mdn.Server(sets, budget_bytes=256 << 20, max_active=8, autotune=False, tile_variant=variant)
    try:
        assert srv.stats()["tile_variant"] == variant
        io = []
        for i, (h, w) in enumerate(sizes * 2):
            x = _frame(h, w, 63000 + i)
            io.append((x, torch.empty_like(x).pin_memory(), i % 2))
        reqs = [(srv.submit(x, y, s), x, y, s) for x, y, s in io]
        got = _drain(srv, len(reqs))
        assert all(r["status"] == 0 for r in got.values())
        for rid, x, y, s in reqs:
            banks, bps = sets[s]
            ref = mdn.denoise_multiscale(x.cuda()[None], banks, mdn.Geometry(3, 3), bps)[0].cpu()
            assert torch.equal(y, ref), (variant, rid, tuple(x.shape))
    finally:
        srv.close()


def test_large_and_small_classes(mdn):
    """Requests of at least 4 M pixels run one per tick in the large class,
    smaller ones batched in the small class; all results equal the per-image
    path's, whatever class or tick they ran in."""
    sets = [_bank_set(mdn, 3, 13)]
    sizes = [(2048, 2048), (240, 320), (97, 131), (2001, 2100), (480, 640), (64, 80)]
    srv = mdn.Server(sets, budget_bytes=1 << 30, max_active=16, autotune=True)
    try:
        io = []
        for i, (h, w) in enumerate(sizes):
            x = _frame(h, w, 64000 + i)
            io.append((x, torch.empty_like(x).pin_memory()))
        reqs = [(srv.submit(x, y, 0), x, y) for x, y in io]
        got = _drain(srv, len(reqs))
        assert all(r["status"] == 0 for r in got.values())
        banks, bps = sets[0]
        for rid, x, y in reqs:
            ref = mdn.denoise_multiscale(x.cuda()[None], banks, mdn.Geometry(3, 3), bps)[0].cpu()
            assert torch.equal(y, ref), tuple(x.shape)
        st = srv.stats()
        assert st["ticks_large"] == 2                      # the two frames of >= 4 M pixels, one tick each
        assert st["ticks"] > st["ticks_large"]
    finally:
        srv.close()


def test_paper_grid_served_with_prepared_banks(mdn):
    """The paper's 16 x 16 x 16 grid (4096 buckets) with 7x7 + 5x5 taps:
    only the fused kernel applies (the tile kernels hold banks of at most
    256 buckets in shared memory); results equal the per-image path run with
    the same banks prepared (the same kernel over a batch)."""
    geom = mdn.Geometry(3, 2)
    rng = np.random.default_rng(14)
    banks = []
    for _ in range(2):
        b = rng.standard_normal((4096, 3, 74)).astype(np.float32) * 0.03
        b += (1.0 - b.sum(axis=2, keepdims=True)) / 74
        banks.append(torch.tensor(b, dtype=torch.float16, device="cuda"))
    bps = [mdn.paper_grid_bparams(l) for l in range(2)]
    srv = mdn.Server([(banks, bps)], budget_bytes=512 << 20, max_active=8, autotune=True, geom=geom)
    try:
        st = srv.stats()
        assert st["tile_variant"] == 3 and st["variant_ms"][0] < 0 and st["variant_ms"][3] > 0
        io = []
        for i, (h, w) in enumerate([(1, 1), (33, 17), (131, 97), (480, 640), (517, 389)]):
            x = _frame(h, w, 65000 + i)
            io.append((x, torch.empty_like(x).pin_memory()))
        reqs = [(srv.submit(x, y, 0), x, y) for x, y in io]
        got = _drain(srv, len(reqs))
        assert all(r["status"] == 0 for r in got.values())
        prepared = [mdn.prepare_bank(b, geom) for b in banks]
        for rid, x, y in reqs:
            ref = mdn.denoise_multiscale(x.cuda()[None], prepared, geom, bps)[0].cpu()
            assert torch.equal(y, ref), tuple(x.shape)
    finally:
        srv.close()


def test_server_rejects_uncompiled_geometry(mdn):
    sets = [_bank_set(mdn, 3, 15)]
    with pytest.raises(mdn.MdnError) as ei:
        mdn.Server(sets, budget_bytes=64 << 20, geom=mdn.Geometry(2, -1))
    assert ei.value.code == 2


@pytest.mark.parametrize("copy_engines", [False, True], ids=["sm_copies", "copy_engines"])
def test_host_buffer_kinds(mdn, copy_engines, monkeypatch):
    """Pinned 16-byte aligned host buffers are moved by the SM copy kernel
    (byte counts that are not a multiple of 16 leave a tail for the copy
    engines); pageable buffers and pinned ones at an odd offset by the copy
    engines; MDN_SERVER_COPY_ENGINES=1 sends everything through the copy
    engines.  Every combination gives the per-image path's results."""
    if copy_engines:
        monkeypatch.setenv("MDN_SERVER_COPY_ENGINES", "1")
    sets = [_bank_set(mdn, 3, 16)]
    srv = mdn.Server(sets, budget_bytes=256 << 20, max_active=8, autotune=False)
    monkeypatch.delenv("MDN_SERVER_COPY_ENGINES", raising=False)

    def odd_offset(h, w, seed):
        base = torch.empty(3 * h * w + 8, dtype=torch.float16).pin_memory()
        v = base[1:1 + 3 * h * w].view(3, h, w)
        v.copy_(_frame(h, w, seed))
        assert v.data_ptr() % 16 != 0
        return v, base

    try:
        keep, io = [], []
        for i, (h, w) in enumerate([(97, 131), (64, 80), (1, 1), (240, 320)]):
            pinned = _frame(h, w, 66000 + i)
            pageable = pinned.clone()
            odd, base = odd_offset(h, w, 66000 + i)
            keep.append(base)
            outs = [torch.empty_like(pinned).pin_memory(), torch.empty_like(pinned)]
            ob = torch.empty(3 * h * w + 8, dtype=torch.float16).pin_memory()
            keep.append(ob)
            outs.append(ob[1:1 + 3 * h * w].view(3, h, w))
            for x in (pinned, pageable, odd):
                for y in outs:
                    io.append((x, y))
        reqs = []
        for x, y in io:
            y.zero_()
            reqs.append((srv.submit(x, y, 0), x, y))
            got = _drain(srv, 1)                           # one at a time: outputs share buffers
            assert all(r["status"] == 0 for r in got.values())
            banks, bps = sets[0]
            ref = mdn.denoise_multiscale(x.contiguous().cuda()[None], banks, mdn.Geometry(3, 3), bps)[0].cpu()
            assert torch.equal(y, ref), (tuple(x.shape), x.is_pinned(), x.data_ptr() % 16, y.data_ptr() % 16)
    finally:
        srv.close()


def test_per_tick_trace(mdn, tmp_path, monkeypatch):
    """MDN_SERVER_TRACE at create: at destroy the server writes one CSV line
    per tick (requests, pixels, host launch / retire times, device phase
    times, request ids) covering every completed request exactly once."""
    path = tmp_path / "trace.csv"
    monkeypatch.setenv("MDN_SERVER_TRACE", str(path))
    sets = [_bank_set(mdn, 3, 17)]
    srv = mdn.Server(sets, budget_bytes=256 << 20, max_active=8, autotune=False)
    monkeypatch.delenv("MDN_SERVER_TRACE")
    try:
        frames = [_frame(h, w, 67000 + i) for i, (h, w) in enumerate([(64, 80), (131, 97), (240, 320), (33, 17)])]
        outs = [torch.empty_like(f).pin_memory() for f in frames]
        ids = [srv.submit(f, o, 0) for f, o in zip(frames, outs)]
        _drain(srv, len(ids))
    finally:
        srv.close()
    lines = path.read_text().strip().splitlines()
    head = lines[0].split(",")
    assert head[:3] == ["tick", "requests", "pixels"] and head[-1] == "ids"
    seen, pix = [], 0
    for ln in lines[1:]:
        f = ln.split(",")
        got = [int(x) for x in f[-1].split(";")]
        assert int(f[1]) == len(got)
        seen += got
        pix += int(f[2])
        launch, retire = float(f[3]), float(f[4])
        assert retire >= launch and all(float(x) >= 0 for x in f[5:10])
    assert sorted(seen) == sorted(ids)
    assert pix == sum(f.shape[1] * f.shape[2] for f in frames)
