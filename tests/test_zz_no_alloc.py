"""mdn_denoise_multiscale_static: the entry point for callers that cannot
allocate device memory (a plug-in whose host application owns all device
allocations, a real-time pipeline that may not allocate on the frame path).
Its scratch is a fixed 48 MiB static device array instead of a caller
workspace.  It runs the same kernels on the same inputs as
mdn_denoise_multiscale, so its results must be identical to that path's,
call after call, even though the array keeps the previous call's contents;
and once the first call on the device has looked up the array, a call must
not change the device's free memory.

Collected last on purpose (file name), and self-contained so that it also
passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import paper_1802_06130_gb300 as mdn
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mdn.build()
    raw = C.CDLL(mdn.build())
    f = raw.mdn_denoise_multiscale_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.POINTER(C.c_void_p),
                  C.c_int32, C.POINTER(mdn.Geometry), C.POINTER(mdn.BucketParams), C.c_void_p,
                  C.POINTER(C.c_void_p), C.c_void_p]
    raw.mdn_last_error.restype = C.c_char_p
    return mdn, raw


def _banks(seed, dtype, D=98, nb=2):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nb):
        b = rng.standard_normal((216, 3, D)).astype(np.float32) * 0.03
        b += (1.0 - b.sum(axis=2, keepdims=True)) / D
        out.append(torch.tensor(b, dtype=dtype, device="cuda"))
    return out


def _call_static(mdn, raw, x, banks, geom, bps, out):
    n, _, h, w = x.shape
    dt = mdn.F32 if x.dtype == torch.float32 else mdn.F16
    levels = 1 if geom.r_coarse < 0 else len(banks) + 1
    barr = (C.c_void_p * len(banks))(*[b.data_ptr() for b in banks])
    parr = (mdn.BucketParams * len(bps))(*bps)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return raw.mdn_denoise_multiscale_static(C.c_void_p(x.data_ptr()), dt, n, h, w, levels, barr, dt,
                                             C.byref(geom), parr, C.c_void_p(out.data_ptr()), None, stream)


@pytest.mark.parametrize("dtype", [torch.float16, torch.float32])
def test_static_scratch_matches_workspace_path(api, dtype):
    mdn, raw = api
    geom = mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    banks = _banks(3, dtype)
    # two calls in a row on different frames: the second one runs on scratch
    # that still holds the first call's data
    for seed, (h, w) in [(50000, (1080, 1920)), (50001, (721, 1283))]:
        z = torch.tensor(synth.noisy_pair(h, w, seed)[0], dtype=dtype, device="cuda")[None]
        ref = mdn.denoise_multiscale(z, banks, geom, bps)
        out = torch.full_like(z, float("nan"))
        rc = _call_static(mdn, raw, z, banks, geom, bps, out)
        assert rc == 0, raw.mdn_last_error()
        torch.cuda.synchronize()
        # same kernels, same inputs: identical results
        assert torch.equal(out, ref), (out.float() - ref.float()).abs().max().item()


def test_static_scratch_single_level_and_empty_batch(api):
    """A 1-level (single-scale) geometry needs no scratch at all, and an empty
    batch (n = 0) is a no-op that succeeds; both through the static entry."""
    mdn, raw = api
    geom = mdn.Geometry(2, -1)
    bps = [mdn.default_bparams(0)]
    banks = _banks(5, torch.float16, D=25, nb=1)
    for seed, (h, w) in [(50010, (256, 256)), (50011, (97, 131))]:
        z = torch.tensor(synth.noisy_pair(h, w, seed)[0], dtype=torch.float16, device="cuda")[None]
        ref = mdn.denoise_multiscale(z, banks, geom, bps)
        out = torch.full_like(z, float("nan"))
        rc = _call_static(mdn, raw, z, banks, geom, bps, out)
        assert rc == 0, raw.mdn_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    empty = torch.empty((0, 3, 64, 64), dtype=torch.float16, device="cuda")
    rc = _call_static(mdn, raw, empty, _banks(6, torch.float16), mdn.Geometry(3, 3),
                      [mdn.default_bparams(0), mdn.default_bparams(1)], torch.empty_like(empty))
    assert rc == 0, raw.mdn_last_error()


def test_static_scratch_allocates_nothing(api):
    """After a first call (which looks up the static array's address), further
    calls leave the device's free memory unchanged: no device allocation."""
    mdn, raw = api
    geom = mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    banks = _banks(7, torch.float16)
    z = torch.tensor(synth.noisy_pair(1080, 1920, 50020)[0], dtype=torch.float16, device="cuda")[None]
    out = torch.empty_like(z)
    assert _call_static(mdn, raw, z, banks, geom, bps, out) == 0, raw.mdn_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call_static(mdn, raw, z, banks, geom, bps, out) == 0, raw.mdn_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_rejects_oversize(api):
    mdn, raw = api
    geom = mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    banks = _banks(4, torch.float16)
    # eight 12 MP FP16 frames need ~330 MB of scratch, more than 48 MiB; the
    # size check runs before any device work, so tiny stand-in tensors suffice
    x = torch.zeros((1, 3, 2, 2), dtype=torch.float16, device="cuda")
    barr = (C.c_void_p * 2)(banks[0].data_ptr(), banks[1].data_ptr())
    parr = (mdn.BucketParams * 2)(*bps)
    rc = raw.mdn_denoise_multiscale_static(C.c_void_p(x.data_ptr()), mdn.F16, 8, 3024, 4032, 3, barr, mdn.F16,
                                           C.byref(geom), parr, C.c_void_p(x.data_ptr()), None, None)
    assert rc == 3
    assert b"48 MiB" in raw.mdn_last_error()
