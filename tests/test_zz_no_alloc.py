"""mdn_denoise_multiscale_static: the entry point for callers that cannot
allocate device memory (a plug-in whose host application owns all device
allocations, a real-time pipeline that may not allocate on the frame path).
Its scratch is a fixed 48 MiB static device array instead of a caller
workspace; its results must match mdn_denoise_multiscale, call after call,
even though the array keeps the previous call's contents.

Collected last on purpose (file name), and self-contained so that it also
passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-4, torch.float16: 2e-3}


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
    barr = (C.c_void_p * len(banks))(*[b.data_ptr() for b in banks])
    parr = (mdn.BucketParams * len(bps))(*bps)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return raw.mdn_denoise_multiscale_static(C.c_void_p(x.data_ptr()), dt, n, h, w, len(banks) + 1, barr, dt,
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
        err = (out.float() - ref.float()).abs().max().item()
        assert err <= TOL[dtype], err


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
