"""GPU check of lddmm_apply_K_noalloc, the K entry point for callers that cannot allocate GPU
memory (a host callback, a real-time loop, a process whose memory another pool holds): its
scratch is a fixed static device array.  Called through the C ABI twice in a row on new data and
compared with lddmm_apply_K (k_mode FP32) of a context, within the FP32 tolerance of the K tests;
also in place (dst = src) and at the limits (an axis of 512, exactly 2^21 voxels).  Kept in a
file collected last so that a failure here never hides the other tests."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import lddmm as L
    L.load()
    return L


def _noalloc(lib, src, dst, shape, h, alpha, gamma, stream):
    Z, Y, X = shape
    return lib.lddmm_apply_K_noalloc(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                     X, Y, Z, h[0], h[1], h[2], alpha, gamma,
                                     ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("shape,h,alpha,gamma", [((29, 20, 33), (1.0, 1.0, 1.0), 0.02, 1.0),
                                                 ((64, 48, 40), (1.0, 2.0, 0.5), 0.5, 1.7),
                                                 ((64, 64, 512), (1.0, 1.0, 1.0), 0.02, 1.0)])
def test_noalloc_matches_context_K_twice(L, shape, h, alpha, gamma, in_place):
    lib = L.load()
    Z, Y, X = shape
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream()
    p = L.default_params(X, Y, Z, hx=h[0], hy=h[1], hz=h[2], alpha=alpha, gamma=gamma, k_mode=0)
    zeros = np.zeros(shape, np.float32)
    with L.Lddmm(p, zeros, zeros, stream=stream) as ctx:
        for call in range(2):
            f = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
            ref = torch.empty_like(f)
            ctx.apply_K(f, ref)
            if in_place:
                out = f.clone()
                rc = _noalloc(lib, out, out, shape, h, alpha, gamma, stream)
            else:
                out = torch.full_like(f, float("nan"))
                rc = _noalloc(lib, f, out, shape, h, alpha, gamma, stream)
            assert rc == L.LDDMM_OK, lib.lddmm_last_error(None)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5, call


def test_noalloc_rejects_oversize_and_host_pointers(L):
    lib = L.load()
    f = torch.zeros((8, 8, 8), device="cuda")
    big = lib.lddmm_apply_K_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                    600, 8, 8, 1.0, 1.0, 1.0, 0.02, 1.0, None)
    assert big == L.LDDMM_ERR_INVALID_ARG
    assert b"512" in lib.lddmm_last_error(None)
    many = lib.lddmm_apply_K_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                     256, 256, 64, 1.0, 1.0, 1.0, 0.02, 1.0, None)
    assert many == L.LDDMM_ERR_INVALID_ARG
    assert b"2^21" in lib.lddmm_last_error(None)
    h = np.zeros((8, 8, 8), np.float32)
    host = lib.lddmm_apply_K_noalloc(ctypes.c_void_p(h.ctypes.data), ctypes.c_void_p(f.data_ptr()),
                                     8, 8, 8, 1.0, 1.0, 1.0, 0.02, 1.0, None)
    assert host == L.LDDMM_ERR_INVALID_ARG
