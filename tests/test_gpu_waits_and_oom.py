"""Failure paths on the GPU, made without faulting it.

* A device allocation that fails inside lddmm_create (injected by LDDMM_TEST_FAIL_ALLOC=k, which
  fails the k-th allocation as if the device were out of memory): the call returns
  LDDMM_ERR_OOM with its reason, and every allocation made before it is released.
* A bounded wait inside the tensor-core DFT pipeline that runs out (LDDMM_TEST_POLL_LIMIT=1: each
  wait gives up after one probe): the kernel drains its copies, frees its tensor memory and sets
  its error flag; the step returns LDDMM_ERR_TIMEOUT; the same context keeps working for calls
  that do not use that pipeline, and a new context without the hook steps normally.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import lddmm as L
    L.load()
    return L


@pytest.fixture(scope="module")
def pair():
    from paper_1605_02060_gb300 import synth
    return synth.ellipsoid_pair(shape=(64, 64, 64), centre=(31.5, 31.5, 31.5), semi_axes=(20, 16, 14),
                                width=12.0, amplitude=3.0, seed=0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_injected_allocation_failure_returns_oom_and_releases_everything(L, pair, monkeypatch):
    I0, I1, M = _dev(pair.I0), _dev(pair.I1), _dev(pair.M)
    p = L.default_params(64, 64, 64, T=10, k_mode=1, flags=1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 5, 12, 20):
        monkeypatch.setenv("LDDMM_TEST_FAIL_ALLOC", str(k))
        with pytest.raises(L.LddmmError) as ei:
            L.Lddmm(p, I0, I1, M)
        assert ei.value.code == L.LDDMM_ERR_OOM, (k, ei.value)
        assert "allocation" in str(ei.value)
        # nothing allocated before the failing call is kept (a context holds ~300 MB here)
        assert abs(torch.cuda.mem_get_info()[0] - free0) < 16 << 20, k
    monkeypatch.setenv("LDDMM_TEST_FAIL_ALLOC", "1000")     # beyond the last allocation
    with L.Lddmm(p, I0, I1, M) as ctx:
        assert np.isfinite(ctx.step()["total"])
    monkeypatch.delenv("LDDMM_TEST_FAIL_ALLOC")
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 16 << 20


def test_device_wait_limit_aborts_the_pipeline_and_context_survives(L, pair, monkeypatch):
    I0, I1, M = _dev(pair.I0), _dev(pair.I1), _dev(pair.M)
    p = L.default_params(64, 64, 64, T=4, k_mode=1)
    with L.Lddmm(p, I0, I1, M) as ref:
        e0 = ref.energy()["total"]
        e_ok = ref.step()["total"]
    monkeypatch.setenv("LDDMM_TEST_POLL_LIMIT", "1")
    ctx = L.Lddmm(p, I0, I1, M)
    monkeypatch.delenv("LDDMM_TEST_POLL_LIMIT")
    try:
        with pytest.raises(L.LddmmError) as ei:
            for _ in range(3):          # one probe per wait: the first pipeline wait gives up
                ctx.step()
        assert ei.value.code == L.LDDMM_ERR_TIMEOUT
        assert "gave up" in str(ei.value)
        # the context is usable: the flows and energies do not use the aborted pipeline
        ctx.set_velocity(np.zeros((4, 3, 64, 64, 64), np.float32))
        assert ctx.energy()["total"] == pytest.approx(e0, rel=1e-12)
    finally:
        ctx.close()
    torch.cuda.synchronize()
    with L.Lddmm(p, I0, I1, M) as fresh:
        assert fresh.step()["total"] == pytest.approx(e_ok, rel=1e-12)
