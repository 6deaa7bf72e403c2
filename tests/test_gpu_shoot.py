"""GPU parity of geodesic shooting (EPDiff in its transport form) against the FP64 oracle.

v_0 is set from the input unchanged; v_1..v_{T-1} come from K |D phi| (D phi)^T (m_0 o phi)
with phi from the forward semi-Lagrangian steps.  Tolerance: relative L2 <= 1e-4 per sample,
the bound of one K application, which dominates the FP32 rounding of the transport.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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
def O():
    from oracle import lddmm as O
    from oracle import shooting as S
    return O, S


@pytest.fixture(scope="module")
def synth():
    from paper_1605_02060_gb300 import synth
    return synth


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape,T,h,kmode", [((32, 32, 32), 4, (1, 1, 1), 0),
                                             ((32, 32, 32), 4, (1, 1, 1), 1),
                                             ((20, 17, 23), 3, (1.0, 1.25, 0.8), 1),
                                             ((8, 10, 260), 4, (1, 1, 1), 1)])
def test_shoot_matches_oracle(L, O, synth, shape, T, h, kmode):
    Or, S = O
    Z, Y, X = shape
    pair = synth.ellipsoid_pair(shape=shape, seed=0)
    v0 = synth.smooth_velocity(1, shape, 3.0, seed=11)[0]
    p = L.default_params(X, Y, Z, T=T, hx=h[0], hy=h[1], hz=h[2], k_mode=kmode)
    ref = S.shoot(v0, Or.Params(T=T, h=h))
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.shoot(_dev(v0))
        v = ctx.get_velocity()
        ctx.shoot(np.ascontiguousarray(v0))          # host input, same result
        vh = ctx.get_velocity()
    assert np.array_equal(v[0], v0)
    assert np.array_equal(v, vh)
    for j in range(1, T):
        assert _rel(ref[j], v0) > 1e-2               # the geodesic moves away from v_0
        assert _rel(v[j] - v0, ref[j] - v0) < 1e-3, j
        assert _rel(v[j], ref[j]) < 1e-4, j


def test_shoot_rejects_bf16_storage_and_rk4(L, synth):
    shape = (16, 16, 16)
    pair = synth.ellipsoid_pair(shape=shape, seed=0)
    v0 = _dev(synth.smooth_velocity(1, shape, 1.0, seed=1)[0])
    for kw in ({"storage": 1}, {"flags": 4}):
        p = L.default_params(16, 16, 16, T=3, **kw)
        with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
            with pytest.raises(L.LddmmError) as ei:
                ctx.shoot(v0)
            assert ei.value.code == L.LDDMM_ERR_INVALID_ARG


def test_shoot_degenerate_cases(L, synth):
    """T = 1 keeps v_0 alone; v_0 = 0 shoots the zero field (no momentum)."""
    shape = (16, 12, 20)
    pair = synth.ellipsoid_pair(shape=shape, seed=0)
    v0 = synth.smooth_velocity(1, shape, 2.0, seed=3)[0]
    p = L.default_params(20, 12, 16, T=1)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.shoot(_dev(v0))
        assert np.array_equal(ctx.get_velocity()[0], v0)
    p = L.default_params(20, 12, 16, T=4)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.set_velocity(_dev(np.ones((4, 3) + shape, np.float32)))
        ctx.shoot(_dev(np.zeros_like(v0)))
        assert not ctx.get_velocity().any()


def test_shoot_full_size_constant_field(L):
    """At 264 x 160 x 228, T = 10, bf16x3 K (the benchmark's configuration): a spatially
    constant v_0 is a fixed point of the shooting (the displacement stays constant, so
    D phi = I and m_0 o phi = m_0 = gamma^2 v_0, and K m_0 = v_0)."""
    shape = (228, 160, 264)
    ones = torch.ones(shape, device="cuda")
    p = L.default_params(264, 160, 228, T=10, k_mode=1)
    c = torch.tensor([0.8, -1.5, 2.25], device="cuda")
    v0 = (c[:, None, None, None] * torch.ones((3,) + shape, device="cuda")).contiguous()
    with L.Lddmm(p, ones, ones, ones) as ctx:
        ctx.shoot(v0)
        v = torch.empty((10, 3) + shape, device="cuda")
        ctx.get_velocity(v)
    err = (v - v0[None]).abs().max().item()
    assert err <= 1e-4 * 2.25, err
