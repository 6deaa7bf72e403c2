"""GPU parity of the §2.7 measures (surface distances, landmark error) through the C ABI against
the FP64 oracle.  With unit spacing every distance is the square root of an integer on both
sides, so the Hausdorff and median distances must agree exactly; with anisotropic spacing the
GPU searches in FP32 and recomputes the winner in FP64 (agreement to 1e-6 relative)."""
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
def OM():
    from oracle import metrics
    return metrics


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _registered(L, synth, shape, steps, h=(1.0, 1.0, 1.0)):
    Z, Y, X = shape
    pair = synth.ellipsoid_pair(shape=shape, centre=((X - 1) / 2, (Y - 1) / 2, (Z - 1) / 2),
                                semi_axes=(X / 3.2, Y / 4.0, Z / 4.5), width=X / 5.0,
                                amplitude=2.0, seed=3)
    p = L.default_params(X, Y, Z, hx=h[0], hy=h[1], hz=h[2], T=4, k_mode=1)
    ctx = L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M))
    for _ in range(steps):
        ctx.step(want_energy=False)
    lab = ctx.transfer_labels(_dev((pair.I0 > 0.5).astype(np.uint16)),
                              torch.empty(shape, dtype=torch.int16, device="cuda"))
    warped = (lab.cpu().numpy() != 0).astype(np.uint8)
    return ctx, pair, warped


@pytest.mark.parametrize("shape,h,steps", [((24, 26, 28), (1.0, 1.0, 1.0), 0),
                                           ((24, 26, 28), (1.0, 1.0, 1.0), 6),
                                           ((20, 22, 32), (1.0, 1.25, 0.8), 4)])
def test_surface_distances_match_oracle(L, OM, shape, h, steps):
    from paper_1605_02060_gb300 import synth
    ctx, pair, warped = _registered(L, synth, shape, steps, h)
    target = (pair.I1 > 0.5).astype(np.uint8)
    with ctx:
        hd, md, na, nb = ctx.surface_distance(_dev(warped), target)   # device and host inputs
    ohd, omd = OM.surface_distances(warped.astype(bool), target.astype(bool), h)
    assert na == int(OM.surface(warped.astype(bool)).sum())
    assert nb == int(OM.surface(target.astype(bool)).sum())
    if h == (1.0, 1.0, 1.0):
        assert hd == ohd and md == omd, (hd, ohd, md, omd)
    else:
        assert abs(hd - ohd) <= 1e-6 * ohd and abs(md - omd) <= 1e-6 * max(omd, 1e-12)


def test_surface_distance_special_cases(L, OM):
    shape = (8, 9, 10)
    a = np.zeros(shape, np.float32)
    p = L.default_params(10, 9, 8)
    with L.Lddmm(p, a, a) as ctx:
        A = np.zeros(shape, np.uint8)
        B = np.zeros(shape, np.uint8)
        A[2, 1, 1] = 1
        B[2, 5, 4] = 1                       # offset (3, 4, 0): 5 voxels
        assert ctx.surface_distance(A, B)[:2] == (5.0, 5.0)
        C = np.zeros(shape, np.uint8)
        C[1:6, 2:7, 1:8] = 1
        assert ctx.surface_distance(C, C)[:2] == (0.0, 0.0)
        with pytest.raises(L.LddmmError) as ei:
            ctx.surface_distance(A, np.zeros(shape, np.uint8))
        assert ei.value.code == L.LDDMM_ERR_INVALID_ARG


def test_landmark_errors_match_oracle(L, OM):
    from paper_1605_02060_gb300 import synth
    shape = (20, 22, 24)
    ctx, pair, _ = _registered(L, synth, shape, 5)
    rng = np.random.default_rng(11)
    xk = rng.uniform(2, 18, size=(64, 3)).astype(np.float32)
    yk = (xk + rng.normal(0, 1.5, size=(64, 3))).astype(np.float32)
    with ctx:
        e = ctx.landmark_error(xk, yk)
        u01 = ctx.get_field(L.LDDMM_FIELD_U01)
        e_dev = ctx.landmark_error(_dev(xk), _dev(yk), torch.empty(64, dtype=torch.float64, device="cuda"))
    ref = OM.landmark_errors(u01.astype(np.float64), xk, yk)
    assert np.max(np.abs(e - ref)) < 1e-5
    assert np.array_equal(e, e_dev.cpu().numpy())


def test_full_size_surface_distance(L, OM):
    """The brain-shaped pair at 264x160x228: the atlas mask against the target mask."""
    from paper_1605_02060_gb300 import synth
    pair, atlas = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    A = (pair.I0 > 0.5).astype(np.uint8)
    B = (pair.I1 > 0.5).astype(np.uint8)
    a = np.zeros(A.shape, np.float32)
    p = L.default_params(264, 160, 228)
    with L.Lddmm(p, a, a) as ctx:
        hd, md, na, nb = ctx.surface_distance(_dev(A), _dev(B))
    ohd, omd = OM.surface_distances(A.astype(bool), B.astype(bool))
    assert hd == ohd and md == omd, (hd, ohd, md, omd)
