"""Pins of the §2.2 preprocessing in the FP64 oracle (CPU): histogram matching and the ball
morphology of the mask generation."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def P():
    from oracle import preprocess
    return preprocess


def _ball_mask(shape, c, r):
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    return ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) <= r * r


def test_matching_an_image_to_itself_is_the_identity(P):
    rng = np.random.default_rng(0)
    I = rng.gamma(2.0, 1.0, size=(10, 11, 12))
    M = np.ones(I.shape)
    xs, ys = P.match_nodes(I, M, I, M)
    assert np.array_equal(xs, ys)
    assert np.allclose(P.histogram_match(I, M, I, M), I, rtol=0, atol=1e-12)


def test_affine_intensity_change_is_recovered(P):
    """I1 = a I0 + b on the same voxels: every quantile of I1 is a q + b (the bins scale with
    the range), so the matched I0 equals I1 exactly up to rounding."""
    rng = np.random.default_rng(1)
    I0 = rng.normal(0.5, 0.15, size=(9, 10, 11))
    M = (rng.random(I0.shape) < 0.7).astype(float)
    I1 = 3.0 * I0 - 0.25
    out = P.histogram_match(I0, M, I1, M)
    assert np.allclose(out[M > 0], I1[M > 0], rtol=0, atol=1e-12)
    assert np.all(out[M == 0] == 0.0)


def test_quantiles_of_a_uniform_ramp(P):
    """Values 0..n-1, each once, with n a multiple of 32: every bin holds n/32 values, so the
    interpolated quantile at f lies within one bin width of f n."""
    n = 64 * 32
    v = np.arange(n, dtype=np.float64)
    w = (n - 1.0) / 32
    for f in (0.1, 0.25, 0.5, 0.8):
        assert abs(P._quantile(v, 0.0, n - 1.0, 32, f) - f * n) < w


def test_map_is_monotone_and_hits_the_nodes(P):
    rng = np.random.default_rng(2)
    I0 = rng.lognormal(0.0, 1.0, size=(8, 9, 10))
    I1 = rng.normal(2.0, 0.3, size=(8, 9, 10))
    M0 = np.ones(I0.shape)
    M1 = (rng.random(I1.shape) < 0.8).astype(float)
    xs, ys = P.match_nodes(I0, M0, I1, M1)
    assert np.all(np.diff(xs) >= 0) and np.all(np.diff(ys) >= 0)
    assert np.allclose(P._map(xs, xs, ys), ys)
    out = P.histogram_match(I0, M0, I1, M1)
    order = np.argsort(I0.ravel())
    assert np.all(np.diff(out.ravel()[order]) >= -1e-12)


@pytest.mark.parametrize("r", [1, 2])
def test_morphology_equals_brute_force(P, r):
    rng = np.random.default_rng(3 + r)
    m = _ball_mask((14, 15, 16), (7.5, 7.0, 6.5), 5.2) | (rng.random((14, 15, 16)) < 0.04)
    m &= ~(rng.random(m.shape) < 0.03)
    opened = P.dilate_brute(P.erode_brute(m, r), r)
    closed = P.erode_brute(P.dilate_brute(opened, r + 1), r + 1)
    got = P.mask_morphology(m.astype(float), 0.5, r, r + 1)
    assert np.array_equal(got, closed)


def test_opening_removes_grains_and_keeps_a_large_ball(P):
    big = _ball_mask((24, 24, 24), (11.5, 11.5, 11.5), 8.0)
    m = big.copy()
    m[1, 1, 1] = m[2, 20, 5] = True              # isolated grains
    got = P.mask_morphology(m.astype(float), 0.5, 1, 0)
    assert not got[1, 1, 1] and not got[2, 20, 5]
    assert np.array_equal(got, P.dilate_brute(P.erode_brute(big, 1), 1))


def test_threshold_is_strict(P):
    """The rough mask is [I > threshold]: voxels exactly at the threshold are background."""
    I = np.zeros((5, 5, 5))
    I[1:4, 1:4, 1:4] = 0.5
    I[2, 2, 2] = 0.7
    m = P.mask_morphology(I, 0.5, 0, 0)
    assert m.sum() == 1 and m[2, 2, 2]
