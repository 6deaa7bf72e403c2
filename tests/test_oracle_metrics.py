"""Pins of the surface and landmark measures of §2.7 in the FP64 oracle (CPU)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def M():
    from oracle import metrics
    return metrics


def _ball(shape, c, r):
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    return ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) <= r * r


def test_surface_of_a_box_is_its_shell(M):
    m = np.zeros((7, 8, 9), bool)
    m[1:6, 2:7, 1:8] = True
    s = M.surface(m)
    inner = np.zeros_like(m)
    inner[2:5, 3:6, 2:7] = True
    assert np.array_equal(s, m & ~inner)
    # a mask touching the grid faces: the face voxels are surface
    full = np.ones((3, 4, 5), bool)
    sf = M.surface(full)
    assert sf.sum() == full.size - 1 * 2 * 3 and not sf[1, 1:3, 1:4].any()


def test_single_voxels_give_the_3_4_5_distance(M):
    A = np.zeros((6, 9, 9), bool)
    B = np.zeros_like(A)
    A[2, 1, 1] = True
    B[2, 5, 4] = True            # offset (3, 4, 0) voxels
    hd, md = M.surface_distances(A, B)
    assert hd == 5.0 and md == 5.0
    hd, md = M.surface_distances(A, B, h=(2.0, 0.5, 1.0))   # (6, 2, 0) -> sqrt(40)
    assert abs(hd - np.sqrt(40.0)) < 1e-12 and abs(md - np.sqrt(40.0)) < 1e-12


def test_identical_masks_are_zero_and_distances_are_symmetric(M):
    A = _ball((16, 17, 18), (8.3, 7.9, 8.1), 5.2)
    B = _ball((16, 17, 18), (9.1, 8.4, 7.2), 4.1)
    assert M.surface_distances(A, A) == (0.0, 0.0)
    assert M.surface_distances(A, B) == M.surface_distances(B, A)


@pytest.mark.parametrize("seed,h", [(0, (1.0, 1.0, 1.0)), (1, (0.5, 1.25, 2.0)), (2, (1.0, 1.0, 3.0))])
def test_distance_transform_route_equals_brute_force(M, seed, h):
    rng = np.random.default_rng(seed)
    A = rng.random((9, 10, 11)) < 0.3
    B = _ball((9, 10, 11), (5.0, 4.5, 4.0), 3.3) | (rng.random((9, 10, 11)) < 0.05)
    hd, md = M.surface_distances(A, B, h)
    hb, mb = M.brute_surface_distances(A, B, h)
    assert abs(hd - hb) < 1e-12 and abs(md - mb) < 1e-12


def test_concentric_balls(M):
    """Ball surfaces of radii 7 and 4 about the same centre: every directed distance lies
    within a voxel diagonal of the radius difference 3."""
    shape = (24, 24, 24)
    A, B = _ball(shape, (11.5, 11.5, 11.5), 7.0), _ball(shape, (11.5, 11.5, 11.5), 4.0)
    hd, md = M.surface_distances(A, B)
    assert 3.0 - np.sqrt(3) <= md <= 3.0 + np.sqrt(3)
    assert 3.0 - np.sqrt(3) <= hd <= 3.0 + 2 * np.sqrt(3)


def test_landmark_error_identity_and_translation(M):
    rng = np.random.default_rng(3)
    shape = (12, 13, 14)
    u = np.zeros((3,) + shape)
    xk = rng.uniform(1, 10, size=(5, 3))
    assert np.allclose(M.landmark_errors(u, xk, xk), 0.0)
    u[0] += 1.5; u[1] -= 0.5; u[2] += 2.0            # phi(x) = x + (1.5, -0.5, 2)
    yk = xk + np.array([1.5, -0.5, 2.0])
    assert np.allclose(M.landmark_errors(u, xk, yk), 0.0, atol=1e-12)
    e = M.landmark_errors(u, xk, xk, h=(2.0, 1.0, 0.5))
    assert np.allclose(e, np.sqrt(3.0 ** 2 + 0.5 ** 2 + 1.0 ** 2))
