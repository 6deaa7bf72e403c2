"""Pins for the FP64 oracle of the warm-start network: the convolution against a library
correlation, adjoint (dot-product) identities for every backward operator, finite differences
through the whole encoder-decoder, and Adam's closed-form first step."""
import numpy as np
import pytest

from oracle import surrogate as S


def _rng(s):
    return np.random.default_rng(s)


def test_conv3d_matches_scipy_correlate_with_zero_padding():
    from scipy import ndimage
    rng = _rng(0)
    x = rng.standard_normal((1, 2, 6, 6, 6))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    y = S.conv3d(x, w, b)
    for o in range(3):
        ref = b[o] + sum(ndimage.correlate(x[0, i], w[o, i].reshape(3, 3, 3), mode="constant")
                         for i in range(2))
        np.testing.assert_allclose(y[0, o], ref, atol=1e-12)


@pytest.mark.parametrize("k", [1, 3])
def test_conv_backward_operators_are_adjoints(k):
    rng = _rng(1)
    x = rng.standard_normal((2, 3, 6, 6, 6))
    w = rng.standard_normal((4, 3, k ** 3))
    dy = rng.standard_normal((2, 4, 6, 6, 6))
    # <conv(x), dy> = <x, dgrad(dy)>
    lhs = (S.conv3d(x, w) * dy).sum()
    np.testing.assert_allclose(lhs, (x * S.conv3d_dgrad(dy, w)).sum(), rtol=1e-12)
    # <conv(x; dw), dy> = <dw, wgrad(x, dy)> and db = sum dy
    dwd = rng.standard_normal(w.shape)
    gw, gb = S.conv3d_wgrad(x, dy, k)
    np.testing.assert_allclose((S.conv3d(x, dwd) * dy).sum(), (dwd * gw).sum(), rtol=1e-12)
    np.testing.assert_allclose(gb, dy.sum(axis=(0, 2, 3, 4)), rtol=1e-12)


def test_pool_and_upsample_adjoints_and_values():
    rng = _rng(2)
    x = rng.standard_normal((1, 2, 4, 4, 4))
    y = rng.standard_normal((1, 2, 2, 2, 2))
    np.testing.assert_allclose((S.pool2(x) * y).sum(), (x * S.pool2_bwd(y)).sum(), rtol=1e-12)
    np.testing.assert_allclose((S.up2(y) * x).sum(), (y * S.up2_bwd(x)).sum(), rtol=1e-12)
    assert S.pool2(x)[0, 1, 1, 0, 1] == x[0, 1, 2:4, 0:2, 2:4].mean()
    assert S.up2(y)[0, 0, 3, 2, 1] == y[0, 0, 1, 1, 0]


def test_network_gradient_matches_finite_differences():
    rng = _rng(3)
    chans = (3, 4, 5)
    shapes = S.layer_shapes(chans, 2, 3)
    params = [(0.3 * rng.standard_normal((co, ci, k ** 3)), 0.1 * rng.standard_normal(co))
              for co, ci, k in shapes]
    x = rng.standard_normal((2, 2, 8, 8, 8))
    t = rng.standard_normal((2, 3, 8, 8, 8))
    y, acts = S.net_forward(params, x, chans)
    loss, dy = S.mse(y, t)
    grads = S.net_backward(params, acts, dy, chans)
    eps = 1e-7      # small enough that no ReLU changes side along the probe direction
    for li in range(len(params)):
        d = rng.standard_normal(params[li][0].shape)
        db = rng.standard_normal(params[li][1].shape)

        def loss_at(s):
            p2 = list(params)
            p2[li] = (params[li][0] + s * d, params[li][1] + s * db)
            return S.mse(S.net_forward(p2, x, chans)[0], t)[0]
        fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
        an = (grads[li][0] * d).sum() + (grads[li][1] * db).sum()
        np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-12)


def test_adam_first_step_is_signed_lr():
    g = np.array([0.5, -2.0, 1e-3])
    w, m, v = S.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-12, 1)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-6)


def test_adam_epsilon_is_added_to_the_root():
    """Adam's denominator is sqrt(v_hat) + eps (Kingma and Ba): a first step with |g| = eps moves
    by lr / 2, and a second step with the same gradient again by lr |g| / (|g| + eps)."""
    eps = 1e-6
    g = np.array([eps, -eps])
    w, m, v = S.adam(np.zeros(2), g, np.zeros(2), np.zeros(2), 0.01, 0.9, 0.999, eps, 1)
    np.testing.assert_allclose(w, -0.005 * np.sign(g), rtol=1e-9)
    w, m, v = S.adam(w, g, m, v, 0.01, 0.9, 0.999, eps, 2)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-9)


def test_layer_shapes_of_the_four_level_network():
    sh = S.layer_shapes((16, 32, 64, 128), 2, 3)
    assert sh[0] == (16, 2, 3) and sh[7] == (128, 128, 3)
    assert sh[8] == (64, 128 + 64, 3) and sh[-2] == (16, 16, 3) and sh[-1] == (3, 16, 1)
    assert len(sh) == 15
