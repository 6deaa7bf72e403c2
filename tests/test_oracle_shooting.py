"""Pins of the geodesic-shooting oracle (CPU)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    from oracle import shooting
    return shooting


def _bump(shape, c, s, amp):
    """A velocity field localised away from the grid faces (components x, y, z)."""
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    g = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    return np.stack([amp[0] * g, amp[1] * g * (x - c[0]) / s, amp[2] * g * (y - c[1]) / s])


def test_ad_star_on_single_modes(S):
    """v = (a sin kx, 0, 0), m = (b cos kx, 0, 0): with central differences D sin = sin(k) cos,
    D cos = -sin(k) sin, so (ad*_v m)_x = 2 m Dv + v Dm = a b sin(k) (2 cos^2 - sin^2); and
    v = (0, f(x), 0), m = (0, g(x), 0): (ad*_v m)_x = (D f) g, the y and z parts vanish."""
    shape = (4, 5, 16)
    x = np.arange(16)[None, None, :] * np.ones(shape)
    k = 2 * np.pi * 3 / 16
    h = (1.0, 1.0, 1.0)
    v = np.zeros((3,) + shape)
    m = np.zeros((3,) + shape)
    v[0] = 0.7 * np.sin(k * x)
    m[0] = 1.3 * np.cos(k * x)
    got = S.ad_star(v, m, h)
    ref = 0.7 * 1.3 * np.sin(k) * (2 * np.cos(k * x) ** 2 - np.sin(k * x) ** 2)
    assert np.allclose(got[0], ref, atol=1e-12) and np.allclose(got[1:], 0.0)
    v[:] = 0.0
    m[:] = 0.0
    v[1] = np.sin(k * x)
    m[1] = 2.0 + np.cos(2 * k * x)
    got = S.ad_star(v, m, h)
    assert np.allclose(got[0], np.sin(k) * np.cos(k * x) * m[1], atol=1e-12)
    assert np.allclose(got[1:], 0.0, atol=1e-12)


def test_transport_of_momentum_under_a_translation_and_a_stretch(S):
    """u = const: |D phi| = 1, D phi = I, so the momentum is only moved; u = (s - 1) x along x:
    D phi = diag(s, 1, 1), so m_x is scaled by s^2 and m_y, m_z by s (|D phi| = s)."""
    shape = (6, 7, 20)
    rng = np.random.default_rng(0)
    m0 = np.broadcast_to(rng.normal(size=(3, 1, 1, 1)), (3,) + shape).copy()
    u = np.zeros((3,) + shape)
    u[0] = 0.75
    assert np.allclose(S.transport_momentum(m0, u, (1.0, 1.0, 1.0)), m0, atol=1e-12)
    x = np.arange(20)[None, None, :] * np.ones(shape)
    u[0] = 0.1 * (x - 10.0)                     # phi_x = 1.1 x - 1 (stays inside near x = 10)
    got = S.transport_momentum(m0, u, (1.0, 1.0, 1.0))[:, :, :, 8:12]
    s = 1.1
    assert np.allclose(got[0], s * s * m0[0, :, :, 8:12], atol=1e-12)
    assert np.allclose(got[1:], s * m0[1:, :, :, 8:12], atol=1e-12)


def test_transport_under_a_shear_at_anisotropic_spacing(S):
    """u_x = c y (voxels) with spacing h: in physical units d phi_x / d y = c h_x / h_y, so
    D phi = [[1, c hx/hy, 0], [0, 1, 0], [0, 0, 1]] and |D phi| = 1; for a constant m0,
    (D phi)^T m0 = (m_x, m_y + c (hx/hy) m_x, m_z).  A transposed Jacobian or an inverted
    spacing ratio gives a different m_x or m_y."""
    shape = (5, 12, 9)
    h = (0.5, 2.0, 1.0)
    c = 0.2
    m0 = np.broadcast_to(np.array([1.5, -0.7, 0.4])[:, None, None, None], (3,) + shape).copy()
    y = np.arange(12)[None, :, None] * np.ones(shape)
    u = np.zeros((3,) + shape)
    u[0] = c * (y - 6.0)
    got = S.transport_momentum(m0, u, h)[:, :, 1:-1, 3:6]   # away from the clamped faces
    r = c * h[0] / h[1]
    assert np.allclose(got[0], 1.5, atol=1e-12)
    assert np.allclose(got[1], -0.7 + r * 1.5, atol=1e-12)
    assert np.allclose(got[2], 0.4, atol=1e-12)


def test_zero_and_constant_fields_are_fixed_points(S):
    from oracle import lddmm as O
    p = O.Params(T=5)
    shape = (6, 7, 8)
    assert not S.shoot(np.zeros((3,) + shape), p).any()
    v0 = np.ones((3,) + shape) * np.array([0.3, -1.2, 2.0])[:, None, None, None]
    assert np.allclose(S.shoot(v0, p), v0[None], atol=1e-12)


def test_the_nonlinearity_is_quadratic(S):
    """The transported momentum departs from m_0 by O(|v|^2): v_j(eps v0) - eps v0 = O(eps^2),
    so halving eps quarters the deviation (a dropped K, or a momentum that is not L^T L v,
    would leave a first-order term)."""
    from oracle import lddmm as O
    p = O.Params(T=4, alpha=0.3)
    v0 = _bump((16, 16, 16), (7.5, 8.0, 7.0), 3.0, (2.0, 1.0, -1.0))
    r = [np.linalg.norm(S.shoot(e * v0, p)[-1] - e * v0) for e in (0.2, 0.1)]
    assert 3.6 < r[0] / r[1] < 4.4


def test_transport_agrees_with_the_eulerian_equation(S):
    """Away from the faces, the momentum transported by the flow and forward Euler on
    dm/dt = -ad*_v m solve the same equation with different O(h^2) spatial errors: at small
    amplitude they agree to within 15% of the change of v for a field of width 4 voxels, and
    the gap narrows as the field gets smoother (width 3 -> 4)."""
    from oracle import lddmm as O
    p = O.Params(T=16, alpha=0.3)
    gap = []
    for s in (3.0, 4.0):
        v0 = _bump((24, 24, 24), (11.5, 12.0, 11.0), s, (0.6, 0.4, -0.3))
        a = S.shoot(v0, p)[-1]
        b = S.shoot_eulerian(v0, p)[-1]
        gap.append(np.abs(a - b).max() / np.abs(a - v0).max())
    assert gap[1] < 0.15 and gap[1] < 0.8 * gap[0]
