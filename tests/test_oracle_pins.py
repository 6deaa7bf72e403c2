"""Pins for the FP64 oracle: closed forms, invariants, library cross-checks and brute force.

Each test fixes a property that the paper's method (§2.4 energy and operator L, the Beg et al.
2005 gradient cited there, §2.5 label pull-back) or plain mathematics determines, chosen so that
a dropped term, a wrong sign, a wrong index or a transposed operand in the oracle fails one of
them.  None of these tests touches the CUDA library.
"""
import math
import os

import numpy as np
import pytest

from oracle import lddmm as O
from paper_1605_02060_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s=0):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- interpolation and stencils

def test_trilinear_reproduces_affine_functions():
    rng = _rng(1)
    Z, Y, X = 7, 9, 11
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    a, b, c, d = 0.7, -1.3, 2.1, 0.25
    f = a * gx + b * gy + c * gz + d
    qx = rng.uniform(0, X - 1, 500)
    qy = rng.uniform(0, Y - 1, 500)
    qz = rng.uniform(0, Z - 1, 500)
    got = O.trilinear(f, qx, qy, qz)
    np.testing.assert_allclose(got, a * qx + b * qy + c * qz + d, rtol=0, atol=1e-12)


def test_trilinear_matches_scipy_map_coordinates_with_clamp():
    from scipy import ndimage
    rng = _rng(2)
    f = rng.standard_normal((6, 8, 10))
    q = [rng.uniform(-3, n + 2, 400) for n in (10, 8, 6)]     # includes points outside
    got = O.trilinear(f, q[0], q[1], q[2])
    ref = ndimage.map_coordinates(f, [q[2], q[1], q[0]], order=1, mode="nearest")
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_fd_gradient_exact_on_linear_and_central_inside():
    Z, Y, X = 5, 6, 7
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    g = O.fd_gradient(3 * gx - 2 * gy + 0.5 * gz)
    np.testing.assert_allclose(g[0], 3.0, atol=1e-12)
    np.testing.assert_allclose(g[1], -2.0, atol=1e-12)
    np.testing.assert_allclose(g[2], 0.5, atol=1e-12)
    q = gx.astype(float) ** 2            # d/dx x^2 = 2x inside (central), one-sided at faces
    gq = O.fd_gradient(q)[0]
    np.testing.assert_allclose(gq[:, :, 1:-1], 2 * gx[:, :, 1:-1], atol=1e-12)
    np.testing.assert_allclose(gq[:, :, 0], 1.0, atol=1e-12)
    np.testing.assert_allclose(gq[:, :, -1], 2 * (X - 1) - 1, atol=1e-12)


def test_jacobian_det_of_affine_map():
    rng = _rng(3)
    A = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    Z, Y, X = 6, 7, 8
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    P = np.stack([gx, gy, gz]).astype(float)
    u = np.einsum("de,exyz->dxyz", A - np.eye(3), P) + np.array([0.3, -0.1, 0.2])[:, None, None, None]
    det = O.jacobian_det(u)
    np.testing.assert_allclose(det, np.linalg.det(A), rtol=1e-12)


# ---------------------------------------------------------------- flows

def _blob_pair(shape=(10, 12, 14)):
    Z, Y, X = shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    I0 = np.exp(-((gx - X / 2) ** 2 / 12 + (gy - Y / 2) ** 2 / 9 + (gz - Z / 2) ** 2 / 7))
    I1 = np.exp(-((gx - X / 2 - 1) ** 2 / 10 + (gy - Y / 2) ** 2 / 9 + (gz - Z / 2 + 0.5) ** 2 / 8))
    return I0, I1


def test_zero_velocity_gives_identity_maps():
    I0, I1 = _blob_pair()
    p = O.Params(T=4)
    v = np.zeros((4, 3) + I0.shape)
    r = O.lddmm_step(v, I0, I1, None, p)
    assert np.all(r.u10 == 0) and np.all(r.u01 == 0)
    assert r.min_det == 1.0
    np.testing.assert_array_equal(r.J0T, I0)
    for j in range(4):
        np.testing.assert_array_equal(r.J1[j], I1)
        np.testing.assert_array_equal(r.W[j], 1.0)
    assert r.E_reg == 0.0
    np.testing.assert_allclose(r.E_data, ((I0 - I1) ** 2).sum() / p.sigma ** 2, rtol=1e-14)


def test_first_step_residual_in_closed_form():
    """From v = 0 the maps are the identity, so b_j = (2/sigma^2) M (I0 - I1) grad_h I0 for every
    j and v_1 = eps K b (Beg's gradient 2v - K b at v = 0).  I0 is a quadratic, on which central
    differences are exact: inside the grid grad_h I0 = (0.01 (2x - z) / hx, 0.04 y / hy,
    -0.01 x / hz).  Anisotropic h and a random weight M make a wrong sign, a dropped weight or
    spacing, or swapped components fail."""
    shape = (6, 7, 8)
    h = (0.5, 2.0, 1.25)
    p = O.Params(T=3, h=h)
    rng = _rng(11)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    I0 = 0.01 * (x * x + 2 * y * y - z * x) + 0.3
    I1 = rng.uniform(0.0, 1.0, shape)
    M = rng.uniform(0.2, 1.0, shape)
    r = O.lddmm_step(np.zeros((3, 3) + shape), I0, I1, M, p)
    g = [0.01 * (2 * x - z) / h[0], 0.04 * y / h[1], -0.01 * x / h[2]]
    inner = (slice(1, -1),) * 3
    for j in range(3):
        for e in range(3):
            ref = 2.0 / p.sigma ** 2 * M * (I0 - I1) * g[e]
            np.testing.assert_allclose(r.b[j, e][inner], ref[inner], rtol=1e-12, atol=1e-12)
        for e in range(3):
            np.testing.assert_allclose(r.v_new[j, e], p.epsilon * O.apply_K(r.b[j, e], p.alpha,
                                                                           p.gamma, h),
                                       rtol=1e-12, atol=1e-15)


def test_empty_mask_update_is_pure_shrinkage():
    """With M = 0 there is no residual (b = 0), so Beg's gradient is 2 v and one step gives
    v_1 = (1 - 2 eps) v exactly, with E_data = 0."""
    shape = (6, 5, 7)
    I0, I1 = _blob_pair(shape)
    v = _rng(12).normal(size=(3, 3) + shape)
    p = O.Params(T=3, h=(1.0, 0.5, 2.0))
    r = O.lddmm_step(v, I0, I1, np.zeros(shape), p)
    assert r.E_data == 0.0 and not r.b.any()
    np.testing.assert_allclose(r.v_new, (1.0 - 2.0 * p.epsilon) * v, rtol=1e-15, atol=0)


def test_W_carries_the_jacobian_of_an_affine_flow():
    """For v_j(x) = A (x - c) the backward maps are affine, phi_{j,1}(x) = B^(T-j) (x - c) + c with
    B = I + dt A (trilinear interpolation and central differences are exact on affine fields), so
    away from the clamped faces W_j = M det(B)^(T-j) for a constant M."""
    n, T = 20, 4
    shape = (n, n, n)
    A = np.array([[0.03, -0.02, 0.01], [0.015, -0.025, 0.02], [-0.01, 0.02, 0.02]])
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64)] * 3, indexing="ij")
    q = np.stack([x - c, y - c, z - c])
    vel = np.einsum("de,e...->d...", A, q)
    v = np.broadcast_to(vel, (T, 3) + shape).copy()
    p = O.Params(T=T)
    M = np.full(shape, 0.75)
    J1, W, u01, _ = O.backward_sweep(v, np.zeros(shape), M, p)
    detB = np.linalg.det(np.eye(3) + A / T)
    inner = (slice(6, -6),) * 3
    for j in range(T):
        np.testing.assert_allclose(W[j][inner], 0.75 * detB ** (T - j), rtol=1e-12)
    Bt = np.linalg.matrix_power(np.eye(3) + A / T, T)
    ref = np.einsum("de,e...->d...", Bt - np.eye(3), q)
    np.testing.assert_allclose(u01[(slice(None),) + inner], ref[(slice(None),) + inner],
                               atol=1e-12)


def test_constant_velocity_is_an_exact_translation():
    shape = (8, 9, 10)
    T = 5
    rng = _rng(4)
    h = (1.0, 1.5, 0.75)
    p = O.Params(T=T, h=h)
    vel = rng.uniform(-2, 2, (T, 3))             # constant in space, varies in time
    v = np.broadcast_to(vel[:, :, None, None, None], (T, 3) + shape).copy()
    I0, I1 = _blob_pair(shape)
    J1, W, u01, min_det = O.backward_sweep(v, I1, np.ones(shape), p)
    b, u10, J0T, _ = O.forward_sweep(v, I0, I1, np.ones(shape), J1, W, p)
    disp = vel.sum(0) / T / np.array(h)          # sum_j dt v_j / h  (voxels)
    for e in range(3):
        np.testing.assert_allclose(u10[e], -disp[e], atol=1e-12)
        np.testing.assert_allclose(u01[e], disp[e], atol=1e-12)
    assert abs(min_det - 1.0) < 1e-12
    # E_reg of a constant field: Lap = 0 so |L v|^2 = gamma^2 |v|^2 per voxel
    er = O.reg_energy(v, p)
    np.testing.assert_allclose(er, (vel ** 2).sum() / T * np.prod(shape) * np.prod(h), rtol=1e-12)


def test_integer_shift_moves_the_template_voxel_by_voxel():
    shape = (8, 10, 12)
    T = 4
    rng = _rng(5)
    I0 = rng.random(shape)
    v = np.zeros((T, 3) + shape)
    v[:, 0] = 2.0          # total x displacement 2 voxels:  phi_10(x) = x - 2
    v[:, 2] = -1.0         # total z displacement -1 voxel:  phi_10(x) = z + 1
    J1, W, u01, _ = O.backward_sweep(v, I0, np.ones(shape), O.Params(T=T))
    _, u10, J0T, _ = O.forward_sweep(v, I0, I0, np.ones(shape), J1, W, O.Params(T=T))
    Z, Y, X = shape
    iz = np.clip(np.arange(Z) + 1, 0, Z - 1)
    ix = np.clip(np.arange(X) - 2, 0, X - 1)
    np.testing.assert_allclose(J0T, I0[iz][:, :, ix], atol=1e-12)


# ---------------------------------------------------------------- the smoothing operator K

def _mode(shape, k, h, kind):
    Z, Y, X = shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    arg = 2 * np.pi * (k[0] * gx / X + k[1] * gy / Y + k[2] * gz / Z)
    return np.cos(arg) if kind == "cos" else np.sin(arg)


@pytest.mark.parametrize("k,kind", [((1, 0, 0), "cos"), ((0, 3, 0), "sin"), ((2, 1, 3), "cos"),
                                    ((5, 4, 2), "sin"), ((6, 5, 4), "cos")])
def test_K_on_a_single_mode(k, kind):
    shape = (9, 10, 12)
    h = (1.0, 2.0, 0.5)
    alpha, gamma = 0.3, 1.7
    f = _mode(shape, k, h, kind)
    lam = sum((2 - 2 * math.cos(2 * math.pi * k[d] / shape[2 - d])) / h[d] ** 2 for d in range(3))
    got = O.apply_K(f, alpha, gamma, h)
    np.testing.assert_allclose(got, f / (gamma + alpha * lam) ** 2, atol=1e-12)


def test_K_single_mode_golden_value():
    """Hand-derived closed form stored in tests/golden: 8^3 grid, mode (1,0,0), h = 1."""
    with open(os.path.join(GOLDEN, "k_single_mode.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for n, kx, ky, kz, alpha, gamma, val in rows:
        n = int(n)
        f = _mode((n, n, n), (int(kx), int(ky), int(kz)), (1, 1, 1), "cos")
        got = O.apply_K(f, float(alpha), float(gamma), (1.0, 1.0, 1.0))
        np.testing.assert_allclose(got, float(val) * f, atol=1e-12)


def test_K_inverts_the_stencil_operator_squared():
    rng = _rng(6)
    f = rng.standard_normal((7, 8, 9))
    h = (1.0, 1.25, 0.8)
    a, g = 0.05, 1.3
    LLf = O.apply_L(O.apply_L(f, a, g, h), a, g, h)
    np.testing.assert_allclose(O.apply_K(LLf, a, g, h), f, atol=1e-11)


def test_K_of_constant():
    f = np.full((5, 6, 7), 3.0)
    np.testing.assert_allclose(O.apply_K(f, 0.02, 2.0, (1, 1, 1)), 3.0 / 4.0, atol=1e-13)


def test_reg_energy_equals_parseval_form():
    rng = _rng(7)
    T, shape = 3, (6, 7, 8)
    h = (1.0, 0.5, 2.0)
    p = O.Params(T=T, alpha=0.1, gamma=1.2, h=h)
    v = rng.standard_normal((T, 3) + shape)
    Z, Y, X = shape
    kz = np.arange(Z)[:, None, None]
    ky = np.arange(Y)[None, :, None]
    kx = np.arange(X)[None, None, :]
    lam = ((2 - 2 * np.cos(2 * np.pi * kx / X)) / h[0] ** 2 + (2 - 2 * np.cos(2 * np.pi * ky / Y)) / h[1] ** 2
           + (2 - 2 * np.cos(2 * np.pi * kz / Z)) / h[2] ** 2)
    s = 0.0
    for j in range(T):
        for e in range(3):
            F = np.fft.fftn(v[j, e])
            s += (np.abs((p.gamma + p.alpha * lam) * F) ** 2).sum() / v[j, e].size
    np.testing.assert_allclose(O.reg_energy(v, p), s / T * np.prod(h), rtol=1e-12)


# ---------------------------------------------------------------- descent and gradient

def test_energy_decreases_at_small_step():
    pair = synth.ellipsoid_pair(shape=(16, 16, 16), centre=(7.5, 7.5, 7.5), semi_axes=(5, 4, 3.5),
                                width=3.0, amplitude=1.5, seed=0)
    p = O.Params(T=4, epsilon=1e-3)
    v = np.zeros((4, 3, 16, 16, 16))
    E = []
    for _ in range(6):
        r = O.lddmm_step(v, pair.I0, pair.I1, pair.M, p)
        E.append(r.E)
        v = r.v_new
    assert all(b < a for a, b in zip(E, E[1:])), E
    # and with a step ten times smaller it still decreases
    r0 = O.lddmm_step(v, pair.I0, pair.I1, pair.M, O.Params(T=4, epsilon=1e-4))
    assert O.energy(r0.v_new, pair.I0, pair.I1, pair.M, p) < r0.E


def _smooth_problem(shape=(8, 8, 8), T=3, seed=8):
    rng = _rng(seed)
    I0, I1 = _blob_pair(shape)
    M = 0.5 + 0.5 * rng.random(shape)
    v = synth.smooth_velocity(T, shape, 0.8, seed).astype(np.float64)
    return I0, I1, M, v


def test_exact_gradient_matches_central_finite_differences():
    I0, I1, M, v = _smooth_problem()
    p = O.Params(T=3, sigma=0.5, alpha=0.05, h=(1.0, 1.1, 0.9))
    E, g = O.energy_grad_exact(v, I0, I1, M, p)
    rng = _rng(9)
    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(v.shape)
        fd = (O.energy(v + eps * d, I0, I1, M, p) - O.energy(v - eps * d, I0, I1, M, p)) / (2 * eps)
        np.testing.assert_allclose((g * d).sum(), fd, rtol=1e-6)


def test_beg_direction_approximates_the_exact_gradient():
    """Beg's body force b_j is the L2 gradient of the data term (with a minus sign), so the
    Euclidean gradient of the discrete data term is close to -dt h^3 b_j on smooth inputs."""
    shape = (16, 16, 16)
    I0, I1 = _blob_pair(shape)
    I0 = 3 * I0
    I1 = 3 * I1
    M = np.ones(shape)
    T = 4
    v = synth.smooth_velocity(T, shape, 0.3, 11).astype(np.float64)
    p = O.Params(T=T, sigma=1.0, alpha=0.02)
    r = O.lddmm_step(v, I0, I1, M, p)
    _, g = O.energy_grad_exact(v, I0, I1, M, p)
    for j in range(T):
        for e in range(3):
            LLv = O.apply_L(O.apply_L(v[j, e], p.alpha, p.gamma, p.h), p.alpha, p.gamma, p.h)
            g[j, e] -= 2.0 / T * LLv
    approx = -r.b / T
    cos = (g * approx).sum() / np.sqrt((g * g).sum() * (approx * approx).sum())
    ratio = np.sqrt((approx * approx).sum() / (g * g).sum())
    assert cos > 0.95, cos
    assert 0.8 < ratio < 1.25, ratio


# ---------------------------------------------------------------- labels, Dice, warps

def test_labels_identity_and_integer_shift():
    rng = _rng(12)
    L0 = rng.integers(0, 60, (6, 7, 8)).astype(np.uint16)
    u = np.zeros((3, 6, 7, 8), np.float32)
    np.testing.assert_array_equal(O.transfer_labels(L0, u), L0)
    u[0] = 1.0
    u[1] = -2.0
    got = O.transfer_labels(L0, u)
    iy = np.clip(np.arange(7) - 2, 0, 6)
    ix = np.clip(np.arange(8) + 1, 0, 7)
    np.testing.assert_array_equal(got, L0[:, iy][:, :, ix])


def test_labels_round_half_up_in_float32():
    L0 = np.arange(4, dtype=np.uint16).reshape(1, 1, 4)
    u = np.zeros((3, 1, 1, 4), np.float32)
    u[0] = np.float32(0.5)                # x + 0.5 rounds up
    np.testing.assert_array_equal(O.transfer_labels(L0, u).ravel(), [1, 2, 3, 3])
    u[0] = np.float32(-0.5)               # x - 0.5 rounds up to x itself
    np.testing.assert_array_equal(O.transfer_labels(L0, u).ravel(), [0, 1, 2, 3])
    u[0] = np.float32(0.4999)             # clearly below the tie: stays
    np.testing.assert_array_equal(O.transfer_labels(L0, u).ravel(), [0, 1, 2, 3])
    # one ulp below 0.5: x + u is rounded to float32 first, which lands on the tie and rounds up
    u[0] = np.nextafter(np.float32(0.5), np.float32(0))
    np.testing.assert_array_equal(O.transfer_labels(L0, u).ravel(), [1, 2, 3, 3])


def test_dice_golden_tiny_volume():
    with open(os.path.join(GOLDEN, "dice_tiny.txt")) as fh:
        lines = [l for l in fh if l.strip() and not l.startswith("#")]
    A = np.array([int(x) for x in lines[0].split()]).reshape(1, 2, 3)
    B = np.array([int(x) for x in lines[1].split()]).reshape(1, 2, 3)
    assert abs(O.dice(A, B) - float(lines[2])) < 1e-12
    assert O.dice(A, A) == 1.0


def test_dice_brute_force():
    rng = _rng(13)
    A = rng.integers(0, 4, (3, 4, 5))
    B = rng.integers(0, 4, (3, 4, 5))
    vals = []
    for l in range(1, 4):
        inter = sum(1 for a, b in zip(A.ravel(), B.ravel()) if a == l and b == l)
        na = sum(1 for a in A.ravel() if a == l)
        nb = sum(1 for b in B.ravel() if b == l)
        if na + nb:
            vals.append(2 * inter / (na + nb))
    assert abs(O.dice(A, B) - np.mean(vals)) < 1e-12


def test_warp_identity_and_shift():
    rng = _rng(14)
    f = rng.random((5, 6, 7))
    u = np.zeros((3, 5, 6, 7))
    np.testing.assert_array_equal(O.warp(f, u), f)
    u[2] = 1.0
    np.testing.assert_allclose(O.warp(f, u), f[np.clip(np.arange(5) + 1, 0, 4)], atol=1e-14)
    u[2] = 0.0
    u[0] = 1.0                                   # (id + u)(x) = x + 1 along x
    u[1] = -1.0                                  # and y - 1
    ref = f[:, np.clip(np.arange(6) - 1, 0, 5)][:, :, np.clip(np.arange(7) + 1, 0, 6)]
    np.testing.assert_allclose(O.warp(f, u), ref, atol=1e-14)


# ---------------------------------------------------------------- multiscale

def test_register_levels_measure_the_same_energy():
    """The energy is a discretised integral, so a coarse level (block means, spacing f h) must
    give the same value as the fine grid where the discretisation is exact: for images that are
    constant on 2x2x2 blocks and v = 0 the data terms agree, and for a spatially constant v the
    regulariser terms agree (|L v|^2 = gamma^2 |v|^2 per unit volume)."""
    rng = _rng(15)
    coarse = (4, 3, 5)
    shape = (8, 6, 10)
    h = (1.0, 1.5, 0.5)
    up = lambda a: np.repeat(np.repeat(np.repeat(a, 2, 0), 2, 1), 2, 2)
    I0 = up(rng.random(coarse))
    I1 = up(rng.random(coarse))
    M = np.ones(shape)
    p = O.Params(T=2, h=h)
    _, e2, _ = O.register(I0, I1, M, p, 1, factors=(2,))
    _, e1, _ = O.register(I0, I1, M, p, 1, factors=(1,))
    assert e2[0][1] == 0.0 and e1[0][1] == 0.0
    np.testing.assert_allclose(e2[0][2], e1[0][2], rtol=1e-12)
    c = np.array([0.4, -0.3, 0.2])[None, :, None, None, None]
    _, e2, _ = O.register(I0, I1, M, p, 1, factors=(2,), v0=c * np.ones((2, 3) + coarse))
    _, e1, _ = O.register(I0, I1, M, p, 1, factors=(1,), v0=c * np.ones((2, 3) + shape))
    np.testing.assert_allclose(e2[0][1], e1[0][1], rtol=1e-12)
    np.testing.assert_allclose(e1[0][1], (c ** 2).sum() * np.prod(shape) * np.prod(h), rtol=1e-12)


def test_downsample_block_mean():
    f = np.arange(4 * 4 * 6, dtype=float).reshape(4, 4, 6)
    d = O.downsample(f, 2)
    assert d.shape == (2, 2, 3)
    assert d[0, 0, 0] == np.mean(f[0:2, 0:2, 0:2])
    g = np.full((5, 7, 9), 2.5)
    np.testing.assert_allclose(O.downsample(g, 4), 2.5)
    assert O.downsample(g, 4).shape == (2, 2, 3)
    # edge replication: the coarse cell over the ragged edge averages replicated values
    h = np.zeros((1, 1, 3))
    h[0, 0, 2] = 8.0
    np.testing.assert_allclose(O.downsample(h, 2)[0, 0, 1], 8.0)


def test_upsample_velocity_reproduces_affine_fields():
    Zc, Yc, Xc = 4, 5, 6
    gz, gy, gx = np.meshgrid(np.arange(Zc), np.arange(Yc), np.arange(Xc), indexing="ij")
    # physical coordinate of coarse voxel i at spacing 4: (i + 0.5) 4 - 0.5
    phys = lambda i, f: (i + 0.5) * f - 0.5
    fc = 4
    field = 0.3 * phys(gx, fc) - 0.2 * phys(gy, fc) + 0.1 * phys(gz, fc) + 1.0
    v = np.broadcast_to(field, (1, 3, Zc, Yc, Xc)).copy()
    ff = 2
    fine = (8, 10, 12)
    up = O.upsample_velocity(v, fine, fc, ff)
    fz, fy, fx = np.meshgrid(np.arange(8), np.arange(10), np.arange(12), indexing="ij")
    ref = 0.3 * phys(fx, ff) - 0.2 * phys(fy, ff) + 0.1 * phys(fz, ff) + 1.0
    inside = (fx >= 1) & (fx <= 10) & (fy >= 1) & (fy <= 8) & (fz >= 1) & (fz <= 6)
    np.testing.assert_allclose(up[0, 0][inside], ref[inside], atol=1e-12)


# --------------------------------------------------------------------------------------------
# RK4 along each time step (the paper's integrator, §2.4)

def _linear_velocity(A, c, shape, T):
    Z, Y, X = shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    q = np.stack([gx - c[0], gy - c[1], gz - c[2]]).astype(np.float64)
    v = np.einsum("ij,jzyx->izyx", A, q)
    return np.broadcast_to(v, (T, 3) + shape).copy()


def test_rk4_matches_the_truncated_exponential_on_a_linear_field():
    """v(x) = A (x - c), held over each step: RK4 advances an affine map by the 4th-order Taylor
    polynomial P of exp(A dt), and trilinear interpolation of affine displacements is exact, so
    inside the grid phi_{0,1}(x) = c + P^T (x - c) and phi_{1,0}(x) = c + Q^T (x - c) with Q the
    polynomial of exp(-A dt), to rounding; the one-lookup scheme is only first order."""
    from oracle import lddmm as O
    rng = np.random.default_rng(7)
    A = 0.25 * rng.standard_normal((3, 3))
    shape, T = (26, 26, 26), 4
    c = (12.5, 12.5, 12.5)
    v = _linear_velocity(A, c, shape, T)
    I = np.zeros(shape)
    p = O.Params(T=T, integrator="rk4")
    _, _, u01, _ = O.backward_sweep(v, I, I, p)
    _, u10, _, _ = O.forward_sweep(v, I, I, I, np.zeros((T,) + shape), np.zeros((T,) + shape), p)

    def taylor(B):
        P, term = np.eye(3), np.eye(3)
        for k in range(1, 5):
            term = term @ B / k
            P = P + term
        return P

    Pf = np.linalg.matrix_power(taylor(A / T), T)
    Pb = np.linalg.matrix_power(taylor(-A / T), T)
    sl = O.Params(T=T)
    _, _, u01_sl, _ = O.backward_sweep(v, I, I, sl)
    z, y, x = np.meshgrid(*[np.arange(10, 16)] * 3, indexing="ij")
    q = np.stack([x - c[0], y - c[1], z - c[2]]).reshape(3, -1)
    exp_f = (Pf - np.eye(3)) @ q
    exp_b = (Pb - np.eye(3)) @ q
    got_f = u01[:, 10:16, 10:16, 10:16].reshape(3, -1)
    got_b = u10[:, 10:16, 10:16, 10:16].reshape(3, -1)
    assert np.max(np.abs(got_f - exp_f)) < 1e-10
    assert np.max(np.abs(got_b - exp_b)) < 1e-10
    # the exact flow differs from RK4 by O(dt^4) and from one lookup per step by O(dt)
    from scipy.linalg import expm
    err_rk = np.max(np.abs(got_f - (expm(A) - np.eye(3)) @ q))
    err_sl = np.max(np.abs(u01_sl[:, 10:16, 10:16, 10:16].reshape(3, -1) - (expm(A) - np.eye(3)) @ q))
    assert err_rk < 1e-3 < err_sl


def test_rk4_equals_one_lookup_for_a_spatially_constant_field():
    from oracle import lddmm as O
    rng = np.random.default_rng(8)
    shape, T = (10, 11, 12), 3
    v = np.broadcast_to(rng.normal(0, 2.0, size=(T, 3, 1, 1, 1)), (T, 3) + shape).copy()
    I1 = rng.random(shape)
    a = O.backward_sweep(v, I1, I1, O.Params(T=T, integrator="rk4"))
    b = O.backward_sweep(v, I1, I1, O.Params(T=T))
    assert np.allclose(a[2], b[2], atol=1e-12) and np.allclose(a[0], b[0], atol=1e-12)


def _affine_chain(A, dt, sign, T, backward):
    """Products of I + sign dt A_j: backward P_j = P_{j+1} (I + dt A_j) with P_T = I; forward
    Q_{j+1} = Q_j (I - dt A_j) with Q_0 = I."""
    out = [None] * (T + 1)
    if backward:
        out[T] = np.eye(3)
        for j in range(T - 1, -1, -1):
            out[j] = out[j + 1] @ (np.eye(3) + sign * dt * A[j])
    else:
        out[0] = np.eye(3)
        for j in range(T):
            out[j + 1] = out[j] @ (np.eye(3) + sign * dt * A[j])
    return out


def test_body_force_at_every_step_of_a_time_varying_affine_flow():
    """For a velocity that is affine in space with a different matrix at every step,
    v_j(x) = H A_j (x - c) (H = diag(h); A_j in voxels per unit time), every map is affine and
    every trilinear lookup and central difference is exact away from the clamped faces:
        phi_{j,1}(x) = c + P_j (x - c),  P_j = P_{j+1} (I + dt A_j),  P_T = I,
        phi_{j,0}(x) = c + Q_j (x - c),  Q_{j+1} = Q_j (I - dt A_j),  Q_0 = I.
    With linear I0 = a0 + g0.x, I1 and M the body force of Beg's gradient at step j is
        b_j = (2/sigma^2) M(phi_{j,1}) det(P_j) (I0(phi_{j,0}) - I1(phi_{j,1})) (Q_j^T g0) / h,
    the spatial gradient of the deformed template I0 o phi_{j,0} (not the template's gradient
    carried along, g0), paired with the target-side terms of the same time t_j.  Pairing J0_j with
    W_{j+1} and J1_{j+1}, taking (grad I0) o phi, or any dropped chain factor fails this at some j.
    The update is then v - eps (2 v - K b) with K the (separately pinned) spectral operator."""
    T = 4
    dt = 1.0 / T
    shape = (30, 32, 36)                                   # Z, Y, X
    h = np.array([1.0, 0.8, 1.25])
    rng = _rng(21)
    A = [0.04 * rng.standard_normal((3, 3)) for _ in range(T)]
    A[1] += 0.06 * np.eye(3)                                # det(I + dt A_j) far from 1
    A[2] -= 0.05 * np.eye(3)
    c = np.array([(n - 1) / 2.0 for n in shape[::-1]])     # (x, y, z) centre
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    q = np.stack([x - c[0], y - c[1], z - c[2]])
    v = np.stack([np.einsum("de,e...->d...", A[j], q) * h[:, None, None, None]
                  for j in range(T)])
    dmax = max(float(np.abs(dt * np.einsum("de,e...->d...", A[j], q)).max()) for j in range(T))
    assert dmax < 1.0
    m = T * (int(np.ceil(dmax)) + 1) + 2                   # exactness margin from the faces
    inner = (slice(m, -m),) * 3
    assert all(n - 2 * m >= 4 for n in shape)
    g0, g1, gm = np.array([0.02, -0.015, 0.03]), np.array([-0.01, 0.025, 0.012]), \
        np.array([0.01, 0.006, -0.008])
    I0 = 0.4 + g0[0] * x + g0[1] * y + g0[2] * z
    I1 = 0.1 + g1[0] * x + g1[1] * y + g1[2] * z
    M = 0.9 + gm[0] * x + gm[1] * y + gm[2] * z
    p = O.Params(T=T, h=tuple(h), epsilon=0.01)
    r = O.lddmm_step(v, I0, I1, M, p)

    P = _affine_chain(A, dt, +1.0, T, backward=True)
    Q = _affine_chain(A, dt, -1.0, T, backward=False)

    def lin(a, g, Mat):                                   # a + g . (c + Mat q)
        pos = c[:, None, None, None] + np.einsum("de,e...->d...", Mat, q)
        return a + np.einsum("d,d...->...", g, pos)

    for j in range(T):
        J1 = lin(0.1, g1, P[j])
        W = lin(0.9, gm, P[j]) * np.linalg.det(P[j])
        J0 = lin(0.4, g0, Q[j])
        grad = Q[j].T @ g0
        np.testing.assert_allclose(r.J1[j][inner], J1[inner], rtol=0, atol=1e-12)
        np.testing.assert_allclose(r.W[j][inner], W[inner], rtol=1e-12, atol=0)
        for e in range(3):
            ref = 2.0 / p.sigma ** 2 * W * (J0 - J1) * grad[e] / h[e]
            np.testing.assert_allclose(r.b[j, e][inner], ref[inner], rtol=0,
                                       atol=1e-10 * float(np.abs(ref[inner]).max()))
    u01 = np.einsum("de,e...->d...", P[0] - np.eye(3), q)
    u10 = np.einsum("de,e...->d...", Q[T] - np.eye(3), q)
    np.testing.assert_allclose(r.u01[(slice(None),) + inner], u01[(slice(None),) + inner], atol=1e-11)
    np.testing.assert_allclose(r.u10[(slice(None),) + inner], u10[(slice(None),) + inner], atol=1e-11)
    np.testing.assert_allclose(r.J0T[inner], lin(0.4, g0, Q[T])[inner], atol=1e-12)
    for j in range(T):
        for e in range(3):
            Kb = O.apply_K(r.b[j, e], p.alpha, p.gamma, p.h)
            np.testing.assert_allclose(r.v_new[j, e], v[j, e] - p.epsilon * (2 * v[j, e] - Kb),
                                       rtol=1e-13, atol=1e-13)


def test_threaded_lookups_give_the_same_bits():
    """Slab-parallel trilinear lookups evaluate every value by the same expression, so a step
    computed with 4 threads equals the single-threaded one bit for bit."""
    shape = (70, 40, 48)
    I0, I1 = _blob_pair(shape)
    v = synth.smooth_velocity(2, shape, 3.0, seed=3)
    p = O.Params(T=2)
    a = O.lddmm_step(v, I0, I1, None, p)
    try:
        O.set_threads(4)
        b = O.lddmm_step(v, I0, I1, None, p)
    finally:
        O.set_threads(1)
    for x, y in ((a.v_new, b.v_new), (a.u10, b.u10), (a.u01, b.u01), (a.J0T, b.J0T), (a.W, b.W)):
        np.testing.assert_array_equal(x, y)
    assert a.E_reg == b.E_reg and a.E_data == b.E_data


def test_resample_between_grids_of_one_box():
    """Cell-centred resampling: the identity on the same grid; a constant stays constant; an
    affine function of the box coordinate (u = (i + 0.5) / n) is reproduced exactly wherever the
    sample point lies inside the source grid, up and down and with different ratios per axis; a
    2x coarsening of a field linear along x gives the mean of each pair."""
    rng = _rng(31)
    f = rng.standard_normal((5, 6, 7))
    np.testing.assert_array_equal(O.resample(f, f.shape), f)
    np.testing.assert_allclose(O.resample(np.full((4, 5, 6), 2.5), (9, 3, 13)), 2.5, rtol=1e-15)
    for src, dst in (((6, 8, 10), (15, 11, 23)), ((20, 12, 16), (7, 5, 6))):
        z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in src], indexing="ij")
        g = 0.3 + 2.0 * x - 1.5 * y + 0.7 * z
        out = O.resample(g, dst)
        Z, Y, X = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in dst], indexing="ij")
        ref = 0.3 + 2.0 * X - 1.5 * Y + 0.7 * Z
        # inside: every sample coordinate between the first and last source cell centre
        ins = ((X >= 0.5 / src[2]) & (X <= 1 - 0.5 / src[2]) & (Y >= 0.5 / src[1]) &
               (Y <= 1 - 0.5 / src[1]) & (Z >= 0.5 / src[0]) & (Z <= 1 - 0.5 / src[0]))
        assert ins.sum() > 20
        np.testing.assert_allclose(out[ins], ref[ins], rtol=0, atol=1e-12)
    h = np.broadcast_to(np.arange(8.0), (4, 4, 8))
    np.testing.assert_allclose(O.resample(h, (4, 4, 4))[0, 0], [0.5, 2.5, 4.5, 6.5], atol=1e-12)
