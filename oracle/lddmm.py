"""FP64 CPU oracle for one gradient-descent iteration of masked LDDMM.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain statement of what the CUDA library
computes; only the tests, the smoke check and the benchmark's CPU-baseline leg may import it.
It shares no code with the CUDA path.

Method (Kutten et al., "Deformably registering and annotating whole CLARITY brains to an atlas
via masked LDDMM", SPIE 2016):

* §2.4: LDDMM minimises, by gradient descent,
      E(v) = int_0^1 ||L v_t||^2 dt + sigma^-2 ||J0 o phi_10 - J1||^2,   L = (-alpha Lap + gamma) I3
  over a time-varying velocity field v; the flow phi is obtained by integrating v.
* §2.3: Mask-LDDMM replaces the images by their masks (the caller passes masks as I0, I1).
* §2.4 / §2.5: the outputs are phi_10 and its inverse; atlas labels are pulled back as
  L0 o phi_10 by nearest-neighbour lookup (§1.5 names nearest-neighbour interpolation).
* The gradient and update rule are those of Beg et al. 2005 (cited in §2.4):
      grad_t = 2 v_t - K[(2/sigma^2) |D phi_t1| (J0_t - J1_t) grad J0_t],   K = (L^T L)^-1,
      v_t <- v_t - eps grad_t,
  with J0_t = I0 o phi_t0, J1_t = I1 o phi_t1.

Readings where the paper is silent:
* Time discretisation: T steps, dt = 1/T, first-order semi-Lagrangian flows (the paper uses
  4 steps of RK4, §2.4; the default here is T steps of one trilinear lookup each, with RK4
  available as integrator="rk4"):
      phi_{j,1}(x) = phi_{j+1,1}(x + dt v_j(x)),  phi_{T,1} = id   (backward sweep)
      phi_{j+1,0}(x) = phi_{j,0}(x - dt v_j(x)),  phi_{0,0} = id   (forward sweep)
  Maps are stored as displacements u = phi - id in voxel units of the grid; velocities are in
  physical units (voxel spacing h per axis), so a step moves dt v / h voxels.
* Interpolation: trilinear with clamp-to-edge coordinates, for displacements and images.
* Stencils: grad J0 and D phi by central differences inside, one-sided at the faces.
* The weight mask M lives in target space, so its time-t pull-back M o phi_{t,1} multiplies the
  residual: b_t = (2/sigma^2) (M o phi_t1) det(D phi_t1) (J0_t - J1_t) grad J0_t.
* K = (gamma - alpha Lap_h)^-2 with the periodic 7-point Laplacian Lap_h; its Fourier symbol is
  (gamma + alpha lambda(k))^-2, lambda(k) = sum_d (2 - 2 cos(2 pi k_d / N_d)) / h_d^2.
* Discrete energy: E = h^3 [dt sum_j sum_x |(gamma - alpha Lap_h) v_j|^2
                            + sigma^-2 sum_x M (I0 o phi_{1,0} - I1)^2],  h^3 = hx hy hz.

Arrays are C-ordered [z][y][x]; vector fields are (3, Z, Y, X) with components (x, y, z).
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Params", "StepResult", "set_threads", "trilinear", "interp_vec", "fd_gradient", "jacobian_det",
    "laplacian_symbol", "apply_K", "apply_L", "backward_sweep", "forward_sweep",
    "reg_energy", "data_energy", "energy", "lddmm_step", "energy_grad_exact",
    "transfer_labels", "warp", "dice", "downsample", "upsample_velocity", "resample", "register",
]


@dataclasses.dataclass
class Params:
    """Problem parameters (§2.4): alpha, gamma in L, sigma in E, T time steps, step size eps."""

    alpha: float = 0.02
    gamma: float = 1.0
    sigma: float = 0.1
    T: int = 10
    epsilon: float = 1e-3
    h: tuple = (1.0, 1.0, 1.0)     # voxel spacing (hx, hy, hz)
    integrator: str = "sl"         # "sl": one lookup per step; "rk4": RK4 along the step (§2.4)


@dataclasses.dataclass
class StepResult:
    v_new: np.ndarray       # (T,3,Z,Y,X) updated velocity
    E_reg: float
    E_data: float
    u10: np.ndarray         # phi_{1,0} - id, voxels (3,Z,Y,X)
    u01: np.ndarray         # phi_{0,1} - id, voxels
    J0T: np.ndarray         # deformed template I0 o phi_{1,0}
    min_det: float          # min over j, x of det D phi_{j,1}
    b: np.ndarray           # (T,3,Z,Y,X) body force before smoothing
    J1: np.ndarray          # (T,Z,Y,X) I1 o phi_{j,1}
    W: np.ndarray           # (T,Z,Y,X) (M o phi_{j,1}) det D phi_{j,1}

    @property
    def E(self):
        return self.E_reg + self.E_data


def _grid(shape):
    Z, Y, X = shape
    return np.meshgrid(np.arange(Z, dtype=np.float64), np.arange(Y, dtype=np.float64),
                       np.arange(X, dtype=np.float64), indexing="ij")


def _axis_weights(q, n):
    """Lower corner index and fraction along one axis, coordinates clamped to [0, n-1]."""
    q = np.clip(q, 0.0, n - 1.0)
    if n == 1:
        return np.zeros(q.shape, np.int64), np.zeros(q.shape), 0
    i0 = np.minimum(np.floor(q).astype(np.int64), n - 2)
    return i0, q - i0, 1


_THREADS = 1


def set_threads(n):
    """Number of host threads for the trilinear lookups (1: none).  Large query arrays are cut
    into slabs along their first axis and each slab is evaluated by the same expression in a
    thread of a pool (NumPy releases the interpreter lock inside array operations); every value
    is computed exactly as in one piece, so results do not depend on the thread count.  FFTs take
    their own `workers` argument."""
    global _THREADS
    _THREADS = max(1, int(n))


def trilinear(f, qx, qy, qz):
    """Trilinear interpolation of f[z,y,x] at voxel coordinates (qx, qy, qz), clamp-to-edge."""
    f = np.asarray(f, dtype=np.float64)
    qx, qy, qz = np.broadcast_arrays(qx, qy, qz)
    if _THREADS > 1 and qx.ndim >= 1 and qx.size >= (1 << 18) and qx.shape[0] >= 2:
        from concurrent.futures import ThreadPoolExecutor
        cuts = np.linspace(0, qx.shape[0], min(_THREADS, qx.shape[0]) + 1).astype(int)
        with ThreadPoolExecutor(len(cuts) - 1) as ex:
            parts = list(ex.map(lambda ab: _trilinear1(f, qx[ab[0]:ab[1]], qy[ab[0]:ab[1]],
                                                       qz[ab[0]:ab[1]]), zip(cuts[:-1], cuts[1:])))
        return np.concatenate(parts, axis=0)
    return _trilinear1(f, qx, qy, qz)


def _trilinear1(f, qx, qy, qz):
    Z, Y, X = f.shape
    ix, tx, sx = _axis_weights(qx, X)
    iy, ty, sy = _axis_weights(qy, Y)
    iz, tz, sz = _axis_weights(qz, Z)
    out = np.zeros(np.broadcast(qx, qy, qz).shape)
    for dz, wz in ((0, 1.0 - tz), (sz, tz)):
        for dy, wy in ((0, 1.0 - ty), (sy, ty)):
            for dx, wx in ((0, 1.0 - tx), (sx, tx)):
                out += wz * wy * wx * f[iz + dz, iy + dy, ix + dx]
    return out


def interp_vec(u, qx, qy, qz):
    """Trilinear interpolation of each component of a vector field (3,Z,Y,X)."""
    return np.stack([trilinear(u[c], qx, qy, qz) for c in range(3)])


def fd_gradient(f):
    """(d/dx, d/dy, d/dz) in voxel units: central inside, one-sided first order at faces."""
    gz, gy, gx = np.gradient(np.asarray(f, np.float64), axis=(0, 1, 2))
    return np.stack([gx, gy, gz])


def jacobian_det(u):
    """det(I + Du) for a displacement u (3,Z,Y,X) in voxels (finite differences as fd_gradient)."""
    D = np.stack([fd_gradient(u[d]) for d in range(3)])  # D[d, e] = du_d / dx_e
    for d in range(3):
        D[d, d] += 1.0
    return (D[0, 0] * (D[1, 1] * D[2, 2] - D[1, 2] * D[2, 1])
            - D[0, 1] * (D[1, 0] * D[2, 2] - D[1, 2] * D[2, 0])
            + D[0, 2] * (D[1, 0] * D[2, 1] - D[1, 1] * D[2, 0]))


def laplacian_symbol(shape, h):
    """lambda(k) = sum_d (2 - 2 cos(2 pi k_d / N_d)) / h_d^2 on the rfftn half-spectrum grid."""
    Z, Y, X = shape
    hx, hy, hz = h
    kz = np.arange(Z)[:, None, None]
    ky = np.arange(Y)[None, :, None]
    kx = np.arange(X // 2 + 1)[None, None, :]
    return ((2 - 2 * np.cos(2 * np.pi * kx / X)) / hx ** 2
            + (2 - 2 * np.cos(2 * np.pi * ky / Y)) / hy ** 2
            + (2 - 2 * np.cos(2 * np.pi * kz / Z)) / hz ** 2)


def apply_K(f, alpha, gamma, h, workers=None):
    """K f = (gamma - alpha Lap_h)^-2 f for a scalar field, by FFT on the periodic grid."""
    from scipy import fft as sfft
    f = np.asarray(f, np.float64)
    lam = laplacian_symbol(f.shape, h)
    F = sfft.rfftn(f, workers=workers)
    F /= (gamma + alpha * lam) ** 2
    return sfft.irfftn(F, s=f.shape, workers=workers)


def apply_L(f, alpha, gamma, h):
    """(gamma - alpha Lap_h) f with the periodic 7-point Laplacian (§2.4's operator L)."""
    f = np.asarray(f, np.float64)
    hx, hy, hz = h
    lap = ((np.roll(f, 1, 2) - 2 * f + np.roll(f, -1, 2)) / hx ** 2
           + (np.roll(f, 1, 1) - 2 * f + np.roll(f, -1, 1)) / hy ** 2
           + (np.roll(f, 1, 0) - 2 * f + np.roll(f, -1, 0)) / hz ** 2)
    return gamma * f - alpha * lap


def _h3(h):
    return float(h[0] * h[1] * h[2])


def _vox(vj, h):
    """Velocity (physical units) -> voxels per unit time, per component."""
    return np.stack([vj[0] / h[0], vj[1] / h[1], vj[2] / h[2]])


def _step_disp(vj, p: Params, sign, grid):
    """Displacement (voxels) of one time step along the characteristic of v_j from each grid
    point: sign dt v_j(x) / h (semi-Lagrangian), or RK4 on dy/dt = sign v_j(y) / h over dt with
    v_j held over the step and read at the stage points by trilinear interpolation (the paper's
    4th-order Runge-Kutta, §2.4).  sign = +1 for phi_{j,1}, -1 for phi_{j+1,0}."""
    gz, gy, gx = grid
    dt = 1.0 / p.T
    k1 = sign * dt * _vox(np.asarray(vj, np.float64), p.h)
    if p.integrator == "sl":
        return k1
    if p.integrator != "rk4":
        raise ValueError("integrator must be 'sl' or 'rk4'")
    vjh = _vox(np.asarray(vj, np.float64), p.h)

    def f(d):
        return sign * dt * interp_vec(vjh, gx + d[0], gy + d[1], gz + d[2])

    k2 = f(0.5 * k1)
    k3 = f(0.5 * k2)
    k4 = f(k3)
    return (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0


def backward_sweep(v, I1, M, p: Params):
    """phi_{j,1} for j = T-1..0, and the target-side terms J1_j = I1 o phi_{j,1},
    W_j = (M o phi_{j,1}) det D phi_{j,1}.  Returns (J1, W, u01, min_det)."""
    T = v.shape[0]
    shape = I1.shape
    dt = 1.0 / T
    gz, gy, gx = _grid(shape)
    u = np.zeros((3,) + shape)                  # phi_{T,1} = id
    J1 = np.empty((T,) + shape)
    W = np.empty((T,) + shape)
    min_det = np.inf
    for j in range(T - 1, -1, -1):
        d = _step_disp(v[j], p, +1.0, (gz, gy, gx))
        u = d + interp_vec(u, gx + d[0], gy + d[1], gz + d[2])
        px, py, pz = gx + u[0], gy + u[1], gz + u[2]
        det = jacobian_det(u)
        min_det = min(min_det, float(det.min()))
        J1[j] = trilinear(I1, px, py, pz)
        W[j] = trilinear(M, px, py, pz) * det
    return J1, W, u, min_det


def forward_sweep(v, I0, I1, M, J1, W, p: Params):
    """phi_{j,0} for j = 0..T, J0_j = I0 o phi_{j,0}, the body force b_j and E_data."""
    T = v.shape[0]
    shape = I0.shape
    dt = 1.0 / T
    gz, gy, gx = _grid(shape)
    u = np.zeros((3,) + shape)                  # phi_{0,0} = id
    b = np.empty((T, 3) + shape)
    c = 2.0 / p.sigma ** 2
    for j in range(T):
        J0 = trilinear(I0, gx + u[0], gy + u[1], gz + u[2])
        g = fd_gradient(J0)
        r = c * W[j] * (J0 - J1[j])
        for e in range(3):
            b[j, e] = r * g[e] / p.h[e]
        d = _step_disp(v[j], p, -1.0, (gz, gy, gx))
        u = d + interp_vec(u, gx + d[0], gy + d[1], gz + d[2])
    J0T = trilinear(I0, gx + u[0], gy + u[1], gz + u[2])
    E_data = data_energy(J0T, I1, M, p)
    return b, u, J0T, E_data


def reg_energy(v, p: Params):
    """dt h^3 sum_j sum_x |(gamma - alpha Lap_h) v_j|^2 (first term of the §2.4 energy)."""
    T = v.shape[0]
    s = 0.0
    for j in range(T):
        for e in range(3):
            s += float((apply_L(v[j, e], p.alpha, p.gamma, p.h) ** 2).sum())
    return s * _h3(p.h) / T


def data_energy(J0T, I1, M, p: Params):
    """sigma^-2 h^3 sum_x M (I0 o phi_10 - I1)^2 (second term of the §2.4 energy, weighted)."""
    r = np.asarray(J0T, np.float64) - np.asarray(I1, np.float64)
    return float((np.asarray(M, np.float64) * r * r).sum()) * _h3(p.h) / p.sigma ** 2


def energy(v, I0, I1, M, p: Params):
    """Discrete §2.4 energy of v (forward sweep only)."""
    T = v.shape[0]
    shape = I0.shape
    dt = 1.0 / T
    gz, gy, gx = _grid(shape)
    u = np.zeros((3,) + shape)
    for j in range(T):
        d = _step_disp(v[j], p, -1.0, (gz, gy, gx))
        u = d + interp_vec(u, gx + d[0], gy + d[1], gz + d[2])
    J0T = trilinear(I0, gx + u[0], gy + u[1], gz + u[2])
    return reg_energy(v, p) + data_energy(J0T, I1, M, p)


def lddmm_step(v, I0, I1, M=None, p: Params = Params(), workers=None) -> StepResult:
    """One gradient-descent iteration (Beg et al. 2005 update, cited in §2.4).

    grad_j = 2 v_j - K b_j;  v_j <- v_j - eps grad_j;  energies are those of the input v.
    """
    v = np.asarray(v, np.float64)
    I0 = np.asarray(I0, np.float64)
    I1 = np.asarray(I1, np.float64)
    M = np.ones_like(I0) if M is None else np.asarray(M, np.float64)
    J1, W, u01, min_det = backward_sweep(v, I1, M, p)
    b, u10, J0T, E_data = forward_sweep(v, I0, I1, M, J1, W, p)
    E_reg = reg_energy(v, p)
    v_new = np.empty_like(v)
    for j in range(v.shape[0]):
        for e in range(3):
            Kb = apply_K(b[j, e], p.alpha, p.gamma, p.h, workers=workers)
            v_new[j, e] = v[j, e] - p.epsilon * (2.0 * v[j, e] - Kb)
    return StepResult(v_new, E_reg, E_data, u10, u01, J0T, min_det, b, J1, W)


# ----------------------------------------------------------------------------------------------
# Exact gradient of the discrete energy (reverse mode of the forward sweep)
# ----------------------------------------------------------------------------------------------

def _trilinear_with_grad(f, qx, qy, qz):
    """Value and coordinate-gradient of the trilinear interpolant (clamped axes have zero slope)."""
    f = np.asarray(f, np.float64)
    Z, Y, X = f.shape

    def ax(q, n):
        inside = (q >= 0.0) & (q <= n - 1.0)
        i0, t, s = _axis_weights(q, n)
        return i0, t, s, inside.astype(np.float64)

    ix, tx, sx, kx = ax(qx, X)
    iy, ty, sy, ky = ax(qy, Y)
    iz, tz, sz, kz = ax(qz, Z)
    val = np.zeros(np.broadcast(qx, qy, qz).shape)
    gx = np.zeros_like(val)
    gy = np.zeros_like(val)
    gz = np.zeros_like(val)
    for dz, wz, dwz in ((0, 1.0 - tz, -1.0), (sz, tz, 1.0)):
        for dy, wy, dwy in ((0, 1.0 - ty, -1.0), (sy, ty, 1.0)):
            for dx, wx, dwx in ((0, 1.0 - tx, -1.0), (sx, tx, 1.0)):
                fv = f[iz + dz, iy + dy, ix + dx]
                val += wz * wy * wx * fv
                gx += wz * wy * dwx * fv
                gy += wz * dwy * wx * fv
                gz += dwz * wy * wx * fv
    return val, gx * kx, gy * ky, gz * kz


def _trilinear_adjoint(g, shape, qx, qy, qz):
    """Transpose of trilinear interpolation: scatter-add g(x) with weights into a grid."""
    Z, Y, X = shape
    ix, tx, sx = _axis_weights(qx, X)
    iy, ty, sy = _axis_weights(qy, Y)
    iz, tz, sz = _axis_weights(qz, Z)
    out = np.zeros(Z * Y * X)
    for dz, wz in ((0, 1.0 - tz), (sz, tz)):
        for dy, wy in ((0, 1.0 - ty), (sy, ty)):
            for dx, wx in ((0, 1.0 - tx), (sx, tx)):
                idx = ((iz + dz) * Y + (iy + dy)) * X + (ix + dx)
                np.add.at(out, idx.ravel(), (wz * wy * wx * g).ravel())
    return out.reshape(shape)


def energy_grad_exact(v, I0, I1, M, p: Params):
    """Euclidean gradient dE/dv of the discrete energy above, by reverse-mode differentiation
    of the forward sweep and of the stencil regulariser.  Returns (E, grad (T,3,Z,Y,X))."""
    if p.integrator != "sl":
        raise ValueError("the exact gradient is built for the semi-Lagrangian flow")
    v = np.asarray(v, np.float64)
    I0 = np.asarray(I0, np.float64)
    I1 = np.asarray(I1, np.float64)
    M = np.ones_like(I0) if M is None else np.asarray(M, np.float64)
    T = v.shape[0]
    shape = I0.shape
    dt = 1.0 / T
    h = p.h
    gz, gy, gx = _grid(shape)
    us = [np.zeros((3,) + shape)]
    for j in range(T):
        d = dt * _vox(v[j], h)
        us.append(-d + interp_vec(us[-1], gx - d[0], gy - d[1], gz - d[2]))
    uT = us[-1]
    J0T, dIx, dIy, dIz = _trilinear_with_grad(I0, gx + uT[0], gy + uT[1], gz + uT[2])
    E = reg_energy(v, p) + data_energy(J0T, I1, M, p)
    c = 2.0 * _h3(h) / p.sigma ** 2 * M * (J0T - I1)
    g = np.stack([c * dIx, c * dIy, c * dIz])       # dE/du_T, per voxel
    grad = np.empty_like(v)
    for j in range(T - 1, -1, -1):
        d = dt * _vox(v[j], h)
        qx, qy, qz = gx - d[0], gy - d[1], gz - d[2]
        # u_{j+1} = -d + U_j(q):  dU/dq is the 3x3 Jacobian of the interpolant of u_j at q
        J = [_trilinear_with_grad(us[j][c_], qx, qy, qz)[1:] for c_ in range(3)]
        for e in range(3):
            s = g[e].copy()
            for c_ in range(3):
                s += g[c_] * J[c_][e]
            grad[j, e] = -(dt / h[e]) * s
        g = np.stack([_trilinear_adjoint(g[c_], shape, qx, qy, qz) for c_ in range(3)])
    for j in range(T):
        for e in range(3):
            LLv = apply_L(apply_L(v[j, e], p.alpha, p.gamma, h), p.alpha, p.gamma, h)
            grad[j, e] += 2.0 * dt * _h3(h) * LLv
    return E, grad


# ----------------------------------------------------------------------------------------------
# Outputs: label transfer (§2.5), warps (§2.4), Dice, multiscale
# ----------------------------------------------------------------------------------------------

def transfer_labels(L0, u10):
    """L0 o phi_10 by nearest neighbour (§2.5; NN interpolation named in §1.5).

    The position x + u is formed and rounded in float32 (floor(q + 0.5), clamped), so that the
    same float32 displacement gives the same labels on any IEEE implementation.
    """
    Z, Y, X = L0.shape
    u = np.asarray(u10, np.float32)
    gz, gy, gx = [a.astype(np.float32) for a in _grid(L0.shape)]
    half = np.float32(0.5)
    ix = np.clip(np.floor((gx + u[0]) + half), 0, X - 1).astype(np.int64)
    iy = np.clip(np.floor((gy + u[1]) + half), 0, Y - 1).astype(np.int64)
    iz = np.clip(np.floor((gz + u[2]) + half), 0, Z - 1).astype(np.int64)
    return np.asarray(L0)[iz, iy, ix]


def warp(img, u):
    """img o (id + u) by trilinear interpolation (deformed template / target, §2.4)."""
    gz, gy, gx = _grid(img.shape)
    u = np.asarray(u, np.float64)
    return trilinear(img, gx + u[0], gy + u[1], gz + u[2])


def dice(A, B):
    """Mean over labels > 0 present in A or B of 2|A=l and B=l| / (|A=l| + |B=l|)."""
    A = np.asarray(A).ravel()
    B = np.asarray(B).ravel()
    labels = np.union1d(np.unique(A), np.unique(B))
    labels = labels[labels > 0]
    if labels.size == 0:
        return 1.0
    vals = []
    for l in labels:
        a = A == l
        b = B == l
        vals.append(2.0 * np.count_nonzero(a & b) / (np.count_nonzero(a) + np.count_nonzero(b)))
    return float(np.mean(vals))


def downsample(f, factor):
    """Block mean over factor^3 blocks; the grid is padded by edge replication to a multiple
    of the factor, so the coarse size is ceil(N_d / factor)."""
    f = np.asarray(f, np.float64)
    if factor == 1:
        return f.copy()
    Z, Y, X = f.shape
    nz, ny, nx = -(-Z // factor), -(-Y // factor), -(-X // factor)
    g = np.pad(f, ((0, nz * factor - Z), (0, ny * factor - Y), (0, nx * factor - X)), mode="edge")
    return g.reshape(nz, factor, ny, factor, nx, factor).mean(axis=(1, 3, 5))


def upsample_velocity(v, fine_shape, f_coarse, f_fine):
    """Trilinear resampling of v (T,3,...) from a grid of spacing f_coarse to one of spacing
    f_fine, with cell-centred coordinates; values are physical so they are not rescaled."""
    v = np.asarray(v, np.float64)
    gz, gy, gx = _grid(fine_shape)
    r = f_fine / f_coarse
    qx, qy, qz = (gx + 0.5) * r - 0.5, (gy + 0.5) * r - 0.5, (gz + 0.5) * r - 0.5
    out = np.empty(v.shape[:2] + tuple(fine_shape))
    for j in range(v.shape[0]):
        for e in range(3):
            out[j, e] = trilinear(v[j, e], qx, qy, qz)
    return out


def resample(f, dst_shape):
    """f sampled on another grid over the same box: trilinear interpolation at cell-centred
    coordinates, q_d = (i_d + 0.5) s_d / d_d - 0.5 source voxels along each axis (clamped).  Used
    by the warm start to move masks to the network's grid and velocities back; a velocity in
    voxels of one grid becomes one in voxels of the other by the ratio of the sizes along its own
    axis, which the caller applies."""
    f = np.asarray(f, np.float64)
    gz, gy, gx = _grid(dst_shape)
    (sz, sy, sx), (dz, dy, dx) = f.shape, tuple(dst_shape)
    return trilinear(f, (gx + 0.5) * sx / dx - 0.5, (gy + 0.5) * sy / dy - 0.5,
                     (gz + 0.5) * sz / dz - 0.5)


def register(I0, I1, M, p: Params, iterations, factors=(1,), v0=None, workers=None):
    """Multiscale gradient descent: at each factor f the inputs are block-averaged by f, the
    spacing is f, and v is carried over by upsample_velocity.  Returns (v, energies, u10)."""
    I0 = np.asarray(I0, np.float64)
    shape = I0.shape
    v = v0
    f_prev = None
    energies = []
    res = None
    for f in factors:
        lvl_shape = tuple(-(-n // f) for n in shape)
        a0, a1, am = downsample(I0, f), downsample(I1, f), downsample(M, f)
        pl = dataclasses.replace(p, h=(p.h[0] * f, p.h[1] * f, p.h[2] * f))
        if v is None:
            v = np.zeros((p.T, 3) + lvl_shape)
        elif f_prev is not None:
            v = upsample_velocity(v, lvl_shape, f_prev, f)
        for _ in range(iterations):
            res = lddmm_step(v, a0, a1, am, pl, workers=workers)
            energies.append((f, res.E_reg, res.E_data))
            v = res.v_new
        f_prev = f
    return v, energies, res
