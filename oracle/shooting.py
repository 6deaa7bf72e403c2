"""FP64 CPU oracle for geodesic shooting of the velocity field (EPDiff).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA path.

LDDMM's minimisers are geodesics (Beg et al. 2005, cited in §2.4): the time-varying field
follows from its initial value v_0 through the Euler-Poincare equation (EPDiff) of the metric
L^T L.  With the momentum m = L^T L v and v = K m (K = (L^T L)^-1, §2.4's smoothing operator),
EPDiff  d m / dt = - ad*_v m  has the solution
    m_t = Ad*_{phi_t^-1} m_0 = |D phi_{t,0}| (D phi_{t,0})^T (m_0 o phi_{t,0}),
the initial momentum transported by the flow (phi_{t,0} carries time-t positions back to 0).

Readings (the paper does not shoot; these are the discrete choices made here):
* phi_{j,0} comes from the same semi-Lagrangian steps as the registration's forward sweep:
  phi_{j+1,0}(x) = phi_{j,0}(x - dt v_j(x)), trilinear, clamp to edge; dt = 1/T.
* m_0 o phi is a trilinear lookup (clamp to edge); D phi is taken by central differences inside
  and one-sided at the faces, in physical units: (D phi)_ik = (h_i / h_k) d phi_i / d x_k in
  voxel coordinates.
* L = gamma - alpha Lap_h (periodic 7-point), so L^T L and K are exact inverses on the grid.
* v_{j+1} = K m_{j+1} for j = 0..T-2, giving the T samples v_0..v_{T-1} the registration uses.

`ad_star` and `shoot_eulerian` (forward Euler on the momentum equation with central
differences) are a second discretisation of the same equation, used only to cross-check the
transport form at small amplitude (forward Euler on this advection is unstable for large
velocities, which is why the transport form is the one built).
"""
from __future__ import annotations

import numpy as np

from . import lddmm as _L

__all__ = ["momentum", "transport_momentum", "shoot", "ddx", "ad_star", "shoot_eulerian"]


def momentum(v, alpha, gamma, h):
    """m = L^T L v = (gamma - alpha Lap_h)^2 v per component."""
    return np.stack([_L.apply_L(_L.apply_L(v[c], alpha, gamma, h), alpha, gamma, h)
                     for c in range(3)])


def transport_momentum(m0, u, h):
    """|D phi| (D phi)^T (m0 o phi) for phi = id + u (u: displacement in voxels, (3,Z,Y,X))."""
    shape = m0.shape[1:]
    gz, gy, gx = _L._grid(shape)
    px, py, pz = gx + u[0], gy + u[1], gz + u[2]
    mm = np.stack([_L.trilinear(m0[c], px, py, pz) for c in range(3)])
    # J[i][k] = d phi_i / d x_k in voxel coordinates (fd_gradient: central inside, one-sided
    # at the faces), then scaled to physical units
    J = np.empty((3, 3) + shape)
    for i in range(3):
        g = _L.fd_gradient(u[i])
        for k in range(3):
            J[i, k] = g[k] + (1.0 if i == k else 0.0)
    h = np.asarray(h, np.float64)
    for i in range(3):
        for k in range(3):
            J[i, k] *= h[i] / h[k]
    det = (J[0, 0] * (J[1, 1] * J[2, 2] - J[1, 2] * J[2, 1])
           - J[0, 1] * (J[1, 0] * J[2, 2] - J[1, 2] * J[2, 0])
           + J[0, 2] * (J[1, 0] * J[2, 1] - J[1, 1] * J[2, 0]))
    out = np.empty_like(mm)
    for k in range(3):            # ((D phi)^T m)_k = sum_i J[i][k] m_i
        out[k] = det * (J[0, k] * mm[0] + J[1, k] * mm[1] + J[2, k] * mm[2])
    return out


def shoot(v0, p: "_L.Params"):
    """v_j for j = 0..T-1 from v_0 (3, Z, Y, X): v_{j+1} = K |D phi| (D phi)^T (m_0 o phi) with
    phi = phi_{j+1,0} from the semi-Lagrangian forward steps of v_0..v_j."""
    v = np.asarray(v0, np.float64)
    shape = v.shape[1:]
    gz, gy, gx = _L._grid(shape)
    m0 = momentum(v, p.alpha, p.gamma, p.h)
    u = np.zeros((3,) + shape)
    out = [v]
    dt = 1.0 / p.T
    for _ in range(p.T - 1):
        d = dt * _L._vox(v, p.h)
        u = -d + _L.interp_vec(u, gx - d[0], gy - d[1], gz - d[2])
        m = transport_momentum(m0, u, p.h)
        v = np.stack([_L.apply_K(m[c], p.alpha, p.gamma, p.h) for c in range(3)])
        out.append(v)
    return np.stack(out)


def ddx(f, axis, h):
    """Central difference along x (axis 0), y (1) or z (2) of f[z][y][x], periodic."""
    ax = {0: 2, 1: 1, 2: 0}[axis]
    return (np.roll(f, -1, ax) - np.roll(f, 1, ax)) / (2.0 * h[axis])


def ad_star(v, m, h):
    """(ad*_v m)_i = sum_j (d_i v_j) m_j + sum_j v_j d_j m_i + m_i div v (components x, y, z)."""
    v = np.asarray(v, np.float64)
    m = np.asarray(m, np.float64)
    div = ddx(v[0], 0, h) + ddx(v[1], 1, h) + ddx(v[2], 2, h)
    out = np.empty_like(m)
    for i in range(3):
        s = m[i] * div
        for j in range(3):
            s = s + ddx(v[j], i, h) * m[j] + v[j] * ddx(m[i], j, h)
        out[i] = s
    return out


def shoot_eulerian(v0, p: "_L.Params"):
    """Forward Euler on dm/dt = -ad*_v m (small amplitudes only; see the module notes)."""
    v = np.asarray(v0, np.float64)
    m = momentum(v, p.alpha, p.gamma, p.h)
    out = [v]
    dt = 1.0 / p.T
    for _ in range(p.T - 1):
        m = m - dt * ad_star(v, m, p.h)
        v = np.stack([_L.apply_K(m[c], p.alpha, p.gamma, p.h) for c in range(3)])
        out.append(v)
    return np.stack(out)
