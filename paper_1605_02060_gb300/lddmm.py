"""Thin ctypes binding of liblddmm (include/lddmm.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; there is no CPU path.  Arrays may be
``torch.Tensor`` (device or host, contiguous) or ``numpy.ndarray``; each is passed to the C
ABI as a raw pointer and the library copies host memory itself (cudaMemcpyDefault).

The functions keep the C names (``lddmm_create``, ``lddmm_step`` ...); :class:`Lddmm` is a
small owner of one context on top of them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblddmm.so")

LDDMM_OK = 0
LDDMM_ERR_INVALID_ARG = -1
LDDMM_ERR_OOM = -2
LDDMM_ERR_CUDA = -3
LDDMM_ERR_NONFINITE = -4
LDDMM_ERR_STATE = -5
LDDMM_ERR_TIMEOUT = -6

LDDMM_K_FP32 = 0
LDDMM_K_BF16X3 = 1
LDDMM_K_BF16 = 2

LDDMM_FIELD_U10 = 0
LDDMM_FIELD_U01 = 1
LDDMM_FIELD_J0 = 2
LDDMM_FIELD_I0 = 3
LDDMM_FIELD_I1 = 4
LDDMM_FIELD_M = 5


class lddmm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_float), ("hy", ctypes.c_float), ("hz", ctypes.c_float),
                ("T", ctypes.c_int),
                ("alpha", ctypes.c_float), ("gamma", ctypes.c_float), ("sigma", ctypes.c_float),
                ("epsilon", ctypes.c_float), ("iterations", ctypes.c_int),
                ("num_levels", ctypes.c_int), ("level_factor", ctypes.c_int * 4),
                ("k_mode", ctypes.c_int), ("flags", ctypes.c_int), ("timeout_s", ctypes.c_float),
                ("storage", ctypes.c_int)]


class lddmm_energy(ctypes.Structure):
    _fields_ = [("total", ctypes.c_double), ("reg", ctypes.c_double), ("data", ctypes.c_double),
                ("min_det", ctypes.c_double), ("iter", ctypes.c_int), ("level", ctypes.c_int),
                ("fold", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class lddmm_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("pad", ctypes.c_int),
                ("total_ms", ctypes.c_double)]


class LddmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("liblddmm error %d: %s" % (code, msg))
        self.code = code


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "lddmm_default_params": (ctypes.c_int, [ctypes.POINTER(lddmm_params), ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lddmm_create": (ctypes.c_int, [ctypes.POINTER(lddmm_params), _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "lddmm_set_images": (ctypes.c_int, [_P, _P, _P, _P]),
    "lddmm_step": (ctypes.c_int, [_P, ctypes.POINTER(lddmm_energy)]),
    "lddmm_register": (ctypes.c_int, [_P, ctypes.POINTER(lddmm_energy), ctypes.c_int]),
    "lddmm_set_level": (ctypes.c_int, [_P, ctypes.c_int]),
    "lddmm_grid": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lddmm_warp": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "lddmm_transfer_labels": (ctypes.c_int, [_P, _P, _P]),
    "lddmm_get_velocity": (ctypes.c_int, [_P, _P]),
    "lddmm_set_velocity": (ctypes.c_int, [_P, _P]),
    "lddmm_get_field": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lddmm_apply_K": (ctypes.c_int, [_P, _P, _P]),
    "lddmm_energy_eval": (ctypes.c_int, [_P, ctypes.POINTER(lddmm_energy)]),
    "lddmm_dice": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    "lddmm_surface_distance": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "lddmm_landmark_error": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "lddmm_shoot": (ctypes.c_int, [_P, _P]),
    "lddmm_histogram_match": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_int, _P, _P]),
    "lddmm_mask_morphology": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_float, ctypes.c_int, ctypes.c_int, _P, _P]),
    "lddmm_energy_grad": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "lddmm_set_timeout": (ctypes.c_int, [_P, ctypes.c_float]),
    "lddmm_apply_K_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                             ctypes.c_float, ctypes.c_float, _P]),
    "lddmm_profile_start": (ctypes.c_int, [_P, ctypes.c_int]),
    "lddmm_profile_stop": (ctypes.c_int, [_P, ctypes.POINTER(lddmm_kernel_stat), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    "lddmm_net_conv3d_fwd": (ctypes.c_int, [_P, _P, _P, _P] + [ctypes.c_int] * 7 + [_P]),
    "lddmm_net_conv3d_dgrad": (ctypes.c_int, [_P, _P, _P, _P] + [ctypes.c_int] * 5 + [_P]),
    "lddmm_net_conv3d_wgrad_scratch": (ctypes.c_int64, [ctypes.c_int] * 5),
    "lddmm_net_conv3d_wgrad": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64]
                               + [ctypes.c_int] * 5 + [_P]),
    "lddmm_net_relu_bwd": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "lddmm_net_pool2": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P]),
    "lddmm_net_up2": (ctypes.c_int, [_P, _P] + [ctypes.c_int] * 6 + [_P]),
    "lddmm_net_copy_channels": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
                                + [ctypes.c_int] * 5 + [_P]),
    "lddmm_net_mse": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "lddmm_net_adam": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int, _P]),
    "lddmm_net_cast_bf16": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "lddmm_resample": (ctypes.c_int, [_P] + [ctypes.c_int] * 3 + [_P] + [ctypes.c_int] * 5
                       + [ctypes.c_float] * 3 + [_P]),
    "lddmm_scale": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_float, _P]),
    "lddmm_last_error": (ctypes.c_char_p, [_P]),
    "lddmm_destroy": (None, [_P]),
}


def load(path: str | None = None):
    """Load liblddmm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("liblddmm.so not built (%s); run __graft_entry__.build() or "
                          "python -m paper_1605_02060_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch.Tensor or numpy.ndarray, got %r" % type(a))


def _check(rc, ctx=None):
    if rc != LDDMM_OK:
        msg = load().lddmm_last_error(ctx)
        raise LddmmError(rc, msg.decode() if msg else "")


def default_params(nx, ny, nz, **kw) -> lddmm_params:
    p = lddmm_params()
    _check(load().lddmm_default_params(ctypes.byref(p), nx, ny, nz))
    for k, v in kw.items():
        if k == "level_factor":
            for i, f in enumerate(v):
                p.level_factor[i] = int(f)
            p.num_levels = len(v)
        else:
            setattr(p, k, v)
    return p


class Lddmm:
    """One registration context (owns an ``lddmm_ctx``).

    ``I0``, ``I1``, ``M``: float32 arrays of shape (nz, ny, nx); ``stream``: a
    ``torch.cuda.Stream`` or raw handle; None = torch's current stream when torch has CUDA
    (so device tensors produced by torch are ordered with the library's work), else the
    legacy default stream.
    """

    def __init__(self, params: lddmm_params, I0, I1, M=None, stream=None):
        lib = load()
        self._keep = (I0, I1, M)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream()
            except ImportError:
                pass
        s = None
        if stream is not None:
            s = ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
        ctx = ctypes.c_void_p()
        rc = lib.lddmm_create(ctypes.byref(params), _ptr(I0), _ptr(I1), _ptr(M), s,
                              ctypes.byref(ctx))
        _check(rc, None)
        self.ctx = ctx
        self.params = params

    def close(self):
        if getattr(self, "ctx", None):
            load().lddmm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls ---------------------------------------------------------------------------------
    def grid(self):
        nx, ny, nz, lv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().lddmm_grid(self.ctx, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz),
                                 ctypes.byref(lv)), self.ctx)
        return nx.value, ny.value, nz.value, lv.value

    @property
    def shape(self):
        nx, ny, nz, _ = self.grid()
        return (nz, ny, nx)

    def step(self, want_energy=True):
        e = lddmm_energy()
        _check(load().lddmm_step(self.ctx, ctypes.byref(e) if want_energy else None), self.ctx)
        return e.as_dict() if want_energy else None

    def register(self):
        n = self.params.num_levels * self.params.iterations
        arr = (lddmm_energy * max(1, n))()
        _check(load().lddmm_register(self.ctx, arr, n), self.ctx)
        return [arr[i].as_dict() for i in range(n)]

    def set_level(self, level):
        _check(load().lddmm_set_level(self.ctx, level), self.ctx)

    def set_images(self, I0, I1, M=None):
        self._keep = (I0, I1, M)
        _check(load().lddmm_set_images(self.ctx, _ptr(I0), _ptr(I1), _ptr(M)), self.ctx)

    def energy(self):
        e = lddmm_energy()
        _check(load().lddmm_energy_eval(self.ctx, ctypes.byref(e)), self.ctx)
        return e.as_dict()

    def get_velocity(self, out=None):
        if out is None:
            out = np.empty((self.params.T, 3) + self.shape, np.float32)
        _check(load().lddmm_get_velocity(self.ctx, _ptr(out)), self.ctx)
        return out

    def set_velocity(self, v):
        _check(load().lddmm_set_velocity(self.ctx, _ptr(v)), self.ctx)

    def get_field(self, which, out=None):
        if out is None:
            lead = (3,) if which in (LDDMM_FIELD_U10, LDDMM_FIELD_U01) else ()
            out = np.empty(lead + self.shape, np.float32)
        _check(load().lddmm_get_field(self.ctx, which, _ptr(out)), self.ctx)
        return out

    def warp(self, src, direction=0, out=None):
        if out is None:
            out = np.empty(self.shape, np.float32)
        _check(load().lddmm_warp(self.ctx, _ptr(src), _ptr(out), direction), self.ctx)
        return out

    def transfer_labels(self, L0, out=None):
        if out is None:
            out = np.empty(self.shape, np.uint16)
        _check(load().lddmm_transfer_labels(self.ctx, _ptr(L0), _ptr(out)), self.ctx)
        return out

    def apply_K(self, src, out=None):
        if out is None:
            out = np.empty(self.shape, np.float32)
        _check(load().lddmm_apply_K(self.ctx, _ptr(src), _ptr(out)), self.ctx)
        return out

    def profile_start(self, max_launches):
        _check(load().lddmm_profile_start(self.ctx, int(max_launches)), self.ctx)

    def profile_stop(self):
        """{kernel name: (launches, total device ms)} since profile_start."""
        arr = (lddmm_kernel_stat * 64)()
        n = ctypes.c_int()
        _check(load().lddmm_profile_stop(self.ctx, arr, 64, ctypes.byref(n)), self.ctx)
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}

    def set_timeout(self, seconds):
        _check(load().lddmm_set_timeout(self.ctx, float(seconds)), self.ctx)

    def energy_grad(self, v=None, grad=None):
        """(E, dE/dv) of the discrete energy, exact reverse mode on the GPU."""
        if grad is None:
            grad = np.empty((self.params.T, 3) + self.shape, np.float32)
        E = ctypes.c_double()
        _check(load().lddmm_energy_grad(self.ctx, _ptr(v), _ptr(grad), ctypes.byref(E)), self.ctx)
        return E.value, grad

    def dice(self, A, B):
        d = ctypes.c_double()
        n = int(np.prod(A.shape))
        _check(load().lddmm_dice(self.ctx, _ptr(A), _ptr(B), n, ctypes.byref(d)), self.ctx)
        return d.value

    def shoot(self, v0):
        """Replace v_j (j = 0..T-1) by the geodesic from v0, float32 (3, nz, ny, nx)."""
        _check(load().lddmm_shoot(self.ctx, _ptr(v0)), self.ctx)

    def surface_distance(self, A, B):
        """(Hausdorff, median, #surface voxels of A, of B) between two uint8 masks (§2.7)."""
        out = (ctypes.c_double * 4)()
        _check(load().lddmm_surface_distance(self.ctx, _ptr(A), _ptr(B), out), self.ctx)
        return out[0], out[1], int(out[2]), int(out[3])

    def landmark_error(self, xk, yk, out=None):
        """|phi(x_k) - y_k| for float32 (n, 3) voxel coordinates (x, y, z); float64 (n,)."""
        n = int(xk.shape[0])
        if out is None:
            out = np.empty(n, np.float64)
        _check(load().lddmm_landmark_error(self.ctx, _ptr(xk), _ptr(yk), n, _ptr(out)), self.ctx)
        return out


def _current_stream():
    """torch's current CUDA stream as a c_void_p (None when torch or CUDA is absent)."""
    try:
        import torch
        if not torch.cuda.is_available():
            return None
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        return None


def histogram_match(I0, M0, I1, M1, out=None, bins=32, points=8):
    """Masked I0 histogram-matched to masked I1 (§2.2), device float32 tensors of one shape."""
    import torch
    if out is None:
        out = torch.empty_like(I0)
    rc = load().lddmm_histogram_match(_ptr(I0), _ptr(M0), _ptr(I1), _ptr(M1), I0.numel(), bins,
                                      points, _ptr(out), _current_stream())
    _check(rc, None)
    return out


def resample(src, dst_shape, ncomp=1, scale=(1.0, 1.0, 1.0), out=None):
    """Trilinear resampling at cell-centred coordinates of device float32 fields
    (..., sz, sy, sx) to (..., dz, dy, dx); field f scaled by scale[f % ncomp]."""
    import torch
    sz, sy, sx = src.shape[-3:]
    dz, dy, dx = dst_shape
    lead = tuple(src.shape[:-3])
    nf = int(np.prod(lead)) if lead else 1
    if out is None:
        out = torch.empty(lead + (dz, dy, dx), dtype=torch.float32, device=src.device)
    _check(load().lddmm_resample(_ptr(src), sx, sy, sz, _ptr(out), dx, dy, dz, nf, ncomp,
                                 float(scale[0]), float(scale[1]), float(scale[2]),
                                 _current_stream()), None)
    return out


def scale_(x, c):
    """x <- c x in place (device float32 tensor)."""
    _check(load().lddmm_scale(_ptr(x), x.numel(), float(c), _current_stream()), None)
    return x


def mask_morphology(I, threshold, r_open, r_close, out=None):
    """[I > threshold] opened with ball(r_open), closed with ball(r_close) (§2.2); device
    float32 (nz, ny, nx) in, uint8 out."""
    import torch
    nz, ny, nx = I.shape
    if out is None:
        out = torch.empty(I.shape, dtype=torch.uint8, device=I.device)
    rc = load().lddmm_mask_morphology(_ptr(I), nx, ny, nz, float(threshold), int(r_open),
                                      int(r_close), _ptr(out), _current_stream())
    _check(rc, None)
    return out


def lddmm_apply_K_noalloc(src, dst, h=(1.0, 1.0, 1.0), alpha=0.02, gamma=1.0, stream=None):
    """K src -> dst for device float32 tensors of shape (nz, ny, nx) without any GPU allocation
    (scratch lives in a fixed static device array; see include/lddmm.h for the limits)."""
    nz, ny, nx = src.shape
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream() if torch.cuda.is_available() else None
        except ImportError:
            stream = None
    s = None if stream is None else ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
    _check(load().lddmm_apply_K_noalloc(_ptr(src), _ptr(dst), nx, ny, nz, h[0], h[1], h[2],
                                        alpha, gamma, s))
    return dst


# C-named module functions (same names as the ABI)
def lddmm_create(params, I0, I1, M=None, stream=None):
    return Lddmm(params, I0, I1, M, stream)


def lddmm_step(ctx: Lddmm, want_energy=True):
    return ctx.step(want_energy)


def lddmm_register(ctx: Lddmm):
    return ctx.register()


def lddmm_warp(ctx: Lddmm, src, direction=0, out=None):
    return ctx.warp(src, direction, out)


def lddmm_transfer_labels(ctx: Lddmm, L0, out=None):
    return ctx.transfer_labels(L0, out)


def lddmm_destroy(ctx: Lddmm):
    ctx.close()
