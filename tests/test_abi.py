"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every entry point
declared in include/lddmm.h, and rejects invalid parameters before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import lddmm as L
    return L.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lddmm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"lddmm_create", "lddmm_step", "lddmm_register", "lddmm_warp",
            "lddmm_transfer_labels"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1605_02060_gb300 import lddmm as L
    assert _declared() <= set(L._SIGS), _declared() - set(L._SIGS)


def test_library_targets_sm_103a():
    from paper_1605_02060_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


@pytest.mark.parametrize("field,value", [("nx", 1), ("T", 0), ("sigma", 0.0), ("epsilon", -1.0),
                                         ("gamma", 0.0), ("num_levels", 5), ("k_mode", 7),
                                         ("flags", 8), ("hx", 0.0)])
def test_invalid_params_rejected_without_gpu(lib, field, value):
    from paper_1605_02060_gb300 import lddmm as L
    p = L.default_params(8, 8, 8)
    setattr(p, field, value)
    a = np.zeros((8, 8, 8), np.float32)
    with pytest.raises(L.LddmmError) as ei:
        L.Lddmm(p, a, a)
    assert ei.value.code == L.LDDMM_ERR_INVALID_ARG


def test_level_schedule_validation(lib):
    from paper_1605_02060_gb300 import lddmm as L
    a = np.zeros((8, 8, 8), np.float32)
    for lf in ([2, 4, 1], [4, 2], [8, 1]):     # not decreasing / not ending at 1 / axis < 2
        p = L.default_params(8, 8, 8, level_factor=lf)
        with pytest.raises(L.LddmmError) as ei:
            L.Lddmm(p, a, a)
        assert ei.value.code == L.LDDMM_ERR_INVALID_ARG


def test_default_params(lib):
    from paper_1605_02060_gb300 import lddmm as L
    p = L.default_params(264, 160, 228)
    assert (p.nx, p.ny, p.nz, p.T) == (264, 160, 228, 10)
    assert abs(p.alpha - 0.02) < 1e-9 and p.gamma == 1.0 and abs(p.sigma - 0.1) < 1e-7
    assert ctypes.sizeof(L.lddmm_energy) == 48


def test_context_free_entry_points_reject_bad_arguments_without_gpu(lib):
    """The §2.2 preprocessing and the context entry points validate their arguments on the host
    (sizes, radii, bin and point counts, NULL pointers) before any CUDA call."""
    from paper_1605_02060_gb300 import lddmm as L
    a = np.zeros(64, np.float32)
    p = a.ctypes.data_as(ctypes.c_void_p)
    cases = [
        lambda: lib.lddmm_histogram_match(p, p, p, p, 64, 0, 8, p, None),      # bins < 1
        lambda: lib.lddmm_histogram_match(p, p, p, p, 64, 32, 65, p, None),    # points > 64
        lambda: lib.lddmm_histogram_match(p, p, p, p, 0, 32, 8, p, None),      # n = 0
        lambda: lib.lddmm_histogram_match(None, p, p, p, 64, 32, 8, p, None),  # NULL image
        lambda: lib.lddmm_mask_morphology(p, 4, 4, 4, 0.5, 17, 1, p, None),    # r_open > 16
        lambda: lib.lddmm_mask_morphology(p, 0, 4, 4, 0.5, 1, 1, p, None),     # empty grid
        lambda: lib.lddmm_shoot(None, p),
        lambda: lib.lddmm_surface_distance(None, p, p, (ctypes.c_double * 4)()),
        lambda: lib.lddmm_landmark_error(None, p, p, 1, p),
    ]
    for i, call in enumerate(cases):
        assert call() == L.LDDMM_ERR_INVALID_ARG, i
