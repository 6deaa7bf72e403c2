"""GPU parity at the benchmark's scale, with maps that have moved several voxels.

* 264x160x228, T = 10 (the benchmark's grid and launch configuration): one iteration from a
  smooth nonzero v_0 whose maps move up to ~8 voxels, so the trilinear lookups leave their
  cells, reach the clamped faces and wrap every DFT tile.  v, phi_10, phi_01, the deformed
  template and the energies against the FP64 oracle (one step: v <= 1e-4, maps and J0 <= 1e-5,
  energies 1e-5 relative); labels bit-exact on the GPU's phi_10 and Dice within 0.005.
* The same step as a precision report for the four storage / product variants, then the maps,
  deformed template, energy and Dice of the updated field against the oracle's.
* The multiscale schedule 4x / 2x / 1x to 132x80x114 (the brain pair at 100 um), T = 10, with
  5 iterations per level instead of 100 so that the FP64 oracle finishes in minutes: the final
  deformed template within 1e-3, the Dice of the transferred atlas labels within 0.005.

The oracle runs its trilinear lookups on all host cores (results do not depend on the thread
count) and its FFTs with scipy workers.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


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
def O():
    from oracle import lddmm as O
    O.set_threads(len(os.sched_getaffinity(0)))
    yield O
    O.set_threads(1)


@pytest.fixture(scope="module")
def full(O):
    """The brain pair at 264x160x228, a smooth v_0 (T = 10) and the oracle's step from it, plus
    the maps, deformed template, energy and labels of the updated field."""
    from paper_1605_02060_gb300 import synth
    pair, _ = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    T = 10
    # a field that keeps its direction over time (so the maps move ~8 voxels) plus a part that
    # varies from step to step
    v0 = (synth.smooth_velocity(1, pair.I0.shape, 8.0, seed=21)
          + synth.smooth_velocity(T, pair.I0.shape, 2.0, seed=22)).astype(np.float32)
    po = O.Params(T=T)
    r = O.lddmm_step(v0, pair.I0, pair.I1, pair.M, po, workers=-1)
    J1, W, u01_1, _ = O.backward_sweep(r.v_new, pair.I1, pair.M, po)
    _, u10_1, J0_1, Ed_1 = O.forward_sweep(r.v_new, pair.I0, pair.I1, pair.M, J1, W, po)
    E_1 = O.reg_energy(r.v_new, po) + Ed_1
    labels_1 = O.transfer_labels(pair.L0, u10_1)
    return dict(pair=pair, T=T, v0=v0, r=dict(v_new=r.v_new, u10=r.u10, u01=r.u01, J0T=r.J0T,
                                                E_reg=r.E_reg, E_data=r.E_data),
                u10_1=u10_1, J0_1=J0_1, E_1=E_1, labels_1=labels_1,
                dice_1=O.dice(labels_1, pair.L1_true))


def test_full_size_step_with_moved_maps(L, O, full):
    pair, T, v0, r = full["pair"], full["T"], full["v0"], full["r"]
    Z, Y, X = pair.I0.shape
    assert np.abs(r["u10"]).max() > 3.0 and np.abs(r["u01"]).max() > 3.0   # the maps moved
    p = L.default_params(X, Y, Z, T=T, k_mode=1)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.set_velocity(_dev(v0))
        u10 = ctx.get_field(L.LDDMM_FIELD_U10)
        u01 = ctx.get_field(L.LDDMM_FIELD_U01)
        J0 = ctx.get_field(L.LDDMM_FIELD_J0)
        labels = ctx.transfer_labels(pair.L0)
        e = ctx.step()
        v1 = ctx.get_velocity()
    assert _rel(u10, r["u10"]) < 1e-5
    assert _rel(u01, r["u01"]) < 1e-5
    assert _rel(J0, r["J0T"]) < 1e-5
    assert _rel(v1, r["v_new"]) < 1e-4
    assert _rel(v1 - v0, r["v_new"] - v0) < 1e-4
    assert abs(e["reg"] - r["E_reg"]) <= 1e-5 * r["E_reg"]
    assert abs(e["data"] - r["E_data"]) <= 1e-5 * r["E_data"]
    # nearest-neighbour labels: bit-exact given the same phi_10
    np.testing.assert_array_equal(labels, O.transfer_labels(pair.L0, u10))
    d_gpu = O.dice(labels, pair.L1_true)
    d_ref = O.dice(O.transfer_labels(pair.L0, r["u10"]), pair.L1_true)
    assert abs(d_gpu - d_ref) < 0.005


VARIANTS = [("fp32 store, fp32 K", 0, 0), ("fp32 store, bf16x3 K", 0, 1),
            ("fp32 store, bf16 K", 0, 2), ("bf16 store, bf16x3 K", 1, 1)]


def test_full_size_precision_report(L, full):
    """One iteration at 264x160x228, T = 10, from the moved v_0, for each precision variant: the
    relative L2 error of v, phi_10, J0 and the energy of the updated field against the FP64
    oracle, and the Dice difference of the transferred labels (run with -s to print)."""
    pair, T, v0 = full["pair"], full["T"], full["v0"]
    Z, Y, X = pair.I0.shape
    rows = {}
    for name, storage, kmode in VARIANTS:
        p = L.default_params(X, Y, Z, T=T, k_mode=kmode, storage=storage)
        with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
            ctx.set_velocity(_dev(v0))
            ctx.step(want_energy=False)
            v1 = torch.empty((T, 3, Z, Y, X), device="cuda")
            ctx.get_velocity(v1)
            u10 = ctx.get_field(L.LDDMM_FIELD_U10)
            J0 = ctx.get_field(L.LDDMM_FIELD_J0)
            E = ctx.energy()["total"]
            labels = ctx.transfer_labels(pair.L0)
            d = ctx.dice(labels, pair.L1_true)
        rows[name] = (_rel(v1.cpu().numpy(), full["r"]["v_new"]), _rel(u10, full["u10_1"]),
                      _rel(J0, full["J0_1"]), abs(E - full["E_1"]) / full["E_1"],
                      abs(d - full["dice_1"]), float(np.mean(labels != full["labels_1"])))
        del v1
    print("\nprecision vs FP64 oracle, brain pair 264x160x228, T=10, one iteration from a smooth v_0")
    print("%-22s %10s %10s %10s %10s %10s %10s" % ("variant", "v", "phi_10", "J0", "E", "dDice",
                                                    "labels!="))
    for name, row in rows.items():
        print("%-22s %10.2e %10.2e %10.2e %10.2e %10.2e %10.2e" % ((name,) + row))
    for n in ("fp32 store, fp32 K", "fp32 store, bf16x3 K"):
        ev, eu, ej, eE, ed, _ = rows[n]
        assert ev < 1e-4 and eu < 1e-5 and ej < 1e-5 and eE < 1e-5 and ed < 0.005, (n, rows[n])
    for n in ("fp32 store, bf16 K", "bf16 store, bf16x3 K"):
        ev, eu, ej, eE, ed, _ = rows[n]
        assert ev < 2e-2 and eu < 2e-2 and ej < 1e-2 and eE < 1e-2 and ed < 0.005, (n, rows[n])


def test_multiscale_brain_132x80x114(L, O):
    """The 4x / 2x / 1x schedule on the 100 um brain pair (levels 33x20x29, 66x40x57,
    132x80x114), T = 10, 5 iterations per level, bf16x3 K: the per-iteration energies, the
    final field, the final deformed template and the Dice of the transferred atlas labels
    against the oracle's schedule."""
    from paper_1605_02060_gb300 import synth
    pair, _ = synth.brain_pair(shape=(114, 80, 132), base_shape=(114, 80, 132), seed=1)
    Z, Y, X = pair.I0.shape
    T, iters = 10, 5
    p = L.default_params(X, Y, Z, T=T, iterations=iters, level_factor=[4, 2, 1], k_mode=1)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        trace = ctx.register()
        v = ctx.get_velocity()
        J0 = ctx.get_field(L.LDDMM_FIELD_J0)
        labels = ctx.transfer_labels(pair.L0)
    po = O.Params(T=T)
    vo, eo, _ = O.register(pair.I0, pair.I1, pair.M, po, iters, factors=(4, 2, 1), workers=-1)
    J1, W, _, _ = O.backward_sweep(vo, pair.I1, pair.M, po)
    _, u10o, J0o, _ = O.forward_sweep(vo, pair.I0, pair.I1, pair.M, J1, W, po)
    assert len(trace) == 3 * iters
    for t, (f, er, ed) in zip(trace, eo):
        assert abs(t["total"] - (er + ed)) <= 1e-4 * (er + ed)
    assert _rel(v, vo) < 1e-3
    assert _rel(J0, J0o) < 1e-3
    d_gpu = O.dice(labels, pair.L1_true)
    d_ref = O.dice(O.transfer_labels(pair.L0, u10o), pair.L1_true)
    assert abs(d_gpu - d_ref) < 0.005
