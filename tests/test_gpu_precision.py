"""Precision form: storage of v and the images in bf16 (FP32 arithmetic, FP64 reductions) and the
precision of the DFT products (FP32, bf16x3, bf16), each compared with the FP64 oracle on the
same registration.  Reported per output (phi_10, deformed template J0, energy, Dice of the
transferred labels); run with -s to print the table."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)
    return t.to(torch.float32).numpy()


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
def problem():
    from oracle import lddmm as O
    from paper_1605_02060_gb300 import synth
    pair, _ = synth.brain_pair(shape=(57, 40, 66), base_shape=(114, 80, 132), seed=1)
    T, iters = 10, 10
    po = O.Params(T=T)
    v = np.zeros((T, 3) + pair.I0.shape)
    E = []
    for _ in range(iters):
        r = O.lddmm_step(v, pair.I0, pair.I1, pair.M, po)
        E.append(r.E)
        v = r.v_new
    J1, W, u01, _ = O.backward_sweep(v, pair.I1, pair.M, po)
    _, u10, J0T, Ed = O.forward_sweep(v, pair.I0, pair.I1, pair.M, J1, W, po)
    Efinal = O.reg_energy(v, po) + Ed
    labels = O.transfer_labels(pair.L0, u10)
    return dict(pair=pair, T=T, iters=iters, v=v, u10=u10, J0T=J0T, E=E, Efinal=Efinal,
                labels=labels, dice=O.dice(labels, pair.L1_true))


VARIANTS = [("fp32 store, fp32 K", 0, 0), ("fp32 store, bf16x3 K", 0, 1),
            ("fp32 store, bf16 K", 0, 2), ("bf16 store, bf16x3 K", 1, 1)]


def _run(L, pb, storage, kmode):
    pair = pb["pair"]
    Z, Y, X = pair.I0.shape
    p = L.default_params(X, Y, Z, T=pb["T"], k_mode=kmode, storage=storage)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        E = [ctx.step()["total"] for _ in range(pb["iters"])]
        u10 = ctx.get_field(L.LDDMM_FIELD_U10)
        J0 = ctx.get_field(L.LDDMM_FIELD_J0)
        Ef = ctx.energy()["total"]
        labels = ctx.transfer_labels(pair.L0)
        v = ctx.get_velocity()
        dice = ctx.dice(labels, pair.L1_true)
    return dict(E=E, u10=u10, J0=J0, Ef=Ef, labels=labels, v=v, dice=dice)


def test_precision_report(L, problem):
    pb = problem
    rows = []
    res = {}
    for name, storage, kmode in VARIANTS:
        r = _run(L, pb, storage, kmode)
        res[name] = r
        rows.append((name, _rel(r["v"], pb["v"]), _rel(r["u10"], pb["u10"]), _rel(r["J0"], pb["J0T"]),
                     abs(r["Ef"] - pb["Efinal"]) / pb["Efinal"], abs(r["dice"] - pb["dice"]),
                     float(np.mean(r["labels"] != pb["labels"]))))
    print("\nprecision vs FP64 oracle, brain pair 66x40x57, T=10, 10 iterations")
    print("%-22s %10s %10s %10s %10s %10s %10s" % ("variant", "v", "phi_10", "J0", "E", "dDice",
                                                    "labels!="))
    for row in rows:
        print("%-22s %10.2e %10.2e %10.2e %10.2e %10.2e %10.2e" % row)
    byname = {r[0]: r for r in rows}
    # float storage with FP32-accurate products: the iteration matches the oracle closely
    for n in ("fp32 store, fp32 K", "fp32 store, bf16x3 K"):
        _, ev, eu, ej, eE, ed, _ = byname[n]
        assert ev < 1e-3 and eu < 1e-3 and ej < 1e-3 and eE < 1e-4 and ed < 0.005, byname[n]
    # reduced precision: bounded, and Dice within 0.005
    for n in ("fp32 store, bf16 K", "bf16 store, bf16x3 K"):
        _, ev, eu, ej, eE, ed, _ = byname[n]
        assert ev < 5e-2 and eu < 5e-2 and ej < 2e-2 and eE < 1e-2 and ed < 0.005, byname[n]


def test_bf16_storage_single_step_matches_oracle_on_quantised_inputs(L):
    """One iteration from a bf16-quantised v: maps and energies see exactly the stored values,
    so they match the oracle fed the same quantised v to FP32 accuracy; the updated v carries one
    bf16 rounding (relative 2^-9)."""
    from oracle import lddmm as O
    from paper_1605_02060_gb300 import synth
    pair = synth.ellipsoid_pair(seed=0)
    T = 10
    v0 = _bf16(synth.smooth_velocity(T, (32, 32, 32), 2.0, seed=4))
    ref = O.lddmm_step(v0, pair.I0, pair.I1, pair.M, O.Params(T=T))
    p = L.default_params(32, 32, 32, T=T, storage=1, k_mode=1)
    with L.Lddmm(p, pair.I0, pair.I1, pair.M) as ctx:
        ctx.set_velocity(v0)
        np.testing.assert_array_equal(ctx.get_velocity(), v0)
        u10 = ctx.get_field(L.LDDMM_FIELD_U10)
        e = ctx.step()
        v1 = ctx.get_velocity()
    assert _rel(u10, ref.u10) < 1e-5
    assert abs(e["total"] - ref.E) <= 1e-5 * ref.E
    assert _rel(v1, ref.v_new) < 4e-3
    # each stored value is the FP32 result rounded once to bf16: within one bf16 ulp
    ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(ref.v_new), 1e-30))) - 7)
    assert np.all(np.abs(v1 - ref.v_new) <= ulp + 1e-6 * np.abs(ref.v_new).max())
