"""The learned warm start at the benchmark's grid: the 64^3 network shipped in the package
(trained on 2000 ellipsoid-union pairs labelled by converged plain LDDMM), its resampling to
264x160x228, and the time to the plain method's final masked-SSD energy and Dice."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import warm64 as W
    assert os.path.exists(W.WEIGHTS)
    return W


def test_converged_plain_stop_rule(W):
    """Plain LDDMM with backtracking stops at the first k >= 10 with |E_{k-10} - E_k| <= 1e-4
    E_k, and its energies never rise."""
    from paper_1605_02060_gb300 import synth
    pr = synth.union_pair((64, 64, 64), seed=1234, amplitude=6.0)
    r = W.converged_plain(W._dev(pr.I0), W._dev(pr.I1), W._dev(pr.M))
    E = r["energies"]
    k = len(E) - 1
    assert r["iterations"] < 500
    assert abs(E[k - 10] - E[k]) <= 1e-4 * E[k]
    assert all(abs(E[i - 10] - E[i]) > 1e-4 * E[i] for i in range(10, k))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(E, E[1:]))
    assert tuple(r["v"].shape) == (10, 3, 64, 64, 64)


def test_prediction_units_and_start_never_above_plain(W):
    """The predicted v_0 comes back on the registration grid, finite, with each component in
    voxels of that grid; the chosen start's energy is at most the plain start's (v = 0 is a
    candidate)."""
    from paper_1605_02060_gb300 import lddmm as L
    from paper_1605_02060_gb300 import synth
    pair, _ = synth.brain_pair(shape=(114, 80, 132), base_shape=(114, 80, 132), seed=1)
    I0, I1, M = W._dev(pair.I0), W._dev(pair.I1), W._dev(pair.M)
    net = W.load_net(W.WEIGHTS)
    v0 = W.predict_v0(net, I0, I1, pair.I0.shape)
    assert tuple(v0.shape) == (3, 114, 80, 132) and bool(torch.isfinite(v0).all())
    p = L.default_params(132, 80, 114, T=10, k_mode=1, flags=1)
    with L.Lddmm(p, I0, I1, M) as ctx:
        e0 = ctx.energy()["total"]
        c, e, cands = W.warm_start(ctx, net, I0, I1)
        assert cands[0] == pytest.approx(e0, rel=1e-12)
        assert e == min(cands) and e <= e0
        assert ctx.energy()["total"] == pytest.approx(e, rel=1e-9)


def test_warm_start_reaches_the_plain_energy_and_dice_in_a_fraction_of_the_iterations(W):
    """At 264x160x228 (the brain pair), plain LDDMM converges in ~200 iterations; from the warm
    start the plain final masked-SSD energy and Dice (within 0.005) are reached in under a
    quarter of them, for the bf16x3 K."""
    net = W.load_net(W.WEIGHTS)
    r = W.measure(net, variants=((1, 0),))
    w = r["warm"][0]
    print("\nplain %d iterations %.3f s; warm %d iterations %.3f s (scale %.3f), speedup %.2f" %
          (r["plain_iterations"], r["plain_wall_s"], w["iterations"], w["wall_s"], w["scale"],
           w["speedup"]))
    assert w["reached"]
    assert w["scale"] > 0
    assert w["iterations"] * 4 < r["plain_iterations"]
