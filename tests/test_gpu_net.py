"""GPU checks of the warm-start network kernels against the FP64 oracle (same bf16-rounded
weights), of whole-network gradients, of Adam, and of the gain of the trained network: a warm
start from its prediction reaches the plain method's energy in fewer iterations."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import lddmm as L
    return L.load()


P = lambda t: ctypes.c_void_p(t.data_ptr())
L_INVALID = -1


def _bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("B,Ci,Co,n,k", [(2, 5, 18, 8, 3), (1, 3, 4, 12, 3), (1, 9, 33, 4, 3),
                                        # input channels in groups of 16: tensor-core path
                                        (2, 16, 3, 8, 1), (2, 16, 32, 8, 3), (1, 32, 16, 12, 3),
                                        (2, 48, 16, 8, 3), (1, 128, 128, 8, 3), (1, 16, 33, 12, 3),
                                        (2, 32, 30, 8, 1)])
def test_conv_kernels_match_oracle(lib, B, Ci, Co, n, k):
    from oracle import surrogate as S
    rng = np.random.default_rng(0)
    x = rng.standard_normal((B, Ci, n, n, n)).astype(np.float32)
    w = rng.standard_normal((Co, Ci, k ** 3)).astype(np.float32)
    b = rng.standard_normal(Co).astype(np.float32)
    dy = rng.standard_normal((B, Co, n, n, n)).astype(np.float32)
    wb = _bf(w)
    wq = wb.float().numpy()
    xd, dyd, bd = (torch.from_numpy(a).cuda() for a in (x, dy, b))
    wbd = wb.cuda()
    y = torch.empty((B, Co, n, n, n), device="cuda")
    assert lib.lddmm_net_conv3d_fwd(P(xd), P(wbd), P(bd), P(y), B, Ci, Co, n, k, 0, 0, None) == 0
    dx = torch.empty_like(xd)
    scratch = torch.empty(Ci * Co * k ** 3, dtype=torch.bfloat16, device="cuda")
    assert lib.lddmm_net_conv3d_dgrad(P(dyd), P(wbd), P(scratch), P(dx), B, Ci, Co, n, k, None) == 0
    dw = torch.zeros((Co, Ci, k ** 3), device="cuda")
    db = torch.zeros(Co, device="cuda")
    nsc = lib.lddmm_net_conv3d_wgrad_scratch(B, Ci, Co, n, k)
    assert nsc > 0
    wsc = torch.empty(nsc, device="cuda")
    assert lib.lddmm_net_conv3d_wgrad(P(xd), P(dyd), P(dw), P(db), P(wsc), nsc - 1, B, Ci, Co, n, k,
                                      None) == L_INVALID
    assert lib.lddmm_net_conv3d_wgrad(P(xd), P(dyd), P(dw), P(db), P(wsc), nsc, B, Ci, Co, n, k,
                                      None) == 0
    # a second call on zeroed sums gives the same bits (fixed-order partial sums, no atomics)
    dw2, db2 = torch.zeros_like(dw), torch.zeros_like(db)
    assert lib.lddmm_net_conv3d_wgrad(P(xd), P(dyd), P(dw2), P(db2), P(wsc), nsc, B, Ci, Co, n, k,
                                      None) == 0
    torch.cuda.synchronize()
    assert torch.equal(dw, dw2) and torch.equal(db, db2)
    assert _rel(y.cpu().numpy(), S.conv3d(x, wq, b)) < 1e-5
    assert _rel(dx.cpu().numpy(), S.conv3d_dgrad(dy, wq)) < 1e-5
    gw, gb = S.conv3d_wgrad(x, dy, k)
    assert _rel(dw.cpu().numpy(), gw) < 1e-5
    assert _rel(db.cpu().numpy(), gb) < 1e-5


def test_resampling_and_loss_kernels(lib):
    from oracle import surrogate as S
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 8, 8, 8)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    p = torch.empty((2, 3, 4, 4, 4), device="cuda")
    assert lib.lddmm_net_pool2(P(xd), P(p), 6, 8, 0, None) == 0
    pb = torch.empty_like(xd)
    assert lib.lddmm_net_pool2(P(p), P(pb), 6, 8, 1, None) == 0
    u = torch.zeros((2, 5, 16, 16, 16), device="cuda")
    assert lib.lddmm_net_up2(P(xd), P(u), 2, 3, 8, 5, 1, 0, None) == 0
    ub = torch.empty_like(xd)
    assert lib.lddmm_net_up2(P(u), P(ub), 2, 3, 8, 5, 1, 1, None) == 0
    t = torch.from_numpy(rng.standard_normal(x.shape).astype(np.float32)).cuda()
    g = torch.empty_like(xd)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.lddmm_net_mse(P(xd), P(t), P(g), xd.numel(), P(loss), None) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), S.pool2(x), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(pb.cpu().numpy(), S.pool2_bwd(S.pool2(x)), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(u[:, 1:4].cpu().numpy(), S.up2(x), rtol=0, atol=0)
    np.testing.assert_allclose(ub.cpu().numpy(), S.up2_bwd(S.up2(x)), rtol=1e-6)
    lo, go = S.mse(x, t.cpu().numpy())
    assert abs(float(loss) / x.size - lo) <= 1e-6 * lo
    assert _rel(g.cpu().numpy(), go) < 1e-6


def test_adam_matches_oracle(lib):
    from oracle import surrogate as S
    rng = np.random.default_rng(2)
    w = rng.standard_normal(1000).astype(np.float32)
    m = np.zeros(1000)
    v = np.zeros(1000)
    wd, md, vd = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (w, m, v))
    wo = w.astype(np.float64)
    for step in range(1, 4):
        g = rng.standard_normal(1000).astype(np.float32)
        gd = torch.from_numpy(g).cuda()
        assert lib.lddmm_net_adam(P(wd), P(gd), P(md), P(vd), None, 1000, 1e-2, 0.9, 0.999, 1e-8,
                                  step, None) == 0
        wo, m, v = S.adam(wo, g.astype(np.float64), m, v, 1e-2, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(wd.cpu().numpy(), wo, rtol=1e-5, atol=1e-6)


def test_network_gradients_match_oracle(lib):
    from oracle import surrogate as S
    from paper_1605_02060_gb300.surrogate import UNet3D
    chans, B, n = (4, 8, 8), 2, 8
    net = UNet3D(chans=chans, cout=3, n=n, batch=B, seed=3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((B, 2, n, n, n)).astype(np.float32)
    t = rng.standard_normal((B, 3, n, n, n)).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda())
    net.loss_and_grad(torch.from_numpy(t).cuda())
    net.backward(net.dy)
    torch.cuda.synchronize()
    params = [(wb.float().cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64))
              for wb, b in zip(net.wb, net.b)]
    yo, acts = S.net_forward(params, x, chans)
    assert _rel(y.cpu().numpy(), yo) < 1e-4
    _, dyo = S.mse(yo, t)
    grads = S.net_backward(params, acts, dyo, chans)
    for i, ((gw, gb), dw, db) in enumerate(zip(grads, net.dw, net.db)):
        assert _rel(dw.cpu().numpy(), gw) < 1e-3, i
        assert _rel(db.cpu().numpy(), gb) < 1e-3, i


def test_trained_network_warm_start_saves_iterations(lib):
    """Train on 240 pairs at 32^3 (x8 mirror images) labelled by 60 plain iterations; training is
    deterministic (fixed-order weight-gradient sums).  On 8 held-out pairs, with backtracking in
    every run so that accepted energies never rise:
    * the prediction is closer to the plain field than v = 0;
    * the warm start (prediction smoothed by gamma^2 K, scale chosen by the energy among
      candidates that include the plain start v = 0) never starts above the plain start, by
      construction, and in practice far below it;
    * ten warm iterations are worth more than twenty plain ones on every pair: plain LDDMM needs
      more than 20 iterations to reach the energy that the warm start reaches within 10.
    The comparison is made at the warm run's energy rather than at a fixed plain target because
    Beg's direction is not the exact gradient of the discrete energy: near a minimum it stops
    being a descent direction, backtracking then shrinks the step to nothing, and plain and warm
    runs come to rest at energies that differ by up to about 2% either way."""
    from paper_1605_02060_gb300 import surrogate as SG
    n, T, iters = 32, 10, 60
    train_pairs = SG.make_pairs(240, n, seed0=1000, amp_max=4.0)
    X, Y = SG.label_pairs(train_pairs, iters, T)
    X, Y = SG.augment_flips(X, Y, T)
    scale = float(np.sqrt((Y ** 2).mean()))
    net = SG.UNet3D(n=n, batch=8, seed=0, out_scale=scale)
    hist = SG.train(net, X, Y, epochs=6, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    rels, start_ratio, k_plain, cs = [], [], [], []
    for pr in SG.make_pairs(8, n, seed0=5000, amp_max=4.0):
        v, _, _, _ = SG.run_plain(pr, iters, T)
        pred = SG.warm_start_field(net, pr, T)
        rels.append(_rel(pred, v.cpu().numpy()))
        _, Ep, _, _ = SG.run_plain(pr, 2 * iters, T, flags=1)      # Ep[k]: E(v_k), v_0 = 0
        _, c, _, _ = SG.run_warm(net, pr, -np.inf, 10, T, flags=1)
        Ew = SG.run_warm.last_energies                              # start, then 10 iterations
        assert len(Ew) == 11
        start_ratio.append(Ew[0] / Ep[0])
        reach = [k for k, e in enumerate(Ep) if e <= Ew[-1]]
        k_plain.append(reach[0] if reach else len(Ep))
        cs.append(c)
    print("\nheld-out prediction rel-L2 %s; chosen scales %s; start energy / plain start %s; plain "
          "iterations to the energy reached within 10 warm iterations: %s" %
          (np.round(rels, 3), cs, np.round(start_ratio, 3), k_plain))
    assert np.mean(rels) < 0.9
    assert max(start_ratio) <= 1.0
    assert np.median(start_ratio) < 0.3, start_ratio
    assert min(k_plain) > 20, k_plain


@pytest.mark.parametrize("src,dst", [((64, 64, 64), (228, 160, 264)), ((57, 40, 66), (16, 16, 16)),
                                     ((5, 7, 9), (5, 7, 9))])
def test_resample_and_scale_match_oracle(lib, src, dst):
    """The warm start's grid changes: a [2][3] stack of vector fields with per-component unit
    scales against the oracle's cell-centred resampling, and x <- c x."""
    from oracle import lddmm as O
    from paper_1605_02060_gb300 import lddmm as L
    rng = np.random.default_rng(6)
    f = rng.standard_normal((2, 3) + src).astype(np.float32)
    sc = (dst[2] / src[2], dst[1] / src[1], dst[0] / src[0])
    out = L.resample(torch.from_numpy(f).cuda(), dst, ncomp=3, scale=sc)
    L.scale_(out, 0.5)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for t in range(2):
        for c in range(3):
            ref = 0.5 * sc[c] * O.resample(f[t, c], dst)
            assert _rel(got[t, c], ref) < 1e-6, (t, c)
