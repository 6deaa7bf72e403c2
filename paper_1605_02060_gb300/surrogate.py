"""Learned warm start for masked LDDMM: a small 3D convolutional encoder-decoder that maps a
template/target mask pair (2 x n^3) to an initial time-varying velocity field (T x 3 x n^3, as
3T output channels) for the optimiser.

Every forward, backward and optimiser step runs in liblddmm's CUDA kernels (lddmm_net_*);
PyTorch only holds device memory.  Architecture (levels l = 0..L-1, channels chans[l]):
  encoder: per level two 3^3 convolutions + ReLU, 2x average pooling between levels;
  decoder: 2x nearest upsampling of the coarser output, concatenation [upsampled, skip], two
           3^3 convolutions + ReLU;
  head:    a 1^3 convolution to 3T output channels (the T velocities of the field).
Weights are kept in FP32 (the optimiser's master copy) and used as bf16 by the products, which
accumulate in FP32.  Targets are velocities of plain LDDMM runs, divided by a fixed scale.

The warm start smooths the prediction with gamma^2 K, lets the energy choose its scale (the
plain start v = 0 is one of the candidates) and continues with plain LDDMM.  Copying a
predicted v_0 to every time step is not used: even the exact v_0 of a plain run, copied to all
t, has a higher energy than the plain field it came from (its regularisation term is several
times larger), because the plain solution's v_t vary along t.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import lddmm as L
from . import synth


def conv_shapes(chans, cin, cout):
    """(Co, Ci, k) of every convolution in execution order."""
    shapes, c = [], cin
    for ch in chans:
        shapes += [(ch, c, 3), (ch, ch, 3)]
        c = ch
    for l in range(len(chans) - 2, -1, -1):
        shapes += [(chans[l], chans[l + 1] + chans[l], 3), (chans[l], chans[l], 3)]
    shapes.append((cout, chans[0], 1))
    return shapes


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _ck(rc):
    if rc != 0:
        raise L.LddmmError(rc, "network kernel failed")


class UNet3D:
    """The encoder-decoder on one GPU, for a fixed batch size and grid size n (a multiple of
    2^(levels-1))."""

    def __init__(self, chans=(16, 32, 64, 128), cin=2, cout=30, n=64, batch=8, seed=0,
                 device="cuda", out_scale=1.0):
        self.lib = L.load()
        self.chans, self.cin, self.cout, self.n, self.B = tuple(chans), cin, cout, n, batch
        self.dev = torch.device(device)
        self.stream = torch.cuda.current_stream(self.dev)
        self.s = ctypes.c_void_p(self.stream.cuda_stream)
        self.out_scale = float(out_scale)
        self.shapes = conv_shapes(self.chans, cin, cout)
        g = torch.Generator().manual_seed(seed)
        self.w, self.wb, self.b, self.dw, self.db = [], [], [], [], []
        self.mw, self.vw, self.mb, self.vb = [], [], [], []
        for co, ci, k in self.shapes:
            std = math.sqrt(2.0 / (ci * k ** 3))
            w = (torch.randn((co, ci, k ** 3), generator=g) * std).to(self.dev)
            if (co, ci, k) == self.shapes[-1]:
                w.mul_(0.1)
            self.w.append(w)
            self.wb.append(torch.empty(w.shape, dtype=torch.bfloat16, device=self.dev))
            _ck(self.lib.lddmm_net_cast_bf16(_p(w), _p(self.wb[-1]), w.numel(), self.s))
            self.b.append(torch.zeros(co, device=self.dev))
            for lst, like in ((self.dw, w), (self.db, self.b[-1]), (self.mw, w), (self.vw, w),
                              (self.mb, self.b[-1]), (self.vb, self.b[-1])):
                lst.append(torch.zeros_like(like))
        maxw = max(co * ci * k ** 3 for co, ci, k in self.shapes)
        self.wT = torch.empty(maxw, dtype=torch.bfloat16, device=self.dev)
        sizes = [n >> l for l in range(len(self.chans))]
        need = [self.lib.lddmm_net_conv3d_wgrad_scratch(batch, ci, co, sizes[self._level(i)], k)
                for i, (co, ci, k) in enumerate(self.shapes)]
        if min(need) < 0:
            raise L.LddmmError(int(min(need)), "bad network shape")
        self.wg_scratch = torch.empty(max(need), device=self.dev)
        self.step_count = 0
        self._alloc()

    def _level(self, i):
        """Pyramid level of convolution i (execution order: encoder, decoder, head)."""
        Lv = len(self.chans)
        if i < 2 * Lv:
            return i // 2
        if i < len(self.shapes) - 1:
            return Lv - 2 - (i - 2 * Lv) // 2
        return 0

    # ------------------------------------------------------------------ buffers
    def _alloc(self):
        B, n, d = self.B, self.n, self.dev
        Lv = len(self.chans)
        self.sizes = [n >> l for l in range(Lv)]
        e = lambda c, m: torch.empty((B, c, m, m, m), device=d)
        self.enc_in = [e(self.cin if l == 0 else self.chans[l - 1], self.sizes[l]) for l in range(Lv)]
        self.enc_mid = [e(c, m) for c, m in zip(self.chans, self.sizes)]
        self.enc_out = [e(c, m) for c, m in zip(self.chans, self.sizes)]
        self.dec_cat = [e(self.chans[l + 1] + self.chans[l], self.sizes[l]) for l in range(Lv - 1)]
        self.dec_mid = [e(self.chans[l], self.sizes[l]) for l in range(Lv - 1)]
        self.dec_out = [e(self.chans[l], self.sizes[l]) for l in range(Lv - 1)]
        self.y = e(self.cout, n)
        # gradients: g_a[l] w.r.t. a level-l output, g_b[l] w.r.t. a level-l middle activation,
        # g_cat[l] w.r.t. a decoder concatenation, g_skip[l] the skip part, g_in[l] w.r.t. an
        # encoder level input (l >= 1)
        self.g_a = [e(c, m) for c, m in zip(self.chans, self.sizes)]
        self.g_b = [e(c, m) for c, m in zip(self.chans, self.sizes)]
        self.g_cat = [e(self.chans[l + 1] + self.chans[l], self.sizes[l]) for l in range(Lv - 1)]
        self.g_skip = [e(c, m) for c, m in zip(self.chans, self.sizes)]
        self.g_in = [None] + [e(self.chans[l - 1], self.sizes[l]) for l in range(1, Lv)]
        self.dy = e(self.cout, n)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=d)

    # ------------------------------------------------------------------ kernels
    def _conv(self, li, x, y, relu, m):
        co, ci, k = self.shapes[li]
        _ck(self.lib.lddmm_net_conv3d_fwd(_p(x), _p(self.wb[li]), _p(self.b[li]), _p(y), self.B,
                                          ci, co, m, k, 1 if relu else 0, 0, self.s))

    def _conv_back(self, li, x_in, g_out, g_in, m, relu_out=None):
        """g_out: gradient w.r.t. this conv's output (post-ReLU when relu_out is given; ReLU
        backward applied in place).  Accumulates dw, db; g_in (may be None) = input gradient."""
        co, ci, k = self.shapes[li]
        if relu_out is not None:
            _ck(self.lib.lddmm_net_relu_bwd(_p(g_out), _p(relu_out), g_out.numel(), self.s))
        _ck(self.lib.lddmm_net_conv3d_wgrad(_p(x_in), _p(g_out), _p(self.dw[li]), _p(self.db[li]),
                                            _p(self.wg_scratch), self.wg_scratch.numel(),
                                            self.B, ci, co, m, k, self.s))
        if g_in is not None:
            _ck(self.lib.lddmm_net_conv3d_dgrad(_p(g_out), _p(self.wb[li]), _p(self.wT), _p(g_in),
                                                self.B, ci, co, m, k, self.s))

    # ------------------------------------------------------------------ forward / backward
    def forward(self, x):
        """x: [B][cin][n^3] float32 on the device.  Returns the output buffer (scaled units)."""
        Lv = len(self.chans)
        self.enc_in[0].copy_(x)
        li = 0
        for l in range(Lv):
            m = self.sizes[l]
            self._conv(li, self.enc_in[l], self.enc_mid[l], True, m)
            self._conv(li + 1, self.enc_mid[l], self.enc_out[l], True, m)
            li += 2
            if l < Lv - 1:
                _ck(self.lib.lddmm_net_pool2(_p(self.enc_out[l]), _p(self.enc_in[l + 1]),
                                             self.B * self.chans[l], m, 0, self.s))
        h = self.enc_out[Lv - 1]
        for l in range(Lv - 2, -1, -1):
            m, cu, cs = self.sizes[l], self.chans[l + 1], self.chans[l]
            _ck(self.lib.lddmm_net_up2(_p(h), _p(self.dec_cat[l]), self.B, cu, m // 2, cu + cs, 0, 0,
                                       self.s))
            _ck(self.lib.lddmm_net_copy_channels(_p(self.enc_out[l]), _p(self.dec_cat[l]), self.B, cs,
                                                 m ** 3, cs, 0, cu + cs, cu, 0, self.s))
            self._conv(li, self.dec_cat[l], self.dec_mid[l], True, m)
            self._conv(li + 1, self.dec_mid[l], self.dec_out[l], True, m)
            li += 2
            h = self.dec_out[l]
        self._conv(li, h, self.y, False, self.n)
        return self.y

    def backward(self, dy):
        """dy: gradient w.r.t. the output buffer.  Fills dw, db (zeroed first)."""
        for t in self.dw + self.db:
            t.zero_()
        Lv = len(self.chans)
        li = len(self.shapes) - 1
        # head (1^3 convolution, no ReLU): gradient w.r.t. the top decoder output
        self._conv_back(li, self.dec_out[0], dy, self.g_a[0], self.n)
        li -= 1
        # decoder levels in the reverse of the forward order
        for l in range(0, Lv - 1):
            m, cu, cs = self.sizes[l], self.chans[l + 1], self.chans[l]
            self._conv_back(li, self.dec_mid[l], self.g_a[l], self.g_b[l], m,
                            relu_out=self.dec_out[l])
            self._conv_back(li - 1, self.dec_cat[l], self.g_b[l], self.g_cat[l], m,
                            relu_out=self.dec_mid[l])
            li -= 2
            _ck(self.lib.lddmm_net_copy_channels(_p(self.g_cat[l]), _p(self.g_skip[l]), self.B, cs,
                                                 m ** 3, cu + cs, cu, cs, 0, 0, self.s))
            _ck(self.lib.lddmm_net_up2(_p(self.g_cat[l]), _p(self.g_a[l + 1]), self.B, cu, m // 2,
                                       cu + cs, 0, 1, self.s))
        # encoder, bottom level first; g_a[l] = gradient w.r.t. enc_out[l]
        for l in range(Lv - 1, -1, -1):
            m = self.sizes[l]
            if l < Lv - 1:
                _ck(self.lib.lddmm_net_pool2(_p(self.g_in[l + 1]), _p(self.g_a[l]),
                                             self.B * self.chans[l], m, 1, self.s))
                _ck(self.lib.lddmm_net_copy_channels(_p(self.g_skip[l]), _p(self.g_a[l]), self.B,
                                                     self.chans[l], m ** 3, self.chans[l], 0,
                                                     self.chans[l], 0, 1, self.s))
            self._conv_back(li, self.enc_mid[l], self.g_a[l], self.g_b[l], m,
                            relu_out=self.enc_out[l])
            self._conv_back(li - 1, self.enc_in[l], self.g_b[l], self.g_in[l], m,
                            relu_out=self.enc_mid[l])
            li -= 2

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for i in range(len(self.shapes)):
            _ck(self.lib.lddmm_net_adam(_p(self.w[i]), _p(self.dw[i]), _p(self.mw[i]), _p(self.vw[i]),
                                        _p(self.wb[i]), self.w[i].numel(), lr, b1, b2, eps,
                                        self.step_count, self.s))
            _ck(self.lib.lddmm_net_adam(_p(self.b[i]), _p(self.db[i]), _p(self.mb[i]), _p(self.vb[i]),
                                        None, self.b[i].numel(), lr, b1, b2, eps, self.step_count,
                                        self.s))

    def loss_and_grad(self, target):
        """MSE of the output against target (same shape, scaled units); fills self.dy."""
        self.loss_dev.zero_()
        _ck(self.lib.lddmm_net_mse(_p(self.y), _p(target), _p(self.dy), self.y.numel(),
                                   _p(self.loss_dev), self.s))
        return self.loss_dev

    def train_step(self, x, target, lr):
        self.forward(x)
        loss = self.loss_and_grad(target)
        self.backward(self.dy)
        self.adam(lr)
        return loss

    def predict(self, x):
        """Velocity prediction [B][3][n^3] in physical units, as a host array (the network works
        in units of out_scale)."""
        return self.forward(x).cpu().numpy() * np.float32(self.out_scale)

    def state(self):
        return {"chans": self.chans, "out_scale": self.out_scale,
                "w": [w.cpu().numpy() for w in self.w], "b": [b.cpu().numpy() for b in self.b]}

    def load_state(self, st):
        for i in range(len(self.shapes)):
            self.w[i].copy_(torch.from_numpy(st["w"][i]))
            self.b[i].copy_(torch.from_numpy(st["b"][i]))
            _ck(self.lib.lddmm_net_cast_bf16(_p(self.w[i]), _p(self.wb[i]), self.w[i].numel(), self.s))
        self.out_scale = float(st["out_scale"])


# ---------------------------------------------------------------------------------------------
# data: mask pairs labelled by plain LDDMM on the GPU

def make_pairs(count, n, seed0, amp_max=8.0):
    """Ellipsoid-union mask pairs at n^3 with RBF warps of amplitude in [amp_max/2, amp_max]."""
    rng = np.random.default_rng(seed0)
    pairs = []
    for i in range(count):
        amp = float(rng.uniform(0.5 * amp_max, amp_max))
        pairs.append(synth.union_pair((n, n, n), seed=seed0 + i, amplitude=amp))
    return pairs


def run_plain(pair, iters, T=10, v0=None, target_energy=None, max_iters=None, k_mode=1, flags=0):
    """Plain LDDMM on one pair.  Returns (v, energies, iterations); with target_energy it stops
    at the first iteration whose energy is <= target (at most max_iters).  flags bit 0:
    backtracking (a step that raises the energy is undone and the step size halved)."""
    n = pair.I0.shape
    p = L.default_params(n[2], n[1], n[0], T=T, k_mode=k_mode, flags=flags)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        if v0 is not None:
            ctx.set_velocity(v0)
        E, it = [], 0
        limit = max_iters if target_energy is not None else iters
        while it < limit:
            e = ctx.step()["total"]
            E.append(e)
            it += 1
            if target_energy is not None and e <= target_energy:
                break
        v = torch.empty((T, 3) + n, device="cuda")
        ctx.get_velocity(v)
        if target_energy is None or (E and E[-1] > target_energy):
            pass
        final = ctx.energy()["total"]
    return v, E, it, final


def label_pairs(pairs, iters, T=10):
    """Inputs (mask pairs) and targets (the whole field v after `iters` plain iterations, as
    3T channels)."""
    X, Y = [], []
    for pr in pairs:
        v, _, _, _ = run_plain(pr, iters, T)
        X.append(np.stack([pr.I0, pr.I1]))
        Y.append(v.reshape((3 * T,) + tuple(v.shape[2:])).cpu().numpy())
    return np.stack(X).astype(np.float32), np.stack(Y).astype(np.float32)


def augment_flips(X, Y, T=10):
    """The 8 mirror images of every sample (flips of x, y and z): the masks flip, and a velocity
    component along a flipped axis changes sign.  X: [S][2][n^3], Y: [S][3T][n^3]."""
    Xs, Ys = [X], [Y]
    for axes in ((4,), (3,), (2,), (4, 3), (4, 2), (3, 2), (4, 3, 2)):
        Xf = np.flip(X, axis=axes)
        Yf = np.flip(Y, axis=axes).copy()
        for ax in axes:
            comp = {4: 0, 3: 1, 2: 2}[ax]      # array axis -> velocity component (x, y, z)
            Yf[:, comp::3] *= -1.0
        Xs.append(np.ascontiguousarray(Xf))
        Ys.append(Yf)
    return np.concatenate(Xs), np.concatenate(Ys)


def train(net, X, Y, epochs, lr=1e-3, seed=0, log=None):
    """Adam on the MSE between net(X) and Y / out_scale, minibatches of net.B."""
    rng = np.random.default_rng(seed)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y / net.out_scale).cuda()
    nb = len(X) // net.B
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(X))
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        for bi in range(nb):
            idx = torch.from_numpy(order[bi * net.B:(bi + 1) * net.B]).cuda()
            tot += net.train_step(Xd[idx], Yd[idx], lr)
        mean = float(tot) / (nb * net.y.numel())
        hist.append(mean)
        if log:
            log(ep, mean)
    return hist


def smooth_prediction(ctx, v, gamma):
    """gamma^2 K applied to each component of the prediction (K = (gamma - alpha Lap)^-2 on the
    context's grid): unit gain at frequency zero, damps the high-frequency part of the network
    error that the regulariser would otherwise take many iterations to remove."""
    out = np.empty_like(v)
    for t in range(v.shape[0]):
        for c in range(v.shape[1]):
            out[t, c] = ctx.apply_K(np.ascontiguousarray(v[t, c])) * np.float32(gamma * gamma)
    return out


def choose_start(ctx, v_pred, scales=(0.0, 0.5, 1.0, 1.5, 2.0, 3.0)):
    """The plain method judges the prediction: among c * v_pred (c = 0 is the plain start v = 0)
    set the one of lowest energy on the context.  Returns (c, energy, energy evaluations)."""
    best = None
    for c in scales:
        ctx.set_velocity(np.ascontiguousarray(v_pred * np.float32(c)))
        e = ctx.energy()["total"]
        if best is None or e < best[1]:
            best = (c, e)
    ctx.set_velocity(np.ascontiguousarray(v_pred * np.float32(best[0])))
    return best[0], best[1], len(scales)


def choose_start_shot(ctx, v0, scales=(0.0, 0.5, 1.0, 1.5, 2.0, 3.0)):
    """The geodesic variant of choose_start: only the initial velocity c * v0 is kept, and the
    context's v_1..v_{T-1} are shot from it (EPDiff); the scale of lowest energy is set.
    Returns (c, energy, energy evaluations)."""
    best = None
    for c in scales:
        ctx.shoot(np.ascontiguousarray(v0 * np.float32(c)))
        e = ctx.energy()["total"]
        if best is None or e < best[1]:
            best = (c, e)
    ctx.shoot(np.ascontiguousarray(v0 * np.float32(best[0])))
    return best[0], best[1], len(scales)


def run_warm(net, pair, target_energy, max_iters, T=10, k_mode=1, flags=0, shoot=False):
    """Warm start (choose_start on the prediction; with shoot=True, choose_start_shot on its
    v_0), then plain LDDMM until the energy reaches target_energy.  Returns (iterations, chosen
    scale, energy evaluations, wall seconds)."""
    n = pair.I0.shape
    p = L.default_params(n[2], n[1], n[0], T=T, k_mode=k_mode, flags=flags)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        v = smooth_prediction(ctx, warm_start_field(net, pair, T), p.gamma)
        c, e, nev = choose_start_shot(ctx, v[0]) if shoot else choose_start(ctx, v)
        run_warm.last_start_energy = e
        run_warm.last_energies = [e]
        it = 0
        while it < max_iters and e > target_energy:
            e = ctx.step()["total"]
            run_warm.last_energies.append(e)
            it += 1
            if e <= target_energy:
                break
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        run_warm.last_dice = mask_dice(ctx, pair)
    return it, c, nev, wall


def run_plain_timed(pair, target_energy, max_iters, T=10, k_mode=1, flags=0):
    """Plain LDDMM from v = 0 until the energy reaches target_energy, timed like run_warm
    (context creation included).  Returns (iterations, wall seconds, Dice of the transferred
    template mask with the target mask)."""
    n = pair.I0.shape
    p = L.default_params(n[2], n[1], n[0], T=T, k_mode=k_mode, flags=flags)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        it, e = 0, float("inf")
        while it < max_iters and e > target_energy:
            e = ctx.step()["total"]
            it += 1
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        d = mask_dice(ctx, pair)
    return it, wall, d


def mask_dice(ctx, pair):
    """Dice of the template mask pulled back through the context's current map (nearest
    neighbour, §2.5) with the target mask."""
    L0 = (pair.I0 > 0.5).astype(np.uint16)
    L1 = (pair.I1 > 0.5).astype(np.uint16)
    return ctx.dice(ctx.transfer_labels(L0), L1)


def warm_start_dice(net, pair, T=10, k_mode=1):
    """Dice with the target mask of the template mask transferred by the surrogate's start alone
    (smoothed and scaled by the energy, no LDDMM iteration)."""
    n = pair.I0.shape
    p = L.default_params(n[2], n[1], n[0], T=T, k_mode=k_mode)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        v = smooth_prediction(ctx, warm_start_field(net, pair, T), p.gamma)
        choose_start(ctx, v)
        return mask_dice(ctx, pair)


def warm_iters_to_dice(net, pair, dice_target, max_iters, T=10, k_mode=1, flags=0):
    """Fewest warm-started iterations whose transferred template mask reaches Dice >=
    dice_target with the target mask (0: the start itself), or None within max_iters."""
    n = pair.I0.shape
    p = L.default_params(n[2], n[1], n[0], T=T, k_mode=k_mode, flags=flags)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        v = smooth_prediction(ctx, warm_start_field(net, pair, T), p.gamma)
        choose_start(ctx, v)
        for it in range(max_iters + 1):
            if mask_dice(ctx, pair) >= dice_target:
                return it
            if it < max_iters:
                ctx.step()
    return None


def run_warm_fixed(net, pair, iters, T=10, k_mode=1, flags=0):
    """Wall seconds of a warm start followed by exactly `iters` iterations (context creation,
    prediction, smoothing and the start's energy evaluations included)."""
    n = pair.I0.shape
    p = L.default_params(n[2], n[1], n[0], T=T, k_mode=k_mode, flags=flags)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        v = smooth_prediction(ctx, warm_start_field(net, pair, T), p.gamma)
        choose_start(ctx, v)
        for _ in range(iters):
            ctx.step(want_energy=False)
        torch.cuda.synchronize()
    return time.perf_counter() - t0


def warm_start_field(net, pair, T=10):
    """The predicted field, shaped [T][3][n^3] (host float32, physical units)."""
    x = torch.from_numpy(np.stack([pair.I0, pair.I1])[None]).cuda()
    if net.B != 1:
        x = x.expand(net.B, *x.shape[1:]).contiguous()
    v = net.predict(x)[0]
    return np.ascontiguousarray(v.reshape((T, 3) + v.shape[1:]), np.float32)
