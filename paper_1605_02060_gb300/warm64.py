"""Learned warm start on a 64^3 network grid for registrations at any grid size.

The network (4 levels, 16/32/64/128 channels, bf16 weights, FP32 accumulation; surrogate.UNet3D)
maps a template/target mask pair on a 64^3 grid covering the whole box to the initial velocity
v_0 (3 x 64^3) of a converged plain LDDMM run on that grid.  Training pairs are ellipsoid-union
masks with RBF warps (amplitude up to 8 voxels); their labels come from plain LDDMM run with
backtracking until the energy stops moving: relative change below 1e-4 over 10 iterations, at
most 500 iterations.

At a registration of size (X, Y, Z) the masks are resampled to 64^3 (cell-centred trilinear),
the predicted v_0 is resampled back with its components scaled to voxels of the registration
grid (x by X/64, y by Y/64, z by Z/64; the network grid is an anisotropic resample of the box),
smoothed by gamma^2 K and copied to every time step.  Among c v_0 for a few scales c the one of
lowest energy is kept (c = 0 is the plain start v = 0, so the warm start never starts above
plain LDDMM); plain iterations follow.  (Shooting v_1..v_{T-1} from v_0 along the geodesic,
EPDiff as lddmm_shoot, is available as an option: at 264x160x228 the shot field grows from step
to step for the predicted v_0 and its energy is not finite, so the copy is the default.)
Every step runs in liblddmm's kernels; PyTorch holds the device memory.

The network trained by the first command below ships as weights/warm64.npz (bf16 weights).

    python -m paper_1605_02060_gb300.warm64 train --out weights.npz [--pairs 2000]
    python -m paper_1605_02060_gb300.warm64 measure [--weights weights.npz]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import lddmm as L
from . import surrogate as SG
from . import synth

NG = 64                     # network grid
CHANS = (16, 32, 64, 128)
SCALES = (0.0, 0.125, 0.25, 0.375, 0.5, 0.75, 1.0)
WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "weights", "warm64.npz")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def converged_plain(I0, I1, M, T=10, tol=1e-4, window=10, cap=500, k_mode=1, storage=0,
                    dice_labels=None, timed=False):
    """Plain LDDMM with backtracking from v = 0 until |E_{k-window} - E_k| <= tol E_k or `cap`
    iterations.  I0, I1, M: device float32 (nz, ny, nx).  Returns a dict: v (device, [T][3][...]),
    energies, iterations, wall seconds (context creation included), and the Dice of
    dice_labels = (L0, L1) transferred through the final map when given."""
    nz, ny, nx = I0.shape
    p = L.default_params(nx, ny, nz, T=T, k_mode=k_mode, storage=storage, flags=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with L.Lddmm(p, I0, I1, M) as ctx:
        E = []
        while len(E) < cap:
            E.append(ctx.step()["total"])
            k = len(E) - 1
            if k >= window and abs(E[k - window] - E[k]) <= tol * abs(E[k]):
                break
        ef = ctx.energy()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out = {"energies": E, "iterations": len(E), "final_energy": ef["total"],
               "final_data": ef["data"], "wall_s": wall}
        if not timed:
            v = torch.empty((T, 3, nz, ny, nx), device="cuda")
            ctx.get_velocity(v)
            out["v"] = v
        if dice_labels is not None:
            out["dice"] = ctx.dice(ctx.transfer_labels(dice_labels[0]), dice_labels[1])
    return out


def make_dataset(count, seed0, T=10, amp_max=8.0, log=None):
    """Mask pairs at 64^3 and the converged plain v_0 of each (3 x 64^3, 64-grid voxels).
    Returns (X [S][2][64^3], Y [S][3][64^3]) as device tensors and the iteration counts."""
    from concurrent.futures import ThreadPoolExecutor
    X = torch.empty((count, 2, NG, NG, NG), device="cuda")
    Y = torch.empty((count, 3, NG, NG, NG), device="cuda")
    iters = []
    rng = np.random.default_rng(seed0)
    amps = [float(rng.uniform(0.5 * amp_max, amp_max)) for _ in range(count)]
    gen = lambda i: synth.union_pair((NG, NG, NG), seed=seed0 + i, amplitude=amps[i])
    t0 = time.perf_counter()
    # the host generates pairs on a thread pool while the GPU labels earlier ones
    with ThreadPoolExecutor(8) as ex:
        pending = [ex.submit(gen, i) for i in range(min(count, 32))]
        for i in range(count):
            pr = pending[i].result()
            if i + 32 < count:
                pending.append(ex.submit(gen, i + 32))
            I0, I1, M = _dev(pr.I0), _dev(pr.I1), _dev(pr.M)
            r = converged_plain(I0, I1, M, T=T)
            X[i, 0].copy_(I0)
            X[i, 1].copy_(I1)
            Y[i].copy_(r["v"][0])
            iters.append(r["iterations"])
            pending[i] = None
            if log and (i + 1) % 100 == 0:
                log("labelled %d/%d pairs, %.0f s, mean iterations %.1f" %
                    (i + 1, count, time.perf_counter() - t0, np.mean(iters)))
    return X, Y, iters


def train(X, Y, epochs, lr=1e-3, batch=8, seed=0, log=None):
    """Adam on the MSE between the network's v_0 and the labels (scaled by their RMS)."""
    scale = float(torch.sqrt((Y.double() ** 2).mean()))
    net = SG.UNet3D(chans=CHANS, cin=2, cout=3, n=NG, batch=batch, seed=seed, out_scale=scale)
    Ys = Y / scale
    rng = np.random.default_rng(seed)
    nb = X.shape[0] // batch
    hist = []
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(X.shape[0])).cuda()
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        for bi in range(nb):
            idx = order[bi * batch:(bi + 1) * batch]
            tot += net.train_step(X[idx], Ys[idx], lr)
        mean = float(tot) / (nb * net.y.numel())
        hist.append(mean)
        if log:
            log("epoch %d loss %.4f (%.1f s)" % (ep, mean, time.perf_counter() - t0))
    return net, hist


def _bf16_bits(a):
    """float32 -> bf16 bit patterns (round to nearest even), as uint16."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def save(net, path, meta=None):
    """Weights as the bf16 the products use (uint16 bit patterns; the optimiser's FP32 master copy
    is not kept), biases float32."""
    st = net.state()
    np.savez(path, out_scale=st["out_scale"], chans=np.array(st["chans"]),
             meta=json.dumps(meta or {}),
             **{"w%d" % i: _bf16_bits(w) for i, w in enumerate(st["w"])},
             **{"b%d" % i: b for i, b in enumerate(st["b"])})


def load_net(path, batch=1):
    d = np.load(path)
    chans = tuple(int(c) for c in d["chans"])
    net = SG.UNet3D(chans=chans, cin=2, cout=3, n=NG, batch=batch, seed=0,
                    out_scale=float(d["out_scale"]))
    n = len(net.shapes)

    def w(i):
        a = d["w%d" % i]
        if a.dtype == np.uint16:                 # bf16 bit patterns
            a = (a.astype(np.uint32) << 16).view(np.float32)
        return np.ascontiguousarray(a, np.float32)
    net.load_state({"w": [w(i) for i in range(n)], "b": [d["b%d" % i] for i in range(n)],
                    "out_scale": float(d["out_scale"])})
    return net


def predict_v0(net, I0, I1, out_shape):
    """v_0 on the registration grid (device [3][nz][ny][nx], voxels of that grid) from device
    masks of that grid."""
    nz, ny, nx = out_shape
    x = torch.empty((net.B, 2, NG, NG, NG), device="cuda")
    L.resample(I0, (NG, NG, NG), out=x[0, 0])
    L.resample(I1, (NG, NG, NG), out=x[0, 1])
    if net.B > 1:
        x[1:].copy_(x[:1].expand(net.B - 1, -1, -1, -1, -1))
    y = net.forward(x)[:1]
    v64 = y[0]
    # network units -> 64-grid voxels (out_scale), then -> registration voxels per axis
    s = net.out_scale
    return L.resample(v64, out_shape, ncomp=3, scale=(s * nx / NG, s * ny / NG, s * nz / NG))


def warm_start(ctx, net, I0, I1, scales=SCALES, shoot=False):
    """Set the context's v to the candidate of lowest energy among c x (the smoothed predicted
    v_0 copied to every time step), c in scales (c = 0: the plain start v = 0).  shoot=True
    shoots v_1..v_{T-1} from c v_0 instead (EPDiff); a shot whose energy is not finite is
    dropped.  Returns (chosen c, its energy, energies of all candidates)."""
    T = ctx.params.T
    shape = tuple(I0.shape)
    v0 = predict_v0(net, I0, I1, shape)
    g2 = ctx.params.gamma ** 2
    for c in range(3):                       # gamma^2 K: unit gain at frequency zero
        ctx.apply_K(v0[c], v0[c])
    L.scale_(v0, g2)
    cand = torch.empty((T, 3) + shape, device="cuda")

    def put(c):
        if c == 0.0:
            cand.zero_()
            ctx.set_velocity(cand)
        elif shoot:
            one = v0.clone()
            L.scale_(one, c)
            ctx.shoot(one)
        else:
            cand.copy_(v0.unsqueeze(0).expand(T, -1, -1, -1, -1))
            L.scale_(cand, c)
            ctx.set_velocity(cand)

    res = []
    for c in scales:
        put(c)
        try:
            res.append(ctx.energy()["total"])
        except L.LddmmError as e:          # a start whose energy is not finite is dropped
            if e.code != L.LDDMM_ERR_NONFINITE:
                raise
            res.append(float("inf"))
    best = int(np.argmin(res))
    put(scales[best])
    return scales[best], res[best], res


def run_warm(net, I0, I1, M, target_data, T=10, k_mode=1, storage=0, cap=500, dice_labels=None,
             dice_target=None):
    """Warm start, then plain iterations (backtracking) until the masked-SSD term of the energy
    is <= target_data and, when dice_labels is given, the Dice of the transferred labels >=
    dice_target.  Wall time from context creation to the last check.  Returns a dict."""
    nz, ny, nx = I0.shape
    p = L.default_params(nx, ny, nz, T=T, k_mode=k_mode, storage=storage, flags=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with L.Lddmm(p, I0, I1, M) as ctx:
        c, e, cands = warm_start(ctx, net, I0, I1)
        t_start = time.perf_counter() - t0
        ed = ctx.energy()["data"]
        E, D = [e], [ed]
        it = 0
        dice = None
        while it < cap:
            if D[-1] <= target_data:
                if dice_labels is None:
                    break
                dice = ctx.dice(ctx.transfer_labels(dice_labels[0]), dice_labels[1])
                if dice >= dice_target:
                    break
            r = ctx.step()
            E.append(r["total"])
            D.append(r["data"])
            it += 1
        # the step reports the energy of the field it started from: the last field's own
        if it:
            last = ctx.energy()
            E.append(last["total"])
            D.append(last["data"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dice_labels is not None and dice is None:
            dice = ctx.dice(ctx.transfer_labels(dice_labels[0]), dice_labels[1])
    return {"scale": c, "start_energy": e, "candidates": cands, "iterations": it,
            "energies": E, "data": D, "wall_s": wall, "start_s": t_start, "dice": dice,
            "reached": min(D) <= target_data and (dice_target is None or (dice or 0) >= dice_target)}


WARM_VARIANTS = ((1, 0), (2, 0), (1, 1))     # (k_mode, storage) of the warm runs


def measure(net, T=10, k_mode=1, variants=WARM_VARIANTS, log=None):
    """Time to the plain method's final masked-SSD energy and Dice at 264x160x228 (the brain
    pair, seed 1).  Plain LDDMM (bf16x3 K unless k_mode says otherwise, float storage) runs from
    v = 0 to convergence (the labels' stop rule); its final E_data = sigma^-2 h^3 sum M
    (I0 o phi_10 - I1)^2 and the Dice D of the transferred template mask are the targets.  Each
    warm variant (k_mode, storage) then iterates from the warm start until E_data <= the plain
    value and Dice >= D - 0.005.  Both wall times start at context creation and include the
    network's prediction, the resampling, the smoothing and the scale search."""
    pair, _ = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    I0, I1, M = _dev(pair.I0), _dev(pair.I1), _dev(pair.M)
    lab = ((pair.I0 > 0.5).astype(np.uint16), (pair.I1 > 0.5).astype(np.uint16))
    plain = converged_plain(I0, I1, M, T=T, k_mode=k_mode, cap=2000, dice_labels=lab, timed=True)
    if log:
        log("plain: %d iterations, %.2f s, E %.4g (data %.4g), Dice %.4f" %
            (plain["iterations"], plain["wall_s"], plain["final_energy"], plain["final_data"],
             plain["dice"]))
    out = {"grid": "264x160x228", "T": T, "plain_k_mode": k_mode,
           "plain_iterations": plain["iterations"], "plain_wall_s": round(plain["wall_s"], 3),
           "plain_final_energy": plain["final_energy"], "plain_final_data": plain["final_data"],
           "plain_start_energy": plain["energies"][0], "plain_dice": round(plain["dice"], 5),
           "warm": []}
    for wk, wst in variants:
        warm = run_warm(net, I0, I1, M, plain["final_data"], T=T, k_mode=wk, storage=wst,
                        cap=plain["iterations"], dice_labels=lab, dice_target=plain["dice"] - 0.005)
        if log:
            log("warm k_mode %d storage %d: scale %.3f, start E %.4g, %d iterations, %.3f s "
                "(start %.3f s), E %.4g, E_data %.4g, Dice %.4f, reached %s" %
                (wk, wst, warm["scale"], warm["start_energy"], warm["iterations"],
                 warm["wall_s"], warm["start_s"], warm["energies"][-1], warm["data"][-1],
                 warm["dice"], warm["reached"]))
        out["warm"].append({
            "k_mode": wk, "storage": wst, "scale": warm["scale"],
            "start_energy": warm["start_energy"], "candidates": warm["candidates"],
            "iterations": warm["iterations"], "wall_s": round(warm["wall_s"], 3),
            "start_s": round(warm["start_s"], 3), "final_data": warm["data"][-1],
            "final_energy": warm["energies"][-1], "dice": round(warm["dice"], 5),
            "reached": bool(warm["reached"]),
            "speedup": round(plain["wall_s"] / warm["wall_s"], 2)})
    return out


def measure_shot_start(net, T=10, k_mode=1):
    """Energies of the shot starts (v_1..v_{T-1} by EPDiff from c v_0) at 264x160x228, for the
    record: at this grid the shot field grows from step to step and its energy is not finite
    for most scales."""
    pair, _ = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    I0, I1, M = _dev(pair.I0), _dev(pair.I1), _dev(pair.M)
    p = L.default_params(264, 160, 228, T=T, k_mode=k_mode, flags=1)
    with L.Lddmm(p, I0, I1, M) as ctx:
        c, e, cands = warm_start(ctx, net, I0, I1, scales=(0.0, 0.1, 0.25, 0.5, 1.0), shoot=True)
    return {"shot_scales": [0.0, 0.1, 0.25, 0.5, 1.0], "shot_energies": cands, "chosen": c}


def surrogate_only_dice(net, T=10, k_mode=1):
    """Dice of the template mask transferred by the warm start alone (no plain iteration) at
    264x160x228, against the target mask."""
    pair, _ = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    I0, I1, M = _dev(pair.I0), _dev(pair.I1), _dev(pair.M)
    p = L.default_params(264, 160, 228, T=T, k_mode=k_mode, flags=1)
    with L.Lddmm(p, I0, I1, M) as ctx:
        warm_start(ctx, net, I0, I1, scales=SCALES[1:])
        return ctx.dice(ctx.transfer_labels((pair.I0 > 0.5).astype(np.uint16)),
                        (pair.I1 > 0.5).astype(np.uint16))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "measure"])
    ap.add_argument("--out", default="warm64.npz")
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--val", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args()
    log = lambda m: print(m, flush=True)
    if args.cmd == "train":
        t0 = time.perf_counter()
        X, Y, its = make_dataset(args.pairs, 1000, log=log)
        t_label = time.perf_counter() - t0
        Xv, Yv, _ = make_dataset(args.val, 3000)
        net, hist = train(X, Y, args.epochs, lr=args.lr, log=log)
        t_train = time.perf_counter() - t0 - t_label
        # held-out error of the predicted v_0 against the converged labels
        rels = []
        for i in range(args.val):
            pred = predict_v0(net, Xv[i, 0], Xv[i, 1], (NG, NG, NG))
            rels.append(float((pred - Yv[i]).norm() / Yv[i].norm()))
        meta = {"pairs": args.pairs, "epochs": args.epochs, "lr": args.lr,
                "label_iterations_mean": float(np.mean(its)), "label_s": round(t_label, 1),
                "train_s": round(t_train, 1), "loss": hist, "val_rel_l2_mean": float(np.mean(rels)),
                "val_rel_l2_median": float(np.median(rels))}
        log(json.dumps(meta))
        save(net, args.out, meta)
    else:
        net = load_net(args.weights)
        res = measure(net, log=log)
        res["surrogate_only_dice"] = surrogate_only_dice(net)
        log(json.dumps(res))
        log(json.dumps(measure_shot_start(net)))


if __name__ == "__main__":
    main()
