"""Benchmark: masked-LDDMM gradient-descent iterations per second at 264x160x228, T = 10.

One step = one full iteration of the hot path on one GPU: backward flow sweep, forward flow
sweep with the masked residual, K = (gamma - alpha Lap)^-2 per time step, the update and the
FP64 energy reductions (all T = 10 time steps).  Inputs: the brain-shaped synthetic atlas/target
mask pair at 264x160x228 (seeded), resident in HBM before the timed region; the working set
(~3 GB: v, per-time-step J1/W, maps, spectra) is far larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): N independent replicas, one per GPU (registrations do not exchange data);
value = iterations of all ranks / max-over-ranks time.  --impl reference times the FP64 CPU
oracle on all host cores: each step is one full T = 10 iteration on the same brain at
132x80x114 (1/8 of the voxels), and the rate is scaled to 264x160x228 by the voxel count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (228, 160, 264)            # (Z, Y, X): 264 x 160 x 228 voxels, 50 um box
BASE = (114, 80, 132)              # generator scale: the 100 um grid
T = 10
METRIC = "LDDMM iters/s at 264x160x228 T=10"
UNIT = "iter/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1605_02060_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


# Algorithmic bytes (or flops) per voxel for one launch of each kernel (fp32 storage): each
# field the kernel reads or writes counts once per launch, a trilinear gather counts the
# gathered field once (the displacements are small, so the corners hit L1/L2).
def algorithmic(kernel, N, dims, kmode, T=10, peaks=None):
    X, Y, Z = dims
    B = {"flow_back_disp": 36, "flow_back_terms": 28, "fwd_residual": 36,
         "fwd_flow": 36, "update": 36,
         # residual b_j and map of step j + 1 over one read of u_j: u_j, I0, J1_j, W_j, v_j in;
         # b_j (split), u_{j+1} out
         "fwd_fused": 60,
         # J0_T = I0 o phi_{1,0} and E_data: u_T, I0, I1, M in; J0_T out
         "fwd_J0T_Edata": 28}
    if kernel in B:
        return {"bound": "hbm", "bytes": B[kernel] * N}
    if kernel == "ereg":             # all T velocity fields read once: 12 B per voxel and step
        return {"bound": "hbm", "bytes": 12 * T * N}
    L = {"K_x_fwd": X, "K_x_inv_update": X, "K_y_fwd": Y, "K_y_inv": Y, "K_z_symbol": Z,
         "K_z_inv": Z, "K_z_fused": Z}[kernel]
    # one DFT pass over 3 components: field in and out (24 B/voxel; the fused update also reads
    # and writes v: 36 B/voxel); the mathematical product is 2 L flops per output value, which
    # the bf16x3 tensor-core form computes three times (hi*hi + hi*lo + lo*hi); the fused z pass
    # (forward product, symbol, inverse product) moves a pass's bytes and computes two products
    nbytes = (36 if kernel == "K_x_inv_update" else 24) * N
    flops = 2.0 * L * 3 * N * (2 if kernel == "K_z_fused" else 1)
    if kmode == 0:
        return {"bound": "alu", "flops": flops, "bytes": nbytes}
    hw_flops = flops * (3 if kmode == 1 else 1)
    if peaks:
        t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
        t_tc = hw_flops / (peaks["bf16_tflops_sustained"] * 1e12)
        if t_hbm >= t_tc:            # the bytes, not the tensor pipe, set this pass's floor
            return {"bound": "hbm", "bytes": nbytes, "flops": flops}
    return {"bound": "tensor", "flops": flops, "hw_flops": hw_flops, "bytes": nbytes}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [l.strip().split(",") for l in self.out.read().splitlines() if l.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


_INPUTS = {}


def make_inputs_full(seed=1):
    """The brain-shaped pair and the atlas grey image at the benchmark's grid (cached)."""
    from paper_1605_02060_gb300 import synth
    if seed not in _INPUTS:
        _INPUTS[seed] = synth.brain_pair(shape=SHAPE, base_shape=BASE, seed=seed)
    return _INPUTS[seed]


def make_inputs(seed=1):
    return make_inputs_full(seed)[0]


SAMPLE_SHAPE = (114, 80, 132)      # the same brain on the 100 um grid: half of each axis


def _oracle_threads():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_iteration(threads):
    """Seconds of one full iteration (T = 10, all time steps, K by FFT) of the FP64 oracle on the
    brain pair at 132x80x114 (the same brain at the 100 um grid, 1/8 of the benchmark's voxels),
    with its trilinear lookups on `threads` host threads and scipy FFT workers.  The oracle's work
    is linear in the voxel count, so the rate at 264x160x228 is 1 / (8 x seconds)."""
    import numpy as np

    from oracle import lddmm as O
    from paper_1605_02060_gb300 import synth
    if "sample" not in _INPUTS:
        _INPUTS["sample"] = synth.brain_pair(shape=SAMPLE_SHAPE, base_shape=BASE, seed=1)[0]
    pair = _INPUTS["sample"]
    O.set_threads(threads)
    v = np.zeros((T, 3) + SAMPLE_SHAPE)
    t0 = time.perf_counter()
    O.lddmm_step(v, pair.I0, pair.I1, pair.M, O.Params(T=T), workers=threads)
    return time.perf_counter() - t0


def _sample_scale():
    return (SHAPE[0] * SHAPE[1] * SHAPE[2]) / float(SAMPLE_SHAPE[0] * SAMPLE_SHAPE[1] * SAMPLE_SHAPE[2])


def _sample_text(threads):
    return ("one full T=10 iteration per step on the same brain at %dx%dx%d (1/%.0f of the "
            "voxels), rate scaled by the voxel count; NumPy/SciPy FP64, trilinear lookups on %d "
            "threads, scipy.fft workers=%d" % (SAMPLE_SHAPE[2], SAMPLE_SHAPE[1], SAMPLE_SHAPE[0],
                                                _sample_scale(), threads, threads))


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    threads = _oracle_threads()
    secs = []
    for i in range(args.warmup + args.steps):
        dt = oracle_iteration(threads)
        if i >= args.warmup:
            secs.append(dt)
    per_step = sum(secs) / len(secs)
    value = 1.0 / (per_step * _sample_scale())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.kmode, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": _sample_text(threads)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(kmode, ws=1, storage=0):
    Z, Y, X = SHAPE
    N = X * Y * Z
    kname = {0: "fp32", 1: "bf16x3", 2: "bf16"}[kmode]
    fields = "fp32 fields" if storage == 0 else "bf16 velocity and images"
    return {"workload": "masked LDDMM %dx%dx%d T=10, brain-shaped atlas/target mask pair (seed 1), "
                        "%s, K via %s DFT products" % (X, Y, Z, fields, kname),
            "grid": [X, Y, Z], "T": T, "alpha": 0.02, "gamma": 1.0, "sigma": 0.1,
            "epsilon": 1e-3, "k_mode": kname, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "working set %.1f GB > L2 (no flush)" % ((2 * T * 3 + 2 * T + 20) * N * 4 / 1e9)}


def run_ours(args):
    import numpy as np
    import torch

    from paper_1605_02060_gb300 import lddmm as L
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    L.load()
    pair = make_inputs()
    Z, Y, X = SHAPE
    N = X * Y * Z
    dev = torch.device("cuda", local)
    I0 = torch.from_numpy(pair.I0).to(dev)
    I1 = torch.from_numpy(pair.I1).to(dev)
    M = torch.from_numpy(pair.M).to(dev)
    stream = torch.cuda.Stream(device=dev)
    p = L.default_params(X, Y, Z, T=T, k_mode=args.kmode, storage=args.storage)
    ctx = L.Lddmm(p, I0, I1, M, stream=stream)
    # warm-up
    for _ in range(args.warmup):
        ctx.step(want_energy=False)
    torch.cuda.synchronize()
    # timed region: K steps with no instrumentation between the kernels (an event pair around
    # every launch adds about 5% to the step)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.step(want_energy=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ws, ms)
    # per-kernel launch times (the kernel table and the roofline): the same K steps again, with
    # a CUDA-event pair around every launch on the context's stream
    launches_per_step = T * 11 + 8
    ctx.profile_start(launches_per_step * args.steps + 64)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.step(want_energy=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_prof = ev0.elapsed_time(ev1)
    prof = ctx.profile_stop()
    value = ws * args.steps / (ms_max / 1000.0)
    e_last = ctx.energy()
    extras = None
    if ws == 1 and not args.no_extras:
        extras = measure_extras(L, I0, I1, M, stream, dev)
        if not args.no_warm_start:
            extras["warm_start"] = measure_warm_start()
    # end to end through the public API with host buffers: every step copies the images in from
    # pinned host memory and reads the energy back
    h0 = torch.from_numpy(pair.I0).pin_memory()
    h1 = torch.from_numpy(pair.I1).pin_memory()
    hm = torch.from_numpy(pair.M).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_images(h0, h1, hm)
        ctx.step(want_energy=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(ws, time.perf_counter() - t0)
    e2e = {"value": ws * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 3 * N * 4,
           "d2h_bytes_per_step": ctypes_sizeof_energy()}
    ctx.close()
    if rank != 0:
        return 0
    # roofline of the dominant kernel
    peaks, src = _peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (nl, tot_ms) = dom
    avg_s = tot_ms / nl / 1000.0
    alg = algorithmic(name, N, (X, Y, Z), args.kmode, T, peaks)
    if args.storage:                 # the table's bytes are those of fp32 storage
        alg = {"bound": "n/a"}
    traffic = _traffic(name) if not args.storage else None
    if alg["bound"] == "hbm":
        achieved = alg["bytes"] / avg_s / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": name,
                "peak_source": src + " (copy bandwidth)",
                "launch_time": LAUNCH_TIME}
    elif alg["bound"] == "tensor":
        achieved = alg["flops"] / avg_s / 1e12
        peak = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": name,
                "peak_source": src + " (bf16 sustained)",
                "launch_time": LAUNCH_TIME,
                # the same launch counted as the tensor cores execute it (the bf16x3 form runs
                # three bf16 products per product) and as HBM bytes
                "hw_flops_per_launch": alg["hw_flops"],
                "hw_frac": alg["hw_flops"] / avg_s / 1e12 / peak,
                "bytes_per_launch": alg["bytes"],
                "bytes_frac": alg["bytes"] / avg_s / 1e9 / peaks["hbm_gbs"]}
    elif alg["bound"] == "n/a":
        roof = {"bound": "n/a", "kernel": name,
                "note": "algorithmic bytes are tabulated for fp32 storage only"}
    else:
        sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12   # FP32 FMA lanes x 2 flop x clock
        achieved = alg["flops"] / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": name,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz,
                "launch_time": LAUNCH_TIME}
    # CPU baseline: the oracle on all host cores, one full T = 10 iteration at 132x80x114
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        threads = _oracle_threads()
        dt = oracle_iteration(threads)
        cpu = {"value": 1.0 / (dt * _sample_scale()), "unit": UNIT, "cores": threads,
               "kind": "oracle", "sample": _sample_text(threads) + "; %.1f s" % dt}
    cfg = workload_config(args.kmode, ws, args.storage)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == 0 else "bf16",
            "data": "synthetic", "config": cfg,
            "clocks": clk, "e2e": e2e, "gpu_launches": int(sum(v[0] for v in prof.values())),
            "profiled_ms_per_step": ms_prof / args.steps,
            "roofline": roof, "cpu_baseline": cpu,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3),
                            "share": round(v[1] / sum(x[1] for x in prof.values()), 4)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "energy_after": e_last["total"], "extras": extras}
    print(json.dumps(line))
    return 0


LAUNCH_TIME = ("mean of CUDA-event pairs around each launch on the launching stream, over a "
               "second run of the same K steps after the timed one")


def _time_steps(L, params, I0, I1, M, stream, warm=2, steps=5):
    import torch
    ctx = L.Lddmm(params, I0, I1, M, stream=stream)
    for _ in range(warm):
        ctx.step(want_energy=False)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ctx.step(want_energy=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    return steps / (e0.elapsed_time(e1) / 1000.0)


def measure_extras(L, I0, I1, M, stream, dev):
    """Secondary measurements reported beside the headline: the same iteration with the other
    precision settings, the exact-gradient (adjoint) evaluation on a 128^3 pair, and the
    surface distances of §2.7 at the benchmark's grid."""
    import numpy as np
    import torch

    from paper_1605_02060_gb300 import synth
    Z, Y, X = SHAPE
    out = {}
    for name, kw in (("bf16_storage_bf16x3_K", dict(k_mode=1, storage=1)),
                     ("fp32_storage_bf16_K", dict(k_mode=2)),
                     ("fp32_storage_fp32_K", dict(k_mode=0))):
        p = L.default_params(X, Y, Z, T=T, **kw)
        out[name + "_iters_per_s"] = round(_time_steps(L, p, I0, I1, M, stream), 2)
    # the paper's integrator: 4 time steps of RK4 along each characteristic (flags bit 2)
    p = L.default_params(X, Y, Z, T=4, k_mode=1, flags=4)
    out["rk4_T4_bf16x3_K_iters_per_s"] = round(_time_steps(L, p, I0, I1, M, stream), 2)
    pair = synth.union_pair((128, 128, 128), seed=100, amplitude=5.0)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    for flags, name in ((0, "adjoint_128cubed_ms"), (2, "adjoint_128cubed_checkpointed_ms")):
        p = L.default_params(128, 128, 128, T=T, flags=flags)
        ctx = L.Lddmm(p, d(pair.I0), d(pair.I1), d(pair.M), stream=stream)
        g = torch.empty((T, 3, 128, 128, 128), device=dev)
        ctx.energy_grad(None, g)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            ctx.energy_grad(None, g)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / 3, 3)
        ctx.close()
    # §2.7 surface measures at the benchmark's grid: the atlas mask after 20 iterations, pulled to
    # target space by its labels, against the target mask (wall time of the C call, host waits)
    p = L.default_params(X, Y, Z, T=T)
    ctx = L.Lddmm(p, I0, I1, M, stream=stream)
    for _ in range(20):
        ctx.step(want_energy=False)
    lab = ctx.transfer_labels((I0 > 0.5).to(torch.int16), torch.empty_like(I0, dtype=torch.int16))
    A = (lab != 0).to(torch.uint8)
    B = (I1 > 0.5).to(torch.uint8)
    A0 = (I0 > 0.5).to(torch.uint8)
    ctx.surface_distance(A0, B)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hd0, md0, _, _ = ctx.surface_distance(A0, B)
    hd, md, na, nb = ctx.surface_distance(A, B)
    dt = (time.perf_counter() - t0) / 2
    # geodesic shooting (EPDiff, transport form) from the v_0 reached after those 20 iterations:
    # T-1 flow steps, transports and K applications (wall time of the C call, host waits)
    vd = torch.empty((T, 3) + tuple(SHAPE), device=dev)
    ctx.get_velocity(vd)
    v0 = vd[0].clone()
    del vd
    ctx.shoot(v0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.shoot(v0)
    torch.cuda.synchronize()
    out["shoot_T10_ms"] = round(1000 * (time.perf_counter() - t0), 2)
    ctx.close()
    # §2.2 preprocessing at the benchmark's grid: target mask from the target intensities
    # (threshold, ball opening r = 1, closing r = 3) and the atlas image histogram-matched to the
    # target (32 bins, 8 points); wall time of the C calls, host waits included
    pair, atlas = make_inputs_full()
    img1 = torch.from_numpy(pair.image1).to(dev)
    img0 = torch.from_numpy(atlas.astype(np.float32)).to(dev)
    L.mask_morphology(img1, 0.025, 1, 3)
    L.histogram_match(img0, I0, img1, I1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.mask_morphology(img1, 0.025, 1, 3)
    t1 = time.perf_counter()
    L.histogram_match(img0, I0, img1, I1)
    t2 = time.perf_counter()
    out["preprocess_ms"] = {"mask_morphology_r1_r3": round(1000 * (t1 - t0), 2),
                            "histogram_match_32_8": round(1000 * (t2 - t1), 2)}
    out["surface_distance"] = {"ms": round(1000 * dt, 2), "surface_voxels": [na, nb],
                               "hausdorff_before": hd0, "median_before": md0,
                               "hausdorff_after_20_iters": hd, "median_after_20_iters": md}
    return out


def measure_warm_start():
    """Time to the plain method's final masked-SSD energy and Dice at 264x160x228 with and without
    the learned warm start (the 64^3 network shipped in the package, trained on 2000 converged
    plain runs): plain LDDMM from v = 0 to convergence, then the warm start until its E_data and
    Dice reach the plain ones, for the bf16x3 K, plain bf16 K and bf16-storage variants.  Wall
    times include context creation, the network's prediction and the scale search."""
    from paper_1605_02060_gb300 import warm64 as W
    if not os.path.exists(W.WEIGHTS):
        return {"unavailable": "no trained network at %s" % os.path.relpath(W.WEIGHTS, ROOT)}
    net = W.load_net(W.WEIGHTS)
    out = W.measure(net)
    out["surrogate_only_dice"] = round(W.surrogate_only_dice(net), 5)
    return out


def ctypes_sizeof_energy():
    import ctypes

    from paper_1605_02060_gb300 import lddmm as L
    return ctypes.sizeof(L.lddmm_energy)


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("csrc_hash") != _csrc_hash():
        return None
    e = d.get("kernels", {}).get(kernel)
    return None if e is None else e.get("dram_bytes_per_launch")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kmode", type=int, default=None, help="0 fp32, 1 bf16x3, 2 bf16")
    ap.add_argument("--storage", type=int, default=0, choices=[0, 1],
                    help="storage of v and the images: 0 fp32 (the metric's), 1 bf16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned warm-start measurement (a few seconds)")
    ap.add_argument("--grid", type=int, nargs=3, default=None, metavar=("X", "Y", "Z"),
                    help="override the 264 160 228 grid (tests only; the metric is quoted on the "
                         "default)")
    args = ap.parse_args()
    global SHAPE, METRIC, SAMPLE_SHAPE
    if args.grid:
        X, Y, Z = args.grid
        SHAPE = (Z, Y, X)
        SAMPLE_SHAPE = tuple((n + 1) // 2 for n in SHAPE)
        METRIC = "LDDMM iters/s at %dx%dx%d T=10" % (X, Y, Z)
    if args.kmode is None:
        args.kmode = DEFAULT_KMODE
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


DEFAULT_KMODE = 1   # tensor-core bf16x3 DFT products (FP32-accurate)

if __name__ == "__main__":
    sys.exit(main())
