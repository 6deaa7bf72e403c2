"""Host-side logic of bench.py (no GPU): the algorithmic bytes and flops behind the roofline, the
choice of the roofline's bound, the clock sampler's reading of nvidia-smi rows, and the rule
that a committed DRAM-traffic capture is reported only for the kernel sources it was taken on."""
import json
import os

import pytest

import bench


N = 1000
DIMS = (10, 20, 5)          # X, Y, Z


@pytest.mark.parametrize("kernel,per_voxel", [("flow_back_disp", 36), ("flow_back_terms", 28),
                                              ("fwd_fused", 60), ("fwd_J0T_Edata", 28)])
def test_flow_kernels_count_their_fields_once(kernel, per_voxel):
    a = bench.algorithmic(kernel, N, DIMS, 1)
    assert a == {"bound": "hbm", "bytes": per_voxel * N}


def test_ereg_reads_every_velocity_field_once():
    a = bench.algorithmic("ereg", N, DIMS, 1, T=7)
    assert a == {"bound": "hbm", "bytes": 12 * 7 * N}


@pytest.mark.parametrize("kernel,L,products,nbytes", [("K_x_fwd", 10, 1, 24), ("K_y_inv", 20, 1, 24),
                                                      ("K_z_fused", 5, 2, 24),
                                                      ("K_x_inv_update", 10, 1, 36)])
def test_dft_pass_flops_and_bytes(kernel, L, products, nbytes):
    # one DFT pass over 3 components: 2 L flops per output value; bf16x3 runs three products
    # per product on the tensor cores, plain bf16 one
    a = bench.algorithmic(kernel, N, DIMS, 1)
    assert a["bound"] == "tensor"
    assert a["flops"] == 2.0 * L * 3 * N * products
    assert a["hw_flops"] == 3 * a["flops"]
    assert a["bytes"] == nbytes * N
    b = bench.algorithmic(kernel, N, DIMS, 2)
    assert b["hw_flops"] == b["flops"]
    c = bench.algorithmic(kernel, N, DIMS, 0)
    assert c["bound"] == "alu" and c["flops"] == a["flops"]


def test_roofline_bound_follows_the_slower_resource():
    # a fast tensor pipe makes the pass HBM-bound, a slow one tensor-bound
    fast = {"hbm_gbs": 1.0, "bf16_tflops_sustained": 1e9}
    slow = {"hbm_gbs": 1e9, "bf16_tflops_sustained": 1e-9}
    assert bench.algorithmic("K_x_fwd", N, DIMS, 1, peaks=fast)["bound"] == "hbm"
    assert bench.algorithmic("K_x_fwd", N, DIMS, 1, peaks=slow)["bound"] == "tensor"


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampled(rows):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.out.write("\n".join(rows) + "\n")
    return s.stop()


def test_clock_sampler_median_and_reasons():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1001.3, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    r = _sampled(rows)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}


def test_clock_sampler_reports_thermal_slowdown():
    rows = ["0, 1500, 2070, 700.0, 0x40, Not Active, Active, Not Active, Not Active"]
    assert _sampled(rows)["reasons"] == ["hw_thermal_slowdown"]


def test_clock_sampler_without_samples_reports_nothing():
    assert _sampled(["not a row"]) is None


def test_traffic_reported_only_for_the_sources_it_was_taken_on(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")
    with open(path) as f:
        d = json.load(f)
    kernel, entry = next(iter(d["kernels"].items()))
    monkeypatch.setattr(bench, "_csrc_hash", lambda: d["csrc_hash"])
    assert bench._traffic(kernel) == entry["dram_bytes_per_launch"]
    assert bench._traffic("no_such_kernel") is None
    monkeypatch.setattr(bench, "_csrc_hash", lambda: "0" * 16)
    assert bench._traffic(kernel) is None


def test_committed_traffic_capture_covers_the_hot_kernels():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    for k in ("flow_back_disp", "flow_back_terms", "fwd_fused", "fwd_J0T_Edata", "ereg",
              "K_x_fwd", "K_y_fwd", "K_z_fused", "K_y_inv", "K_x_inv_update"):
        e = d["kernels"][k]
        assert e["read"] > 0 and abs(e["dram_bytes_per_launch"] - e["read"] - e["write"]) <= 1
