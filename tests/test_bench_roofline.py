"""The benchmark's roofline arithmetic (host logic, no GPU).

The per-kernel rooflines of the benchmark line are computed on the host from CUDA-event times the
step reports.  These tests feed `bench.kernel_rooflines` the per-step figures of a 1,022,138-tet
mixed-precision step and check:

* the algorithmic bytes per launch against the per-unit cost model: the assembly's connectivity,
  coordinates, BDF history, each block value once and the right-hand side; the F pass's
  sub-block records, row pointers and seven per-node vector touches; the SpMV's blocks, columns,
  row pointers and two vectors;
* achieved = work / event time, and frac = achieved / peak, for each kernel;
* the dominant kernel, which is the one with the most device time per step;
* the ncu-derived `traffic`.  It is reported only for the launch shape and precision it was
  captured on: the persistent double-float assembly and the staged BF16 F pass.

The clock record of the timed region (nvidia-smi samples) is checked as well: the median SM
clock, the maximum clock and the throttle reasons seen.  Only this process's GPU counts.
"""
import pytest

T, V, NNZB = 1_022_138, 174_868, 2_606_308       # the 1.02M-tet Poiseuille cylinder


def _stats(asm_ms, mode, its, f_ms, spmv_ms, steps=10):
    # Arnoldi steps average `its` over the steps; four SpMV launches timed per step
    lo = int(its)
    n_hi = round((its - lo) * steps)
    out = []
    for k in range(steps):
        out.append({"ms_assembly_kernels": asm_ms, "n_assembly_launches": 1 if mode == 3 else 19,
                    "assembly_mode": mode, "iterations": lo + (1 if k < n_hi else 0),
                    "ms_fpass_median": f_ms, "n_fpass": 4, "ms_spmv": 4 * spmv_ms, "n_spmv": 4})
    return out


@pytest.fixture(scope="module")
def bench():
    import bench as B

    return B


def test_mixed_step_rooflines(bench):
    peaks, _ = bench._peaks()
    hbm = peaks["hbm_gbs"]
    roof, k = bench.kernel_rooflines(_stats(2.0857, 3, 19.8, 0.02022, 0.0363), T, V, NNZB, "mixed")

    # assembly: 16 B connectivity per element; per node 3 x 8 B coordinates and 8 x 8 B of history;
    # 16 values x 8 B per block (FP32 high + low parts); 4 x 8 B of right-hand side per node
    a = k["assembly"]
    assert a["hbm_view"]["algorithmic_bytes"] == 370_945_792
    assert a["bound"] == "alu" and a["peak"] == pytest.approx(2 * 35.96)
    assert a["achieved"] == pytest.approx(2948 * T / 2.0857e-3 / 1e12, rel=1e-4)
    assert a["frac"] == pytest.approx(0.0201, abs=5e-5)
    assert a["hbm_view"]["frac"] == pytest.approx(370_945_792 / 2.0857e-3 / 1e9 / hbm, abs=5e-5)
    assert a["traffic"] == bench.ASM_DD_PERSISTENT_DRAM_BYTES_PER_ELEMENT * T
    assert a["launches_per_step"] == 1

    # staged BF16 F pass: 12 BF16 values per block record (the column rides in its padding), the
    # row pointers, and per node d_old, r, x, diag(F)^-1 read and r, d, x written in FP32 (16 B each)
    f = k["f_pass"]
    assert f["algorithmic_bytes_per_launch"] == 82_836_084
    assert f["achieved"] == pytest.approx(82_836_084 / 0.02022e-3 / 1e9, rel=1e-4)
    assert f["frac"] == pytest.approx(f["achieved"] / hbm, abs=5e-5)
    assert f["launches_per_step"] == pytest.approx(5 * 19.8)      # (6 F steps - 1) per application
    assert f["traffic"] == int(bench.FPASS_BF16_DRAM_BYTES_PER_BLOCK * NNZB)

    # FP32 SpMV: 16 x 4 B values + a 4 B column per block, row pointers, x read and y written
    s = k["spmv"]
    assert s["algorithmic_bytes_per_launch"] == 183_524_196
    assert s["achieved"] == pytest.approx(183_524_196 / 0.0363e-3 / 1e9, rel=1e-4)
    assert s["ms_per_step"] == pytest.approx(0.0363 * 19.8, rel=1e-4)

    # the assembly takes the most device time per step here (2.09 against 2.00 and 0.72 ms)
    assert roof["kernel"] == a["kernel"] and roof["frac"] == a["frac"]
    assert set(roof["dominant_of"]) == {"assembly", "f_pass", "spmv"}
    assert max(roof["dominant_of"].values()) == roof["dominant_of"]["assembly"]


def test_dominant_kernel_follows_the_krylov_count(bench):
    # more Arnoldi steps per time step: the F passes grow, the assembly does not
    roof, k = bench.kernel_rooflines(_stats(2.0857, 3, 27.0, 0.02022, 0.0363), T, V, NNZB, "mixed")
    assert k["f_pass"]["ms_per_step"] > k["assembly"]["ms_per_step"]
    assert roof["kernel"] == k["f_pass"]["kernel"] and roof["bound"] == "hbm"


def test_traffic_only_for_the_captured_shape_and_precision(bench):
    _, k = bench.kernel_rooflines(_stats(2.18, 2, 19.8, 0.02022, 0.0363), T, V, NNZB, "mixed")
    assert k["assembly"]["traffic"] is None                      # chunk colours: not captured
    _, k = bench.kernel_rooflines(_stats(2.0857, 3, 19.8, 0.0233, 0.0363), T, V, NNZB, "mixed", bf16=False)
    assert k["f_pass"]["traffic"] is None                        # plain FP32 F pass: not captured
    # plain FP32 pass: 12 x 4 B values and a 4 B column per block
    assert k["f_pass"]["algorithmic_bytes_per_launch"] == NNZB * 52 + 4 * (V + 1) + V * 16 * 7


def test_fp64_step_rooflines(bench):
    _, k = bench.kernel_rooflines(_stats(9.5, 1, 18.2, 0.06, 0.07), T, V, NNZB, "fp64")
    a = k["assembly"]
    assert a["peak"] == pytest.approx(1.00) and a["traffic"] is None
    assert a["frac"] == pytest.approx(2948 * T / 9.5e-3 / 1e12 / 1.00, abs=5e-5)
    # FP64 F sub-blocks (12 x 8 B + a 4 B column) and FP64 vectors (32 B per node touch)
    assert k["f_pass"]["algorithmic_bytes_per_launch"] == NNZB * 100 + 4 * (V + 1) + V * 32 * 7
    # FP64 SpMV: 16 x 8 B values + a 4 B column per block, row pointers, x and y (32 B per node each)
    assert k["spmv"]["algorithmic_bytes_per_launch"] == NNZB * 132 + 4 * (V + 1) + 2 * 32 * V
    assert k["spmv"]["traffic"] is None


class _FakeSmi:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_from_samples(bench, monkeypatch):
    # nvidia-smi rows: index, clocks.sm, clocks.max.sm, power.draw, active reasons, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    monkeypatch.setenv("LOCAL_RANK", "0")
    c = bench.Clocks()
    c.proc = _FakeSmi()
    c.samples = [
        ["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1980", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2070", "2070", "950.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1", "900", "2070", "300.0", "0x8", "Active", "Not Active", "Not Active", "Not Active"],  # other GPU
    ]
    rec = c.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]           # kept and noted; the other GPU's slowdown is not ours
    c = bench.Clocks()
    c.proc = _FakeSmi()
    c.samples = [["0", "1500", "2070", "1200.0", "0x2", "Not Active", "Active", "Not Active", "Not Active"]]
    assert c.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi(bench):
    assert bench.Clocks().stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_line():
    """`bench.py --impl reference`: the FP64 oracle on the host cores, on a bounded sample of the
    headline workload, prints one JSON line with the main arm's metric, unit, direction and workload
    name, its cpu_baseline record and an end-to-end entry with no host-device bytes."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--cpu-sample-tets", "20000"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "steps/s" and d["higher_is_better"]
    assert d["metric"].startswith("time steps/s at 1M P1 tets")
    assert d["config"] == {"workload": "poiseuille_cylinder_1022138_tets"}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "sample" in cb
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
