"""The benchmark's reference arm (the oracle on the host cores) prints one JSON
line with the keys the benchmark contract names; run on the small workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "maxcut_d6_kron_cap16", "--steps", "2", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["higher_is_better"] is False and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "maxcut_d6_kron_cap16"


def test_batch_partition_covers_every_order_of_the_batch():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_11890_gb300 import inputs
    insts = inputs.batch_maxcut(64, 0)
    assert {i["d"] for i in insts} == set(range(6, 12))
    shards = bench.partition_batch([i["d"] for i in insts], 4, 64)
    assert all(len(sh) > 0 for sh in shards)


def test_clock_summary_reads_throttle_reasons_and_median_clock():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "2010", "2070", "1390", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2070", "2070", "950", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.Clocks(0).summary()["reasons"] == ["unsampled"]


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_seed(5, 0) == 5 and bench.replica_seed(5, 3) == 8
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]          # no process group: identity
    assert bench.gather_results({3: (0, 1.0, 4)}, 1) == {3: (0, 1.0, 4)}
    assert set(bench.WORKLOADS) >= {"maxcut_d10_kron_er_cap64", "maxcut_d6_kron_cap16",
                                     "maxcut_batch64_d6to11_cap64"}


def test_dual_residual_bound_proves_the_weighted_workload_uncertifiable_at_cap_64():
    # Kronecker OR Erdos-Renyi graph with weights U[0.5, 1.5], n = 2^10, cap 64:
    # every iterate Z of TT rank <= 65 leaves rel_d above 0.2, three orders of
    # magnitude above eps_d = 2e-4
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_11890_gb300 import inputs
    w = inputs.maxcut_kron_er(10, 0)["weights"]
    lb = bench.dual_residual_lower_bound(w, 64)
    assert lb["rel_d_lower_bound"] > 0.2 and not lb["certifiable"]
    assert lb["bond"] == 5
    # the bound shrinks as the cap grows and vanishes once the cap covers
    # every unfolding rank (at most 4^5 = 1024 at the middle bond)
    assert bench.dual_residual_lower_bound(w, 256)["rel_d_lower_bound"] < lb["rel_d_lower_bound"]
    assert bench.dual_residual_lower_bound(w, 1024)["rel_d_lower_bound"] == 0.0


def test_dual_residual_bound_is_zero_for_low_rank_objectives():
    # unit-weight Kronecker graphs: C has TT rank <= 4, nothing forces a residual
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_11890_gb300 import inputs
    lb = bench.dual_residual_lower_bound(inputs.maxcut_kron(8, 0)["weights"], 16)
    assert lb["rel_d_lower_bound"] < 1e-12 and lb["certifiable"]


def test_roofline_choice_names_the_kernel_with_the_most_device_time():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    peaks = {"bf16_tflops_sustained": 1716.8, "sm_max_mhz": 2070.0}
    zero3 = (0.0, 0.0, 0)
    # FP64: eight times the sampled GEMM time above the local solves' time -> the GEMM kernel, FP64 peak
    r = bench.roofline_choice("fp64", peaks, "measured", contraction=(1e9, 0.5), tc=zero3,
                              local=(4e11, 0.6, 260, 224, 36), gemm64=(1.6e10, 0.2, 4000))
    assert r[0] == "alu" and r[2] == 1.25 and r[5].startswith("gemm_nd_kernel<double>")
    assert abs(r[1] - 1.6e10 / 0.2 / 1e12) < 1e-12
    # FP64 with the local solves leading and most of them on FP32 factors -> the FP32 ALU peak
    r = bench.roofline_choice("fp64", peaks, "measured", contraction=(1e9, 0.5), tc=zero3,
                              local=(4e11, 2.0, 260, 224, 36), gemm64=(1.6e10, 0.2, 4000))
    assert r[5].startswith("dense local solves") and abs(r[2] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    # ... and on FP64 factors -> the FP64 peak
    r = bench.roofline_choice("fp64", peaks, "measured", contraction=(1e9, 0.5), tc=zero3,
                              local=(4e11, 2.0, 260, 10, 0), gemm64=(1.6e10, 0.2, 4000))
    assert r[2] == 1.25
    # TF32: the tensor-core GEMM against half the BF16 sustained peak
    r = bench.roofline_choice("tf32", peaks, "measured", contraction=(1e9, 0.5), tc=(2e12, 0.01, 100),
                              local=(4e11, 0.1, 260, 260, 0), gemm64=zero3)
    assert r[0] == "tensor" and abs(r[2] - 858.4) < 1e-9 and r[5].startswith("tc_gemm_kernel")
    assert abs(r[1] - 200.0) < 1e-9
