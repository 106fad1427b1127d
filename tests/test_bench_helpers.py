"""Host-side helpers of bench.py (no GPU): the nvidia-smi clock summary that decides which
throttle reasons a bench line reports."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _clocks_from(lines):
    c = bench.Clocks(0)
    import tempfile
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    return c.summary()


def test_clock_summary_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _clocks_from(rows)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    rows = [
        "0, 1500, 2070, 1300.0, 0x0000000000000048, Active, Not Active, Active, Not Active",
        "0, [N/A], 2070, 1300.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _clocks_from(rows)
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500.0 and s["samples"] == 2


def test_clock_summary_without_nvidia_smi_output():
    s = _clocks_from([])
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]


def test_host_cpu_reports_core_count_and_model():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["nproc"] >= 1
    assert isinstance(h["machine"], str) and h["machine"]
    assert h["model"] is None or isinstance(h["model"], str)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host) on a small lattice of the
    same recipe: one JSON line with the keys the benchmark contract names."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--dims", "16,16,32", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["higher_is_better"] is True and line["config"]["workload"] == "fiber16x16x32_mixed"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_code_digest_ignores_comments_and_whitespace_only():
    src = "__global__ void k(float* a) {\n    a[0] = 1.0f;  // set\n}\n"
    same = "/* kernel */\n__global__ void k(float* a)\n{ a[0] = 1.0f; }  // other words\n"
    changed = "__global__ void k(float* a) {\n    a[0] = 2.0f;  // set\n}\n"
    assert bench.code_digest([src]) == bench.code_digest([same])
    assert bench.code_digest([src]) != bench.code_digest([changed])


def test_kernel_traffic_scales_with_the_cells_and_names_its_kernel():
    """The committed DRAM bytes per cell of the current kernel code, scaled to a launch's
    cells; unknown kernels have none."""
    per, stale = {}, set()
    for line in open(os.path.join(ROOT, "profiles", "sweep_fp32_traffic.txt")):
        if line.startswith("kernel="):
            kv = dict(x.split("=", 1) for x in line.split())
            if kv["source_sha"] == bench.kernel_source_digest(kv["kernel"]):
                per[kv["kernel"]] = float(kv["dram_bytes_per_cell"])
            else:
                stale.add(kv["kernel"])
    for kernel in stale - set(per):       # taken on other kernel code: reported as null
        assert bench.kernel_traffic(1000, kernel) is None
    for kernel, b in per.items():
        assert bench.kernel_traffic(1000, kernel) == b * 1000
        assert bench.kernel_traffic(2 ** 25, kernel) == b * 2 ** 25
        assert b >= bench.SWEEP_BYTES_PER_CELL - 0.5    # no launch moves less than its inputs
    assert bench.kernel_traffic(1000, "no_such_kernel") is None


def test_oracle_baselines_on_every_core_and_to_steady_state():
    """The CPU baseline's all-core figure runs one spawned process per slab at once and
    adds their cell updates; the serial time to steady state runs the oracle's loop to the
    tolerance."""
    from tests._cases import fiber_case
    case = fiber_case((16, 16, 32))
    rate, workers, sec = bench.oracle_all_cores(case, n_planes=8, sweeps=5)
    assert workers == min(os.cpu_count() or 1, 4) and rate > 0 and sec > 0
    t, n = bench.oracle_time_to_steady(case, 1e-8)
    assert t > 0 and 0 < n < 100000
