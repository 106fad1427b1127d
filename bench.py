"""Benchmark: steady state-of-charge solve on one GB300 (replicas for --gpus N > 1).

Step = one cold-start solve (s = s_in everywhere) to residual 1e-8 of the 256x256x512
fiber lattice (porosity 0.85, d ~ U[6,10] cells, potential flow at 0.5 cm/s,
eta = -0.05 V, s_in = 0.3) in mixed precision: FP32 correction sweeps with FP64 defect
checks. value = lattice cells x sweeps / step time (GCell-updates/s), whole job.

Prints one JSON line. ``--impl reference`` times the CPU oracle instead (explicit FP64
CSR sweeps of the same workload on a bounded sample of it).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCell-updates/s + time-to-steady (res 1e-8) of SOC sweep, % HBM peak, vs FP64"
UNIT = "GCell-updates/s"
# algorithmic bytes per cell of one FP32 correction launch (one sweep or a two-sweep
# pass), global-step kernels of the batched path: delta in + out (8), FP32 forcing r (4),
# three FP32 face velocities (12), one mask bit (1/8)
SWEEP_BYTES_PER_CELL = 4 + 4 + 4 + 12 + 0.125
# local-step kernels (every single-lattice workload): the same with the FP32 step field
# (4) in place of the mask
DT_SWEEP_BYTES_PER_CELL = 4 + 4 + 4 + 12 + 4


def pass_kernel(kname):
    """(sweeps per launch, kernel description) of an FP32 kernel name of the binding."""
    if not kname or kname == "plain":
        return 1, "sweep32d_kernel (one sweep)"
    shape = kname.rsplit("_", 1)[1]
    if kname.startswith("three_sweep"):
        return 3, ("sweep32t3_kernel (three-sweep TMA-staged pass, coefficients of the older "
                   "levels in tensor memory, %s launch, %d delta stages)" % (
                       shape, 5 if kname.startswith("three_sweep5") else 4))
    return 2, ("sweep32tbd_kernel (two-sweep TMA-staged pass, %s launch, %d TMA stages)" % (
        shape, 4 if kname.startswith("blocked4") else 3))
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dims", default="256,256,512")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--workload", default="mixed",
                    choices=["mixed", "batch48", "upsample", "adjoint", "nernst", "logpile"],
                    help="mixed: the 256x256x512 mixed-precision solve (default); batch48: the "
                         "48-lattice batched workload; upsample: 128x128x256 -> 256x256x512 -> "
                         "512x512x1024 iterative upsampling; adjoint: gradients of I_tot, U "
                         "and U_mt on the 128x128x256 differentiation workload; nernst: the "
                         "Nernst model against the SBV FP64 solve on 48x48x96 and 128x128x256; "
                         "logpile: the paper's reference reaction case on its logpile lattice "
                         "at 5, 2.5 and 1.25 um")
    ap.add_argument("--logpile-h", default="10,5,2.5,1.25",
                    help="logpile workload: cell sizes in um (each must divide the box)")
    ap.add_argument("--fp32-kernel", default="auto",
                    choices=["auto", "plain", "blocked", "blocked_persistent", "blocked_chunked",
                             "blocked4_persistent", "blocked4_chunked",
                             "three_sweep_persistent", "three_sweep_chunked",
                             "three_sweep5_persistent", "three_sweep5_chunked"],
                    help="FP32 correction kernel: chosen by the autotuner (default), one sweep "
                         "per launch, or TMA-staged passes (variant autotuned; two-sweep "
                         "passes persistent, or one (tile, z chunk) item per CTA; blocked4: "
                         "four TMA stages; three_sweep: three sweeps a pass with four (or "
                         "five) delta stages)")
    ap.add_argument("--logpile-flow", default="potential", choices=["potential", "stokes"],
                    help="logpile workload: potential flow at the paper's 10 Pa flow rate "
                         "(default) or the Stokes flow at 10 Pa (matrix-free MINRES with a multigrid "
                         "preconditioner)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 comparison, U_mt, e2e and CPU-baseline legs")
    return ap.parse_args()


from paper_2502_08034_gb300.workflows import reduce_over_ranks, upsample_chain  # noqa: E402


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_case(dims, device):
    from paper_2502_08034_gb300 import synth
    return synth.large_mixed_case(dims=dims, flow_device=device)


def peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def code_digest(sources):
    """Digest of C/CUDA source texts with comments and whitespace removed."""
    import re
    h = hashlib.sha256()
    for src in sources:
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def kernel_source_digest(kernel=None):
    """Digest of the kernel sources' code (comments and whitespace removed, so that a
    comment edit does not void the traffic figures taken on the same code); the
    three-sweep pass adds its own header."""
    names = ["soc_kernels.cuh", "sweep_tb.cuh", "sweep_dt.cuh"]
    if kernel and kernel.startswith("three_sweep"):
        names.append("sweep_t3.cuh")
    return code_digest(open(os.path.join(ROOT, "paper_2502_08034_gb300", "csrc", name)).read()
                       for name in names)


def kernel_traffic(n_cells, kernel):
    """DRAM bytes per launch of the sweep kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "sweep_fp32_traffic.txt")
    if not os.path.exists(p):
        return None
    digest = kernel_source_digest(kernel)
    for line in open(p):
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if (parts.get("source_sha") == digest and parts.get("kernel") == kernel
                and "dram_bytes_per_cell" in parts):
            return float(parts["dram_bytes_per_cell"]) * n_cells
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def host_cpu():
    """The host the oracle baseline ran on: logical CPUs and the CPU model (from
    /proc/cpuinfo: "model name" on x86, implementer / part codes on Arm)."""
    info = {"nproc": os.cpu_count(), "machine": os.uname().machine, "model": None}
    try:
        fields = {}
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
        if fields.get("model name"):
            info["model"] = fields["model name"]
        elif fields.get("CPU part"):
            info["model"] = "implementer %s part %s" % (fields.get("CPU implementer"),
                                                       fields["CPU part"])
    except OSError:
        pass
    return info


def oracle_sample(case, n_planes=16, sweeps=40, repeats=1):
    """Time the CPU oracle's explicit FP64 sweeps (Algorithm 7 style, scipy CSR matvec,
    one core) on the first ``n_planes`` z-planes of the workload."""
    import numpy as np

    from oracle import soc
    nz = n_planes
    p = soc.Problem(np.ascontiguousarray(case.solid[:nz]), case.U[:nz], case.V[:nz],
                    case.W[:nz + 1], case.h, case.D, case.s_in, k0=case.k0, eta=case.eta)
    op = soc.assemble(p)
    s0 = soc.initial_state(op, case.s_in)
    n = case.dims[0] * case.dims[1] * nz
    best = float("inf")
    for _ in range(repeats):
        t0 = time.perf_counter()
        soc.explicit_iterate(op, 0.4, 0.0, s0=s0, max_steps=sweeps, check_every=sweeps + 1,
                             local_dt=True)
        best = min(best, time.perf_counter() - t0)
    return n * sweeps / best / 1e9, best, n, sweeps


_SLAB_BARRIER = None


def _slab_init(barrier):
    global _SLAB_BARRIER
    _SLAB_BARRIER = barrier


def _oracle_slab(task):
    """One worker of the all-core oracle figure: assemble the oracle operator of a slab of
    z-planes, wait for every worker, then time its explicit FP64 sweeps."""
    import numpy as np

    from oracle import soc
    solid, U, V, W, h, D, s_in, k0, eta, sweeps = task
    p = soc.Problem(np.ascontiguousarray(solid), U, V, W, h, D, s_in, k0=k0, eta=eta)
    op = soc.assemble(p)
    s0 = soc.initial_state(op, s_in)
    _SLAB_BARRIER.wait()
    t0 = time.perf_counter()
    soc.explicit_iterate(op, 0.4, 0.0, s0=s0, max_steps=sweeps, check_every=sweeps + 1,
                         local_dt=True)
    return solid.size * sweeps, time.perf_counter() - t0


def oracle_all_cores(case, n_planes=16, sweeps=20):
    """The oracle on every host core: one process per core (spawned, not forked), each
    sweeping its own slab of ``n_planes`` z-planes of the workload at the same time.
    Returns (cell-updates/s over all workers, workers, seconds of the slowest)."""
    import multiprocessing as mp
    workers = max(1, min(os.cpu_count() or 1, case.dims[2] // n_planes))
    tasks = []
    for q in range(workers):
        a, b = q * n_planes, (q + 1) * n_planes
        tasks.append((case.solid[a:b].copy(), case.U[a:b].copy(), case.V[a:b].copy(),
                      case.W[a:b + 1].copy(), case.h, case.D, case.s_in, case.k0, case.eta,
                      sweeps))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    with ctx.Pool(workers, initializer=_slab_init, initargs=(barrier,)) as pool:
        res = pool.map(_oracle_slab, tasks)
    slowest = max(t for _, t in res)
    return sum(n for n, _ in res) / slowest / 1e9, workers, slowest


def oracle_time_to_steady(case, tol):
    """Serial wall time of the oracle's Algorithm 7 loop (local steps, FP64 CSR, one
    core) from the cold start s = s_in to tau RMS(RHS) < tol, with its sweep count."""
    import numpy as np

    from oracle import soc
    p = soc.Problem(np.ascontiguousarray(case.solid), case.U, case.V, case.W, case.h, case.D,
                    case.s_in, k0=case.k0, eta=case.eta)
    op = soc.assemble(p)
    t0 = time.perf_counter()
    _, n = soc.explicit_iterate(op, 0.4, tol, s0=soc.initial_state(op, case.s_in),
                                check_every=50, local_dt=True)
    return time.perf_counter() - t0, n


def run_reference(args, dims):
    rank, world, local = dist_env()
    if rank != 0:
        return
    t0 = time.time()
    case = make_case(dims, "cuda" if _cuda() else "cpu")
    setup_s = time.time() - t0
    import numpy as np  # noqa: F401
    for _ in range(args.warmup):
        oracle_sample(case, sweeps=5)
    times, rates = [], []
    n = sweeps = 0
    for _ in range(args.steps):
        rate, sec, n, sweeps = oracle_sample(case, sweeps=20)
        times.append(sec)
        rates.append(rate)
    total = sum(times)
    value = n * sweeps * len(times) / total / 1e9
    sample = ("explicit FP64 CSR sweeps (scipy, 1 thread) of the first 16 z-planes "
              "(%dx%dx16 = %d cells) of the workload, %d sweeps per step" %
              (dims[0], dims[1], n, sweeps))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "fiber%dx%dx%d_mixed" % dims, "dims": list(dims),
                      "porosity": round(case.porosity, 4), "fiber_d": "U[6,10] cells",
                      "u_mean_m_s": case.u_mean, "eta_V": case.eta, "s_in": case.s_in,
                      "tol": args.tol, "sample": "16 z-planes"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample, "host": host_cpu()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "setup_s": setup_s}
    print(json.dumps(out), flush=True)


def _cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def run_batch(args):
    """48 lattices (64^3 .. 192x192x384) in one batched solve per step."""
    import torch

    from paper_2502_08034_gb300 import _build, rfb, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    t0 = time.time()
    cases = synth.batch_cases(48, flow_device="cuda:%d" % local, tol=args.tol)
    setup_s = time.time() - t0
    solvers = [rfb.Solver.from_case(c, device_inputs=True) for c in cases]
    stream = torch.cuda.Stream()
    batch = rfb.Batch(solvers)
    batch.set_stream(stream)
    args_ = ([c.s_in for c in cases], [c.eta for c in cases], [args.tol] * len(cases))

    def step():
        for s in solvers:
            s.reset_state()
        return batch.solve(*args_)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    outs = []
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            outs.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1)
    cells = sum(c.n * r["sweeps"] for res, _ in outs for c, r in zip(cases, res))
    n_total = sum(c.n for c in cases)
    info = outs[-1][1]
    peak, peak_kind = peak_hbm()
    # algorithmic bytes per launch: the two-sweep pass moves 28 B a cell for two sweeps,
    # the one-sweep kernel 24.125 B for one; sweep_ms is the autotuner's time per sweep
    passes = info["pass_stages"] > 0
    achieved = (DT_SWEEP_BYTES_PER_CELL / 2 if passes else SWEEP_BYTES_PER_CELL) * n_total / \
        (info["sweep_ms"] / 1e3) / 1e9
    out = {"metric": METRIC, "value": cells / (elapsed / 1e3) / 1e9, "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "batch48", "lattices": len(cases), "cells": n_total,
                      "tol": args.tol, "l2": "inputs larger than L2"},
           "time_to_last_converged_ms": elapsed / args.steps,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": ("batch_tbd_kernel (two-sweep pass over all 48 lattices, "
                                   "%d-column tiles, %d TMA stages)" % (
                                       info["pass_tile_cols"], info["pass_stages"])
                                   if passes else
                                   "batch_sweep_kernel (one sweep of all 48 lattices)"),
                        "note": "per sweep: algorithmic bytes of a launch / launches per sweep",
                        "peak_kind": peak_kind},
           "batch_info": info, "clocks": clk.summary(),
           "sweeps": [r["sweeps"] for r in outs[-1][0]],
           "max_residual": max(r["residual"] for r in outs[-1][0]),
           "setup_s": setup_s}
    print(json.dumps(out), flush=True)
    batch.close()
    for s in solvers:
        s.close()


def run_upsample(args):
    """The largest single-GPU run: the same analytic fibers at 128x128x256 (h = 5 um),
    256x256x512 and 512x512x1024 (h = 1.25 um, d = 8, porosity 0.82), 1 cm/s,
    eta = -0.10 V, s_in = 0.5; each level warm-started from the prolonged coarser one."""
    import torch

    from paper_2502_08034_gb300 import _build, rfb, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    t0 = time.time()
    cases = synth.upsampling_cases(flow_device="cuda:%d" % local)
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()
    solvers = [rfb.Solver.from_case(c, device_inputs=True, stream=stream) for c in cases]
    for _ in range(args.warmup):
        upsample_chain(solvers, cases, args.tol, umt=False)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    runs = []
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            runs.append(upsample_chain(solvers, cases, args.tol, umt=False))
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1)
    levels, _ = runs[-1]
    cells = sum(c.n * r["sweeps"] for res, _ in runs for c, r in zip(cases, res))
    fine = solvers[-1]
    u_mt, ru = fine.umt(args.tol, precision="mixed")
    # cold start of the finest level for comparison
    fine.reset_state()
    cold = fine.solve(cases[-1].s_in, cases[-1].eta, args.tol, precision="mixed")

    # What the warm start saves, level by level: the residual every 200 sweeps of each
    # level's solve from a cold start (s = s_in) and from the prolonged coarser solution,
    # for the 256x256x512 level (prolonged from 128x128x256, whose fibers are 2 cells
    # across) and the 512x512x1024 level (prolonged from 256x256x512, fibers 4 cells across)
    def history(sv, case, warm_from):
        if warm_from is None:
            sv.reset_state()
        else:
            sv.upsample_from(warm_from)
        hist = []
        for _ in range(200):
            r = sv.step(case.s_in, case.eta, 200, precision="mixed")
            hist.append(r["residual"])
            if r["residual"] <= args.tol:
                break
        return hist

    upsample_gain = []
    for q in (1, 2):
        solvers[q - 1].reset_state()
        upsample_chain(solvers[:q], cases[:q], args.tol, umt=False)
        warm = history(solvers[q], cases[q], solvers[q - 1])
        coldh = history(solvers[q], cases[q], None)
        upsample_gain.append({"level": list(cases[q].dims), "from": list(cases[q - 1].dims),
                              "coarse_fiber_cells": 8.0 / 2 ** (2 - (q - 1)),
                              "residual_every_200_sweeps_warm": warm,
                              "residual_every_200_sweeps_cold": coldh,
                              "sweeps_warm": 200 * len(warm), "sweeps_cold": 200 * len(coldh)})
    peak, peak_kind = peak_hbm()
    N = cases[-1].n
    fr = levels[-1]
    kname, _, _ = fine.tuned_fp32_kernel()
    depth, kdesc = pass_kernel(kname)
    launches_fine = (fr["sweeps"] + depth - 1) // depth
    # algorithmic bytes per launch (a pass reads and writes each cell once)
    achieved = DT_SWEEP_BYTES_PER_CELL * N * launches_fine / (fr["sweep_ms"] / 1e3) / 1e9
    effective = DT_SWEEP_BYTES_PER_CELL * N * fr["sweeps"] / (fr["sweep_ms"] / 1e3) / 1e9
    out = {"metric": METRIC, "value": cells / (elapsed / 1e3) / 1e9, "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "upsample_512x512x1024", "levels": [list(c.dims) for c in cases],
                      "porosity_finest": round(cases[-1].porosity, 4), "tol": args.tol},
           "levels": [{"dims": list(c.dims), "sweeps": r["sweeps"], "time_ms": r["time_ms"],
                       "residual": r["residual"]} for c, r in zip(cases, levels)],
           "finest": {"I_tot_A": fr["I_tot"], "U": fr["U"],
                      "mass_balance_rel": fr["mass_balance_rel"], "U_mt": u_mt,
                      "U_mt_sweeps": ru["sweeps"]},
           "cold_start_finest": {"sweeps": cold["sweeps"], "time_ms": cold["time_ms"]},
           "upsample_gain": upsample_gain,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak,
                        "traffic": kernel_traffic(N, kname) if depth > 1 else None,
                        "kernel": "%s on the finest level" % kdesc,
                        "bytes_per_cell_per_launch": DT_SWEEP_BYTES_PER_CELL,
                        "peak_kind": peak_kind},
           "effective_bandwidth": {"value": effective, "unit": "GB/s", "frac": effective / peak,
                                   "note": "28 B per cell per sweep x sweeps/s, finest level"},
           "clocks": clk.summary(), "setup_s": setup_s}
    print(json.dumps(out), flush=True)
    for s in solvers:
        s.close()


def run_nernst(args):
    """Nernst model (FP64) against the SBV FP64 solve of the same problem: the 48x48x96 plain
    workload (d = 8, porosity 0.8, 1 cm/s, eta = -0.10 V, s_in = 0.5) and a 128x128x256
    lattice of the same recipe, each at the workload's k0 = 1e-7 m/s and at the paper's
    7.2e-5 m/s, to residual 1e-10; omega = 1. value: cell-updates/s of the Nernst solves."""
    import dataclasses

    import numpy as np
    import torch

    from paper_2502_08034_gb300 import _build, rfb, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    tol = 1e-10
    stream = torch.cuda.current_stream()
    rows, cells, nernst_ms, sweep_ms, sweeps_n = [], 0.0, 0.0, 0.0, 0
    with Clocks(local) as clk:
        for dims in ((48, 48, 96), (128, 128, 256)):
            base = synth.fiber_channel_case(dims=dims, flow_device="cuda:%d" % local)
            for k0 in (base.k0, 7.2e-5):
                case = dataclasses.replace(base, k0=k0)
                with rfb.Solver.from_case(case, stream=stream) as sv:
                    for _ in range(max(1, args.warmup)):
                        sv.reset_state()
                        sv.solve(case.s_in, case.eta, tol, precision="fp64")
                        sv.reset_state()
                        sv.solve_nernst(case.s_in, case.eta, tol)
                    sv.reset_state()
                    r_sbv = sv.solve(case.s_in, case.eta, tol, precision="fp64")
                    s_sbv = sv.get_state()
                    res = []
                    for _ in range(args.steps):
                        sv.reset_state()
                        res.append(sv.solve_nernst(case.s_in, case.eta, tol))
                    s_n = sv.get_state()
                r_n = res[-1]
                n = case.n
                cells += n * sum(r["sweeps"] for r in res)
                nernst_ms += sum(r["time_ms"] for r in res)
                sweep_ms += sum(r["sweep_ms"] for r in res)
                sweeps_n += n * sum(r["sweeps"] for r in res)
                rows.append({"dims": list(dims), "k0": k0,
                             "sbv": {"sweeps": r_sbv["sweeps"], "time_ms": r_sbv["time_ms"]},
                             "nernst": {"sweeps": r_n["sweeps"], "time_ms": r_n["time_ms"],
                                        "residual": r_n["residual"]},
                             "maxabs_state_difference": float(np.abs(s_n - s_sbv).max()),
                             "I_tot_A": r_n["I_tot"]})
    # FP64-ALU roofline of the Nernst step: ~16 FP64 flops a cell (7 FMAs of the operator,
    # the update) against the nominal 1.25 TFLOP/s FP64 rate of GB300
    achieved = 16.0 * sweeps_n / (sweep_ms / 1e3) / 1e12
    out = {"metric": METRIC, "value": cells / (nernst_ms / 1e3) / 1e9, "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": nernst_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "nernst_48x48x96_128x128x256", "tol": tol, "omega": 1.0},
           "cases": rows,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                        "frac": achieved / 1.25, "traffic": None,
                        "kernel": "nernst_interior_kernel + nernst_elec_kernel (FP64)",
                        "peak_kind": "nominal FP64"},
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_logpile(args):
    """The paper's reference reaction case on its logpile lattice (Sec. IV): 10 Pa flow
    rate, applied reducing voltage 0, k0 = 7.2e-5 m/s, s_in = 1.73e-7, residual 1e-6 (the
    paper's tolerance), with potential flow scaled to the paper's 10 Pa flow rate or
    (--logpile-flow stokes) the Stokes flow at 10 Pa on each lattice. Mixed-precision
    solves at h = 10, 5, 2.5 and 1.25 um (the last is the paper's 1024 x 512 x 128 = 2^26
    cells), with U, I_tot and U_mt beside the paper's U = 0.243 and I = 0.09 mA, and the
    FP64 solve of the finest level for comparison; at 10 and 5 um also the Butler-Volmer
    model with electromigration refined from the SBV state, beside the paper's model
    comparison. value: cell-updates/s of the timed finest-level mixed solves."""
    import numpy as np
    import torch

    from paper_2502_08034_gb300 import _build, rfb, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    tol = 1e-6
    stream = torch.cuda.current_stream()
    levels, t_setup = [], time.time()
    with Clocks(local) as clk:
        for h in sorted((float(x) * 1e-6 for x in args.logpile_h.split(",")), reverse=True):
            case = synth.logpile_case(h, flow_device="cuda:%d" % local, flow=args.logpile_flow)
            with rfb.Solver.from_case(case, stream=stream) as sv:
                finest = h == min(float(x) * 1e-6 for x in args.logpile_h.split(","))
                for _ in range(max(1, args.warmup) if finest else 0):
                    sv.reset_state()
                    sv.solve(case.s_in, case.eta, tol, precision="mixed")
                res = []
                for _ in range(args.steps if finest else 1):
                    sv.reset_state()
                    res.append(sv.solve(case.s_in, case.eta, tol, precision="mixed"))
                s_mixed = sv.get_state() if finest else None
                u_mt, _ = sv.umt(tol, precision="mixed")
                row = {"h_um": h * 1e6, "dims": list(case.dims),
                       "porosity": round(case.porosity, 5),
                       "q_mL_h": case.info["q_m3_s"] * 3.6e9, "sweeps": res[-1]["sweeps"],
                       "time_to_steady_ms": res[-1]["time_ms"], "U": res[-1]["U"],
                       "I_tot_mA": res[-1]["I_tot"] * 1e3, "U_mt": u_mt,
                       "mass_balance_rel": res[-1]["mass_balance_rel"]}
                if h > 4.9e-6:
                    # the Butler-Volmer model with electromigration refined from the SBV
                    # state (Sec. III.C), against the paper's model comparison (Sec. V:
                    # RMS difference of s from SBV 8.61e-4; phi_L mean 0.16 mV, max 0.47 mV)
                    sv.reset_state()
                    sv.solve(case.s_in, case.eta, 1e-10, precision="fp64")
                    s_sbv = sv.get_state()
                    rb = sv.solve_bv(case.s_in, case.eta, 1e-8, start="sbv")
                    g = sv.get_bv_state()
                    fl = case.solid.ravel() == 0
                    s_bv = g["R"][fl] / (g["O"][fl] + g["R"][fl])
                    row["bv"] = {"rms_s_minus_sbv": float(np.sqrt(np.mean((s_bv - s_sbv[fl]) ** 2))),
                                 "phi_mean_mV": rb["phi_mean"] * 1e3,
                                 "phi_min_mV": rb["phi_min"] * 1e3,
                                 "phi_max_mV": rb["phi_max"] * 1e3, "U": rb["U"],
                                 "I_tot_mA": rb["I_tot"] * 1e3, "sweeps": rb["sweeps"],
                                 "potential_solves": rb["cycles"],
                                 "cg_iterations": rb["cg_iterations"],
                                 "time_ms": rb["time_ms"], "residual": rb["residual"]}
                if finest:
                    sv.reset_state()
                    r64 = sv.solve(case.s_in, case.eta, tol, precision="fp64")
                    row["fp64_time_to_steady_ms"] = r64["time_ms"]
                    row["mixed_minus_fp64_maxabs_s"] = float(np.abs(sv.get_state() - s_mixed).max())
                    n_fine, steps_fine = case.n, res
            levels.append(row)
    ms = sum(r["time_ms"] for r in steps_fine)
    cells = n_fine * sum(r["sweeps"] for r in steps_fine)
    out = {"metric": METRIC, "value": cells / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64",
           "data": "synthetic (the paper's logpile geometry, %s flow)" % args.logpile_flow,
           "config": {"workload": "logpile1024x512x128_sbv_10Pa", "tol": tol,
                      "precision": "mixed", "flow": args.logpile_flow,
                      "q_m3_s": (synth.LOGPILE_Q_10PA if args.logpile_flow == "potential"
                                 else "the Stokes flow rate at 10 Pa of each level (q_mL_h)"),
                      "eta_V": 0.0, "k0_m_s": 7.2e-5},
           "paper": {"U": 0.243, "I_tot_mA": 0.09, "time_steps_to_tol": 125000,
                     "bv_rms_s_minus_sbv": 8.61e-4, "bv_phi_mean_mV": 0.16,
                     "bv_phi_max_mV": 0.47},
           "levels": levels,
           "setup_s": time.time() - t_setup, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """Differentiation workload: 128x128x256, porosity 0.8, d = 8, lognormal (sigma 0.3)
    area multipliers on wall cells; step = FP64 solve to 1e-12 + U_mt solve + the three
    adjoint solves (I_tot, U, U_mt) with their gradients."""
    import torch

    from paper_2502_08034_gb300 import _build, rfb, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    t0 = time.time()
    case = synth.adjoint_case(flow_device="cuda:%d" % local)
    m = synth.lognormal_area_mult(case.solid, 0.3, 40)
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()
    sv = rfb.Solver.from_case(case, area_mult=m, device_inputs=True, stream=stream)
    grad = torch.empty(case.n, dtype=torch.float64, device="cuda")

    def step():
        sv.reset_state()
        fwd = sv.solve(case.s_in, case.eta, 1e-12, precision="fp64")
        sv.umt(1e-12, precision="fp64")
        adj = [sv.adjoint(o, 1e-11, out=grad)[2] for o in ("I_tot", "U", "U_mt")]
        return fwd, adj

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    outs = []
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            outs.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1)
    fwd, adj = outs[-1]
    sweeps = fwd["sweeps"] + sum(a["sweeps"] for a in adj)
    # the same adjoints in mixed precision (FP32 transposed correction sweeps, double-float
    # defects, FP64 confirmation): time and gradient difference from the FP64 ones
    mixed = []
    for o in ("I_tot", "U", "U_mt"):
        g64, b64, _ = sv.adjoint(o, 1e-11)
        gmx, bmx, rm = sv.adjoint(o, 1e-11, precision="mixed")
        scale = float(abs(g64).max()) or 1.0
        mixed.append({"objective": o, "sweeps": rm["sweeps"], "time_ms": rm["time_ms"],
                      "relative_residual": rm["residual"],
                      "max_rel_diff_d_area_mult": float(abs(gmx - g64).max()) / scale,
                      "rel_diff_d_beta": abs(bmx - b64) / abs(b64)})
    out = {"metric": METRIC, "value": case.n * sweeps * args.steps / (elapsed / 1e3) / 1e9,
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "adjoint_128x128x256", "tol_forward": 1e-12,
                      "tol_adjoint": 1e-11},
           "forward": {"sweeps": fwd["sweeps"], "time_ms": fwd["time_ms"]},
           "adjoints": [{"objective": o, "sweeps": a["sweeps"], "time_ms": a["time_ms"],
                         "relative_residual": a["residual"]}
                        for o, a in zip(("I_tot", "U", "U_mt"), adj)],
           "adjoints_mixed": mixed,
           "clocks": clk.summary(), "setup_s": setup_s}
    print(json.dumps(out), flush=True)
    sv.close()


def main():
    args = parse()
    dims = tuple(int(x) for x in args.dims.split(","))
    if args.impl == "reference":
        run_reference(args, dims)
        return
    if args.workload == "batch48":
        run_batch(args)
        return
    if args.workload == "upsample":
        run_upsample(args)
        return
    if args.workload == "adjoint":
        run_adjoint(args)
        return
    if args.workload == "nernst":
        run_nernst(args)
        return
    if args.workload == "logpile":
        run_logpile(args)
        return
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2502_08034_gb300 import _build, rfb
    if rank == 0 or world == 1:
        _build.build()
    if dist:
        dist.barrier()
    t0 = time.time()
    case = make_case(dims, "cuda:%d" % local)
    setup_case_s = time.time() - t0
    stream = torch.cuda.current_stream()
    t0 = time.time()
    sv = rfb.Solver.from_case(case, device_inputs=True, stream=stream)
    torch.cuda.synchronize()
    create_s = time.time() - t0
    N = sv.n_cells

    def step(precision="mixed", tol=args.tol):
        sv.reset_state()
        return sv.solve(case.s_in, case.eta, tol, precision=precision,
                        fp32_kernel=args.fp32_kernel)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = sv.kernel_launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    results = []
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            results.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    clocks = clk.summary()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = sv.kernel_launches - launches0
    sweeps = sum(r["sweeps"] for r in results)
    elapsed_ms, units = reduce_over_ranks(dist, elapsed_ms, N * sweeps, device="cuda")
    value = units / (elapsed_ms / 1e3) / 1e9
    sweep_ms = sum(r["sweep_ms"] for r in results)
    peak, peak_kind = peak_hbm()
    # algorithmic bytes per launch: a launch reads each cell's correction, forcing, three
    # face velocities and step once and writes the correction once, whether it applies
    # one sweep or a two-sweep pass
    kname, tuned_plain_ms, tuned_blocked_ms = sv.tuned_fp32_kernel()
    if args.fp32_kernel not in ("auto", "blocked"):
        kname = args.fp32_kernel
    depth, kdesc = pass_kernel(kname)   # one launch per `depth` sweeps
    kernel_launches = (sweeps + depth - 1) // depth
    achieved = DT_SWEEP_BYTES_PER_CELL * N * kernel_launches / (sweep_ms / 1e3) / 1e9
    effective = DT_SWEEP_BYTES_PER_CELL * N * sweeps / (sweep_ms / 1e3) / 1e9
    traffic = kernel_traffic(N, kname)
    # measured DRAM bytes per launch over the launch time: the kernel's % of HBM peak
    launch_s = (sweep_ms / 1e3) / max(1, kernel_launches)
    dram_frac = traffic / launch_s / 1e9 / peak if traffic else None
    last = results[-1]

    extras = {}
    e2e = None
    cpu = None
    if not args.no_extras:
        # FP64 path on the same workload and tolerance ("vs FP64")
        r64 = step("fp64")
        # accuracy of the mixed state against the FP64 one (both at the same tol)
        s64 = sv.get_state()
        r32 = step("mixed")
        s32 = sv.get_state()
        fluid = case.solid.ravel() == 0
        extras["fp64"] = {"time_to_steady_ms": r64["time_ms"], "sweeps": r64["sweeps"],
                          "GCell_updates_per_s": N * r64["sweeps"] / r64["time_ms"] / 1e6,
                          "sweep_kernel_GCell_per_s": N * r64["sweeps"] / r64["sweep_ms"] / 1e6}
        extras["mixed_vs_fp64_speedup"] = r64["time_ms"] / r32["time_ms"]
        # both states are at residual <= tol but stop after different sweep counts (the
        # check schedules differ), so they differ by the iteration's remaining error there
        extras["mixed_minus_fp64_at_tol_maxabs_s"] = float(np.abs(s32[fluid] - s64[fluid]).max())
        # the precision alone: the FP64 path after the mixed solve's number of sweeps
        sv.reset_state()
        sv.step(case.s_in, case.eta, r32["sweeps"], precision="fp64")
        s64n = sv.get_state()
        extras["mixed_minus_fp64_same_sweeps_maxabs_s"] = float(
            np.abs(s32[fluid] - s64n[fluid]).max())
        u, ru = sv.umt(args.tol, precision="mixed")
        extras["U_mt"] = u
        extras["U_mt_time_ms"] = ru["time_ms"]
        extras["U_mt_sweeps"] = ru["sweeps"]
        # end to end through the C ABI with host buffers: create from the host arrays
        # (copied to the device inside the call), solve, read the state back to host
        # memory; the host buffers are pinned, as a user streaming lattices would keep them
        def pinned(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hin = [pinned(a) for a in (case.solid, case.U, case.V, case.W)]
        h2d = sum(a.nbytes for a in hin)
        d2h = N * 8
        host_s = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        e2e_t, e2e_sw = 0.0, 0
        parts = np.zeros(4)
        reps = max(1, min(args.steps, 2))
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sh = rfb.Solver(case.dims, case.h, *hin, case.D, case.k0, case.alpha, case.n_e,
                            case.T, case.c0)
            t1 = time.perf_counter()
            rr = sh.solve(case.s_in, case.eta, args.tol, precision="mixed")
            t2 = time.perf_counter()
            sh.get_state(host_s)
            t3 = time.perf_counter()
            sh.close()
            t4 = time.perf_counter()
            e2e_t += t4 - t0
            e2e_sw += rr["sweeps"]
            parts += np.array([t1 - t0, t2 - t1, t3 - t2, t4 - t3]) * 1e3
        e2e = {"value": world * N * e2e_sw / e2e_t / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h + 8 * 16),
               "ms_per_step": {"create": parts[0] / reps, "solve": parts[1] / reps,
                               "state_to_host": parts[2] / reps, "destroy": parts[3] / reps}}
        if rank == 0 and world == 1:
            from paper_2502_08034_gb300 import synth
            rate, sec, n_s, sw = oracle_sample(case, sweeps=40)
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "explicit FP64 CSR sweeps (scipy, 1 thread) on the first 16 "
                             "z-planes (%d cells) of the workload, %d sweeps, %.1f s" %
                             (n_s, sw, sec), "host": host_cpu()}
            # the same sweeps on every core at once (one slab of 16 planes per process)
            arate, workers, asec = oracle_all_cores(case)
            cpu["all_cores"] = {"value": arate, "unit": UNIT, "cores": workers,
                                "sample": "%d processes, each 20 sweeps of its own 16-plane "
                                          "slab, %.1f s for the slowest" % (workers, asec)}
            # serial time to steady state: measured on the small workloads, extrapolated
            # (serial rate x the sweeps the same local-step iteration needs) on this one
            small = {}
            c1 = synth.fiber_channel_case(flow_device="cuda:%d" % local)
            t1, n1 = oracle_time_to_steady(c1, c1.tol)
            small["fiber48x48x96_tol1e-10"] = {"seconds": t1, "sweeps": n1, "measured": True}
            q0 = synth.batch_instance_params(0)
            c0 = synth.build_case("batch00", q0["dims"], q0["porosity"], 8.0, q0["seed"],
                                  q0["u_mean"], q0["eta"], q0["s_in"], args.tol,
                                  flow_device="cuda:%d" % local)
            t0_, n0 = oracle_time_to_steady(c0, args.tol)
            small["batch_lattice0_64x64x64_tol%g" % args.tol] = {"seconds": t0_, "sweeps": n0,
                                                                 "measured": True}
            small["this_workload"] = {"seconds": N * sweeps / args.steps / (rate * 1e9),
                                      "sweeps": sweeps / args.steps, "measured": False,
                                      "note": "extrapolated: serial rate x sweeps to tol"}
            cpu["time_to_steady_serial"] = small

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
               "data": "synthetic",
               "config": {"workload": "fiber%dx%dx%d_mixed" % dims, "dims": list(dims),
                          "porosity": round(case.porosity, 4), "fiber_d": "U[6,10] cells",
                          "u_mean_m_s": case.u_mean, "eta_V": case.eta, "s_in": case.s_in,
                          "tol": args.tol, "precision": "mixed", "dt_mode": "local",
                          "parallelism": "replicas" if world > 1 else "1 GPU",
                          "l2": "inputs larger than L2 (%.0f MB of fields)" %
                                (N * 28 / 1e6)},
               "time_to_steady_ms": elapsed_ms / args.steps,
               "sweeps_per_step": sweeps / args.steps,
               "residual": last["residual"], "I_tot_A": last["I_tot"], "U": last["U"],
               "mass_balance_rel": last["mass_balance_rel"],
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                            "kernel": kdesc, "sweeps_per_launch": depth,
                            "autotuner_ms_per_sweep": {"plain": tuned_plain_ms,
                                                       "blocked": tuned_blocked_ms},
                            "bytes_per_cell_per_launch": DT_SWEEP_BYTES_PER_CELL,
                            "dram_frac": dram_frac, "nominal_peak_gbs": 7900.0,
                            "peak_kind": peak_kind},
               "effective_bandwidth": {"value": effective, "unit": "GB/s",
                                       "frac": effective / peak,
                                       "note": "28 B per cell per sweep x sweeps/s"},
               "sweep_kernel_ms_per_sweep": sweep_ms / sweeps,
               "check_ms_per_check": (sum(r["check_ms"] for r in results) /
                                      max(1, sum(r["checks"] - 1 for r in results))),
               "fluid_GCell_updates_per_s": value * sv.n_fluid / N,
               "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "gpu_launches": launches,
               "setup_s": {"case": setup_case_s, "create": create_s}}
        out.update(extras)
        print(json.dumps(out), flush=True)
    sv.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
