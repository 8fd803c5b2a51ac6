#!/usr/bin/env python
"""Benchmark: DOF/s solved to 1e-10 relative residual on one or more GB300s.

Workload (one step = one full solve): periodic unit cube, 16^3 elements, P = 8
(2,985,984 DOFs), nodal f ~ N(0, 1) from seed 2 made compatible (zero integral
mean), weak rhs b = M f, standalone V(1,1) multigrid with N_O = 1 node-layer
overlap, FP64, from u = 0 to ||b - A u|| <= 1e-10 ||b||.  Inputs are resident
in HBM when timing starts; L2 is flushed (256 MiB write) between steps.

Also reported: the same solves through the host-buffer API (e2e); the
standalone MG with the multigrid in double-float (df64); the mixed-precision
solver (FP32 V-cycle inside the outer CG) on the same problem with the outer
iteration in FP64 (mixed), with q = A p in double-float (mixed_df64) and with
the whole outer iteration in double-float (mixed_df64_all); the level
kernels against their rooflines (the FP64 / FP32 pipe at the sampled clock
for the fast diagonalisation, HBM for the residual and the scatter); the
anisotropic 48x8x8, P = 16 box (mixed MG-CG, N_O = 1, 2, 4, and N_O = 4 with
the double-float outer iteration; key "c3"); the 4^3, P = 32 cube with the
smoother's contractions on the tensor cores and on the CUDA cores (key "c4");
a graded 16^3, P = 8 mesh (element widths varying by a factor 4 along every
axis: FP64 MG and mixed MG-CG, with the outer iteration in FP64 and in
double-float; key "graded"); the 512-request serving stream
(N_O = 1 and 4, and N_O = 4 without grouped launches; key "serving"); and the
FP64 CPU oracle timed on the host cores on a bounded sample of the workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mg|reference]
Multi-GPU (N > 1, launched with torch.distributed.run): every rank solves its
own replica of the problem (weak scaling, no collective on the data path).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF/s solved to 1e-10 rel. residual, mixed vs FP64 on GB300; p50/p99 latency"
TC_MODE = {"off": False, "on": True, "auto": "auto"}
WORKLOAD = {
    "workload": "periodic unit cube, 16^3 elements, P=8 (2,985,984 DOFs), nodal f ~ N(0,1) seed 2 with zero mean, "
                "standalone V(1,1) multigrid, N_O=1 node layer, FP64, u0 = 0, tol 1e-10",
    "lengths": [1.0, 1.0, 1.0],
    "elements": [16, 16, 16],
    "P": 8,
    "overlap_layers": 1,
    "penalty": "2 x stability threshold",
    "tol": 1e-10,
    "solver": "MG V(1,1)",
    "seed": 2,
}
# Other configurations (same timing code; `--workload NAME`).  The default
# bench line is WORKLOAD above (cube16_p8).
WORKLOADS = {
    "sines4_p4": dict(workload="periodic unit cube, 4^3 elements, P=4 (8,000 DOFs), manufactured sines "
                        "(f = 12 pi^2 sin 2pi x sin 2pi y sin 2pi z), standalone V(1,1) MG, N_O=1, FP64, tol 1e-10",
               lengths=[1.0, 1.0, 1.0], elements=[4, 4, 4], P=4, overlap_layers=1, rhs="sines", precision="fp64",
               use_cg=False),
    "cube16_p8": dict(WORKLOAD, rhs="gaussian", precision="fp64", use_cg=False),
    "box48x8x8_p16": dict(workload="periodic box [0,48]x[0,1]x[0,1], 48x8x8 elements, P=16 (15,092,736 DOFs), N_O node layers, "
                        "zero-mean Gaussian f (seed 3), FP32 V(1,1) preconditioner inside FP64 inexact PCG, tol 1e-10",
               lengths=[48.0, 1.0, 1.0], elements=[48, 8, 8], P=16, overlap_layers=1, rhs="gaussian", seed=3,
               precision="mixed", use_cg=True),
    "ar48_p16": dict(workload="periodic box [0,48]x[0,24]x[0,1], 8^3 elements (aspect 48:24:1), P=16 (2,515,456 DOFs), "
                            "N_O node layers, zero-mean Gaussian f (seed 3), FP32 V(1,1) in FP64 PCG, tol 1e-10",
                   lengths=[48.0, 24.0, 1.0], elements=[8, 8, 8], P=16, overlap_layers=1, rhs="gaussian", seed=3,
                   precision="mixed", use_cg=True),
    "ar48max_p16": dict(workload="Table 2 robust method at AR = 48: periodic box [0,48]x[0,24]x[0,1], 8^3 elements, "
                             "P=16 (2,515,456 DOFs), delta_O,i = min(0.08 max_j dx_j, dx_i) (N_O = 4, 6, 17 in x, y, z "
                             "on the finest level), variable V-cycle N_s,l = (1,1) x 3^(L-l), zero-mean Gaussian f "
                             "(seed 3), MG-CG, tol 1e-10",
                    lengths=[48.0, 24.0, 1.0], elements=[8, 8, 8], P=16, overlap_layers=1, overlap_mode="max",
                    overlap_frac=0.08, ns_growth=3, rhs="gaussian", seed=3, precision="fp64", use_cg=True),
    "cube4_p32": dict(workload="periodic unit cube, 4^3 elements, P=32 (2,299,968 DOFs), f = 8 random Fourier modes "
                        "(|k|_inf <= 8, seed 4), FP32 V(1,1) preconditioner in FP64 PCG, N_O=1, tol 1e-10",
               lengths=[1.0, 1.0, 1.0], elements=[4, 4, 4], P=32, overlap_layers=1, rhs="fourier", seed=4,
               precision="mixed", use_cg=True),
}
WORKLOADS["serving512"] = dict(workload="serving stream: 512 solve requests, Poisson arrivals at 200/s (seed 5), periodic box "
                                "[0,AR]x[0,1]x[0,1], AR ~ U[1,8], n^3 elements with n in {4,8,16,24,32}, P in {2,4,8,16}, "
                                "N_O=4 (default; --overlap), Gaussian f, FP32 V(1,1) in a PCG whose outer iteration runs in "
                                "double-float (convergence confirmed on the true residual), tol 1e-10, "
                                "admitted by HBM footprint (smallest work first with aging; MG_SERVING_POLICY=fcfs "
                                "for first come first served), "
                                "one context and stream per slot; requests of <= 2^20 DOFs and one order admitted "
                                "together are solved as one batch (MG_SERVING_BATCH=1: groups of one; MG_SERVING_BATCH_DOFS=0: "
                                "no batched path)")
WORKLOADS["serving512_small"] = dict(workload="serving stream of small requests only: 512 solve requests, Poisson arrivals at "
                                     "5000/s (seed 5: the server is saturated), periodic box [0,AR]x[0,1]x[0,1], AR ~ U[1,8], n^3 elements with "
                                     "n in {4,8}, P in {2,4,8} (1,728 to 373,248 DOFs), N_O=4, Gaussian f, FP32 V(1,1) "
                                     "in PCG (outer iteration in double-float), tol 1e-10; the regime where launches, "
                                     "not arithmetic, bound the throughput (MG_SERVING_BATCH_DOFS=0: no batched path)",
                                     sizes=[4, 8], orders=[2, 4, 8], rate=5000.0)
WORKLOADS["batch16_p4"] = dict(workload="16 independent small problems solved together (mg_solve_batch: one launch per "
                                         "sweep for all): periodic boxes [0,AR]x[0,1]x[0,1], AR ~ U[1,8], n^3 elements "
                                         "with n in {4,5,6,7,8} (seed 7), P=4, N_O=1, Gaussian f, FP32 V(1,1) in FP64 "
                                         "PCG (outer A p in double-float), tol 1e-10; compared with the same 16 solves "
                                         "one after another (mg_solve each)",
                                problems=16, P=4, sizes=[4, 5, 6, 7, 8], aspect=[1.0, 8.0], seed=7,
                                overlap_layers=1, precision="mixed", use_cg=True)


def cosine_widths(n, length, amp, phase):
    """Smoothly graded periodic widths: h_i proportional to
    1 + amp cos(2 pi (i + 1/2) / n + phase), scaled to sum to `length`
    (largest / smallest width (1 + amp) / (1 - amp) at most)."""
    h = 1.0 + amp * np.cos(2.0 * np.pi * (np.arange(n) + 0.5) / n + phase)
    return h * (length / h.sum())


WORKLOADS["graded16_p8"] = dict(workload="graded periodic unit cube: 16^3 elements whose widths follow "
                                         "1 + 0.6 cos(2 pi (i + 1/2) / 16 + phase) per axis (phases 0, 2 pi/3, "
                                         "4 pi/3; widths 0.025 to 0.1, ratio 4), P=8 (2,985,984 DOFs), N_O=1, "
                                         "nodal f ~ N(0,1) seed 2, standalone V(1,1) MG, FP64, tol 1e-10; "
                                         "per-line eigenbases (graded kernels)",
                                lengths=[1.0, 1.0, 1.0], elements=[16, 16, 16], P=8, overlap_layers=1,
                                rhs="gaussian", seed=2, precision="fp64", use_cg=False,
                                widths=[cosine_widths(16, 1.0, 0.6, 2.0 * np.pi * d / 3.0).tolist()
                                        for d in range(3)])
FP32_FLOP_PER_CLK_PER_SM = 256    # 128 FP32 FMA lanes per SM
TF32_PER_BF16 = 1.1 / 2.25         # nominal dense tensor rates per GPU

# bounded sample of the workload for the CPU oracle (same P, overlap, tol; smaller mesh)
ORACLE_SAMPLE = {"elements": [6, 6, 6], "P": 8}
FLUSH_BYTES = 256 << 20
FP64_FLOP_PER_CLK_PER_SM = 4      # 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal at 2070 MHz, 152 SMs)
NUM_SMS = 152


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mg", choices=["mg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / mixed / roofline legs")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 48x8x8, P=16 (c3) and serving-stream keys of the default line")
    ap.add_argument("--workload", default="cube16_p8", choices=sorted(WORKLOADS))
    ap.add_argument("--overlap", type=int, default=None, help="override N_O of the workload")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"], help="override the workload's precision")
    ap.add_argument("--cg", action="store_true", help="solve the workload with MG-CG instead of its default solver")
    ap.add_argument("--fdm-operands", default="fp32", choices=["fp32", "bf16", "fp8"],
                    help="mixed runs: the FP32 smoother's contractions with operands rounded to BF16 or to FP8 "
                         "E4M3 with power-of-two scales per line and per factor column (a precision study of "
                         "BF16 / FP8 tensor-core contractions, run on the CUDA cores)")
    ap.add_argument("--fdm-bf16", action="store_true", help="the same as --fdm-operands bf16")
    ap.add_argument("--autotune", action="store_true",
                    help="--workload runs: time each level's kernel variants at setup and keep the fastest "
                         "(mg_opts.autotune)")
    ap.add_argument("--outer-all", action="store_true",
                    help="mixed MG-CG runs: the whole outer iteration (vectors, inner products, updates and "
                         "q = A p) in double-float arithmetic")
    ap.add_argument("--outer-df64", action="store_true",
                    help="mixed runs: outer operator products q = A p in double-float (FP32-pair) arithmetic")
    ap.add_argument("--tensor-cores", default="off", choices=["off", "on", "auto"],
                    help="FP32 smoother contractions in the mixed runs: CUDA cores, tensor cores (tcgen05, "
                         "TF32) where the tiles fit, or per level the faster of the two (timed at setup)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(x, device=None):
    """Max of a float over all ranks of the default process group (identity
    without one); device = the tensor device the backend needs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, dofs_per_rank, steps, max_seconds):
    """Whole-job DOF/s: every rank solves its own replica; the job time is the
    slowest rank's."""
    return world * dofs_per_rank * steps / max_seconds


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.lines = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        self.cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"] + sel

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def measured_traffic(record="fdm_fp64_16x16x16_p8_m11.json"):
    """DRAM bytes per launch of a fine-level smoother from a committed ncu
    capture (profiles/<record>), or None if the kernel source changed since
    it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest() != rec["source_sha256"]:
            return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def profile_shares(s, total_ms):
    """Share of the profiled step time of every kernel group; "other" is the
    rest: launch gaps and the host synchronisations of the stopping test."""
    out = {}
    for kind in s.PROFILE_KINDS:
        ms, _ = s.profile_result(kind)
        out[kind] = round(ms / max(total_ms, 1e-9), 4)
    out["other"] = round(1.0 - sum(out.values()), 4)
    return out


def clock_mhz(clock_info, pk):
    """Median SM clock sampled under load (nvidia-smi), else the peaks file's maximum."""
    v = (clock_info or {}).get("sm_mhz")
    return (float(v), "median SM clock sampled during the timed steps") if v else \
        (float(pk.get("sm_max_mhz", 2070.0)), "maximum SM clock (no clock samples)")


def fdm_executed_ops(md):
    """Arithmetic instructions the even/odd fast diagonalisation executes per
    subdomain of m_x x m_y x m_z: per direction d, m^3 / m_d lines, each
    transformed forward and backward with (h+1)^2 + h^2 multiply-adds and 2h
    additions (h = (m_d - 1) / 2); plus m^3 multiplications by 1/(lam sum)."""
    m3 = md[0] * md[1] * md[2]
    ops = m3
    for m in md:
        h = (m - 1) // 2
        ops += 2 * (m3 // m) * (2 * h + (h + 1) ** 2 + h * h)
    return ops


def fdm_dense_flop(md):
    """Dense-equivalent flops of one subdomain solve (6 dense 1D products and
    the division): 4 (m_x + m_y + m_z) m^3 + m^3 = 12 m^4 + m^3 for a cube."""
    m3 = md[0] * md[1] * md[2]
    return 4 * sum(md) * m3 + m3


def level_widths(s, lev):
    n = 2 ** lev + 1
    return [n + 2 * s.layers(lev, d) for d in range(3)]


def fdm_roofline(s, lev, fp64, clk, clk_basis, pk, traffic=None):
    """Roofline of the smoother's gather + fast diagonalisation on one level,
    from the CUDA-event durations of its profiled launches.  ALU bound: the
    achieved rate counts every executed arithmetic instruction of the method
    as 2 flop (FMA-equivalent) against the pipe's FMA rate at the sampled clock;
    the dense-equivalent rate (the 12 m^4 + m^3 count) is given beside it."""
    ms, cnt = s.profile_result("fdm", lev)
    if not cnt:
        return None
    t = ms / cnt / 1e3
    md = level_widths(s, lev)
    Ne = int(np.prod(s.counts))
    per_clk = FP64_FLOP_PER_CLK_PER_SM if fp64 else FP32_FLOP_PER_CLK_PER_SM
    peak = NUM_SMS * per_clk * clk * 1e6
    graded = getattr(s, "widths", None) is not None
    # graded meshes: whole 1D products (a subdomain line has no reflection
    # symmetry), 2 m^3 m_d multiply-adds per direction and m^3 divisions
    ops = Ne * (sum(2 * int(np.prod(md)) * m for m in md) + int(np.prod(md)) if graded else fdm_executed_ops(md))
    dense = Ne * fdm_dense_flop(md)
    vb = 8 if fp64 else 4
    algo_bytes = vb * (s.num_dofs(lev) + Ne * md[0] * md[1] * md[2])
    m = md[0] if md[0] == md[1] == md[2] else "x".join(str(v) for v in md)
    if not fp64 and s.fdm_tensor_cores(lev) == 1:
        # tcgen05 TF32 contractions: the dense count is what the tensor cores
        # execute (no even/odd split), against the TF32 dense peak
        tpeak = float(pk["bf16_tflops"]) * TF32_PER_BF16 * 1e12
        return {
            "kernel": "k_fdm_tc<%s> (level %d gather + fast diagonalisation on the tensor cores, TF32)" % (m, lev),
            "bound": "tensor", "achieved": dense / t / 1e12, "peak": tpeak / 1e12, "unit": "TFLOP/s",
            "frac": dense / t / tpeak, "traffic": traffic, "flop_per_launch": dense,
            "avg_launch_ms": t * 1e3, "launches_timed": cnt,
            "hbm": {"algorithmic_bytes_per_launch": algo_bytes, "achieved_gbs": algo_bytes / t / 1e9,
                    "frac": algo_bytes / t / 1e9 / float(pk["hbm_gbs"])},
            "peak_basis": "TF32 dense: measured bf16 burst %.1f TFLOP/s x the nominal TF32 / BF16 ratio %.4f "
                          "(1.1 / 2.25 PFLOP/s)" % (float(pk["bf16_tflops"]), TF32_PER_BF16),
        }
    if graded:
        kname = "k_gfdm<%s> (m = %s, per-line eigenbases)" % ("double" if fp64 else "float", m)
    elif fp64:
        kname = "k_fdm_m<double, %s>" % m
    else:
        kname = {0: "k_fdm_c<%s>", 1: "k_fdm_m<float, %s>",
                 2: "k_fdm_xy / k_fdm_z / k_fdm_yx<%s> (split over three kernels)"}.get(
                     s.kernel_variants(lev)["fdm"], "k_fdm_c<%s>") % m
    return {
        "kernel": kname + " (level %d gather + fast diagonalisation)" % lev,
        "bound": "alu", "achieved": 2.0 * ops / t / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
        "frac": 2.0 * ops / t / peak, "traffic": traffic,
        "executed_ops_per_launch": ops, "avg_launch_ms": t * 1e3, "launches_timed": cnt,
        "dense_equivalent": {"flop_per_launch": dense, "achieved_tflops": dense / t / 1e12,
                             "frac_of_peak": dense / t / peak},
        "hbm": {"algorithmic_bytes_per_launch": algo_bytes, "achieved_gbs": algo_bytes / t / 1e9,
                "frac": algo_bytes / t / 1e9 / float(pk["hbm_gbs"])},
        "peak_basis": "%s pipe: %d SMs x %d flop/clk (FMA-equivalent) x %.0f MHz (%s); derived, the peaks file has "
                      "no %s entry" % ("FP64" if fp64 else "FP32", NUM_SMS, per_clk, clk, clk_basis,
                                       "FP64" if fp64 else "FP32"),
    }


def hbm_roofline(s, kind, lev, bytes_per_launch, name, pk):
    """HBM roofline of a streaming kernel group: algorithmic bytes per launch
    over its mean CUDA-event duration, against the measured copy bandwidth."""
    ms, cnt = s.profile_result(kind, lev)
    if not cnt:
        return None
    t = ms / cnt / 1e3
    return {"kernel": name, "bound": "hbm", "achieved": bytes_per_launch / t / 1e9, "peak": float(pk["hbm_gbs"]),
            "unit": "GB/s", "frac": bytes_per_launch / t / 1e9 / float(pk["hbm_gbs"]), "traffic": None,
            "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": t * 1e3, "launches_timed": cnt}


def level_rooflines(s, lev, fp64, clk, clk_basis, pk, traffic=None):
    """Rooflines of the three level kernels of the smoothing step on level lev
    (residual, gather + fast diagonalisation, weighted scatter); the first is
    the dominant one by time."""
    vb = 8 if fp64 else 4
    N = s.num_dofs(lev)
    md = level_widths(s, lev)
    Ne = int(np.prod(s.counts))
    tname = "double" if fp64 else "float"
    out = []
    r = fdm_roofline(s, lev, fp64, clk, clk_basis, pk, traffic)
    if r:
        out.append(r)
    if getattr(s, "widths", None) is not None:
        oname = "k_gsipg<%s, %d>" % (tname, 2 ** lev + 1)
    else:
        oname = "k_sipg_n<double, %d>" % (2 ** lev + 1) if fp64 else "k_sipg_c<%d>" % (2 ** lev + 1)
    r = hbm_roofline(s, "sipg", lev, 3 * vb * N, "%s (level %d residual r = f - A u: reads u, f, writes r)"
                     % (oname, lev), pk)
    if r:
        out.append(r)
    r = hbm_roofline(s, "scatter", lev, vb * (Ne * md[0] * md[1] * md[2] + 2 * N),
                     "k_scatter_e<%s, %d> (level %d weighted scatter: reads the corrections and u, writes u)"
                     % (tname, 2 ** lev + 1, lev), pk)
    if r:
        out.append(r)
    out.sort(key=lambda d: -d["avg_launch_ms"] * d["launches_timed"])
    return out


def profile_levels(s, steps):
    """Device ms per step for every kernel group and level (CUDA events)."""
    out = {}
    for kind in s.PROFILE_KINDS:
        for lev in range(s.L + 1):
            ms, cnt = s.profile_result(kind, lev)
            if cnt:
                out["%s@%d" % (kind, lev)] = round(ms / steps, 4)
    return out


def oracle_sample_solve(seed=2):
    """The FP64 CPU oracle on the bounded sample: returns (DOFs, solve seconds,
    setup seconds, iterations)."""
    from oracle.multigrid import Hierarchy, solve_mg
    from oracle.sipg import Mesh, weak_rhs
    from paper_1612_04796_gb300 import inputs
    counts, P = ORACLE_SAMPLE["elements"], ORACLE_SAMPLE["P"]
    t0 = time.perf_counter()
    mesh = Mesh(WORKLOAD["lengths"], counts)
    H = Hierarchy(mesh, P, n_o=WORKLOAD["overlap_layers"])
    N = H.A.shape[0]
    b = weak_rhs(mesh, P, inputs.gaussian(N, seed))
    t1 = time.perf_counter()
    _, its, _ = solve_mg(H, b, tol=WORKLOAD["tol"])
    t2 = time.perf_counter()
    return N, t2 - t1, t1 - t0, its


def sample_text(N, its):
    c = ORACLE_SAMPLE["elements"]
    return ("FP64 oracle (numpy/scipy, assembled SIPG matrix, direct subdomain solves) solving the same problem "
            "class on %dx%dx%d elements, P=%d (%d DOFs, %d V(1,1) cycles to 1e-10), solve time only"
            % (c[0], c[1], c[2], ORACLE_SAMPLE["P"], N, its))


def compact_line(line):
    """An extra configuration's line without the keys the main line already has."""
    drop = ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "unit")
    out = {k: v for k, v in line.items() if k not in drop}
    out["unit"] = line["unit"]
    return out


def run_reference(args):
    """Reference arm: the CPU oracle, on the host cores, each step one solve of
    the bounded sample.  Rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    times = []
    N = its = 0
    for step in range(args.warmup + args.steps):
        N, t, _, its = oracle_sample_solve()
        if step >= args.warmup:
            times.append(t)
    total = sum(times)
    value = N * len(times) / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, sample=ORACLE_SAMPLE),
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores, "kind": "oracle",
                         "sample": sample_text(N, its)},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_mg(args):
    import torch
    import torch.distributed as dist

    import paper_1612_04796_gb300 as pkg
    from paper_1612_04796_gb300 import inputs

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(x, dev)

    pkg.load_library()
    W = WORKLOAD
    s = pkg.MGSolver(W["lengths"], W["elements"], W["P"], overlap=W["overlap_layers"], device=dev)
    N = s.num_dofs()
    f_nodal = torch.tensor(inputs.gaussian(N, W["seed"]), device=dev)
    b = s.rhs(f_nodal)
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        u.zero_()
        s.solve(b, u, tol=W["tol"])
    barrier()

    def timed_steps(solver, uvec, use_cg=False):
        ms, its_l = [], []
        for step in range(args.steps):
            flush.fill_(step & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            uvec.zero_()
            _, its, _, _ = solver.solve(b, uvec, tol=W["tol"], use_cg=use_cg)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            its_l.append(its)
        return ms, its_l

    clocks = ClockSampler(dev.index)
    clocks.start()
    launches0 = s.kernel_launches()
    barrier()
    step_ms, iters = timed_steps(s, u)
    barrier()
    launches = s.kernel_launches() - launches0
    clock_info = clocks.stop()
    total_s = max_over_ranks(sum(step_ms) / 1e3)
    value = weak_scaling_value(world, N, args.steps, total_s)
    # per-kernel device times: the same steps again with CUDA events around
    # every kernel group (eager launches instead of graph replays)
    s.profile(True)
    prof_ms, _ = timed_steps(s, u)
    s.profile(False)

    # roofline of the dominant kernel: the smoother's fast diagonalisation on the
    # fine level (FP64-pipe bound), with the other level kernels beside it
    pk, pk_kind = peaks()
    clk, clk_basis = clock_mhz(clock_info, pk)
    kern = level_rooflines(s, s.L, True, clk, clk_basis, pk, traffic=measured_traffic())
    roofline = dict(kern[0])
    roofline["traffic_source"] = "profiles/fdm_fp64_16x16x16_p8_m11.md (ncu dram__bytes_read+write of one launch)"
    roofline["other_kernels"] = kern[1:]
    roofline["time_share_of_step"] = profile_shares(s, sum(prof_ms))
    roofline["ms_per_step_by_kernel_level"] = profile_levels(s, args.steps)
    roofline["timing"] = ("kernel durations from CUDA events around each kernel group over %d profiled steps of the "
                          "same workload run right after the timed steps (eager launches: %.3f ms per step)"
                          % (args.steps, sum(prof_ms) / args.steps))

    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(W, dofs=N, iterations=int(statistics.median(iters)),
                       l2="flushed (256 MiB write) between steps", parallelism="replicas" if world > 1 else "1 GPU"),
        "gpu_launches": launches, "clocks": clock_info, "roofline": roofline,
    }

    if not args.no_extras:
        # e2e: the same solves through the host-buffer entry point (pinned memory)
        f_host = b.cpu().pin_memory()
        u_host = torch.zeros(N, dtype=torch.float64).pin_memory()
        s.solve_host(f_host, u_host, tol=W["tol"])
        barrier()
        t0 = time.perf_counter()
        for _ in range(max(3, args.steps // 3)):
            u_host.zero_()
            s.solve_host(f_host, u_host, tol=W["tol"])
        k_e2e = max(3, args.steps // 3)
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        line["e2e"] = {"value": world * N * k_e2e / e2e_s, "unit": "DOF/s", "h2d_bytes_per_step": 2 * N * 8,
                       "d2h_bytes_per_step": N * 8, "steps": k_e2e}

        # mixed precision: FP32 V(1,1) preconditioner inside FP64 inexact PCG, with the outer
        # products q = A p in FP64 ("mixed") and in double-float pairs ("mixed_df64")
        def mixed_leg(outer_df64):
            sm_ = pkg.MGSolver(W["lengths"], W["elements"], W["P"], overlap=W["overlap_layers"], precision="mixed",
                               device=dev, tensor_cores=TC_MODE[args.tensor_cores], outer_df64=outer_df64)
            um = torch.zeros(N, dtype=torch.float64, device=dev)
            for _ in range(args.warmup):
                um.zero_()
                sm_.solve(b, um, tol=W["tol"], use_cg=True)
            barrier()
            ck = ClockSampler(dev.index)
            ck.start()
            mix_ms, its_ml = timed_steps(sm_, um, use_cg=True)
            barrier()
            ck_info = ck.stop()
            sm_.profile(True)
            mix_prof_ms, _ = timed_steps(sm_, um, use_cg=True)
            sm_.profile(False)
            true_rel = float(torch.linalg.norm(s.residual(um, b)) / torch.linalg.norm(b))
            err = float(torch.max(torch.abs(um - u)) / torch.max(torch.abs(u)))
            mix_total = max_over_ranks(sum(mix_ms) / 1e3)
            leg = {"value": world * N * args.steps / mix_total, "unit": "DOF/s",
                   "ms_per_step": sum(mix_ms) / args.steps, "iterations": its_ml[-1],
                   "solver": "MG-CG: FP32 V(1,1) preconditioner, FP64 inexact PCG",
                   "outer_operator": {False: "FP64", True: "double-float (FP32 pairs, ~48-bit)",
                                      "all": "double-float, with the outer vectors, inner products and updates "
                                             "(FP32 pairs, ~48-bit)"}[outer_df64],
                   "fdm_tensor_cores": args.tensor_cores,
                   "fdm_tensor_cores_by_level": [sm_.fdm_tensor_cores(l) for l in range(1, sm_.L + 1)],
                   "true_relres_fp64": true_rel, "max_rel_diff_vs_fp64_solution": err,
                   "time_share_of_step": profile_shares(sm_, sum(mix_prof_ms)),
                   "ms_per_step_by_kernel_level": profile_levels(sm_, args.steps), "clocks": ck_info}
            clk_m, clk_b = clock_mhz(ck_info, pk)
            kern = level_rooflines(sm_, sm_.L, False, clk_m, clk_b, pk)
            leg["roofline"] = dict(kern[0], other_kernels=kern[1:])
            sm_.close()
            return leg

        # the standalone MG of the main line with the multigrid in double-float arithmetic
        sd = pkg.MGSolver(W["lengths"], W["elements"], W["P"], overlap=W["overlap_layers"], precision="df64",
                          device=dev)
        ud = torch.zeros(N, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            ud.zero_()
            sd.solve(b, ud, tol=W["tol"])
        barrier()
        ck = ClockSampler(dev.index)
        ck.start()
        df_ms, its_d = timed_steps(sd, ud, use_cg=False)
        barrier()
        df_clocks = ck.stop()
        sd.profile(True)
        df_prof_ms, _ = timed_steps(sd, ud, use_cg=False)
        sd.profile(False)
        line["df64"] = {"value": world * N * args.steps / max_over_ranks(sum(df_ms) / 1e3), "unit": "DOF/s",
                        "ms_per_step": sum(df_ms) / args.steps, "iterations": its_d[-1],
                        "solver": "MG V(1,1), multigrid in double-float (FP32 pairs, ~48-bit), FP64 residual",
                        "dtype": "f32x2",
                        "true_relres_fp64": float(torch.linalg.norm(s.residual(ud, b)) / torch.linalg.norm(b)),
                        "max_rel_diff_vs_fp64_solution": float(torch.max(torch.abs(ud - u)) / torch.max(torch.abs(u))),
                        "time_share_of_step": profile_shares(sd, sum(df_prof_ms)),
                        "ms_per_step_by_kernel_level": profile_levels(sd, args.steps), "clocks": df_clocks}
        sd.close()

        line["mixed"] = mixed_leg(args.outer_df64)
        if not args.outer_df64:
            line["mixed_df64"] = mixed_leg(True)
        line["mixed_df64_all"] = mixed_leg("all")

    if not args.no_configs and world == 1:
        # the metric's own configurations beside the main line: the anisotropic
        # 48x8x8, P = 16 box (mixed MG-CG, every overlap the configuration
        # lists, outer iteration in FP64 as the configuration states; and N_O = 4
        # with the double-float outer iteration) and the 512-request serving
        # stream (N_O = 1 and 4, and N_O = 4 without grouped launches)
        line["c3"] = {}
        for no in (1, 2, 4):
            line["c3"]["n_o_%d" % no] = compact_line(workload_line("box48x8x8_p16", 3, 2, overlap=no))
        line["c3"]["n_o_4_outer_df64"] = compact_line(workload_line("box48x8x8_p16", 3, 2, overlap=4,
                                                                    outer_df64="all"))
        # the P = 32 cube: the FP32 smoother's contractions on the tensor cores
        # where timing at setup prefers them (TF32 inputs, FP32 accumulation), and
        # on the CUDA cores; outer iteration in double-float
        line["c4"] = {}
        for tcm in ("auto", "off"):
            line["c4"]["tensor_cores_" + tcm] = compact_line(workload_line("cube4_p32", 5, 3, outer_df64="all",
                                                                           tensor_cores=tcm))
        # a graded mesh (element widths varying smoothly by a factor 4 along
        # every axis) of the 16^3, P = 8 size: FP64 MG and mixed MG-CG
        line["graded"] = {"fp64_mg": compact_line(workload_line("graded16_p8", 5, 3)),
                          "mixed_mgcg": compact_line(workload_line("graded16_p8", 5, 3, precision="mixed",
                                                                   cg=True)),
                          "mixed_mgcg_outer_df64": compact_line(workload_line("graded16_p8", 5, 3,
                                                                              precision="mixed", cg=True,
                                                                              outer_df64="all"))}
        line["serving"] = {}
        for no in (1, 4):
            line["serving"]["n_o_%d" % no] = compact_line(serving_line("serving512", no))
        # the same stream with every request solved on its own (no grouped launches)
        line["serving"]["n_o_4_unbatched"] = compact_line(serving_line("serving512", 4, batch_dofs=0))

    if rank == 0 and not args.no_cpu_baseline:
        Ns, ts, _, its_s = oracle_sample_solve()
        line["cpu_baseline"] = {"value": Ns / ts, "unit": "DOF/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": sample_text(Ns, its_s)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def workload_line(name, steps, warmup, overlap=None, precision=None, cg=False, outer_df64=False,
                  tensor_cores="off", fdm_operands="fp32", autotune=False):
    """One configuration: DOF/s of full solves (inputs resident, L2 flushed
    between solves), per-kernel device times and the rooflines of the
    fine-level kernels.  Returns the JSON line as a dict."""
    import torch

    import paper_1612_04796_gb300 as pkg
    from paper_1612_04796_gb300 import inputs

    W = dict(WORKLOADS[name])
    if overlap is not None:
        W["overlap_layers"] = overlap
    if precision is not None:
        W["precision"] = precision
    if cg:
        W["use_cg"] = True
    dev = torch.device("cuda", torch.cuda.current_device())
    pkg.load_library()
    extra = {k: W[k] for k in ("overlap_mode", "overlap_frac", "ns_growth") if k in W}
    extra["autotune"] = autotune
    extra_mixed = dict(extra, tensor_cores=TC_MODE[tensor_cores], outer_df64=outer_df64,
                       fdm_operands=fdm_operands)
    if "widths" in W:
        extra["widths"] = W["widths"]
        extra_mixed = {k: v for k, v in extra_mixed.items() if k not in ("tensor_cores", "fdm_operands")}
        extra_mixed["widths"] = W["widths"]
    s = pkg.MGSolver(W["lengths"], W["elements"], W["P"], overlap=W["overlap_layers"], precision=W["precision"],
                     device=dev, **(extra_mixed if W["precision"] == "mixed" else extra))
    s64 = s if W["precision"] == "fp64" else pkg.MGSolver(W["lengths"], W["elements"], W["P"],
                                                          overlap=W["overlap_layers"], device=dev, **extra)
    N = s.num_dofs()
    x, y, z = (t.cpu().numpy() for t in s.node_coords())
    if W["rhs"] == "sines":
        f = inputs.sines(x, y, z, W["lengths"])[1]
    elif W["rhs"] == "fourier":
        f = inputs.eval_fourier(inputs.fourier_modes(W["seed"]), x, y, z, W["lengths"])
    else:
        f = inputs.gaussian(N, W.get("seed", 2))
    b = s.rhs(torch.tensor(f, device=dev))
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run(k):
        ms, its = [], []
        for step in range(k):
            flush.fill_(step & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u.zero_()
            _, it, _, _ = s.solve(b, u, tol=1e-10, maxit=200, use_cg=W["use_cg"])
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(it)
        return ms, its

    run(warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    l0 = s.kernel_launches()
    ms, its = run(steps)
    launches = s.kernel_launches() - l0
    clock_info = clocks.stop()
    s.profile(True)
    prof_ms, _ = run(steps)
    s.profile(False)
    true_rel = float(torch.linalg.norm(s64.residual(u, b)) / torch.linalg.norm(b))
    W["autotune"] = autotune
    W["kernel_variants_by_level"] = [s.kernel_variants(l) for l in range(1, s.L + 1)]
    if W["precision"] == "mixed":
        W["fdm_tensor_cores"] = tensor_cores
        W["outer_operator"] = {False: "FP64", True: "double-float (FP32 pairs)",
                               "all": "double-float outer iteration (FP32 pairs)"}[outer_df64]
        W["fdm_tensor_cores_by_level"] = [s.fdm_tensor_cores(l) for l in range(1, s.L + 1)]
        W["fdm_operands"] = {"fp32": "FP32", "bf16": "BF16-rounded (FP32 accumulation)",
                             "fp8": "FP8 E4M3-rounded with power-of-two scales per line and per factor "
                                    "column (FP32 accumulation)"}[fdm_operands]
    fp64 = W["precision"] == "fp64"
    pk, _ = peaks()
    clk, clk_basis = clock_mhz(clock_info, pk)
    traffic = measured_traffic("gfdm_fp64_graded16_p8_m11.json") if name == "graded16_p8" and fp64 else None
    kern = level_rooflines(s, s.L, fp64, clk, clk_basis, pk, traffic=traffic)
    for k in kern:
        if traffic is not None and k["kernel"].startswith("k_gfdm"):
            k["traffic_source"] = "profiles/gfdm_fp64_graded16_p8_m11.md (ncu dram__bytes_read+write of one launch)"
    vb = 8 if fp64 else 4
    if "widths" in W:
        W["element_widths"] = {"min": min(min(w) for w in W["widths"]), "max": max(max(w) for w in W["widths"])}
    line = {
        "metric": METRIC, "value": N * steps / (sum(ms) / 1e3), "unit": "DOF/s", "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": sum(ms) / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32 multigrid / f64 outer",
        "data": "synthetic",
        "config": dict({k: v for k, v in W.items() if k != "widths"}, dofs=N,
                       iterations=int(statistics.median(its)), name=name,
                       true_relres=true_rel, l2="flushed (256 MiB write) between steps; fine-level vectors "
                       "%.0f MB each" % (vb * N / 1e6)),
        "gpu_launches": launches, "clocks": clock_info,
        "roofline": dict(kern[0], other_kernels=kern[1:], time_share_of_step=profile_shares(s, sum(prof_ms)),
                         ms_per_step_by_kernel_level=profile_levels(s, steps)),
    }
    if s64 is not s:
        s64.close()
    s.close()
    return line


def run_workload(args):
    """One configuration other than the default line (`--workload NAME`)."""
    line = workload_line(args.workload, args.steps, args.warmup, overlap=args.overlap, precision=args.precision,
                         cg=args.cg, outer_df64="all" if args.outer_all else args.outer_df64,
                         tensor_cores=args.tensor_cores,
                         fdm_operands="bf16" if args.fdm_bf16 else args.fdm_operands, autotune=args.autotune)
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Many small problems: DOF/s of solving all of them with one batched
    call (every sweep one grouped launch) against the same solves made one
    after another on the same stream."""
    import torch

    import paper_1612_04796_gb300 as pkg
    from paper_1612_04796_gb300 import inputs

    W = dict(WORKLOADS[args.workload])
    dev = torch.device("cuda", torch.cuda.current_device())
    pkg.load_library()
    rng = np.random.default_rng(W["seed"])
    probs = []
    for i in range(W["problems"]):
        n = int(rng.choice(W["sizes"]))
        ar = float(rng.uniform(*W["aspect"]))
        s = pkg.MGSolver((ar, 1.0, 1.0), (n, n, n), W["P"], overlap=W["overlap_layers"], precision=W["precision"],
                         device=dev, outer_df64=True)
        b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), W["seed"] * 1000 + i), device=dev))
        probs.append((s, b, torch.zeros(s.num_dofs(), dtype=torch.float64, device=dev)))
    dofs = sum(s.num_dofs() for s, _, _ in probs)
    solvers = [p[0] for p in probs]
    stream = torch.cuda.current_stream(dev)

    def run(batched, k, batch_solvers=None):
        ms, its = [], None
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            for _, _, u in probs:
                u.zero_()
            if batched:
                _, its, _, sts = pkg.solve_batch(batch_solvers or solvers, [b for _, b, _ in probs],
                                                 [u for _, _, u in probs], tol=1e-10, maxit=200)
                assert all(v == 0 for v in sts), sts
            else:
                its = [s.solve(b, u, tol=1e-10, maxit=200, use_cg=True)[1] for s, b, u in probs]
            e1.record(stream)
            e1.synchronize()
            ms.append(max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3))
        return ms, its

    run(True, args.warmup)
    run(False, args.warmup)
    clocks = ClockSampler(dev.index)
    clocks.start()
    lb0 = solvers[0].batch_launches()
    ms_b, its_b = run(True, args.steps)
    launches_b = solvers[0].batch_launches() - lb0
    u_b = [u.clone() for _, _, u in probs]  # the batched solutions
    ls0 = sum(s.kernel_launches() for s in solvers)
    ms_s, its_s = run(False, args.steps)
    launches_s = sum(s.kernel_launches() for s in solvers) - ls0
    clock_info = clocks.stop()
    assert its_b == its_s
    # batched against one by one: the batched kernels are separate compilations
    # of the same code, equal to rounding (bit for bit where the compiler
    # contracted alike)
    identical = all(torch.equal(a, u) for a, (_, _, u) in zip(u_b, probs))
    max_rel_diff = max(float((a - u).abs().max() / u.abs().max()) for a, (_, _, u) in zip(u_b, probs))
    # the same batch with every grouped launch in persistent form (one wave of
    # blocks looping over the problems' blocks; the first context's option
    # decides): a twin of the first problem's context with persistent="always"
    s0 = solvers[0]
    sp = pkg.MGSolver(s0.lengths, s0.counts, W["P"], overlap=W["overlap_layers"], precision=W["precision"],
                      device=dev, outer_df64=True, persistent="always")
    run(True, args.warmup, [sp] + solvers[1:])
    ms_p, its_p = run(True, args.steps, [sp] + solvers[1:])
    identical_p = its_p == its_b and all(torch.equal(a, u) for a, (_, _, u) in zip(u_b, probs))
    sp.close()
    tb, ts = statistics.median(ms_b), statistics.median(ms_s)
    line = {
        "metric": METRIC, "value": dofs / (tb / 1e3), "unit": "DOF/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 multigrid / f64 outer", "data": "synthetic",
        "config": dict(W, name=args.workload, total_dofs=dofs, dofs_each=[s.num_dofs() for s in solvers],
                       iterations=its_b, l2="inputs L2-resident (small problems; the point is launch overhead)"),
        "gpu_launches": launches_b // args.steps,
        "one_by_one": {"value": dofs / (ts / 1e3), "ms_per_step": ts, "gpu_launches": launches_s // args.steps},
        "speedup_vs_one_by_one": ts / tb, "bitwise_identical_to_one_by_one": identical,
        "max_rel_diff_vs_one_by_one": max_rel_diff, "clocks": clock_info,
        "persistent_always": {"value": dofs / (statistics.median(ms_p) / 1e3), "ms_per_step": statistics.median(ms_p),
                              "bitwise_identical_to_batched": identical_p},
    }
    print(json.dumps(line), flush=True)


def serving_line(name, overlap=None, n_req=None, batch_dofs=None):
    """The serving stream: throughput (DOFs solved / makespan) and per-request
    latency (arrival to result on the host) percentiles.  Returns the JSON line
    as a dict."""
    import torch

    from paper_1612_04796_gb300.serving import Server, latency_summary, request_stream
    n_req = int(os.environ.get("MG_SERVING_REQUESTS", "512")) if n_req is None else n_req
    overlap = 4 if overlap is None else overlap
    slots = int(os.environ.get("MG_SERVING_SLOTS", "8"))
    policy = os.environ.get("MG_SERVING_POLICY", "smallest")
    W = WORKLOADS[name]
    reqs = request_stream(seed=5, n_requests=n_req, overlap=overlap, sizes=tuple(W.get("sizes", (4, 8, 16, 24, 32))),
                          orders=tuple(W.get("orders", (2, 4, 8, 16))), rate=W.get("rate", 200.0))
    batch_max = int(os.environ.get("MG_SERVING_BATCH", "16"))
    if batch_dofs is None:
        batch_dofs = int(os.environ.get("MG_SERVING_BATCH_DOFS", str(1 << 20)))
    srv = Server(slots=slots, keep_solution=False, policy=policy, batch_max=batch_max, batch_dofs=batch_dofs)
    # warm-up: small requests of every order (module loading, first captures)
    warm = request_stream(seed=6, n_requests=64, sizes=(4,), overlap=overlap)[:8]
    srv.serve(warm, realtime=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(srv.device.index)
    clocks.start()
    t0 = time.perf_counter()
    res = srv.serve(reqs, realtime=True)
    torch.cuda.synchronize()
    makespan = time.perf_counter() - t0
    clock_info = clocks.stop()
    ok = [r for r, q in zip(res, reqs) if r.error is None]
    dofs = sum(q.dofs for r, q in zip(res, reqs) if r.error is None)
    summ = latency_summary(res)
    line = {
        "metric": METRIC, "value": dofs / makespan, "unit": "DOF/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": makespan * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 multigrid / f64 outer", "data": "synthetic",
        "config": dict(W, name=name, requests=len(reqs), slots=slots, overlap_layers=overlap,
                       hbm_budget_gb=srv.budget / 1e9, total_dofs=dofs,
                       admission=policy + (" (aging after %.0f s)" % srv.max_wait
                                           if policy == "smallest" else ""),
                       outer_operator={False: "FP64", True: "double-float (FP32 pairs)",
                                       "all": "double-float outer iteration (FP32 pairs)"}[srv.outer_df64],
                       batch_max=srv.batch_max, batch_dofs=srv.batch_dofs),
        "latency": summ, "max_concurrent": srv.max_active,
        "batched_requests": int(sum(r.batch > 1 for r in res)),
        "mean_batch": float(np.mean([r.batch for r in res])),
        "failed_requests": len(res) - len(ok),
        "iterations": {"median": float(np.median([r.iterations for r in ok])),
                       "max": int(max(r.iterations for r in ok))},
        "max_relres": float(max(r.relres for r in ok)), "clocks": clock_info,
    }
    srv.close()
    return line


def run_serving(args):
    print(json.dumps(serving_line(args.workload, args.overlap)), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("serving512", "serving512_small"):
        run_serving(args)
    elif args.workload == "batch16_p4":
        run_batch(args)
    elif args.workload != "cube16_p8" or args.precision is not None or args.cg:
        run_workload(args)
    else:
        run_mg(args)


if __name__ == "__main__":
    main()
