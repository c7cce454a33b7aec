#!/usr/bin/env python
"""Benchmark: grid-point x field RK4 updates per second on one spherical shell.

Default workload (the full-RK4 single-shell configuration): 33 x 48 x 96 shell,
r in [1.8, 11], 50 GHG fields, Kerr-Schild Schwarzschild plus a seeded l <= 4
perturbation of amplitude 1e-4, Yn filter (L = 46) on every stage right-hand
side, dt = 0.25 min dx.  A "step" is one full RK4 step: four evaluations of
derivatives + GHG right-hand side + boundary condition + Yn filter, and the
stage updates.  Inputs are synthetic (seeded generator).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Multi-GPU (torchrun): one independent shell per rank
(replicas, weak scaling, no data-path collective); value = all ranks' units
divided by the slowest rank's time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pt·field RK4 updates/s, mixed vs FP64 path on GB300 at ≤1e-10 err vs FP64 oracle"
UNIT = "pt·field/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ks_33x48x96")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the shorter measurements of the 58-field 65x96x192 shell and of the "
                         "256-shell batch that a default run adds to its line")
    ap.add_argument("--filter", default="yn", choices=["yn", "y", "yg"],
                    help="filter of the single-shell workloads: tensor Yn (default), scalar Y, graded Yg")
    ap.add_argument("--sweep", default=None,
                    help="comma list of n: time the Cartesian derivatives of 50 fields on n x n x 2n shells "
                         "by the mixed and FP64 matrix paths and the FFT path, print one JSON line and exit")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one eager RK4 step with per-group device times and print them "
                         "(the fixed launch sequence used for profiler captures)")
    ap.add_argument("--profile-graph", action="store_true",
                    help="run one RK4 step through the captured step graph (as the timed steps run) "
                         "and exit: the launch sequence of the launch-list capture")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist.get_rank(), int(os.environ.get("LOCAL_RANK", "0")), ws, dist


def _max_over_ranks(t_ms, dist):
    """The slowest rank's time (host-side all-reduce over the gloo group)."""
    if not dist:
        return t_ms
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _workload(name):
    from paper_1104_3408_gb300 import inputs
    w = dict(inputs.WORKLOADS[name])
    w["name"] = name
    return w


def _state(w):
    from paper_1104_3408_gb300 import inputs
    return inputs.kerr_schild_state(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"],
                                    n_fields=w.get("n_fields", 50), amp=w["amp"], ell=w["ell"],
                                    seed=w["seed"])


def _peaks():
    """(HBM GB/s, sustained BF16 TFLOP/s, source)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return (p.get("hbm_gbs", 6800.0), p.get("bf16_tflops_sustained", p.get("bf16_tflops", 1700.0)),
                "measured")
    return 6800.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) > 8:
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _time_steps(sh, u, dt, K, flush, torch, use_async=True):
    """K single RK4 steps, L2 flushed (256 MiB write) before each; CUDA events
    on the launching stream around each step.  use_async: the steps go
    through cffyn_rk4_step_async (the host queues every step without waiting,
    so each step's events bracket its device work alone; the status words are
    checked after the last); else through the synchronising cffyn_rk4_step
    (the traced graph, whose trace needs it).  Returns total ms."""
    from paper_1104_3408_gb300 import cffyn
    st = torch.cuda.current_stream()
    status = torch.zeros(K, dtype=torch.int32).pin_memory()
    total = 0.0
    evs = []
    for i in range(K):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        if use_async:
            sh.rk4_step_async(u, status[i:i + 1], dt, 1, st)
        else:
            sh.rk4_step(u, dt, 1)
        b.record(st)
        evs.append((a, b))
    torch.cuda.synchronize()
    cffyn.check_status(status)
    for a, b in evs:
        total += a.elapsed_time(b)
    return total


# Kernel families of the step and the trace phases each one runs in.
FAMILIES = {
    "k_op_tc": ["d_r", "d_theta_phi", "dft_fwd", "project", "dft_inv"],
    "k_reconstruct": ["reconstruct"],
    "k_rhs_gamma": ["rhs_gamma"],
    "k_rhs_quad": ["rhs_quad"],
    "k_rhs_pp": ["rhs_pp"],
    "k_decompose": ["decompose"],
    "k_field_exp": ["field_exp"],
}
# BF16 digit-pair products per operator product: i + j <= 6 of 6 x 6 digits
# for the derivatives, i + j <= 5 for the filter's DFTs and projections
PAIRS = {"d_r": 26, "d_theta_phi": 26, "dft_fwd": 21, "project": 21, "dft_inv": 21}
# FP64 operations of one evaluation of the pointwise right-hand side per point
# (eqs. gdot, Phidot, Pidot with their 3+1 quantities and Christoffel
# symbols), counted on the oracle's own formulation by oracle/flops.py
# (tests/test_oracle_flops.py checks this figure); the chain rule adds
# 15 per pt-field (eq. dvdx).
RHS_OPS_PER_POINT = 6418.0
# FP32 instructions per FP64-equivalent operation of the double-float
# arithmetic of the mixed path's pointwise kernels: an addition is TwoSum
# (6) + 2 + a fast renormalisation (3) = 11, a product is 1 + 1 FMA + 2 + 1
# + 3 = 8; the whole-step bound takes the mean, 9.5.
FF_INSTR_PER_OP = 9.5
# SM count and FP32 lanes per SM of the GB300 (the FP32 pipe's instruction
# peak is SMs x lanes x SM clock).
SMS, FP32_LANES = 152, 128


def _op_flops(w, phase):
    """Method FP64 flops of one operator group over all fields (one stage):
    the per-pt-field figures 2 n_r (d_r), 4N (d_theta, K = 2N) + 4N (d_phi),
    and 8N + 2(L+1) for the filter split as DFT 4N + projection 2(L+1) +
    inverse DFT 4N."""
    n_r, N, J, L, nv = w["n_r"], w["n_theta"], w["n_phi"], w["L"], w["n_fields"]
    per = {"d_r": 2 * n_r, "d_theta_phi": 8 * N, "dft_fwd": 4 * N,
           "project": 2 * (L + 1), "dft_inv": 4 * N}[phase]
    return float(per) * n_r * N * J * nv


def _pointwise_bytes(w, phase):
    """Algorithmic HBM bytes of one launch of a pointwise kernel: the 8-byte
    values it must read and write per point (stage average for the update)."""
    n_r, N, J, L, nv = w["n_r"], w["n_theta"], w["n_phi"], w["L"], w["n_fields"]
    P8 = n_r * N * J * 8.0
    vals = {"rhs_gamma": 96, "rhs_quad": 100, "rhs_pp": 240, "decompose": 2 * nv,
            "reconstruct": 4.5 * nv,
            "field_exp": nv}[phase]
    return vals * P8


def _op_sources_sha():
    """sha256 of the sources that define the operator kernel k_op_tc."""
    import hashlib
    h = hashlib.sha256()
    for name in ("ops.cu", "tc.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1104_3408_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _op_traffic(w):
    """DRAM bytes per step of the operator family from the committed
    single-kernel capture summary profiles/k_op_tc_dram_<workload>.md, or
    None when there is none or it was taken on other kernel sources."""
    import re
    path = os.path.join(ROOT, "profiles", f"k_op_tc_dram_{w['name']}.md")
    if not os.path.exists(path):
        return None, "no single-kernel DRAM capture of k_op_tc for this workload"
    with open(path) as fh:
        text = fh.read()
    sha = re.search(r"sources_sha256:\s*([0-9a-f]{64})", text)
    val = re.search(r"dram_bytes_per_step:\s*([0-9.eE+]+)", text)
    if not sha or not val:
        return None, "capture summary without sources_sha256 / dram_bytes_per_step"
    if sha.group(1) != _op_sources_sha():
        return None, "capture taken on other k_op_tc sources (stale)"
    return float(val.group(1)), f"profiles/k_op_tc_dram_{w['name']}.md"


def _whole_step_bound(w, ms_step, hbm, bf16s, sm_mhz):
    """The whole-step roofline of the method: T_bound = max(operator work /
    tensor peak, algorithmic bytes / HBM peak) + right-hand-side work / ALU
    peak, per RK4 step (four substeps).  Operator work: the method's FP64
    flops 2n_r + 16N + 2(L+1) per pt-field per substep (no emulation
    overhead).  Bytes: 40 per pt-field per substep (read the stage state and
    u_n, read and write the accumulator, write the next stage).  Right-hand
    side: RHS_OPS_PER_POINT + 15 n_v (chain rule) FP64-equivalent operations
    per point, each FF_INSTR_PER_OP FP32 instructions on the FP32 pipe
    (SMS x FP32_LANES x the measured median SM clock)."""
    n_r, N, J, L, nv = w["n_r"], w["n_theta"], w["n_phi"], w["L"], w["n_fields"]
    P = n_r * N * J
    units = 4.0 * P * nv
    t_tensor = (2 * n_r + 16 * N + 2 * (L + 1)) * units / (bf16s * 1e12)
    t_hbm = 40.0 * units / (hbm * 1e9)
    clk = (sm_mhz or 2070.0) * 1e6
    t_alu = 4.0 * P * (RHS_OPS_PER_POINT + 15 * nv) * FF_INSTR_PER_OP / (SMS * FP32_LANES * clk)
    t_bound = max(t_tensor, t_hbm) + t_alu
    return {"t_tensor_ms": t_tensor * 1e3, "t_hbm_ms": t_hbm * 1e3, "t_rhs_alu_ms": t_alu * 1e3,
            "t_bound_ms": t_bound * 1e3, "ms_per_step": ms_step, "frac": t_bound * 1e3 / ms_step,
            "rhs_ops_per_point": RHS_OPS_PER_POINT + 15 * nv, "ff_instr_per_op": FF_INSTR_PER_OP,
            "sm_mhz": clk / 1e6}


def _roofline(w, per_step, launches, hbm, bf16s, peak_kind):
    """Roofline of the dominant kernel family of the traced step (largest device
    time per step).  The operator family is a dense contraction on the tensor
    cores: achieved = the method's own FP64 operator flops (2n_r + 16N +
    2(L+1) per pt-field per substep) / the family's traced time, against the
    sustained BF16 peak (it runs inside a long step).  The split-precision
    scheme issues 26 (derivatives) or 21 (filter) BF16 digit-pair products per
    such flop: that utilisation of the tensor pipe is reported beside it as
    tensor_pipe_frac.  Pointwise families are compared with HBM on their
    algorithmic bytes."""
    fam_ms = {f: sum(per_step.get(ph, 0.0) for ph in phs) for f, phs in FAMILIES.items()}
    dom = max(fam_ms, key=fam_ms.get)
    t = fam_ms[dom] * 1e-3
    nl = sum(launches.get(ph, 0) for ph in FAMILIES[dom])
    if dom == "k_op_tc":
        fl = sum(4 * _op_flops(w, ph) for ph in FAMILIES[dom])  # 4 stages
        achieved = fl / t / 1e12
        issued = sum(PAIRS[ph] * 4 * _op_flops(w, ph) for ph in FAMILIES[dom]) / t / 1e12
        byts = 4 * 8.0 * w["n_fields"] * w["n_r"] * w["n_theta"] * w["n_phi"] * (
            6 + 2 + 4 * (2 * w["L"] + 1) / w["n_phi"])
        per_launch = {}
        for ph in FAMILIES[dom]:
            tl = per_step[ph] * 1e-3
            per_launch[ph] = {"ms_per_step": per_step[ph], "launches_per_step": launches[ph],
                              "method_tflops": 4 * _op_flops(w, ph) / tl / 1e12,
                              "tensor_pipe_frac": PAIRS[ph] * 4 * _op_flops(w, ph) / tl / 1e12 / bf16s}
        traffic, tsrc = _op_traffic(w)
        return {"bound": "tensor", "kernel": "k_op_tc (all operator launches of the step)",
                "achieved": achieved, "peak": bf16s, "unit": "TFLOP/s", "frac": achieved / bf16s,
                "traffic": traffic, "traffic_source": tsrc,
                "traffic_scope": "DRAM bytes per step, all k_op_tc launches",
                "peak_source": f"bf16_tflops_sustained ({peak_kind})",
                "work": "the method's FP64 operator flops, 2n_r + 16N + 2(L+1) per pt-field per substep "
                        "(no emulation overhead)",
                "tensor_pipe_frac": issued / bf16s,
                "issued_bf16_tflops": issued,
                "issued_work": "26 (derivatives) or 21 (filter) BF16 digit-pair products per method flop",
                "hbm_view": {"algorithmic_GBps": byts / t / 1e9, "frac": byts / t / 1e9 / hbm},
                "ms_per_step": fam_ms[dom], "launches_per_step": nl, "per_phase": per_launch}
    byts = sum(launches[ph] * _pointwise_bytes(w, ph) for ph in FAMILIES[dom])
    achieved = byts / t / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "peak_source": f"hbm_gbs ({peak_kind})",
            "ms_per_step": fam_ms[dom], "launches_per_step": nl}


def run_ours(args, rank, local_rank, ws, dist, acc_steps=100):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn

    torch.cuda.set_device(local_rank)
    w = _workload(args.workload)
    n_r, N, J, L = w["n_r"], w["n_theta"], w["n_phi"], w["L"]
    P = n_r * N * J
    units_per_step = P * w["n_fields"]
    u0 = _state(w)

    fk = {"yn": cffyn.FILTER_YN, "y": cffyn.FILTER_Y, "yg": cffyn.FILTER_YG}[args.filter]
    sh = cffyn.Shell(n_r, N, J, w["r_in"], w["r_out"], L, n_fields=w["n_fields"],
                     precision=cffyn.MIXED, filter_kind=fk)
    dt = w["lam"] * sh.default_dt() / 0.25
    u = torch.from_numpy(u0).cuda()
    sh.init_gauge_from_state(u)
    uf = torch.empty_like(u)
    sh.filter(u, uf)
    u.copy_(uf)
    for _ in range(max(args.warmup, 3)):
        sh.rk4_step(u, dt, 1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    # keep the GPU loaded for ~1 s before the timed region so that the 200 ms
    # clock samples cover a loaded period that ends in the timed region
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        sh.rk4_step(u, dt, 1)
    torch.cuda.synchronize()
    # timed region 1 (the value): K steps of the plain step graph
    t_ms = _time_steps(sh, u, dt, args.steps, flush, torch)
    torch.cuda.synchronize()
    # the same K steps through the synchronising call (each step's events
    # then also hold the host's wake-up after the step): reported beside
    t_sync_ms = _time_steps(sh, u, dt, args.steps, flush, torch, use_async=False)
    torch.cuda.synchronize()
    # kernel launches per step of the plain graph (its capture counted them;
    # it runs the filter as two chains, so it launches more than the traced one)
    launches_plain = sh.get_trace()[1]
    if dist:
        dist.barrier()
    # timed region 2 (the roofline): K steps of the traced graph, whose event
    # nodes between kernel groups give every group's device time
    sh.set_trace(True)
    sh.rk4_step(u, dt, 1)          # capture the traced graph outside the timed region
    sh.set_trace(True)             # reset totals
    torch.cuda.synchronize()
    t_traced_ms = _time_steps(sh, u, dt, args.steps, flush, torch, use_async=False)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    trace_ms, launches, tsteps = sh.get_trace()
    sh.set_trace(False)
    t_max = _max_over_ranks(t_ms, dist)
    value = units_per_step * args.steps * ws / (t_max * 1e-3)

    if rank != 0:
        return None

    # ---- dominant kernel family, live from the traced timed region
    hbm, bf16s, peak_kind = _peaks()
    per_step = {k: v / max(tsteps, 1) for k, v in trace_ms.items()}
    roof = _roofline(w, per_step, launches, hbm, bf16s, peak_kind)
    roof["whole_step"] = _whole_step_bound(w, t_max / args.steps, hbm, bf16s,
                                           clk.get("sm_mhz") if clk else None)

    # ---- plain FP64 GPU path on the same workload
    fp64 = None
    if not args.no_fp64:
        s64 = cffyn.Shell(n_r, N, J, w["r_in"], w["r_out"], L, n_fields=w["n_fields"],
                          precision=cffyn.FP64, filter_kind=fk)
        v = torch.from_numpy(u0).cuda()
        s64.init_gauge_from_state(v)
        vf = torch.empty_like(v)
        s64.filter(v, vf)
        v.copy_(vf)
        for _ in range(2):
            s64.rk4_step(v, dt, 1)
        k64 = max(2, min(args.steps, 5))
        t64 = _time_steps(s64, v, dt, k64, flush, torch)
        fp64_value = units_per_step * k64 / (t64 * 1e-3)
        # accuracy: acc_steps steps of both paths from the same filtered state
        a = torch.from_numpy(u0).cuda()
        sh.init_gauge_from_state(a)
        sh.filter(a, uf)
        a.copy_(uf)
        b = a.clone()
        sh.rk4_step(a, dt, acc_steps)
        s64.rk4_step(b, dt, acc_steps)
        err = float((a - b).abs().max() / b.abs().max())
        s64.destroy()
        fp64 = {"value": fp64_value, "steps": k64, "mixed_over_fp64": value / ws / fp64_value,
                f"err_fields_{acc_steps}_steps_vs_fp64_gpu": err}

    # ---- end to end through the C-ABI with host buffers
    e2e = _e2e(sh, u0, u, dt, max(3, min(args.steps, 10)), units_per_step)

    # ---- CPU oracle on a bounded sample
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = _cpu_baseline(w, u0)

    # the step graph's kernel nodes, plus the pair copy of the state that
    # every mixed-path step call launches ahead of the graph (k_to_store)
    launches_per_step = sum(launches_plain.values()) + 1
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: bf16-digit tensor products (exact fp32 sums, int64 recombination), "
                 "fp32-pair pointwise, f64 state",
        "data": "synthetic (seeded Kerr-Schild + l<=4 perturbation, amplitude 1e-4)",
        "config": {"workload": w["name"], "n_r": n_r, "n_theta": N, "n_phi": J,
                   "n_fields": w["n_fields"], "L": L, "r": [w["r_in"], w["r_out"]],
                   "dt": dt, "filter": {"yn": "Yn", "y": "Y", "yg": "Yg"}[args.filter] + " on every stage rhs",
                   "precision": "mixed",
                   "parallelism": f"replicas x{ws}",
                   "l2": "flushed (256 MiB write) before every timed step",
                   "timing": "CUDA events around each step's cffyn_rk4_step_async call on the launching "
                             "stream; status words checked after the last step"},
        "roofline": roof,
        "ms_per_step_sync_call": t_sync_ms / args.steps,
        "ms_per_step_traced": t_traced_ms / args.steps,
        "phase_ms_per_step": per_step,
        "launches_per_step": launches_plain,
        "launches_per_step_traced": launches,
        "gpu_launches": launches_per_step * args.steps,
        "fp64_gpu": fp64,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    sh.destroy()
    return out


def _e2e(sh, u0, u, dt, ke, units_per_step):
    """The metric end to end through the public API with the state in pinned
    host memory: every timed step copies its input in from the host and its
    result back.  `value`: ke independent problems through cffyn.HostStepper
    (each problem's copies overlapped with its neighbours' steps on two copy
    streams); `serial`: the same with copy in, step and copy out one after
    the other on one stream."""
    import torch
    from paper_1104_3408_gb300 import cffyn
    hu = torch.from_numpy(u0).pin_memory()
    hout = torch.empty_like(hu).pin_memory()
    st = torch.cuda.current_stream()
    nbytes = int(u.numel() * 8)

    def timed(fn):
        fn(1)  # captures the step graph for this state buffer
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn(ke)
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    hs = cffyn.HostStepper(sh, u)
    ms_pipe = timed(lambda n: hs.run([hu] * n, [hout] * n, dt, 1, st))
    dbuf = torch.empty_like(u)

    def serial(n):
        for _ in range(n):
            dbuf.copy_(hu, non_blocking=True)
            sh.rk4_step(dbuf, dt, 1)
            hout.copy_(dbuf, non_blocking=True)
    ms_ser = timed(serial)
    return {"value": units_per_step * ke / (ms_pipe * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": ke,
            "how": "cffyn.HostStepper: ke independent problems from pinned host memory, each "
                   "problem's copy in / copy out overlapped with the neighbouring problems' steps",
            "serial": {"value": units_per_step * ke / (ms_ser * 1e-3),
                       "how": "copy in, step, copy out in turn on one stream"}}


def _oracle_state(w, u0):
    """The bench state with the gauge source of 54/58-field states filled in
    (H_a = -Gamma_a in fields 50..53), as the library's gauge initialisation does."""
    from oracle import ghg
    if w["n_fields"] == 50:
        return u0
    u = u0.copy()
    u[50:54] = ghg.gauge_source_from_state(u[:50].reshape(50, -1)).reshape((4,) + u.shape[1:])
    return u


def _shell_units(d):
    return d["n_r"] * d["n_theta"] * d["n_phi"] * 50


def _shells_for_rank(descs, rank, ws):
    """Greedy longest-first assignment of the batch's shells to ranks by
    points x fields; returns this rank's shell indices."""
    order = sorted(range(len(descs)), key=lambda i: (-_shell_units(descs[i]), i))
    load = [0] * ws
    mine = []
    for i in order:
        r = min(range(ws), key=lambda k: (load[k], k))
        load[r] += _shell_units(descs[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def run_batch(args, rank, local_rank, ws, dist):
    """The uneven-shell batch: every shell of this rank advanced by one batch
    RK4 step per graph launch (cffyn_batch_rk4_step).  Across ranks the shells
    are split by cost (total work fixed: strong scaling)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn, inputs

    torch.cuda.set_device(local_rank)
    w = _workload(args.workload)
    descs = inputs.shell_batch(w["n_shells"], seed=w["seed"])
    mine = _shells_for_rank(descs, rank, ws)

    def state(d):
        return inputs.kerr_schild_state(d["n_r"], d["n_theta"], d["n_phi"], d["r_in"], d["r_out"],
                                        amp=d["amp"], ell=d["ell"], seed=d["seed"])

    def make(d, prec):
        sh = cffyn.Shell(d["n_r"], d["n_theta"], d["n_phi"], d["r_in"], d["r_out"], d["L"],
                         precision=prec)
        u = torch.from_numpy(state(d)).cuda()
        sh.init_gauge_from_state(u)
        v = torch.empty_like(u)
        sh.filter(u, v)
        return sh, v

    t_setup = time.perf_counter()
    shells, us = zip(*[make(descs[i], cffyn.MIXED) for i in mine])
    shells, us = list(shells), list(us)
    t_setup = time.perf_counter() - t_setup
    units = sum(_shell_units(descs[i]) for i in mine)
    units_all = sum(_shell_units(d) for d in descs)
    b = cffyn.Batch(shells)
    st = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        b.rk4_step(us, None, 1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        b.rk4_step(us, None, 1)
    torch.cuda.synchronize()
    a_ev = torch.cuda.Event(enable_timing=True)
    b_ev = torch.cuda.Event(enable_timing=True)
    a_ev.record(st)
    b.rk4_step(us, None, args.steps)
    b_ev.record(st)
    torch.cuda.synchronize()
    t_ms = a_ev.elapsed_time(b_ev)
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    t_max = _max_over_ranks(t_ms, dist)
    value = units_all * args.steps / (t_max * 1e-3) if dist else units * args.steps / (t_max * 1e-3)
    if rank != 0:
        b.destroy()
        return None

    # ---- the same shells stepped one by one (no batch), mixed and FP64
    def loop_rate(shs, vs, k):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(k):
            for sh, v in zip(shs, vs):
                sh.rk4_step(v, 0.0, 1)
        e1.record(st)
        torch.cuda.synchronize()
        return units * k / (e0.elapsed_time(e1) * 1e-3)

    for sh, v in zip(shells, us):
        sh.rk4_step(v, 0.0, 1)      # capture each shell's own graph
    mixed_loop = loop_rate(shells, us, 2)
    # kernel launches of one shell's step (the same sequence for every
    # 50-field mixed shell and for every stacked class of the batch), counted
    # by the capture of its step graph
    shells[0].rk4_step(us[0], 0.0, 1)
    launches_per_shell_step = sum(shells[0].get_trace()[1].values())
    fp64 = None
    if not args.no_fp64:
        s64, v64 = zip(*[make(descs[i], cffyn.FP64) for i in mine])
        for sh, v in zip(s64, v64):
            sh.rk4_step(v, 0.0, 1)
        fp64_loop = loop_rate(s64, v64, 1)
        # accuracy: 100 steps of the first 8 shells, mixed batch vs FP64 loop
        k8 = min(8, len(mine))
        s8, u8 = zip(*[make(descs[i], cffyn.MIXED) for i in mine[:k8]])
        b8 = cffyn.Batch(list(s8))
        _, r8 = zip(*[make(descs[i], cffyn.FP64) for i in mine[:k8]])
        b8.rk4_step(list(u8), None, 100)
        for sh, v in zip(s64[:k8], r8):
            sh.rk4_step(v, 0.0, 100)
        err = max(float((x - y).abs().max() / y.abs().max()) for x, y in zip(u8, r8))
        b8.destroy()
        for sh in list(s8) + list(s64):
            sh.destroy()
        fp64 = {"per_shell_loop_value": fp64_loop, "batch_over_fp64_loop": value / fp64_loop,
                "err_fields_100_steps_vs_fp64_gpu": err, "err_shells": k8}

    # ---- end to end with host buffers: copy in, one batch step, copy out
    hs = [u.cpu().pin_memory() for u in us]
    hout = [torch.empty_like(h).pin_memory() for h in hs]
    ke = 3

    def timed_e2e(fn):
        fn(1)  # captures the step graphs for these state buffers
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn(ke)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    hstep = cffyn.HostStepper(b, us)
    ms_pipe = timed_e2e(lambda n: hstep.run([hs] * n, [hout] * n, None, 1, st))

    def serial(n):
        for _ in range(n):
            for u, h in zip(us, hs):
                u.copy_(h, non_blocking=True)
            b.rk4_step(us, None, 1)
            for u, h in zip(us, hout):
                h.copy_(u, non_blocking=True)
    ms_ser = timed_e2e(serial)
    del hstep
    nbytes = int(sum(u.numel() for u in us) * 8)
    e2e = {"value": units * ke / (ms_pipe * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": ke,
           "how": "cffyn.HostStepper over the batch: ke independent batch problems from pinned host "
                  "memory, each problem's copies overlapped with the neighbouring problems' steps",
           "serial": {"value": units * ke / (ms_ser * 1e-3),
                      "how": "copy in, batch step, copy out in turn on one stream"}}

    # ---- whole-step tensor roofline (a lower bound of the operator family's share)
    hbm, bf16s, peak_kind = _peaks()
    fl = issued = 0.0
    for i in mine:
        d = descs[i]
        deriv = 2 * d["n_r"] + 8 * d["n_theta"]
        filt = 8 * d["n_theta"] + 2 * (d["L"] + 1)
        fl += 4.0 * (deriv + filt) * _shell_units(d)
        issued += 4.0 * (26 * deriv + 21 * filt) * _shell_units(d)
    achieved = fl * args.steps / (t_ms * 1e-3) / 1e12
    roof = {"bound": "tensor", "kernel": "k_op_tc (operator work over the whole batch step time)",
            "achieved": achieved, "peak": bf16s, "unit": "TFLOP/s", "frac": achieved / bf16s,
            "traffic": None, "traffic_source": "no single-kernel capture of the batch",
            "peak_source": f"bf16_tflops_sustained ({peak_kind})",
            "work": "the method's FP64 operator flops, 2n_r + 16N + 2(L+1) per pt-field per substep",
            "tensor_pipe_frac": issued * args.steps / (t_ms * 1e-3) / 1e12 / bf16s,
            "scope": "divides by the whole step (all kernel families), so it is a lower bound "
                     "of the operator kernels' own fraction"}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        d = descs[mine[0]]
        wd = dict(d, n_fields=50, name="batch shell 0")
        cpu = _cpu_baseline(wd, state(d))
        cpu["sample"] = ("one RK4 stage of the batch's first shell "
                         f"({d['n_r']}x{d['n_theta']}x{d['n_phi']}) = 1/4 step; numpy FP64")
    nshapes = {}
    for i in mine:
        k = f"{descs[i]['n_r']}x{descs[i]['n_theta']}x{descs[i]['n_phi']}"
        nshapes[k] = nshapes.get(k, 0) + 1
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "mixed: bf16-digit tensor products (exact fp32 sums, int64 recombination), "
                 "fp32-pair pointwise, f64 state",
        "data": "synthetic (seeded Kerr-Schild + l<=4 perturbations, amplitudes log-uniform "
                "1e-6..1e-3)",
        "config": {"workload": w["name"], "n_shells": len(descs), "shells_this_rank": len(mine),
                   "pt_field_per_step": units_all, "shapes": nshapes, "n_fields": 50,
                   "L": "n_theta - 2", "r": [1.8, 11.0], "filter": "Yn on every stage rhs",
                   "precision": "mixed", "parallelism": f"shells split by cost over {ws} rank(s)",
                   "l2": f"inputs larger than L2 ({units * 8 / 1e9:.1f} GB of state per rank)",
                   "setup_s": t_setup},
        "roofline": roof,
        "mixed_per_shell_loop_value": mixed_loop,
        "batch_over_mixed_loop": value / mixed_loop,
        "gpu_launches": launches_per_shell_step * b.units() * args.steps,
        "launches_per_class_step": launches_per_shell_step,
        "classes": b.units(),
        "fp64_gpu": fp64,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    b.destroy()
    for sh in shells:
        sh.destroy()
    return out


def _cpu_baseline(w, u0, nthreads=None):
    """The oracle, as it stands, on one RK4 stage (derivatives + right-hand side
    + boundary + Yn filter) of the same workload: a quarter of a step."""
    import oracle
    t0 = time.perf_counter()
    sh = oracle.OracleShell(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"], w["L"],
                            n_fields=w["n_fields"])
    u0 = _oracle_state(w, u0)
    sh.init_gauge_from_state(u0)
    _ = sh.sf
    t1 = time.perf_counter()
    k = sh.stage(u0)
    t2 = time.perf_counter()
    del k
    units = w["n_r"] * w["n_theta"] * w["n_phi"] * w["n_fields"] / 4.0
    return {"value": units / (t2 - t1), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one RK4 stage (rhs + BC + Yn filter) of the same shell = 1/4 step; "
                      f"setup {t1 - t0:.1f} s excluded; numpy FP64",
            "seconds": t2 - t1}


def run_reference(args, rank):
    """Reference arm: the CPU oracle on the host cores, same workload and metric;
    each step is one RK4 stage sample (a quarter of a full step)."""
    if rank != 0:
        return None
    w = _workload(args.workload)
    u0 = _oracle_state(w, _state(w))
    import oracle
    sh = oracle.OracleShell(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"], w["L"],
                            n_fields=w["n_fields"])
    sh.init_gauge_from_state(u0)
    _ = sh.sf
    for _ in range(min(args.warmup, 1)):
        sh.stage(u0)
    budget = 240.0
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sh.stage(u0)
        times.append(time.perf_counter() - t0)
        if sum(times) > budget:
            break
    units = w["n_r"] * w["n_theta"] * w["n_phi"] * w["n_fields"] / 4.0
    value = units * len(times) / sum(times)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": len(times),
        "steps_requested": args.steps, "warmup": min(args.warmup, 1),
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": w["name"], "n_r": w["n_r"], "n_theta": w["n_theta"],
                   "n_phi": w["n_phi"], "n_fields": w["n_fields"], "L": w["L"],
                   "step": "one RK4 stage (rhs + BC + Yn filter) = 1/4 RK4 step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "one RK4 stage of the same shell per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_profile_step(args):
    """One eager RK4 step of the workload (mixed path): gauge from the state,
    then Shell.profile_step.  Launch order: the three gauge-derivative operator
    launches, then per stage the groups of cffyn_profile_step."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn

    w = _workload(args.workload)
    sh = cffyn.Shell(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"], w["L"],
                     n_fields=w["n_fields"], precision=cffyn.MIXED)
    u = torch.from_numpy(_state(w)).cuda()
    sh.init_gauge_from_state(u)
    prof = sh.profile_step(u)
    torch.cuda.synchronize()
    sh.destroy()
    return {"workload": w["name"], "profile_step_ms": {k: t for k, (t, n) in prof.items()},
            "launches": {k: n for k, (t, n) in prof.items()}}


def run_graph_step(args):
    """One RK4 step of the workload through cffyn_rk4_step (mixed path): the
    gauge from the state, then the step graph's launches (the pair copy of the
    state, then per stage its kernel nodes, the filter as two chains)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn

    w = _workload(args.workload)
    sh = cffyn.Shell(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"], w["L"],
                     n_fields=w["n_fields"], precision=cffyn.MIXED)
    u = torch.from_numpy(_state(w)).cuda()
    sh.init_gauge_from_state(u)
    sh.rk4_step(u, 0.0, 1)
    torch.cuda.synchronize()
    launches = sh.get_trace()[1]
    sh.destroy()
    return {"workload": w["name"], "launches": launches}


def run_derivs_sweep(args):
    """Cartesian derivatives of 50 fields on shells n_r x n x 2n (n_r = n) by
    three methods: the split-precision matrices on the tensor cores (MIXED),
    the FP64 matrices, and FP64 FFTs (cuFFT; cffyn_derivs_fft): the GB300
    analogue of the paper's matrix-vs-FFT comparison (Sec. 5, Fig. mmfft), for
    the whole derivative rather than one transform.  CUDA events on the
    launching stream, median of 5 calls after 2 warm-up calls, L2 flushed
    before each call."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn, inputs

    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    nv = 50
    rows = []
    for n in [int(x) for x in args.sweep.split(",")]:
        base = inputs.band_limited_fields(n, n, 2 * n, 1.8, 11.0, n_fields=5, seed=n)
        u = torch.from_numpy(np.ascontiguousarray(np.tile(base, (nv // 5, 1, 1, 1)))).cuda()
        shells = {"matrix_mixed": cffyn.Shell(n, n, 2 * n, 1.8, 11.0, n - 2, precision=cffyn.MIXED),
                  "matrix_fp64": cffyn.Shell(n, n, 2 * n, 1.8, 11.0, n - 2, precision=cffyn.FP64)}
        calls = {"matrix_mixed": lambda o: shells["matrix_mixed"].derivs(u, o),
                 "matrix_fp64": lambda o: shells["matrix_fp64"].derivs(u, o),
                 "fft_fp64": lambda o: shells["matrix_fp64"].derivs_fft(u, o)}
        outs, ms = {}, {}
        for name, fn in calls.items():
            o = torch.empty((3,) + tuple(u.shape), dtype=torch.float64, device="cuda")
            for _ in range(2):
                fn(o)
            times = []
            for _ in range(5):
                flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(st)
                fn(o)
                b.record(st)
                b.synchronize()
                times.append(a.elapsed_time(b))
            ms[name] = statistics.median(times)
            outs[name] = o
        ref = outs["matrix_fp64"]
        scale = float(ref.abs().max())
        units = float(n * n * 2 * n * nv)
        rows.append({"n_r": n, "n_theta": n, "n_phi": 2 * n, "ms": ms,
                     "pt_field_per_s": {k: units / (v * 1e-3) for k, v in ms.items()},
                     "rel_diff_vs_matrix_fp64": {k: float((outs[k] - ref).abs().max()) / scale
                                                 for k in ("matrix_mixed", "fft_fp64")}})
        for sh in shells.values():
            sh.destroy()
        del outs, u
        torch.cuda.empty_cache()
    return {"mode": "derivs_sweep", "fields": nv, "method_note":
            "matrix_mixed: split-precision BF16 digit products on tcgen05 (k_op_tc); matrix_fp64: "
            "FP64 matrices (k_op_fp64); fft_fp64: cuFFT D2Z/Z2D with the library's own extension, "
            "recurrence and transpose kernels; all followed by the same chain-rule kernel",
            "timing": "median of 5 calls after 2 warm-ups, CUDA events, L2 flushed before each call",
            "rows": rows}


def run_other_workloads(args, local_rank):
    """Shorter measurements of the other two throughput configurations on the
    same GPU, after the main line: the 58-field 65 x 96 x 192 shell (5 timed
    steps, FP64 path beside it, fields compared after 10 steps) and the batch
    of 256 uneven shells (5 timed batch steps, per-shell loops beside it).
    Same timing rules as the main line; no CPU baseline."""
    import copy

    import torch
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "config", "roofline", "fp64_gpu", "e2e",
            "clocks", "gpu_launches", "mixed_per_shell_loop_value", "batch_over_mixed_loop", "classes")
    res = {}
    for name, fn in (("ks_65x96x192_58f", lambda a: run_ours(a, 0, local_rank, 1, None, acc_steps=10)),
                     ("batch_256", lambda a: run_batch(a, 0, local_rank, 1, None))):
        a = copy.copy(args)
        a.workload, a.steps, a.warmup, a.no_cpu_baseline = name, 5, 3, True
        try:
            r = fn(a)
            res[name] = {k: r[k] for k in keep if k in r}
        except Exception as e:  # recorded in the line, never hides the main value
            res[name] = {"error": repr(e)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return res


def main():
    args = _args()
    if args.profile_step:
        print(json.dumps(run_profile_step(args)), flush=True)
        return
    if args.profile_graph:
        print(json.dumps(run_graph_step(args)), flush=True)
        return
    if args.sweep:
        print(json.dumps(run_derivs_sweep(args)), flush=True)
        return
    rank, local_rank, ws, dist = _dist()
    batch = "n_shells" in _workload(args.workload)
    if args.impl == "reference":
        out = run_reference(args, rank) if not batch else {
            "impl": "reference", "unavailable": "the reference arm times the oracle on the "
            "single-shell workloads only"}
    elif batch:
        out = run_batch(args, rank, local_rank, ws, dist)
    else:
        out = run_ours(args, rank, local_rank, ws, dist)
        if ws == 1 and not args.no_other_workloads and args.workload == "ks_33x48x96":
            out["other_workloads"] = run_other_workloads(args, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
