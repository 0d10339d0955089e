#!/usr/bin/env python
"""Benchmark: Rand-QLP time-to-factor and A-pass GB/s on one GB300.

Workload: A = U_r diag(exp(-i/50)) V_r^T + 1e-6 G / sqrt(n), 20000 x 20000
FP32 (Haar U_r, V_r, r = 1000), k = 200, p = 10, q = 2, Gaussian Omega
20000 x 210. One step = one full factorisation A -> (Q, L, P) through the
C ABI with A resident in HBM. value = GB/s of A streamed by the 2q + 2
passes over A (aggregate over ranks), ms_per_step = time to factor.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16x3|auto]
  (auto = the BF16-split tensor-core form; the plain FP32 form is timed beside it)
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

For N > 1 (torchrun) every rank factors its own replica (the path does not
shard across GPUs: replicas only, weak scaling), timing is max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Rand-QLP time & A-pass GB/s at 20k², k=200: BF16-split+learned q vs FP32"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
# GB300: 152 SMs x 128 FP32 lanes x 2 flop/FMA at the maximum SM clock.
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16x3"])
    ap.add_argument("--m", type=int, default=20000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the plain FP32 form")
    ap.add_argument("--sample", type=int, default=0,
                    help="rows/cols of the oracle's sample block (0 = default for the workload)")
    return ap.parse_args()


def workload_name(a):
    return f"rand_qlp {a.m}x{a.n} k={a.k} p={a.p} q={a.q}"


def apass_bytes(a):
    return (2 * a.q + 2) * a.m * a.n * 4


# ------------------------------------------------------------------ inputs

def make_inputs(a, device):
    from paper_2110_01011_gb300 import inputs
    sig = inputs.exp_spectrum(1000, 50.0)
    A = inputs.low_rank_matrix_torch(a.m, a.n, sig, 1e-6, seed=1002, rank=1000, device=device)
    Om = inputs.omega_torch(a.m, a.k + a.p, seed=2002, device=device)
    return A, Om


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle baseline

def oracle_inputs(a, S, A=None):
    """The leading S x S block of the workload's A (same generator and seed)
    and the matching Omega rows, in float64 on the host."""
    import numpy as np
    import torch

    from paper_2110_01011_gb300 import inputs
    if A is None:
        sig = inputs.exp_spectrum(1000, 50.0)
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        A = inputs.low_rank_matrix_torch(a.m, a.n, sig, 1e-6, seed=1002, rank=1000, device=dev)
    As = A[:S, :S].double().cpu().numpy()
    Om = inputs.omega(a.m, a.k + a.p, seed=2002)[:S].astype(np.float64)
    return As, Om


def oracle_time(a, As, Om):
    """One run of the FP64 oracle chain on the sample; returns (GB/s, s, cores)."""
    from oracle import rqlp_oracle as orc
    S = As.shape[0]
    t0 = time.perf_counter()
    orc.rand_qlp(As, Om, a.q)
    dt = time.perf_counter() - t0
    gbs = (2 * a.q + 2) * S * S * 4 / dt / 1e9
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    return gbs, dt, cores


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    S = a.sample or 2000
    As, Om = oracle_inputs(a, S)
    vals = []
    for i in range(a.warmup + a.steps):
        gbs, dt, cores = oracle_time(a, As, Om)
        if i >= a.warmup:
            vals.append((gbs, dt))
    gbs = statistics.median(v[0] for v in vals)
    ms = statistics.median(v[1] for v in vals) * 1e3
    sample = f"FP64 oracle chain on the leading {S}x{S} block of the workload's A, q={a.q}, d={a.k + a.p}"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": sample, "parallelism": "cpu"},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def kernel_sha():
    h = hashlib.sha256()
    for f in ("gemm_simt.cu", "tc_gemm.cu"):
        p = os.path.join(ROOT, "paper_2110_01011_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:12]


def traffic_for(kernel, sha):
    """DRAM bytes per launch recorded from an ncu capture of this exact kernel source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    for line in open(TRAFFIC_FILE):
        f = line.split()
        if len(f) >= 3 and f[0] == kernel and f[1] == sha:
            return float(f[2])
    return None


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    from paper_2110_01011_gb300 import rqlp
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    lib = rqlp.load()
    del lib
    # The headline form is the BF16-split tensor-core path; FP32 is timed beside it.
    prec = {"fp32": rqlp.PREC_FP32, "bf16x3": rqlp.PREC_BF16X3}.get(a.precision, rqlp.PREC_BF16X3)
    d = a.k + a.p

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    A, Om = make_inputs(a, dev)
    opts = rqlp._opts(prec)
    wsb = rqlp.rqlp_workspace_bytes(a.m, a.n, a.k, a.p, a.q, opts)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
    Q = torch.empty(a.m, d, device=dev)
    L = torch.empty(d, d, device=dev)
    P = torch.empty(a.n, d, device=dev)
    info = torch.empty(2, dtype=torch.int32, device=dev)
    diag = torch.empty(4, dtype=torch.float64, device=dev)
    out = (Q, L, P, info, diag)

    def step():
        rqlp.factor(A, a.k, a.p, a.q, Om, precision=prec, workspace=ws, out=out)

    for _ in range(a.warmup):
        step()
    barrier()
    status = int(info[0].item())
    rqlp.rqlp_profile_read()          # drop records from the warm-up
    rqlp.rqlp_profile_enable(True)
    clocks = ClockSampler(local)
    l0 = rqlp.rqlp_kernel_launches()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    for _ in range(a.steps):
        step()
    e1.record(st)
    barrier()
    launches = rqlp.rqlp_kernel_launches() - l0
    rqlp.rqlp_profile_enable(False)
    ck = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms_total], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    recs = rqlp.rqlp_profile_read()
    ms_step = ms_total / a.steps
    value = world * apass_bytes(a) / (ms_step * 1e-3) / 1e9

    # Dominant kernel: the pass over A (A^T X / A X products), timed per launch.
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    by_tag = {0: [r[0] for r in recs if r[1] == 0], 1: [r[0] for r in recs if r[1] == 1]}
    dom = max(by_tag, key=lambda t: sum(by_tag[t]))
    pass_ms = statistics.mean(by_tag[dom]) if by_tag[dom] else float("nan")
    flops = 2.0 * a.m * a.n * d
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    kname = {0: "pass_AX", 1: "pass_AtX"}[dom]
    sha = kernel_sha()
    if prec == rqlp.PREC_FP32:
        peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (pass_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"}
    else:
        # The split form's algorithm is three BF16 products per pass (A_hi X_hi +
        # A_hi X_lo + A_lo X_hi); the pass timed is a power-pass / projection one.
        peak = peaks.get("bf16_tflops_sustained", 1683.0)
        mma_flops = 3 * flops
        roof = {"bound": "tensor", "achieved": mma_flops / (pass_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "flops_per_launch": mma_flops,
                "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (of measured)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.setdefault("flops_per_launch", flops)
    roof["traffic"] = traffic_for(f"{kname}_{'fp32' if prec == 0 else 'bf16x3'}", sha)
    roof["kernel"] = kname
    roof["launch_ms"] = pass_ms
    roof["hbm_gbs"] = a.m * a.n * 4 / (pass_ms * 1e-3) / 1e9
    roof["hbm_frac_of_measured"] = roof["hbm_gbs"] / peaks.get("hbm_gbs", 6761.6)

    # Accuracy of the timed form (Q L P^T = A P~ P~^T, so the residual follows from
    # ||A||_F^2 - ||L||_F^2) and the plain-FP32 form timed on the same inputs.
    dg = diag.cpu().tolist()
    relres = (max(dg[2], 0.0) / dg[0]) ** 0.5 if dg[0] > 0 else float("nan")
    compare = {"form": "fp32" if prec == rqlp.PREC_FP32 else "bf16x3", "rel_residual": relres}
    if prec != rqlp.PREC_FP32 and not a.no_compare:
        out32 = (torch.empty_like(Q), torch.empty_like(L), torch.empty_like(P), torch.empty_like(info),
                 torch.empty_like(diag))
        ws32 = torch.empty(rqlp.rqlp_workspace_bytes(a.m, a.n, a.k, a.p, a.q, rqlp._opts(rqlp.PREC_FP32)) + 256,
                           dtype=torch.uint8, device=dev)
        rqlp.factor(A, a.k, a.p, a.q, Om, precision=rqlp.PREC_FP32, workspace=ws32, out=out32)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nf = 3
        f0.record(st)
        for _ in range(nf):
            rqlp.factor(A, a.k, a.p, a.q, Om, precision=rqlp.PREC_FP32, workspace=ws32, out=out32)
        f1.record(st)
        barrier()
        d32 = out32[4].cpu().tolist()
        compare["fp32_ms_per_step"] = f0.elapsed_time(f1) / nf
        compare["fp32_rel_residual"] = (max(d32[2], 0.0) / d32[0]) ** 0.5
        compare["speedup_vs_fp32"] = compare["fp32_ms_per_step"] / ms_step
        # ||L_split - L_fp32|| on the leading-k diagonal (both against the same A)
        l16 = torch.diagonal(L)[: a.k].double()
        l32 = torch.diagonal(out32[1])[: a.k].double()
        compare["lead_k_Lii_rel_diff_vs_fp32"] = float(((l16 - l32).abs() / l32.abs()).max())
        del ws32, out32
        torch.cuda.empty_cache()

    # End to end through the host-buffer entry point (pinned buffers).
    e2e = None
    if not a.no_e2e:
        hA = A.cpu().pin_memory()
        hO = Om.cpu().pin_memory()
        hout = (torch.empty(a.m, d).pin_memory(), torch.empty(d, d).pin_memory(),
                torch.empty(a.n, d).pin_memory(), torch.zeros(2, dtype=torch.int32),
                torch.zeros(4, dtype=torch.float64))
        hws = torch.empty(rqlp.rqlp_host_workspace_bytes(a.m, a.n, a.k, a.p, a.q, opts) + 256,
                          dtype=torch.uint8, device=dev)
        torch.cuda.empty_cache()
        for _ in range(max(1, a.warmup)):
            rqlp.factor_host(hA, a.k, a.p, a.q, hO, precision=prec, workspace=hws, out=hout)
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            rqlp.factor_host(hA, a.k, a.p, a.q, hO, precision=prec, workspace=hws, out=hout)
        barrier()
        dt = (time.perf_counter() - t0) / a.steps
        if world > 1:
            t = torch.tensor([dt], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        h2d = 4 * (a.m * a.n + a.m * d)
        d2h = 4 * (a.m * d + d * d + a.n * d) + 8 + 32
        e2e = {"value": world * apass_bytes(a) / dt / 1e9, "unit": "GB/s", "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    A_keep = A
    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        S = a.sample or 4000
        gbs, dt, cores = oracle_time(a, *oracle_inputs(a, S, A_keep))
        cpu = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle chain on the leading {S}x{S} block of the workload's A "
                         f"(q={a.q}, d={d}), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == rqlp.PREC_FP32 else "bf16x3",
                "data": "synthetic",
                "config": {"workload": workload_name(a), "m": a.m, "n": a.n, "k": a.k, "p": a.p,
                           "q": a.q, "precision": "fp32" if prec == 0 else "bf16x3",
                           "A_bytes_per_step": apass_bytes(a),
                           "l2": "inputs larger than L2 (A is %.1f GB)" % (a.m * a.n * 4 / 1e9),
                           "parallelism": "replicas" if world > 1 else "single"},
                "status": status, "clocks": ck, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "compare": compare,
                "gpu_launches": launches, "kernel_sha": sha}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
