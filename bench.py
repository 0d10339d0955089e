#!/usr/bin/env python
"""Benchmark: Rand-QLP time-to-factor and A-pass GB/s on one GB300.

Workload: A = U_r diag(exp(-i/50)) V_r^T + 1e-6 G / sqrt(n), 20000 x 20000
FP32 (Haar U_r, V_r, r = 1000), k = 200, Gaussian Omega 20000 x 220 rounded
to BF16-representable values (its first k + p columns are the sketch's test
matrix; every form then sketches with the same one).

Headline (``--form learned``, the default): the BF16-split tensor-core form
with (q, p) predicted by the trained network for the excess rank-k error that
the plain FP32 form reaches with the fixed q = 2, p = 10 on the same matrix
(equal accuracy). One step = one rqlp_factor_learned call (probe, prediction,
chain) with A resident in HBM. value = GB/s of A streamed by the 2q + 2 passes
over A (aggregate over ranks), ms_per_step = time to factor. The plain FP32
form and the split form with the fixed (2, 10) are timed beside it.
``--form fixed`` times rqlp_factor with --precision and --q/--p instead.

A ``batched`` object times the batched form on 512 uneven problems (m in
[256, 4096], n in [256, 2048], k in [8, 64], p = 5, q = 1; half exponential,
half polynomial spectra) as one graph launch after autotuning.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form learned|fixed]
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
    ap.add_argument("--form", default="learned", choices=["learned", "fixed", "batched"],
                    help="batched: only the batched leg, printed as its own line")
    ap.add_argument("--target", type=float, default=None,
                    help="learned form: this request instead of the excess error FP32 (2, 10) reaches")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16x3"],
                    help="--form fixed: the form timed (auto = bf16x3)")
    ap.add_argument("--parts", type=int, default=0, choices=[0, 2, 3],
                    help="BF16 parts per pass operand of the split form (0 = the library's automatic choice)")
    ap.add_argument("--m", type=int, default=20000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the plain FP32 form")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched form")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--no-autotune", action="store_true", help="batched leg: default tile shapes")
    ap.add_argument("--batched-precision", default="both", choices=["both", "fp32", "bf16x3"],
                    help="batched leg: FP32 products, BF16x3 tensor-core passes, or both (value = BF16x3)")
    ap.add_argument("--sample", type=int, default=0,
                    help="rows/cols of the oracle's sample block (0 = default for the workload)")
    ap.add_argument("--log", default=None, help="also append the JSON line to this JSONL file")
    return ap.parse_args()


def emit(a, line):
    """The run's one JSON line on stdout (and appended to --log)."""
    text = json.dumps(line)
    print(text, flush=True)
    if a.log:
        with open(a.log, "a") as f:
            f.write(text + "\n")


def workload_name(a):
    return f"rand_qlp {a.m}x{a.n} k={a.k} p={a.p} q={a.q}"


def apass_bytes(a):
    return (2 * a.q + 2) * a.m * a.n * 4


# ------------------------------------------------------------------ inputs

SPECTRUM_RANK = 1000


def spectrum():
    from paper_2110_01011_gb300 import inputs
    return inputs.exp_spectrum(SPECTRUM_RANK, 50.0)


def make_inputs(a, device):
    """A and an Omega wide enough for the probe (k + 20 columns)."""
    from paper_2110_01011_gb300 import inputs
    A = inputs.low_rank_matrix_torch(a.m, a.n, spectrum(), 1e-6, seed=1002, rank=SPECTRUM_RANK, device=device)
    # BF16-representable, so that every form sketches with the same test matrix
    Om = inputs.omega_torch(a.m, a.k + 20, seed=2002, device=device, bf16_exact=True)
    return A, Om


def tail2(a):
    """sum_{i > k} sigma_i^2 of the workload (the noise floor adds ~1e-12 m)."""
    sig = spectrum()
    return float((sig[a.k:] ** 2).sum()) + 1e-12 * a.m


class Accuracy:
    """Accuracy of a factorisation from its P, evaluated directly in FP64:
    ||A - A P_j P_j^T||_F for the leading j = k columns (the excess rank-k
    error eps = that / (sum_{i>k} sigma_i^2)^(1/2) - 1) and for all d columns
    (relative to ||A||_F). The identity ||A||^2 - ||L||^2 is not used here:
    at a 3e-4 relative tail the rounding of L itself would dominate it."""

    def __init__(self, a, A):
        self.a = a
        self.A64 = A.double()
        self.nA = float(self.A64.norm())

    def resid(self, P, j):
        Pj = P[:, :j].double()
        return float((self.A64 - (self.A64 @ Pj) @ Pj.T).norm())

    def __call__(self, P):
        r_k = self.resid(P, self.a.k)
        return {"excess_error": r_k / tail2(self.a) ** 0.5 - 1.0,
                "rel_residual": self.resid(P, P.shape[1]) / self.nA}


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
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        A = inputs.low_rank_matrix_torch(a.m, a.n, spectrum(), 1e-6, seed=1002, rank=SPECTRUM_RANK, device=dev)
    As = A[:S, :S].double().cpu().numpy()
    Om = inputs.omega(a.m, a.k + 20, seed=2002, bf16_exact=True)[:S, :a.k + a.p].astype(np.float64)
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
    emit(a, line)


# ------------------------------------------------------------------ our arm

def kernel_sha(prec):
    """Hash of the source file that holds the dominant kernel of this precision."""
    f = "gemm_simt.cu" if prec == 0 else "tc_gemm.cu"   # 0: FP32 form
    p = os.path.join(ROOT, "paper_2110_01011_gb300", "csrc", f)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:12]


def traffic_for(kernel, sha):
    """DRAM bytes per launch recorded from an ncu capture of this exact kernel source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    for line in open(TRAFFIC_FILE):
        f = line.split()
        if len(f) >= 3 and f[0] == kernel and f[1] == sha:
            return float(f[2])
    return None


class Ctx:
    """Ranks of one job (one process per GPU; replicas, no data-path
    collective): a barrier that also drains the device, and the maximum of a
    per-rank time over the ranks."""

    def __init__(self, world, rank, dev):
        self.world, self.rank, self.dev = world, rank, dev

    def barrier(self):
        import torch
        import torch.distributed as dist
        if self.world > 1:
            dist.barrier()
        if self.dev.type == "cuda":
            torch.cuda.synchronize(self.dev)

    def max_over_ranks(self, x):
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return x
        t = torch.tensor([x], device=self.dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def time_steps(ctx, fn, steps):
    """ms per step of fn over `steps` calls (CUDA events on the current stream)."""
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.barrier()
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    ctx.barrier()
    return ctx.max_over_ranks(e0.elapsed_time(e1) / steps)


def fixed_runner(a, A, Om, q, p, prec, dev, small_fp64=False, fused=False):
    import torch

    from paper_2110_01011_gb300 import rqlp
    d = a.k + p
    parts = a.parts if prec == rqlp.PREC_BF16X3 else 0
    opts = rqlp._opts(prec, small_fp64, parts=parts, fused=fused)
    ws = torch.empty(rqlp.rqlp_workspace_bytes(a.m, a.n, a.k, p, q, opts) + 256, dtype=torch.uint8, device=dev)
    out = (torch.empty(a.m, d, device=dev), torch.empty(d, d, device=dev), torch.empty(a.n, d, device=dev),
           torch.empty(2, dtype=torch.int32, device=dev), torch.empty(4, dtype=torch.float64, device=dev))
    Omp = Om[:, :d]

    def step():
        rqlp.factor(A, a.k, p, q, Omp, precision=prec, small_fp64=small_fp64, workspace=ws, out=out, parts=parts,
                    fused=fused)
    return step, out


def learned_runner(a, A, Om, params, target, prec, dev):
    import torch

    from paper_2110_01011_gb300 import rqlp
    w = a.k + 20
    nb = rqlp.rqlp_learned_workspace_bytes(a.m, a.n, a.k, rqlp._opts(prec))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    out = (torch.empty(a.m, w, device=dev), torch.empty(w, w, device=dev), torch.empty(a.n, w, device=dev),
           torch.empty(2, dtype=torch.int32, device=dev), torch.empty(4, dtype=torch.float64, device=dev))
    res = {}

    def step():
        Q, L, P, info, diag, qp = rqlp.factor_learned(A, a.k, Om, params, target, precision=prec, workspace=ws,
                                                      out=out)
        res["out"] = (Q, L, P, info, diag)
        res["qp"] = qp
    return step, res


def pass_products(prec, three_part, x_has_low=True):
    """BF16 MMA products per element pair of a split-form pass: six with three
    parts; with two, three (two when X is BF16-exact, e.g. a rounded Omega)."""
    if prec == 0:
        return 1
    if three_part:
        return 6
    return 3 if x_has_low else 2


def three_part_auto(a, p):
    """The library's automatic part count (three when p < 5 or m n <= 2^27)."""
    if a.parts:
        return a.parts == 3
    return p < 5 or a.m * a.n <= (1 << 27)


def roofline(a, recs, d, prec, peaks, dev, three_part, q, ms_step):
    """Roofline of the dominant kernel (the pass over A that takes the most
    time, per launch, against the burst peak: each launch runs alone inside
    the step) and of the whole chain (the slower of A's bytes over HBM and the
    passes' MMA flops at the tensor peak, against the step time)."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    by_tag = {0: [r[0] for r in recs if r[1] == 0], 1: [r[0] for r in recs if r[1] == 1]}
    dom = max(by_tag, key=lambda t: sum(by_tag[t]))
    pass_ms = statistics.mean(by_tag[dom]) if by_tag[dom] else float("nan")
    npad = max(16, -(-d // 16) * 16)
    flops = 2.0 * a.m * a.n * d
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    kname = {0: "pass_AX", 1: "pass_AtX"}[dom]
    sha = kernel_sha(prec)
    hbm = peaks.get("hbm_gbs", 6761.6)
    burst = peaks.get("bf16_tflops", 1889.1)
    sust = peaks.get("bf16_tflops_sustained", 1683.0)
    if prec == rqlp.PREC_FP32:
        peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (pass_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "flops_per_launch": flops}
    else:
        # MMA flops as issued: N = round16(d) columns, products per element pair
        mma = pass_products(prec, three_part) * 2.0 * a.m * a.n * npad
        roof = {"bound": "tensor", "achieved": mma / (pass_ms * 1e-3) / 1e12, "peak": burst,
                "unit": "TFLOP/s", "flops_per_launch": mma,
                "peak_source": "MEASURED_PEAKS bf16_tflops (burst, of measured)",
                "frac_of_sustained": mma / (pass_ms * 1e-3) / 1e12 / sust}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_for(f"{kname}_{'fp32' if prec == 0 else 'bf16x3'}", sha)
    roof["kernel"] = kname
    roof["launch_ms"] = pass_ms
    roof["launches_timed"] = len(by_tag[dom])
    part_bytes = 4 if prec == 0 else (6 if three_part else 4)
    roof["hbm_gbs"] = a.m * a.n * part_bytes / (pass_ms * 1e-3) / 1e9
    roof["hbm_frac_of_measured"] = roof["hbm_gbs"] / hbm
    # the chain: 2q + 2 passes over A
    npass = 2 * q + 2
    chain_bytes = npass * a.m * a.n * part_bytes
    if prec == rqlp.PREC_FP32:
        chain_flops = npass * flops
        t_flops = chain_flops / (roof["peak"] * 1e12)
        peak_name = "derived FP32"
        t_flops_s = t_flops
    else:
        # the sketch multiplies a BF16-exact Omega (two products with two parts)
        chain_flops = (pass_products(prec, three_part, False) + (npass - 1) * pass_products(prec, three_part)) \
            * 2.0 * a.m * a.n * npad
        t_flops = chain_flops / (burst * 1e12)
        t_flops_s = chain_flops / (sust * 1e12)
        peak_name = "measured bf16 burst (sustained beside it)"
    t_bytes = chain_bytes / (hbm * 1e9)
    roof_ms, roof_ms_s = 1e3 * max(t_bytes, t_flops), 1e3 * max(t_bytes, t_flops_s)
    roof["chain"] = {"passes": npass, "A_bytes": chain_bytes, "mma_flops": chain_flops,
                     "roofline_ms": roof_ms, "bound": "hbm" if t_bytes >= t_flops else "tensor",
                     "frac": roof_ms / ms_step, "frac_sustained": roof_ms_s / ms_step, "peak": peak_name}
    return roof, sha


def batched_leg(a, ctx):
    """512 uneven problems (m in [256, 4096], n in [256, 2048], k in [8, 64],
    p = 5, q = 1) as one graph launch after autotuning, with the passes over
    A as grouped BF16x3 tensor-core passes and/or as FP32 products."""
    import torch

    from paper_2110_01011_gb300 import inputs, rqlp
    probs = inputs.random_batch(a.batch, seed=4004)
    t0 = time.perf_counter()
    As = [inputs.low_rank_matrix_reflect(pr.m, pr.n, pr.sigma(), pr.seed, ctx.dev) for pr in probs]
    Os = [inputs.omega_torch(pr.m, pr.d, pr.seed + 1, ctx.dev) for pr in probs]
    gen_s = time.perf_counter() - t0
    q = probs[0].q
    abytes = sum((2 * q + 2) * pr.m * pr.n * 4 for pr in probs)

    def one(prec):
        b = rqlp.Batch(As, Os, [pr.k for pr in probs], [pr.p for pr in probs], q, precision=prec)
        tune = None if a.no_autotune else b.autotune(reps=2)
        for _ in range(max(1, a.warmup)):
            b.launch()
        ctx.barrier()
        l0 = rqlp.rqlp_kernel_launches()
        reps = max(3, a.steps)
        ms = time_steps(ctx, b.launch, reps)
        launches = (rqlp.rqlp_kernel_launches() - l0) // reps
        bad = int((b.info[:, 0] != 0).sum().item())
        res = {"ms_per_batch": ms, "value": ctx.world * abytes / (ms * 1e-3) / 1e9, "unit": "GB/s",
               "problems_per_s": ctx.world * len(probs) / (ms * 1e-3), "graph_kernels": launches, "tuning": tune,
               "nonzero_status": bad}
        # leading-k diagonals of L for the agreement check between the forms
        diags[prec] = [torch.diagonal(b.L[i])[:probs[i].k].double().cpu() for i in range(len(probs))]
        orth = [float(torch.linalg.norm(b.Q[i].double().T @ b.Q[i].double()
                                        - torch.eye(probs[i].d, dtype=torch.float64, device=ctx.dev)))
                for i in range(min(32, len(probs)))]
        res["max_orth_Q_first32"] = max(orth)
        b.close()
        return res

    runs = {}
    diags = {}
    if a.batched_precision in ("both", "bf16x3"):
        runs["bf16x3"] = one(rqlp.PREC_BF16X3)
    if a.batched_precision in ("both", "fp32"):
        runs["fp32"] = one(rqlp.PREC_FP32)
    head = "bf16x3" if "bf16x3" in runs else "fp32"
    out = dict(runs[head])
    if len(diags) == 2:
        # Parity with the FP64 oracle is a GPU test (the bench's first 32
        # problems); here the two forms are checked against each other.
        rel = [float(((diags[1][i] - diags[0][i]).abs() / diags[0][i].abs()).max()) for i in range(len(probs))]
        out["agreement"] = {"max_rel_Lii_diff_bf16x3_vs_fp32": max(rel),
                            "median_rel_Lii_diff": statistics.median(rel), "problems": len(rel)}
    out.update({"problems": len(probs), "A_bytes_per_batch": abytes, "generate_s": gen_s, "precision": head,
                "workload": f"{len(probs)} problems, m in [256,4096], n in [256,2048], k in [8,64], p=5, q={q}, "
                            "half exp / half poly spectra"})
    if head == "bf16x3" and "fp32" in runs:
        out["fp32"] = runs["fp32"]
        out["speedup_vs_fp32"] = runs["fp32"]["ms_per_batch"] / runs["bf16x3"]["ms_per_batch"]
    del As, Os
    torch.cuda.empty_cache()
    return out


def h2d_copy_gbs(hA, dev):
    """Pinned host-to-device copy rate of A alone on this machine (GB/s, CUDA
    events around three plain copies): the floor that the end-to-end call's
    copy of A cannot beat, reported beside its time."""
    import torch
    dst = torch.empty(hA.shape, dtype=hA.dtype, device=dev)
    dst.copy_(hA, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        dst.copy_(hA, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    del dst
    return hA.numel() * hA.element_size() / ms / 1e6


def e2e_learned(a, ctx, A, Om, params, target, prec, steps, warmup):
    """End to end through the public C ABI with host buffers:
    rqlp_factor_learned_host takes pinned host A and Omega, copies A by row
    blocks while the probe sketch runs on the blocks that have landed, factors,
    and copies Q, L, P back, every step."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    w = a.k + 20
    hA, hO = A.cpu().pin_memory(), Om.cpu().pin_memory()
    out = (torch.empty(a.m, w).pin_memory(), torch.empty(w, w).pin_memory(), torch.empty(a.n, w).pin_memory(),
           torch.zeros(2, dtype=torch.int32), torch.zeros(4, dtype=torch.float64))
    nb = rqlp.rqlp_learned_host_workspace_bytes(a.m, a.n, a.k, rqlp._opts(prec))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=ctx.dev)
    qp = None
    for _ in range(max(1, warmup)):
        qp = rqlp.factor_learned_host(hA, a.k, hO, params, target, precision=prec, workspace=ws, out=out)[5]
    ctx.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        qp = rqlp.factor_learned_host(hA, a.k, hO, params, target, precision=prec, workspace=ws, out=out)[5]
    ctx.barrier()
    dt = ctx.max_over_ranks((time.perf_counter() - t0) / steps)
    d = a.k + qp[1]
    h2d = 4 * (a.m * a.n + a.m * w)
    d2h = 4 * (a.m * d + d * d + a.n * d) + 8 + 32 + 8
    return {"value": ctx.world * (2 * qp[0] + 2) * a.m * a.n * 4 / dt / 1e9, "unit": "GB/s", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "qp": list(qp),
            "api": "rqlp_factor_learned_host", "h2d_copy_gbs": h2d_copy_gbs(hA, ctx.dev)}


def e2e_fixed(a, ctx, A, Om, q, p, prec, steps, warmup):
    import torch

    from paper_2110_01011_gb300 import rqlp
    d = a.k + p
    hA = A.cpu().pin_memory()
    hO = Om[:, :d].contiguous().cpu().pin_memory()
    hout = (torch.empty(a.m, d).pin_memory(), torch.empty(d, d).pin_memory(), torch.empty(a.n, d).pin_memory(),
            torch.zeros(2, dtype=torch.int32), torch.zeros(4, dtype=torch.float64))
    hws = torch.empty(rqlp.rqlp_host_workspace_bytes(a.m, a.n, a.k, p, q, rqlp._opts(prec)) + 256,
                      dtype=torch.uint8, device=ctx.dev)
    for _ in range(max(1, warmup)):
        rqlp.factor_host(hA, a.k, p, q, hO, precision=prec, workspace=hws, out=hout)
    ctx.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        rqlp.factor_host(hA, a.k, p, q, hO, precision=prec, workspace=hws, out=hout)
    ctx.barrier()
    dt = ctx.max_over_ranks((time.perf_counter() - t0) / steps)
    return {"value": ctx.world * (2 * q + 2) * a.m * a.n * 4 / dt / 1e9, "unit": "GB/s", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": 4 * (a.m * a.n + a.m * d),
            "d2h_bytes_per_step": 4 * (a.m * d + d * d + a.n * d) + 8 + 32, "api": "rqlp_factor_host",
            "h2d_copy_gbs": h2d_copy_gbs(hA, ctx.dev)}


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    from paper_2110_01011_gb300 import learn, rqlp
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    ctx = Ctx(world, rank, dev)
    rqlp.load()
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    if a.form == "batched":
        ck = ClockSampler(local)
        bt = batched_leg(a, ctx)
        clocks = ck.stop()
        if rank == 0:
            line = {"metric": "batched Rand-QLP A-pass GB/s", "value": bt["value"], "unit": "GB/s", "n_gpus": world,
                    "steps": max(3, a.steps), "warmup": max(1, a.warmup), "ms_per_step": bt["ms_per_batch"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "bf16x3" if bt["precision"] == "bf16x3" else "f32",
                    "data": "synthetic", "config": {"workload": bt["workload"], "l2": "inputs larger than L2"},
                    "clocks": clocks, "batched": bt}
            emit(a, line)
        if world > 1:
            dist.destroy_process_group()
        return
    A, Om = make_inputs(a, dev)

    params = None
    learned_note = None
    if a.form == "learned":
        if os.path.exists(learn.WEIGHTS):
            params = torch.from_numpy(learn.load_weights()).to(dev)
        else:
            learned_note = "no trained weights in the package: fixed (q, p) timed instead"
    form = "learned" if params is not None else "fixed"

    compare = {}
    acc = Accuracy(a, A)
    # The plain FP32 form with the fixed (2, 10): its time and the accuracy the
    # learned form is asked to match.
    target = None
    if (form == "learned" and a.target is None) or (form == "fixed" and not a.no_compare and a.precision != "fp32"):
        step32, out32 = fixed_runner(a, A, Om, 2 if form == "learned" else a.q, 10 if form == "learned" else a.p,
                                     rqlp.PREC_FP32, dev)
        step32()
        ctx.barrier()
        ms32 = time_steps(ctx, step32, 3)
        acc32 = acc(out32[2])
        compare.update({"fp32_fixed_qp": [2, 10] if form == "learned" else [a.q, a.p], "fp32_ms_per_step": ms32,
                        "fp32_rel_residual": acc32["rel_residual"], "fp32_excess_error": acc32["excess_error"]})
        target = min(max(acc32["excess_error"], 1e-3), 0.5)
        del out32, step32
        torch.cuda.empty_cache()
    if form == "learned" and a.target is not None:
        target = a.target

    prec = rqlp.PREC_BF16X3
    if form == "fixed":
        prec = {"fp32": rqlp.PREC_FP32, "bf16x3": rqlp.PREC_BF16X3}.get(a.precision, rqlp.PREC_BF16X3)
        step, out = fixed_runner(a, A, Om, a.q, a.p, prec, dev)
        res = None
        q_used, p_used = a.q, a.p
    else:
        step, res = learned_runner(a, A, Om, params, target, prec, dev)

    for _ in range(a.warmup):
        step()
    ctx.barrier()
    if res is not None:
        q_used, p_used = res["qp"]
        out = res["out"]
    status = int(out[3][0].item())
    rqlp.rqlp_profile_read()          # drop records from the warm-up
    rqlp.rqlp_profile_enable(True)
    clocks = ClockSampler(local)
    l0 = rqlp.rqlp_kernel_launches()
    ms_step = time_steps(ctx, step, a.steps)
    launches = rqlp.rqlp_kernel_launches() - l0
    rqlp.rqlp_profile_enable(False)
    ck = clocks.stop()
    recs = rqlp.rqlp_profile_read()
    if res is not None:
        q_used, p_used = res["qp"]
        out = res["out"]
    d = a.k + p_used
    abytes = (2 * q_used + 2) * a.m * a.n * 4
    value = world * abytes / (ms_step * 1e-3) / 1e9
    roof, sha = roofline(a, recs, d, prec, peaks, dev, prec == rqlp.PREC_BF16X3 and three_part_auto(a, p_used),
                         q_used, ms_step)

    compare.update({"form": ("learned_" if form == "learned" else "fixed_") + ("fp32" if prec == 0 else "bf16x3"),
                    "qp": [q_used, p_used], **acc(out[2])})
    if target is not None:
        compare["requested_excess_error"] = target
    if "fp32_ms_per_step" in compare:
        compare["speedup_vs_fp32"] = compare["fp32_ms_per_step"] / ms_step
    if form == "learned" and not a.no_compare:
        # the split form with the fixed (2, 10): what the prediction changed
        s16, o16 = fixed_runner(a, A, Om, 2, 10, rqlp.PREC_BF16X3, dev)
        s16()
        ctx.barrier()
        compare["bf16x3_fixed_ms_per_step"] = time_steps(ctx, s16, 3)
        acc16 = acc(o16[2])
        compare["bf16x3_fixed_excess_error"] = acc16["excess_error"]
        compare["bf16x3_fixed_rel_residual"] = acc16["rel_residual"]
        del s16, o16
        torch.cuda.empty_cache()
        # FP64 d x d factors (Cholesky and the QR of R^T) on the same split form
        s64, o64 = fixed_runner(a, A, Om, 2, 10, rqlp.PREC_BF16X3, dev, small_fp64=True)
        s64()
        ctx.barrier()
        compare["bf16x3_fixed_small_fp64_ms_per_step"] = time_steps(ctx, s64, 3)
        del s64, o64
        torch.cuda.empty_cache()
        # power passes fused as A^T (A P~) over L2-sized row panels
        sfu, ofu = fixed_runner(a, A, Om, 2, 10, rqlp.PREC_BF16X3, dev, fused=True)
        sfu()
        ctx.barrier()
        compare["bf16x3_fixed_fused_power_ms_per_step"] = time_steps(ctx, sfu, 3)
        compare["bf16x3_fixed_fused_power_excess_error"] = acc(ofu[2])["excess_error"]
        del sfu, ofu
        torch.cuda.empty_cache()
        # the bench matrix's excess errors for every (q, p) (one width-(k + 20)
        # FP32 chain, FP64 residuals) and the network's picks across requests
        tab = learn.eps_table(A, Om, a.k, tail2(a))
        compare["eps_table"] = {f"q{q_}_p{p_}": float(tab[qi][pi]) for qi, q_ in enumerate(learn.Q_CHOICES)
                                for pi, p_ in enumerate(learn.P_CHOICES)}
        sweep = []
        for t in sorted({0.1, 0.05, 0.03, float(target), 0.015, 0.01}, reverse=True):
            stp, rs = learned_runner(a, A, Om, params, t, prec, dev)
            stp()
            ctx.barrier()
            ms_t = time_steps(ctx, stp, 3)
            qt, pt = rs["qp"]
            bq, bp = learn.label_from_table(tab, a.k, t)
            sweep.append({"request": t, "qp": [qt, pt], "table_eps": float(tab[learn.Q_CHOICES.index(qt)]
                                                                           [learn.P_CHOICES.index(pt)]),
                          "ms_per_step": ms_t, "cheapest_feasible": [learn.Q_CHOICES[bq], learn.P_CHOICES[bp]]
                          if tab[bq][bp] <= t else None})
            del stp, rs
        compare["request_sweep"] = sweep
        torch.cuda.empty_cache()
    if learned_note:
        compare["learned"] = learned_note

    e2e = None
    if not a.no_e2e:
        torch.cuda.empty_cache()
        if form == "learned":
            e2e = e2e_learned(a, ctx, A, Om, params, target, prec, a.steps, a.warmup)
        else:
            e2e = e2e_fixed(a, ctx, A, Om, a.q, a.p, prec, a.steps, a.warmup)

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        S = a.sample or 4000
        import argparse as _ap
        ao = _ap.Namespace(**vars(a))
        ao.q, ao.p = q_used, p_used
        gbs, dt, cores = oracle_time(ao, *oracle_inputs(ao, S, A))
        cpu = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle chain on the leading {S}x{S} block of the workload's A "
                         f"(q={q_used}, d={d}), {dt:.1f} s"}

    del A, Om, acc
    torch.cuda.empty_cache()
    batched = None if a.no_batched else batched_leg(a, ctx)

    if rank == 0:
        ao = argparse.Namespace(**vars(a))
        ao.q, ao.p = q_used, p_used
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == rqlp.PREC_FP32 else "bf16x3",
                "data": "synthetic",
                "config": {"workload": workload_name(ao), "m": a.m, "n": a.n, "k": a.k, "p": p_used, "q": q_used,
                           "form": compare["form"], "A_bytes_per_step": abytes,
                           "l2": "inputs larger than L2 (A is %.1f GB)" % (a.m * a.n * 4 / 1e9),
                           "parallelism": "replicas" if world > 1 else "single"},
                "status": status, "clocks": ck, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "compare": compare, "batched": batched,
                "gpu_launches": launches, "kernel_sha": sha}
        emit(a, line)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
