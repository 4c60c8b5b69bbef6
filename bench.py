#!/usr/bin/env python
"""Benchmark of the 4D HOTRG coarse-graining step (arXiv:1906.06060, Sec. 2) on GB300.

Workload: 4D Ising, beta = 0.1497, h = 0, Dcut = 10 (the 40-step flow to 1024^4). A bench
"step" is one coarse-graining step of the whole path (Gram matrices, eigensolver, operand
construction, squeeze GEMM, epilogue, norm/ln accumulation). W warm-up steps (W >= 3 reaches
the steady-state bond dimensions 10^4) run untimed, then K steady-state steps are timed with CUDA
events on the library's stream. Metric: algorithmic TFLOP/s of the squeeze (2 prod(chi_b) P^3
per step = 2 Dcut^15 at steady state; split-precision extra passes are not counted).

At h = 0 the squeeze runs block-sparse by default (opts.z2: the spin-flip parity structure leaves
two dense GEMM blocks per chunk, about a quarter of the flops; --no-z2 for the dense squeeze).
"value" keeps the chi-rule count above as the unit of work in both cases; "executed_tflops" is
what the kernels computed.

Default precision schedule (|delta f / f| = 2.2e-8 against the FP64 GPU path after 8 steps at
Dcut = 10): steps 1-3 in FP64, steps 4-6 in BF16X6, then FP16X3 (fp16 hi + lo planes of power-of-two
scaled operands, three products). With the default W = 12 the timed steps are FP16X3 steps; with
W = 3 the first three are BF16X6 steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp16x3|bf16x3|bf16x6|fp64 ...]
    python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample

Other workloads of the same path (same JSON line; e2e and the CPU baseline only for the default):
    --workload scan    batched temperature scan: beta in linspace(0.1490, 0.1505, n) x h in {0, 1e-5}
                       (2n instances, default n = 64), Dcut = 8, one context, graph-captured steps
    --workload deriv   d lnZ/d beta and d lnZ/d h through the eigendecomposition: beta in
                       linspace(0.1494, 0.1500, n) (default n = 16), h = 1e-6, Dcut = 10
    --instances n      fewer instances of a scan / deriv workload (a bounded sample of it)
    --workload accuracy  per-step |delta(lnZ/N)| / |lnZ/N| of split-precision schedules against the
                       FP64 GPU flow (--ref-steps of it, timed step by step) and the oracle's golden
    --workload gemm    the tcgen05 squeeze GEMM alone (--gemm-shape M,N,K --npass)
    --workload phase   X^(n) flows at the temperatures --temps (h = 0), classified ordered /
                       disordered (Sec. 3: T_c(Dcut = 13) = 6.650365(5) on 1024^4)

Multi-GPU (torchrun, one process per GPU): the single-flow workload does not shard, so each rank
runs an independent replica; value = total flops of all ranks / max time over ranks.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4D HOTRG TFLOP/s & % tensor peak at Dcut=10, mixed vs FP64, |Δf/f|≤1e-7"
GEMM_SRC = os.path.join(ROOT, "paper_1906_06060_gb300", "csrc", "gemm_tc.cu")
# committed ncu summaries of the Dcut = 10 BF16X3 squeeze GEMM: dense and block-sparse launches
PROFILE = {False: os.path.join(ROOT, "profiles", "ncu_squeeze_gemm_dcut10_summary.md"),
           True: os.path.join(ROOT, "profiles", "ncu_squeeze_gemm_z2_dcut10_summary.md")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=12)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16x3",
                    choices=["bf16x3", "bf16x4", "bf16x6", "fp16x3", "fp16x4", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--kblock", type=int, default=64)
    ap.add_argument("--fold-group", type=int, default=0)
    ap.add_argument("--cta-group", type=int, default=0, choices=[0, 1, 2],
                    help="CTAs per squeeze-GEMM output tile: 2 = CTA pairs (256 x 256 tiles), 1 = single CTAs "
                         "(128 x 256); 0 = the library default (pairs for the block-sparse squeeze), autotuned")
    ap.add_argument("--x6-steps", type=int, default=6)
    ap.add_argument("--workload", default="flow", choices=["flow", "scan", "deriv", "accuracy", "gemm", "phase"])
    ap.add_argument("--temps", default="6.650355,6.650375",
                    help="phase workload: temperatures T = 1/beta of the X^(n) flows (h = 0)")
    ap.add_argument("--gemm-shape", default="10000,40000,10000",
                    help="gemm workload: M,N,K of the squeeze GEMM alone (default: a quarter of one Dcut=10 chunk)")
    ap.add_argument("--npass", type=int, default=3, help="gemm workload: split products (1, 3, 4 or 6)")
    ap.add_argument("--ref-steps", type=int, default=8,
                    help="accuracy workload: steps of the FP64 GPU reference flow (0: read the committed one)")
    ap.add_argument("--flow-steps", type=int, default=40, help="accuracy workload: steps of each split flow")
    ap.add_argument("--schedules", default="fp16x3:3:6,bf16x3:3:12,bf16x3:3:0,bf16x6:3:0,fp16x3:3:0,fp16x4:3:0",
                    help="accuracy workload: precision:fp64_steps:x6_steps of each split flow")
    ap.add_argument("--instances", type=int, default=0)
    ap.add_argument("--group", type=int, default=0,
                    help="instances per squeeze GEMM launch (0: for a scan the largest of 64, 32, 16, 8 "
                         "whose workspaces fit 80%% of the free device memory, else the library default)")
    ap.add_argument("--dcut", type=int, default=0)
    ap.add_argument("--beta", type=float, default=0.1497)
    ap.add_argument("--h", type=float, default=0.0)
    ap.add_argument("--no-z2", action="store_true",
                    help="dense squeeze at h = 0 (default: the zero-field block-sparse squeeze)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default GEMM tile configuration (default: autotune after the warm-up steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-slices", type=int, default=2)
    ap.add_argument("--log-jsonl", default="",
                    help="flow workload: write one JSON record per step of the e2e flow to this file")
    a = ap.parse_args()
    if not a.dcut:
        a.dcut = 8 if a.workload == "scan" else 10
    return a


def instances(a):
    """(betas, hs) of the workload's instances."""
    import numpy as np
    if a.workload == "scan":
        n = a.instances or 64
        b = [float(x) for x in np.linspace(0.1490, 0.1505, n)]
        return b + b, [0.0] * n + [1e-5] * n
    if a.workload == "deriv":
        n = a.instances or 16
        return [float(x) for x in np.linspace(0.1494, 0.1500, n)], [1e-6] * n
    return [a.beta], [a.h]


def use_z2(a):
    """The zero-field block-sparse squeeze applies to instances with h = 0 when no derivative in
    h is taken (a scan puts its h = 0 instances into a block-sparse context of their own)."""
    _, hs = instances(a)
    return (not a.no_z2) and a.workload != "deriv" and any(h == 0.0 for h in hs)


def groups(a):
    """(betas, hs, z2) of the contexts that run the workload's instances."""
    betas, hs = instances(a)
    if not use_z2(a):
        return [(betas, hs, False)]
    zero = [i for i, h in enumerate(hs) if h == 0.0]
    rest = [i for i, h in enumerate(hs) if h != 0.0]
    out = [([betas[i] for i in zero], [0.0] * len(zero), True)]
    if rest:
        out.append(([betas[i] for i in rest], [hs[i] for i in rest], False))
    return out


def workload_config(a):
    betas, hs = instances(a)
    if a.workload == "scan":
        what = (f"4D Ising HOTRG batched temperature scan: {len(betas)} instances (beta in "
                f"linspace(0.1490, 0.1505, {len(betas) // 2}) x h in {{0, 1e-5}}), Dcut={a.dcut}: steady-state "
                f"steps of the 40-step flows to 1024^4, one context, graph-captured steps")
    elif a.workload == "deriv":
        what = (f"4D Ising HOTRG with d lnZ/d beta and d lnZ/d h through the eigendecomposition: "
                f"{len(betas)} instances (beta in linspace(0.1494, 0.1500, {len(betas)}), h = 1e-6), "
                f"Dcut={a.dcut}: steady-state steps of the 40-step flow to 1024^4; flops counted: forward "
                f"squeeze + two tangent contractions over a doubled k range (5x the forward)")
    else:
        what = (f"4D Ising HOTRG, beta={a.beta}, h={a.h}, Dcut={a.dcut}: steady-state "
                f"coarse-graining steps (bond dims {a.dcut}^4) of the 40-step flow to 1024^4")
    return {"workload": what, "instances": len(betas),
            "d": 4, "Dcut": a.dcut, "beta": a.beta if len(betas) == 1 else [min(betas), max(betas)],
            "h": a.h if len(hs) == 1 else sorted(set(hs)), "precision": a.precision,
            "timed_steps": [a.warmup + 1, a.warmup + a.steps],
            "fp64_steps": a.fp64_steps, "x6_steps": a.x6_steps, "kblock": a.kblock,
            "z2_block_sparse": use_z2(a),
            "contexts": [{"instances": len(g[0]), "z2": g[2]} for g in groups(a)],
            "fold_group": a.fold_group, "cta_group": a.cta_group,
            "l2": "inputs larger than L2 (T 800 MB fp64, GEMM operands several GB per step)",
            "parallelism": "replicas" if a.gpus > 1 else "single GPU"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def steady_flops(dcut):
    return 2.0 * float(dcut) ** 15


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(dcut, slices):
    """Time the FP64 oracle's squeeze on `slices` slices of a steady-state step (random T with
    bond dims dcut^4 and random orthonormal isometries: the cost does not depend on the values).
    Returns (seconds, algorithmic flops)."""
    import numpy as np
    from oracle import hotrg_ref as R
    rng = np.random.default_rng(0)
    D = dcut
    T = rng.standard_normal((D,) * 8)
    T /= np.linalg.norm(T)
    U = {}
    for b in (1, 2, 3):
        q, _ = np.linalg.qr(rng.standard_normal((D * D, D)))
        U[b] = q.reshape(D, D, D)
    t0 = time.perf_counter()
    R.squeeze(T, T, 0, U, max_slices=slices)
    dt = time.perf_counter() - t0
    return dt, slices * 2.0 * float(D) ** 12


def cpu_threads():
    return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)


def run_reference(a, rank, world):
    if rank != 0:
        return None
    for _ in range(a.warmup):
        oracle_sample(a.dcut, a.cpu_slices)
    times, flops = [], 0.0
    for _ in range(a.steps):
        dt, f = oracle_sample(a.dcut, a.cpu_slices)
        times.append(dt)
        flops += f
    total = sum(times)
    value = flops / total / 1e12
    sample = (f"{a.cpu_slices} slice(s) of one steady-state Dcut={a.dcut} squeeze per step "
              f"(2 Dcut^12 flops each), oracle/hotrg_ref.py squeeze(), FP64 NumPy/BLAS")
    return {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(a),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- GPU arm
def effective_cta_group(a, tuned):
    """CTAs per squeeze-GEMM tile in the timed steps: the autotuner's choice, else --cta-group,
    else the library default (pairs for the block-sparse squeeze)."""
    for t in tuned or []:
        if isinstance(t, dict) and "cta_group" in t:
            return int(t["cta_group"])
    return a.cta_group or (2 if use_z2(a) else 1)


def traffic_from_profile(z2, cta_group):
    """Per-launch DRAM bytes of the squeeze GEMM (dense or block-sparse launch) from the
    committed ncu summary, valid only if the kernel source is unchanged since the capture and the
    launch uses the capture's CTA group (pairs and single CTAs move different bytes)."""
    try:
        with open(PROFILE[bool(z2)]) as fh:
            text = fh.read()
    except OSError:
        return None
    with open(GEMM_SRC, "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()[:16]
    kv = {}
    for line in text.splitlines():
        if "=" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("gemm_tc_sha") != sha or kv.get("cta_group", "1") != str(cta_group):
        return None
    try:
        return float(kv["traffic_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def over_ranks(dist, ms, flops, executed, device):
    """Whole-job figures of a replica run: the slowest rank's time and every rank's flops summed
    (the replicas run independent flows; this is the only collective, outside the timed region)."""
    if dist is None:
        return ms, flops, executed
    import torch
    buf = torch.tensor([ms, flops, executed], dtype=torch.float64, device=device)
    mx = buf.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = buf.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def squeeze_group(a, torch=None):
    """Instances per squeeze GEMM launch: --group, or for a scan the largest of 64, 32, 16, 8 whose
    contexts' workspaces together fit in 80 % of the free device memory."""
    if a.group > 0 or a.workload != "scan":
        return a.group
    from paper_1906_06060_gb300 import workspace_bytes
    free = torch.cuda.mem_get_info()[0] if torch is not None else float("inf")
    for g in (64, 32, 16, 8):
        need = sum(workspace_bytes(4, a.dcut, a.precision, len(b), a.fp64_steps, x6_steps=a.x6_steps, z2=z2,
                                   group=g) for b, _, z2 in groups(a))
        if need <= 0.8 * free:
            return g
    return 1


def run_ours(a, rank, world, dist):
    import torch
    from paper_1906_06060_gb300 import HOTRG
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    kw = dict(precision=a.precision, fp64_steps=a.fp64_steps, x6_steps=a.x6_steps, kblock=a.kblock, fold_group=a.fold_group,
              cta_group=a.cta_group, stream=stream)

    def barrier():
        if dist:
            dist.barrier()

    if a.workload == "deriv":
        kw["derivatives"] = "eig"
    kw["group"] = squeeze_group(a, torch)
    # one context per group (a scan's h = 0 instances run block-sparse in a context of their own);
    # all contexts step on the same stream, one after the other
    flows = [HOTRG(4, b, h, a.dcut, z2=z2, **kw) for b, h, z2 in groups(a)]
    for _ in range(a.warmup):
        for flow in flows:
            flow.step()
    for flow in flows:
        flow.free_energy()
    # the squeeze GEMM's tile configuration for the steady shape, picked by the library's
    # autotuner on the last warm-up step's operands (outside the timed region)
    tuned = []
    # only when the last warm-up step ran the GEMM the timed steps run (a two-plane split step)
    if not a.no_autotune and a.precision != "fp64" and a.warmup > max(a.fp64_steps, a.x6_steps):
        for flow in flows:
            try:
                tuned.append(flow.autotune())
            except Exception as exc:  # the last warm-up step ran in FP64: nothing to tune
                tuned.append({"skipped": str(exc)})
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    for flow in flows:
        flow.timing_start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        ev0.record(stream)
        for _ in range(a.steps):
            for flow in flows:
                flow.step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ts = [flow.timing_stop() for flow in flows]
    t = {k: sum(x[k] for x in ts) for k in ts[0]}
    ms = ev0.elapsed_time(ev1)
    lnz = flows[0].free_energy()[0][0]
    flow_obs = [flows[0].observables(i) for i in range(flows[0].batch)] if a.workload == "deriv" else []
    for flow in flows:
        flow.close()
    # unit of work: the chi-rule count 2 prod(chi_b) P^3 per step and instance (also with the
    # block-sparse squeeze, which computes about a quarter of it: reported as executed_*)
    step_flops = t["dense_step_flops"] * (5.0 if a.workload == "deriv" else 1.0)
    executed_flops = t["step_flops"] * (5.0 if a.workload == "deriv" else 1.0)
    ms_max, flops_all, exec_all = over_ranks(dist, ms, step_flops, executed_flops, dev)
    if rank != 0:
        return None
    value = flops_all / (ms_max * 1e-3) / 1e12
    pk, src = peaks()
    gemm_ms = t["ms_gemm"] / max(1, t["gemm_launches"])
    achieved = (t["gemm_flops"] / max(1, t["gemm_launches"])) / (gemm_ms * 1e-3) / 1e12
    peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            # the committed ncu summaries are of the steady-step three-product GEMM (fp16 and bf16
            # planes move the same bytes), scaled to Dcut = 10
            "traffic": (traffic_from_profile(use_z2(a), effective_cta_group(a, tuned))
                        if (a.workload == "flow" and a.dcut == 10 and a.precision in ("bf16x3", "fp16x3"))
                        else None),
            "peak_source": f"{src} bf16 sustained (kernel timed inside long steps)",
            "kernel": "k_gemm_split (tcgen05 squeeze GEMM)" if a.precision != "fp64" else "k_gemm_f64",
            "tensor_pipe_tflops": (t["gemm_tensor_flops"] / max(1, t["gemm_launches"])) / (gemm_ms * 1e-3) / 1e12,
            "note": "achieved counts the algorithmic flops the GEMM launches execute (2MNK; with the "
                    "block-sparse squeeze only its two blocks per chunk); the split passes multiply tensor "
                    "work by 3 (bf16x3) or 6 (bf16x6)"}
    if a.precision == "fp64":
        # the FMA-chain microbenchmark measures less than the FP64 GEMM itself sustains (1.06 against
        # 1.248 TFLOP/s at Dcut = 10), so the nominal rate is the tighter bound; both are reported
        from paper_1906_06060_gb300 import fp64_fma_tflops
        roof.update({"bound": "alu", "peak": 1.25, "peak_source": "nominal GB300 FP64 rate",
                     "frac": achieved / 1.25, "fp64_fma_microbenchmark_tflops": fp64_fma_tflops()})
    if a.workload == "deriv":
        o = [flow_obs[i] for i in range(len(flow_obs))]
        extra = {"internal_energy": [x["internal_energy"] for x in o], "magnetization": [x["magnetization"] for x in o]}
    else:
        extra = {}
    out = {"metric": METRIC, "value": value, "unit": "TFLOP/s",
           "value_basis": "dense-equivalent: the chi-rule count 2 prod(chi_b) P^3 per step (2 Dcut^15 at steady "
                          "state) whether or not the block-sparse squeeze skips its zero blocks; executed_tflops "
                          "is what the kernels computed (about a quarter of it at h = 0)",
           "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None,
           # the squeeze's operand type in the timed steps (split into hi + lo planes, FP32 accumulation;
           # Gram matrices, eigensolver, norms and ln sums in FP64)
           "dtype": "f64" if a.precision == "fp64" else ("fp16" if a.precision.startswith("fp16") else "bf16"),
           "data": "synthetic", "config": workload_config(a),
           "steps_per_s": a.steps / (ms_max * 1e-3), "roofline": roof,
           "executed_tflops": exec_all / (ms_max * 1e-3) / 1e12,
           "executed_flops_fraction": exec_all / flops_all if flops_all else None,
           "phases_ms_per_step": {k[3:]: v / a.steps for k, v in t.items() if k.startswith("ms_")},
           "gpu_launches": int(t["kernel_launches"]), "lnz_per_site_after": lnz, **extra}
    out["config"]["squeeze_group"] = kw["group"] or "library default (up to 8)"
    out["config"]["autotune"] = tuned or "off"
    out["clocks"] = clk.summary()
    return out



# ----------------------------------------------------------------------------- accuracy workload
ACCURACY_PROFILE = os.path.join(ROOT, "profiles", "accuracy_fp64_vs_split_dcut10.md")
ORACLE_GOLDEN_D10 = os.path.join(ROOT, "tests", "golden", "flow_d4_b0.1497_h0_D10_n4.json")


def stored_fp64_reference(path=None):
    """Per-step ln Z/N of the FP64 GPU flow recorded in the committed accuracy summary
    ("- fp64_lnz_step_<n> = <value>" lines), or {} if there is none."""
    path = path or ACCURACY_PROFILE
    out = {}
    try:
        with open(path) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith("- fp64_lnz_step_") and "=" in line:
                    k, v = line[2:].split("=", 1)
                    out[int(k.strip()[len("fp64_lnz_step_"):])] = float(v)
    except (OSError, ValueError):
        return {}
    return out


def oracle_golden_lnz(path=None):
    """Per-step ln Z/N of the FP64 oracle's Dcut = 10 flow (tests/golden, written by the oracle)."""
    path = path or ORACLE_GOLDEN_D10
    try:
        with open(path) as fh:
            g = json.load(fh)
    except (OSError, ValueError):
        return {}
    return {st["step"]: st["lnz"] for st in g["steps"]}


def run_accuracy(a):
    """|delta(ln Z/N)| / |ln Z/N| of split-precision schedules against the FP64 GPU path after every
    step (4D, h = 0, both block-sparse; --no-z2 for dense), with the FP64 steps timed one by one."""
    import torch
    from paper_1906_06060_gb300 import HOTRG, fp64_fma_tflops
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    z2 = use_z2(a)
    out = {"workload": "accuracy", "d": 4, "beta": a.beta, "h": a.h, "Dcut": a.dcut, "z2_block_sparse": z2}
    out["fp64_fma_tflops"] = fp64_fma_tflops(stream=stream)
    ref, ref_src = {}, None
    if a.ref_steps > 0:
        steps = []
        # the workspace plan covers only the states these steps reach (Dcut = 13 in FP64 would
        # otherwise plan steady-state FP64 buffers of about 100 GB)
        with HOTRG(4, a.beta, a.h, a.dcut, precision="fp64", z2=z2, stream=stream, graphs=False,
                   max_steps=a.ref_steps) as f:
            for n in range(1, a.ref_steps + 1):
                f.timing_start()
                f.step()
                t = f.timing_stop()
                lnz = float(f.free_energy()[0][0])
                ob = f.observables()
                ref[n] = lnz
                steps.append({"step": n, "lnz": lnz, "ln_c": ob["last_ln_c"], "x": ob["x_indicator"],
                              "ms": t["ms_step"], "ms_gemm": t["ms_gemm"], "gemm_flops": t["gemm_flops"],
                              "dense_flops": t["dense_step_flops"]})
                print(json.dumps({"fp64_step": steps[-1]}), file=sys.stderr, flush=True)
        out["fp64_steps"] = steps
        ref_src = "FP64 GPU flow of this run"
    else:
        ref = stored_fp64_reference()
        ref_src = f"FP64 GPU flow recorded in {os.path.relpath(ACCURACY_PROFILE, ROOT)}"
    oracle = oracle_golden_lnz() if (a.dcut == 10 and a.beta == 0.1497 and a.h == 0.0) else {}
    out["reference"] = ref_src
    out["fp64_vs_oracle"] = {str(n): abs(ref[n] - v) / abs(v) for n, v in oracle.items() if n in ref}
    sched = []
    for spec in [x for x in a.schedules.split(",") if x]:
        prec, f64, x6 = spec.split(":")
        lnzs = []
        t0 = time.perf_counter()
        with HOTRG(4, a.beta, a.h, a.dcut, precision=prec, fp64_steps=int(f64), x6_steps=int(x6), z2=z2,
                   stream=stream, max_steps=a.flow_steps) as f:
            for _ in range(a.flow_steps):
                f.step()
                lnzs.append(float(f.free_energy()[0][0]))
            lnc = [float(x) for x in f.ln_norms()]
        wall = time.perf_counter() - t0
        rel = {str(n): abs(lnzs[n - 1] - v) / abs(v) for n, v in ref.items() if n <= len(lnzs)}
        rel_o = {str(n): abs(lnzs[n - 1] - v) / abs(v) for n, v in oracle.items() if n <= len(lnzs)}
        sched.append({"precision": prec, "fp64_steps": int(f64), "x6_steps": int(x6), "wall_s": wall,
                      "lnz": lnzs, "ln_c": lnc, "rel_err_vs_fp64": rel, "rel_err_vs_oracle": rel_o})
        print(json.dumps({"schedule": spec, "rel_err_vs_fp64": rel, "wall_s": wall}), file=sys.stderr, flush=True)
    out["schedules"] = sched
    return out


# ----------------------------------------------------------------------------- GEMM alone
def run_gemm(a):
    """The tcgen05 squeeze GEMM alone through the C ABI (hotrg_gemm_split) on seeded Gaussian
    operands: one warm-up launch (it also splits the FP32 operands into bf16 planes), then K timed
    launches with CUDA events. The default shape is a quarter of one Dcut = 10 chunk's N range
    (M = P = 10^4, N = 4 x 10^4, K = 10^4: 3.6 GB of operands and output, larger than L2)."""
    import torch
    from ctypes import c_void_p
    from paper_1906_06060_gb300 import _lib
    from paper_1906_06060_gb300._lib import check
    M, N, K = (int(x) for x in a.gemm_shape.split(","))
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g = torch.Generator(device=dev).manual_seed(0)
    A = torch.randn((M, K), device=dev, generator=g, dtype=torch.float32)
    Bt = torch.randn((N, K), device=dev, generator=g, dtype=torch.float32)
    C = torch.empty((M, N), device=dev, dtype=torch.float32)
    nbytes = lib.hotrg_gemm_scratch_bytes(M, N, K)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()

    def launch():
        check(lib.hotrg_gemm_split(c_void_p(A.data_ptr()), A.stride(0), c_void_p(Bt.data_ptr()), Bt.stride(0),
                                   c_void_p(C.data_ptr()), C.stride(0), M, N, K, a.npass, a.kblock, a.fold_group,
                                   c_void_p(scratch.data_ptr()), nbytes, c_void_p(s.cuda_stream)),
              "hotrg_gemm_split")

    for _ in range(max(1, a.warmup)):
        launch()
    check(lib.hotrg_gemm_status(c_void_p(scratch.data_ptr()), c_void_p(s.cuda_stream)), "gemm status")
    times = []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        launch()
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    check(lib.hotrg_gemm_status(c_void_p(scratch.data_ptr()), c_void_p(s.cuda_stream)), "gemm status")
    flops = 2.0 * M * N * K
    best = min(times)
    return {"workload": "gemm", "M": M, "N": N, "K": K, "npass": a.npass, "kblock": a.kblock,
            "fold_group": a.fold_group, "ms": times,
            "note": "each timed launch includes the FP32 -> bf16 plane split of A and Bt",
            "alg_tflops": flops / (best * 1e-3) / 1e12, "tensor_tflops": a.npass * flops / (best * 1e-3) / 1e12}


# ----------------------------------------------------------------------------- X^(n) phase flows
def run_phase(a):
    """X^(n) flows (Sec. 3, Eq. (x)) of the 4D Ising model at h = 0 at the given temperatures, each
    its own context (block-sparse squeeze, the precision schedule of --precision / --fp64-steps /
    --x6-steps), --flow-steps steps (40: the 1024^4 lattice); every flow classified from its
    converged tail (paper_1906_06060_gb300.phase). Progress goes to stderr one line per step."""
    import torch
    from paper_1906_06060_gb300 import HOTRG, phase
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    temps = [float(t) for t in a.temps.split(",") if t]
    flows = []
    for T in temps:
        xs, lnz, ms = [], [], []
        with HOTRG(4, 1.0 / T, 0.0, a.dcut, precision=a.precision, fp64_steps=a.fp64_steps, x6_steps=a.x6_steps,
                   z2=not a.no_z2, stream=stream, max_steps=a.flow_steps) as f:
            for n in range(1, a.flow_steps + 1):
                t0 = time.perf_counter()
                f.step()
                ob = f.observables()
                ms.append(1e3 * (time.perf_counter() - t0))
                xs.append(ob["x_indicator"])
                lnz.append(ob["lnz_per_site"])
                print(json.dumps({"T": T, "n": n, "x": xs[-1], "lnz": lnz[-1], "ms": ms[-1]}), file=sys.stderr,
                      flush=True)
        flows.append({"T": T, "beta": 1.0 / T, "x": xs, "lnz": lnz, "ms_per_step": ms,
                      "phase": phase.classify(xs)})
    br = phase.bracket([fl["beta"] for fl in flows], [fl["phase"] for fl in flows])
    return {"workload": "phase", "d": 4, "h": 0.0, "Dcut": a.dcut, "steps": a.flow_steps,
            "precision": a.precision, "fp64_steps": a.fp64_steps, "x6_steps": a.x6_steps, "z2": not a.no_z2,
            "flows": flows, "beta_bracket": br,
            "T_bracket": [1.0 / br[1], 1.0 / br[0]] if br else None}

def e2e(a):
    """Same metric through the public API from host inputs: context creation (beta, h copied
    from host), W + K steps with the free energy read back to the host after every step."""
    import torch
    from paper_1906_06060_gb300 import HOTRG
    torch.cuda.synchronize()
    nsteps = a.warmup + a.steps
    t0 = time.perf_counter()
    flow = HOTRG(4, a.beta, a.h, a.dcut, precision=a.precision, fp64_steps=a.fp64_steps, x6_steps=a.x6_steps,
                 kblock=a.kblock, fold_group=a.fold_group, cta_group=a.cta_group, z2=use_z2(a))
    flops = 0.0
    dims = [2, 2, 2, 2]
    records = []
    lnzs = []
    for n in range(nsteps):
        ax = 3 - (n % 4)
        P = math.prod(dims)
        chi = [min(dims[b] ** 2, a.dcut) for b in range(4) if b != ax]
        flops += 2.0 * math.prod(chi) * P ** 3
        dims = [dims[b] if b == ax else min(dims[b] ** 2, a.dcut) for b in range(4)]
        ts = time.perf_counter()
        flow.step()
        lnzs.append(float(flow.free_energy()[0][0]))
        if a.log_jsonl:
            rec = flow.step_record()
            rec["wall_ms"] = 1e3 * (time.perf_counter() - ts)
            records.append(rec)
    dt = time.perf_counter() - t0
    flow.close()
    if a.log_jsonl:
        # written after the timed flow (the records' queries are inside it: they synchronise anyway)
        with open(a.log_jsonl, "w") as fh:
            for rec in records:
                fh.write(json.dumps(rec) + "\n")
    out = {"value": flops / dt / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 16.0 / nsteps,
           "d2h_bytes_per_step": 3 * 8 + 4, "steps": nsteps,
           "note": "wall clock: context creation + every step + host read of ln Z/N after each step"}
    return out, lnzs


def accuracy_line(a, lnzs):
    """|delta(lnZ/N)| / |lnZ/N| of this run's flow after each step against the FP64 GPU flow of the
    committed accuracy summary (steps 1-8, same configuration) and the oracle's golden (steps 1-4)."""
    if not (a.dcut == 10 and a.beta == 0.1497 and a.h == 0.0):
        return None
    ref, ora = stored_fp64_reference(), oracle_golden_lnz()
    rel = {str(n): abs(lnzs[n - 1] - v) / abs(v) for n, v in sorted(ref.items()) if n <= len(lnzs)}
    rel_o = {str(n): abs(lnzs[n - 1] - v) / abs(v) for n, v in sorted(ora.items()) if n <= len(lnzs)}
    return {"rel_err_vs_fp64_gpu": rel, "rel_err_vs_oracle": rel_o,
            "lnz_per_site_last": lnzs[-1] if lnzs else None,
            "basis": "ln Z/N of the e2e flow (this run, this schedule) after each step, against the FP64 GPU "
                     "flow recorded in profiles/accuracy_fp64_vs_split_dcut10.md and the FP64 oracle's "
                     "tests/golden/flow_d4_b0.1497_h0_D10_n4.json; the measured tail beyond step 8 "
                     "is in that summary"}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        if a.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        # the reference arm (the CPU oracle) needs no GPU: its ranks meet over gloo
        td.init_process_group("nccl" if a.impl == "ours" else "gloo")
        dist = td
    if a.impl == "reference":
        out = run_reference(a, rank, world)
        if out:
            print(json.dumps(out))
        if dist:
            dist.destroy_process_group()
        return
    if a.workload in ("accuracy", "gemm", "phase"):
        from paper_1906_06060_gb300 import build
        build.build()
        run = {"accuracy": run_accuracy, "gemm": run_gemm, "phase": run_phase}[a.workload]
        print(json.dumps(run(a)))
        return
    if a.warmup < 3:
        print("warm-up must be >= 3 steps", file=sys.stderr)
        sys.exit(2)
    from paper_1906_06060_gb300 import build
    build.build()
    out = run_ours(a, rank, world, dist)
    if out is not None:
        if not a.no_e2e and a.workload == "flow":
            out["e2e"], lnzs = e2e(a)
            acc = accuracy_line(a, lnzs)
            if acc:
                out["accuracy"] = acc
        if not a.no_cpu_baseline and world == 1 and a.workload == "flow":
            dt, f = oracle_sample(a.dcut, a.cpu_slices)
            out["cpu_baseline"] = {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_threads(),
                                   "kind": "oracle",
                                   "sample": f"{a.cpu_slices} slice(s) of one steady-state Dcut={a.dcut} "
                                             f"squeeze (2 Dcut^12 flops each, {dt:.1f} s), FP64 NumPy/BLAS"}
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
