#!/usr/bin/env python
"""Benchmark of the per-cell chemistry + properties step (arXiv 2312.05800).

One step = one pass of the hot path over one batch of synthetic cells: the
composition advanced over dt = 1 us and the properties of the advanced state.

Workload (seeded, synthetic): the 30-species / 180-reaction C/H/O/N
mechanism, 2,097,152 cells sampled along algebraic stratified premixed
profiles (phi 0.5-1.2, 5 % log-normal Y noise), 1 atm. Inputs (about 0.5 GB
of FP64 state) are larger than L2, so no flush is needed between steps.

Paths (see --path):
  "ann" (default): chem_step_ann (the Box-Cox / Z-score MLP 32-1600-800-400-29 on
      the tensor cores, BF16 with FP32 accumulation) then props_eval, on
      4,194,304 cells. The network is trained first (untimed) on pairs the GPU
      stiff integrator generates; its error against a tight stiff integration
      is measured on held-out cells and printed with the throughput, beside the
      plain method (stiff + props) timed on a sample of the same cells. Side
      lines, outside the timed region: the random-data generation of Sec. 3.1
      on the same cells ("hfrd") and one training step at batch 4096 with and
      without the physics terms ("training_step").
  "stiff": chem_step_stiff (FP64 Rodas3 at rtol 1e-2: of rtol 1e-3, 3e-3, 1e-2,
      3e-2 and 1e-1, the loosest whose error against a tight integration meets
      the learned step's bars, 1e-3 relative on dY of the major species and 2 K,
      with a factor 2 to spare) followed by props_eval (FP32 arithmetic on the
      FP64 state), 2,097,152 cells. The same setting integrates the learned
      step's out-of-distribution cells.

Contract: python bench.py --gpus N --steps K --warmup W [--impl reference]
prints one JSON line. Under torchrun each rank runs its own shard (the cells
are independent: weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NCELLS = 2097152
NCELLS_ANN = 4194304
DT = 1.0e-6
TIGHT_OPTS = dict(rtol=1e-6, atol_Y=1e-13, atol_T=1e-6, h0=1e-9, max_steps=20000)
STIFF_OPTS = dict(rtol=1e-2, atol_Y=1e-8, atol_T=1e-2, h0=1e-9, max_steps=10000)
STIFF_MODE = 1                  # CHEM_ODE_MIXED on the GPU at the throughput setting (the oracle is FP64)
PARITY_OPTS = dict(rtol=1e-9, atol_Y=1e-15, atol_T=1e-9, h0=1e-9, max_steps=10000)
MECH = "c2"
ORACLE_ACC_CELLS = 4096          # default count of held-out cells whose learned-step error is measured against the oracle
E2E_PARTS = 4                   # parts of the end-to-end step whose host copies overlap the others' compute
HIDDEN = {"c2": (1600, 800, 400), "c5": (2048, 1024, 512)}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of the network's tensor-core launches of one
# 262,144-cell chunk of the timed step, from one capture of the current kernels; a mechanism without
# a capture reports null.
# DRAM bytes (read + write) of the network's tensor-core launches for one 262,144-cell chunk (ncu
# dram__bytes_read.sum + dram__bytes_write.sum of layer 1, layer 2 and the fused layers 3-4; the
# capture is summarised in profiles/gemm_layers_c2_262k_chunk_traffic.md)
GEMM_CHUNK_TRAFFIC = {"c2": {"gemm_tn_kernel<256> 1600x96": 50694144 + 783133440,
                              "gemm_tn_kernel<208> 800x1600": 841469696 + 387382784,
                              "gemm_fused34_kernel 400x800+29x400": 426411008 + 25097728}}
CELLS = {("ann", "c2"): NCELLS_ANN, ("stiff", "c2"): NCELLS, ("ann", "c5"): 16777216, ("stiff", "c5"): 1048576}
SEED = 2002
METRIC = "chem+props cells/s at stated dY/T error: ANN (BF16/FP8) vs stiff integrator, 1 GB300"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk/SM x 2 flop x max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FFMA/clk/SM x 2 flop x max SM clock


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over the ranks (the slowest rank's time): an all-reduce on the process group's
    device (CPU tensors under gloo, the rank's GPU under nccl)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cpu") if dist.get_backend() == "gloo" else torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / seconds


def shard_seed(base: int, rank: int) -> int:
    """Each rank draws its own cells (independent shards, no collective on the data path)."""
    return base + 1000 * rank


def stiff_flops_per_step(N: int, R: int, n_tb: int, n_troe: int) -> float:
    """Algorithmic FP64 flops of one Rodas3 step (exp/log counted as 20 flops):
    3 right-hand sides (species thermo 20N, per reaction 2 exp + 12, third-body
    sums 2N each, Troe 5 transcendental + 30), the analytic Jacobian (chain rule
    4 n^2, third-body rank-1 terms 12 N per reaction with a third body, sparse
    terms 72 per reaction), LU 2/3 n^3 and four solves 2 n^2 each."""
    n = N + 1
    rhs = 20 * N + R * (2 * 20 + 12) + n_tb * 2 * N + n_troe * (5 * 20 + 30)
    jac = 4 * n * n + n_tb * 12 * N + 72 * R
    return 3 * rhs + jac + (2.0 / 3.0) * n ** 3 + 4 * 2 * n * n


def pasr_rhs_flops(N: int, R: int, n_tb: int, n_troe: int) -> float:
    """FP64 flops of one reactor right-hand side (the rhs term of stiff_flops_per_step) plus the
    species times (a division and a comparison per species)."""
    return 20 * N + R * (2 * 20 + 12) + n_tb * 2 * N + n_troe * (5 * 20 + 30) + 2 * N


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def stiff_workload(mech) -> str:
    return "%s stratified-profile cells, %d species / %d reactions, dt 1 us" % (MECH, mech.N, mech.R)


def ann_workload(mech) -> str:
    widths = [mech.N + 2, *HIDDEN[MECH], mech.N - 1]
    return "ANN chemistry + props: %s, MLP %s" % (stiff_workload(mech), "-".join(str(w) for w in widths))


def make_inputs(rank: int, ncells: int = NCELLS):
    from paper_2312_05800_gb300 import synth
    mech = synth.get_mech(MECH)
    T, p, Y = synth.states_profiles(mech, ncells, shard_seed(SEED, rank), ld=synth.padded_ld(ncells))
    return mech, T, p, Y


def run_cpu_oracle(mech, T, p, Y, ncells: int):
    """The oracle (stiff + props) on the first ncells cells; returns seconds."""
    import numpy as np
    import oracle as O
    Ts, ps, Ys = T[:ncells].copy(), p[:ncells].copy(), Y[:, :ncells].copy()
    t0 = time.perf_counter()
    T1, Y1, st, ns = O.step_stiff(mech, Ts, ps, Ys, DT, **STIFF_OPTS)
    O.props(mech, T1, ps, Y1)
    el = time.perf_counter() - t0
    assert np.all(st == 0)
    return el


def omp_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    """The oracle, as it stands, on the host cores: the same path and metric as
    our arm, each step a bounded sample of the workload."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle as O
    O.build()
    from paper_2312_05800_gb300 import synth
    if args.path == "ann":
        smech = synth.get_mech(MECH)
        T, p, Y = synth.states_profiles(smech, 8192, 2003, ld=8192)
        sample = 4096
        for _ in range(args.warmup):
            cpu_baseline_ann(smech, T, p, Y, sample)
        vals = [cpu_baseline_ann(smech, T, p, Y, sample)["value"] for _ in range(args.steps)]
        v = statistics.median(vals)
        cfg = {"workload": ann_workload(smech), "path": "oracle ANN step (FP64) + props",
               "cells_per_step": sample}
        desc = "first %d cells per step: oracle ANN step (FP64) + props" % sample
    else:
        mech, T, p, Y = make_inputs(0, 8192)
        sample = 4096
        for _ in range(args.warmup):
            run_cpu_oracle(mech, T, p, Y, sample)
        v = sample / statistics.median([run_cpu_oracle(mech, T, p, Y, sample) for _ in range(args.steps)])
        cfg = {"workload": stiff_workload(mech), "path": "oracle stiff+props", "cells_per_step": sample, "rtol": STIFF_OPTS["rtol"]}
        desc = "first %d cells per step: oracle stiff + props at rtol %g" % (sample, STIFF_OPTS["rtol"])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": omp_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_stiff(args, rank, world, local):
    import torch
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y = make_inputs(rank, NCELLS)
    N = mech.N
    dm = binding.Mech(mech)
    dev = torch.device("cuda", local)
    T0 = torch.from_numpy(T).to(dev)
    p0 = torch.from_numpy(p).to(dev)
    Y0 = torch.from_numpy(Y).to(dev)
    Tw, Yw = T0.clone(), Y0.clone()
    status = torch.zeros(NCELLS, dtype=torch.int32, device=dev)
    nsteps = torch.zeros(NCELLS, dtype=torch.int32, device=dev)
    cp = torch.empty(NCELLS, dtype=torch.float32, device=dev)
    hh, mu, lam = torch.empty_like(cp), torch.empty_like(cp), torch.empty_like(cp)
    Dk = torch.empty(N, NCELLS, dtype=torch.float32, device=dev)
    opts = binding.make_opts(mode=STIFF_MODE, **STIFF_OPTS)
    stream = torch.cuda.current_stream(dev)

    def step():
        Tw.copy_(T0)
        Yw.copy_(Y0)
        binding.chem_step_stiff(dm, NCELLS, NCELLS, DT, opts, Tw, p0, Yw, status, nsteps, stream)
        binding.props_eval(dm, NCELLS, NCELLS, binding.CHEM_F64_IN_F32, Tw, p0, Yw, cp, hh, mu, lam, Dk, stream)

    # the dominant kernel (the stiff integrator) timed alone on the same stream
    def stiff_only():
        binding.chem_step_stiff(dm, NCELLS, NCELLS, DT, opts, Tw, p0, Yw, status, nsteps, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert int((status != 0).sum()) == 0, "cells failed in warm-up"
    rank_barrier(world)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ev[2 * i].record(stream)
            Tw.copy_(T0)
            Yw.copy_(Y0)
            kev[2 * i].record(stream)
            stiff_only()
            kev[2 * i + 1].record(stream)
            binding.props_eval(dm, NCELLS, NCELLS, binding.CHEM_F64_IN_F32, Tw, p0, Yw, cp, hh, mu, lam, Dk, stream)
            ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
    rank_barrier(world)
    torch.cuda.synchronize()
    step_ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]
    kern_ms = [kev[2 * i].elapsed_time(kev[2 * i + 1]) for i in range(args.steps)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world)
    value = job_rate(NCELLS * args.steps, world, total_s)
    steps_total = float(nsteps.double().sum().item())

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Th = torch.from_numpy(T).pin_memory()
    ph = torch.from_numpy(p).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    Tout = torch.empty_like(Th).pin_memory()
    Yout = torch.empty_like(Yh).pin_memory()
    sout = torch.empty(NCELLS, dtype=torch.int32).pin_memory()
    pout = [torch.empty(NCELLS, dtype=torch.float32).pin_memory() for _ in range(4)]
    Dout = torch.empty(N, NCELLS, dtype=torch.float32).pin_memory()
    h2d = Th.numel() * 8 + ph.numel() * 8 + Yh.numel() * 8
    d2h = Tout.numel() * 8 + Yout.numel() * 8 + sout.numel() * 4 + 4 * NCELLS * 4 + Dout.numel() * 4
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        Tw.copy_(Th, non_blocking=True)
        p0.copy_(ph, non_blocking=True)
        Yw.copy_(Yh, non_blocking=True)
        binding.chem_step_stiff(dm, NCELLS, NCELLS, DT, opts, Tw, p0, Yw, status, nsteps, stream)
        binding.props_eval(dm, NCELLS, NCELLS, binding.CHEM_F64_IN_F32, Tw, p0, Yw, cp, hh, mu, lam, Dk, stream)
        Tout.copy_(Tw, non_blocking=True)
        Yout.copy_(Yw, non_blocking=True)
        sout.copy_(status, non_blocking=True)
        for o, d in zip(pout, (cp, hh, mu, lam)):
            o.copy_(d, non_blocking=True)
        Dout.copy_(Dk, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_value = world * NCELLS * e2e_steps / e2e_s

    # the integrator at the parity setting (rtol 1e-9) on a sample of the same cells
    nt = min(16384, NCELLS)
    Tw.copy_(T0)
    Yw.copy_(Y0)
    e0.record(stream)
    binding.chem_step_stiff(dm, nt, NCELLS, DT, binding.make_opts(**PARITY_OPTS), Tw, p0, Yw, status, nsteps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tight = {"value": nt / (e0.elapsed_time(e1) / 1e3), "unit": "cells/s", "rtol": PARITY_OPTS["rtol"],
             "sample": "first %d cells, stiff only" % nt,
             "mean_steps_per_cell": float(nsteps[:nt].double().mean().item()),
             "failed_cells": int((status[:nt] != 0).sum().item())}
    dgemm = measure_dgemm_tflops(dev)

    flops_step = stiff_flops_per_step(N, mech.R, int((mech.rtype != 0).sum()), int((mech.rtype == 2).sum()))
    kern_s = statistics.mean(kern_ms) / 1e3
    achieved = steps_total * flops_step / kern_s / 1e12
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": stiff_workload(mech),
                       "path": "stiff+props (Rodas3 rtol %g in the mixed mode, FP32 props)" % STIFF_OPTS["rtol"],
                       "cells_per_gpu": NCELLS,
                       "l2": "inputs larger than L2 (0.5 GB FP64 state)",
                       "mean_steps_per_cell": steps_total / NCELLS, "parallelism": "replicas" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "kernel": "stiff_kernel", "flops_per_step": flops_step,
                         "peak_source": "FP64 nominal: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz",
                         "dgemm_tflops_measured": dgemm},
            "stiff_parity_setting": tight,
            "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        sample = 8192
        el = run_cpu_oracle(mech, T, p, Y, sample)
        line["cpu_baseline"] = {"value": sample / el, "unit": "cells/s", "cores": omp_threads(), "kind": "oracle",
                                "sample": "first %d of the %d cells, stiff + props at the same rtol" % (sample, NCELLS)}
    return line




def measure_dgemm_tflops(dev) -> float:
    """FP64 throughput of cuBLAS DGEMM (4096^3, CUDA events): a measured ceiling for FP64 arithmetic."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        torch.matmul(a, b)
    e1.record()
    torch.cuda.synchronize()
    return 5 * 2.0 * 4096 ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12


def measured_peak(key: str, fallback: float):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key]), "measured"
    except Exception:
        return fallback, "fallback"


def gemm_traffic(ncells: int, kernel=None):
    """DRAM bytes from GEMM_CHUNK_TRAFFIC (one ncu capture of a 262,144-cell chunk of the current
    kernels) scaled to ncells: of one launch kernel, or (kernel None) of all the network's tensor-core
    launches; None when that launch was not captured for this mechanism."""
    t = GEMM_CHUNK_TRAFFIC.get(MECH)
    if t is None:
        return None
    if kernel is None:
        return sum(t.values()) * ncells / 262144
    return t[kernel] * ncells / 262144 if kernel in t else None


def fusion_text(mask: int) -> str:
    """The layer launches that the autotuned fusion mask gives."""
    from paper_2312_05800_gb300 import binding
    return "layer 1, layer 2, " + ("layers 3-4 fused" if mask & binding.CHEM_FUSE_34 else "layer 3, layer 4")


def dominant_gemm(dom, ncells: int, chunk: int, widths, peak: float, steps: int):
    """The longest-running tensor-core kernel of the step: its share of the GEMM time and its own
    roofline fraction on its algorithmic flops per launch (the fused output layers: 2 (h2 h3 + h3
    n_out) per cell; a single layer: 2 fan_in fan_out per cell; chunk cells per launch)."""
    if dom is None:
        return None
    name, (launches, ms, _, _) = dom
    if name.startswith("gemm_fused34"):
        per_cell = 2.0 * (widths[2] * widths[3] + widths[3] * widths[4])
    else:
        shape = name.split()[-1]                      # "N x K" of the launch
        n_out, k_in = (int(x) for x in shape.split("x"))
        fan_in = widths[0] if n_out == widths[1] else k_in
        per_cell = 2.0 * fan_in * n_out
    cells_per_launch = ncells * steps / launches
    avg_ms = ms / launches
    achieved = cells_per_launch * per_cell / (avg_ms / 1e3) / 1e12
    return {"kernel": name, "launches": launches, "avg_ms": avg_ms, "cells_per_launch": cells_per_launch,
            "mflop_per_cell": per_cell / 1e6, "achieved": achieved, "frac": achieved / peak}


def roofline_line(dom, peak: float, src: str, agg_achieved, agg_traffic, mflop_cell: float, widths, net, gemm):
    """The roofline object of the step: the dominant (longest) tensor-core launch on its algorithmic
    flops per launch and its ncu DRAM bytes per launch, with the aggregate of all the network's
    tensor-core launches (the method's 2 sum fan_in fan_out per cell) beside it."""
    out = {"bound": "tensor", "achieved": dom["achieved"] if dom else None, "peak": peak, "unit": "TFLOP/s",
           "frac": dom["frac"] if dom else None,
           "traffic": gemm_traffic(dom["cells_per_launch"], dom["kernel"]) if dom else None,
           "traffic_unit": "DRAM bytes (read + write) per launch: ncu dram__bytes of the launch on one "
                           "262,144-cell chunk, scaled to the launch's cells",
           "kernel": dom["kernel"] if dom else None, "launches": dom["launches"] if dom else None,
           "avg_ms": dom["avg_ms"] if dom else None, "cells_per_launch": dom["cells_per_launch"] if dom else None,
           "work": ("%.4f MFLOP per cell (2 fan_in fan_out of the layer)" % dom["mflop_per_cell"]) if dom else None,
           "peak_source": src,
           "mlp_aggregate": {
               "achieved": agg_achieved, "frac": (agg_achieved / peak) if agg_achieved else None,
               "traffic": agg_traffic,
               "traffic_unit": "DRAM bytes (read + write) of the network's tensor-core launches per step",
               "kernel": "every tensor-core launch of the network per step (%s); CUDA events around each launch"
                         % fusion_text(net.fusion),
               "work": "%.4f MFLOP per cell: 2 sum fan_in x fan_out over %s (first layer K = N + 2, not the "
                       "device's three-term K)" % (mflop_cell, "-".join(str(w) for w in widths)),
               "per_shape": {k: {"launches": v[0], "ms": v[1],
                                 "tflops": v[2] / (v[1] / 1e3) / 1e12 if v[1] > 0 else None}
                             for k, v in gemm.items()}}}
    return out


def guarded(fn):
    """A side line of the bench: its result, or the error that stopped it (the headline stays)."""
    try:
        return fn()
    except Exception as e:          # reported in the line, never allowed to end the run
        return {"error": "%s: %s" % (type(e).__name__, e)}


def props_full_line(prof, ncells: int, steps: int, N: int):
    """The full properties pass of the timed steps (cp, h, mu, lambda, D_k) on the FP32 CUDA cores: its
    algorithmic flops per cell, about 16 N^2 + 30 N (the Wilke pair terms of mu and lambda and the
    diffusion resistance sums over species pairs, plus the per-species fits), over its time in the
    library's profiler, against the nominal FP32 rate (no measured FP32 peak is available)."""
    ms = sum(v[1] for k, v in prof.items() if k.startswith("props_kernel")) / steps
    if ms <= 0:
        return None
    flop = 16 * N * N + 30 * N
    tf = ncells * flop / (ms / 1e3) / 1e12
    return {"ms_per_step": ms, "cells_per_launch": ncells,
            "roofline": {"bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tf / FP32_PEAK_TFLOPS, "flops_per_cell": flop, "kernel": "props_kernel",
                         "peak_source": "FP32 nominal: 152 SM x 128 FMA/clk x 2 x 2.07 GHz"}}


def bench_hfrd(dm, smech, T, p, Y, T0, p0, Y0, n: int, ld: int, dev, reps: int = 5):
    """chem_hfrd_perturb (Sec. 3.1: Eq. 1-4, the renormalisation and the Table 1 filter) on the bench's n
    cells as base states, with seeded uniform draws c in [-1, 1] made on the device: time per launch
    (CUDA events, after two warm-up launches). Its FP64 work per state, with a power as one exp and one
    log at 20 flops each (the stiff kernel's convention): Eq. 1-3 12 flops, Eq. 4 42 per non-bath
    species, the sum and the scaling 2 per non-bath species, the scale factor 2, the element moles 9 per
    species, the ratios 6: 53 N - 24 flops, about 2 flops per byte of its reads (2N + 5) x 8 and writes
    (N + 2) x 8 + 1, ten
    times the FP64 ridge, so the roofline is the FP64 rate; the HBM fraction is reported beside it."""
    import torch
    from paper_2312_05800_gb300 import binding, synth
    N, b = smech.N, smech.bath
    prm = binding.hfrd_params(T_min=float(T[:n].min()), T_max=float(T[:n].max()), p_min=float(p[:n].min()),
                              p_max=float(p[:n].max()), Yb_min=float(Y[b, :n].min()), Yb_max=float(Y[b, :n].max()))
    gen = torch.Generator(device=dev)
    gen.manual_seed(2085)
    c = torch.rand((3 + N, ld), dtype=torch.float64, device=dev, generator=gen) * 2.0 - 1.0
    T2 = torch.empty(ld, dtype=torch.float64, device=dev)
    p2 = torch.empty_like(T2)
    Y2 = torch.empty((N, ld), dtype=torch.float64, device=dev)
    keep = torch.empty(ld, dtype=torch.uint8, device=dev)
    chon = synth.element_table(smech)
    stream = torch.cuda.current_stream(dev)

    def call():
        binding.chem_hfrd_perturb(dm, prm, chon, n, ld, T0, p0, Y0, c, T2, p2, Y2, keep, stream)

    for _ in range(2):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    per_state = (2 * N + 5) * 8 + (N + 2) * 8 + 1
    flop_state = 53 * N - 24
    gbs = n * per_state / (ms / 1e3) / 1e9
    hbm, hbm_src = measured_peak("hbm_gbs", 6800.0)
    tf = n * flop_state / (ms / 1e3) / 1e12
    return {"value": n / (ms / 1e3), "unit": "states/s", "ms": ms, "launches": reps,
            "kept_fraction": float(keep[:n].float().mean().item()),
            "roofline": {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tf / FP64_PEAK_TFLOPS, "flops_per_state": flop_state,
                         "peak_source": "FP64 nominal: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz", "kernel": "hfrd_kernel",
                         "hbm": {"achieved_GBps": gbs, "peak_GBps": hbm, "frac": gbs / hbm,
                                 "bytes_per_state": per_state, "peak_source": hbm_src}},
            "workload": "chem_hfrd_perturb on the %d bench cells as base states, seeded uniform draws" % n}


def bench_train_step(dm, smech, hidden, dev, batch: int = 4096, steps: int = 20, pairs: int = 65536):
    """mlp_train_step (Sec. 3.2: forward, the Eq. 5 loss, back-propagation, Adam) at the bench's batch on
    a fresh handle and freshly integrated pairs: ms per step with Eq. 5 alone and with the two physics
    terms (weights 0.1, scales fitted on the pairs), each after three warm-up steps, CUDA events on the
    launching stream; the tensor-core rate on the algorithmic flops of a step (the forward product, dW
    and dX of every layer, the first layer without dX) against the measured BF16 peak."""
    import torch
    from paper_2312_05800_gb300 import binding, train
    data = train.make_training_set(dm, smech, pairs, seed=2107)
    net = binding.Mlp(dm, hidden=hidden, dt=DT, seed=3007, chunk=pairs, max_batch=batch)
    try:
        train.fit_norm(net, data)
        s_m, s_q = net.fit_physics_scales(data.n, data.ld, data.T, data.Y, data.Y1)
        loss = torch.zeros(4, dtype=torch.float32, device=dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(2108)
        rows = [torch.randperm(data.n, generator=gen, device=dev)[:batch].to(torch.int32) for _ in range(steps)]
        stream = torch.cuda.current_stream(dev)

        def timed():
            for i in range(3):
                binding.mlp_train_step(net, batch, rows[i], data.ld, data.T, data.p, data.Y, data.Y1, 1e-4, loss)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(steps):
                binding.mlp_train_step(net, batch, rows[i], data.ld, data.T, data.p, data.Y, data.Y1, 1e-4, loss)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

        ms_l1 = timed()
        net.set_physics_loss(0.1, 0.1, s_m, s_q)
        ms_phys = timed()
        err = net.error()
    finally:
        net.free()
    widths = [smech.N + 2, *hidden, smech.N - 1]
    fwd = 2.0 * sum(a * b_ for a, b_ in zip(widths[:-1], widths[1:]))
    flop = batch * (3.0 * fwd - 2.0 * widths[0] * widths[1])
    peak, src = measured_peak("bf16_tflops", 1900.0)
    tf = flop / (ms_l1 / 1e3) / 1e12
    return {"batch": batch, "steps": steps, "ms_per_step": ms_l1, "ms_per_step_physics_terms": ms_phys,
            "physics_terms_overhead": ms_phys / ms_l1 - 1.0, "physics_scales": [s_m, s_q], "device_error": err,
            "mflop_per_sample": flop / batch / 1e6,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "peak_source": src},
            "workload": "%d GPU-integrated pairs, network %s, one Adam step per batch"
                        % (pairs, "-".join(str(w) for w in widths))}


def accuracy(mech, T0, Y0, Ta, Ya, Tr, Yr, n):
    """Per major species relative L2 of dY, and |T error| max / p99.9, against a reference."""
    import numpy as np
    major = [k for k in range(mech.N) if k != mech.bath and Y0[k, :n].mean() >= 1e-2]
    rel = {}
    for k in major:
        dr = Yr[k, :n] - Y0[k, :n]
        da = Ya[k, :n] - Y0[k, :n]
        rel[str(k)] = float(np.linalg.norm(da - dr) / max(np.linalg.norm(dr), 1e-300))
    terr = np.abs(Ta[:n] - Tr[:n])
    return {"dY_rel_l2_major": rel, "dY_rel_l2_major_max": max(rel.values()) if rel else None,
            "T_err_max_K": float(terr.max()), "T_err_p999_K": float(np.percentile(terr, 99.9)), "cells": int(n)}


def bench_ann(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2312_05800_gb300 import binding, synth, train
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    smech = synth.get_mech(MECH)
    dm = binding.Mech(smech)
    N = smech.N
    hidden = HIDDEN[MECH]
    # ---- training (untimed): GPU stiff pairs, statistics, Adam on Eq. 5
    net = binding.Mlp(dm, hidden=hidden, dt=DT, seed=3003, chunk=args.chunk, max_batch=4096)
    fp8 = not args.untrained and not args.no_fp8
    if args.untrained:
        t_data = t_train = 0.0
        hist = [float("nan")]
    else:
        t0 = time.perf_counter()
        data = train.make_training_set(dm, smech, args.train_pairs, seed=shard_seed(2103, rank))
        t_data = time.perf_counter() - t0
        train.fit_norm(net, data)
        t0 = time.perf_counter()
        hist = train.train(net, data, epochs=args.epochs, batch=4096, lr0=args.lr)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        # out-of-distribution guard fitted on the training states; off-grid cells fall back to stiff
        binding.chem_mlp_fit_ood_multi(net, dm, data.n, data.ld, data.T, data.p, data.Y,
                                       [smech.roles[r] for r in args.ood_species.split(",")], 64, args.ood_kmin)
        if fp8:
            # E4M3 activation scales from the BF16 forward of training states
            binding.chem_mlp_calibrate_fp8(net, min(data.n, 262144), data.ld, data.T, data.p, data.Y)
    tiles = binding.chem_mlp_autotune(net, min(args.chunk, 524288))
    # ---- the paper's model form: one network per species (Sec. 3.2), trained on the same pairs
    ens = None
    ens_train = None
    if args.ens_epochs > 0 and not args.untrained:
        ens = binding.Mlp(dm, hidden=hidden, dt=DT, seed=3004, chunk=args.ens_chunk, max_batch=4096, ensemble=True)
        train.fit_norm(ens, data)
        t0 = time.perf_counter()
        ens_hist = train.train(ens, data, epochs=args.ens_epochs, batch=4096, lr0=args.ens_lr)
        torch.cuda.synchronize()
        ens_train = {"pairs": args.train_pairs, "epochs": args.ens_epochs, "batch": 4096,
                     "loss_first_epoch": ens_hist[0], "loss_last_epoch": ens_hist[-1],
                     "train_s": time.perf_counter() - t0}
        binding.chem_mlp_fit_ood_multi(ens, dm, data.n, data.ld, data.T, data.p, data.Y,
                                       [smech.roles[r] for r in args.ood_species.split(",")], 64, args.ood_kmin)
        ens_tiles = binding.chem_mlp_autotune(ens, min(args.ens_chunk, 262144))
    if not args.untrained:
        del data
    fb_opts = binding.make_opts(mode=STIFF_MODE, **STIFF_OPTS)
    # ---- inference workload
    ncells = args.cells
    T, p, Y = synth.states_profiles(smech, ncells, shard_seed(2003, rank), ld=synth.padded_ld(ncells))
    ld = T.shape[0]
    T0 = torch.from_numpy(T).to(dev)
    p0 = torch.from_numpy(p).to(dev)
    Y0 = torch.from_numpy(Y).to(dev)
    Tw, Yw = T0.clone(), Y0.clone()
    status = torch.zeros(ld, dtype=torch.int32, device=dev)
    cp = torch.empty(ld, dtype=torch.float32, device=dev)
    hh, mu, lam = torch.empty_like(cp), torch.empty_like(cp), torch.empty_like(cp)
    Dk = torch.empty(N, ld, dtype=torch.float32, device=dev)
    # ---- accuracy on held-out cells against a tight stiff integration
    ne = min(args.eval_cells, ncells) if not args.untrained else 4
    Ta, Ya = T0.clone(), Y0.clone()
    binding.chem_step_ann(dm, net, ne, ld, DT, binding.CHEM_PREC_BF16, fb_opts, Ta, p0, Ya, status)
    Tr, Yr = T0.clone(), Y0.clone()
    binding.chem_step_stiff(dm, ne, ld, DT, binding.make_opts(**TIGHT_OPTS), Tr, p0, Yr, status)
    Ts, Ys = T0.clone(), Y0.clone()
    binding.chem_step_stiff(dm, ne, ld, DT, binding.make_opts(mode=STIFF_MODE, **STIFF_OPTS), Ts, p0, Ys, status)
    T8, Y8 = T0.clone(), Y0.clone()
    if fp8:
        binding.chem_step_ann(dm, net, ne, ld, DT, binding.CHEM_PREC_FP8, fb_opts, T8, p0, Y8, status)
    Te, Ye = T0.clone(), Y0.clone()
    if ens is not None:
        binding.chem_step_ann(dm, ens, ne, ld, DT, binding.CHEM_PREC_BF16, fb_opts, Te, p0, Ye, status)
    torch.cuda.synchronize()
    Ta, Ya, Tr, Yr, Ts, Ys, T8, Y8, Te, Ye = [x.cpu().numpy() for x in (Ta, Ya, Tr, Yr, Ts, Ys, T8, Y8, Te, Ye)]
    acc_ann = accuracy(smech, T, Y, Ta, Ya, Tr, Yr, ne)
    acc_stiff = accuracy(smech, T, Y, Ts, Ys, Tr, Yr, ne)
    acc_fp8 = accuracy(smech, T, Y, T8, Y8, Tr, Yr, ne) if fp8 else None
    acc_ens = accuracy(smech, T, Y, Te, Ye, Tr, Yr, ne) if ens is not None else None
    # the learned steps' results on the first cells, for the oracle-referenced accuracy of the CPU leg
    no = min(args.oracle_cells, ne)
    first = {"ann": (Ta[:no].copy(), Ya[:, :no].copy())}
    if fp8:
        first["fp8"] = (T8[:no].copy(), Y8[:, :no].copy())
    if ens is not None:
        first["ensemble"] = (Te[:no].copy(), Ye[:, :no].copy())
    del Ta, Ya, Tr, Yr, Ts, Ys, T8, Y8, Te, Ye

    def step(st=stream, prec=binding.CHEM_PREC_BF16):
        Tw.copy_(T0)
        Yw.copy_(Y0)
        binding.chem_step_ann_props(dm, net, ncells, ld, DT, prec, fb_opts, Tw, p0, Yw, status, cp, hh, mu, lam, Dk,
                                    st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert net.error() == 0
    rank_barrier(world)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    binding.chem_prof_enable(True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")          # lets a profiler select the timed launches
        ev[0].record(stream)
        for _ in range(args.steps):
            step()
        ev[1].record(stream)
        torch.cuda.synchronize()
        rank_barrier(world)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    prof = binding.chem_prof_read()
    binding.chem_prof_enable(False)
    n_fallback = int((status[:ncells] == binding.CELL_FALLBACK).sum().item())
    n_failed = int((status[:ncells] >= 2).sum().item())
    # the same step captured once as a CUDA graph and replayed
    graph = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream(dev)
    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        step(None)
    gs.synchronize()
    with torch.cuda.graph(graph):
        step(None)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / args.steps
    del graph
    # ---- the HBM-bound part of props_eval alone: thermo only (cp, h) from the FP64 state
    binding.props_eval(dm, ncells, ld, binding.CHEM_F64_IN_F32, Tw, p0, Yw, cp, hh, None, None, None, stream)
    g0.record(stream)
    for _ in range(args.steps):
        binding.props_eval(dm, ncells, ld, binding.CHEM_F64_IN_F32, Tw, p0, Yw, cp, hh, None, None, None, stream)
    g1.record(stream)
    torch.cuda.synchronize()
    th_ms = g0.elapsed_time(g1) / args.steps
    th_bytes = ncells * ((N + 1) * 8 + 2 * 4)
    hbm_peak, hbm_src = measured_peak("hbm_gbs", 6800.0)
    props_thermo = {"ms": th_ms, "bytes_per_cell": (N + 1) * 8 + 2 * 4,
                    "achieved_GBps": th_bytes / (th_ms / 1e3) / 1e9, "peak_GBps": hbm_peak,
                    "frac": th_bytes / (th_ms / 1e3) / 1e9 / hbm_peak, "peak_source": hbm_src,
                    "note": "props_eval with mu, lambda, D_k null: NASA-7 cp and h only (reads T and Y in FP64, "
                            "writes cp, h in FP32; p is not read)"}
    # ---- the same step with the hidden-to-hidden layers on E4M3 operands
    fp8_line = None
    if fp8:
        for _ in range(args.warmup):
            step(prec=binding.CHEM_PREC_FP8)
        torch.cuda.synchronize()
        binding.chem_prof_enable(True)
        g0.record(stream)
        for _ in range(args.steps):
            step(prec=binding.CHEM_PREC_FP8)
        g1.record(stream)
        torch.cuda.synchronize()
        prof8 = binding.chem_prof_read()
        binding.chem_prof_enable(False)
        f8_ms = g0.elapsed_time(g1) / args.steps
        g8 = {k: v for k, v in prof8.items() if k.startswith("gemm_")}
        e8 = {k: v for k, v in g8.items() if "e4m3" in k}
        e8_ms, e8_fl = sum(v[1] for v in e8.values()), sum(v[2] for v in e8.values())
        peak8 = measured_peak("bf16_tflops", 1900.0)[0] * 2.0
        fp8_line = {"value": world * ncells / (f8_ms / 1e3), "unit": "cells/s", "ms_per_step": f8_ms,
                    "accuracy_vs_tight_stiff": acc_fp8, "act_scales": [float(v) for v in
                                                                      binding.chem_mlp_get_fp8_scales(net)],
                    "e4m3_gemm_roofline": {"bound": "tensor", "achieved": e8_fl / (e8_ms / 1e3) / 1e12 if e8_ms else None,
                                           "peak": peak8, "unit": "TFLOP/s",
                                           "frac": (e8_fl / (e8_ms / 1e3) / 1e12 / peak8) if e8_ms else None,
                                           "peak_source": "measured BF16 x 2 (the nominal FP8 / BF16 ratio)"},
                    "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof8.items()},
                    "layers": "h1 -> h2 and h2 -> h3 on E4M3 operands (per-row weight scales, per-tensor "
                              "activation scales), first and output layers BF16"}
    # ---- PaSR scaling (Sec. 4.1) of the learned step's result, timed alone
    rng_t = np.random.default_rng(2071)
    tt = torch.from_numpy(10.0 ** rng_t.uniform(-6, -2, ld)).to(dev)
    tk = torch.from_numpy(10.0 ** rng_t.uniform(-7, -3, ld)).to(dev)
    kap = torch.empty(ld, dtype=torch.float64, device=dev)
    tcd = torch.empty_like(kap)
    step()
    Tp, Yp = Tw.clone(), Yw.clone()
    binding.chem_pasr(dm, ncells, ld, 1e-6, T0, p0, Y0, tt, tk, Tp, Yp, tcd, kap, stream)
    torch.cuda.synchronize()
    kap_med = float(kap[:ncells].median().item())
    g0.record(stream)
    for _ in range(2):
        binding.chem_pasr(dm, ncells, ld, 1e-6, T0, p0, Y0, tt, tk, Tp, Yp, tcd, kap, stream)
    g1.record(stream)
    torch.cuda.synchronize()
    pasr_ms = g0.elapsed_time(g1) / 2
    rhs_fl = pasr_rhs_flops(smech.N, smech.R, int((smech.rtype != 0).sum()), int((smech.rtype == 2).sum()))
    pasr_line = {"ms": pasr_ms, "cells_per_s": ncells / (pasr_ms / 1e3), "kappa_median": kap_med,
                 "roofline": {"bound": "alu", "achieved": ncells * rhs_fl / (pasr_ms / 1e3) / 1e12,
                              "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": ncells * rhs_fl / (pasr_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                              "flops_per_cell": rhs_fl},
                 "workload": "chem_pasr on the learned step's result: FP64 reactor rates at the state before "
                             "the step, tau_c, kappa with seeded Taylor / Kolmogorov times, scaled (T, Y)"}
    del Tp, Yp, tt, tk, kap, tcd
    # ---- the per-species ensemble through the same call
    ens_line = None
    if ens is not None:
        def ens_step():
            Tw.copy_(T0)
            Yw.copy_(Y0)
            binding.chem_step_ann_props(dm, ens, ncells, ld, DT, binding.CHEM_PREC_BF16, fb_opts, Tw, p0, Yw, status,
                                        cp, hh, mu, lam, Dk, stream)

        ens_steps = max(1, min(args.steps, 5))
        for _ in range(min(args.warmup, 2)):
            ens_step()
        torch.cuda.synchronize()
        assert ens.error() == 0
        binding.chem_prof_enable(True)
        g0.record(stream)
        for _ in range(ens_steps):
            ens_step()
        g1.record(stream)
        torch.cuda.synchronize()
        profe = binding.chem_prof_read()
        binding.chem_prof_enable(False)
        e_ms = g0.elapsed_time(g1) / ens_steps
        ge = {k: v for k, v in profe.items() if k.startswith("gemm_")}
        ge_ms, ge_fl = sum(v[1] for v in ge.values()), sum(v[2] for v in ge.values())
        bf_peak = measured_peak("bf16_tflops", 1900.0)[0]
        ens_line = {"value": world * ncells / (e_ms / 1e3), "unit": "cells/s", "ms_per_step": e_ms,
                    "steps": ens_steps,
                    "model": "%d networks %d-%s-1 (one per non-bath species), BF16 tcgen05 grouped GEMMs"
                             % (N - 1, N + 2, "-".join(str(h) for h in hidden)),
                    "mflop_per_cell": 2.0 * (N - 1) * ((N + 2) * hidden[0] + hidden[0] * hidden[1] +
                                                       hidden[1] * hidden[2] + hidden[2]) / 1e6,
                    "accuracy_vs_tight_stiff": acc_ens, "training": ens_train, "autotuned_tiles": ens_tiles,
                    "fallback_cells_per_step": int((status[:ncells] == binding.CELL_FALLBACK).sum().item()),
                    "gemm_roofline": {"bound": "tensor", "achieved": ge_fl / (ge_ms / 1e3) / 1e12 if ge_ms else None,
                                      "peak": bf_peak, "unit": "TFLOP/s",
                                      "frac": (ge_fl / (ge_ms / 1e3) / 1e12 / bf_peak) if ge_ms else None,
                                      "peak_source": "measured",
                                      "per_shape": {k: {"launches": v[0], "ms": v[1],
                                                        "tflops": v[2] / (v[1] / 1e3) / 1e12 if v[1] > 0 else None}
                                                    for k, v in ge.items()}},
                    "kernels_ms_per_step": {k: v[1] / ens_steps for k, v in profe.items()},
                    "chunk": args.ens_chunk}
        ens.free()
    total_s = max_over_ranks(ev[0].elapsed_time(ev[1]) / 1e3, world)
    value = job_rate(ncells * args.steps, world, total_s)
    # every tensor-core launch of the network (single layers and the fused output layers); the work
    # is the method's: 2 sum fan_in fan_out per cell with the first layer's true K of N + 2 inputs
    # (the device's three-term first layer triples K but is not the method's work)
    gemm = {k: v for k, v in prof.items() if k.startswith("gemm_")}
    g_ms = sum(v[1] for v in gemm.values())
    widths = [N + 2, *hidden, N - 1]
    mflop_cell = 2.0 * sum(a * b for a, b in zip(widths[:-1], widths[1:])) / 1e6
    g_fl = ncells * args.steps * mflop_cell * 1e6
    peak, src = measured_peak("bf16_tflops", 1900.0)
    achieved = g_fl / (g_ms / 1e3) / 1e12 if g_ms > 0 else None
    dom = max(gemm.items(), key=lambda kv: kv[1][1]) if gemm else None
    dom_line = dominant_gemm(dom, ncells, args.chunk, widths, peak, args.steps)
    # ---- the plain method on a sample of the same cells (stiff at the throughput setting + props)
    ns = min(args.stiff_sample, ncells)
    torch.cuda.synchronize()
    Tw.copy_(T0)
    Yw.copy_(Y0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    binding.chem_step_stiff(dm, ns, ld, DT, binding.make_opts(mode=STIFF_MODE, **STIFF_OPTS), Tw, p0, Yw, status, None,
                            stream)
    binding.props_eval(dm, ns, ld, binding.CHEM_F64_IN_F32, Tw, p0, Yw, cp, hh, mu, lam, Dk, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    stiff_value = ns / (e0.elapsed_time(e1) / 1e3)
    # ---- batched + fallback: the same cells with 2 % moved off the manifold (T +/- 300 K, Y noise 0.2)
    T4, Y4, moved = synth.perturb_off_manifold(T, Y, ncells, 0.02, shard_seed(2004, rank))
    T4d, Y4d = torch.from_numpy(T4).to(dev), torch.from_numpy(Y4).to(dev)
    Tw.copy_(T4d)
    Yw.copy_(Y4d)
    torch.cuda.synchronize()
    binding.chem_prof_enable(True)
    e0.record(stream)
    binding.chem_step_ann_props(dm, net, ncells, ld, DT, binding.CHEM_PREC_BF16, fb_opts, Tw, p0, Yw, status, cp, hh,
                                mu, lam, Dk, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    prof4 = binding.chem_prof_read()
    binding.chem_prof_enable(False)
    st4 = status[:ncells].cpu().numpy()
    mv = moved[:ncells]
    flagged = st4 == binding.CELL_FALLBACK
    c4_ms = e0.elapsed_time(e1)
    ne4 = min(args.eval_cells, ncells)
    Tr4, Yr4 = T4d.clone(), Y4d.clone()
    binding.chem_step_stiff(dm, ne4, ld, DT, binding.make_opts(**TIGHT_OPTS), Tr4, p0, Yr4, status)
    acc_c4 = accuracy(smech, T4, Y4, Tw.cpu().numpy(), Yw.cpu().numpy(), Tr4.cpu().numpy(), Yr4.cpu().numpy(), ne4)
    batched = {"value": ncells / (c4_ms / 1e3), "unit": "cells/s", "ms_per_step": c4_ms,
               "perturbed_cells": int(mv.sum()), "fallback_cells": int(flagged.sum()),
               "recall": float(flagged[mv].mean()), "false_positive_rate": float(flagged[~mv].mean()),
               "failed_cells": int((st4 >= 2).sum()),
               "fallback_ms": sum(v[1] for k, v in prof4.items() if "fallback" in k),
               "accuracy_vs_tight_stiff": acc_c4,
               "workload": "the same %d cells with a seeded 2 %% moved off the manifold (T +/- 300 K, "
                           "Y x exp(0.2 xi)); guard + stiff fallback (rtol %g) in the step" % (ncells, STIFF_OPTS["rtol"])}
    del T4d, Y4d, Tr4, Yr4

    # ---- end to end through the C ABI with pinned host buffers. The cells go in E2E_PARTS parts (each
    # its own SoA arrays on host and device); the host-to-device copies of part i + 1 and the
    # device-to-host copies of part i - 1 run on two copy streams while part i steps, so the copies
    # hide behind the computation.
    e2e_steps = max(1, min(args.steps, 3))
    parts = []
    sub = (ncells // E2E_PARTS + 3) // 4 * 4
    for c0 in range(0, ncells, sub):
        n_i = min(sub, ncells - c0)
        ld_i = synth.padded_ld(n_i)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hT, hp, hY = pin(T[c0:c0 + n_i]), pin(p[c0:c0 + n_i]), pin(Y[:, c0:c0 + n_i])
        if ld_i != n_i:
            hT = pin(np.pad(T[c0:c0 + n_i], (0, ld_i - n_i), constant_values=300.0))
            hp = pin(np.pad(p[c0:c0 + n_i], (0, ld_i - n_i), constant_values=synth.P_ATM))
            hY = pin(np.pad(Y[:, c0:c0 + n_i], ((0, 0), (0, ld_i - n_i))))
        d = dict(n=n_i, ld=ld_i, hT=hT, hp=hp, hY=hY,
                 T=torch.empty(ld_i, dtype=torch.float64, device=dev), p=torch.empty(ld_i, dtype=torch.float64,
                                                                                      device=dev),
                 Y=torch.empty(N, ld_i, dtype=torch.float64, device=dev),
                 st=torch.empty(ld_i, dtype=torch.int32, device=dev),
                 props=[torch.empty(ld_i, dtype=torch.float32, device=dev) for _ in range(4)],
                 Dk=torch.empty(N, ld_i, dtype=torch.float32, device=dev),
                 oT=torch.empty(ld_i, dtype=torch.float64).pin_memory(),
                 oY=torch.empty(N, ld_i, dtype=torch.float64).pin_memory(),
                 ost=torch.empty(ld_i, dtype=torch.int32).pin_memory(),
                 oprops=[torch.empty(ld_i, dtype=torch.float32).pin_memory() for _ in range(4)],
                 oDk=torch.empty(N, ld_i, dtype=torch.float32).pin_memory(),
                 ev_in=torch.cuda.Event(), ev_done=torch.cuda.Event(), ev_out=torch.cuda.Event())
        parts.append(d)
    h2d = sum((q["hT"].numel() + q["hp"].numel() + q["hY"].numel()) * 8 for q in parts)
    d2h = sum((q["oT"].numel() + q["oY"].numel()) * 8 + q["ost"].numel() * 4 + 4 * q["ld"] * 4 + q["oDk"].numel() * 4
              for q in parts)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_step():
        for q in parts:
            s_in.wait_event(q["ev_out"])           # the previous step's results of this part are on the host
            with torch.cuda.stream(s_in):
                q["T"].copy_(q["hT"], non_blocking=True)
                q["p"].copy_(q["hp"], non_blocking=True)
                q["Y"].copy_(q["hY"], non_blocking=True)
                q["ev_in"].record(s_in)
        for q in parts:
            stream.wait_event(q["ev_in"])
            binding.chem_step_ann_props(dm, net, q["n"], q["ld"], DT, binding.CHEM_PREC_BF16, fb_opts, q["T"], q["p"],
                                        q["Y"], q["st"], *q["props"], q["Dk"], stream)
            q["ev_done"].record(stream)
            s_out.wait_event(q["ev_done"])
            with torch.cuda.stream(s_out):
                q["oT"].copy_(q["T"], non_blocking=True)
                q["oY"].copy_(q["Y"], non_blocking=True)
                q["ost"].copy_(q["st"], non_blocking=True)
                for o_, d_ in zip(q["oprops"], q["props"]):
                    o_.copy_(d_, non_blocking=True)
                q["oDk"].copy_(q["Dk"], non_blocking=True)
                q["ev_out"].record(s_out)

    for q in parts:
        q["ev_out"].record(stream)
    e2e_step()                                   # warm: the parts' first calls
    torch.cuda.synchronize()
    e0.record(stream)
    s_in.wait_event(e0)
    for _ in range(e2e_steps):
        e2e_step()
    for q in parts:
        stream.wait_event(q["ev_out"])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = world * ncells * e2e_steps / (e0.elapsed_time(e1) / 1e3)
    assert all(int((q["ost"][:q["n"]] >= 2).sum()) == 0 for q in parts)
    del parts
    # ---- the upstream and training rows beside the step (outside the timed region)
    hfrd_line = guarded(lambda: bench_hfrd(dm, smech, T, p, Y, T0, p0, Y0, ncells, ld, dev))
    train_line = None if args.untrained else guarded(lambda: bench_train_step(dm, smech, hidden, dev))
    chunks = (ncells + args.chunk - 1) // args.chunk
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": ann_workload(smech),
                       "path": "chem_step_ann_props: BF16 tcgen05 GEMMs (FP32 accumulation); out-of-distribution "
                               "cells to the FP64 stiff integrator; then the FP32 properties of the advanced "
                               "state, after the fallback",
                       "cells_per_gpu": ncells, "l2": "inputs larger than L2 (1 GB FP64 state)",
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "accuracy": {"ann_vs_tight_stiff": acc_ann, "stiff_throughput_setting_vs_tight_stiff": acc_stiff,
                         "reference": "chem_step_stiff rtol 1e-6 on the first %d cells" % ne},
            "stiff": {"value": stiff_value, "unit": "cells/s",
                      "path": "chem_step_stiff rtol %g (mixed mode) + props_eval" % STIFF_OPTS["rtol"],
                      "sample": "first %d of the %d cells, one step" % (ns, ncells),
                      "ann_speedup": value / stiff_value},
            "training": {"pairs": args.train_pairs, "epochs": args.epochs, "batch": 4096,
                         "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "data_s": t_data,
                         "train_s": t_train},
            "roofline": roofline_line(dom_line, peak, src, achieved, gemm_traffic(ncells), mflop_cell, widths, net,
                                      gemm),
            "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
            "guard": {"ood": not args.untrained,
                      "grid": "64^3 over (T, h/R, Y_s) for s in %s, neighbourhood >= %d; outside any grid -> fallback"
                      % (args.ood_species, args.ood_kmin), "fallback_cells_per_step": n_fallback, "failed_cells": n_failed,
                      "fallback_rtol": STIFF_OPTS["rtol"], "fallback_mode": "mixed (CHEM_ODE_MIXED)"},
            "autotuned_tiles": tiles,
            "graph": {"ms_per_step": graph_ms, "cells_per_s": world * ncells / (graph_ms / 1e3),
                      "note": "the whole step captured once as a CUDA graph and replayed"},
            "batched_fallback": batched,
            "fp8": fp8_line,
            "ensemble": ens_line,
            "pasr": pasr_line,
            "props_thermo": props_thermo,
            "props_full": guarded(lambda: props_full_line(prof, ncells, args.steps, N)),
            "hfrd": hfrd_line,
            "training_step": train_line,
            "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "overlap": "%d parts of the cells; host-to-device and device-to-host copies on two streams "
                               "beside the compute stream" % E2E_PARTS},
            # the library's kernel launches of the timed steps, counted by its profiler (per chunk: the
            # prologue, the tensor-core layers and the epilogue; per step: the fallback and props)
            "gpu_launches": int(sum(v[0] for v in prof.values())),
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_ann(smech, T, p, Y)
        line["cpu_baseline"]["one_core"] = cpu_baseline_one_core()
        if not args.untrained and no > 0:
            # the FP64 oracle's integration (parity setting) of the first held-out cells: the error of
            # each learned step against it
            To, Yo, so, t_or = oracle_reference(smech, T, p, Y, no)
            ref = "oracle stiff integration (FP64, rtol %g) of the first %d held-out cells (%.1f s on %d host " \
                  "cores)" % (PARITY_OPTS["rtol"], no, t_or, omp_threads())
            line["accuracy"]["ann_vs_oracle"] = accuracy(smech, T, Y, *first["ann"], To, Yo, no)
            line["accuracy"]["oracle_reference"] = ref
            line["accuracy"]["oracle_failed_cells"] = int((so != 0).sum())
            if line.get("fp8") and "fp8" in first:
                line["fp8"]["accuracy_vs_oracle"] = accuracy(smech, T, Y, *first["fp8"], To, Yo, no)
            if line.get("ensemble") and "ensemble" in first:
                line["ensemble"]["accuracy_vs_oracle"] = accuracy(smech, T, Y, *first["ensemble"], To, Yo, no)
    return line


def oracle_reference(smech, T, p, Y, n):
    """The oracle's FP64 stiff integration over dt at the parity setting of the first n cells (the
    reference of the learned step's error). Returns (T, Y, status, seconds)."""
    import oracle as O
    O.build()
    t0 = time.perf_counter()
    To, Yo, so, _ = O.step_stiff(smech, T[:n].copy(), p[:n].copy(), Y[:, :n].copy(), DT, **PARITY_OPTS)
    return To, Yo, so, time.perf_counter() - t0


def cpu_baseline_ann(smech, T, p, Y, sample=4096):
    """The oracle's learned step + props (FP64, numpy matmul and the C oracle) on a sample."""
    import oracle as O
    from oracle import ann as A
    from oracle import mlp as M
    from paper_2312_05800_gb300 import synth
    O.build()
    widths = [smech.N + 2, *HIDDEN[MECH], smech.N - 1]
    layers = synth.mlp_layers(widths, 3003)
    x = M.features(T[:sample], p[:sample], Y[:, :sample])
    mu_x, sd_x = M.zscore_stats(x)
    stats = (mu_x, sd_x, np.zeros(smech.N - 1), np.full(smech.N - 1, 1e-5))
    t0 = time.perf_counter()
    T1, Y1 = A.step_ann(smech, layers, stats, T[:sample].copy(), p[:sample].copy(), Y[:, :sample].copy())
    O.props(smech, T1, p[:sample].copy(), Y1)
    el = time.perf_counter() - t0
    return {"value": sample / el, "unit": "cells/s", "cores": omp_threads(), "kind": "oracle",
            "sample": "first %d of the cells: oracle ANN step (FP64) + props" % sample}


def _oracle_one_core(q, mech_name: str, sample: int):
    """Spawned child: the oracle's learned step + props with every thread pool sized to one."""
    global MECH
    MECH = mech_name
    from paper_2312_05800_gb300 import synth
    smech = synth.get_mech(mech_name)
    T, p, Y = synth.states_profiles(smech, sample, 2003, ld=synth.padded_ld(sample))
    cpu_baseline_ann(smech, T, p, Y, sample)                 # warm: builds and loads the C oracle
    q.put(cpu_baseline_ann(smech, T, p, Y, sample)["value"])


def cpu_baseline_one_core(sample: int = 1024):
    """cells/s of the oracle on one host core: a spawned process whose OpenMP and BLAS pools are set to
    one thread before it loads numpy (a pool forked from this process would carry its threads)."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    import queue as queue_mod
    v, why = None, None
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        proc = ctx.Process(target=_oracle_one_core, args=(q, MECH, sample))
        proc.start()
        t_end = time.time() + 600
        while v is None and time.time() < t_end:
            try:
                v = q.get(timeout=2)
            except queue_mod.Empty:
                if not proc.is_alive():
                    why = "the one-core oracle process exited with code %s" % proc.exitcode
                    break
        if v is None and why is None:
            why = "the one-core oracle run exceeded 600 s"
        proc.join(timeout=30)
        if proc.is_alive():
            proc.terminate()
    except Exception as e:          # the baseline is reported, never allowed to end the run
        why = "one-core oracle run failed: %s" % e
    finally:
        for k, v0 in old.items():
            if v0 is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v0
    if v is None:
        return {"value": None, "unit": "cells/s", "cores": 1, "error": why}
    return {"value": v, "unit": "cells/s", "cores": 1, "sample": "%d cells, same oracle path" % sample}


def main():
    global NCELLS, MECH
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="ann", choices=["ann", "stiff"])
    ap.add_argument("--mech", default=MECH, choices=sorted(HIDDEN),
                    help="mechanism (c2: 30 species, MLP 1600/800/400; c5: 53 species, MLP 2048/1024/512)")
    ap.add_argument("--no-fp8", action="store_true", help="skip the E4M3 variant of the learned step")
    ap.add_argument("--ood-species", default="oxidizer,co2",
                    help="comma-separated species roles of the guard's grids (one grid per role, at most two)")
    ap.add_argument("--chunk", type=int, default=2097152,
                    help="cells per inference chunk of the network (sets the activation workspace)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=None,
                    help="cells per GPU (default 4,194,304 for ann, 2,097,152 for stiff); smaller values only for "
                         "profiling captures")
    ap.add_argument("--train-pairs", type=int, default=2097152)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--ens-lr", type=float, default=1e-3, help="first learning rate of the ensemble's training")
    ap.add_argument("--eval-cells", type=int, default=32768)
    ap.add_argument("--oracle-cells", type=int, default=ORACLE_ACC_CELLS,
                    help="held-out cells integrated by the FP64 oracle on the host cores for the oracle-referenced "
                         "accuracy (the oracle's time grows with the mechanism: fewer for c5)")
    ap.add_argument("--stiff-sample", type=int, default=262144)
    ap.add_argument("--ood-kmin", type=int, default=1,
                    help="training states the 3x3x3 neighbourhood of a cell's bin must hold for the network")
    ap.add_argument("--ens-epochs", type=int, default=30,
                    help="epochs of the per-species ensemble's training (0, or --untrained: no ensemble line)")
    ap.add_argument("--ens-chunk", type=int, default=262144,
                    help="cells per inference chunk of the ensemble (G x 2800 BF16 activations per cell)")
    ap.add_argument("--untrained", action="store_true",
                    help="profiling captures only: skip training and the accuracy check (kernel times do not "
                         "depend on the weights)")
    args = ap.parse_args()
    MECH = args.mech
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    if args.cells is None:
        args.cells = CELLS[(args.path, MECH)]
    NCELLS = args.cells
    if NCELLS % 4:
        raise SystemExit("--cells must be a multiple of 4")
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2312_05800_gb300 import build
    build.build()
    if args.path == "ann":
        line = bench_ann(args, rank, world, local)
    else:
        line = bench_stiff(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
