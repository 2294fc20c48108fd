#!/usr/bin/env python
"""Benchmark of the per-cell chemistry + properties step (arXiv 2312.05800).

One step = one pass of the hot path over one batch of synthetic cells: the
composition advanced over dt = 1 us and the properties of the advanced state.

Workload (seeded, synthetic): the 30-species / 180-reaction C/H/O/N
mechanism, 2,097,152 cells sampled along algebraic stratified premixed
profiles (phi 0.5-1.2, 5 % log-normal Y noise), 1 atm. Inputs (about 0.5 GB
of FP64 state) are larger than L2, so no flush is needed between steps.

Paths (see --path): "stiff" = chem_step_stiff (FP64 Rodas3 at rtol 1e-3, the
loosest setting tried; its error against a tight integration is far inside the
ANN bars) followed by props_eval (FP32 arithmetic on the FP64 state).

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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NCELLS = 2097152
DT = 1.0e-6
STIFF_OPTS = dict(rtol=1e-3, atol_Y=1e-9, atol_T=1e-3, h0=1e-9, max_steps=10000)
MECH = "c2"
SEED = 2002
METRIC = "chem+props cells/s at stated dY/T error: ANN (BF16/FP8) vs stiff integrator, 1 GB300"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk/SM x 2 flop x max SM clock


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


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


def make_inputs(rank: int, ncells: int = NCELLS):
    from paper_2312_05800_gb300 import synth
    mech = synth.get_mech(MECH)
    T, p, Y = synth.states_profiles(mech, ncells, SEED + 1000 * rank, ld=synth.padded_ld(ncells))
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
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle as O
    O.build()
    mech, T, p, Y = make_inputs(0)
    sample = 4096
    for _ in range(args.warmup):
        run_cpu_oracle(mech, T, p, Y, sample)
    times = [run_cpu_oracle(mech, T, p, Y, sample) for _ in range(args.steps)]
    v = sample / statistics.median(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c2 stratified-profile cells, 30 species / 180 reactions, dt 1 us",
                       "path": "stiff+props", "cells_per_step": sample, "rtol": STIFF_OPTS["rtol"]},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": omp_threads(), "kind": "oracle",
                             "sample": "first %d of the %d cells per step" % (sample, NCELLS)},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global NCELLS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="stiff", choices=["stiff"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=NCELLS,
                    help="cells per GPU; smaller values only for profiling captures (the bench line uses the default)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    NCELLS = args.cells
    if NCELLS % 4:
        raise SystemExit("--cells must be a multiple of 4")
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2312_05800_gb300 import binding, build
    build.build()
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
    opts = binding.make_opts(**STIFF_OPTS)
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
    if world > 1:
        torch.distributed.barrier()
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
    if world > 1:
        torch.distributed.barrier()
    step_ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]
    kern_ms = [kev[2 * i].elapsed_time(kev[2 * i + 1]) for i in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * NCELLS * args.steps / total_s
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

    flops_step = stiff_flops_per_step(N, mech.R, int((mech.rtype != 0).sum()), int((mech.rtype == 2).sum()))
    kern_s = statistics.mean(kern_ms) / 1e3
    achieved = steps_total * flops_step / kern_s / 1e12
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c2 stratified-profile cells, 30 species / 180 reactions, dt 1 us",
                       "path": "stiff+props (FP64 Rodas3 rtol 1e-3, FP32 props)", "cells_per_gpu": NCELLS,
                       "l2": "inputs larger than L2 (0.5 GB FP64 state)",
                       "mean_steps_per_cell": steps_total / NCELLS, "parallelism": "replicas" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "kernel": "stiff_kernel", "flops_per_step": flops_step,
                         "peak_source": "FP64 nominal: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz"},
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
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
