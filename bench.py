"""Throughput of the over-relaxed diffusive integer lattice gas on GB300.

One bench step = the D2Q5 16384^2 workload (mean 10 per velocity,
omega_eff 1.8, theta 1/3): 500 fused flip+collision+streaming time steps and
the observables at the end (mass, column sums, S(k) and A^LG for axis modes
1..64).  Metric: node updates per second (GNUPS).  The state (5.4 GB
double-buffered) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank advances its own lattice (replica = rank):
weak scaling, no collective on the data path.  --impl reference times the CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_01380_gb300 import inputs  # noqa: E402

METRIC = "GNUPS (node-updates/s) D2Q5 ILG+flip vs HBM roofline; batched vs plain; p99"
BYTES_PER_NU = 20  # read + write of 5 uint16 occupations


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.unlink(self.path)
        except Exception:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample(cfg, side=512, steps=8):
    """The oracle on a side x side window of the workload for `steps` steps
    (light-cone patch from its own initial state).  Returns (node updates, s)."""
    import oracle as O
    ref = O.Lattice(**cfg)
    t0 = time.perf_counter()
    ref.window(0, 0, side, side, steps)
    dt = time.perf_counter() - t0
    nu = sum((side + 2 * (steps - k)) ** 2 for k in range(steps))
    return nu, dt


def run_reference(args, cfg, world, rank):
    if rank != 0:
        return
    side, steps = 512, 8
    oracle_sample(cfg, 64, 2)  # build / load the oracle
    for _ in range(args.warmup):
        oracle_sample(cfg, side, steps)
    tot_nu, tot_t = 0, 0.0
    for _ in range(args.steps):
        nu, dt = oracle_sample(cfg, side, steps)
        tot_nu += nu
        tot_t += dt
    v = tot_nu / tot_t / 1e9
    sample = f"oracle light-cone window {side}x{side} after {steps} steps of the 16384^2 workload (its own initial state)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GNUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic", "config": {"workload": "large_d2q5 (sampled)", "Lx": cfg["Lx"], "Ly": cfg["Ly"]},
            "cpu_baseline": {"value": v, "unit": "GNUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GNUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=inputs.LARGE_D2Q5["Lx"], help="lattice side (default 16384)")
    ap.add_argument("--tsteps", type=int, default=inputs.LARGE_D2Q5["steps"], help="lattice steps per bench step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    cfg = {k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}
    cfg.update(Lx=args.side, Ly=args.side, replica=rank)
    if args.impl == "reference":
        run_reference(args, cfg, world, rank)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2203_01380_gb300 import binding as B

    stream = torch.cuda.current_stream(dev)
    modes = inputs.LARGE_MODES
    T = args.tsteps
    lat = B.Lattice(**cfg, stream=stream)
    lat.init()
    nodes = cfg["Lx"] * cfg["Ly"]

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        lat.step(T)
        lat.observables(modes)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(dev.index) as clk:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for e0, e1, e2 in ev:
            e0.record(stream)
            lat.step(T)
            e1.record(stream)
            obs = lat.observables(modes)
            e2.record(stream)
        end.record(stream)
        barrier()
    total_ms = start.elapsed_time(end)
    step_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    obs_ms = sum(b.elapsed_time(c) for _, b, c in ev)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    nu = float(nodes) * T * args.steps * world
    value = nu / (total_ms / 1e3) / 1e9
    launch_ms = step_ms / (T * args.steps)
    achieved_gbs = nodes * BYTES_PER_NU / (launch_ms / 1e3) / 1e9
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    launches = args.steps * (T + 2)

    e2e = None
    if not args.no_e2e:
        host = torch.empty(lat.size, dtype=torch.uint16, pin_memory=True)
        hnp = host.numpy()
        lat.get_state(hnp.reshape(lat.shape))
        res = torch.empty(lat.size, dtype=torch.uint16, pin_memory=True).numpy()
        barrier()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        e_start.record(stream)
        for _ in range(args.steps):
            lat.set_state(hnp, 0)
            lat.step(T)
            lat.observables(modes)
            lat.get_state(res.reshape(lat.shape))
        e_end.record(stream)
        barrier()
        e_ms = e_start.elapsed_time(e_end)
        if world > 1:
            tt = torch.tensor([e_ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e_ms = float(tt.item())
        e2e = {"value": nu / (e_ms / 1e3) / 1e9, "unit": "GNUPS",
               "h2d_bytes_per_step": int(lat.size * 2 + 8 * len(modes)),
               "d2h_bytes_per_step": int(lat.size * 2 + 8 + 32 * len(modes))}

    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        side, csteps = 512, 8
        oracle_sample(cfg, 64, 2)
        nu_c, dt_c = 0, 0.0
        t_begin = time.perf_counter()
        while time.perf_counter() - t_begin < 10.0:
            n_, d_ = oracle_sample(cfg, side, csteps)
            nu_c += n_
            dt_c += d_
        cpu = {"value": nu_c / dt_c / 1e9, "unit": "GNUPS", "cores": 1, "kind": "oracle",
               "sample": f"oracle (single thread) light-cone windows {side}x{side} after {csteps} steps of the same workload, ~10 s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GNUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": f"large_d2q5: D2Q5 {cfg['Lx']}x{cfg['Ly']}, Poisson mean 10 per velocity, "
                                   f"omega_eff 1.8, {T} steps + observables (S(k), m=1..64) per bench step",
                       "Lx": cfg["Lx"], "Ly": cfg["Ly"], "steps_per_bench_step": T, "modes": len(modes),
                       "parallelism": f"replicas x{world}",
                       "l2": "no flush: the double-buffered state is larger than L2"},
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                         "frac": achieved_gbs / peak, "traffic": None,
                         "kernel": "step_generic_kernel<5>", "launch_ms": launch_ms,
                         "algorithmic_bytes_per_launch": nodes * BYTES_PER_NU},
            "observables_ms_per_step": obs_ms / args.steps,
            "cpu_baseline": cpu,
            "check": {"mass": obs["mass"], "t": obs["t"]},
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
