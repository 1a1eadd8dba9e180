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
import math
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
# random numbers of the method per D2Q5 node update: eight 32-bit words (thinning of
# the five velocities, the rest share, the axis and sign words of the moving
# particles), i.e. two Philox4x32-10 blocks
PHILOX_BLOCKS_PER_NU = 2
SMS = 152
# DRAM bytes (read + write) of one 16384^2 launch of a step kernel, from an ncu
# capture of the same kernel (scaled from a smaller lattice by node count); only
# kernels unchanged since their capture are listed
TRAFFIC_BYTES_PER_LAUNCH = {"seg8": 5.187e9, "warpv8": 5.168e9}


def json_default(o):
    """numpy scalars and arrays in the line as plain JSON values."""
    if hasattr(o, "tolist"):
        return o.tolist()
    raise TypeError(f"{type(o).__name__} is not JSON serialisable")


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
        self._summary = None

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
        if self._summary is None:
            self._summary = self._read()
        return self._summary

    def _read(self):
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


def rank_workload(cfg: dict, rank: int) -> dict:
    """Weak scaling: every rank advances its own lattice of the workload, told apart
    by the replica word of its random numbers."""
    c = dict(cfg)
    c["replica"] = rank
    return c


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (the job's time); no reduction with one rank."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample(cfg, side=512, steps=8, x0=0, y0=0):
    """The oracle on a side x side window of the workload for `steps` steps
    (light-cone patch from its own initial state).  Returns (node updates, s)."""
    import oracle as O
    ref = O.Lattice(**cfg)
    t0 = time.perf_counter()
    ref.window(x0, y0, side, side, steps)
    dt = time.perf_counter() - t0
    nu = sum((side + 2 * (steps - k)) ** 2 for k in range(steps))
    return nu, dt


def oracle_worker(cfg, side, steps, x0, seconds):
    """One process of the all-cores oracle sample: windows at x0, x0 + side, ...
    until `seconds` have passed.  Returns (node updates, busy seconds)."""
    nu, busy, k = 0, 0.0, 0
    while busy < seconds:
        n_, d_ = oracle_sample(cfg, side, steps, (x0 + k * side) % cfg["Lx"], 0)
        nu += n_
        busy += d_
        k += 1
    return nu, busy


def oracle_all_cores(cfg, side, steps, seconds):
    """The oracle, unchanged, in one process per host core (spawned: the parent may
    already hold a CUDA context).  Returns (node updates per second, processes)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        pool.starmap(oracle_sample, [(cfg, 64, 2)] * n)  # load the oracle in every process
        t0 = time.perf_counter()
        res = pool.starmap(oracle_worker, [(cfg, side, steps, k * 997 * side, seconds) for k in range(n)])
        wall = time.perf_counter() - t0
    return sum(r[0] for r in res) / wall, n


KERNEL_NAMES = {"vec8": "step_vec_kernel<5, 8>", "vec4": "step_vec_kernel<5, 4>", "node": "step_kernel<5>",
                "tb2": "step_tb_kernel (depth 2)", "tb4": "step_tb_kernel (depth 4)", "seg8": "step_seg_kernel<5, 8>",
                "warpv8": "step_warp_kernel<5, flip, 64 rows, 8 nodes per lane, 384 threads>",
                "warpv4": "step_warp_kernel<5, flip, 64 rows, 4 nodes per lane, 640 threads>"}


def hbm_roofline(nodes, launch_ms, choice):
    """The HBM roofline of the dominant kernel: every occupation read and written
    once (20 B per D2Q5 node update) per launch, against the measured copy bandwidth."""
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    achieved = nodes * BYTES_PER_NU / (launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(choice), "kernel": KERNEL_NAMES.get(choice, choice),
            "launch_ms": launch_ms, "algorithmic_bytes_per_launch": nodes * BYTES_PER_NU,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if pk else "fallback 6800 GB/s (of fallback)"}


def alu_roofline(B, nodes, launch_ms, stream):
    """The integer bound beside it: the method's random numbers (two Philox4x32-10
    blocks per node update) against the Philox block rate of this GPU, measured here
    by ilg_int_peak (1 s of CUDA-event-timed blocks on every SM); and the rate of an
    even mix of 3-input logic and multiply-add lane-operations for context."""
    ph = B.int_peak(0, 1.0, stream)
    mix = B.int_peak(4, 1.0, stream)
    achieved = PHILOX_BLOCKS_PER_NU * nodes / (launch_ms / 1e3)
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": ph["rate"] / 1e9,
            "unit": "G Philox4x32-10 blocks/s", "frac": achieved / ph["rate"],
            "blocks_per_node_update": PHILOX_BLOCKS_PER_NU,
            "peak_source": "ilg_int_peak kind 0, measured in this run (of measured)",
            "int_lane_ops_peak": {"value": mix["rate"] / 1e12, "unit": "T int32 lane-ops/s",
                                  "kind": "even mix of lop3 and 32-bit multiply-add (ilg_int_peak kind 4)"}}


def measure_batched(torch, B, dev, rings=4096, T=5000, sample=64):
    """4096 D1Q3 rings, 5000 steps in one persistent launch, against one context per
    ring on a stratified sample of the rings (every rings/sample-th ring in order of
    length), each created and initialised before its timing and timed over the same
    5000 steps with CUDA events on its stream; the sampled rings' final states must be
    identical in both runs.  The plain time of all rings is the sample's time scaled by
    rings/sample (each sampled ring stands for that many rings of similar length).
    Fewer rings or steps only for profiling captures."""
    reps = inputs.batch_replicas(rings)
    nodes = sum(r["Lx"] for r in reps)
    st = torch.cuda.Stream(dev)
    by_len = sorted(range(len(reps)), key=lambda i: reps[i]["Lx"])
    idx = [by_len[k] for k in np.linspace(0, len(reps) - 1, min(sample, len(reps))).astype(int)]
    with B.Batch(reps, stream=st) as bat:
        bat.init()
        tuning = bat.autotune(50)
        bat.run(20)
        bat.init()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        bat.run(T)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        batch_states = {i: bat.get_state(i)[0] for i in idx}
    # one context per sampled ring, created and initialised outside the timed region
    with B.Lattice(**reps[idx[-1]], stream=st) as warm:
        warm.init()
        warm.step(50)
    plain_ms, plain_nu, same = 0.0, 0, True
    for i in idx:
        with B.Lattice(**reps[i], stream=st) as lat:
            lat.init()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(st)
            lat.step(T)
            b.record(st)
            torch.cuda.synchronize(dev)
            plain_ms += a.elapsed_time(b)
            plain_nu += reps[i]["Lx"] * T
            same &= bool(np.array_equal(lat.get_state()[0], batch_states[i]))
    v = nodes * T / (ms / 1e3) / 1e9
    plain_all_ms = plain_ms * len(reps) / len(idx)
    return {"workload": f"batch_d1q3: {rings} rings, L log-uniform [64, 8192], n0 uniform [5, 200], "
                        f"omega_eff uniform [0.2, 1.95], {T} steps, one persistent graph-captured launch",
            "value": v, "unit": "GNUPS", "ms": ms, "node_updates": nodes * T,
            "plain_per_ring_launch": {
                "value": plain_nu / (plain_ms / 1e3) / 1e9, "unit": "GNUPS", "ms_sample": plain_ms,
                "ms_all_rings_estimated": plain_all_ms,
                "sample": f"{len(idx)} rings evenly spaced in order of length, one context each, created and "
                          f"initialised before timing, {T} steps each (one launch per step) timed with CUDA events",
                "identical_results": same},
            "speedup_vs_plain": plain_all_ms / ms, "autotune": tuning}


FP64_LANES_PER_SM_CYCLE = 2.0   # GB300 nominal 1.25 TFLOP/s fp64 = 2 fused multiply-add lanes per SM per cycle at 2070 MHz
LB_FP64_OPS_PER_NU = 15         # D2Q5: 4 adds, 2 multiplies, 9 fused multiply-adds, one fp64 lane-op each
LB_BYTES_PER_NU = 80            # 5 doubles read + 5 written


def measure_lb(torch, B, dev, clocks, side=None):
    """Lattice Boltzmann comparator (Sec. IV) on the 16384^2 D2Q5 lattice, 100 steps."""
    cfg = dict(inputs.LB_D2Q5)
    if side:
        cfg.update(Lx=side, Ly=side)
    oj, om = B.lb_rates(cfg["omega_eff"])
    kw = {k: v for k, v in cfg.items() if k not in ("omega_eff", "steps")}
    st = torch.cuda.Stream(dev)
    T = 100
    with B.LB(omega_j=oj, omega=om, stream=st, **kw) as lb:
        lb.init()
        lb.step(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        lb.step(T)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / T
        mass = lb.observables()["mass"]
    nodes = kw["Lx"] * kw["Ly"]
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = FP64_LANES_PER_SM_CYCLE * SMS * mhz * 1e6 / 1e9
    ach = LB_FP64_OPS_PER_NU * nodes / (ms / 1e3) / 1e9
    gbs = LB_BYTES_PER_NU * nodes / (ms / 1e3) / 1e9
    pk = peaks()
    hpk = pk["hbm_gbs"] if pk else 6800.0
    return {"workload": f"lb_d2q5: D2Q5 {kw['Lx']}x{kw['Ly']} fp64, omega^j {oj}, omega {om:.2f}, {T} steps",
            "value": nodes / (ms / 1e3) / 1e9, "unit": "GNUPS", "ms_per_step": ms,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G fp64 lane-ops/s", "frac": ach / peak,
                         "kernel": "lb_step_kernel<5>", "fp64_ops_per_node_update": LB_FP64_OPS_PER_NU,
                         "peak_source": "nominal 1.25 TFLOP/s fp64 (2 FMA lanes per SM per cycle) at the measured SM clock"},
            "hbm": {"achieved": gbs, "peak": hpk, "unit": "GB/s", "frac": gbs / hpk},
            "mass": mass}


def measure_ensemble(torch, B, dev):
    """512 replicas of the L = 320 ring (Sec. V, Fig. 1) for 2000 steps with the
    on-device ensemble statistics of mode 1; the decay of the replica-mean
    amplitude fitted to exp(-D k^2 t) against D = theta (1/omega^j - 1/2)."""
    cfg = dict(inputs.ENSEMBLE_D1Q3)
    R, T = cfg.pop("replicas"), cfg.pop("steps")
    reps = [dict(cfg, replica=r) for r in range(R)]
    st = torch.cuda.Stream(dev)
    with B.Batch(reps, stream=st) as bat:
        bat.init()
        tuning = bat.autotune(50)
        bat.ensemble(10)
        bat.init()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        stats = bat.ensemble(T, mode=1)
        wall = time.perf_counter() - t0
    L = cfg["Lx"]
    amp = stats["mean_im"] / (L / 2.0)
    ts = np.arange(T + 1)
    sel = ts >= 200
    slope = np.polyfit(ts[sel], np.log(amp[sel]), 1)[0]
    k2 = (2 * np.pi / L) ** 2
    oj = cfg["omega_eff"]
    D_theory = cfg["theta"] * (1.0 / oj - 0.5)
    return {"workload": f"ensemble_d1q3: {R} replicas of a D1Q3 ring L={L}, n0 {cfg['n0']:.2f}, sine amplitude "
                        f"{cfg['amp']}, omega_eff {oj}, {T} steps, statistics of mode 1 at every step",
            "value": R * L * T / wall / 1e9, "unit": "GNUPS", "seconds": wall,
            "amplitude": {"t0": float(amp[0]), "t_end": float(amp[-1]),
                          "sd_of_mean_t_end": float(math.sqrt(stats["var_im"][-1] / R) / (L / 2.0))},
            "diffusion": {"fitted": float(-slope / k2), "theory": D_theory, "fit": "ln <A(t)>, t in [200, 2000]"},
            "structure_factor_t0_over_mass": float(stats["cov_re"][0] / (cfg["n0"] * 3 * L)), "autotune": tuning}


def measure_particle(torch, B, dev, side):
    """The main workload with the particle (reference) sampler: one word per particle."""
    cfg = {k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}
    cfg.update(Lx=side, Ly=side, sampler=B.SAMPLER_PARTICLE)
    st = torch.cuda.Stream(dev)
    T = 20
    with B.Lattice(**cfg, stream=st) as lat:
        lat.init()
        lat.step(2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        lat.step(T)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / T
    return {"workload": f"large_d2q5 with the particle sampler: D2Q5 {side}x{side}, {T} steps",
            "value": side * side / (ms / 1e3) / 1e9, "unit": "GNUPS", "ms_per_step": ms,
            "kernel": "step_kernel<5> (general path, one Philox word per particle)"}


def measure_sweep(torch, B, dev):
    """The omega sweep workload as stated: D2Q5 1024^2, mean 50 per velocity + a sine of
    amplitude 20 along x, 1000 steps per omega_eff, each autotuned.  The steps are timed
    with CUDA events; A^LG of mode 1 is read every 10 steps (outside the timed steps) and
    ln A(t) fitted over t in [100, 1000] for the diffusion constant, against
    D = theta (1/omega^j - 1/2) (Sec. IV) and against the lattice Boltzmann comparator's
    mean amplitude from the same initial means (the exact ensemble mean, Sec. IV)."""
    out = {}
    st = torch.cuda.Stream(dev)
    every = 10
    for c in inputs.SWEEP_D2Q5:
        T = c["steps"]
        cfg = {k: v for k, v in c.items() if k != "steps"}
        k2 = (2.0 * math.pi / cfg["Lx"]) ** 2
        with B.Lattice(**cfg, stream=st) as lat:
            lat.init()
            tun = lat.autotune(10)
            ts, amps, step_ms = [0], [lat.observables([(1, 0)])["amp"][0]], 0.0
            for k in range(T // every):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                lat.step(every)
                e1.record(st)
                torch.cuda.synchronize(dev)
                step_ms += e0.elapsed_time(e1)
                ts.append((k + 1) * every)
                amps.append(lat.observables([(1, 0)])["amp"][0])
        oj, om = B.lb_rates(cfg["omega_eff"])
        with B.LB(omega_j=oj, omega=om, stream=st, **cfg) as lb:
            lb.init()
            lb.step(T)
            a_lb = float(lb.observables([(1, 0)])["amp"][0])
        ts, amps = np.array(ts, dtype=float), np.array(amps)
        sel = ts >= 100
        (slope, icpt), cov = np.polyfit(ts[sel], np.log(amps[sel]), 1, cov=True)
        D_theory = cfg["theta"] * (1.0 / oj - 0.5)
        rho = cfg["n0"] * 5
        out[str(cfg["omega_eff"])] = {
            "value": cfg["Lx"] * cfg["Ly"] * T / (step_ms / 1e3) / 1e9, "unit": "GNUPS", "ms_per_step": step_ms / T,
            "kernel": tun["choice"],
            "diffusion": {"fitted": float(-slope / k2), "stderr": float(math.sqrt(cov[0, 0]) / k2),
                          "theory": D_theory, "fit": f"ln A^LG(t), t in [100, {T}], every {every} steps"},
            "amplitude": {"t0": float(amps[0]), "t_end": float(amps[-1]), "lb_mean_t_end": a_lb,
                          "sd_single_sample": math.sqrt(2.0 * rho / (cfg["Lx"] * cfg["Ly"]))}}
    return {"workload": "sweep_d2q5: D2Q5 1024x1024, Poisson mean 50 per velocity + sine amplitude 20, "
                        "1000 steps per omega_eff (0.5, 1.0, 1.5, 1.9)", "omega_eff": out}


def measure_ring(torch, B, dev):
    """The D1Q3 ring workload as stated: L = 256, mean 30 per velocity + a sine of
    amplitude 10, omega_eff 1.5, 2000 steps, the full state and the mode-1 amplitude
    after every step.  Through ilg_batch_run_record (one ring held in shared memory
    for all steps, the states and amplitudes recorded on the device, one copy to the
    host; wall clock of the whole call), and through one context stepping once per
    call with the state and the amplitude read back after every step."""
    cfg = {k: v for k, v in inputs.RING_D1Q3.items() if k != "steps"}
    T = inputs.RING_D1Q3["steps"]
    L = cfg["Lx"]
    st = torch.cuda.Stream(dev)
    with B.Batch([cfg], stream=st) as bat:
        bat.init()
        bat.run_record(T)          # graph capture and the record's allocation
        bat.init()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        amp, states = bat.run_record(T, 1)
        wall = time.perf_counter() - t0
    lat_s = []
    with B.Lattice(**cfg, stream=st) as lat:
        lat.init()
        buf = np.empty(lat.shape, dtype=np.uint16)
        for _ in range(T):
            t0 = time.perf_counter()
            lat.step(1)
            a_ctx = lat.observables([(1, 0)])["amp"][0]
            lat.get_state(buf)
            lat_s.append(time.perf_counter() - t0)
    same = bool(np.array_equal(states[0][-1], buf)) and bool(abs(a_ctx - amp[0][-1]) <= 1e-12 * max(1.0, abs(a_ctx)))
    lat_s = np.array(lat_s)
    return {"workload": f"ring_d1q3: D1Q3 ring L={L}, Poisson mean 30 per velocity + sine amplitude 10, omega_eff 1.5, "
                        f"{T} steps, state and A^LG of mode 1 after every step",
            "value": L * T / wall / 1e9, "unit": "GNUPS", "latency_per_step_us": 1e6 * wall / T,
            "call_s": wall, "path": "ilg_batch_run_record (wall clock, host copy of the 3 MB record included)",
            "one_context_one_step_per_call": {
                "value": L * T / lat_s.sum() / 1e9, "unit": "GNUPS",
                "latency_us": {"p50": float(1e6 * np.percentile(lat_s, 50)), "p99": float(1e6 * np.percentile(lat_s, 99))}},
            "amplitude": {"t1": float(amp[0][0]), "t_end": float(amp[0][-1])}, "identical_results": same}


def measure_d2q9(torch, B, dev, side):
    """The D2Q9 lattice (9 velocities, product weights) on the main workload's size,
    through the default staged warp step and the other applicable step kernels, each
    event-timed on its own context from the same initial state (identical results:
    the same mass and mode amplitudes after the same steps)."""
    cfg = {k: v for k, v in inputs.LARGE_D2Q9.items() if k != "steps"}
    cfg.update(Lx=side, Ly=side)
    st = torch.cuda.Stream(dev)
    T = 20
    nodes = side * side
    pk = peaks()
    hpk = pk["hbm_gbs"] if pk else 6800.0
    names = {6: "step_warp_kernel<9>, 4-node vectors collided in shared memory, 512 threads per SM (default)",
             7: "step_warp_kernel<9>, 4-node vectors collided in shared memory, 640 threads per SM",
             2: "step9_pair_kernel (node-parallel, two nodes of a row per thread)"}
    kernels, obs = {}, []
    for cand in (6, 7, 2):
        with B.Lattice(**cfg, stream=st) as lat:
            lat.set_step_kernel(cand)
            lat.init()
            lat.step(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(st)
            lat.step(T)
            e1.record(st)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / T
            o = lat.observables(modes=[(1, 0), (0, 1), (5, 0)])
            obs.append((o["mass"], tuple(o["re"]), tuple(o["im"])))
        kernels[cand] = {"kernel": names[cand], "value": nodes / (ms / 1e3) / 1e9, "ms_per_step": ms}
    best = kernels[6]
    gbs = 36 * nodes / (best["ms_per_step"] / 1e3) / 1e9
    return {"workload": f"large_d2q9: D2Q9 {side}x{side}, Poisson mean 10 per velocity, omega_eff 1.8, {T} steps",
            "value": best["value"], "unit": "GNUPS", "ms_per_step": best["ms_per_step"],
            "hbm": {"achieved": gbs, "peak": hpk, "unit": "GB/s", "frac": gbs / hpk,
                    "bytes_per_node_update": 36},
            "kernel": best["kernel"],
            "kernels": {k["kernel"]: {"value": k["value"], "ms_per_step": k["ms_per_step"]} for k in kernels.values()},
            "identical_results": bool(all(x == obs[0] for x in obs))}


def measure_e2e_one_context(torch, lat, args, modes, stream, dev, world, nu, barrier):
    """The e2e metric through one context: every bench step copies its state in from and
    out to pinned host memory around its steps and observables, one after another."""
    host = torch.empty(lat.size, dtype=torch.uint16, pin_memory=True).numpy()
    lat.get_state(host.reshape(lat.shape))
    res = torch.empty(lat.size, dtype=torch.uint16, pin_memory=True).numpy()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lat.set_state(host, 0)
        lat.step(args.tsteps)
        lat.observables(modes)
        lat.get_state(res.reshape(lat.shape))
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    return {"value": nu / (ms / 1e3) / 1e9, "unit": "GNUPS",
            "h2d_bytes_per_step": int(lat.size * 2 + 8 * len(modes)),
            "d2h_bytes_per_step": int(lat.size * 2 + 8 + 32 * len(modes)),
            "how": "one context: each bench step's state copied in from and out to pinned host memory "
                   "through ilg_set_state / ilg_get_state around its steps"}


def measure_e2e(torch, B, lat, cfg, args, modes, stream, dev, world, nu, barrier):
    """The metric end to end through the C ABI with host buffers: every bench step
    copies its initial state in from pinned host memory (ilg_set_state), takes its
    steps and observables, and copies the final state out (ilg_get_state).  Two
    contexts on two streams, each driven by its own host thread, take alternate bench
    steps, so one step's copies overlap the other's kernels (each result is the one a
    single context gives: the same input, the same counter-keyed random numbers)."""
    st2 = torch.cuda.Stream(dev)
    lat2 = B.Lattice(**cfg, stream=st2)
    if args.kernel:
        lat2.set_step_kernel(B.CONTEXT_CANDIDATES.index(args.kernel))
    else:
        lat2.init()
        lat2.autotune(20)
    host = torch.empty(lat.size, dtype=torch.uint16, pin_memory=True).numpy()
    lat.get_state(host.reshape(lat.shape))
    res = [torch.empty(lat.size, dtype=torch.uint16, pin_memory=True).numpy() for _ in range(2)]
    lats = [lat, lat2]
    T = args.tsteps

    def bench_step(i, before=None, done=None):
        lats[i].set_state(host, 0)
        if before is not None:
            before.wait()  # the previous bench step's kernels have finished
        lats[i].step(T)
        if done is not None:
            done.set()
        lats[i].observables(modes)
        lats[i].get_state(res[i].reshape(lat.shape))

    errors = []
    # bench step k takes its steps only after step k - 1 has taken its own, so the two
    # contexts' kernels run one after the other and each step's copies overlap the
    # other context's kernels instead of coinciding with them
    stepped = [threading.Event() for _ in range(args.steps)]

    def worker(i):
        try:
            for k in range(i, args.steps, 2):
                bench_step(i, stepped[k - 1] if k > 0 else None, stepped[k])
        except Exception as ex:  # reported after the join
            errors.append(ex)
            for ev in stepped:
                ev.set()

    bench_step(1)  # the second context's warm-up
    barrier()
    e_start, e_end, e_b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e_start.record(stream)
    st2.wait_event(e_start)
    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    e_b.record(st2)
    stream.wait_event(e_b)
    e_end.record(stream)
    barrier()
    if errors:
        raise errors[0]
    same = bool(np.array_equal(res[0], res[1])) if args.steps > 1 else True
    e_ms = max_over_ranks(e_start.elapsed_time(e_end), world, dev)
    lat2.close()
    # the same bench steps one after another through the one context (no overlap)
    s_start, s_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    s_start.record(stream)
    for _ in range(args.steps):
        bench_step(0)
    s_end.record(stream)
    barrier()
    s_ms = max_over_ranks(s_start.elapsed_time(s_end), world, dev)
    return {"value": nu / (e_ms / 1e3) / 1e9, "unit": "GNUPS",
            "h2d_bytes_per_step": int(lat.size * 2 + 8 * len(modes)),
            "d2h_bytes_per_step": int(lat.size * 2 + 8 + 32 * len(modes)),
            "how": "two contexts on two streams take alternate bench steps from two host threads, each "
                   "step's kernels after the previous step's; each step's state copied in from and out to "
                   "pinned host memory through ilg_set_state / ilg_get_state, its copies overlapping the "
                   "other context's kernels",
            "identical_results": same,
            "one_context": {"value": nu / (s_ms / 1e3) / 1e9, "unit": "GNUPS",
                            "how": "the same bench steps in sequence through one context"}}


def serve_stream(B, reqs, slots, smallest_first):
    """Submit requests at their arrival times; returns results, wall time, stats."""
    with B.Server(5, 48 << 30, max_slots=slots, quantum=32) as srv:
        srv.set_policy(smallest_first)
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            dt = r["arrive"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            srv.submit(i, **{k: v for k, v in r.items() if k != "arrive"})
        srv.wait_idle(1800)
        wall = time.perf_counter() - t0
        res = srv.poll(4096)
        st = srv.stats()
    return res, wall, st


def latency_summary(res):
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    queue = np.array([r["t_admit"] - r["t_submit"] for r in res])
    return ({"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            {"p50": float(np.percentile(queue, 50)), "p99": float(np.percentile(queue, 99))})


def measure_serving(torch, B, dev, n_requests=200):
    """Poisson arrivals (200/s) of D2Q5 requests, submitted in real time: every
    request admitted at once (arrival order), and least-work-first admission into 32
    slots; against the same requests run one after another, one context each (created
    and initialised outside the timing, each request's steps timed with CUDA events),
    at identical results (mass and A^LG of every request)."""
    reqs = inputs.serve_requests(n_requests)
    tot = sum(r["Lx"] * r["Ly"] * r["steps"] for r in reqs)
    res, wall, st = serve_stream(B, reqs, 512, False)
    lat_all, queue_all = latency_summary(res)
    res2, wall2, st2 = serve_stream(B, reqs, 32, True)
    lat_sm, queue_sm = latency_summary(res2)
    served = {r["id"]: r for r in res}
    stream = torch.cuda.Stream(dev)
    plain_ms, same = 0.0, True
    for i, r in enumerate(reqs):
        with B.Lattice(**{k: v for k, v in r.items() if k not in ("arrive", "steps")}, stream=stream) as one:
            one.init()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            one.step(r["steps"])
            b.record(stream)
            torch.cuda.synchronize(dev)
            plain_ms += a.elapsed_time(b)
            o = one.observables([(1, 0)])
            same &= bool(served[i]["mass"] == o["mass"]) and bool(served[i]["amp"] == o["amp"][0])
    return {"workload": f"serve_d2q5: {n_requests} requests, Poisson arrivals 200/s, side log-uniform [64, 2048], "
                        "steps log-uniform [100, 10000], n0 uniform [5, 100], omega_eff 1.5",
            "aggregate": {"value": tot / wall / 1e9, "unit": "GNUPS"}, "offered_node_updates": tot,
            "latency_s": lat_all, "queueing_s": queue_all,
            "completed": len(res), "wall_s": wall, "peak_resident": st["peak_resident"],
            "least_work_first_32_slots": {"aggregate": {"value": tot / wall2 / 1e9, "unit": "GNUPS"},
                                          "latency_s": lat_sm, "queueing_s": queue_sm, "completed": len(res2),
                                          "wall_s": wall2},
            "one_context_per_request": {
                "value": tot / (plain_ms / 1e3) / 1e9, "unit": "GNUPS", "steps_s": plain_ms / 1e3,
                "how": "every request alone in turn, created and initialised outside the timing, its steps timed "
                       "with CUDA events (no arrival times: the GPU time of the plain launches alone)",
                "identical_results": bool(same)},
            "speedup_vs_one_context_per_request": (plain_ms / 1e3) / wall}


def main_config(cfg, T, nmodes, world):
    """The `config` object of both arms' lines: the main workload."""
    return {"workload": f"large_d2q5: D2Q5 {cfg['Lx']}x{cfg['Ly']}, Poisson mean 10 per velocity, "
                        f"omega_eff 1.8, {T} steps + observables (S(k), m=1..{nmodes}) per bench step",
            "Lx": cfg["Lx"], "Ly": cfg["Ly"], "steps_per_bench_step": T, "modes": nmodes,
            "parallelism": f"replicas x{world}",
            "l2": "no flush: the double-buffered state is larger than L2"}


def run_reference(args, cfg, world, rank):
    """The oracle as the reference arm: every step runs one light-cone window per host
    core, in parallel processes (spawned), on the same workload."""
    if rank != 0:
        return
    import multiprocessing as mp
    side, steps = 512, 8
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    tot_nu, tot_t = 0, 0.0
    with ctx.Pool(n) as pool:
        pool.starmap(oracle_sample, [(cfg, 64, 2)] * n)  # build / load the oracle everywhere
        jobs = [(cfg, side, steps, (k * 997 * side) % cfg["Lx"], 0) for k in range(n)]
        for _ in range(args.warmup):
            pool.starmap(oracle_sample, jobs)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            res = pool.starmap(oracle_sample, jobs)
            tot_t += time.perf_counter() - t0
            tot_nu += sum(r[0] for r in res)
    v = tot_nu / tot_t / 1e9
    sample = (f"oracle light-cone windows {side}x{side} after {steps} steps of the 16384^2 workload (its own "
              f"initial state), one window per host core per step, {n} processes")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GNUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic", "config": main_config(cfg, args.tsteps, len(inputs.LARGE_MODES), world),
            "cpu_baseline": {"value": v, "unit": "GNUPS", "cores": n, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GNUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=inputs.LARGE_D2Q5["Lx"], help="lattice side (default 16384)")
    ap.add_argument("--side-y", type=int, default=0, help="rows of the lattice (default: --side; profiling only)")
    ap.add_argument("--tsteps", type=int, default=inputs.LARGE_D2Q5["steps"], help="lattice steps per bench step")
    ap.add_argument("--kernel", default="", choices=["", "vec8", "vec4", "node", "seg8", "warpv8", "warpv4"],
                    help="fixed single-step kernel instead of the autotuner's choice (profiling: under ncu the "
                         "tuner's timings are not the run's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip every measurement beyond the main workload")
    ap.add_argument("--extra", default="tb,batched,lb,ensemble,particle,d2q9,sweep,ring,serving",
                    help="comma-separated measurements beyond the main workload")
    ap.add_argument("--lb-side", type=int, default=0, help="side of the lattice Boltzmann workload (default 16384)")
    ap.add_argument("--batch-rings", type=int, default=4096, help="rings of the batched workload (profiling only)")
    ap.add_argument("--batch-steps", type=int, default=5000, help="steps of the batched workload (profiling only)")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests of the serving workload (profiling only)")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    cfg = {k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}
    cfg.update(Lx=args.side, Ly=args.side_y or args.side)
    cfg = rank_workload(cfg, rank)
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
    if args.kernel:
        lat.set_step_kernel(B.CONTEXT_CANDIDATES.index(args.kernel))
        tuning = {"choice": args.kernel, "fixed": True}
    else:
        tuning = lat.autotune(20)   # launch shape chosen by timing (outside the timed region)

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
    total_ms = max_over_ranks(start.elapsed_time(end), world, dev)
    step_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    obs_ms = sum(b.elapsed_time(c) for _, b, c in ev)
    nu = float(nodes) * T * args.steps * world
    value = nu / (total_ms / 1e3) / 1e9
    launch_ms = step_ms / (T * args.steps)
    launches = args.steps * (T + 2)

    e2e = None
    if not args.no_e2e:
        try:
            e2e = measure_e2e(torch, B, lat, cfg, args, modes, stream, dev, world, nu, barrier)
        except (RuntimeError, MemoryError, B.IlgError) as ex:
            # a second context or three pinned state buffers did not fit: one context alone
            torch.cuda.synchronize(dev)
            e2e = measure_e2e_one_context(torch, lat, args, modes, stream, dev, world, nu, barrier)
            e2e["pipelined_unavailable"] = str(ex).splitlines()[0][:200]

    alu = alu_roofline(B, nodes, launch_ms, stream) if rank == 0 else None

    extra = {}
    if rank == 0 and world == 1 and not args.no_modes:
        # temporal blocking on the same workload: steps per launch against single steps
        tb = {}
        parts = set(args.extra.split(","))
        for depth in ((2, 4) if "tb" in parts else ()):
            lat.set_temporal_blocking(depth)
            lat.step(2 * depth)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            ea.record(stream)
            lat.step(100)
            eb.record(stream)
            torch.cuda.synchronize(dev)
            tb[str(depth)] = {"value": nodes * 100 / (ea.elapsed_time(eb) / 1e3) / 1e9, "unit": "GNUPS"}
        lat.set_temporal_blocking(0)
        if tb:
            extra["temporal_blocking"] = {"steps_per_launch": tb, "single_step_kernel": {"value": value, "unit": "GNUPS"},
                                          "tile": "44 - 2 depth nodes per side, with a halo of depth nodes"}
        if "batched" in parts:
            extra["batched"] = measure_batched(torch, B, dev, args.batch_rings, args.batch_steps)
        if "lb" in parts:
            extra["lattice_boltzmann"] = measure_lb(torch, B, dev, clk.summary(), args.lb_side)
        if "ensemble" in parts:
            extra["ensemble"] = measure_ensemble(torch, B, dev)
        if "particle" in parts:
            extra["particle_sampler"] = measure_particle(torch, B, dev, args.side)
        if "d2q9" in parts:
            extra["d2q9"] = measure_d2q9(torch, B, dev, args.side)
        if "sweep" in parts:
            extra["sweep"] = measure_sweep(torch, B, dev)
        if "ring" in parts:
            extra["ring"] = measure_ring(torch, B, dev)
        if "serving" in parts:
            extra["serving"] = measure_serving(torch, B, dev, args.serve_requests)

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
        rate, nproc = oracle_all_cores(cfg, side, csteps, 10.0)
        cpu = {"value": rate / 1e9, "unit": "GNUPS", "cores": nproc, "kind": "oracle",
               "sample": f"oracle light-cone windows {side}x{side} after {csteps} steps of the same workload, "
                         f"one process per host core for ~10 s each",
               "single_thread": {"value": nu_c / dt_c / 1e9, "unit": "GNUPS", "cores": 1,
                                 "sample": f"the same windows in one thread, ~10 s"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GNUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": main_config(cfg, T, len(modes), world),
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": launches,
            "autotune": tuning,
            "roofline": hbm_roofline(nodes, launch_ms, tuning["choice"]),
            "alu_roofline": alu,
            "observables_ms_per_step": obs_ms / args.steps,
            "cpu_baseline": cpu,
            **extra,
            "check": {"mass": obs["mass"], "t": obs["t"]},
        }
        print(json.dumps(line, default=json_default), flush=True)
    lat.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
