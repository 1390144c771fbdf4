"""Benchmark: fused FP32 fluctuating D3Q19 LB + bead-spring chain step on GB300, in MLUPS
(million lattice-node updates per second) and as a fraction of the HBM roofline, beside the
plain FP64 path on the same GPU and the FP64 CPU oracle.

Workload: L = 128 periodic box (2,097,152 nodes), rho = 1, eta = eta_b = 3, kT = 1, a = 1,
h = 0.01, one chain of N = 128 beads (m = 1, FENE k = 30, R0 = 1.5, WCA eps = sigma = 1,
zeta = 20.8) started as a self-avoiding walk with bond 0.97, fluid at rest, full
thermalization, seed 3.  The two population buffers (2 x 159 MB in FP32) are larger than
the 129 MB L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank runs an independent replica of the
workload (own seed): the method has no exchange between independent boxes, so the job
scales weakly with no data-path collective; the MAX of the ranks' timed regions is used.
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
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline: fused FP32 LB+chain vs plain FP64, same GPU"
L_BENCH, N_BENCH, SEED = 128, 128, 3
PARAMS = dict(rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0)
CHAIN = dict(m=1.0, zeta=20.8, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0)
BYTES_PER_NODE = {"f32": 19 * 4 * 2, "f64": 19 * 8 * 2, "bf16": 19 * 2 * 2}  # algorithmic: 19 reads + 19 writes
# FP64 operations per node update of the plain FP64 kernel with noise (ncu op counts at L = 128:
# (DADD + DMUL + 2 DFMA) / nodes = 2.223e9 / 2,097,152); that kernel is bound by FP64 arithmetic
FP64_FLOPS_PER_NODE = 797
# GB300's dense FP64 rate: 152 SMs x 2 FP64 FMA per SM and clock x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 1.26
KERNEL_SOURCES = ["paper_0903_5067_gb300/csrc/lb_device.cuh", "paper_0903_5067_gb300/csrc/d3q19.cuh",
                  "paper_0903_5067_gb300/csrc/philox.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "lb_step_f32_L128_traffic.json")


def workload_name(L=L_BENCH, N=N_BENCH):
    return (f"fluctuating D3Q19 LB, periodic L={L} box ({L ** 3:,} nodes) + FENE/WCA chain N={N}, "
            f"full thermalization, 1 coupled step = 1 LB + 1 MD step")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic():
    """DRAM bytes per launch of the FP32 LB kernel from the committed ncu summary, or None
    when the kernel sources changed since it was taken."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as fh:
        d = json.load(fh)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling while the timed work runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, directory: str | None = None):
        import tempfile

        self.index = index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        if not rows:
            return None
        powered = [r for r in rows if r[2] > 0.5 * max(x[2] for x in rows)] or rows
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, flag in zip(names, r[3]):
                if flag.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in powered), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(powered)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """MAX of a per-rank scalar over the job (identity when ws == 1)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, seconds: float, ws: int, device=None):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    tmax = max_over_ranks(seconds, ws, device)
    return units_per_rank * ws / tmax, tmax


_ORACLE_WORKER = """
import os, sys, time, json
sys.path.insert(0, {root!r})
from oracle import lbchain as o
from paper_0903_5067_gb300 import inputs
fp = o.FluidParams(L={L}, seed={seed}, **{params!r})
cp = o.ChainParams(N={N}, **{chain!r})
st = o.init_state(fp, cp, inputs.chain_walk({N}, L={L}, bond=0.97, seed={seed}, self_avoiding=True))
st = o.run(st, fp, cp, {warmup})
print("READY", flush=True)
sys.stdin.readline()
t = time.perf_counter()
st = o.run(st, fp, cp, {steps})
print(json.dumps({{"seconds": time.perf_counter() - t}}), flush=True)
"""


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu), for the baseline's record."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine() or "unknown"


def host_memory_bytes() -> int:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def cpu_oracle_run(L: int, N: int, steps: int, procs: int = 1, warmup: int = 0, seed: int = SEED,
                   timeout: float = 900.0):
    """Time the FP64 oracle as it stands on `procs` host cores: `procs` fresh single-threaded
    processes, each an independent replica of the workload on an L^3 box (seeds seed, seed+1,
    ...), each running `warmup` untimed steps, then released together for `steps` timed
    coupled steps.  Returns (seconds of the slowest process, node updates of all processes)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1")
    ps = []
    try:
        for p in range(procs):
            code = _ORACLE_WORKER.format(root=ROOT, L=L, N=N, seed=seed + p, params=PARAMS, chain=CHAIN,
                                         warmup=warmup, steps=steps)
            ps.append(subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                                       stderr=subprocess.PIPE, text=True, env=env))
        t_end = time.time() + timeout
        for pr in ps:  # every replica initialised and warmed up
            line = pr.stdout.readline()
            if line.strip() != "READY" or time.time() > t_end:
                raise RuntimeError("oracle worker failed: " + pr.stderr.read()[-2000:])
        for pr in ps:
            pr.stdin.write("GO\n")
            pr.stdin.flush()
        secs = []
        for pr in ps:
            out, err = pr.communicate(timeout=max(1.0, t_end - time.time()))
            if pr.returncode != 0:
                raise RuntimeError("oracle worker failed: " + err[-2000:])
            secs.append(json.loads(out.strip().splitlines()[-1])["seconds"])
    finally:
        for pr in ps:
            if pr.poll() is None:
                pr.kill()
    return max(secs), procs * L ** 3 * steps


def cpu_oracle_sample(L: int, N: int, steps: int, seed: int, timeout: float = 900.0, warmup: int = 0):
    """Seconds per coupled step of the FP64 oracle on one host core (see cpu_oracle_run)."""
    t, _ = cpu_oracle_run(L, N, steps, 1, warmup, seed, timeout)
    return t / steps


def oracle_procs(L: int) -> int:
    """Host cores for the all-core oracle timing: every core, but no more replicas than half
    the host memory holds (the oracle needs about 1.5 KB per node of an L^3 box)."""
    cores = os.cpu_count() or 1
    mem = host_memory_bytes()
    if mem:
        cores = max(1, min(cores, int(0.5 * mem / (1500.0 * L ** 3))))
    return cores


def cpu_baseline_record():
    """The oracle on the full L=128, N=128 workload: one step single-threaded, and one step on
    every host core (independent replicas, released together)."""
    t1, n1 = cpu_oracle_run(L_BENCH, N_BENCH, 1, 1)
    P = oracle_procs(L_BENCH)
    tp, npn = cpu_oracle_run(L_BENCH, N_BENCH, 1, P)
    return {"value": npn / tp / 1e6, "unit": "MLUPS", "cores": P, "kind": "oracle", "cpu_model": cpu_model(),
            "host_cores": os.cpu_count(),
            "sample": f"1 coupled step of the full L={L_BENCH}, N={N_BENCH} workload (FP64) in each of {P} "
                      f"single-threaded processes (independent replicas) released together; value = node "
                      f"updates of all of them / the slowest one's time",
            "single_thread": {"value": n1 / t1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": f"1 coupled step of the full L={L_BENCH}, N={N_BENCH} workload, FP64"}}


def run_reference(args):
    """The FP64 oracle on the host cores, same workload/metric/unit: every core runs an
    independent replica (its own seed), all released together; each step a sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    budget = 150.0  # seconds for the timed and warm-up steps together
    L = L_BENCH
    P = oracle_procs(L)
    probe, _ = cpu_oracle_run(L, N_BENCH, 1, P)

    def chain_for(Ls):
        return N_BENCH if Ls >= 64 else (64 if Ls >= 32 else 8)

    sample = f"full L={L} workload per core, 1 coupled step per step"
    if probe * (args.steps + args.warmup) > budget:
        for Ls in (96, 64, 48, 32, 24, 16):
            L = Ls
            P = oracle_procs(L)
            probe, _ = cpu_oracle_run(L, chain_for(L), 1, P)
            if probe * (args.steps + args.warmup) <= budget:
                break
        sample = f"L={L} sub-box of the workload per core (same fluid, chain N={chain_for(L)}), 1 coupled step per step"
    t, nodes = cpu_oracle_run(L, chain_for(L), args.steps, P, warmup=args.warmup, timeout=3600)
    value = nodes / t / 1e6
    sample += f"; {P} single-threaded processes (independent replicas, seeds {SEED}..{SEED + P - 1}) released together"
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "L": L_BENCH, "N": N_BENCH, "seed": SEED},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": P, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge

    ge.build()
    from paper_0903_5067_gb300 import inputs, lb

    # CPU baseline first (a fresh process, before this process does GPU work)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record()

    L, N, seed = L_BENCH, N_BENCH, SEED + 1000 * rank
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)

    def make(prec):
        sim = lb.Simulation(L=L, seed=seed, precision=prec, **PARAMS)
        sim.add_chain(N, x0=X0, **CHAIN)
        return sim

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    sim = make(lb.LB_FP32)
    sim.step(args.warmup)
    sim.sync()

    clocks = ClockSampler(local, args.clocks_dir)
    with clocks:
        # timed region: K fused steps, inputs resident in HBM
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        barrier()
        t32 = e0.elapsed_time(e1) / 1e3
        sim.sync()
        # roofline pass: events around every LB launch (same stream)
        lb.lb_set_timing(sim.ctx, True)
        sim.step(args.steps)
        ms_k, nk = lb.lb_get_timing(sim.ctx)
        lb.lb_set_timing(sim.ctx, False)
        sim.sync()
        # plain FP64 path on the same GPU, same workload
        k64 = max(3, args.steps // 20)
        s64 = make(lb.LB_FP64)
        s64.step(max(1, args.warmup // 20))
        s64.sync()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(k64)
        f1.record(stream)
        barrier()
        t64 = f0.elapsed_time(f1) / 1e3
        s64.sync()
        s64.close()
    obs = sim.observables()
    sim.close()

    # batched replicas: the 64-box ensemble (5,242,368 nodes per step), autotuned tile shape,
    # 16-step CUDA graphs; whole-ensemble MLUPS
    batch = None
    if not args.no_batch:
        bL, bN, bseeds, bX = inputs.c4_ensemble(base_seed=100 + 1000 * rank)
        bt = lb.Batch(bL, bN, bseeds, bX, precision=lb.LB_FP32, **PARAMS, **CHAIN)
        shape = lb.lb_batch_autotune(bt.b)
        kb = max(32, (args.steps // 10) // 16 * 16)
        bt.step(32)
        bt.sync()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        bt.step(kb)
        g1.record(stream)
        barrier()
        tb = g0.elapsed_time(g1) / 1e3
        bt.sync()
        nodes = lb.lb_batch_nodes(bt.b)
        bt.close()
        bval, _ = aggregate_throughput(nodes * kb / 1e6, tb, ws, dev)
        batch = {"value": bval, "unit": "MLUPS", "replicas": len(bL), "nodes_per_step": nodes, "steps": kb,
                 "ms_per_step": tb / kb * 1e3, "threads": shape[0], "blocks_per_sm": shape[1],
                 "hbm_frac": BYTES_PER_NODE["f32"] * nodes / (tb / kb) / 1e9 / measured_peaks()[0],
                 "workload": "64 replicas, L in {16,24,32,48,64}, N in {8,16,32,64}, FP32, graph-captured"}

    # the same kernel without noise (fluid and beads): the memory-bound reference point; and
    # the FP32 coupled step at L=256 (16.8 M nodes, 2.55 GB of populations) far above L2
    variants = None
    if not args.no_variants:
        def timed_steps(sim, k):
            sim.step(3)
            sim.sync()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            sim.step(k)
            a1.record(stream)
            torch.cuda.synchronize()
            return a0.elapsed_time(a1) / 1e3 / k

        sq = make(lb.LB_FP32)
        sq.set_options(noise_fluid=0, noise_beads=0)
        kq = max(20, args.steps // 5)
        tq = timed_steps(sq, kq)
        sq.close()
        s256 = lb.Simulation(L=256, seed=seed, precision=lb.LB_FP32, **PARAMS)
        s256.add_chain(N, x0=inputs.chain_walk(N, L=256, bond=0.97, seed=seed, self_avoiding=True), **CHAIN)
        k256 = max(10, args.steps // 40)
        t256 = timed_steps(s256, k256)
        s256.close()
        sb = make(lb.LB_BF16)  # BF16 storage of the deviations, FP32 arithmetic
        kb16 = max(20, args.steps // 5)
        tb16 = timed_steps(sb, kb16)
        sb.close()
        peak_q = measured_peaks()[0]
        variants = {
            "noise_off_L128": {"value": L ** 3 / tq / 1e6, "unit": "MLUPS", "ms_per_step": tq * 1e3, "steps": kq,
                               "hbm_frac": BYTES_PER_NODE["f32"] * L ** 3 / tq / 1e9 / peak_q},
            "L256": {"value": 256 ** 3 / t256 / 1e6, "unit": "MLUPS", "ms_per_step": t256 * 1e3, "steps": k256,
                     "hbm_frac": BYTES_PER_NODE["f32"] * 256 ** 3 / t256 / 1e9 / peak_q},
            "bf16_storage_L128": {"value": L ** 3 / tb16 / 1e6, "unit": "MLUPS", "ms_per_step": tb16 * 1e3,
                                  "steps": kb16,
                                  "hbm_frac": BYTES_PER_NODE["bf16"] * L ** 3 / tb16 / 1e9 / peak_q},
        }

    # chain observables (Sec. III A/B) on a recorded trajectory: 1000 frames of the N=128
    # chain in an L=32 box; each analysis kernel timed once after a warm-up call
    observ = None
    if not args.no_observables:
        from paper_0903_5067_gb300 import analysis as an

        so = lb.Simulation(L=32, seed=seed, precision=lb.LB_FP32, **PARAMS)
        so.add_chain(N, x0=inputs.chain_walk(N, L=32, bond=0.97, seed=seed, self_avoiding=True), **CHAIN)
        so.record_trajectory(stride=1, capacity=1000)
        so.step(999)
        traj = so.trajectory()
        so.close()
        T_o = traj.shape[0]
        ks = [0.1 * (1.25 ** q) for q in range(16)]

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            a0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - a0) * 1e3, r

        t_msd, _ = timed(lambda: an.msd(traj, 500))
        t_rouse, _ = timed(lambda: an.rouse_correlation(an.rouse_modes(traj), 500))
        t_sk, _ = timed(lambda: an.static_sk(traj, ks))
        t_skt, _ = timed(lambda: an.dynamic_sk(traj, ks[:4], 100, origin_stride=20))
        observ = {"frames": T_o, "N": N, "msd_ms": t_msd, "rouse_ms": t_rouse, "static_sk_ms": t_sk,
                  "dynamic_sk_ms": t_skt,
                  "static_sk_pairs_per_s": len(ks) * T_o * N * (N - 1) / 2 / (t_sk / 1e3),
                  "work": "g1/g2/g3 to lag 500; Rouse modes p=1..127 and correlation to lag 500; S(k) at 16 k; "
                          "S(k,t) at 4 k, lags 0..100, origins every 20 frames; FP64, host-timed with sync"}

    # the adjoint of the coupled step (gradient of sum_b |x_b(T) - x_b(0)|^2 with respect to the
    # initial positions and zeta, noise held fixed): L = 32, N = 16, T = 100, checkpoints every
    # 10 steps, FP32; one call runs the forward pass, the checkpointed recomputation and the
    # reverse sweep
    adj = None
    if not args.no_adjoint:
        Xa = inputs.chain_walk(16, L=32, bond=0.97, seed=7, self_avoiding=True)
        calls = []
        for rep in range(3):
            sa = lb.Simulation(L=32, seed=7, precision=lb.LB_FP32, **PARAMS)
            sa.add_chain(16, x0=Xa, **CHAIN)
            sa._bind()
            torch.cuda.synchronize()
            ta = time.perf_counter()
            lb.lb_adjoint_displacement(sa.ctx, 100, 10, 16)
            torch.cuda.synchronize()
            calls.append(time.perf_counter() - ta)
            sa.close()
        ta = min(calls[1:])
        fwd = []
        for rep in range(3):
            sf = lb.Simulation(L=32, seed=7, precision=lb.LB_FP32, **PARAMS)
            sf.add_chain(16, x0=Xa, **CHAIN)
            sf._bind()
            torch.cuda.synchronize()
            tf = time.perf_counter()
            sf.step(100)
            sf.sync()
            fwd.append(time.perf_counter() - tf)
            sf.close()
        tf = min(fwd[1:])
        adj = {"L": 32, "N": 16, "steps": 100, "checkpoint_every": 10, "ms_per_call": ta * 1e3,
               "us_per_step_forward_and_reverse": ta / 100 * 1e6, "forward_ms": tf * 1e3,
               "adjoint_over_forward": ta / tf,
               "work": "forward 100 steps with checkpoints, recomputation of each 10-step segment and the "
                       "reverse sweep (adjoint LB and bead kernels); FP32; host-timed, best of 2 after one "
                       "warm-up call; forward_ms: the same 100 steps through lb_step alone"}

    # Brownian dynamics with hydrodynamic interaction (Sec. II C): 64 chains of the paper's
    # production model (N = 32), one thread block per chain, RPY mobility and Fixman's
    # Chebyshev square root (degree 20, 20 power iterations for the bounds) every step
    bd = None
    if not args.no_bd:
        Xb = np.stack([inputs.chain_walk(32, L=1000, bond=0.97, seed=100 + r, self_avoiding=True) for r in range(64)])
        sbd = lb.BD(Xb, precision=lb.LB_FP32, seed=2)
        sbd.step(20)
        sbd.sync()
        kbd = max(200, args.steps // 5)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        sbd.step(kbd)
        b1.record(stream)
        torch.cuda.synchronize()
        tbd = b0.elapsed_time(b1) / 1e3 / kbd
        sbd.close()
        bd = {"chains": 64, "N": 32, "steps": kbd, "us_per_step": tbd * 1e6, "chain_steps_per_s": 64 / tbd,
              "work": "per chain and step: RPY mobility (96 x 96), 40 power-iteration and 20 Chebyshev "
                      "mat-vecs, FENE + WCA, Ito-Euler update; FP32, HI on"}

    cost = cost_scaling(stream) if args.cost_scaling else None

    value, tmax = aggregate_throughput(L ** 3 * args.steps / 1e6, t32, ws, dev)
    v64, _ = aggregate_throughput(L ** 3 * k64 / 1e6, t64, ws, dev)

    # end to end through the C ABI with host buffers: upload the initial state, K steps each
    # followed by a read-back of the beads, download the final populations
    n0 = torch.empty((19, L, L, L), dtype=torch.float64, pin_memory=True).numpy()
    nout = torch.empty((19, L, L, L), dtype=torch.float64, pin_memory=True).numpy()
    # two pinned bead buffers: the read-back of step k travels while step k+1 is queued
    xb = [torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    vb = [torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    ctx = lb.lb_create(L, PARAMS["rho"], PARAMS["eta"], PARAMS["eta_b"], PARAMS["kT"], PARAMS["h"], PARAMS["a"],
                       seed, lb.LB_FP32)
    lb.lb_add_chain(ctx, N, CHAIN["m"], CHAIN["zeta"], CHAIN["k_fene"], CHAIN["R0"], CHAIN["eps"], CHAIN["sigma"],
                    x0=X0)
    lb.lb_set_stream(ctx, stream.cuda_stream)
    lb.lb_get_populations(ctx, n0)  # the initial (rest) state, as host input; allocates the workspace
    ke = args.steps
    barrier()
    t0 = time.perf_counter()
    lb.lb_set_populations(ctx, n0)  # synchronising
    t1 = time.perf_counter()
    pending = []
    for k in range(ke):
        lb.lb_step(ctx, 1)
        pending.append(lb.lb_get_beads_async(ctx, xb[k % 2], vb[k % 2], 3 * N))
        if len(pending) == 2:  # step k-1's beads are on the host before buffer reuse
            lb.lb_wait(ctx, pending.pop(0))
    for t in pending:
        lb.lb_wait(ctx, t)
    t2 = time.perf_counter()
    lb.lb_get_populations(ctx, nout)  # synchronising
    barrier()
    te = time.perf_counter() - t0
    e2e_phases = {"upload_ms": (t1 - t0) * 1e3, "steps_ms": (t2 - t1) * 1e3,
                  "download_ms": (time.perf_counter() - t2) * 1e3}
    lb.lb_destroy(ctx)
    e2e_val, _ = aggregate_throughput(L ** 3 * ke / 1e6, te, ws, dev)
    h2d = n0.nbytes / ke
    d2h = nout.nbytes / ke + xb[0].nbytes + vb[0].nbytes

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    # the LB kernel's average launch duration from the timed region: K chained steps with one LB
    # launch each.  The LB launches follow one another (each waits, through the bead kernel of
    # its step, for the previous one to complete) and the bead kernel runs beside them, so the
    # region's time per step bounds the kernel's duration from above.  The roofline pass's
    # events around every (then unchained) launch add the launch gap; reported beside it.
    avg_kernel_s = t32 / args.steps
    achieved = BYTES_PER_NODE["f32"] * L ** 3 / avg_kernel_s / 1e9
    unchained_s = ms_k / max(nk, 1) / 1e3
    # per step: bead kernel + LB kernel
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(), "L": L, "N": N, "seed": SEED, "precision": "FP32 deviations",
                   "noise": "full thermalization + bead Langevin", "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (2 x 159 MB population buffers > 129 MB), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(), "kernel": "k_lb_step<float,float,DEV,NOISE>",
                     "algorithmic_bytes_per_node": BYTES_PER_NODE["f32"], "avg_launch_ms": avg_kernel_s * 1e3,
                     "timing": "CUDA events around the K chained steps of the timed region on the launching "
                               "stream / K LB launches (an upper bound of the launch duration: the bead kernel "
                               "runs beside each LB kernel)",
                     "unchained_launch_ms": unchained_s * 1e3,
                     "unchained_frac": BYTES_PER_NODE["f32"] * L ** 3 / unchained_s / 1e9 / peak,
                     "peak_kind": f"{peak_kind} (STREAM copy, burst)"},
        "fp64_plain": {"value": v64, "unit": "MLUPS", "steps": k64, "ms_per_step": t64 / k64 * 1e3,
                       "roofline_frac": BYTES_PER_NODE["f64"] * L ** 3 / (t64 / k64) / 1e9 / peak,
                       "roofline": {"bound": "fp64",
                                    "achieved": FP64_FLOPS_PER_NODE * L ** 3 / (t64 / k64) / 1e12,
                                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                    "frac": FP64_FLOPS_PER_NODE * L ** 3 / (t64 / k64) / 1e12 / FP64_PEAK_TFLOPS,
                                    "flops_per_node": FP64_FLOPS_PER_NODE,
                                    "peak_kind": "nominal (152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz)"},
                       "fp32_over_fp64": value / v64},
        "bead_steps_per_s": N * args.steps * ws / tmax,
        "batch_c4": batch,
        "observables_f3": observ,
        "bd_f4": bd,
        "cost_scaling": cost,
        "adjoint_c5": adj,
        "variants": variants,
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "phases": e2e_phases,
                "path": "C ABI, pinned host buffers: set_populations, K x (step + asynchronous bead read-back, each waited for one step later), get_populations"},
        # per step one bead launch (a cluster grid) and one LB launch; lb_step leaves the last
        # step's force correction pending (applied when the fluid is next read, after the
        # timed region)
        "gpu_launches": 2 * args.steps,
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
        "check": {"mass": obs[1], "bead_temperature": obs[15]},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# the paper's production model in MD/LB units (Sec. II E): dt_MD = 0.01, dtau_LB = 0.02
PAPER = dict(rho=0.864, eta=0.864 * 2.8, eta_b=0.864 * 2.8, kT=1.2, h=0.02, a=1.0, m=1.0, zeta=20.8, k_fene=7.0,
             R0=2.0, eps=1.0, sigma=1.0)


def cost_scaling(stream):
    """Cost of each method per chain and time unit as the chain grows (Sec. IV): the LB side
    runs, like the paper, three boxes per N with sqrt<R_e^2>/L = 0.5, 0.4, 0.3 (R_e from the
    Table 1 BD value at N = 32 scaled by N^0.588), each as a batch of 64 replicas with two MD
    steps per LB step; the BD side runs 64 chains of the same N with RPY and the Chebyshev
    square root at its production time step.  Device time with CUDA events."""
    import math

    import numpy as np
    import torch
    from paper_0903_5067_gb300 import inputs, lb

    out = []
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for N in (16, 32, 64):
        re = math.sqrt(99.22) * (N / 32.0) ** 0.588
        Ls = [max(8, int(round(re / f))) for f in (0.5, 0.4, 0.3)]
        lb_cost = 0.0
        for Lb in Ls:
            seeds = [7000 + 97 * Lb + r for r in range(64)]
            X = [inputs.chain_walk(N, L=Lb, bond=0.97, seed=sd, self_avoiding=True) for sd in seeds]
            b = lb.Batch([Lb] * 64, [N] * 64, seeds, X, precision=lb.LB_FP32, md_substeps=2, **PAPER)
            b.step(5)
            e0, e1 = ev(), ev()
            e0.record(stream)
            b.step(100)
            e1.record(stream)
            torch.cuda.synchronize()
            lb_cost += e0.elapsed_time(e1) / 1e3 / (64 * 100 * PAPER["h"])
            b.close()
        Xb = np.stack([inputs.chain_walk(N, L=1000, bond=0.97, seed=300 + r, self_avoiding=True) for r in range(64)])
        zeta = lb.zeta_eff(20.8, PAPER["eta"])
        dt = 0.005 * zeta / (4.0 * PAPER["k_fene"])
        sb = lb.BD(Xb, kT=PAPER["kT"], zeta=zeta, eta_s=PAPER["eta"], dt=dt, k_fene=PAPER["k_fene"],
                   R0=PAPER["R0"], precision=lb.LB_FP32, seed=5)
        sb.step(20)
        e0, e1 = ev(), ev()
        e0.record(stream)
        sb.step(400)
        e1.record(stream)
        torch.cuda.synchronize()
        bd_cost = e0.elapsed_time(e1) / 1e3 / (64 * 400 * dt)
        sb.close()
        out.append({"N": N, "L": Ls, "lb_s_per_chain_time_unit": lb_cost, "bd_s_per_chain_time_unit": bd_cost,
                    "lb_over_bd": lb_cost / bd_cost})
    lg = np.log([r["N"] for r in out])
    return {"points": out,
            "lb_exponent": float(np.polyfit(lg, np.log([r["lb_s_per_chain_time_unit"] for r in out]), 1)[0]),
            "bd_exponent": float(np.polyfit(lg, np.log([r["bd_s_per_chain_time_unit"] for r in out]), 1)[0]),
            "work": "FP32; LB: 64 replicas per box, 100 LB steps (200 MD steps) timed after 5; BD: 64 chains, "
                    "400 steps timed after 20, dt = 0.005 zeta_eff / (4 k)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="where the nvidia-smi clock samples of the timed region are written (default: temp dir)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-observables", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-bd", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--cost-scaling", action="store_true",
                    help="also time LB against BD per chain and time unit for N = 16, 32, 64 (Sec. IV)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
