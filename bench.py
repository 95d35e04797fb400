"""Benchmark: monomer Monte-Carlo moves per second of the SCMF cycle
(sweep + occupation count + field update), arXiv:1711.03828.

Default workload: the lamella-forming diblock melt at scale, 4,194,304 chains
of N=32 (134,217,728 particles) in a 32^3 R_e0 box, 192^3 grid, chiN=30,
kappaN=50.  One step = one SCMF cycle of every particle.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) the workload's chains
are sharded over the ranks (strong scaling: the same 134 M-particle system on
N GPUs) and every cycle sums the occupation numbers over the ranks with one
NCCL all-reduce before each rank's field update, the one exchange of the
method (Sec. 3.1.1).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "monomer MC moves/s incl. field update"
UNIT = "moves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="melt_large",
                    choices=["melt_large", "melt_mid", "melt_small", "melt_slow", "melt_subbox",
                             "melt_tiny", "arch_large", "arch_mid", "abc_large",
                             "batch64", "decorrelation", "precision"])
    ap.add_argument("--move", default="uniform", choices=["uniform", "smc", "learned"],
                    help="trial moves: uniform displacement or smart Monte Carlo")
    ap.add_argument("--iteration", default="set", choices=["set", "molecule"],
                    help="particle visiting scheme: independent sets (even/odd chain positions) "
                         "or molecule-parallel with random particle choice")
    ap.add_argument("--learned-net", default="mma_sync", choices=["mma_sync", "umma", "fp32"],
                    help="network evaluator of the learned move: warp-level mma.sync (default), "
                         "tcgen05 with the accumulator in tensor memory, or FP32 on the CUDA cores")
    ap.add_argument("--grid-dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="storage type of the omega grids (energies stay FP32)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


GRID_DTYPES = {"f32": 0, "bf16": 1, "f16": 2}


def workload(name, replica=0, grid_dtype="f32", move="uniform", learned_net="mma_sync",
             iteration="set"):
    from paper_1711_03828_gb300 import workloads
    d = getattr(workloads, name)(seed=1)
    d.replica_id = replica
    d.grid_dtype = GRID_DTYPES[grid_dtype]
    d.move = {"uniform": 0, "smc": 1, "learned": 2}[move]
    d.flags |= {"mma_sync": 0, "umma": 4, "fp32": 2}[learned_net] if d.move == 2 else 0
    if iteration == "molecule":
        d.set_order = 2
    return d


def setup_architectures(target, d, seed=1, name="arch_large"):
    """Molecules of the architectures of workloads.arch_large (or, for
    abc_large, the three-type molecules of workloads.abc_molecules with their
    chi matrix), one drawn per molecule, on a library System or an oracle
    System (the same arrays)."""
    import numpy as np
    from paper_1711_03828_gb300 import workloads
    if name.startswith("abc_"):
        mols = workloads.abc_molecules()
        target.set_types(3, workloads.ABC_CHI_N)
    else:
        mols = workloads.arch_large_molecules()
    words, starts = workloads.encode_architectures(mols)
    arch = np.random.default_rng(seed + 17).integers(0, len(mols), d.n_chains).astype(np.uint8)
    pos = workloads.architecture_positions(d, mols, arch, seed=seed + 29)
    target.set_topology(words, starts, arch)
    return pos


def uses_architectures(name):
    return name.startswith("arch_") or name.startswith("abc_")


def config_of(d, name, l2_note):
    extra = {}
    if name.startswith("arch_"):
        extra["architectures"] = ("three-arm star (11,10,10), comb (16 + 4x4), ring (32), "
                                  "linear diblock; one drawn per molecule")
    if name.startswith("abc_"):
        extra["architectures"] = ("three types A, B, C (chi N: AB 30, AC 15, BC 40): ABC "
                                  "triblock, three-arm star with one arm per type, ABC ring; "
                                  "one drawn per molecule")
    return {**extra,"workload": f"{name}: {d.n_chains} chains x N={d.N}, box {d.box_Re} R_e0, grid "
                        f"{d.grid}, chiN={d.chiN}, kappaN={d.kappaN}",
            "n_chains": d.n_chains, "N": d.N, "particles": d.M, "grid": list(d.grid),
            "box_Re": list(d.box_Re), "chiN": d.chiN, "kappaN": d.kappaN,
            "move": {0: "uniform", 1: "smart Monte Carlo", 2: "learned MH proposal"}[d.move],
            "set_order": {0: "random per chain and sweep", 1: "even first",
                          2: "molecule-parallel, random particle per attempt"}[d.set_order],
            "grid_dtype": {0: "f32", 1: "bf16", 2: "f16"}[d.grid_dtype], "l2": l2_note}


# --------------------------------------------------------------------------
# CPU oracle timing (the baseline; never tuned)
# --------------------------------------------------------------------------
def oracle_rate(name, seconds, max_steps=None):
    """Oracle cycles (sweep + histogram + fields) on a 4^3 R_e0 sub-box of the
    workload (same N, density, grid spacing, chiN).  Returns (moves/s, cores,
    sample, steps)."""
    import oracle
    from paper_1711_03828_gb300 import workloads
    d = workload(name)
    sub = workloads.scaled(d, (4.0, 4.0, 4.0))
    o = oracle.System(sub.n_chains, sub.N, sub.f, sub.box_Re, sub.grid, sub.chiN, sub.kappaN,
                      seed=sub.seed)
    if uses_architectures(name):
        pos = setup_architectures(o, sub, name=name)
        p = oracle.Positions(pos[0].copy(), pos[1].copy(), pos[2].copy())
    else:
        p = o.init_chains()
    types = name.startswith("abc_")

    def fields():
        if types:
            return None, None, o.fields_types(o.histogram_types(p))
        return (*o.fields(*o.histogram(p)), None)

    wA, wB, wT = fields()
    steps = 0
    t0 = time.perf_counter()
    while True:
        o.sweep(p, wA, wB, steps, w_types=wT)
        wA, wB, wT = fields()
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and steps >= max_steps) or (max_steps is None and el >= seconds):
            break
    sample = (f"oracle cycles on a 4^3 R_e0 sub-box of the workload ({sub.n_chains} chains x "
              f"N={sub.N}, grid {sub.grid}, chiN={sub.chiN}): {steps} cycles, {el:.2f} s")
    return sub.M * steps / el, oracle.num_threads(), sample, steps, el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import build as ob
    if not os.path.exists(os.path.join(ROOT, "oracle", "liboracle.so")):
        ob.build()
    total = args.warmup + args.steps
    # warm-up cycles are not timed: run them first
    oracle_rate(args.workload, 0.0, max_steps=max(args.warmup, 1))
    rate, cores, sample, steps, el = oracle_rate(args.workload, 0.0, max_steps=args.steps)
    d = workload(args.workload)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(d, args.workload, "CPU"),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    _ = total


# --------------------------------------------------------------------------
# Clock sampling during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.lines = []
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            time.sleep(0.3)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for l in self.proc.stdout:
            self.lines.append(l.strip())

    def __exit__(self, *a):
        if self.proc is None:
            self.out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        import statistics
        self.out = {"sm_mhz": statistics.median(sm) if sm else None,
                    "sm_max_mhz": max(mx) if mx else None,
                    "power_w_max": max(pw) if pw else None,
                    "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = json.load(f)
        return float(v["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


SWEEP_SOURCES = ("sweep.cu", "pair_body.cuh", "common.cuh")


def kernel_source_hash(sources=SWEEP_SOURCES):
    """sha256 over the sources of a sweep kernel (by default the pair kernel's
    sweep.cu, pair_body.cuh, common.cuh), so that a stored traffic figure is
    used only while the kernel it was taken on is unchanged."""
    import hashlib
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1711_03828_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(workload_name):
    """DRAM bytes per sweep launch from the committed ncu capture, if it was
    taken on this workload with the sweep kernel source as it is now."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", f"sweep_traffic_{workload_name}.json")) as f:
            t = json.load(f)
        if kernel_source_hash(tuple(t.get("sources", SWEEP_SOURCES))) != t["kernel_src_sha256"]:
            return None
        return t["dram_bytes_read"] + t["dram_bytes_write"]
    except (OSError, KeyError, ValueError):
        return None


def sweep_kernel_name(d, architectures=False):
    """The sweep kernel libsoma launches for this description."""
    if architectures:
        return "sweep_molecule_topology_kernel" if d.set_order == 2 else "sweep_topology_kernel"
    pair = d.N % 2 == 0 and d.N <= 64
    if d.move == 1:
        return "sweep_smc_pair_kernel" if pair else "sweep_smc_kernel"
    if d.move == 2:
        if not pair or d.flags & 2:
            return "sweep_learned_kernel"
        return "sweep_learned_umma_kernel" if d.flags & 4 else "sweep_learned_tc_kernel"
    if d.set_order == 2:
        return "sweep_molecule_kernel"
    return "sweep_pair_kernel" if pair else "sweep_uniform_kernel"


def sweep_kernel_bytes(d, n_types=0):
    """Algorithmic bytes of one sweep-kernel launch: every position read and
    written once (24 B per particle), each omega plane read once and the
    occupation grid written once (12 B per cell for FP32 omega; with n_t
    types one FP32 field plane and one 32-bit count plane per type)."""
    cells = d.grid[0] * d.grid[1] * d.grid[2]
    if n_types:
        return 24 * d.M + cells * 8 * n_types
    wb = 4 if d.grid_dtype == 0 else 2
    return 24 * d.M + cells * (2 * wb + 4)


def field_kernel_bytes(d, n_types=0):
    """Counts read, the next sweep's counts cleared, fields written."""
    cells = d.grid[0] * d.grid[1] * d.grid[2]
    if n_types:
        return cells * 12 * n_types
    wb = 4 if d.grid_dtype == 0 else 2
    return cells * (4 + 4 + 2 * wb)


def run_sharded(args, rank, world):
    """One rank of the chain-sharded cycle: this rank's share of the
    workload's chains, one NCCL all-reduce of the packed counts per cycle."""
    import ctypes

    import torch
    import torch.distributed as tdist
    from paper_1711_03828_gb300 import System, _abi
    from paper_1711_03828_gb300.shard import ShardedRun, shard_desc

    if uses_architectures(args.workload) or args.move == "learned":
        raise SystemExit("bench.py --gpus N > 1 shards the linear-chain workloads with uniform "
                         "or smart Monte Carlo moves")
    whole = workload(args.workload, grid_dtype=args.grid_dtype, move=args.move,
                     iteration=args.iteration)
    d = shard_desc(whole, world, rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = System(d, stream=stream)
    run = ShardedRun(s, d.cells, "cuda")
    run.start()
    run.cycle(args.warmup)
    s.sync()
    t_before = s.timing()
    tdist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        run.cycle(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    tdist.barrier()
    t = torch.tensor([ev0.elapsed_time(ev1)], device="cuda")
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    ms = float(t.item())
    launches = s.timing()["kernel_launches"] - t_before["kernel_launches"]
    value = whole.M * args.steps / (ms * 1e-3)
    s.set_timing(True)
    run.cycle(min(args.steps, 100))
    tk = s.timing()
    s.set_timing(False)
    sweep_ms = tk["ms_sweep"] / max(tk["sweep_launches"], 1)
    field_ms = tk["ms_fields"] / max(tk["field_launches"], 1)
    peak, peak_kind = measured_peak_hbm()
    achieved = sweep_kernel_bytes(d) / (sweep_ms * 1e-3) / 1e9
    # end to end: every step uploads this rank's positions from pinned host
    # memory, runs one sharded cycle (exchange included) and reads the summed
    # occupation numbers back
    host_pos = torch.empty(3 * d.M, dtype=torch.float32, pin_memory=True)
    _abi.soma_get_positions(s.h, ctypes.c_void_p(host_pos.data_ptr()), 3 * d.M, 0)
    host_n = torch.empty(d.cells, dtype=torch.int32, pin_memory=True)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    tdist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _abi.soma_set_positions(s.h, ctypes.c_void_p(host_pos.data_ptr()), 3 * d.M, 0)
        run.start()
        run.cycle(1)
        _abi.soma_get_density(s.h, ctypes.c_void_p(host_n.data_ptr()), d.cells, 0)
    torch.cuda.synchronize()
    t = torch.tensor([time.perf_counter() - t0], device="cuda")
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    e2e = {"value": whole.M * e2e_steps / float(t.item()), "unit": UNIT,
           "h2d_bytes_per_step": 12 * d.M, "d2h_bytes_per_step": 4 * d.cells,
           "steps": e2e_steps, "per_rank": True}
    obs = s.observables()
    acc = torch.tensor([float(obs["accepted"]), float(obs["attempted"])], device="cuda",
                       dtype=torch.float64)
    tdist.all_reduce(acc)
    s.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**config_of(whole, args.workload,
                                   f"inputs larger than L2 ({12 * d.M / 1e9:.2f} GB of positions "
                                   "per rank)" if 12 * d.M > 129e6 else
                                   f"inputs L2-resident ({12 * d.M / 1e6:.1f} MB per rank)"),
                       "parallelism": f"chains sharded over {world} ranks, one NCCL all-reduce "
                                      f"of the {4 * d.cells / 1e6:.1f} MB count grid per cycle"},
            "roofline": {"bound": "hbm", "kernel": sweep_kernel_name(d), "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None,
                         "bytes_per_launch": sweep_kernel_bytes(d), "ms_per_launch": sweep_ms,
                         "field_kernel_ms": field_ms},
            "e2e": e2e, "clocks": clk.out, "gpu_launches": int(launches),
            "acceptance": float(acc[0].item()) / max(float(acc[1].item()), 1.0),
        }
        print(json.dumps(line), flush=True)
    tdist.destroy_process_group()


def run_ours(args):
    import torch
    import torch.distributed as tdist

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if world > 1:
        return run_sharded(args, rank, world)
    from paper_1711_03828_gb300 import System, _abi

    d = workload(args.workload, replica=rank, grid_dtype=args.grid_dtype, move=args.move,
                 learned_net=args.learned_net, iteration=args.iteration)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = System(d, stream=stream)
    if uses_architectures(args.workload):
        s.set_positions(setup_architectures(s, d, name=args.workload))
        s.sort_molecules()   # the generator's molecules are in random spatial order
        s.update_fields()
    train_log = None
    if d.move == 2:  # train the proposal on this system's plain-method configurations
        train_log = s.train_proposal(steps=200, batch=16384, sweeps_between=1, lr=3e-3)

    def barrier():
        if world > 1:
            tdist.barrier()

    # warm-up, then the timed cycles on the production path (CUDA graph of
    # 16 cycles, no per-kernel events)
    s.sweep(args.warmup)
    s.sync()
    t_before = s.timing()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        s.sweep(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    t_after = s.timing()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    launches = t_after["kernel_launches"] - t_before["kernel_launches"]
    value = d.M * args.steps * world / (ms * 1e-3)
    # per-kernel device times for the roofline: the same cycles launched one by
    # one with CUDA events around every kernel on the system's stream
    s.set_timing(True)
    s.sweep(min(args.steps, 200))
    tk = s.timing()
    sweep_ms = tk["ms_sweep"] / max(tk["sweep_launches"], 1)
    field_ms = tk["ms_fields"] / max(tk["field_launches"], 1)
    s.set_timing(False)
    peak, peak_kind = measured_peak_hbm()
    n_types = 3 if args.workload.startswith("abc_") else 0
    achieved = sweep_kernel_bytes(d, n_types) / (sweep_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: every step copies the
    # positions in from pinned memory, runs one cycle and reads the occupation
    # grid back
    host_pos = torch.empty(3 * d.M, dtype=torch.float32, pin_memory=True)
    import ctypes
    _abi.soma_get_positions(s.h, ctypes.c_void_p(host_pos.data_ptr()), 3 * d.M, 0)
    n_words = d.cells * (n_types or 1)   # the packed A | B grid, or one plane per type
    host_n = torch.empty(n_words, dtype=torch.int32, pin_memory=True)
    read_counts = _abi.soma_get_type_counts if n_types else _abi.soma_get_density
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _abi.soma_set_positions(s.h, ctypes.c_void_p(host_pos.data_ptr()), 3 * d.M, 0)
        _abi.soma_sweep(s.h, 1)
        read_counts(s.h, ctypes.c_void_p(host_n.data_ptr()), n_words, 0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": d.M * e2e_steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 12 * d.M, "d2h_bytes_per_step": 4 * n_words,
           "steps": e2e_steps}
    obs = s.observables()
    s.close()

    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(d, args.workload,
                            f"inputs larger than L2 ({12 * d.M / 1e9:.2f} GB of positions)"
                            if 12 * d.M > 129e6 else
                            f"inputs L2-resident ({12 * d.M / 1e6:.2f} MB of positions): a "
                            "latency figure, not a bandwidth one"),
        "roofline": {"bound": "hbm",
                     "kernel": sweep_kernel_name(d, uses_architectures(args.workload)),
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": measured_traffic(args.workload)
                     if args.grid_dtype == "f32" and args.move == "uniform" else None,
                     "bytes_per_launch": sweep_kernel_bytes(d, n_types), "ms_per_launch": sweep_ms,
                     "field_kernel_ms": field_ms,
                     "field_kernel_gbs": field_kernel_bytes(d, n_types) / (field_ms * 1e-3) / 1e9},
        "e2e": e2e,
        "clocks": clk.out,
        "gpu_launches": int(launches),
        "acceptance": obs["accepted"] / max(obs["attempted"], 1),
    }
    if train_log is not None:
        line["training"] = train_log
    if not args.no_cpu_baseline and world == 1:
        rate, cores, sample, _, _ = oracle_rate(args.workload, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def run_batch(args):
    """64 independent melts (uneven sizes) advanced by one batched launch per
    cycle, against the same 64 systems advanced by 64 sequential launches."""
    import torch
    from paper_1711_03828_gb300 import Batch, System, workloads

    torch.cuda.set_device(0)
    descs = workloads.batch_replicas(64, seed=1)
    M = sum(d.M for d in descs)
    cells = sum(d.cells for d in descs)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b = Batch(descs, stream=stream)
    table = b.autotune(cycles_per_candidate=3)
    b.sweep(args.warmup)
    b.sync()
    b.set_timing(True)
    t_before = b.timing()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        b.sweep(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    t_after = b.timing()
    b.set_timing(False)
    sweep_ms = t_after["ms_sweep"] / max(t_after["sweep_launches"] - t_before["sweep_launches"], 1)
    # graph replay (no per-kernel events) for the batched value
    torch.cuda.synchronize()
    ev0.record(stream)
    b.sweep(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_graph = ev0.elapsed_time(ev1)
    b.close()
    singles = [System(d, stream=stream) for d in descs]
    for s_ in singles:
        s_.sweep(args.warmup)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        for s_ in singles:
            s_.sweep(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_seq = ev0.elapsed_time(ev1)
    for s_ in singles:
        s_.close()
    peak, peak_kind = measured_peak_hbm()
    bytes_launch = 24 * M + 12 * cells
    line = {
        "metric": METRIC, "value": M * args.steps / (ms_graph * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batch64: 64 independent diblock melts, {M} particles in total "
                               "(L in {2,3,4,6,8} R_e0, N in {16,32,64}, f in {0.3,0.5}, "
                               "chiN in [10,40]), one batched launch per cycle under a CUDA graph",
                   "particles": M, "cells": cells, "tuned_shape": min(table, key=lambda t: t["ms_per_cycle"]),
                   "l2": f"inputs larger than L2 ({12 * M / 1e9:.2f} GB of positions)"},
        "sequential": {"value": M * args.steps / (ms_seq * 1e-3), "unit": UNIT,
                       "ms_per_step": ms_seq / args.steps,
                       "how": "the same 64 systems, one soma_sweep(1) per system per cycle "
                              "(2 launches each)"},
        "eager_events": {"ms_per_step": ms / args.steps, "sweep_kernel_ms": sweep_ms},
        "roofline": {"bound": "hbm", "kernel": "sweep_batch_kernel",
                     "achieved": bytes_launch / (sweep_ms * 1e-3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": bytes_launch / (sweep_ms * 1e-3) / 1e9 / peak,
                     "peak_kind": peak_kind, "traffic": None},
        "clocks": clk.out,
        "gpu_launches": 2 * args.steps,
        "autotune": table,
    }
    print(json.dumps(line), flush=True)


def tau_int(x, c=5.0):
    """Integrated autocorrelation time (in samples) of series x (T, chains),
    chain-averaged autocorrelation, Sokal's automatic window (W >= c tau)."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    x = x - x.mean(0)
    T = x.shape[0]
    f = np.fft.rfft(x, n=2 * T, axis=0)
    acf = np.fft.irfft(f * np.conj(f), n=2 * T, axis=0)[:T].mean(1) / np.arange(T, 0, -1)
    rho = acf / acf[0]
    tau = 0.5
    for W in range(1, T):
        tau += rho[W]
        if W >= c * tau:
            break
    return float(tau), int(W)


def run_decorrelation(args):
    """R_e^2 decorrelations per second of the uniform, smart Monte Carlo and
    learned moves on the slow melt (N=64, chiN=40, kappaN=50): tau_int of the
    per-chain R_e^2 and of S(q*) on an 8x8x4 R_e0 box, wall time per cycle at
    the 67M-particle scale, decorrelations/s = chains * cycles/s / (2 tau)."""
    import numpy as np
    import torch
    from paper_1711_03828_gb300 import System, workloads

    torch.cuda.set_device(0)
    dev = torch.device("cuda")
    big = workloads.melt_slow()
    every, T, equil = 10, max(args.steps, 400), 1000
    seeds = (1, 2)
    # train the learned proposal on plain-method configurations of the small
    # box: 2000 Adam steps, five plain sweeps between steps (10^4 sweeps of
    # plain-method trajectories)
    tr = System(workloads.melt_slow(n_chains=16384, box_Re=(8.0, 8.0, 4.0), grid=(48, 48, 24),
                                    move=2, seed=101))
    tr.sweep(200)
    train_log = tr.train_proposal(steps=2000, batch=16384, sweeps_between=5, lr=3e-3)
    W = tr.get_proposal_weights()
    tr.close()
    # q*: the strongest low-q shell after equilibration (uniform moves)
    ms_all = [(i, j, k) for i in range(-4, 5) for j in range(-4, 5) for k in range(0, 3)
              if 0 < i * i + j * j + k * k <= 16]
    res = {}
    q_star = None
    for name, move, order in (("uniform", 0, 0), ("smc", 1, 0), ("learned", 2, 0),
                              ("uniform_molecule", 0, 2)):
        taus_re, taus_sq = [], []
        for seed in seeds:
            d = workloads.melt_slow(n_chains=16384, box_Re=(8.0, 8.0, 4.0), grid=(48, 48, 24),
                                    move=move, set_order=order, seed=seed)
            s = System(d)
            if move == 2:
                s.set_proposal_weights(W)
            s.sweep(equil)
            if q_star is None:
                sq = s.structure_factor(ms_all)
                q_star = [ms_all[int(np.argmax(sq))]]
            pos = torch.empty(3 * d.M, dtype=torch.float32, device=dev)
            re2, sqs = [], []
            for t in range(T):
                s.sweep(every)
                s.get_positions(out=pos)
                P = pos.view(3, d.n_chains, d.N)
                re2.append(((P[:, :, -1] - P[:, :, 0]) ** 2).sum(0).double().cpu().numpy())
                sqs.append(float(s.structure_factor(q_star)[0]))
            s.close()
            tr_, w_ = tau_int(np.asarray(re2))
            taus_re.append(tr_)
            taus_sq.append(tau_int(np.asarray(sqs))[0])
        tau_re, w_re = float(np.mean(taus_re)), w_
        tau_sq = float(np.mean(taus_sq))
        # wall time per cycle at scale
        b = System(workloads.melt_slow(move=move, set_order=order))
        if move == 2:
            b.set_proposal_weights(W)
        b.sweep(3)
        import time as _t
        b.sync()
        t0 = _t.perf_counter()
        b.sweep(20)
        b.sync()
        ms_cycle = (_t.perf_counter() - t0) * 1e3 / 20
        b.close()
        tau_sweeps = tau_re * every
        # error of the seed mean from the seeds' spread (the autocorrelation is
        # averaged over 16,384 chains, so one run's estimate scatters far less
        # than a single series' would)
        err = float(np.std(taus_re, ddof=1) / np.sqrt(len(seeds))) * every
        dps = big.n_chains * (1e3 / ms_cycle) / (2 * tau_sweeps)
        res[name] = {"tau_int_Re2_sweeps": tau_sweeps, "tau_int_Re2_err": err,
                     "tau_int_Re2_per_seed": [t * every for t in taus_re], "window": w_re * every,
                     "tau_int_Sq_sweeps": tau_sq * every,
                     "tau_int_Sq_per_seed": [t * every for t in taus_sq],
                     "ms_per_cycle_67M": ms_cycle,
                     "decorrelations_per_s": dps, "decorrelations_per_s_err": dps * err / tau_sweeps}
    line = {"metric": "R_e^2 decorrelations/s (learned vs plain)", "unit": "decorrelations/s",
            "value": res["learned"]["decorrelations_per_s"], "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "slow melt: tau_int on 16,384 chains x N=64 in 8x8x4 R_e0 "
                                   "(48x48x24 grid), wall time on 1,048,576 chains in 32x32x16 R_e0 "
                                   "(192x192x96 grid), chiN=40, kappaN=50",
                       "sampling": f"every {every} cycles, {T} samples after {equil} cycles, "
                                   f"seeds {list(seeds)}",
                       "q_star": q_star[0]},
            "moves": res, "training": train_log}
    print(json.dumps(line), flush=True)


def batch_means(x, n_batches=8):
    """Mean and standard error of a time series by batch means."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    b = len(x) // n_batches
    m = x[:b * n_batches].reshape(n_batches, b).mean(1)
    return float(x.mean()), float(m.std(ddof=1) / np.sqrt(n_batches))


def run_precision(args):
    """Precision of the 16-bit field grids at scale: the 134M-particle lamellar
    melt from one seed with FP32, BF16 and FP16 omega, 1000 SCMF cycles each;
    time averages over the last 800 cycles (a sample every 10 cycles, batch
    means over 8 batches) of the total energy per particle (FP64 on the GPU),
    <R_e^2>/R_e0^2 and S(q*), q* the shell |m| (grid wave vectors) with the
    largest S averaged over up to 32 wave vectors of the shell, chosen on the
    FP32 run after 200 cycles and used for all three."""
    import numpy as np
    import torch
    from paper_1711_03828_gb300 import System

    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    shells = {}
    for r in range(4, 33):
        # wave vectors of the shell |m| = r (rounded), half space, up to 32 of them
        ms = [(i, j, k) for i in range(-r, r + 1) for j in range(-r, r + 1) for k in range(0, r + 1)
              if round(np.sqrt(i * i + j * j + k * k)) == r and (k > 0 or j > 0 or (j == 0 and i > 0))]
        idx = rng.choice(len(ms), size=min(32, len(ms)), replace=False)
        shells[r] = [ms[i] for i in sorted(idx)]
    equil, total, every = 200, 1000, 10
    res, q_shell = {}, None
    for name in ("f32", "bf16", "f16"):
        d = workload("melt_large", grid_dtype=name)
        s = System(d)
        s.sweep(equil)
        if q_shell is None:
            avg = {r: float(np.mean(s.structure_factor(m))) for r, m in shells.items()}
            q_shell = max(avg, key=avg.get)
        E, R, S = [], [], []
        t0 = time.perf_counter()
        for _ in range((total - equil) // every):
            s.sweep(every)
            o = s.observables()
            E.append(o["E_tot"] / d.M)
            R.append(o["Re2_rel"])
            S.append(float(np.mean(s.structure_factor(shells[q_shell]))))
        wall = time.perf_counter() - t0
        s.close()
        res[name] = {"E_per_particle": batch_means(E), "Re2_rel": batch_means(R),
                     "S_qstar": batch_means(S), "samples": len(E), "wall_s": wall}
    for name in ("bf16", "f16"):
        for k in ("E_per_particle", "Re2_rel", "S_qstar"):
            m0, e0 = res["f32"][k]
            m1, e1 = res[name][k]
            res[name][k + "_vs_f32_sigma"] = (m1 - m0) / max(np.hypot(e0, e1), 1e-300)
    line = {"metric": "observables with 16-bit field grids vs FP32 (config 4)",
            "n_gpus": 1, "data": "synthetic", "dtype": "f32 positions and energies",
            "config": {"workload": "melt_large: 4194304 chains x N=32, box 32^3 R_e0, grid 192^3, "
                                   "chiN=30, kappaN=50, seed 1",
                       "cycles": total, "averaged": f"cycles {equil}..{total}, every {every}",
                       "q_star_shell": q_shell},
            "results": res}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "decorrelation":
        run_decorrelation(args)
    elif args.workload == "precision":
        run_precision(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
