"""Benchmark: GCAMPS T-gates/s on seeded T-doped random Clifford brickwork circuits.

Workload (one step = one pass of the whole hot path over one batch):
  qubit and qutrit circuits (d = 2 and d = 3), n = 32 qudits, 24 brickwork layers of random
  two-qudit Cliffords, 32 T gates (each followed by disentangling), chi_max = 256, SVD cutoff
  1e-12, complex128; seeds 1..8 for each d (16 circuits per step; one thread-block cluster per
  circuit, 16 CTAs for qutrits and 4 for qubits: the qutrit circuits are the slow ones, and their
  exact class evaluations spread over the cluster's CTAs).  Every step starts from |0...0> with
  C = I (reset kernel) and runs the full gate list in one engine launch per d, the qutrit launch
  first.

value  : T gates of all circuits / device time of the timed steps (CUDA events on the engine's
         stream; L2 flushed with a 512 MiB write before every step, outside the event pair).
e2e    : same metric through the C ABI with the gate list in pinned host memory, copied to the
         device inside the timed region, and per-circuit counters read back every step.
Multi-GPU: circuits are independent; each rank runs the same per-rank batch with its own seeds
(weak scaling, no collective on the data path).

--impl reference runs the FP64 CPU oracle on a bounded sample of the same workload.

Other workloads (--workload): batched (uneven qutrit circuits in one graph-captured launch),
gradient (forward run + adjoint gradient), chi-layers (the bond dimension after every layer of the
Fig. 4 circuit family, the experiment of Fig. 5a; with --impl reference the oracle runs it).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N, LAYERS, T, CHI, CUTOFF = 32, 24, 32, 256, 1e-12
SEEDS_PER_D = 8
WORKLOAD = "gcamps-brickwork-n32-L24-T32-chi256-d2+d3-8seeds"
METRIC = "T-gates/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 nominal (profiling recipe table), used only without a measurement
# GB300 FP32 (non-tensor) nominal: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAKS_FILE = os.path.join(ROOT, "profiles", "arith_peaks_gb300.json")


def arith_peaks():
    """(FP64 peak, FP32 peak, source): the measured multiply-add rates of profiles/arith_peaks_gb300.json
    (python -m paper_2511_06672_gb300.peaks), else the nominal figures."""
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return (float(p["fp64_fma_tflops"]), float(p["fp32_fma_tflops"]),
                f"measured ({os.path.relpath(PEAKS_FILE, ROOT)}, {p.get('when', '?')})")
    except (OSError, ValueError, KeyError):
        return FP64_NOMINAL_TFLOPS, FP32_NOMINAL_TFLOPS, "nominal (no measurement committed)"
ENGINE_SRCS = [os.path.join(ROOT, "paper_2511_06672_gb300", "csrc", f)
               for f in ("gcamps_device.cuh", "gcamps_engine.cu", "gcamps_internal.h")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_run_dram_bench_workload.txt")


def engine_source_hash() -> str:
    """sha256 over the sources of the benchmark's kernel (device code, its translation unit, the layout)."""
    import hashlib
    h = hashlib.sha256()
    for f in ENGINE_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def engine_traffic():
    """DRAM bytes per k_run launch from the committed ncu summary, if it was taken on these engine
    sources (sha256 recorded beside it); else None."""
    try:
        want = engine_source_hash()
        kv = dict(line.strip().split("=", 1) for line in open(TRAFFIC_FILE) if "=" in line and not line.startswith("#"))
        if kv.get("engine_sha256") == want:
            return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def progress(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def rank_seeds(rank: int, per_rank: int = SEEDS_PER_D):
    """Seeds of one rank's circuits: each rank runs its own circuits (weak scaling, no collective on the
    data path)."""
    return [1 + s + rank * per_rank for s in range(per_rank)]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank time over all ranks (the value itself for one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank count over all ranks (the value itself for one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units_per_rank_step: float, steps: int, world: int, max_time_s: float) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return units_per_rank_step * steps * world / max_time_s


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_ops(G, d, rank):
    from synth import brickwork_circuit
    import numpy as np
    ops, begin = [], [0]
    for seed in rank_seeds(rank):
        o = G.ops_from_gates(brickwork_circuit(N, d, LAYERS, T, seed), d)
        ops.append(o)
        begin.append(begin[-1] + len(o))
    return np.concatenate(ops), np.array(begin, dtype=np.int32)


def bench_circuits(rank: int = 0):
    """The benchmark's circuits of one rank, (d, seed), in the order the CPU oracle runs them: qubit and qutrit
    circuits of each seed in turn."""
    return [(d, seed) for seed in rank_seeds(rank) for d in (2, 3)]


def cpu_oracle_sample(budget_s=None):
    """Time the oracle (as it stands, one thread) on whole benchmark circuits in bench_circuits order: all 16
    (budget_s None), or as many as start within budget_s seconds.  Returns (T gates / s, seconds, names,
    per-circuit seconds)."""
    from synth import brickwork_circuit
    from oracle.gcamps import GCAMPS
    t_gates, names, secs = 0, [], []
    t0 = time.perf_counter()
    for d, seed in bench_circuits(0):
        if budget_s is not None and names and time.perf_counter() - t0 > budget_s:
            break
        c0 = time.perf_counter()
        g = GCAMPS(N, d, chi_max=CHI, cutoff=CUTOFF)
        for gt in brickwork_circuit(N, d, LAYERS, T, seed):
            g.apply_gate(gt)
            if not hasattr(gt, "sp_index"):
                g.disentangle()
                t_gates += 1
        names.append(f"d{d}s{seed}")
        secs.append(time.perf_counter() - c0)
    el = time.perf_counter() - t0
    return t_gates / el, el, names, secs


def cpu_baseline_subprocess(budget_s: float):
    """The oracle's bounded sample in a fresh single-threaded process (BLAS threads pinned to 1 before numpy
    loads): the GPU arm's cpu_baseline."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1", RANK="0",
               WORLD_SIZE="1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ref-budget-s", str(budget_s),
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    line = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": line["value"], "unit": "T-gates/s", "cores": 1, "kind": "oracle",
            "sample": line["cpu_baseline"]["sample"]}


def _oracle_whole_circuit(shape):
    """One whole batched-workload circuit through the oracle (a pool worker): (T gates, seconds)."""
    from synth import brickwork_circuit
    from oracle.gcamps import GCAMPS
    n, layers, t, seed, d, chi = shape
    t0 = time.perf_counter()
    g = GCAMPS(n, d, chi_max=chi, cutoff=CUTOFF)
    tg = 0
    for gt in brickwork_circuit(n, d, layers, t, seed):
        g.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            g.disentangle()
            tg += 1
    return tg, time.perf_counter() - t0


def cpu_oracle_pool_sample(shapes, d: int, chi: int, budget_s: float, procs: int):
    """The oracle on all host cores, one process per circuit (spawned workers, one BLAS thread each):
    circuits of ``shapes`` are started in order while fewer than ``budget_s`` seconds have passed, and
    the ones in flight are then finished.  Returns (T gates / wall seconds, wall seconds, circuits)."""
    import multiprocessing as mp
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    todo = [(n, layers, t, seed, d, chi) for n, layers, t, seed in shapes]
    t_gates, done = 0, 0
    with ctx.Pool(procs) as pool:
        t0 = time.perf_counter()
        pending = []
        nxt = 0
        while nxt < len(todo) and len(pending) < procs:
            pending.append(pool.apply_async(_oracle_whole_circuit, (todo[nxt],)))
            nxt += 1
        while pending:
            ready = [r for r in pending if r.ready()]
            if not ready:
                time.sleep(0.01)
                continue
            for r in ready:
                pending.remove(r)
                tg, _sec = r.get()
                t_gates += tg
                done += 1
                if nxt < len(todo) and time.perf_counter() - t0 < budget_s:
                    pending.append(pool.apply_async(_oracle_whole_circuit, (todo[nxt],)))
                    nxt += 1
        wall = time.perf_counter() - t0
    return t_gates / wall, wall, done


def run_batched_reference(args):
    """--impl reference for the batched workload: the oracle on every host core (rank 0 only), each
    step a bounded sample of the circuits rank 0 runs, in order."""
    from synth import batched_workload
    rank, _world, _ = dist_env()
    if rank != 0:
        return 0
    procs = os.cpu_count() or 1
    shapes = batched_workload(args.batched_count, seed0=0, n_range=(16, args.batched_nmax),
                              layer_range=(16, args.batched_nmax))
    tg_total, wall_total, circuits = 0.0, 0.0, 0
    for i in range(args.warmup + args.steps):
        rate, wall, done = cpu_oracle_pool_sample(shapes, 3, 128, args.ref_step_s, procs)
        if i >= args.warmup:
            tg_total += rate * wall
            wall_total += wall
            circuits += done
    value = tg_total / wall_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "T-gates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall_total / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"gcamps-batched-{args.batched_count}-qutrit-n16..{args.batched_nmax}"
                               f"-L16..{args.batched_nmax}-T=n-chi128"},
        "cpu_baseline": {"value": value, "unit": "T-gates/s", "cores": procs, "kind": "oracle",
                         "sample": f"{circuits} whole circuits over {args.steps} steps, circuits started "
                                   f"in order for ~{args.ref_step_s}s per step, one process per circuit"},
        "e2e": {"value": value, "unit": "T-gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def init_ranks():
    """Process group for N > 1 (NCCL with a GPU, else gloo); returns (rank, world, local)."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def finish_ranks():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


def run_batched(args):
    """The batched form: 256 independent qutrit circuits of uneven size (n and layers uniform in
    [16, 48], n T gates each, chi_max = 128) in one handle; every step is one reset and one engine
    launch over all of them, captured once in a CUDA graph and replayed.  The CTAs per circuit are
    picked by measurement during the warm-up (2, 4 or 8: the autotuned shape)."""
    import ctypes as C
    import numpy as np
    import torch
    from synth import batched_workload, brickwork_circuit
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    d, chi = 3, 128
    count = args.batched_count
    shapes = batched_workload(count, seed0=rank * count, n_range=(16, args.batched_nmax),
                              layer_range=(16, args.batched_nmax))
    ops, begin = [], [0]
    for n, layers, t, seed in shapes:
        o = G.ops_from_gates(brickwork_circuit(n, d, layers, t, seed), d)
        ops.append(o)
        begin.append(begin[-1] + len(o))
    ops = np.concatenate(ops)
    stream = torch.cuda.Stream()
    sizes = [int(x) for x in args.batched_clusters.split(",")]
    sim = G.Simulator([x[0] for x in shapes], d, chi_max=chi, cutoff=CUTOFF, stream=stream, cluster_size=max(sizes))
    ops_dev = torch.from_numpy(ops.view(np.uint8)).to(f"cuda:{local}")
    begin_dev = torch.from_numpy(np.array(begin, dtype=np.int32)).to(f"cuda:{local}")
    lib = G._native.load()
    torch.cuda.synchronize()

    def step():
        rc = lib.gcamps_reset(sim._h)
        if rc == 0:
            rc = lib.gcamps_run_device(sim._h, C.c_void_p(ops_dev.data_ptr()), C.c_void_p(begin_dev.data_ptr()))
        if rc:
            raise RuntimeError(lib.gcamps_last_error(sim._h).decode())

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    tune = {}
    for cs in sizes:                 # autotune the CTAs per circuit on the workload itself
        sim.set_cluster_size(cs)
        tune[cs] = timed(step)
        progress(f"batched: {cs} CTAs per circuit: {tune[cs]:.2f} s")
    best = min(tune, key=tune.get)
    sim.set_cluster_size(best)
    graph = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        graph = g
    except Exception as ex:          # run uncaptured if this torch build cannot capture the launch
        progress(f"batched: graph capture failed ({ex}); launching directly")
    def replay():
        with torch.cuda.stream(stream):   # a graph replays on the current stream: make it the handle's
            graph.replay()

    run = replay if graph is not None else step
    for _ in range(max(0, args.warmup - 3)):
        timed(run)
    sim.sync()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = [timed(run) for _ in range(args.steps)]
    torch.cuda.synchronize()
    clk = clocks.stop()
    total = max_over_ranks(sum(times), device=f"cuda:{local}")
    stats = [sim.stats(c) for c in range(len(shapes))]
    if any(st["status"] for st in stats):
        raise RuntimeError("device status set")
    tg = sum(st["t_gates"] for st in stats)
    line = {
        "metric": METRIC, "value": aggregate_rate(tg, args.steps, world, total), "unit": "T-gates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"gcamps-batched-{count}-qutrit-n16..{args.batched_nmax}-L16..{args.batched_nmax}-T=n-chi128",
                   "circuits_per_rank": count,
                   "d": d, "chi_max": chi, "cutoff": CUTOFF, "cluster_ctas_per_circuit": best,
                   "autotune_s": {str(k): round(v, 3) for k, v in tune.items()},
                   "graph_captured": graph is not None, "parallelism": f"replicas x{world}",
                   "l2": "inputs (MPS, scratch) far larger than L2"},
        "candidates_per_s": sum(st["candidates_scored"] for st in stats) * args.steps * world / total,
        "max_chi": max(st["max_chi"] for st in stats),
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        procs = os.cpu_count() or 1
        rate, wall, done = cpu_oracle_pool_sample(shapes, d, chi, args.ref_step_s, procs)
        line["cpu_baseline"] = {"value": rate, "unit": "T-gates/s", "cores": procs, "kind": "oracle",
                                "sample": f"{done} whole circuits of this workload in order, one process per "
                                          f"circuit, {wall:.1f}s wall"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_gradient(args):
    """The differentiation form: qutrits n = 24, 20 layers, 48 parametrised gates
    diag(1, e^{i th}, e^{-i th}) (synth.param_phase_circuit, seed 1), chi_max = 256; one step = a forward
    run with snapshots and the adjoint gradient of Re<Z_0 Z_12> with respect to every gate's phases.
    Reports gradients/s, the split between the two passes, and whether the backward pass stayed exact
    (GCAMPS_ECHI otherwise)."""
    import numpy as np
    import torch
    from synth import param_phase_circuit
    rank, world, local = init_ranks()
    torch.cuda.set_device(local)
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    d, n, layers, ngates, chi = 3, 24, 20, 48, 256
    gates, _ = param_phase_circuit(n, d, layers, ngates, 1 + rank)
    if 0 < args.grad_prefix < ngates:   # the circuit up to its grad_prefix-th parametrised gate
        k, cut = 0, len(gates)
        for i, g in enumerate(gates):
            if not hasattr(g, "sp_index"):
                k += 1
                if k == args.grad_prefix:
                    cut = i + 1
                    break
        gates = gates[:cut]
    nparam = sum(1 for g in gates if not hasattr(g, "sp_index"))
    ops = G.ops_from_gates(gates, d)
    x = np.zeros(n, dtype=np.int32)
    z = np.zeros(n, dtype=np.int32)
    z[0] = z[12] = 1
    sim = G.Simulator(n, d, chi_max=chi, cutoff=1e-12, snapshot_entries=1 << 27, snapshot_max_gates=ngates)
    fwd, bwd, exact, err = [], [], True, ""
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        sim.reset()
        sim.run(ops)
        sim.sync()
        t1 = time.perf_counter()
        try:
            val, grad = sim.expect_gradient(x, z)
        except G.GcampsError as ex:
            exact, err = False, str(ex)
            val, grad = float("nan"), None
        t2 = time.perf_counter()
        progress(f"gradient step {i}: forward {t1 - t0:.2f} s, adjoint {t2 - t1:.2f} s")
        if i >= args.warmup:
            fwd.append(t1 - t0)
            bwd.append(t2 - t1)
        if not exact:
            break
    st = sim.stats()
    total = max_over_ranks(sum(fwd) + sum(bwd), device=f"cuda:{local}")
    line = {
        "metric": "gradients/s", "value": aggregate_rate(1, len(fwd), world, total) if exact and total > 0 else None,
        "unit": "gradients/s",
        "n_gpus": world, "steps": len(fwd), "warmup": args.warmup, "ms_per_step": 1e3 * total / max(1, len(fwd)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gcamps-gradient-qutrit-n24-L20-48params-chi256", "observable": "Re<Z_0 Z_12>",
                   "parametrised_gates_run": nparam, "timing": "host wall clock around synchronising calls"},
        "forward_s": float(np.mean(fwd)) if fwd else None, "adjoint_s": float(np.mean(bwd)) if bwd else None,
        "value_re": val, "exact": exact, "error": err, "max_chi": st["max_chi"],
        "forward_discarded_weight": st["discarded_weight"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    finish_ranks()
    return 0


def bond_dims_per_layer(layer_items, run_layer, bond_dims, budget_s: float = float("inf")):
    """Run a circuit one layer at a time (``run_layer`` on each item) and read the bond dimensions
    after every layer; stops early once ``budget_s`` seconds have passed.  Returns (dims per layer,
    seconds per layer)."""
    dims, secs = [], []
    t0 = time.perf_counter()
    for item in layer_items:
        t1 = time.perf_counter()
        run_layer(item)
        dims.append([int(c) for c in bond_dims()])
        secs.append(time.perf_counter() - t1)
        if time.perf_counter() - t0 > budget_s:
            break
    return dims, secs


def scaled_max_chi(dims_per_layer, n: int, d: int):
    """Largest bond dimension after each layer over the largest Schmidt rank d^floor(n/2) of n qudits
    (the bond-dimension axis of the paper's Fig. 5a; its layer axis is layers / n)."""
    full = d ** (n // 2)
    return [max(ds) / full for ds in dims_per_layer]


def chi_layer_shapes(args):
    ds = [int(v) for v in args.chi_layers_d.split(",") if v]
    ns = [int(v) for v in args.chi_layers_n.split(",") if v]
    return [(d, n, args.chi_layers_factor * n) for d in ds for n in ns]


def _curve_entry(d, n, layers, dims, secs):
    return {"d": d, "n": n, "layers_run": len(dims), "layers": layers,
            "scaled_layers": [round((k + 1) / n, 4) for k in range(len(dims))],
            "scaled_max_chi": [round(v, 6) for v in scaled_max_chi(dims, n, d)],
            "max_chi": [max(ds) for ds in dims], "seconds": round(sum(secs), 4)}


def run_chi_layers(args):
    """The bond-dimension-per-layer experiment of Fig. 5a on the circuit family of Fig. 4 (a random
    Clifford on all qudits, then a T gate on qudit 0, per layer; synth.layered_t_circuit, seed 1 plus
    the rank), run through the library one layer per launch with chi_max = d^floor(n/2) (no
    truncation by the bond cap) and cutoff 1e-12.  value = T gates / host wall time over all curves."""
    import torch
    from synth import layered_t_circuit
    rank, world, local = init_ranks()
    torch.cuda.set_device(local)
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    curves, total_t, total_s = [], 0, 0.0
    for d, n, layers in chi_layer_shapes(args):
        gates, ends = layered_t_circuit(n, d, layers, 1 + rank)
        starts = [0] + ends[:-1]
        layer_ops = [G.ops_from_gates(gates[a:b], d) for a, b in zip(starts, ends)]
        csize = args.cluster_qutrit if d == 3 else args.cluster_qubit
        sim = G.Simulator(n, d, chi_max=d ** (n // 2), cutoff=CUTOFF, cluster_size=csize or args.cluster,
                          score_kind=args.chi_layers_score_kind)
        dims, secs = bond_dims_per_layer(layer_ops, sim.run, sim.bond_dims, args.chi_layers_budget_s)
        sim.close()
        curves.append(_curve_entry(d, n, layers, dims, secs))
        total_t += len(dims)
        total_s += sum(secs)
        progress(f"chi-layers d={d} n={n}: {len(dims)} layers in {sum(secs):.2f} s")
    t_max = max_over_ranks(total_s, device=f"cuda:{local}")
    units = sum_over_ranks(total_t, device=f"cuda:{local}")   # ranks may stop at different layers
    line = {
        "metric": METRIC, "value": units / t_max if t_max > 0 else None,
        "unit": "T-gates/s", "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * t_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gcamps-fig4-layers-T-on-qudit-0", "chi_max": "d^floor(n/2)", "cutoff": CUTOFF,
                   "score_kind": args.chi_layers_score_kind,
                   "timing": "host wall clock around one synchronising launch per layer"},
        "curves": curves,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    finish_ranks()
    return 0


def run_chi_layers_reference(args):
    """The same experiment with the oracle on the host (rank 0 only), each curve bounded by
    --chi-layers-budget-s seconds."""
    rank, _world, _ = dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from synth import layered_t_circuit
    from oracle.gcamps import GCAMPS
    curves, total_t, total_s = [], 0, 0.0
    for d, n, layers in chi_layer_shapes(args):
        gates, ends = layered_t_circuit(n, d, layers, 1)
        starts = [0] + ends[:-1]
        ref = GCAMPS(n, d, chi_max=d ** (n // 2), cutoff=CUTOFF, score_kind=args.chi_layers_score_kind)

        def run_layer(gs, ref=ref):
            for gt in gs:
                ref.apply_gate(gt)
                if not hasattr(gt, "sp_index"):
                    ref.disentangle()

        dims, secs = bond_dims_per_layer([gates[a:b] for a, b in zip(starts, ends)], run_layer,
                                         ref.mps.bond_dims, args.chi_layers_budget_s)
        curves.append(_curve_entry(d, n, layers, dims, secs))
        total_t += len(dims)
        total_s += sum(secs)
    value = total_t / total_s if total_s > 0 else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "T-gates/s", "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * total_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gcamps-fig4-layers-T-on-qudit-0", "chi_max": "d^floor(n/2)", "cutoff": CUTOFF,
                   "score_kind": args.chi_layers_score_kind},
        "cpu_baseline": {"value": value, "unit": "T-gates/s", "cores": 1, "kind": "oracle",
                         "sample": f"layers until {args.chi_layers_budget_s} s per curve"},
        "e2e": {"value": value, "unit": "T-gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "curves": curves,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_case(args):
    """One seeded benchmark-family circuit (or a batch of consecutive seeds), reset and run in one engine
    launch per repetition: for profiling one launch (ncu) and for the per-phase cycle profile of the
    engine.  Prints one JSON line per repetition."""
    import numpy as np
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    from synth import brickwork_circuit
    ops, begin = [], [0]
    for b in range(args.case_batch):
        o = G.ops_from_gates(brickwork_circuit(args.case_n, args.case_d, args.case_layers, args.case_t,
                                               args.case_seed + b), args.case_d)
        if args.case_t_prefix > 0:   # the circuit up to the disentangling after its first case_t_prefix T gates
            ends = np.nonzero(o["kind"] == G.OP_DISENTANGLE)[0]
            if len(ends) > args.case_t_prefix:
                o = o[: ends[args.case_t_prefix - 1] + 1]
        ops.append(o)
        begin.append(begin[-1] + len(o))
    ops = np.concatenate(ops)
    sim = G.Simulator(args.case_n, args.case_d, chi_max=args.case_chi, cutoff=CUTOFF, batch=args.case_batch,
                      cluster_size=args.cluster, precision=args.case_precision)
    if args.exact_cta is not None:
        sim.set_exact_cta(args.exact_cta)
    for r in range(args.case_repeat):
        sim.reset()
        t0 = time.perf_counter()
        sim.run(ops, np.array(begin, dtype=np.int32))
        sim.sync()
        el = time.perf_counter() - t0
        st = [sim.stats(c) for c in range(args.case_batch)]
        line = {"workload": "case", "rep": r, "seconds": el, "d": args.case_d, "n": args.case_n,
                "layers": args.case_layers, "t_gates": args.case_t, "chi_max": args.case_chi,
                "seed": args.case_seed, "batch": args.case_batch, "cluster": args.cluster,
                "t_prefix": args.case_t_prefix, "precision": args.case_precision,
                "stats": st[0] if args.case_batch == 1 else st,
                "profile": [sim.profile(c) for c in range(args.case_batch)]}
        print(json.dumps(line), flush=True)
    sim.close()
    return 0


PREC_N, PREC_LAYERS, PREC_T, PREC_CHI = 64, 40, 64, 1024
PREC_WORKLOAD = "gcamps-brickwork-n64-L40-T64-chi1024-d3"


def weyl_probes(n: int):
    """Weyl strings whose expectation both forms report: Z_j (every 4th qudit), Z_0 Z_{n/5}, X_j Z_{j+1}."""
    probes = []
    for j in range(0, n, 4):
        x, z = [0] * n, [0] * n
        z[j] = 1
        probes.append((x, z))
    x, z = [0] * n, [0] * n
    z[0], z[n // 5] = 1, 1
    probes.append((x, z))
    for j in range(0, n - 1, 8):
        x, z = [0] * n, [0] * n
        x[j], z[j + 1] = 1, 1
        probes.append((x, z))
    return probes


def run_precision(args):
    """The precision form against the FP64 form on the precision configuration: qutrits, n = 64, 40 brickwork
    layers, 64 T gates, chi_max = 1024, cutoff 1e-12, seeds 1..S, each circuit up to its --prec-prefix-th T
    gate, one circuit at a time (a handle of this shape reserves about 37 GB).  Per seed and form: W warm-up and
    K timed launches (device time, L2 flushed before each).  value = T-gates/s of the precision form over all
    seeds; fp64 = the same for the FP64 form.  Errors of the precision run against the FP64 run: |<W>|
    differences for the probe strings (each form in its own Clifford frame), and, replaying the FP64 decisions,
    the fidelity |<M|M'>|^2 (equal tableaux checked bit for bit)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    from synth import brickwork_circuit
    seeds = [1 + s + rank * args.prec_seeds for s in range(args.prec_seeds)]
    dev = f"cuda:{local}"
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    probes = weyl_probes(PREC_N)
    acc = {0: {"t": 0.0, "tg": 0, "max_chi": 0, "visits": 0, "exact": 0, "tensor_flops": 0.0},
           1: {"t": 0.0, "tg": 0, "max_chi": 0, "visits": 0, "exact": 0, "tensor_flops": 0.0}}
    werr, fid_err, same_dec, e2e_t, e2e_tg, per_seed = 0.0, 0.0, 0, 0.0, 0, []
    clocks = ClockSampler(local)
    clocks.start()
    for sd in seeds:
        o = G.ops_from_gates(brickwork_circuit(PREC_N, 3, PREC_LAYERS, PREC_T, sd), 3)
        ends = np.nonzero(o["kind"] == G.OP_DISENTANGLE)[0]
        if 0 < args.prec_prefix < len(ends):   # the circuit up to the disentangling after its prefix-th T gate
            o = o[: ends[args.prec_prefix - 1] + 1]
        tg = int(np.sum(o["kind"] == G.OP_NONCLIFFORD))
        ops_dev = torch.from_numpy(o.view(np.uint8)).to(dev)
        begin_dev = torch.tensor([0, len(o)], dtype=torch.int32, device=dev)
        sims, secs = {}, {}
        for prec in (0, 1):
            stream = torch.cuda.Stream()
            sim = G.Simulator(PREC_N, 3, chi_max=PREC_CHI, cutoff=CUTOFF, stream=stream, cluster_size=16,
                              precision=prec)
            for _ in range(args.warmup):
                sim.reset()
                sim.run_device(ops_dev.data_ptr(), begin_dev.data_ptr())
            sim.sync()
            times = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.reset()
                sim.run_device(ops_dev.data_ptr(), begin_dev.data_ptr())
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
            st = sim.stats()
            if st["status"]:
                raise RuntimeError(f"device status {st['status']} (seed {sd}, precision {prec})")
            a = acc[prec]
            a["t"] += sum(times)
            a["tg"] += tg * args.steps
            a["max_chi"] = max(a["max_chi"], st["max_chi"])
            a["visits"] += st["bonds_visited"]
            a["exact"] += st["vn_evaluations"]
            a["tensor_flops"] += st["tensor_flops"] * args.steps
            sims[prec], secs[prec] = sim, sum(times) / args.steps
        for x, z in probes:
            werr = max(werr, abs(sims[1].expect_weyl(x, z) - sims[0].expect_weyl(x, z)))
        dec0 = sims[0].decisions()
        same_dec += sims[1].decisions() == dec0
        # e2e of the precision form through the C ABI: host gate list copied in, bond dimensions read back
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sims[1].reset()
        sims[1].run(o)
        dims = sims[1].bond_dims()
        e2e_t += time.perf_counter() - t0
        e2e_tg += tg
        sims[1].close()
        rep = G.Simulator(PREC_N, 3, chi_max=PREC_CHI, cutoff=CUTOFF, cluster_size=16, precision=1)
        rep.set_replay(dec0)
        rep.run(o)
        rep.sync()
        ea, pa = sims[0].tableau()
        eb, pb = rep.tableau()
        if not (np.array_equal(ea, eb) and np.array_equal(pa, pb)):
            raise RuntimeError("replayed tableau differs")
        fid_err = max(fid_err, 1.0 - abs(sims[0].overlap(rep)) ** 2)
        rep.close()
        sims[0].close()
        per_seed.append({"seed": sd, "t_gates": tg, "fp64_s": round(secs[0], 4), "precision_s": round(secs[1], 4)})
        progress(f"precision workload seed {sd}: fp64 {secs[0]:.3f} s, precision {secs[1]:.3f} s")
    clk = clocks.stop()
    v = {p: acc[p]["tg"] / acc[p]["t"] for p in (0, 1)}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        tf32_peak, tf32_src = bf16 * 1.1 / 2.25, "measured bf16 burst x nominal tf32/bf16 ratio (1.1/2.25)"
    except (OSError, ValueError, KeyError):
        tf32_peak, tf32_src = 1900.0 * 1.1 / 2.25, "fallback bf16 x nominal tf32/bf16 ratio"
    tc_ach = acc[1]["tensor_flops"] / acc[1]["t"] / 1e12
    summary = lambda p: {"value": v[p], "seconds": acc[p]["t"], "max_chi": acc[p]["max_chi"],  # noqa: E731
                         "bond_visits": acc[p]["visits"], "exact_evaluations": acc[p]["exact"],
                         "tensor_flops_per_step": acc[p]["tensor_flops"] / args.steps}
    line = {
        "metric": "T-gates/s (precision form)", "value": v[1], "unit": "T-gates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * acc[1]["t"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 contractions (tf32x3 tensor cores), f64 eigen/SVD/score", "data": "synthetic",
        "config": {"workload": PREC_WORKLOAD, "n": PREC_N, "layers": PREC_LAYERS, "t_gates": PREC_T,
                   "chi_max": PREC_CHI, "cutoff": CUTOFF, "d": 3, "seeds": seeds,
                   "t_gate_prefix": args.prec_prefix if args.prec_prefix > 0 else PREC_T,
                   "l2": "512 MiB flush before every timed launch", "step": "one launch per seed, in turn"},
        "fp64": summary(0), "precision": summary(1), "speedup_vs_fp64": v[1] / v[0], "per_seed": per_seed,
        "errors_vs_fp64": {"max_abs_weyl_expectation": werr, "probes_per_circuit": len(probes),
                           "replay_fidelity_error": fid_err, "circuits_with_identical_decisions": same_dec},
        "roofline": {"bound": "tensor", "achieved": tc_ach, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": tc_ach / tf32_peak, "traffic": None, "peak_source": tf32_src,
                     "kernel": "k_run_tc (tensor-core Grams of CTA-level class evaluations)"},
        "e2e": {"value": e2e_tg / e2e_t, "unit": "T-gates/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": 4 * (PREC_N - 1), "note": "one C-ABI run per seed, gate list from host"},
        "gpu_launches": 2 * len(seeds) * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", RANK="0", WORLD_SIZE="1")
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                            "precision", "--ref-budget-s", "20", "--prec-seeds", str(args.prec_seeds), "--prec-prefix",
                            str(args.prec_prefix), "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                           text=True, timeout=900)
        ref = json.loads(r.stdout.strip().splitlines()[-1])
        line["cpu_baseline"] = {k: ref["cpu_baseline"][k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def precision_oracle_sample(seeds, prefix, budget_s=None):
    """The FP64 oracle (one thread) on the precision workload's circuits, each up to its prefix-th T gate, seeds in
    order (those that start within budget_s seconds).  Returns (T gates / s, seconds, seeds run)."""
    from synth import brickwork_circuit
    from oracle.gcamps import GCAMPS
    t0 = time.perf_counter()
    tg, done = 0, []
    for sd in seeds:
        if budget_s is not None and done and time.perf_counter() - t0 > budget_s:
            break
        g = GCAMPS(PREC_N, 3, chi_max=PREC_CHI, cutoff=CUTOFF)
        k = 0
        for gt in brickwork_circuit(PREC_N, 3, PREC_LAYERS, PREC_T, sd):
            g.apply_gate(gt)
            if not hasattr(gt, "sp_index"):
                g.disentangle()
                k += 1
                if 0 < prefix <= k:
                    break
        tg += k
        done.append(sd)
    el = time.perf_counter() - t0
    return tg / el, el, done


def run_precision_reference(args):
    """--impl reference --workload precision: the oracle on the precision workload (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    seeds = [1 + s for s in range(args.prec_seeds)]
    rate, el, done = precision_oracle_sample(seeds, args.prec_prefix, args.ref_budget_s)
    line = {
        "impl": "reference", "metric": "T-gates/s (precision form)", "value": rate, "unit": "T-gates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": PREC_WORKLOAD, "n": PREC_N, "layers": PREC_LAYERS, "t_gates": PREC_T,
                   "chi_max": PREC_CHI, "cutoff": CUTOFF, "d": 3, "seeds": seeds,
                   "t_gate_prefix": args.prec_prefix if args.prec_prefix > 0 else PREC_T,
                   "l2": "512 MiB flush before every timed launch", "step": "one launch per seed, in turn"},
        "cpu_baseline": {"value": rate, "unit": "T-gates/s", "cores": 1, "kind": "oracle",
                         "sample": f"seeds {done} up to T gate {args.prec_prefix} ({el:.1f} s, 1 thread)"},
        "e2e": {"value": rate, "unit": "T-gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """--impl reference: the FP64 CPU oracle (as it stands, one thread) on the GPU arm's own 16 circuits, one
    whole pass of them in the timed region, split over the --steps steps in bench_circuits order (with
    --ref-budget-s: only the circuits that start within that many seconds).  Warm-up steps run the first
    circuit."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_sample(budget_s=0.0)
    rate, el, names, secs = cpu_oracle_sample(budget_s=args.ref_budget_s)
    full = args.ref_budget_s is None
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "T-gates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(world if full else 1),
        "cpu_baseline": {"value": rate, "unit": "T-gates/s", "cores": 1, "kind": "oracle",
                         "sample": (f"all {len(names)} benchmark circuits once" if full and len(names) == 2 * SEEDS_PER_D
                                    else f"{len(names)} whole circuits {','.join(names)}") + f" ({el:.1f} s, 1 thread)",
                         "seconds_per_circuit": {n_: round(t_, 3) for n_, t_ in zip(names, secs)}},
        "e2e": {"value": rate, "unit": "T-gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_config(world: int) -> dict:
    """The workload of both arms (the same dict in the GPU line and the reference line)."""
    return {"workload": WORKLOAD, "n": N, "layers": LAYERS, "t_gates": T, "chi_max": CHI, "cutoff": CUTOFF,
            "d": [2, 3], "seeds_per_d": SEEDS_PER_D, "circuits_per_rank": 2 * SEEDS_PER_D,
            "l2": "512 MiB flush before every timed step", "parallelism": f"replicas x{world}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gcamps", choices=["gcamps", "reference"])
    ap.add_argument("--prec-seeds", type=int, default=8, help="precision workload: circuits per rank")
    ap.add_argument("--grad-prefix", type=int, default=0,
                    help="gradient workload: parametrised gates run (0: all 48)")
    ap.add_argument("--prec-prefix", type=int, default=48,
                    help="precision workload: T gates run per circuit (0: all 64; past about 48 T gates most seeds "
                         "reach 243 x 243 two-site tensors, where one T gate takes tens of seconds in FP64)")
    ap.add_argument("--workload", default="bench",
                    choices=["bench", "batched", "gradient", "chi-layers", "case", "precision"],
                    help="bench: the 16-circuit n=32 workload; batched: uneven qutrit circuits in one launch; "
                         "gradient: forward + adjoint; chi-layers: bond dimension after every layer (Fig. 5a); "
                         "case: one seeded circuit per launch with its engine profile (for ncu)")
    ap.add_argument("--case-d", type=int, default=3)
    ap.add_argument("--case-n", type=int, default=12)
    ap.add_argument("--case-layers", type=int, default=10)
    ap.add_argument("--case-t", type=int, default=12)
    ap.add_argument("--case-chi", type=int, default=64)
    ap.add_argument("--case-seed", type=int, default=1)
    ap.add_argument("--case-batch", type=int, default=1)
    ap.add_argument("--case-repeat", type=int, default=2)
    ap.add_argument("--case-t-prefix", type=int, default=0, help="run only up to the K-th T gate (0: all)")
    ap.add_argument("--case-precision", type=int, default=0, choices=[0, 1], help="0 FP64, 1 precision form")
    ap.add_argument("--chi-layers-d", default="2,3")
    ap.add_argument("--chi-layers-n", default="6,8")
    ap.add_argument("--chi-layers-factor", type=int, default=2, help="layers = this x n")
    ap.add_argument("--chi-layers-budget-s", type=float, default=60.0, help="per curve; later layers are skipped")
    ap.add_argument("--chi-layers-score-kind", type=int, default=0, choices=[0, 1, 2],
                    help="disentangler score: 0 von Neumann, 1 Renyi-2, 2 weight rank (bond-dimension criterion)")
    ap.add_argument("--batched-count", type=int, default=64)
    ap.add_argument("--batched-nmax", type=int, default=24, help="n and layers uniform in [16, this]")
    ap.add_argument("--batched-clusters", default="8,4", help="CTAs per circuit tried by the autotuner")
    ap.add_argument("--ref-step-s", type=float, default=8.0, help="batched reference arm: seconds per step")
    ap.add_argument("--ref-budget-s", type=float, default=None,
                    help="bench reference arm: only the circuits that start within this many seconds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sm-ids", action="store_true", help="print the SM each CTA of each circuit ran on")
    ap.add_argument("--exact-cta", type=int, default=None,
                    help="exact class evaluations of m <= 27 one per CTA from this m on (library default 10)")
    ap.add_argument("--cluster", type=int, default=8, help="CTAs per circuit (thread-block cluster)")
    ap.add_argument("--cluster-qubit", type=int, default=4, help="CTAs per qubit circuit (0: --cluster)")
    ap.add_argument("--cluster-qutrit", type=int, default=16, help="CTAs per qutrit circuit (0: --cluster)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload == "chi-layers":
            return run_chi_layers_reference(args)
        if args.workload == "batched":
            return run_batched_reference(args)
        if args.workload == "precision":
            return run_precision_reference(args)
        if args.workload == "gradient":
            if dist_env()[0] == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle's gradient is a dense "
                                  "state-vector adjoint; 3^24 amplitudes at n = 24 do not fit in host memory"}),
                      flush=True)
            return 0
        return run_reference(args)
    if args.workload == "case":
        return run_case(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "chi-layers":
        return run_chi_layers(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "gradient":
        return run_gradient(args)

    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G

    stream = torch.cuda.Stream()
    streams = {2: torch.cuda.Stream(), 3: torch.cuda.Stream()}   # the two handles run concurrently
    sims, ops_host, ops_dev, begin_dev = {}, {}, {}, {}
    cluster = {2: args.cluster_qubit or args.cluster, 3: args.cluster_qutrit or args.cluster}
    for d in (2, 3):
        sims[d] = G.Simulator(N, d, chi_max=CHI, cutoff=CUTOFF, batch=SEEDS_PER_D, stream=streams[d],
                              cluster_size=cluster[d])
        if args.exact_cta is not None:
            sims[d].set_exact_cta(args.exact_cta)
        o, b = workload_ops(G, d, rank)
        # e2e inputs live in pinned host memory
        o_pin = torch.from_numpy(o.view(np.uint8).copy()).pin_memory().numpy().view(G.OP_DTYPE)
        b_pin = torch.from_numpy(b.copy()).pin_memory().numpy()
        ops_host[d] = (o_pin, b_pin)
        ops_dev[d] = torch.from_numpy(o.view(np.uint8)).to(f"cuda:{local}")
        begin_dev[d] = torch.from_numpy(b).to(f"cuda:{local}")
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    lib = G._native.load()
    import ctypes as C

    def launch_all(events=None):
        """One step: back to |0...0> and C = I, then the full gate list of every circuit (one
        engine launch per d).  The qubit and qutrit handles run on their own streams, forked from
        and joined back into `stream`.  `events`: optional (start, end) CUDA-event pairs recorded
        around each engine launch on its stream."""
        fork = torch.cuda.Event()
        fork.record(stream)
        for i, d in enumerate((2, 3)):   # the order of the end-to-end loop below
            s = sims[d]
            streams[d].wait_event(fork)
            rc = lib.gcamps_reset(s._h)
            if events is not None:
                events[i][0].record(streams[d])
            if rc == 0:
                rc = lib.gcamps_run_device(s._h, C.c_void_p(ops_dev[d].data_ptr()),
                                           C.c_void_p(begin_dev[d].data_ptr()))
            if events is not None:
                events[i][1].record(streams[d])
            if rc:
                raise RuntimeError(lib.gcamps_last_error(s._h).decode())
            join = torch.cuda.Event()
            join.record(streams[d])
            stream.wait_event(join)

    # warm-up (also checks status)
    progress("handles ready; warm-up")
    for w in range(args.warmup):
        t0 = time.perf_counter()
        launch_all()
        stream.synchronize()
        progress(f"warm-up step {w}: {time.perf_counter() - t0:.2f} s")
    for d in (2, 3):
        sims[d].sync()

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, engine_times = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        ev0, ev1 = mk(), mk()
        inner = [(mk(), mk()), (mk(), mk())]
        ev0.record(stream)
        launch_all(inner)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        engine_times.extend(a.elapsed_time(b) / 1e3 for a, b in inner)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_time = max_over_ranks(sum(times), device=f"cuda:{local}")
    stats = {d: [sims[d].stats(c) for c in range(SEEDS_PER_D)] for d in (2, 3)}
    for d in (2, 3):
        for st in stats[d]:
            if st["status"] != 0:
                raise RuntimeError(f"device status {st['status']}")
    tg_per_step = sum(st["t_gates"] for d in (2, 3) for st in stats[d])
    cand_per_step = sum(st["candidates_scored"] for d in (2, 3) for st in stats[d])
    value = aggregate_rate(tg_per_step, args.steps, world, total_time)
    cand_rate = aggregate_rate(cand_per_step, args.steps, world, total_time)
    vn_frac = sum(st["vn_evaluations"] for d in (2, 3) for st in stats[d]) / max(1, cand_per_step)
    # algorithmic work (the exhaustive search: every class of every visit scored exactly, the per-class
    # count of the scope table) and the FP64 work the engine executed (the classes its bounds left)
    flops_per_launch = sum(st["algorithmic_flops"] for d in (2, 3) for st in stats[d]) / 2.0
    executed_per_launch = sum(st["scoring_flops"] for d in (2, 3) for st in stats[d]) / 2.0
    screen_per_launch = sum(st["screen_flops"] for d in (2, 3) for st in stats[d]) / 2.0
    launch_s = sum(engine_times) / len(engine_times)
    achieved = flops_per_launch / launch_s / 1e12
    screen_achieved = screen_per_launch / launch_s / 1e12
    fp64_peak, fp32_peak, peak_src = arith_peaks()
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": engine_traffic(),
                "kernel": "k_run (engine, one launch per d)", "flops_per_launch": flops_per_launch,
                "launch_ms": 1e3 * launch_s, "peak_source": "FP64 fma, " + peak_src,
                "flops_definition": "K classes x (8 d^2 R C + 4 m (m + 1) M + (16/3) m^3) FP64 flops per bond visit "
                                    "with m > 1 (every class scored exactly, as the exhaustive search does)",
                "executed_fp64": {"flops_per_launch": executed_per_launch,
                                  "achieved": executed_per_launch / launch_s / 1e12,
                                  "frac": executed_per_launch / launch_s / 1e12 / fp64_peak},
                "fp32_screen": {"flops_per_launch": screen_per_launch, "achieved": screen_achieved,
                                "peak": fp32_peak, "frac": screen_achieved / fp32_peak,
                                "peak_source": "FP32 fma, " + peak_src}}

    progress(f"timed steps: {[round(t, 3) for t in times]}")
    if args.sm_ids:
        for d in (2, 3):
            for c in range(SEEDS_PER_D):
                progress(f"d{d} circuit {c} SM ids: {sims[d].profile(c)['sm_ids']}")
    # end to end: host gate lists, copies and readback inside the timed region
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e2e_times = []
    h2d = sum(ops_host[d][0].nbytes + ops_host[d][1].nbytes for d in (2, 3))
    d2h = 0
    for _ in range(max(2, args.steps)):
        flush.fill_(1.0)   # L2 flushed as before the device-timed steps, outside the timed region
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d in (2, 3):
            sims[d].reset()
            sims[d].run(*ops_host[d])
        res = []
        for d in (2, 3):
            for c in range(SEEDS_PER_D):
                res.append(sims[d].bond_dims(c))
        e2e_times.append(time.perf_counter() - t0)
        d2h = sum(len(r) * 4 for r in res)
    e2e_total = max_over_ranks(sum(e2e_times), device=f"cuda:{local}")   # slowest rank, as for value
    e2e_value = aggregate_rate(tg_per_step, len(e2e_times), world, e2e_total)

    line = {
        "metric": METRIC, "value": value, "unit": "T-gates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(world),
        "launch": {"cluster_ctas_per_circuit": {"d2": cluster[2], "d3": cluster[3]}},
        "candidates_per_s": cand_rate,
        "vn_evaluated_fraction": vn_frac,
        "e2e": {"value": e2e_value, "unit": "T-gates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * 2 * args.steps,
        "roofline": roofline,
        "clocks": clk,
    }
    progress(f"e2e steps: {[round(t, 3) for t in e2e_times]}")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(15.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for d in (2, 3):
        sims[d].close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
