"""Throughput of the mesh-registration hot path on GB300.

One step = one whole registration of one 512x512 image pair with a ~20k-node
mesh: B-spline prefilter of both images, node samples of Re, pixel ->
triangle map, 200 iterations (sampling, Eq. 9-10 force, semi-implicit
umbrella solve by Jacobi-PCG), dense warp and MSD, all on the device.
Metric: registrations/s (and node-iterations/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--mode S1] [--config 1]

--config 3 times the batched form instead: one step registers 256 pairs of
uneven size (sides 96-768, 500-40k nodes, 100 iterations each) in one CUDA
graph launch around one persistent kernel, with the team shape chosen by the
library's autotuner before timing.

The default run (config 1) also times the other forms briefly and reports
them under "forms": the batched engine on the 256-pair workload (FP32, and
with BF16- and FP16-stored coefficients), the same pairs through one-pair
handles on 8 CUDA streams (the plain FP32 form), and the differentiation
form (--no-forms skips them).  Its line carries "parity": the timed run's final node
displacements and MSD against one full FP64 oracle registration of the same
pair.

--impl reference times the FP64 CPU oracle on the host cores instead: each
timed step is one whole registration (all iterations) of the same pair.
Under torchrun (N > 1) every rank registers its own pairs on its own GPU
(independent replicas, weak scaling); rank 0 prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1411_2141_gb300 import inputs  # noqa: E402

MODE_NAMES = {"S0": "explicit Eq.5+Eq.14", "S1": "umbrella-implicit solve",
              "S2": "P1-FEM-implicit solve"}
SOLVER_NAMES = {"chebyshev": "Jacobi-Chebyshev semi-iteration, verified residual",
                "cg": "Jacobi-PCG", "none": "no solve"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=1)
    p.add_argument("--mode", default="S1", choices=["S0", "S1", "S2"])
    p.add_argument("--grad", default="G0", choices=["G0", "G1"])
    p.add_argument("--solver", default="auto", choices=["auto", "cg", "chebyshev"],
                   help="linear solve of the semi-implicit forms (auto: Chebyshev for S1, CG for S2)")
    p.add_argument("--neighbour-sync", action="store_true",
                   help="synchronise the Chebyshev steps by neighbour blocks instead of the grid "
                        "barrier (the library's option; measured slower on the 512^2 pair)")
    p.add_argument("--coeff", default="fp32", choices=["fp32", "bf16", "fp16"],
                   help="storage of Te's spline coefficients (bf16, fp16: the precision form)")
    p.add_argument("--team", default=None,
                   help="config 3: fixed team shape 'ctas,block[,blocks_per_sm]' instead of "
                        "the autotuner")
    p.add_argument("--teams", type=int, default=0,
                   help="config 3 with --team: number of teams (0 = as many as are co-resident)")
    p.add_argument("--pairs", type=int, default=0,
                   help="config 3: only the first N pairs of the batch (small profiling case)")
    p.add_argument("--single", action="store_true",
                   help="config 3: register the pairs one after another with the one-pair "
                        "engine (the plain FP32 form) instead of the batched engine")
    p.add_argument("--streams", type=int, default=8,
                   help="differentiation form and --single: CUDA streams the pairs are spread over")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--operator", action="store_true",
                   help="config 3: also time the batched system-matrix product y = A x (the "
                        "standalone SpMV) against the HBM roofline")
    p.add_argument("--checkpoint", type=int, default=0,
                   help="config 4: keep every C-th state of the unroll and recompute the "
                        "segments in the backward pass (0: keep every state)")
    p.add_argument("--no-forms", action="store_true",
                   help="config 1: skip the short runs of the batched, plain-on-streams and "
                        "differentiation forms")
    return p.parse_args()


# ------------------------------------------------------------- bytes model
def algorithmic_bytes_per_iteration(n_v: int, n_t: int, nnz: int, mode: str, cg_its: float,
                                    solver: str = "cg") -> float:
    """Compulsory bytes of one iteration of the iteration kernel (each array
    read or written once; gathers of neighbours counted once per node).
    cg_its: mean iterations (CG) or steps (Chebyshev) of a solve."""
    sample = n_v * (8 + 8 + 4 + 4)                          # V, u, Re(V) in; f out
    force = 4 * (n_v + 1) + 4 * 3 * n_t + 12 * n_t + 8 * n_v  # inc CSR, triangles, F out
    if mode == "S0":
        update = 4 * (n_v + 1) + 4 * nnz + 8 * n_v + 8 * n_v + 8 * n_v  # graph, u0 out/in, u out
        return sample + force + update
    graph = 4 * (n_v + 1) + 4 * nnz
    if mode == "S1" and solver == "chebyshev":
        # first phase: graph, x in; b out, previous b in (verification); d, x' out;
        # 1/diag(A); the two earlier iterates in and this one out (extrapolated guess)
        first = graph + 8 * n_v + 16 * n_v + 16 * n_v + 8 * n_v + 8 * n_v + 4 * n_v + 24 * n_v
        # each further step: graph, x and b in, d in and out, 1/diag(A), x' out
        step = graph + 8 * n_v + 16 * n_v + 16 * n_v + 4 * n_v + 8 * n_v
        return sample + force + first + max(cg_its - 1.0, 0.0) * step
    vals = (8 * nnz + 8 * n_v) if mode == "S2" else 0
    init = graph + vals + 8 * n_v + 16 * n_v + 8 * n_v + 8 * n_v + 4 * n_v   # u, b, r, z out, dinv
    cg1 = graph + vals / 2 + 8 * n_v * 3 + 16 * n_v + 8 * n_v * 3           # z, p, x, b in; p', q, rt out
    cg2 = 8 * n_v * 4 + 4 * n_v + 8 * n_v * 3                                # p, q, x, r in; x, r, z out
    return sample + force + init + cg_its * (cg1 + cg2)


def solver_of(args) -> str:
    """The linear solver the run uses: the library's default is Chebyshev
    semi-iteration for S1 and CG for S2 (--solver overrides)."""
    if args.mode == "S1" and args.solver in ("auto", "chebyshev"):
        return "chebyshev"
    return "cg" if args.mode != "S0" else "none"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: wait (before the timed region)
            # for its first sample so that the samples cover the region
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU side
def oracle_registration(case, mode: str, grad: str, n_iter: int | None = None):
    """One whole registration by the FP64 oracle (set-up, n_iter iterations,
    default the workload's full count, and the MSD): (seconds, u, MSD)."""
    from oracle import register
    t0 = time.perf_counter()
    pb = register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau, mode, grad)
    u, _ = pb.run(case.spec.n_iter if n_iter is None else n_iter)
    msd = pb.msd(u)
    return time.perf_counter() - t0, u, msd


def host_cpu() -> dict:
    """The host cores the oracle runs on (it uses one of them)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "processor name"):
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model}


def parity_against_oracle(u, msd, u_ref, msd_ref, u_tol: float = 1e-4, msd_rtol: float = 1e-5) -> dict:
    """Node displacements and MSD of a GPU run against the FP64 oracle's."""
    du = float(np.abs(np.asarray(u, np.float64) - u_ref).max())
    dm = float(abs(msd - msd_ref) / msd_ref)
    return {"max_du_px": du, "msd_rel": dm, "u_tol_px": u_tol, "msd_rtol": msd_rtol,
            "pass": bool(du <= u_tol and dm <= msd_rtol)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.config == 3:
        return run_reference_batch(args)
    if args.config == 4:
        return run_reference_adjoint(args)
    spec = inputs.config_spec(args.config)
    case = inputs.make_case(spec)
    for _ in range(args.warmup):   # warm-up: set-up and a short run, untimed
        oracle_registration(case, args.mode, args.grad, n_iter=2)
    times = []
    for _ in range(args.steps):
        t, _, _ = oracle_registration(case, args.mode, args.grad)
        times.append(t)
    sec = sum(times)
    value = args.steps / sec
    line = {
        "impl": "reference", "metric": "registrations/s", "value": value, "unit": "registrations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, case),
        "node_iters_per_s": value * case.n_nodes * spec.n_iter,
        "cpu_baseline": {"value": value, "unit": "registrations/s", "cores": 1, "kind": "oracle",
                         "host": host_cpu(),
                         "sample": f"per step: one whole registration (set-up, all {spec.n_iter} "
                                   f"iterations, MSD), numpy/scipy FP64, 1 thread"},
        "e2e": {"value": value, "unit": "registrations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def launches_per_registration(args, n_iter: int) -> int:
    """Our kernels in one timed step: prefilter (row and column pass) of Re
    and Te, [BF16 copy], Re at the nodes, [Re at edge midpoints], pixel map
    (fill + map), the persistent iteration kernel and its energy pass per
    1024-iteration chunk, the warp's per-triangle affine records, warp + MSD
    and the final MSD sum."""
    chunks = (n_iter + 1023) // 1024
    return (4 + (args.coeff != "fp32") + 1 + 2 + 2 * chunks + 3)


def run_reference_adjoint(args):
    from oracle import adjoint, register
    cases = adjoint_cases(args.pairs)
    K = cases[0].spec.n_iter
    total, n = 0.0, 0
    for step in range(args.warmup + args.steps):
        c = cases[step % len(cases)]
        t0 = time.perf_counter()
        pb = register.Problem(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, "S0", "G1")
        adjoint.unrolled_grad(pb, _smooth_u0(c).astype(np.float64), K)
        if step >= args.warmup:
            total += time.perf_counter() - t0
            n += 1
    value = n / total
    line = {
        "impl": "reference", "metric": "unrolled gradients/s", "value": value,
        "unit": "gradients/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / n, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"config4: pairs of 256x256, gradient through {K} iterations",
                   "pairs": len(cases), "iterations": K},
        "cpu_baseline": {"value": value, "unit": "gradients/s", "cores": 1, "kind": "oracle",
                         "sample": "per step: one pair's set-up, forward iterations and adjoint"},
        "e2e": {"value": value, "unit": "gradients/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_batch(args):
    cases = batch_cases(args.pairs)
    n_iter = cases[0].spec.n_iter
    for _ in range(args.warmup):
        oracle_registration(cases[0], args.mode, args.grad, n_iter=2)
    measured, est, pick = 0.0, 0.0, None
    for _ in range(args.steps):
        t, t_all, pick = oracle_batch_time(cases, args.mode, args.grad, n_sample_pairs=4)
        measured += t
        est += t_all
    value = args.steps * len(cases) / est
    sample = (f"per step: whole registrations ({n_iter} iterations) of {len(pick)} of the "
              f"{len(cases)} pairs, spread over the size range; the rate per node applied to "
              f"the whole batch (ms_per_step is the measured time of the sampled pairs)")
    line = {
        "impl": "reference", "metric": "registrations/s", "value": value, "unit": "registrations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * measured / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batch_workload_config(args, cases),
        "cpu_baseline": {"value": value, "unit": "registrations/s", "cores": 1, "kind": "oracle",
                         "host": host_cpu(), "sample": sample},
        "e2e": {"value": value, "unit": "registrations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, case):
    s = case.spec
    return {"workload": f"config{args.config}: {s.side}x{s.side} pair, {case.n_nodes}-node mesh, "
                        f"{s.n_iter} iterations, {args.mode} {MODE_NAMES[args.mode]}"
                        f"{' (' + SOLVER_NAMES[solver_of(args)] + ')' if args.mode != 'S0' else ''}, "
                        f"{args.grad} {'mesh gradient Eq.9-10' if args.grad == 'G0' else 'spline gradient'}"
                        + (f", {args.coeff.upper()}-stored Te coefficients" if args.coeff != "fp32" else ""),
            "image": [s.side, s.side], "nodes": case.n_nodes, "triangles": case.n_tris,
            "iterations": s.n_iter, "mode": args.mode, "grad": args.grad, "coeff": args.coeff,
            "solver": solver_of(args), "alpha": s.alpha, "tau": s.tau,
            "l2": "flushed between timed steps (256 MiB write, then 256 MiB read); the step's own working set is L2-resident",
            "parallelism": f"replicas x{args.gpus} (one pair per GPU per step)"}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (x itself when world == 1)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def pair_cost(case) -> float:
    """Work of one pair when a batch is split over ranks: its node-iterations
    plus its pixels (the set-up and the warp)."""
    return float(case.n_nodes) * case.spec.n_iter + float(case.Re.size)


def lpt_partition(costs, world: int) -> list[list[int]]:
    """Greedy longest-processing-time split of independent pairs over ranks:
    pairs in decreasing cost (ties by index), each to the rank with the
    smallest total so far (ties: lowest rank).  Deterministic, so every rank
    computes the same split; each rank's list is in ascending pair order."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += costs[k]
    return [sorted(p) for p in parts]


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second of the slowest rank (weak scaling)."""
    return units_per_rank * world / seconds


PROFILE_C1 = ("k_implicit_512px_20k_nodes.md",
              ["device_common.cuh", "iterate_common.cuh", "iterate_body.cuh", "iterate.cu",
               "mreg_internal.h"])
PROFILE_C2 = ("k_implicit_2048px_250k_nodes.md",
              ["device_common.cuh", "iterate_common.cuh", "iterate_body.cuh", "iterate.cu",
               "mreg_internal.h"])
PROFILE_ONE_PAIR = {1: PROFILE_C1, 2: PROFILE_C2}
PROFILE_OP = ("k_batch_apply_256_uneven_pairs.md", ["operator.cu", "mreg_internal.h"])
PROFILE_C3 = ("k_batch_256_uneven_pairs.md",
              ["device_common.cuh", "iterate_common.cuh", "iterate_body.cuh", "batch.cu",
               "setup_common.cuh", "mreg_internal.h"])


def profiled_traffic(profile, shape=None):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since the capture, the summary has no full-size
    capture, or (batched form) the launch's team shape is not the profiled one."""
    import hashlib
    import re
    name, sources = profile
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"source sha256 \([^)]*\): ([0-9a-f]+)", text)
    m_bytes = re.search(r"DRAM bytes per launch: (\d+)", text)
    if not (m_hash and m_bytes):
        return None
    if shape is not None:
        m_shape = re.search(r"team shape \(ctas,block,blocks_per_sm\): (\d+),(\d+),(\d+)", text)
        if not m_shape or tuple(int(x) for x in m_shape.groups()) != tuple(shape):
            return None
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1411_2141_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return int(m_bytes.group(1)) if h.hexdigest()[:len(m_hash.group(1))] == m_hash.group(1) else None


class L2Flush:
    """Evicts L2 (129 MB) between timed launches: writes a 256 MiB buffer,
    then reads another 256 MiB, so that the written lines are back in DRAM
    before the timed region starts and the timed kernel finds L2 holding
    only unrelated clean lines (a dirty L2 would make it pay for the
    flush's own write-backs)."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.r = torch.zeros(32 << 20, dtype=torch.int64, device=dev)
        self.out = torch.empty((), dtype=torch.int64, device=dev)

    def fill_(self, v):
        import torch
        self.w.fill_(v)
        torch.sum(self.r, dim=0, out=self.out)


def peak_hbm():
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        with open(pk_path) as fh:
            peaks = json.load(fh)
    return float(peaks.get("hbm_gbs", 6800.0)), ("measured" if "hbm_gbs" in peaks else "fallback")


# --------------------------------------------------------------- GPU side
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1411_2141_gb300 import mreg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    mreg.load()
    spec = inputs.config_spec(args.config)
    case = inputs.make_case(spec)
    n_iter = spec.n_iter
    stream = torch.cuda.current_stream()
    Re_d = torch.from_numpy(case.Re).to(dev)
    Te_d = torch.from_numpy(case.Te).to(dev)
    coeff = args.coeff
    reg = mreg.Registration(case.V, case.T, Re_d, Te_d, spec.alpha, spec.tau,
                            mode=args.mode, grad=args.grad, coeff=coeff, solver=args.solver,
                            neighbour_sync=args.neighbour_sync, stream=stream)
    msd_dev = torch.empty(1, dtype=torch.float64, device=dev)
    flush = L2Flush(dev)

    def one_registration(ev_iter=None):
        reg.reset(stream)
        if ev_iter is not None:
            ev_iter[0].record(stream)
        reg.step(n_iter, stream)
        if ev_iter is not None:
            ev_iter[1].record(stream)
        reg.warp(None, msd_dev, stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        one_registration()
    torch.cuda.synchronize()
    st = reg.stats(stream)
    cg_hist = reg.get_field(mreg.MREG_FIELD_PCG_ITERS)
    cg_mean = float(cg_hist.mean()) if args.mode != "S0" and len(cg_hist) else 0.0

    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    it_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                    # evict L2 between timed steps
        starts[k].record(stream)
        one_registration(it_ev[k])
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    iter_ms = [a.elapsed_time(b) for a, b in it_ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    msd = float(msd_dev.item())
    st = reg.stats(stream)
    u_gpu = reg.get_u(stream=stream)   # the last timed registration's result

    # end to end through the public API with host buffers (create from host
    # arrays, iterate, MSD and u back to the host, destroy)
    e2e = None
    if not args.no_e2e:
        Re_h = torch.from_numpy(case.Re).pin_memory().numpy()
        Te_h = torch.from_numpy(case.Te).pin_memory().numpy()
        e2e_steps = max(3, min(args.steps, 10))
        alloc = mreg.TorchAllocator()   # device memory from PyTorch's caching allocator

        def e2e_once():
            with mreg.Registration(case.V, case.T, Re_h, Te_h, spec.alpha, spec.tau,
                                   mode=args.mode, grad=args.grad, coeff=coeff, solver=args.solver,
                                   stream=stream, allocator=alloc) as r:
                r.step(n_iter, stream)
                m = r.msd(stream)
                u = r.get_u(stream=stream)
            return m, u
        e2e_once()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_once()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = case.Re.nbytes + case.Te.nbytes + case.V.nbytes + case.T.nbytes
        d2h = 8 + case.V.nbytes
        e2e = {"value": whole_job_rate(e2e_steps, world, e2e_s), "unit": "registrations/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": e2e_steps,
               "includes": "create from host arrays (device memory from PyTorch's caching "
                           "allocator), set-up, iterations, MSD and u back to the host, destroy"}

    if rank != 0:
        reg.close()
        return None
    value = whole_job_rate(args.steps, world, total_s)
    e = np.sort(np.concatenate([case.T[:, [0, 1]], case.T[:, [1, 2]], case.T[:, [2, 0]]]), axis=1)
    nnz = 2 * len(np.unique(e, axis=0))          # off-diagonal entries of the node graph
    per_iter = algorithmic_bytes_per_iteration(case.n_nodes, case.n_tris, nnz, args.mode, cg_mean,
                                               solver_of(args))
    it_ms = statistics.mean(iter_ms)
    achieved = per_iter * n_iter / (it_ms / 1e3) / 1e9
    peak, peak_src = peak_hbm()
    traffic = (profiled_traffic(PROFILE_ONE_PAIR[args.config])
               if args.config in PROFILE_ONE_PAIR
               and (args.mode, args.grad, args.coeff) == ("S1", "G0", "fp32") else None)
    line = {
        "metric": "registrations/s", "value": value, "unit": "registrations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, case),
        "node_iters_per_s": value * case.n_nodes * n_iter,
        "msd": msd, "cg_iters_mean": cg_mean,
        "iteration_kernel_ms": it_ms,
        "roofline": {"kernel": ("k_explicit" if args.mode == "S0" else "k_implicit")
                               + " (persistent: sample + force + update or solve, all iterations)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "peak_source": peak_src,
                     "basis": "algorithmic bytes per launch / launch time, against the HBM copy "
                              "peak; the working set is L2-resident at this size, so the kernel "
                              "is bound by latency (grid barriers, dependent L2 round trips), "
                              "not by DRAM",
                     "algorithmic_bytes_per_launch": per_iter * n_iter,
                     "traffic": traffic,
                     "dram_gbs": (traffic / (it_ms / 1e3) / 1e9 if traffic else None)},
        "clocks": clk,
        "gpu_launches": launches_per_registration(args, n_iter) * args.steps,
        "launch": {"grid": st["grid_blocks"], "block": st["block_size"]},
    }
    if e2e is not None:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        # one whole oracle registration of the same pair: the timed CPU
        # baseline, and the reference the timed GPU run is checked against
        t_reg, u_ref, msd_ref = oracle_registration(case, args.mode, args.grad)
        line["cpu_baseline"] = {
            "value": 1.0 / t_reg, "unit": "registrations/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"one whole registration (set-up, all {n_iter} iterations, MSD), "
                      f"numpy/scipy FP64, 1 thread"}
        line["parity"] = parity_against_oracle(u_gpu, msd, u_ref, msd_ref)
        line["parity"]["what"] = ("final node displacements and MSD of the last timed "
                                  "registration against the FP64 oracle's")
    reg.close()
    return line

# ---------------------------------------------------------- batched form
BATCH_LAUNCHES = 9   # prefilter rows + columns, Re at nodes, pixel fill + map,
                     # persistent iteration kernel, energy sums, warp, MSD sums
# kernels of one unrolled gradient: the forward persistent launch and its energy
# sums, the three warp-adjoint passes and their energy sum, the adjoint
# recursion (one cooperative launch)
ADJOINT_LAUNCHES = 7


def adjoint_launches(n_iter: int, every: int) -> int:
    """Kernels of one unrolled gradient with checkpoints every `every`
    iterations (0: every state kept): per segment a forward launch and its
    energy sums, and (when there are several segments) the recomputation
    with its energy sums and one adjoint launch; the warp adjoint's three
    passes and energy sum once."""
    segs = 1 if every <= 0 or every >= n_iter else -(-n_iter // every)
    return 4 + (2 * segs + segs if segs == 1 else 5 * segs)


def batch_workload_config(args, cases, shape=None):
    sides = [c.spec.side for c in cases]
    nodes = [c.n_nodes for c in cases]
    n_iter = cases[0].spec.n_iter
    cfg = {"workload": f"config3: batch of {len(cases)} pairs, sides {min(sides)}-{max(sides)} px "
                       f"(log-uniform), {min(nodes)}-{max(nodes)} nodes ({sum(nodes)} total), "
                       f"{n_iter} iterations each, {args.mode} {MODE_NAMES[args.mode]}"
                       f"{' (' + SOLVER_NAMES[solver_of(args)] + ')' if args.mode != 'S0' else ''}, "
                       f"{args.grad}",
           "pairs": len(cases), "pixels": int(sum(s * s for s in sides)), "nodes": int(sum(nodes)),
           "triangles": int(sum(c.n_tris for c in cases)), "iterations": n_iter,
           "mode": args.mode, "grad": args.grad, "coeff": args.coeff,
           "alpha": cases[0].spec.alpha, "tau": cases[0].spec.tau,
           "l2": "flushed between timed steps (256 MiB write, then 256 MiB read); the packed batch (~1.3 GB) exceeds L2",
           "parallelism": f"replicas x{args.gpus} (the whole batch per GPU per step)"}
    if args.gpus > 1:
        cfg["parallelism"] = (f"the batch split over {args.gpus} GPUs by greedy LPT on "
                              f"node-iterations + pixels; this config describes rank 0's share")
    if shape is not None:
        cfg["team"] = {"ctas": shape[0], "block": shape[1], "blocks_per_sm": shape[2],
                       "teams": shape[3]}
    return cfg


def batch_cases(n_pairs: int = 0):
    return inputs.make_cases(inputs.batched_specs(3, n_pairs or None))


def oracle_batch_time(cases, mode: str, grad: str, n_sample_pairs: int = 4):
    """The FP64 oracle on the batched workload: whole registrations (all
    iterations) of n_sample_pairs pairs spread over the size range.  Returns
    the seconds they took, the seconds the whole batch would take at the same
    rate per node, and the pairs picked."""
    order = np.argsort([c.n_nodes for c in cases])
    pick = [int(order[round(k * (len(order) - 1) / max(1, n_sample_pairs - 1))])
            for k in range(n_sample_pairs)]
    t_pick = sum(oracle_registration(cases[k], mode, grad)[0] for k in pick)
    scale = sum(c.n_nodes for c in cases) / sum(cases[k].n_nodes for k in pick)
    return t_pick, t_pick * scale, pick


def run_ours_batch_single(args, rank, world, local_rank, cases=None):
    """The batched workload through the one-pair engine: every pair has its
    own handle (created before timing); a step registers all pairs one after
    another (reset + iterations + warp/MSD each), as the plain FP32 form
    would."""
    import torch
    from paper_1411_2141_gb300 import mreg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    mreg.load()
    cases = cases or batch_cases(args.pairs)
    n_iter = cases[0].spec.n_iter
    stream = torch.cuda.current_stream()
    regs = [mreg.Registration(c.V, c.T, torch.from_numpy(c.Re).to(dev),
                              torch.from_numpy(c.Te).to(dev), c.spec.alpha, c.spec.tau,
                              mode=args.mode, grad=args.grad, coeff=args.coeff, solver=args.solver,
                              stream=stream) for c in cases]
    msd_dev = torch.empty(len(cases), dtype=torch.float64, device=dev)
    flush = L2Flush(dev)

    side = [torch.cuda.Stream(device=dev) for _ in range(max(1, args.streams))]

    def one_step():
        for s in side:
            s.wait_stream(stream)
        for k, r in enumerate(regs):
            sk = side[k % len(side)]
            r.reset(sk)
            r.step(n_iter, sk)
            r.warp(None, msd_dev[k:k + 1], sk)
        for s in side:
            stream.wait_stream(s)
    for _ in range(args.warmup):
        flush.fill_(1)
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        one_step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_s = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3, world, dev)
    if rank != 0:
        for r in regs:
            r.close()
        return None
    value = whole_job_rate(args.steps * len(cases), world, total_s)
    cfg = batch_workload_config(args, cases)
    cfg["engine"] = ("one-pair grid engine, pairs in sequence (the plain FP32 form)"
                     if len(side) == 1 else
                     f"one-pair grid engine (the plain FP32 form), pairs spread over {len(side)} "
                     f"CUDA streams")
    line = {
        "metric": "registrations/s", "value": value, "unit": "registrations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "node_iters_per_s": value / len(cases) * sum(c.n_nodes for c in cases) * n_iter,
        "msd_mean": float(msd_dev.double().mean().item()), "clocks": clk,
        "gpu_launches": sum(launches_per_registration(args, n_iter) for _ in cases) * args.steps,
    }
    for r in regs:
        r.close()
    return line


def operator_bytes(n_v: int, nnz: int, mode: str) -> float:
    """Compulsory bytes of y = A x for one mesh: the column indices (and for
    S2 the stored off-diagonal values and diagonal), x read once and y
    written once (both float2).  The row structure is not counted: the
    batched product's sliced layout reads one 16-byte record per 32 rows
    (0.5 B per row) and no row pointers; its padding entries are overhead."""
    vals = (4 * nnz + 4 * n_v) if mode == "S2" else 0
    return 4 * nnz + vals + 8 * n_v + 8 * n_v


def measure_operator(b, cases, nnz, mode, dev, stream, flush, launches: int = 20) -> dict:
    """The batched operator y = A x (every pair's system matrix, one launch)
    timed with CUDA events on the launching stream, L2 flushed before each
    launch, against the HBM roofline."""
    import torch
    n = sum(c.n_nodes for c in cases)
    g = torch.Generator(device=dev).manual_seed(11)
    x = torch.randn((n, 2), dtype=torch.float32, device=dev, generator=g)
    y = torch.empty_like(x)
    for _ in range(3):
        b.apply_operator(x, y, stream)
    evs = []
    for k in range(launches):
        flush.fill_(k & 0xFF)
        a_ev = torch.cuda.Event(enable_timing=True)
        e_ev = torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        b.apply_operator(x, y, stream)
        e_ev.record(stream)
        evs.append((a_ev, e_ev))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(e) for a, e in evs)
    nbytes = sum(operator_bytes(c.n_nodes, z, mode) for c, z in zip(cases, nnz))
    peak, peak_src = peak_hbm()
    achieved = nbytes / (ms / 1e3) / 1e9
    return {"kernel": "k_batch_apply (y = A x with every pair's system matrix, one launch)",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "algorithmic_bytes_per_launch": nbytes, "launch_ms": ms, "launches": launches,
            "l2": "flushed before every launch (256 MiB write, then 256 MiB read)",
            "traffic": profiled_traffic(PROFILE_OP) if mode == "S1" and len(cases) == 256 else None}


def run_ours_batch(args, rank, world, local_rank, cases=None):
    import torch
    from paper_1411_2141_gb300 import mreg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    mreg.load()
    cases = cases or batch_cases(args.pairs)
    n_total = len(cases)
    split = world > 1
    if split:   # pairs are independent: each rank registers its LPT share of the batch
        cases = [cases[k] for k in lpt_partition([pair_cost(c) for c in cases], world)[rank]]
    n_iter = cases[0].spec.n_iter
    stream = torch.cuda.current_stream()
    coeff = args.coeff
    pairs = [(c.V, c.T, c.Re, c.Te) for c in cases]
    b = mreg.Batch(pairs, cases[0].spec.alpha, cases[0].spec.tau, mode=args.mode, grad=args.grad,
                   coeff=coeff, solver=args.solver, stream=stream)
    if args.team:
        vals = [int(x) for x in args.team.split(",")]
        ctas, block, per_sm = (vals + [1])[:3]
        b.close()
        b = mreg.Batch(pairs, cases[0].spec.alpha, cases[0].spec.tau, mode=args.mode,
                       grad=args.grad, coeff=coeff, team_ctas=ctas, block_size=block,
                       team_blocks_per_sm=per_sm, grid_blocks=args.teams, solver=args.solver,
                       stream=stream)
        tune_s, tune_ms = 0.0, {}
    else:
        t0 = time.perf_counter()
        (ctas, block, per_sm), tune_ms = b.tune(n_iter, stream)
        tune_s = time.perf_counter() - t0
    shape = b.shape()
    flush = L2Flush(dev)
    for _ in range(args.warmup):
        flush.fill_(1)
        b.run(n_iter, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iter_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        b.run(n_iter, stream)
        ends[k].record(stream)
        iter_ms.append(b.iterate_ms())   # waits for this step's kernel only
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    msd = b.msd(stream)
    cg = []
    nnz_total, per_iter_total, nnzs = 0, 0.0, []
    for k, c in enumerate(cases):
        its = b.get_field(k, mreg.MREG_FIELD_PCG_ITERS)
        cgm = float(its.mean()) if args.mode != "S0" and len(its) else 0.0
        cg.append(cgm)
        e = np.sort(np.concatenate([c.T[:, [0, 1]], c.T[:, [1, 2]], c.T[:, [2, 0]]]), axis=1)
        nnz = 2 * len(np.unique(e, axis=0))
        nnz_total += nnz
        nnzs.append(nnz)
        per_iter_total += algorithmic_bytes_per_iteration(c.n_nodes, c.n_tris, nnz, args.mode, cgm,
                                                          solver_of(args))

    op = (measure_operator(b, cases, nnzs, args.mode, dev, stream, flush)
          if getattr(args, "operator", False) and args.mode != "S0" else None)
    e2e = None
    if not args.no_e2e:
        pinned = [(c.V, c.T, torch.from_numpy(c.Re).pin_memory().numpy(),
                   torch.from_numpy(c.Te).pin_memory().numpy()) for c in cases]
        e2e_steps = max(2, min(args.steps, 3))
        alloc = mreg.TorchAllocator()   # device memory from PyTorch's caching allocator

        def e2e_once():
            with mreg.Batch(pinned, cases[0].spec.alpha, cases[0].spec.tau, mode=args.mode,
                            grad=args.grad, coeff=coeff, team_ctas=ctas, block_size=block,
                            team_blocks_per_sm=per_sm, solver=args.solver, stream=stream,
                            allocator=alloc) as bb:
                bb.run(n_iter, stream)
                m = bb.msd(stream)
                us = [bb.get_u(k, stream) for k in range(len(cases))]
            return m, us
        e2e_once()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_once()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = sum(c.Re.nbytes + c.Te.nbytes + c.V.nbytes + c.T.nbytes for c in cases)
        d2h = 8 * len(cases) + sum(c.V.nbytes for c in cases)
        e2e = {"value": (e2e_steps * n_total / e2e_s if split
                         else whole_job_rate(e2e_steps * len(cases), world, e2e_s)),
               "unit": "registrations/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
               "note": "each step creates the batch from pinned host arrays (host topology "
                       "build of every mesh included; device memory from PyTorch's caching "
                       "allocator), runs it, reads MSD and u, destroys it"}
    if rank != 0:
        b.close()
        return None
    # split: the ranks registered the n_total pairs together (strong scaling)
    value = (args.steps * n_total / total_s if split
             else whole_job_rate(args.steps * len(cases), world, total_s))
    it_ms = statistics.mean(iter_ms)
    achieved = per_iter_total * n_iter / (it_ms / 1e3) / 1e9
    peak, peak_src = peak_hbm()
    before = np.array([np.mean((c.Re.astype(np.float64) - c.Te) ** 2) for c in cases])
    line = {
        "metric": "registrations/s", "value": value, "unit": "registrations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": batch_workload_config(args, cases, shape),
        "node_iters_per_s": value / len(cases) * sum(c.n_nodes for c in cases) * n_iter,
        "msd_mean": float(msd.mean()), "msd_ratio_mean": float((msd / before).mean()),
        "cg_iters_mean": float(np.mean(cg)),
        "iteration_kernel_ms": it_ms,
        "autotune": ({"seconds": tune_s, "chosen": [ctas, block, per_sm],
                      "ms": {f"{c}x{k}/{m}": v for (c, k, m), v in tune_ms.items()}}
                     if tune_ms else {"fixed": [ctas, block, per_sm]}),
        "roofline": {"kernel": "k_batch (persistent: every pair's sample + force + solve loop)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": per_iter_total * n_iter,
                     "traffic": (profiled_traffic(PROFILE_C3, (ctas, block, per_sm))
                                 if not args.pairs and (args.mode, args.grad, args.coeff)
                                 == ("S1", "G0", "fp32") else None)},
        "clocks": clk,
        "gpu_launches": BATCH_LAUNCHES * args.steps,
    }
    if op is not None:
        line["operator_roofline"] = op
    if e2e is not None:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        _, t_all, pick = oracle_batch_time(cases, args.mode, args.grad)
        line["cpu_baseline"] = {
            "value": len(cases) / t_all, "unit": "registrations/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"whole registrations ({n_iter} iterations) of {len(pick)} of the "
                      f"{len(cases)} pairs spread over the size range, the rate per node "
                      f"applied to the whole batch; numpy/scipy FP64, 1 thread"}
    b.close()
    return line

# ------------------------------------------------- differentiation form
def adjoint_cases(n_pairs: int = 0):
    return inputs.make_cases(inputs.batched_specs(4, n_pairs or None))


def _smooth_u0(c):
    x = c.V[:, 0].astype(np.float64)
    y = c.V[:, 1].astype(np.float64)
    s = c.spec.side
    return np.stack([np.sin(2 * np.pi * x / s), np.cos(2 * np.pi * y / s)], axis=1).astype(np.float32)


def run_ours_adjoint(args, rank, world, local_rank):
    """One step = the gradient of the warp energy after a 20-iteration
    unrolled registration (explicit form, spline gradient) with respect to
    the starting displacement, for each of the 64 pairs: 20 forward
    iterations with every state kept, the warp energy and its adjoint, and
    20 adjoint steps."""
    import torch
    from paper_1411_2141_gb300 import mreg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    mreg.load()
    cases = adjoint_cases(args.pairs)
    K = cases[0].spec.n_iter
    stream = torch.cuda.current_stream()
    regs = [mreg.Registration(c.V, c.T, torch.from_numpy(c.Re).to(dev), torch.from_numpy(c.Te).to(dev),
                              c.spec.alpha, c.spec.tau, mode="S0", grad="G1", stream=stream)
            for c in cases]
    u0 = [torch.from_numpy(_smooth_u0(c)).to(dev) for c in cases]
    E = torch.empty(len(cases), dtype=torch.float64, device=dev)
    g = [torch.empty_like(u) for u in u0]
    flush = L2Flush(dev)

    # Each pair's launches fill only a fraction of the GPU (a 5k-node pair's
    # grid is ~20 blocks), so the pairs are spread over several streams and
    # run concurrently; every handle owns its buffers, so the results do not
    # depend on the stream count.
    side = [torch.cuda.Stream(device=dev) for _ in range(max(1, args.streams))]

    def one_step():
        for s in side:
            s.wait_stream(stream)
        for k, r in enumerate(regs):
            r.unroll_grad(u0[k], K, E[k:k + 1], g[k], side[k % len(side)],
                          checkpoint_every=args.checkpoint)
        for s in side:
            stream.wait_stream(s)
    for _ in range(args.warmup):
        flush.fill_(1)
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        one_step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_s = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3, world, dev)

    # the dominant kernel: the forward iteration kernel (K explicit iterations
    # of one pair, the launch the gradient's forward run makes), timed per pair
    # with CUDA events on the launching stream, after the timed region
    fw_ms = []
    for k, r in enumerate(regs):
        a_ev = torch.cuda.Event(enable_timing=True)
        b_ev = torch.cuda.Event(enable_timing=True)
        flush.fill_(k & 0xFF)
        a_ev.record(stream)
        r.step(K, stream)
        b_ev.record(stream)
        fw_ms.append((a_ev, b_ev))
    torch.cuda.synchronize()
    fw_ms = [a_ev.elapsed_time(b_ev) for a_ev, b_ev in fw_ms]

    # end to end through the public API: every step copies each pair's u0 from
    # pinned host memory, runs its unrolled gradient and reads the gradient and
    # the energy back into pinned host memory
    e2e = None
    if not args.no_e2e:
        u0_h = [torch.from_numpy(_smooth_u0(c)).pin_memory() for c in cases]
        g_h = [torch.empty(u.shape, dtype=u.dtype).pin_memory() for u in u0_h]
        E_h = torch.empty(len(cases), dtype=torch.float64).pin_memory()
        u0_d = [torch.empty(u.shape, dtype=u.dtype, device=dev) for u in u0_h]
        e2e_steps = max(2, min(args.steps, 5))

        def e2e_once():
            for s in side:
                s.wait_stream(stream)
            for k, r in enumerate(regs):
                sk = side[k % len(side)]
                with torch.cuda.stream(sk):
                    u0_d[k].copy_(u0_h[k], non_blocking=True)
                    r.unroll_grad(u0_d[k], K, E[k:k + 1], g[k], sk, checkpoint_every=args.checkpoint)
                    g_h[k].copy_(g[k], non_blocking=True)
            for s in side:
                stream.wait_stream(s)
            E_h.copy_(E, non_blocking=True)
            torch.cuda.synchronize()
        e2e_once()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_once()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = sum(u.numel() * u.element_size() for u in u0_h)
        e2e = {"value": whole_job_rate(e2e_steps * len(cases), world, e2e_s), "unit": "gradients/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d + 8 * len(cases)),
               "steps": e2e_steps}
    if rank != 0:
        for r in regs:
            r.close()
        return None
    value = whole_job_rate(args.steps * len(cases), world, total_s)
    fw_bytes = []
    for c in cases:
        e = np.sort(np.concatenate([c.T[:, [0, 1]], c.T[:, [1, 2]], c.T[:, [2, 0]]]), axis=1)
        nnz = 2 * len(np.unique(e, axis=0))
        fw_bytes.append(algorithmic_bytes_per_iteration(c.n_nodes, c.n_tris, nnz, "S0", 0.0) * K)
    peak, peak_src = peak_hbm()
    achieved = statistics.mean(fw_bytes) / (statistics.mean(fw_ms) / 1e3) / 1e9
    line = {
        "metric": "unrolled gradients/s", "value": value, "unit": "gradients/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"config4: {len(cases)} pairs of 256x256, {cases[0].n_nodes}-node "
                               f"meshes, gradient of the warp energy through {K} explicit "
                               f"iterations (spline gradient) with respect to u0"
                               + (f", states checkpointed every {args.checkpoint} iterations "
                                  f"(segments recomputed in the backward pass)"
                                  if 0 < args.checkpoint < K else ", every state kept"),
                   "checkpoint_every": args.checkpoint,
                   "pairs": len(cases), "iterations": K, "streams": len(side),
                   "l2": "flushed between timed steps (256 MiB write, then 256 MiB read)",
                   "parallelism": f"replicas x{args.gpus}"},
        "energy_mean": float(E.mean().item()),
        "roofline": {"kernel": "k_explicit (the forward run: K explicit iterations of one pair, "
                               "one persistent launch; timed per pair after the timed region)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": statistics.mean(fw_bytes),
                     "launch_ms": statistics.mean(fw_ms), "traffic": None},
        "clocks": clk,
        "gpu_launches": len(cases) * adjoint_launches(K, args.checkpoint) * args.steps,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        from oracle import adjoint, register
        c = cases[0]
        t0 = time.perf_counter()
        pb = register.Problem(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, "S0", "G1")
        adjoint.unrolled_grad(pb, _smooth_u0(c).astype(np.float64), K)
        t1 = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / t1, "unit": "gradients/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "one pair: set-up, 20 forward iterations and the adjoint "
                                          "recursion, numpy/scipy FP64, 1 thread"}
    for r in regs:
        r.close()
    return line



FORM_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "iteration_kernel_ms",
             "cg_iters_mean", "msd_mean", "clocks", "gpu_launches")


def _form_summary(line: dict, what: str) -> dict:
    out = {"what": what}
    out.update({k: line[k] for k in FORM_KEYS if k in line})
    if "roofline" in line:
        out["roofline"] = {k: line["roofline"][k] for k in ("kernel", "achieved", "frac", "peak")}
    if "team" in line.get("config", {}):
        out["team"] = line["config"]["team"]
    if "operator_roofline" in line:
        out["operator_roofline"] = line["operator_roofline"]
    return out


def run_forms(args, rank, world, local_rank) -> dict | None:
    """Short runs (3 warm-up and 3 timed steps each, L2 flushed between
    steps) of the other forms, reported beside the one-pair line."""
    import copy
    sub = copy.copy(args)
    sub.steps, sub.warmup, sub.no_cpu_baseline, sub.no_e2e, sub.pairs = 3, 3, True, True, 0
    sub.mode, sub.grad, sub.coeff, sub.team, sub.teams = "S1", "G0", "fp32", None, 0
    cases = batch_cases()
    forms = {}
    sub.config = 3
    sub.operator = True
    line = run_ours_batch(sub, rank, world, local_rank, cases)
    sub.operator = False
    if line is not None:
        forms["batched_fp32"] = _form_summary(
            line, "config 3: 256 uneven pairs, 100 iterations each, batched engine (one CUDA-graph "
                  "launch, autotuned team shape), FP32")
        sub.team = ",".join(str(x) for x in line["autotune"]["chosen"])
    for storage in ("bf16", "fp16"):
        sub.coeff = storage
        line = run_ours_batch(sub, rank, world, local_rank, cases)
        if line is not None:
            forms[f"batched_{storage}"] = _form_summary(
                line, f"the same batch with {storage.upper()}-stored Te coefficients (the precision "
                      f"form), the team shape the FP32 run's autotuner chose")
    sub.coeff, sub.team = "fp32", None
    line = run_ours_batch_single(sub, rank, world, local_rank, cases)
    if line is not None:
        forms["plain_fp32_streams"] = _form_summary(
            line, f"the same 256 pairs through one-pair handles (the plain FP32 form), pairs "
                  f"spread over {sub.streams} CUDA streams")
    del cases
    sub.config = 4
    for every in (0, 5):
        sub.checkpoint = every
        line = run_ours_adjoint(sub, rank, world, local_rank)
        if line is not None:
            key = "differentiation" if every == 0 else "differentiation_checkpointed"
            forms[key] = _form_summary(
                line, "config 4: gradient of the warp energy through 20 unrolled explicit "
                      f"iterations, 64 pairs of 256x256, {sub.streams} CUDA streams"
                      + (f", states checkpointed every {every} iterations" if every else ""))
    return forms if rank == 0 else None


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.config == 4:
            line = run_ours_adjoint(args, rank, world, local_rank)
        elif args.config == 3 and args.single:
            line = run_ours_batch_single(args, rank, world, local_rank)
        elif args.config == 3:
            line = run_ours_batch(args, rank, world, local_rank)
        else:
            line = run_ours(args, rank, world, local_rank)
            if args.config == 1 and not args.no_forms:
                forms = run_forms(args, rank, world, local_rank)
                if line is not None:
                    line["forms"] = forms
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
