"""Throughput of the mesh-registration hot path on GB300.

One step = one whole registration of one 512x512 image pair with a ~20k-node
mesh: B-spline prefilter of both images, node samples of Re, pixel ->
triangle map, 200 iterations (sampling, Eq. 9-10 force, semi-implicit
umbrella solve by Jacobi-PCG), dense warp and MSD, all on the device.
Metric: registrations/s (and node-iterations/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--mode S1] [--config 1]

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sample of each registration, extrapolated to the full iteration
count).  Under torchrun (N > 1) every rank registers its own pairs on its
own GPU (independent replicas, weak scaling); rank 0 prints one JSON line.
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

MODE_NAMES = {"S0": "explicit Eq.5+Eq.14", "S1": "umbrella-implicit solve (Jacobi-PCG)",
              "S2": "P1-FEM-implicit solve (Jacobi-PCG)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=1)
    p.add_argument("--mode", default="S1", choices=["S0", "S1", "S2"])
    p.add_argument("--grad", default="G0", choices=["G0", "G1"])
    p.add_argument("--coeff", default="fp32", choices=["fp32", "bf16"],
                   help="storage of Te's spline coefficients (bf16: the precision form)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------- bytes model
def algorithmic_bytes_per_iteration(n_v: int, n_t: int, nnz: int, mode: str, cg_its: float) -> float:
    """Compulsory bytes of one iteration of the iteration kernel (each array
    read or written once; gathers of neighbours counted once per node)."""
    sample = n_v * (8 + 8 + 4 + 4)                          # V, u, Re(V) in; f out
    force = 4 * (n_v + 1) + 4 * 3 * n_t + 12 * n_t + 8 * n_v  # inc CSR, triangles, F out
    if mode == "S0":
        update = 4 * (n_v + 1) + 4 * nnz + 8 * n_v + 8 * n_v + 8 * n_v  # graph, u0 out/in, u out
        return sample + force + update
    graph = 4 * (n_v + 1) + 4 * nnz
    vals = (8 * nnz + 8 * n_v) if mode == "S2" else 0
    init = graph + vals + 8 * n_v + 16 * n_v + 8 * n_v + 8 * n_v + 4 * n_v   # u, b, r, z out, dinv
    cg1 = graph + vals / 2 + 8 * n_v * 3 + 16 * n_v + 8 * n_v * 3           # z, p, x, b in; p', q, rt out
    cg2 = 8 * n_v * 4 + 4 * n_v + 8 * n_v * 3                                # p, q, x, r in; x, r, z out
    return sample + force + init + cg_its * (cg1 + cg2)


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
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
def oracle_registration_time(case, mode: str, grad: str, sample_iters: int = 20):
    """Seconds of one registration by the FP64 oracle: set-up, a bounded run
    of sample_iters iterations extrapolated to the full count, and the MSD."""
    from oracle import register
    t0 = time.perf_counter()
    pb = register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau, mode, grad)
    t1 = time.perf_counter()
    u, _ = pb.run(sample_iters)
    t2 = time.perf_counter()
    pb.msd(u)
    t3 = time.perf_counter()
    n = case.spec.n_iter
    return (t1 - t0) + (t2 - t1) * n / sample_iters + (t3 - t2), sample_iters


def run_reference(args, rank, world):
    if rank != 0:
        return
    spec = inputs.config_spec(args.config)
    case = inputs.make_case(spec)
    for _ in range(args.warmup):
        oracle_registration_time(case, args.mode, args.grad, sample_iters=2)
    times = []
    for _ in range(args.steps):
        t, sample_iters = oracle_registration_time(case, args.mode, args.grad)
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
                         "sample": f"per step: full set-up + {sample_iters} of {spec.n_iter} "
                                   f"iterations (time scaled x{spec.n_iter / sample_iters:g}) + MSD"},
        "e2e": {"value": value, "unit": "registrations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def launches_per_registration(args, n_iter: int) -> int:
    """Our kernels in one timed step: prefilter (row and column pass) of Re
    and Te, [BF16 copy], Re at the nodes, [Re at edge midpoints], pixel map
    (fill + scan), the persistent iteration kernel and its energy pass per
    1024-iteration chunk, warp + MSD and the final MSD sum."""
    chunks = (n_iter + 1023) // 1024
    return (4 + (args.coeff == "bf16") + 1 + 2 + 2 * chunks + 2)


def workload_config(args, case):
    s = case.spec
    return {"workload": f"config{args.config}: {s.side}x{s.side} pair, {case.n_nodes}-node mesh, "
                        f"{s.n_iter} iterations, {args.mode} {MODE_NAMES[args.mode]}, "
                        f"{args.grad} {'mesh gradient Eq.9-10' if args.grad == 'G0' else 'spline gradient'}"
                        + (", BF16-stored Te coefficients" if args.coeff == "bf16" else ""),
            "image": [s.side, s.side], "nodes": case.n_nodes, "triangles": case.n_tris,
            "iterations": s.n_iter, "mode": args.mode, "grad": args.grad, "coeff": args.coeff,
            "alpha": s.alpha, "tau": s.tau,
            "l2": "flushed between timed steps (256 MiB write); the step's own working set is L2-resident",
            "parallelism": f"replicas x{args.gpus} (one pair per GPU per step)"}


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
    bf16 = args.coeff == "bf16"
    reg = mreg.Registration(case.V, case.T, Re_d, Te_d, spec.alpha, spec.tau,
                            mode=args.mode, grad=args.grad, coeff_bf16=bf16, stream=stream)
    msd_dev = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

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
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    msd = float(msd_dev.item())
    st = reg.stats(stream)

    # end to end through the public API with host buffers (create from host
    # arrays, iterate, MSD and u back to the host, destroy)
    e2e = None
    if not args.no_e2e:
        Re_h = torch.from_numpy(case.Re).pin_memory().numpy()
        Te_h = torch.from_numpy(case.Te).pin_memory().numpy()
        e2e_steps = max(3, min(args.steps, 10))

        def e2e_once():
            with mreg.Registration(case.V, case.T, Re_h, Te_h, spec.alpha, spec.tau,
                                   mode=args.mode, grad=args.grad, coeff_bf16=bf16,
                                   stream=stream) as r:
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
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = case.Re.nbytes + case.Te.nbytes + case.V.nbytes + case.T.nbytes
        d2h = 8 + case.V.nbytes
        e2e = {"value": e2e_steps * world / e2e_s, "unit": "registrations/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": e2e_steps}

    if rank != 0:
        return
    value = args.steps * world / total_s
    e = np.sort(np.concatenate([case.T[:, [0, 1]], case.T[:, [1, 2]], case.T[:, [2, 0]]]), axis=1)
    nnz = 2 * len(np.unique(e, axis=0))          # off-diagonal entries of the node graph
    per_iter = algorithmic_bytes_per_iteration(case.n_nodes, case.n_tris, nnz, args.mode, cg_mean)
    it_ms = statistics.mean(iter_ms)
    achieved = per_iter * n_iter / (it_ms / 1e3) / 1e9
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        with open(pk_path) as fh:
            peaks = json.load(fh)
    peak = float(peaks.get("hbm_gbs", 6800.0))
    line = {
        "metric": "registrations/s", "value": value, "unit": "registrations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, case),
        "node_iters_per_s": value * case.n_nodes * n_iter,
        "msd": msd, "cg_iters_mean": cg_mean,
        "iteration_kernel_ms": it_ms,
        "roofline": {"kernel": "k_iterate (persistent: sample + force + solve, all iterations)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                     "algorithmic_bytes_per_launch": per_iter * n_iter,
                     "traffic": None},
        "clocks": clk,
        "gpu_launches": launches_per_registration(args, n_iter) * args.steps,
        "launch": {"grid": st["grid_blocks"], "block": st["block_size"]},
    }
    if e2e is not None:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        t_reg, sample_iters = oracle_registration_time(case, args.mode, args.grad)
        line["cpu_baseline"] = {
            "value": 1.0 / t_reg, "unit": "registrations/s", "cores": 1, "kind": "oracle",
            "sample": f"one registration: full set-up + {sample_iters} of {n_iter} iterations "
                      f"(time scaled x{n_iter / sample_iters:g}) + MSD, numpy/scipy FP64, 1 thread"}
    print(json.dumps(line), flush=True)
    reg.close()


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
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
