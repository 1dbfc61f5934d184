"""Oracle runs for the GPU tests, in worker processes.

The functions here take a case's seeded spec (not its arrays), rebuild the
case in the worker and run the FP64 oracle on it, so that many pairs can be
checked in parallel on the host cores while the GPU test runs.  They import
neither torch nor the CUDA library; start their pool with the "spawn"
method.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

from oracle import register
from paper_1411_2141_gb300 import inputs


def registration(job):
    """(spec, mode, grad, quad, n_iter) -> (u, per-iteration data energy, MSD)
    of the oracle's registration of the case the spec describes."""
    spec, mode, grad, quad, n = job
    c = inputs.make_case(spec)
    pb = register.Problem(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, mode, grad, quad)
    u, e = pb.run(n)
    return u, e, pb.msd(u)


def pool(processes: int | None = None) -> cf.ProcessPoolExecutor:
    n = processes or max(1, min(16, os.cpu_count() or 1))
    return cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn"))
