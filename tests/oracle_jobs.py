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

import numpy as np

from oracle import bspline, register
from paper_1411_2141_gb300 import inputs


def round_coefficients(c: np.ndarray, storage: str, flip_ties: bool = False) -> np.ndarray:
    """The values a 16-bit copy of FP32 coefficients holds, as FP64: FP32
    rounding of c, then round to nearest even to BF16 (the top 16 bits of the
    FP32 pattern) or to IEEE FP16.

    flip_ties: where the FP32 value lies within 4 FP32 ulps of the midpoint
    between two 16-bit values, take the other one.  Two FP32 computations of
    the same coefficients (the library's prefilter and the oracle's, rounded)
    differ by a few ulps, so they can round to different 16-bit neighbours
    exactly there; running the method on both roundings bounds what that
    ambiguity can change."""
    f = np.ascontiguousarray(c, dtype=np.float32)
    if storage == "fp16":
        q = f.astype(np.float16)
        qa = np.abs(q)
        up = np.nextafter(qa, np.float16(np.inf))
        dn = np.nextafter(qa, np.float16(0.0))
        qa, up, dn = (x.astype(np.float64) for x in (qa, up, dn))
    else:
        b = f.view(np.uint32).astype(np.uint64)
        qb = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
        q = qb.view(np.float32)
        mag = qb & np.uint32(0x7FFFFFFF)
        up = (mag + np.uint32(0x10000)).view(np.float32).astype(np.float64)
        dn = np.where(mag >= 0x10000, mag - np.uint32(0x10000), 0).astype(np.uint32) \
            .view(np.float32).astype(np.float64)
        qa = np.abs(q).astype(np.float64)
    q = q.astype(np.float64)
    if not flip_ties:
        return q
    fa = np.abs(f).astype(np.float64)
    other = np.where(fa > qa, up, dn)
    ulp = np.spacing(np.abs(f)).astype(np.float64)
    near = np.abs(fa - 0.5 * (qa + other)) <= 4.0 * ulp
    return np.where(near, np.sign(f) * other, q)


def registration(job):
    """(spec, mode, grad, quad, n_iter) -> (u, per-iteration data energy, MSD)
    of the oracle's registration of the case the spec describes."""
    spec, mode, grad, quad, n = job
    c = inputs.make_case(spec)
    pb = register.Problem(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, mode, grad, quad)
    u, e = pb.run(n)
    return u, e, pb.msd(u)


def registration_rounded_coefficients(job):
    """(spec, mode, grad, quad, n_iter, storage[, flip_ties]) -> as
    registration(), with Te's spline coefficients rounded as a 16-bit copy
    stores them (see round_coefficients) and everything else in FP64: the
    method as the precision form defines it, the reference for that form's
    parity."""
    spec, mode, grad, quad, n, storage = job[:6]
    flip = bool(job[6]) if len(job) > 6 else False
    c = inputs.make_case(spec)
    pb = register.Problem(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, mode, grad, quad)
    q = round_coefficients(pb.cTe, storage, flip)
    pb.cTe = q
    pb.te_sampler = lambda x, y: bspline.evaluate(q, x, y, grad=True)
    u, e = pb.run(n)
    return u, e, pb.msd(u)


def registration_and_sensitivity(job):
    """As registration(), plus the trajectory's sensitivity to rounding at
    FP32 level: the largest node difference between the FP64 run and a second
    oracle run whose iterate is rounded to FP32 after every iteration.  Where
    the deformed mesh folds, Eq. 9's triangle gradient changes sign with the
    deformed area, the force is discontinuous in u, and rounding differences
    can grow to a visible fraction of a pixel; the sensitivity measures that
    from the oracle alone."""
    spec, mode, grad, quad, n = job
    c = inputs.make_case(spec)
    pb = register.Problem(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, mode, grad, quad)
    u, e = pb.run(n)
    v = np.zeros_like(u)
    for _ in range(n):
        v, _ = pb.step(v)
        v = v.astype(np.float32).astype(np.float64)
    return u, e, pb.msd(u), float(np.abs(u - v).max())


def pool(processes: int | None = None) -> cf.ProcessPoolExecutor:
    n = processes or max(1, min(16, os.cpu_count() or 1))
    return cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn"))
