"""Autotuner for the launch shapes of an MDSystem.

The paper found thread-block size to matter little on its GPU and warned that this need not hold
elsewhere (Sec. 4.1 item 2).  On GB300 the residency of the fused step kernel and the number of
neighbour-matrix loads each thread keeps in flight decide its speed, so they are measured on the
system itself: every candidate advances the live system by a number of steps timed with CUDA
events on the library's stream.  Step kernels 1-3 and builds 2, 4 and 32 perform the same
arithmetic in the same order; the list-free step kernel (4) and the sub-cell build (1) sum each
force in another order, and the half-list kernel (5) adds through atomics in no fixed order, so
choosing them changes the trajectory at the rounding level only.

Search: coordinate descent over (step kernel, ctas_per_sm, nbr_batch, atom_threads) for the step
-- the per-thread kernel at register-bound residencies with 1, 2 or 4 lanes per atom, the list-free
and half-list kernels, and on request the shared-memory ring and the staged-neighbour kernel (2
and 3, slower on every measured workload) at the residencies their shared memory allows -- then
build_batch and build_stage for the neighbour build (timed over steps that include rebuilds).
Results are cached per GPU and workload signature in a JSON file.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import binding as B

CTAS = (4, 8, 12, 16)          # per-thread step kernel (register-bound residency)
CTAS_RING = (2, 3, 4, 6)       # shared-memory ring step kernel (shared-memory-bound residency)
CTAS_STAGED = (4, 6, 8)        # staged-neighbour step kernel (register- and shared-memory-bound)
CTAS_CELLS = (4, 8, 12)        # list-free and half-list step kernels (register-bound residency)
NBR_BATCH = (2, 4, 8)
NBR_BATCH_TPA = (2, 4)         # with 2 or 4 lanes per atom
ATOM_THREADS = (2, 4)
BUILD_BATCH = (1, 2, 4, 32)
BUILD_STAGE = (2, 1)           # the build writes W entry by entry, or rows from shared memory


def signature(system) -> str:
    p = system.params
    dev = torch.cuda.get_device_name(system.device)
    return (f"{dev}|prec{p.precision}|n{system.n}|rep{system.nrep}|rc{p.rc:.4f}|skin{p.skin:.3f}|"
            f"rho{system.n / float((system.boxes.prod(axis=1)).sum()):.3f}")


def _time_steps(system, steps: int) -> float:
    s = system.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    system.integrate(steps)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(system, steps: int = 128, cache: str | None = None, verbose: bool = False,
         step_kernels=(1, 4, 5)) -> dict:
    """Pick the step kernel and its launch shape, then the build's, for this system; returns the
    choice and timings.  step_kernels: the step kernels to try (md_adjoint needs one that reads W:
    1, 2 or 3)."""
    key = signature(system)
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                best = table[key]["best"]
                system.set_tuning(**best)
                return table[key]
        except (OSError, ValueError, KeyError):
            pass
    t_start = time.perf_counter()
    steps = max(32, (steps // 16) * 16)           # whole 16-step graph replays
    trials = {}

    def trial(**kw):
        system.set_tuning(**kw)
        system.integrate(16)                       # capture the graph outside the timing
        ms = _time_steps(system, steps)
        trials[json.dumps(kw, sort_keys=True)] = ms
        if verbose:
            print(f"tune {kw}: {ms * 1e3:.1f} us/step", flush=True)
        return ms

    cur = system.tuning()
    best = {k: cur[k] for k in ("ctas_per_sm", "nbr_batch", "build_batch", "step_kernel", "build_stage",
                                "atom_threads")}
    best_ms = trial(**best)
    fp64 = system.params.precision == B.MD_FP64
    kernels = (1,) if fp64 else tuple(step_kernels)
    shapes = []                                    # (step kernel, lanes per atom, residencies, batches)
    for sk in kernels:
        ctas = {1: CTAS, 2: CTAS_RING, 3: CTAS_STAGED, 4: CTAS_CELLS, 5: CTAS_CELLS}[sk]
        shapes.append((sk, 1, ctas, NBR_BATCH if sk < 4 else (2,)))
        if sk == 1 and not fp64:
            shapes += [(1, t, CTAS, NBR_BATCH_TPA) for t in ATOM_THREADS]
    for sk, tpa, ctas_set, nbs in shapes:
        for ctas in ctas_set:
            for nb in nbs:
                cand = dict(best, ctas_per_sm=ctas, nbr_batch=nb, step_kernel=sk, atom_threads=tpa)
                if json.dumps(cand, sort_keys=True) in trials:
                    continue
                ms = trial(**cand)
                if ms < best_ms:
                    best, best_ms = cand, ms
    for bb in BUILD_BATCH:
        for stage in (BUILD_STAGE if bb != 32 else (best["build_stage"],)):
            cand = dict(best, build_batch=bb, build_stage=stage)
            if json.dumps(cand, sort_keys=True) in trials:
                continue
            ms = trial(**cand)
            if ms < best_ms:
                best, best_ms = cand, ms
    system.set_tuning(**best)
    result = {"best": best, "ms_per_step": best_ms, "trials": trials, "signature": key,
              "seconds": time.perf_counter() - t_start}
    if cache:
        try:
            table = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    table = json.load(f)
            table[key] = result
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        except (OSError, ValueError):
            pass
    return result
