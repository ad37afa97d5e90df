"""Autotuner for the launch shapes of an MDSystem.

The paper found thread-block size to matter little on its GPU and warned that this need not hold
elsewhere (Sec. 4.1 item 2).  On GB300 the residency of the fused step kernel and the number of
neighbour-matrix loads each thread keeps in flight decide its speed, so they are measured on the
system itself: every candidate advances the live system by a number of steps timed with CUDA
events on the library's stream.  Step kernels 1-3 and builds 2, 4 and 32 perform the same
arithmetic in the same order; the list-free step kernel (4) and the sub-cell build (1) sum each
force in another order, and the half-list kernel (5) adds through atomics in no fixed order, so
choosing them changes the trajectory at the rounding level only.

Search: coordinate descent over (step kernel, ctas_per_sm, nbr_batch) for the step -- the
per-thread kernel at register-bound residencies, the list-free and half-list kernels, and on
request the shared-memory ring and the staged-neighbour kernel (2 and 3, slower on every measured
workload) at the residencies their shared memory allows -- then build_batch and build_stage for
the neighbour build, then the reorder policy (every 100 steps or at every rebuild: the paper's
reorder, Sec. 4.1 item 1, is a trade between the reorder's cost and the locality it restores).

Measurement: each candidate runs with direct launches and the library's per-phase CUDA events,
and is scored as (step-phase ms per step) + (rebuild-phase ms per rebuild) x (rebuilds per step
over the whole search).  Timing whole steps instead would let the number of rebuilds that fall in
a trial (one rebuild of the 16.4M-atom LJ fluid costs as much as ten steps) decide between shapes
a few per cent apart.  The chosen shape is then used with graphs as before.  Results are cached
per GPU and workload signature in a JSON file.
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
REBUILD_PHASES = ("bin", "build")
REORDER = (100, -1)            # reorder every 100 steps, or at every rebuild
BUILD_BATCH = (1, 2, 4, 32)
BUILD_STAGE = (2, 1)           # the build writes W entry by entry, or rows from shared memory


def signature(system) -> str:
    p = system.params
    dev = torch.cuda.get_device_name(system.device)
    return (f"{dev}|prec{p.precision}|n{system.n}|rep{system.nrep}|rc{p.rc:.4f}|skin{p.skin:.3f}|"
            f"rho{system.n / float((system.boxes.prod(axis=1)).sum()):.3f}")


def _counts(system):
    pr = system.props()
    return sum(int(p["rebuilds"]) for p in pr), sum(int(p.get("reorders", 0)) for p in pr)


class _Rate:
    """Rebuilds per step over every trial so far (the same physical system throughout), and the
    last measured cost of one reorder."""
    steps = 0
    rebuilds = 0
    reorder_ms = None


def _time_steps(system, steps: int, rate: _Rate = None) -> float:
    """Score of the current launch shape in ms per step (see the module docstring)."""
    ro = system.tuning().get("reorder_every", 100)
    r0, o0 = _counts(system)
    system.set_timing(True)
    system.integrate(steps)
    ph = system.timing()
    system.set_timing(False)
    r1, o1 = _counts(system)
    k, kr = r1 - r0, o1 - o0
    step_ms = ph["step"][0] / steps
    rebuild_ms = sum(ph[name][0] for name in REBUILD_PHASES)
    reorder_ms = ph["reorder"][0]
    if rate is None:
        return step_ms + (rebuild_ms + reorder_ms) / steps
    rate.steps += steps
    rate.rebuilds += k
    per_step = rate.rebuilds / rate.steps
    score = step_ms + (rebuild_ms / k * per_step if k else rebuild_ms / steps)
    # reorders: every rebuild (ro = -1) or about every ro steps, at the cost of one measured reorder
    if kr:
        rate.reorder_ms = reorder_ms / kr
    if rate.reorder_ms is not None:
        score += rate.reorder_ms * (per_step if ro < 0 else 1.0 / max(ro, 1))
    return score


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

    rate = _Rate()
    use_graph = system.tuning()["use_graph"]

    def trial(**kw):
        system.set_tuning(use_graph=2, **kw)
        system.integrate(16)                       # first launches outside the timing
        ms = _time_steps(system, steps, rate)
        trials[json.dumps(kw, sort_keys=True)] = ms
        if verbose:
            print(f"tune {kw}: {ms * 1e3:.1f} us/step", flush=True)
        return ms

    cur = system.tuning()
    best = {k: cur[k] for k in ("ctas_per_sm", "nbr_batch", "build_batch", "step_kernel", "build_stage",
                                "reorder_every")}
    best_ms = trial(**best)
    kernels = (1,) if system.params.precision == B.MD_FP64 else tuple(step_kernels)
    for sk in kernels:
        for ctas in {1: CTAS, 2: CTAS_RING, 3: CTAS_STAGED, 4: CTAS_CELLS, 5: CTAS_CELLS}[sk]:
            for nb in (NBR_BATCH if sk < 4 else (2,)):
                cand = dict(best, ctas_per_sm=ctas, nbr_batch=nb, step_kernel=sk)
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
    if best["step_kernel"] != 4:          # the list-free kernel reorders at every rebuild anyway
        for ro in REORDER:
            cand = dict(best, reorder_every=ro)
            if json.dumps(cand, sort_keys=True) in trials:
                continue
            ms = trial(**cand)
            if ms < best_ms:
                best, best_ms = cand, ms
    system.set_tuning(use_graph=use_graph, **best)
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
