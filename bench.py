"""Throughput of the MD hot path on GB300: particle-timesteps per second.

One "step" is one leapfrog time step of the whole hot path: the fused force + integration
kernel, the refresh criterion, and (when the criterion fires) cell binning, ordering, reorder and
the neighbour-matrix rebuild.  Default workload: WCA fluid, fcc 100^3 = 4,000,000 atoms at
density 0.8, T = 1, skin 0.4, FP32 pair forces with FP64 state and reductions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload wca4m|lj16m|batch512]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the same workload

Under torchrun (N > 1) every rank advances its own independent copy of the workload (the path has
no exchange between replicas); value = atoms x steps over all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WCA_RC = 2.0 ** (1.0 / 6.0)
WORKLOADS = {
    # fcc n^3 cells, density, temperature, cutoff, skin
    "wca4m": dict(ncell=100, rho=0.8, T=1.0, rc=WCA_RC, skin=0.4, desc="WCA fluid, fcc 100^3 = 4,000,000 atoms"),
    "lj16m": dict(ncell=160, rho=0.8442, T=0.72, rc=2.5, skin=0.3, desc="LJ r_c=2.5 shifted, fcc 160^3 = 16,384,000 atoms"),
    "batch512": dict(nrep=512, nmin=500, nmax=32000, rhomin=0.6, rhomax=0.9, T=1.0, rc=WCA_RC, skin=0.4,
                     desc="512 WCA replicas, N ~ U{500..32000}, rho ~ U[0.6, 0.9]"),
}
METRIC = "particle-timesteps/s"
RULE = "vmax"          # rebuild when the accumulated max-velocity bound on displacement exceeds skin/2
UNIT = "particle-steps/s"
DT = 0.005
SEED = {"wca4m": 2, "lj16m": 3, "batch512": 4}


def combine_ranks(ms: float, atoms: int, steps: int, device=None):
    """(max time over ranks in ms, total atoms, whole-job particle-steps/s); one process per GPU."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    a = torch.tensor([float(atoms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    ms_max, total = float(t.item()), int(a.item())
    return ms_max, total, total * steps / (ms_max * 1e-3)


def code_hash(paths) -> str:
    """sha256 (16 hex digits) of C/CUDA sources (one path or a list) with comments and whitespace
    removed, so that only code changes invalidate a capture taken on them."""
    import hashlib
    import re
    src = ""
    for path in ([paths] if isinstance(paths, str) else paths):
        with open(path) as f:
            src += f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def traffic_per_atom(kernel: str):
    """DRAM bytes per atom of a kernel from its committed ncu capture, if its code is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)[kernel]
        src = rec["source"]
        sha = code_hash([os.path.join(ROOT, p) for p in ([src] if isinstance(src, str) else src)])
        return float(rec["dram_bytes_per_atom"]) if sha == rec["code_sha256_16"] else None
    except (OSError, KeyError, ValueError):
        return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_inputs(name, rank=0, ncell=0):
    from paper_2003_14061_gb300 import inputs
    w = WORKLOADS[name]
    seed = SEED[name] + 1000 * rank
    if name == "batch512":
        specs = inputs.replica_specs(w["nrep"], w["nmin"], w["nmax"], w["rhomin"], w["rhomax"], seed)
        states = inputs.replica_states(specs, w["T"], seed)
        x = np.concatenate([s[0] for s in states])
        v = np.concatenate([s[1] for s in states])
        return x, v, dict(n_rep=[s[0] for s in specs], boxes=np.stack([s[2] for s in states]))
    x, box = inputs.fcc_lattice(ncell or w["ncell"], w["rho"])
    v = inputs.maxwell(x.shape[0], w["T"], seed)
    return x, v, dict(box=box)


class NvmlClocks:
    """Read-only NVML queries (libnvidia-ml through ctypes) of one GPU: SM clock, its maximum and
    the active clock-event reason bits.  Nothing is set."""

    def __init__(self, dev_index: int = 0):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        rc = -1
        try:
            import torch
            pr = torch.cuda.get_device_properties(dev_index)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h))
        except Exception:
            rc = -1
        if rc != 0 and self.lib.nvmlDeviceGetHandleByIndex_v2(int(dev_index), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle for the device")
        self._u = ctypes.c_uint()
        self._r = ctypes.c_ulonglong()
        self._getr = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        """(sm_mhz, sm_max_mhz, reason_bits)"""
        ct = self.ct
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(self._u))          # NVML_CLOCK_SM
        sm = float(self._u.value)
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(self._u))
        mx = float(self._u.value)
        self._getr(self.h, ct.byref(self._r))
        return sm, mx, int(self._r.value)


class ClockSampler:
    """SM clock and clock-event reasons sampled while the timed region runs.

    A background thread polls the source every `period` seconds, with one sample at entry and one
    at exit as well, so a timed region of a few milliseconds still has samples.  The source is
    NVML (read-only); without it, `nvidia-smi --query-gpu ... -lms 5` is read instead."""

    # clock-event reason bits of NVML (nvml.h)
    REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                   0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period=0.002, source=None):
        self.index = index
        self.period = period
        self.src = source
        self.samples = []
        self.proc = None
        self.lines = []
        self.kind = None

    def _poll(self):
        import time as _t
        while not self._stop.is_set():
            try:
                self.samples.append(self.src.sample())
            except Exception:
                return
            _t.sleep(self.period)

    def __enter__(self):
        import threading
        if self.src is None:
            try:
                self.src = NvmlClocks(self.index)
            except Exception:
                self.src = None
        if self.src is not None:
            self.kind = "nvml"
            self._stop = threading.Event()
            try:
                self.samples.append(self.src.sample())
            except Exception:
                pass
            self._th = threading.Thread(target=self._poll, daemon=True)
            self._th.start()
            return self
        try:
            self.kind = "nvidia-smi"
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "5"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.src is not None and self.kind == "nvml":
            self._stop.set()
            self._th.join(timeout=2)
            try:
                self.samples.append(self.src.sample())
            except Exception:
                pass
        elif self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        for smhz, mmhz, bits in self.samples:
            sm.append(smhz)
            mx = mmhz
            for b, nm in self.REASON_BITS.items():
                if bits & b:
                    reasons.add(nm)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": self.kind}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "source": self.kind}


def algorithmic_bytes_per_atom_step(mean_nbrs: float, precision: str = "mixed", rule: str = "vmax") -> float:
    """Bytes the fused step must move per atom (W counted at its mean row length).

    mixed: read pos32 16 + count 4 + W 4m + x 24 + v 24; write x 24 + v 24 + pos32 16.
    The max-displacement rule also reads the position at the last rebuild (16).
    """
    ref = 16.0 if rule == "disp" else 0.0
    if precision == "mixed":
        return 132.0 + ref + 4.0 * mean_nbrs
    if precision == "fp32":
        return 16 + 4 + 12 + 16 + 12 + ref + 4.0 * mean_nbrs
    return 32 + 4 + 24 + 24 + 24 + 24 + 32 + ref + 4.0 * mean_nbrs


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(x, v, box, rc, steps, threads):
    """Particle-steps/s of the FP64 oracle on the given state (host cores)."""
    import oracle
    oracle.set_threads(threads)
    p = oracle.pot(rc=rc)
    t0 = time.perf_counter()
    oracle.run(x, v, box, p, dt=DT, nsteps=steps, with_props=False)
    dt = time.perf_counter() - t0
    return x.shape[0] * steps / dt, dt


def run_gb300(args, rank, world, local_rank):
    import torch
    from paper_2003_14061_gb300.system import MDSystem

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOADS[args.workload]
    x, v, geo = make_inputs(args.workload, rank, args.ncell)
    n = x.shape[0]
    s = MDSystem(x, v, device=dev, rc=w["rc"], skin=w["skin"], dt=DT, precision=args.precision, reorder_every=100,
                 rebuild_rule=RULE, props_every=args.props_every, **geo)
    if args.ctas_per_sm or args.nbr_batch or args.build_batch:
        s.set_tuning(ctas_per_sm=args.ctas_per_sm, nbr_batch=args.nbr_batch, build_batch=args.build_batch)
    tuned = None
    if args.tune:
        from paper_2003_14061_gb300 import tune as gtune
        s.integrate(max(args.warmup // 2, 16))     # melt first: tune on the fluid
        # the neighbour-matrix kernel (the paper's method, deterministic); the list-free and
        # half-list kernels are forms of their own
        tuned = gtune.tune(s, steps=args.tune_steps, step_kernels=(1,))
    if args.no_graph:          # direct launches (ncu cannot profile kernels of graphs with IF nodes)
        s.set_tuning(use_graph=2)
    stream = s.stream
    # warm-up (also melts the lattice: timed steps see a fluid)
    s.integrate(args.warmup)
    torch.cuda.synchronize()
    rb0 = [p["rebuilds"] for p in s.props()]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s.timing()                                  # reset launch counters
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        s.integrate(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    issued = s.timing()
    props = s.props()
    rebuilds_timed = sum(p["rebuilds"] - r0 for p, r0 in zip(props, rb0))
    # kernels that ran: the library counts the host-issued ones and, inside captured graphs, the
    # kernels of every rebuild sequence whose IF node opened (a device counter it reads back)
    graph_mode = s.tuning()["use_graph"] == 1
    launches = sum(p[2] for p in issued.values())
    mean_nbrs = float(np.average([p["mean_nbrs"] for p in props], weights=s.n_rep))
    if world > 1:
        ms, total_atoms, value = combine_ranks(ms, n, args.steps, device=dev)
    else:
        total_atoms = n
        value = total_atoms * args.steps / (ms * 1e-3)

    # per-kernel durations: the same workload continued with direct launches, every phase
    # bracketed by CUDA events on the library's stream (graph replays cannot be split per kernel)
    s.set_tuning(use_graph=2)
    s.set_timing(True)
    s.integrate(min(args.steps, args.phase_steps))
    phases = s.timing()
    s.set_timing(False)
    s.set_tuning(use_graph=2 if args.no_graph else 1)
    step_ms, step_calls, step_launches = phases["step"]
    # with the props in every step, every timed launch is the step kernel's props form
    mode = {"mixed": "MD_MIXED", "fp32": "MD_FP32", "fp64": "MD_FP64"}[args.precision]
    roof_kernel = (f"k_step_sm<{mode}, props>" if args.props_every == 1 else f"k_step_sm<{mode}>") \
        if args.precision != "fp64" else "k_step<MD_FP64>"
    peak, peak_kind = load_peaks()
    bpa = algorithmic_bytes_per_atom_step(mean_nbrs, args.precision, RULE)
    per_launch_ms = step_ms / max(step_calls, 1)
    achieved = bpa * n / (per_launch_ms * 1e-3) / 1e9

    # end to end through the public API with host buffers: every step the library's step (with the
    # energy reduction F2 fused) and a device-to-host read of that step's props row into pinned
    # memory; the state goes host-to-device at the start and device-to-host at the end
    e2e_steps = min(args.steps, args.e2e_steps)
    se = MDSystem(x, v, device=dev, rc=w["rc"], skin=w["skin"], dt=DT, precision=args.precision, reorder_every=100,
                  rebuild_rule=RULE, props_every=1, **geo)
    se.set_tuning(**{k: s.tuning()[k] for k in ("ctas_per_sm", "nbr_batch", "build_batch", "build_stage", "step_kernel",
                                                     "reorder_every")})
    se.integrate(32)                                     # capture its graphs outside the timing:
    se.integrate(1)                                      # the 16-step ones and the one-step ones
    se.integrate(1)                                      # from either position buffer
    xh = torch.from_numpy(x).pin_memory()
    vh = torch.from_numpy(v).pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    vo = torch.empty_like(vh).pin_memory()
    rows = torch.empty((e2e_steps, se.nrep, 9), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    se.set_state(xh, vh)
    for k in range(e2e_steps):
        se.integrate(1)
        se.props_latest_into(rows[k])
    se.state_into(xo, vo)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = total_atoms * e2e_steps / e2e_s
    e2e_energy = float(rows[-1, 0, 1] + rows[-1, 0, 2]) / n
    se.close()
    props_bytes = 9 * 8 * s.nrep

    result = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            threads = os.cpu_count() or 1
            if args.workload == "batch512":
                from paper_2003_14061_gb300 import inputs
                specs = inputs.replica_specs(8, 500, 32000, 0.6, 0.9, SEED["batch512"])
                sts = inputs.replica_states(specs, 1.0, SEED["batch512"])
                atoms, secs = 0, 0.0
                for xs, vs, bs in sts:
                    r, dtt = cpu_oracle_rate(xs, vs, bs, w["rc"], 10, threads)
                    atoms += xs.shape[0] * 10
                    secs += dtt
                rate, sample = atoms / secs, "first 8 replicas of the batch recipe, 10 steps each"
            else:
                steps_cpu = args.cpu_steps
                rate, _ = cpu_oracle_rate(x, v, geo["box"], w["rc"], steps_cpu, threads)
                sample = f"{steps_cpu} steps of the full {n}-atom system from its initial state"
            one = None
            if args.workload != "batch512" and args.cpu_steps_1t > 0:
                r1, s1 = cpu_oracle_rate(x, v, geo["box"], w["rc"], args.cpu_steps_1t, 1)
                one = {"value": r1, "unit": UNIT, "cores": 1, "seconds": s1,
                       "sample": f"{args.cpu_steps_1t} steps of the full {n}-atom system, one thread"}
            cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                   "cpu_model": cpu_model(), "nproc": os.cpu_count(), "single_thread": one,
                   "note": "the FP64 oracle as written: OpenMP over atoms in its force loop, its kick-drift loop serial"}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp32": "f32", "fp64": "f64"}[args.precision], "data": "synthetic",
            "config": {"workload": w["desc"] if not args.ncell else f"{w['desc']} (resized: fcc {args.ncell}^3)",
                       "atoms_per_gpu": n, "precision": {"mixed": "FP32 pair forces, FP64 state",
                                                        "fp32": "FP32 pair forces and state",
                                                        "fp64": "FP64 throughout"}[args.precision],
                       "skin": w["skin"], "rc": w["rc"], "dt": DT, "reorder_every": 100,
                       "rebuild_rule": "accumulated bound dt*max|v| on the largest displacement since the last rebuild > skin/2 (the paper's criterion; the exact-displacement rule is the form wca4m_mixed_disp)",
                       "l2": "inputs larger than L2 (state %.2f GB)" % (s.workspace_bytes / 1e9),
                       "mean_neighbours": mean_nbrs,
                       "rebuilds_per_100_steps": 100.0 * rebuilds_timed / max(s.nrep, 1) / args.steps,
                       "cuda_graph": graph_mode,
                       "props_every": args.props_every,
                       "reductions": ("every step: max |v| (refresh criterion) and, fused into the step kernel, "
                                      "U, K, virial, pressure and momentum into the device time series"
                                      if args.props_every == 1 else
                                      "every step: max |v| (refresh criterion); U, K, virial, pressure and "
                                      "momentum fused into every %d-th step" % args.props_every
                                      if args.props_every > 1 else
                                      "every step: max |v| (refresh criterion) only; the energy/virial reductions "
                                      "are the forms wca4m_mixed_props1/_props10 and the e2e loop")},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": (lambda b: None if b is None else b * n)(traffic_per_atom(roof_kernel)),
                         "kernel": roof_kernel,
                         "bytes_per_atom": bpa, "peak_kind": peak_kind},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 48.0 * total_atoms / e2e_steps,
                    "d2h_bytes_per_step": props_bytes + 48.0 * total_atoms / e2e_steps, "steps": e2e_steps,
                    "per_step_result": "props row (step, U, K, W, P, momentum, vmax) to pinned host memory",
                    "energy_per_atom_last": e2e_energy},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "tuning": s.tuning(),
            "tune_trials_us_per_step": {k: round(v * 1e3, 1) for k, v in (tuned or {}).get("trials", {}).items()},
            "phases_ms_direct": {k: round(vv[0], 3) for k, vv in phases.items()},
            "phase_steps_direct": min(args.steps, args.phase_steps),
            "kernel_ms_per_launch": per_launch_ms,
        }
    s.close()
    if rank == 0 and world == 1 and args.forms and not args.ncell:
        result["forms"] = measure_forms(args, dev)
    return result


def _event_ms(s, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    fn()
    e1.record(s.stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def measure_form(label, x, v, geo, dev, precision, rc, skin, steps, warmup, tune=True, rule="vmax",
                 props_every=0, fixed=None):
    """Particle-steps/s of one form of the hot path, with its step-kernel roofline fraction."""
    from paper_2003_14061_gb300 import tune as gtune
    from paper_2003_14061_gb300.system import MDSystem
    s = MDSystem(x, v, device=dev, rc=rc, skin=skin, dt=DT, precision=precision, reorder_every=100,
                 rebuild_rule=rule, props_every=props_every, **geo)
    s.integrate(max(warmup // 2, 16))
    if fixed:
        s.set_tuning(**fixed)
    elif tune:
        gtune.tune(s, steps=64, step_kernels=(1,))    # the neighbour-matrix kernel; 4 and 5 have forms of their own
    s.integrate(max(warmup // 2, 16))
    p0 = s.props()
    ms = _event_ms(s, lambda: s.integrate(steps))
    p1 = s.props()
    n = s.n
    mean_nbrs = float(np.average([p["mean_nbrs"] for p in p1], weights=s.n_rep))
    s.set_tuning(use_graph=2)
    s.set_timing(True)
    s.integrate(min(steps, 200))
    ph = s.timing()
    s.set_timing(False)
    step_ms = ph["step"][0] / max(ph["step"][1], 1)
    peak, kind = load_peaks()
    bpa = algorithmic_bytes_per_atom_step(mean_nbrs, precision, rule)
    if fixed and fixed.get("step_kernel") == 4:
        bpa = algorithmic_bytes_per_atom_step(0.0, precision, rule) - 4.0    # no W and no neighbour counts
    elif fixed and fixed.get("step_kernel") == 5:
        bpa += 40.0       # half W (mean_nbrs is the half count) + the FP32 force buffers read and cleared
    achieved = bpa * n / (step_ms * 1e-3) / 1e9
    out = {"label": label, "value": n * steps / (ms * 1e-3), "unit": UNIT, "atoms": n, "replicas": s.nrep,
           "steps": steps, "ms_per_step": ms / steps, "precision": precision, "props_every": props_every,
           "mean_neighbours": mean_nbrs,
           "rebuilds_per_100_steps": 100.0 * sum(a["rebuilds"] - b["rebuilds"] for a, b in zip(p1, p0)) / s.nrep / steps,
           "kernel_ms_per_launch": step_ms, "tuning": s.tuning(),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "bytes_per_atom": bpa, "peak_kind": kind},
           "energy_per_atom": float(np.average([p["E_per_atom"] for p in p1], weights=s.n_rep))}
    s.close()
    return out


def measure_dynamics(dev, n_edge=100, every=10, nsamples=100, nlag=50, origin_every=10):
    """VACF, MSD and the self-diffusion coefficient of the SP fluid at density 1.0, T = 1, with
    the throughput of the steps and samples together.  The start is the paper's (Sec. 3.1): a
    simple cubic grid (spacing 1.0 < r_c, so it melts), brought to T = 1 by rescaling the
    velocities every 100 steps for 500 steps before the measurement."""
    from paper_2003_14061_gb300 import inputs
    from paper_2003_14061_gb300.system import MDSystem
    x, box = inputs.cubic_lattice(n_edge, 1.0)
    v = inputs.maxwell(x.shape[0], 1.0, 7)
    s = MDSystem(x, v, box, device=dev, rc=WCA_RC, skin=0.4, dt=DT, precision="mixed", reorder_every=100)
    for _ in range(5):
        s.integrate(100)
        xs, vs, _ = s.state()
        vs -= vs.mean(0)
        vs *= math.sqrt(3.0 * (vs.shape[0] - 1) / float((vs * vs).sum()))
        s.set_state(xs, vs)
    s.integrate(100)
    T_start = float(s.props()[0]["K"]) * 2.0 / (3.0 * (s.n - 1))
    s.dyn_begin(nlag, origin_every)

    def loop():
        for k in range(nsamples):
            if k:
                s.integrate(every)
            s.dyn_sample()

    ms = _event_ms(s, loop)
    vacf, msd, cnt = s.dyn_result()
    n = s.n
    T = every * DT
    lags = np.arange(nlag) * T
    half = nlag // 2
    slope = np.polyfit(lags[half:], msd[half:], 1)[0]
    kmin = int(np.argmin(vacf))
    s.close()
    steps = (nsamples - 1) * every
    return {"label": "SP fluid rho = 1.0, T = 1 (simple cubic %d^3 start, melted) = %d atoms: VACF and MSD every %d "
                     "steps" % (n_edge, n, every), "temperature_at_start": T_start,
            "value": n * steps / (ms * 1e-3), "unit": UNIT, "steps": steps, "samples": nsamples,
            "ms_per_step_with_samples": ms / steps, "vacf0": float(vacf[0]), "vacf_min": float(vacf[kmin]),
            "vacf_min_time": float(lags[kmin]), "diffusion_D": float(slope / 6.0),
            "msd_last": float(msd[-1]), "lag_time": T, "origins_at_last_lag": int(cnt[-1]),
            "vacf": [round(float(a), 6) for a in vacf], "msd": [round(float(a), 6) for a in msd]}


def measure_forms(args, dev):
    """The other forms of the hot path, each reported beside the main line."""
    from paper_2003_14061_gb300 import inputs
    from paper_2003_14061_gb300.system import MDSystem
    forms = {}
    t0 = time.perf_counter()
    # plain FP32 (pair forces and state) on the main workload
    x, v, geo = make_inputs("wca4m")
    forms["wca4m_fp32"] = measure_form("WCA fcc 100^3, FP32 state", x, v, geo, dev, "fp32", WCA_RC, 0.4,
                                       args.form_steps, 200)
    # the main workload with the energy/virial/momentum reductions (F2) fused into every step, and
    # into every 10th step
    forms["wca4m_mixed_props1"] = measure_form("WCA fcc 100^3, MIXED, U/K/W/P/momentum reduced every step", x, v,
                                               geo, dev, "mixed", WCA_RC, 0.4, args.form_steps, 200, props_every=1)
    forms["wca4m_mixed_props10"] = measure_form("WCA fcc 100^3, MIXED, U/K/W/P/momentum reduced every 10 steps", x,
                                                v, geo, dev, "mixed", WCA_RC, 0.4, args.form_steps, 200,
                                                props_every=10)
    # the list-free step kernel (no neighbour matrix; the cell-block alternative of Sec. 4.2 item
    # 1), A/B against the neighbour-matrix kernel on the main workload
    forms["wca4m_mixed_list_free"] = measure_form("WCA fcc 100^3, MIXED, list-free step kernel (27 cells every step)",
                                                  x, v, geo, dev, "mixed", WCA_RC, 0.4, args.form_steps, 200,
                                                  fixed=dict(step_kernel=4, ctas_per_sm=8))
    # the half neighbour list with Newton's third law (the variant Sec. 2.3 rejects), A/B
    forms["wca4m_mixed_half_list"] = measure_form("WCA fcc 100^3, MIXED, half neighbour list + atomic reactions",
                                                  x, v, geo, dev, "mixed", WCA_RC, 0.4, args.form_steps, 200,
                                                  fixed=dict(step_kernel=5, ctas_per_sm=8))
    # the main workload with the exact-displacement refresh rule (reads the positions at the last
    # rebuild every step)
    forms["wca4m_mixed_disp"] = measure_form("WCA fcc 100^3, MIXED, rebuild on max |x - x_ref| > skin/2", x, v, geo,
                                             dev, "mixed", WCA_RC, 0.4, args.form_steps, 200, rule="disp")
    # the LJ liquid (r_c = 2.5, shifted), 16,384,000 atoms
    w = WORKLOADS["lj16m"]
    x, v, geo = make_inputs("lj16m")
    forms["lj16m_mixed"] = measure_form(w["desc"], x, v, geo, dev, "mixed", w["rc"], w["skin"],
                                        max(args.form_steps // 4, 100), 100)
    forms["lj16m_mixed_half_list"] = measure_form(w["desc"] + ", half neighbour list + atomic reactions", x, v, geo,
                                                  dev, "mixed", w["rc"], w["skin"], max(args.form_steps // 8, 50), 100,
                                                  fixed=dict(step_kernel=5, ctas_per_sm=8, build_batch=32))
    del x, v
    # 512 independent replicas of uneven size in one persistent launch per step
    w = WORKLOADS["batch512"]
    x, v, geo = make_inputs("batch512")
    forms["batch512_mixed"] = measure_form(w["desc"], x, v, geo, dev, "mixed", w["rc"], w["skin"],
                                           args.form_steps, 200)
    # physics measurement: the SP fluid at density 1.0 (Sec. 4.1 item 7), VACF and MSD of atoms
    # followed by their ids, sampled every 10 steps over 1000 steps
    forms["sp_rho1_dynamics"] = measure_dynamics(dev)
    # FP64 cell list (skin 0, rebuilt every step), 2048 atoms: L2-resident, steps/s is the figure
    xl, box = inputs.fcc_lattice(8, 0.8)
    vl = inputs.maxwell(xl.shape[0], 1.0, 1)
    s = MDSystem(xl, vl, box, device=dev, rc=WCA_RC, skin=0.0, dt=DT, precision="fp64", reorder_every=100)
    s.integrate(100)
    ms = _event_ms(s, lambda: s.integrate(1000))
    forms["wca2048_fp64_celllist"] = {"label": "WCA fcc 8^3 = 2048 atoms, FP64, cell list rebuilt every step",
                                      "value": 2048 * 1000 / (ms * 1e-3), "unit": UNIT,
                                      "steps_per_s": 1000 / (ms * 1e-3), "ms_per_step": ms / 1000,
                                      "note": "working set in L2; no HBM roofline"}
    s.close()
    # adjoint: 32,000 atoms, 400 steps, checkpoints every 20
    xa, boxa = inputs.fcc_subset(32000, 0.8, seed=5)
    va = inputs.maxwell(32000, 1.0, seed=6)
    s = MDSystem(xa, va, boxa, device=dev, rc=WCA_RC, skin=0.4, dt=DT, precision="mixed")
    from paper_2003_14061_gb300 import tune as gtune
    # launch shapes for this 32k-atom system: the adjoint reads W, so kernels 1-3 (the
    # shared-memory ring, kernel 2, wins at this L2-resident size)
    gtune.tune(s, steps=64, step_kernels=(1, 2, 3))
    s.adjoint(400, 20)                                     # warm-up (workspace, graphs, lazy loads)
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    s.adjoint(400, 20)
    secs = time.perf_counter() - t
    forms["adjoint32k"] = {"label": "adjoint, WCA 32,000 atoms, 400 steps, checkpoints every 20",
                           "value": 400 / secs, "unit": "grad-steps/s", "seconds_per_gradient": secs,
                           "particle_grad_steps_per_s": 32000 * 400 / secs,
                           "tuning": s.tuning(),
                           "note": "a grad-step = forward step + recomputed step + reverse step; working set in L2"}
    s.close()
    forms["seconds"] = time.perf_counter() - t0
    return forms


def run_reference(args):
    """The FP64 CPU oracle on a bounded sample of the same workload (host cores)."""
    import oracle
    from paper_2003_14061_gb300 import inputs
    w = WORKLOADS[args.workload]
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    p = oracle.pot(rc=w["rc"])
    # calibrate the per-atom-step cost on a small system of the same recipe
    rho = w.get("rho", 0.75)
    xc, bc = inputs.fcc_lattice(16, rho)
    vc = inputs.maxwell(xc.shape[0], w["T"], 1)
    t0 = time.perf_counter()
    oracle.run(xc, vc, bc, p, dt=DT, nsteps=2, with_props=False)
    per = (time.perf_counter() - t0) / (2 * xc.shape[0])
    budget = args.ref_seconds
    natoms = budget / max(per * (args.steps + args.warmup), 1e-12)
    full = 4 * w["ncell"] ** 3 if "ncell" in w else 8_300_000
    ncell = max(6, min(int((min(natoms, full) / 4.0) ** (1.0 / 3.0)), w.get("ncell", 10 ** 6)))
    x, box = inputs.fcc_lattice(ncell, rho)
    v = inputs.maxwell(x.shape[0], w["T"], SEED[args.workload])
    x, v, _, _ = oracle.run(x, v, box, p, dt=DT, nsteps=args.warmup, with_props=False)
    t0 = time.perf_counter()
    oracle.run(x, v, box, p, dt=DT, nsteps=args.steps, with_props=False)
    secs = time.perf_counter() - t0
    value = x.shape[0] * args.steps / secs
    sample = f"fcc {ncell}^3 = {x.shape[0]} atoms of the same recipe, {args.steps} steps"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "device": "host cores (the FP64 oracle)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "atoms": x.shape[0]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=300)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="wca4m", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"],
                    help="precision of the timed system (the default is the benchmark's)")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--ncell", type=int, default=0, help="fcc cells per axis (smaller case for profiling)")
    ap.add_argument("--nbr-batch", type=int, default=0)
    ap.add_argument("--build-batch", type=int, default=0)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--tune", type=int, default=1, help="1: autotune launch shapes during warm-up")
    ap.add_argument("--tune-steps", type=int, default=128)
    ap.add_argument("--forms", type=int, default=1, help="1: also measure the FP32, LJ, batched, FP64 and adjoint forms")
    ap.add_argument("--form-steps", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--phase-steps", type=int, default=400)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--cpu-steps-1t", type=int, default=2, help="steps of the one-thread oracle timing (0: skip)")
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--props-every", type=int, default=1,
                    help="steps between fused reductions of U, K, virial, pressure and momentum (0: none)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_gb300(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
