"""Plain FP64 CPU oracle for short-range pair-force molecular dynamics.

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU-baseline leg of the
benchmark are the only callers.  Nothing here is shared with, or imported by, the CUDA
library; both sides receive the same seeded inputs from ``paper_2003_14061_gb300.inputs``.

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it with gcc and
wraps each entry point with numpy marshalling.  What every function follows in the paper
(Rapaport, arXiv 2003.14061) is listed in the header of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPROPS = 8
PROP_NAMES = ("U", "K", "W", "P", "px", "py", "pz", "vmax")


class Pot(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("rc", ctypes.c_double),
                ("shift", ctypes.c_int32), ("rc_scales_with_sigma", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -ffp-contract=off, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        d = ctypes.c_double
        P = ctypes.POINTER(Pot)
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        lib.orc_pair.argtypes = [P, d, dp, dp]
        lib.orc_forces_brute.argtypes = [i64, dp, dp, P, dp, dp, dp, dp]
        lib.orc_forces_cells.argtypes = [i64, dp, dp, P, dp, dp, dp, dp]
        lib.orc_force_on_atoms.argtypes = [i64, dp, dp, P, dp, dp, dp, dp, i64, dp, dp, dp]
        lib.orc_cells.argtypes = [i64, dp, dp, d, dp, dp]
        lib.orc_cell_order.argtypes = [i64, dp, i64, dp, dp]
        lib.orc_neighbours.argtypes = [i64, dp, dp, d, d, i32, dp, dp, dp, dp]
        lib.orc_neighbours_sample.argtypes = [i64, dp, dp, d, d, i32, i64, dp, i64, dp, dp]
        lib.orc_props.argtypes = [i64, dp, dp, dp, P, d, dp]
        lib.orc_run.argtypes = [i64, dp, dp, dp, P, d, d, i64, i32, d, dp, dp]
        lib.orc_force_jvp.argtypes = [i64, dp, dp, P, dp, dp]
        lib.orc_param_grads.argtypes = [i64, dp, dp, P, dp, dp, dp, dp]
        lib.orc_adjoint.argtypes = [i64, dp, dp, dp, P, d, d, i64, dp, dp, dp, dp, dp, dp]
        lib.orc_loss.argtypes = [i64, dp, dp, dp, P, d, d, i64, dp]
        lib.orc_dynamics.argtypes = [i64, dp, dp, dp, P, d, d, i64, i32, i32, i32, dp, dp, dp]
        C = ctypes.POINTER(Chains)
        lib.orc_chain_forces.argtypes = [i64, dp, dp, C, dp, dp, dp]
        lib.orc_run_chains.argtypes = [i64, dp, dp, dp, P, C, d, d, i64, dp]
        for name in ("orc_forces_brute", "orc_forces_cells", "orc_force_on_atoms", "orc_cells",
                     "orc_cell_order", "orc_neighbours", "orc_neighbours_sample", "orc_props", "orc_run", "orc_force_jvp",
                     "orc_param_grads", "orc_adjoint", "orc_loss", "orc_dynamics", "orc_chain_forces",
                     "orc_run_chains"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def pot(eps=1.0, sigma=1.0, rc=2.0 ** (1.0 / 6.0), shift=True, rc_scales_with_sigma=None):
    """Pair-potential parameters.  By default r_c moves with sigma only for the WCA cutoff."""
    if rc_scales_with_sigma is None:
        rc_scales_with_sigma = abs(rc / sigma - 2.0 ** (1.0 / 6.0)) < 1e-12
    return Pot(float(eps), float(sigma), float(rc), int(bool(shift)), int(bool(rc_scales_with_sigma)))


class Chains(ctypes.Structure):
    _fields_ = [("len", ctypes.c_int32), ("pad", ctypes.c_int32), ("kb", ctypes.c_double), ("r0", ctypes.c_double),
                ("ka", ctypes.c_double), ("kd", ctypes.c_double)]


def chains(length, kb=30.0, r0=1.5, ka=0.0, kd=0.0):
    """Chains of `length` consecutive ids: FENE bonds (kb, r0), bending ka, dihedral kd."""
    return Chains(int(length), 0, float(kb), float(r0), float(ka), float(kd))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def pair(p: Pot, r2: float):
    """(u, g) of the pair at squared distance r2; the force on i is g * (x_i - x_j)."""
    u = ctypes.c_double()
    g = ctypes.c_double()
    _load().orc_pair(ctypes.byref(p), float(r2), ctypes.byref(u), ctypes.byref(g))
    return u.value, g.value


def forces(x, box, p: Pot, method: str = "cells"):
    """Return (F [n,3], u_atom [n], U, W) from the definition (brute) or over cells."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    n = x.shape[0]
    f = np.zeros((n, 3))
    ua = np.zeros(n)
    U = ctypes.c_double()
    W = ctypes.c_double()
    fn = _load().orc_forces_brute if method == "brute" else _load().orc_forces_cells
    _check(fn(n, _ptr(x), _ptr(box), ctypes.byref(p), _ptr(f), _ptr(ua), ctypes.byref(U),
              ctypes.byref(W)), "forces")
    return f, ua, U.value, W.value


def cells(x, box, r_cell):
    """N1: (n_cells_per_axis [3], cell id per atom)."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    n = x.shape[0]
    nc = np.zeros(3, dtype=np.int32)
    cell = np.zeros(n, dtype=np.int32)
    _check(_load().orc_cells(n, _ptr(x), _ptr(box), float(r_cell), _ptr(nc), _ptr(cell)), "cells")
    return nc, cell


def cell_order(cell, ncells):
    """N2-N4: (start [ncells+1], order [n]) with ascending indices inside each cell."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    n = cell.shape[0]
    start = np.zeros(int(ncells) + 1, dtype=np.int64)
    order = np.zeros(max(n, 1), dtype=np.int64)
    _check(_load().orc_cell_order(n, _ptr(cell), int(ncells), _ptr(start), _ptr(order)), "cell_order")
    return start, order[:n]


def force_on_atoms(x, box, p: Pot, atoms):
    """Forces and u_i on the listed atoms only (definition over cells of side >= r_c)."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    n = x.shape[0]
    nc, cell = cells(x, box, p.rc)
    start, order = cell_order(cell, int(np.prod(nc.astype(np.int64))))
    atoms = np.ascontiguousarray(atoms, dtype=np.int64)
    f = np.zeros((atoms.shape[0], 3))
    ua = np.zeros(atoms.shape[0])
    order = np.ascontiguousarray(order, dtype=np.int64)
    _check(_load().orc_force_on_atoms(n, _ptr(x), _ptr(box), ctypes.byref(p), _ptr(nc), _ptr(cell),
                                      _ptr(start), _ptr(order), atoms.shape[0], _ptr(atoms), _ptr(f),
                                      _ptr(ua)), "force_on_atoms")
    return f, ua


def neighbours(x, box, rc, skin, fp32: bool = True):
    """N5 neighbour sets: (n_cells_per_axis, counts [n], offsets [n+1], nbrs [sum counts])."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    n = x.shape[0]
    nc = np.zeros(3, dtype=np.int32)
    counts = np.zeros(max(n, 1), dtype=np.int64)
    lib = _load()
    _check(lib.orc_neighbours(n, _ptr(x), _ptr(box), float(rc), float(skin), int(fp32), _ptr(nc),
                              _ptr(counts), None, None), "neighbours(count)")
    counts = counts[:n]
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    nbrs = np.zeros(max(int(offsets[-1]), 1), dtype=np.int64)
    counts2 = np.zeros(max(n, 1), dtype=np.int64)
    _check(lib.orc_neighbours(n, _ptr(x), _ptr(box), float(rc), float(skin), int(fp32), _ptr(nc),
                              _ptr(counts2), _ptr(offsets), _ptr(nbrs)), "neighbours(fill)")
    return nc, counts, offsets, nbrs[: int(offsets[-1])]


def neighbours_sample(x, box, rc, skin, atoms, cap, fp32: bool = True):
    """Neighbour sets of the listed atoms: (counts [s], nbrs [s, cap] ascending, -1 padded)."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    atoms = np.ascontiguousarray(atoms, dtype=np.int64)
    counts = np.zeros(atoms.shape[0], dtype=np.int64)
    nb = np.full((atoms.shape[0], int(cap)), -1, dtype=np.int64)
    _check(_load().orc_neighbours_sample(x.shape[0], _ptr(x), _ptr(box), float(rc), float(skin), int(fp32),
                                         atoms.shape[0], _ptr(atoms), int(cap), _ptr(counts), _ptr(nb)),
           "neighbours_sample")
    return counts, nb


def props(x, v, box, p: Pot, mass=1.0):
    """[U, K, W, P, px, py, pz, vmax] at the given state."""
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    box = _f64(box, (3,))
    out = np.zeros(NPROPS)
    _check(_load().orc_props(x.shape[0], _ptr(x), _ptr(v), _ptr(box), ctypes.byref(p), float(mass),
                             _ptr(out)), "props")
    return out


def run(x, v, box, p: Pot, mass=1.0, dt=0.005, nsteps=1, rule=0, skin=0.0, with_props=True):
    """KDK leapfrog for nsteps.  Returns (x, v, props [nsteps+1, 8] or None, rebuilds)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    box = _f64(box, (3,))
    pr = np.zeros((int(nsteps) + 1, NPROPS)) if with_props else None
    rb = ctypes.c_int64()
    _check(_load().orc_run(x.shape[0], _ptr(x), _ptr(v), _ptr(box), ctypes.byref(p), float(mass),
                           float(dt), int(nsteps), int(rule), float(skin), _ptr(pr), ctypes.byref(rb)),
           "run")
    return x, v, pr, rb.value


def force_jvp(x, box, p: Pot, lam):
    x = _f64(x, (-1, 3))
    lam = _f64(lam, (-1, 3))
    box = _f64(box, (3,))
    out = np.zeros_like(x)
    _check(_load().orc_force_jvp(x.shape[0], _ptr(x), _ptr(box), ctypes.byref(p), _ptr(lam), _ptr(out)),
           "force_jvp")
    return out


def param_grads(x, box, p: Pot):
    """(dF/deps [n,3], dF/dsigma [n,3], dU/deps, dU/dsigma)."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    fe = np.zeros_like(x)
    fs = np.zeros_like(x)
    ue = ctypes.c_double()
    us = ctypes.c_double()
    _check(_load().orc_param_grads(x.shape[0], _ptr(x), _ptr(box), ctypes.byref(p), _ptr(fe), _ptr(fs),
                                   ctypes.byref(ue), ctypes.byref(us)), "param_grads")
    return fe, fs, ue.value, us.value


def adjoint(x0, v0, box, p: Pot, mass=1.0, dt=0.005, nsteps=1):
    """Loss and its gradients: (loss, dL/deps, dL/dsigma, dL/dv0 [n,3], x_S, v_S)."""
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    box = _f64(box, (3,))
    n = x0.shape[0]
    loss = ctypes.c_double()
    ge = ctypes.c_double()
    gs = ctypes.c_double()
    gv = np.zeros((n, 3))
    xs = np.zeros((n, 3))
    vs = np.zeros((n, 3))
    _check(_load().orc_adjoint(n, _ptr(x0), _ptr(v0), _ptr(box), ctypes.byref(p), float(mass), float(dt),
                               int(nsteps), ctypes.byref(loss), ctypes.byref(ge), ctypes.byref(gs),
                               _ptr(gv), _ptr(xs), _ptr(vs)), "adjoint")
    return loss.value, ge.value, gs.value, gv, xs, vs


def loss(x0, v0, box, p: Pot, mass=1.0, dt=0.005, nsteps=1):
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    box = _f64(box, (3,))
    out = ctypes.c_double()
    _check(_load().orc_loss(x0.shape[0], _ptr(x0), _ptr(v0), _ptr(box), ctypes.byref(p), float(mass),
                            float(dt), int(nsteps), ctypes.byref(out)), "loss")
    return out.value


def dynamics(x0, v0, box, p: Pot, mass=1.0, dt=0.005, nsamples=1, every=1, nlag=1, origin_every=1):
    """VACF and MSD per atom over lags 0..nlag-1 (samples every `every` steps, a new origin every
    `origin_every` samples): (vacf [nlag], msd [nlag], counts [nlag]) as averages per atom and
    origin, and the number of origins that reached each lag."""
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    box = _f64(box, (3,))
    n = x0.shape[0]
    vacf = np.zeros(int(nlag))
    msd = np.zeros(int(nlag))
    cnt = np.zeros(int(nlag), dtype=np.int64)
    _check(_load().orc_dynamics(n, _ptr(x0), _ptr(v0), _ptr(box), ctypes.byref(p), float(mass), float(dt),
                                int(nsamples), int(every), int(nlag), int(origin_every), _ptr(vacf), _ptr(msd),
                                _ptr(cnt)), "dynamics")
    with np.errstate(invalid="ignore", divide="ignore"):
        return vacf / (n * cnt), msd / (n * cnt), cnt


def chain_forces(x, box, ch: Chains):
    """(F [n,3], U, W) of the chain terms alone."""
    x = _f64(x, (-1, 3))
    box = _f64(box, (3,))
    f = np.zeros_like(x)
    U = ctypes.c_double()
    W = ctypes.c_double()
    _check(_load().orc_chain_forces(x.shape[0], _ptr(x), _ptr(box), ctypes.byref(ch), _ptr(f), ctypes.byref(U),
                                    ctypes.byref(W)), "chain_forces")
    return f, U.value, W.value


def run_chains(x, v, box, p: Pot, ch: Chains, mass=1.0, dt=0.005, nsteps=1):
    """KDK leapfrog with pair and chain forces.  Returns (x, v, props [nsteps+1, 8])."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    box = _f64(box, (3,))
    pr = np.zeros((int(nsteps) + 1, NPROPS))
    _check(_load().orc_run_chains(x.shape[0], _ptr(x), _ptr(v), _ptr(box), ctypes.byref(p), ctypes.byref(ch),
                                  float(mass), float(dt), int(nsteps), _ptr(pr)), "run_chains")
    return x, v, pr
