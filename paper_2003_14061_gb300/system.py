"""MDSystem: the C ABI of libgbmd.so with a torch-owned device workspace.

PyTorch provides the device memory (one uint8 tensor) and the stream; every computation is a
call into the library.  Host arrays are numpy float64; device tensors may be passed instead for
the initial state and for state exchange (their data pointers go straight to the ABI).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B

_PREC = {"fp64": B.MD_FP64, "mixed": B.MD_MIXED, "fp32": B.MD_FP32}
_RULE = {"vmax": B.MD_REBUILD_VMAX, "disp": B.MD_REBUILD_DISP, "every": B.MD_REBUILD_EVERY}
WCA_RC = 2.0 ** (1.0 / 6.0)


def make_params(*, eps=1.0, sigma=1.0, mass=1.0, rc=WCA_RC, skin=0.4, dt=0.005, shift=True,
                precision="mixed", reorder_every=100, nbr_capacity=0, rebuild_rule="vmax",
                props_every=0, cell_block=0, n=0, box=(1.0, 1.0, 1.0)) -> B.md_params:
    p = B.md_params()
    p.n = int(n)
    for a in range(3):
        p.box[a] = float(box[a])
    p.eps, p.sigma, p.mass, p.rc, p.skin, p.dt = map(float, (eps, sigma, mass, rc, skin, dt))
    p.shift_energy = int(bool(shift))
    p.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    p.reorder_every = int(reorder_every)
    p.nbr_capacity = int(nbr_capacity)
    p.rebuild_rule = _RULE[rebuild_rule] if isinstance(rebuild_rule, str) else int(rebuild_rule)
    p.props_every = int(props_every)
    p.cell_block = int(cell_block)
    return p


def _ptr(a):
    """(pointer, keepalive) for a float64 [n,3] numpy array or a contiguous torch tensor."""
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            a = a.to(torch.float64).contiguous()
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data_as(ctypes.c_void_p), arr


class MDSystem:
    """One system (``box`` given) or a batch of independent replicas (``n_rep`` and ``boxes``)."""

    def __init__(self, x0, v0, box=None, *, n_rep=None, boxes=None, device=None, stream=None, **kw):
        self.lib = B.lib()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if n_rep is None:
            n = int(np.asarray(x0.shape[0]))
            self.n_rep = np.array([n], dtype=np.int64)
            self.boxes = np.asarray(box, dtype=np.float64).reshape(1, 3).copy()
        else:
            self.n_rep = np.ascontiguousarray(n_rep, dtype=np.int64)
            self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        self.n = int(self.n_rep.sum())
        self.params = make_params(n=self.n_rep[0], box=self.boxes[0], **kw)
        nrep = len(self.n_rep)
        nbytes = self.lib.md_workspace_bytes_batch(ctypes.byref(self.params), nrep,
                                                   self.n_rep.ctypes.data_as(ctypes.c_void_p),
                                                   self.boxes.ctypes.data_as(ctypes.c_void_p))
        if nbytes == 0:
            raise B.MDError(-1, "md_workspace_bytes_batch", B.last_error())
        self.workspace_bytes = int(nbytes)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        xp, xk = _ptr(x0)
        vp, vk = _ptr(v0)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            B.check(self.lib.md_create_batch(ctypes.byref(self.params), nrep,
                                             self.n_rep.ctypes.data_as(ctypes.c_void_p),
                                             self.boxes.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.c_void_p(self.workspace.data_ptr()),
                                             self.workspace_bytes, xp, vp,
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)),
                    "md_create_batch")
        self.h = handle
        del xk, vk

    # -- lifecycle ---------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the hot path ------------------------------------------------------------------------
    def _call(self, name, *args):
        with torch.cuda.device(self.device):
            return B.call(name, self.h, *args)

    def bin_cells(self):
        self._call("md_bin_cells")

    def build_neighbours(self):
        self._call("md_build_neighbours")

    def compute_forces(self):
        self._call("md_compute_forces")

    def integrate(self, nsteps: int):
        self._call("md_integrate", int(nsteps))

    # -- results -----------------------------------------------------------------------------
    @property
    def nrep(self) -> int:
        return int(self.lib.md_nrep(self.h))

    @property
    def nbr_capacity(self) -> int:
        return int(self.lib.md_nbr_capacity(self.h))

    def cells_per_axis(self, r: int = 0):
        nc = np.zeros(3, dtype=np.int32)
        self._call("md_cells_per_axis", int(r), nc.ctypes.data_as(ctypes.c_void_p))
        return nc

    def props(self):
        out = (B.md_props * self.nrep)()
        self._call("md_reduce_props", ctypes.cast(out, ctypes.c_void_p))
        return [o.as_dict() for o in out]

    def series(self, max_rows: int = 1024):
        buf = np.zeros((self.nrep, max_rows, B.SERIES_COLS))
        rows = ctypes.c_int32()
        self._call("md_get_series", buf.ctypes.data_as(ctypes.c_void_p), int(max_rows), ctypes.byref(rows))
        return buf[:, : rows.value]

    def props_latest_into(self, dst: torch.Tensor):
        """Queue a copy of the latest props row ([nrep, 9] float64) into dst (pinned or device)."""
        self._call("md_props_latest", ctypes.c_void_p(dst.data_ptr()))

    def clear_series(self):
        self._call("md_clear_series")

    def state(self, x=True, v=True, f=False):
        """(x, v, f) in id order as numpy [n,3] float64 (None where not requested)."""
        out = [np.zeros((self.n, 3)) if w else None for w in (x, v, f)]
        ptrs = [o.ctypes.data_as(ctypes.c_void_p) if o is not None else None for o in out]
        self._call("md_get_state", *ptrs)
        return tuple(out)

    def state_into(self, x: torch.Tensor = None, v: torch.Tensor = None, f: torch.Tensor = None):
        """Write the state into device (or pinned host) float64 tensors of shape [n,3]."""
        ptrs = [ctypes.c_void_p(t.data_ptr()) if t is not None else None for t in (x, v, f)]
        self._call("md_get_state", *ptrs)

    def set_state(self, x, v):
        xp, xk = _ptr(x)
        vp, vk = _ptr(v)
        self._call("md_set_state", xp, vp)

    def cells(self):
        out = np.zeros(self.n, dtype=np.int32)
        self._call("md_get_cells", out.ctypes.data_as(ctypes.c_void_p))
        return out

    def neighbours(self, cap: int = None):
        cap = int(cap or self.nbr_capacity)
        counts = np.zeros(self.n, dtype=np.int32)
        nb = np.full((self.n, cap), -1, dtype=np.int32)
        self._call("md_get_neighbours", counts.ctypes.data_as(ctypes.c_void_p),
                   nb.ctypes.data_as(ctypes.c_void_p), cap)
        return counts, nb

    def check(self):
        self._call("md_check")

    def debug_set_error(self, status: str):
        """Latch a device error as a failing kernel would (tests of the reporting path)."""
        code = {v: k for k, v in B.STATUS.items()}[status]
        self._call("md_debug_set_error", int(code))

    def adjoint(self, nsteps: int, ckpt_every: int = 20, dv0_out: torch.Tensor = None):
        """Loss L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2 and (dL/deps, dL/dsigma, dL/dv0).

        The state is left at its initial value.  dv0_out (float64 [n,3], device or pinned host)
        receives dL/dv0 in place; otherwise a numpy array is returned."""
        nb = self.lib.md_adjoint_workspace_bytes(self.h, int(nsteps), int(ckpt_every))
        if nb == 0:
            raise B.MDError(-1, "md_adjoint_workspace_bytes", B.last_error())
        if getattr(self, "_adj_ws", None) is None or self._adj_ws.numel() < nb:
            with torch.cuda.device(self.device):
                self._adj_ws = torch.empty(int(nb), dtype=torch.uint8, device=self.device)
        loss, ge, gs = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        if dv0_out is not None:
            gv, gptr = dv0_out, ctypes.c_void_p(dv0_out.data_ptr())
        else:
            gv = np.zeros((self.n, 3))
            gptr = gv.ctypes.data_as(ctypes.c_void_p)
        self._call("md_adjoint", ctypes.c_void_p(self._adj_ws.data_ptr()), int(self._adj_ws.numel()), int(nsteps),
                   int(ckpt_every), ctypes.byref(loss), ctypes.byref(ge), ctypes.byref(gs), gptr)
        return loss.value, ge.value, gs.value, gv

    def set_chains(self, length: int, fene_k: float = 30.0, fene_r0: float = 1.5, bend_k: float = 0.0,
                   dihedral_k: float = 0.0):
        """Polymer chains of `length` consecutive ids in every replica (0 removes them)."""
        c = B.md_chains(int(length), 0, float(fene_k), float(fene_r0), float(bend_k), float(dihedral_k))
        self._call("md_set_chains", ctypes.byref(c))

    # -- VACF / MSD of atoms followed by their ids --------------------------------------------
    def dyn_begin(self, nlag: int, origin_every: int):
        """Start a VACF / MSD measurement with its device buffer (torch-owned)."""
        nb = self.lib.md_dyn_workspace_bytes(self.h, int(nlag), int(origin_every))
        if nb == 0:
            raise B.MDError(-1, "md_dyn_workspace_bytes", B.last_error())
        with torch.cuda.device(self.device):
            self._dyn_ws = torch.empty(int(nb), dtype=torch.uint8, device=self.device)
        self._dyn_nlag = int(nlag)
        self._call("md_dyn_begin", ctypes.c_void_p(self._dyn_ws.data_ptr()), int(nb), int(nlag), int(origin_every))

    def dyn_sample(self):
        self._call("md_dyn_sample")

    def dyn_result(self):
        """(vacf [nlag], msd [nlag], counts [nlag]): averages per atom and origin."""
        n = self._dyn_nlag
        vacf, msd = np.zeros(n), np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        self._call("md_dyn_get", vacf.ctypes.data_as(ctypes.c_void_p), msd.ctypes.data_as(ctypes.c_void_p),
                   cnt.ctypes.data_as(ctypes.c_void_p))
        return vacf, msd, cnt

    def set_tuning(self, ctas_per_sm: int = 0, nbr_batch: int = 0, build_batch: int = 0, use_graph: int = 0,
                   step_kernel: int = 0, build_stage: int = 0, reorder_every: int = 0):
        """Launch shapes (0 keeps the current value); use_graph: 1 = CUDA graphs, 2 = direct;
        step_kernel: 1 = per-thread loads with L2 prefetch, 2 = bulk-copy shared-memory ring,
        3 = staged cell-row windows in shared memory, 4 = list-free (27 cells every step),
        5 = half neighbour list with atomic reactions; build_stage: 1 = the build writes W rows
        from shared memory, 2 = entry by entry; reorder_every: reorder by cell every that many
        steps (at a rebuild), -1 = at every rebuild."""
        t = B.md_tuning(int(ctas_per_sm), int(nbr_batch), int(build_batch), int(use_graph), int(step_kernel),
                        int(build_stage), int(reorder_every))
        self._call("md_set_tuning", ctypes.byref(t))

    def set_timing(self, enable: bool = True):
        self._call("md_set_timing", int(bool(enable)))

    def timing(self):
        """{phase: (ms, calls, launches)} since the last call (waits for the stream)."""
        ms = np.zeros(B.NPHASE)
        calls = np.zeros(B.NPHASE, dtype=np.int64)
        launches = np.zeros(B.NPHASE, dtype=np.int64)
        self._call("md_get_timing", ms.ctypes.data_as(ctypes.c_void_p), calls.ctypes.data_as(ctypes.c_void_p),
                   launches.ctypes.data_as(ctypes.c_void_p))
        return {name: (float(ms[k]), int(calls[k]), int(launches[k])) for k, name in enumerate(B.PHASES)}

    def tuning(self):
        t = B.md_tuning()
        self._call("md_get_tuning", ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in t._fields_}
