"""md_forces_static: forces without any device allocation, checked against md_compute_forces
and against the FP64 oracle.

The entry point serves callers that cannot allocate device memory where they need forces (code
inside a runtime that owns the allocator and hands out only pre-planned buffers, plug-ins where
cudaMalloc's synchronisation is not allowed).  Its scratch lives in a fixed device array inside
the library, so two calls in a row must each reproduce the forces of the regular entry point, and
a request beyond the array's stated limits must be refused.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2003_14061_gb300 import binding as B
from paper_2003_14061_gb300 import inputs
from paper_2003_14061_gb300.system import WCA_RC, MDSystem, make_params

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("ncell,rho,rc,amp", [(6, 0.8, WCA_RC, 0.15), (7, 0.8442, 2.5, 0.08)])
def test_static_scratch_forces_match_regular_entry_point(ncell, rho, rc, amp):
    x, box = inputs.fcc_lattice(ncell, rho)
    x = inputs.perturb(x, box, amp, seed=ncell)
    n = x.shape[0]
    v = inputs.maxwell(n, 1.0, seed=3)
    s = MDSystem(x, v, box, rc=rc, skin=0.3, precision="mixed")
    _, _, f_ref = s.state(x=False, v=False, f=True)          # md_get_state -> md_compute_forces path
    U_ref = s.props()[0]["U"]
    p = make_params(n=n, box=box, rc=rc)
    L = B.lib()
    xd = torch.from_numpy(x).to("cuda")
    fd = torch.empty_like(xd)
    ud = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):                                        # the array keeps the last call's contents
        fd.fill_(float("nan"))
        ud.fill_(float("nan"))
        rc_ = L.md_forces_static(ctypes.byref(p), n, ctypes.c_void_p(xd.data_ptr()),
                                 ctypes.c_void_p(fd.data_ptr()), ctypes.c_void_p(ud.data_ptr()), stream)
        assert rc_ == 0, B.last_error()
        torch.cuda.synchronize()
        f = fd.cpu().numpy()
        assert rel_l2(f, f_ref) <= 1e-5
        assert abs(0.5 * float(ud.sum()) - U_ref) / n <= 1e-6
    s.close()


def test_static_scratch_rejects_oversized_requests():
    L = B.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 65537
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    f = torch.empty_like(x)
    p = make_params(n=n, box=(45.0, 45.0, 45.0))
    rc_ = L.md_forces_static(ctypes.byref(p), n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                             None, stream)
    assert B.STATUS[rc_] == "MD_ERR_INVALID_ARG" and "65536" in B.last_error()
    # too many cells: 80^3 cells of side >= rc
    p = make_params(n=1000, box=(80 * 1.13,) * 3)
    rc_ = L.md_forces_static(ctypes.byref(p), 1000, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                             None, stream)
    assert B.STATUS[rc_] == "MD_ERR_INVALID_ARG" and "cells" in B.last_error()


def _static_forces(p, x):
    L = B.lib()
    n = x.shape[0]
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
    fd = torch.full_like(xd, float("nan"))
    ud = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc_ = L.md_forces_static(ctypes.byref(p), n, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(fd.data_ptr()),
                             ctypes.c_void_p(ud.data_ptr()), stream)
    assert rc_ == 0, B.last_error()
    torch.cuda.synchronize()
    return fd.cpu().numpy(), ud.cpu().numpy()


@pytest.mark.parametrize("ncell,rho,rc,amp", [(6, 0.8, WCA_RC, 0.15), (7, 0.8442, 2.5, 0.08)])
def test_static_scratch_forces_match_oracle(ncell, rho, rc, amp):
    # positions up to four box lengths outside the box: wrapped by the call; forces and u_i
    # against the FP64 oracle on the in-box positions, and identical bits on a repeated call
    x, box = inputs.fcc_lattice(ncell, rho)
    x = inputs.perturb(x, box, amp, seed=ncell + 10)
    k = np.random.default_rng(ncell).integers(-4, 5, x.shape)
    p = make_params(n=x.shape[0], box=box, rc=rc)
    f, u = _static_forces(p, x + k * box)
    of, ou, U, _ = oracle.forces(x, box, oracle.pot(rc=rc))
    assert rel_l2(f, of) <= 1e-5
    assert np.abs(u - ou).max() <= 1e-5 * (np.abs(ou).max() + 1.0)
    assert abs(0.5 * u.sum() - U) / x.shape[0] <= 1e-6
    f2, u2 = _static_forces(p, x + k * box)
    assert np.array_equal(f, f2) and np.array_equal(u, u2)
