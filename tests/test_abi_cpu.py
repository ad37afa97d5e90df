"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU, exports every
symbol include/gbmd.h declares, and its host-side planning rejects bad parameters."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2003_14061_gb300 import binding as B
from paper_2003_14061_gb300.system import WCA_RC, make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "gbmd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = B.lib()
    syms = header_symbols()
    assert len(syms) >= 20
    for name in syms:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTS) == syms


def test_nvidia_so_is_native_sm103a():
    path = B.lib_path()
    assert os.path.exists(path)
    blob = open(path, "rb").read()
    assert b"sm_103a" in blob or b"sm_103" in blob


def _bytes(**kw):
    p = make_params(**kw)
    return B.lib().md_workspace_bytes(ctypes.byref(p))


def test_workspace_sizing_and_argument_checks():
    ok = _bytes(n=2048, box=(13.68, 13.68, 13.68))
    assert ok > 0 and ok % 256 == 0
    # bigger systems need more workspace
    assert _bytes(n=4096, box=(17.2, 17.2, 17.2)) > ok
    # fewer than 3 cells of side rc + skin
    assert _bytes(n=100, box=(4.0, 4.0, 4.0)) == 0
    assert "fewer than 3 cells" in B.last_error()
    # more than 1023 cells per axis
    assert _bytes(n=100, box=(2000.0, 10.0, 10.0), skin=0.0) == 0
    assert "1023" in B.last_error()
    for bad in (dict(eps=-1.0), dict(dt=0.0), dict(skin=-0.1), dict(precision=7), dict(rebuild_rule=9),
                dict(reorder_every=-1)):
        assert _bytes(n=2048, box=(13.68,) * 3, **bad) == 0, bad


def test_batch_sizing():
    L = B.lib()
    p = make_params()
    n = np.array([500, 1000, 129], dtype=np.int64)
    boxes = np.array([[8.5] * 3, [10.7] * 3, [6.0] * 3])
    nb = L.md_workspace_bytes_batch(ctypes.byref(p), 3, n.ctypes.data_as(ctypes.c_void_p),
                                    boxes.ctypes.data_as(ctypes.c_void_p))
    assert nb > 0
    boxes[2] = 3.0
    assert L.md_workspace_bytes_batch(ctypes.byref(p), 3, n.ctypes.data_as(ctypes.c_void_p),
                                      boxes.ctypes.data_as(ctypes.c_void_p)) == 0


def test_null_handles_fail_cleanly():
    L = B.lib()
    assert L.md_integrate(None, 1) == -1
    assert L.md_reduce_props(None, None) == -1
    assert L.md_destroy(None) == -1
    assert L.md_nrep(None) == 0


def test_slot_and_cell_limits():
    # 2^26 atom slots: just below is accepted, just above is refused
    p = make_params(n=(1 << 26) - 128, box=(460.0, 460.0, 460.0), skin=0.0)
    assert B.lib().md_workspace_bytes(ctypes.byref(p)) > 0
    p = make_params(n=(1 << 26) + 1, box=(460.0, 460.0, 460.0), skin=0.0)
    assert B.lib().md_workspace_bytes(ctypes.byref(p)) == 0
    assert "2^26" in B.last_error()


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of md_params, md_props and md_tuning against the header, compiled as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"md_params": B.md_params, "md_props": B.md_props, "md_tuning": B.md_tuning, "md_chains": B.md_chains}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gbmd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            *key, val = ln.split()
            got[tuple(key)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def _create_status(n, box, **kw):
    """md_create's status for a system whose host-side plan fails (no device work is reached)."""
    L = B.lib()
    p = make_params(n=n, box=box, **kw)
    x = np.zeros((n, 3))
    v = np.zeros((n, 3))
    h = ctypes.c_void_p()
    fake_ws = ctypes.c_void_p(1 << 20)          # never touched: the plan is refused first
    rc = L.md_create(ctypes.byref(p), fake_ws, 1 << 30, x.ctypes.data_as(ctypes.c_void_p),
                     v.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(h))
    return B.STATUS[rc], h.value


def test_create_reports_box_and_cell_errors():
    # 2 cells of side r_c + skin along an axis (L = 3.0 < 3 (2^(1/6) + 0.4))
    assert _create_status(64, (3.0, 10.0, 10.0)) == ("MD_ERR_BOX_TOO_SMALL", None)
    assert "fewer than 3 cells" in B.last_error()
    # 1024 cells along x
    assert _create_status(64, (1024 * 1.6, 10.0, 10.0)) == ("MD_ERR_CELL_OVERFLOW", None)
    assert "1023" in B.last_error()
    assert _create_status(64, (10.0, 10.0, 10.0), eps=float("nan")) == ("MD_ERR_INVALID_ARG", None)
