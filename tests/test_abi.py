"""The C-ABI library loads and exports every symbol the header declares.

Host-only calls (descriptor validation and workspace sizing) run without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_03876_gb300.build import build

    build()
    from paper_1908_03876_gb300 import _lib

    return _lib.load(), _lib


def _header_symbols():
    syms = set()
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            with open(os.path.join(ROOT, "include", name)) as fh:
                text = fh.read()
            syms |= set(re.findall(r"^(?:cx_status|const char\*|size_t|int)\s+(cx\w*_\w+)\s*\(", text, flags=re.M))
    return sorted(syms)


def test_exports_every_declared_symbol(lib):
    so, mod = lib
    syms = _header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(so, s), s
    assert sorted(mod.EXPORTS) == syms


def test_struct_layout_matches_header(lib, tmp_path):
    """ctypes Desc/StepInfo layouts equal the C layouts compiled from the header."""
    so, mod = lib
    fields = [f for f, _ in mod.Desc._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cxlbm.h"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(cx_problem_desc), sizeof(cx_step_info));']
    lines += [f'printf("%zu\\n", offsetof(cx_problem_desc, {f}));' for f in fields]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    assert int(out[0]) == ctypes.sizeof(mod.Desc)
    assert int(out[1]) == ctypes.sizeof(mod.StepInfo)
    for f, off in zip(fields, out[2:]):
        assert getattr(mod.Desc, f).offset == int(off), f


def _desc(mod, **kw):
    d = mod.Desc()
    d.nx, d.ny, d.n_steps, d.lattice, d.precision, d.ckpt_every = 64, 48, 20, 9, 32, 5
    d.tau, d.d_u, d.d_v = 1.0, 1.0, 1.0
    d.D_u = (ctypes.c_double * 3)(0.05, 0.0, 0.05)
    d.D_v = (ctypes.c_double * 3)(0.2, 0.0, 0.2)
    d.u_target = ctypes.c_void_p(0x1000)
    d.s = (ctypes.c_double * 7)(*([1.0] * 7))
    d.source_order = 2
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_workspace_size_and_validation(lib):
    so, mod = lib
    n = ctypes.c_size_t(0)
    assert so.cx_workspace_size(ctypes.byref(_desc(mod)), ctypes.byref(n)) == 0
    plane = 64 * 48
    # at least: 4 population buffers + 4 checkpoints + tape of 5 steps
    assert n.value >= (4 + 4) * 2 * 9 * plane * 4 + 5 * 3 * plane * 4
    n64 = ctypes.c_size_t(0)
    assert so.cx_workspace_size(ctypes.byref(_desc(mod, precision=64)), ctypes.byref(n64)) == 0
    assert n64.value > n.value
    bad = [dict(lattice=7), dict(precision=16), dict(nx=2), dict(n_steps=0), dict(d_u=0.0),
           dict(source_order=3), dict(aniso=1), dict(adv=1), dict(lattice=5, adv=1, a=ctypes.c_void_p(8)),
           dict(ctrl_nx=10, ctrl_ny=10, ctrl_x0=60), dict(alpha=-1.0), dict(u_target=None)]
    for kw in bad:
        assert so.cx_workspace_size(ctypes.byref(_desc(mod, **kw)), ctypes.byref(n)) == 1, kw
    d = _desc(mod)
    d.s[3] = 2.5
    assert so.cx_workspace_size(ctypes.byref(d), ctypes.byref(n)) == 1


def test_create_rejects_bad_workspace_without_gpu(lib):
    so, mod = lib
    h = ctypes.c_void_p()
    # misaligned or too small workspaces are refused before any device work
    assert so.cx_create(ctypes.byref(_desc(mod)), ctypes.c_void_p(0x1001), 1 << 30, None, ctypes.byref(h)) == 2
    assert so.cx_create(ctypes.byref(_desc(mod)), ctypes.c_void_p(0x1000), 16, None, ctypes.byref(h)) == 2
    assert so.cx_status_string(6) == b"line search failed"


def test_batch_descriptors_must_share_schedule(lib):
    so, mod = lib
    d = (mod.Desc * 2)(_desc(mod), _desc(mod, nx=40, ny=24))
    n = ctypes.c_size_t(0)
    assert so.cx_batch_workspace_size(d, 2, ctypes.byref(n)) == 0
    single = ctypes.c_size_t(0)
    assert so.cx_workspace_size(ctypes.byref(d[0]), ctypes.byref(single)) == 0
    assert n.value > single.value
    for kw in (dict(n_steps=21), dict(precision=64), dict(lattice=5), dict(ckpt_every=7)):
        bad = (mod.Desc * 2)(_desc(mod), _desc(mod, **kw))
        assert so.cx_batch_workspace_size(bad, 2, ctypes.byref(n)) == 1, kw
    assert so.cx_batch_workspace_size(d, 0, ctypes.byref(n)) == 1


def test_arc_desc_layout_matches_header(lib, tmp_path):
    """ctypes Desc3 layout equals cx3_desc compiled from include/cxarc.h."""
    so, mod = lib
    fields = [f for f, _ in mod.Desc3._fields_]
    src = tmp_path / "layout3.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cxarc.h"', "int main(void){",
             'printf("%zu\\n", sizeof(cx3_desc));']
    lines += [f'printf("%zu\\n", offsetof(cx3_desc, {f}));' for f in fields]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout3"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    assert int(out[0]) == ctypes.sizeof(mod.Desc3)
    for f, off in zip(fields, out[1:]):
        assert getattr(mod.Desc3, f).offset == int(off), f


def _desc3(mod, **kw):
    d = mod.Desc3()
    d.nx, d.ny, d.n_steps, d.precision, d.ckpt_every = 40, 24, 12, 32, 5
    d.tau, d.d = 1.0, 1.0
    d.D_u = (ctypes.c_double * 3)(0.05, 0.0, 0.05)
    d.D_v = (ctypes.c_double * 3)(0.2, 0.0, 0.2)
    d.D_w = (ctypes.c_double * 3)(0.1, 0.0, 0.1)
    d.u_target = ctypes.c_void_p(0x1000)
    d.s = (ctypes.c_double * 7)(*([1.0] * 7))
    d.source_order = 2
    d.ctrl_species = 2
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_arc_workspace_size_and_validation(lib):
    so, mod = lib
    n = ctypes.c_size_t(0)
    assert so.cx3_workspace_size(ctypes.byref(_desc3(mod)), ctypes.byref(n)) == 0
    plane = 40 * 24 + 24  # rounded up to 64
    # at least: 4 population buffers of 27 planes, 3 checkpoint slots of 30 planes, 5 tape steps of 6 planes
    assert n.value >= (4 * 27 + 3 * 30 + 5 * 6) * plane * 4
    n64 = ctypes.c_size_t(0)
    assert so.cx3_workspace_size(ctypes.byref(_desc3(mod, precision=64)), ctypes.byref(n64)) == 0
    assert n64.value > n.value
    bad = [dict(precision=16), dict(nx=2), dict(n_steps=0), dict(d=0.0), dict(source_order=3), dict(aniso=1),
           dict(aniso=2), dict(adv=1), dict(ctrl_species=0), dict(ctrl_species=3), dict(alpha=-1.0),
           dict(u_target=None), dict(chi1=float("nan")), dict(ckpt_every=-1)]
    for kw in bad:
        assert so.cx3_workspace_size(ctypes.byref(_desc3(mod, **kw)), ctypes.byref(n)) == 1, kw
    d = _desc3(mod)
    d.s[2] = 2.0
    assert so.cx3_workspace_size(ctypes.byref(d), ctypes.byref(n)) == 1
    h = ctypes.c_void_p()
    assert so.cx3_create(ctypes.byref(_desc3(mod)), ctypes.c_void_p(0x1001), 1 << 30, None, ctypes.byref(h)) == 2
    assert so.cx3_create(ctypes.byref(_desc3(mod)), ctypes.c_void_p(0x1000), 16, None, ctypes.byref(h)) == 2


def test_d3q19_desc_layout_and_validation(lib, tmp_path):
    """ctypes Desc3D layout equals cx3d_desc of include/cx3d.h; host-side
    validation and workspace sizing of the D3Q19 solver."""
    so, mod = lib
    fields = [f for f, _ in mod.Desc3D._fields_]
    src = tmp_path / "layout3d.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cx3d.h"', "int main(void){",
             'printf("%zu\\n", sizeof(cx3d_desc));']
    lines += [f'printf("%zu\\n", offsetof(cx3d_desc, {f}));' for f in fields]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout3d"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    assert int(out[0]) == ctypes.sizeof(mod.Desc3D)
    for f, off in zip(fields, out[1:]):
        assert getattr(mod.Desc3D, f).offset == int(off), f

    def desc(**kw):
        d = mod.Desc3D()
        d.nx, d.ny, d.nz, d.n_steps, d.precision, d.ckpt_every = 12, 10, 8, 9, 32, 4
        d.tau, d.d_u, d.d_v = 1.0, 1.0, 1.0
        d.D_u = (ctypes.c_double * 6)(0.05, 0, 0, 0.05, 0, 0.05)
        d.D_v = (ctypes.c_double * 6)(0.2, 0, 0, 0.2, 0, 0.2)
        d.u_target = ctypes.c_void_p(0x1000)
        d.s = (ctypes.c_double * 7)(*([1.0] * 7))
        d.source_order = 2
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    n = ctypes.c_size_t(0)
    assert so.cx3d_workspace_size(ctypes.byref(desc()), ctypes.byref(n)) == 0
    plane = 12 * 10 * 8
    assert n.value >= (4 * 38 + 3 * 39 + 4 * 4) * plane * 4
    for kw in (dict(nz=2), dict(precision=16), dict(n_steps=0), dict(d_v=0.0), dict(aniso=1), dict(aniso=2),
               dict(adv=1), dict(adv=3, a=ctypes.c_void_p(8)), dict(alpha=-1.0), dict(u_target=None),
               dict(source_order=0)):
        assert so.cx3d_workspace_size(ctypes.byref(desc(**kw)), ctypes.byref(n)) == 1, kw
    h = ctypes.c_void_p()
    assert so.cx3d_create(ctypes.byref(desc()), ctypes.c_void_p(0x1001), 1 << 30, None, ctypes.byref(h)) == 2
    # a tensor that is not positive definite is refused before any device work
    bad = desc()
    bad.D_u = (ctypes.c_double * 6)(0.05, 0.2, 0, 0.05, 0, 0.05)
    assert so.cx3d_create(ctypes.byref(bad), ctypes.c_void_p(0x1000), 1 << 30, None, ctypes.byref(h)) == 5
