"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/l2xfer.h with struct layouts that match the binding.
(No compute calls: these run without a GPU.)"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1810_13046_gb300 as l2x

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "l2xfer.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(l2x_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = l2x.load_library()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", l2x.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (l2x_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "l2xfer.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(l2x_grid), sizeof(l2x_mesh),"
        " sizeof(l2x_opts), sizeof(l2x_info), offsetof(l2x_info, cg_residual), offsetof(l2x_opts, force_scale));"
        "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(l2x._Grid), ctypes.sizeof(l2x._Mesh), ctypes.sizeof(l2x._Opts),
                    ctypes.sizeof(l2x._Info), l2x._Info.cg_residual.offset, l2x._Opts.force_scale.offset]


def test_status_strings_and_defaults():
    lib = l2x.load_library()
    for s in range(10):
        assert lib.l2x_status_string(s)
    o = l2x._Opts()
    lib.l2x_default_opts(ctypes.byref(o))
    assert (o.path, o.precision, o.cg_max_iter, o.force_mode) == (l2x.FUSED, l2x.FP64, 200, l2x.DUAL)
    assert o.cg_rtol == 1e-13 and o.force_scale == 1.0


def test_invalid_arguments_are_rejected_without_a_gpu():
    """Argument validation happens on the host before any CUDA call."""
    lib = l2x.load_library()
    g = l2x._Grid()
    g.dim = 4
    m = l2x._Mesh()
    m.dim = 4
    h = ctypes.c_void_p()
    st = lib.l2x_build_coupling(ctypes.byref(g), ctypes.byref(m), None, None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"dim" in lib.l2x_last_error()
    assert lib.l2x_destroy(None) == 0
    assert lib.l2x_set_step_work_shape(None, 64) == 1


def test_bad_multiplier_space_is_rejected_without_a_gpu():
    lib = l2x.load_library()
    g = l2x._Grid()
    g.dim, g.staggered = 2, 0
    for k in range(2):
        g.ncell[k] = 4
        g.h[k] = 0.25
    m = l2x._Mesh()
    m.dim, m.n_nodes, m.n_elems = 2, 3, 1
    m.coords = m.elems = 16  # never dereferenced: validation fails first
    o = l2x._Opts()
    lib.l2x_default_opts(ctypes.byref(o))
    assert o.multiplier == l2x.STANDARD_BASIS
    o.multiplier = 7
    h = ctypes.c_void_p()
    assert lib.l2x_build_coupling(ctypes.byref(g), ctypes.byref(m), ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert b"multiplier" in lib.l2x_last_error()


def test_stretched_axis_is_validated_without_a_gpu():
    """A stretched node array that does not increase strictly is rejected before any CUDA call."""
    import numpy as np
    lib = l2x.load_library()
    grid = l2x.Grid(2, (4, 4), (0.25, 0.25), (0.0, 0.0), False,
                    (np.array([0.0, 0.2, 0.5, 0.5, 1.0]), np.linspace(0.0, 1.0, 5)))
    g, keep = l2x._as_cgrid(grid)
    m = l2x._Mesh()
    m.dim, m.n_nodes, m.n_elems = 2, 3, 1
    m.coords = m.elems = 16  # never dereferenced: validation fails first
    h = ctypes.c_void_p()
    assert lib.l2x_build_coupling(ctypes.byref(g), ctypes.byref(m), None, None, ctypes.byref(h)) == 1
    assert b"increase" in lib.l2x_last_error()


_NULL_SWEEP = r'''
import ctypes, sys
import paper_1810_13046_gb300 as l2x
lib = l2x.load_library()
names = sys.argv[1].split(",")
free_ok = {"l2x_destroy", "l2x_graph_destroy"}
not_taking_a_handle = {"l2x_kernel_launch_count", "l2x_status_string", "l2x_last_error", "l2x_default_opts",
                       "l2x_build_coupling"}
checked = 0
for n in names:
    fn = getattr(lib, n)
    if n in not_taking_a_handle or fn.argtypes is None:
        continue
    args = []
    for t in fn.argtypes:
        if t in (ctypes.c_double,):
            args.append(0.0)
        elif t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64):
            args.append(0)
        else:
            args.append(None)
    st = fn(*args)
    want = 0 if n in free_ok else 1
    if st != want:
        print("BAD", n, st)
        sys.exit(1)
    checked += 1
print("checked", checked)
'''


def test_every_entry_point_rejects_null_arguments_without_a_gpu():
    """Every call that takes a handle, a graph or device norms returns
    L2X_EINVAL for NULL on the host (the destroy calls accept NULL), so a
    caller's mistake is a status, never a crash.  Runs in a child process."""
    l2x.load_library()
    names = ",".join(_declared())
    out = subprocess.run([__import__("sys").executable, "-c", _NULL_SWEEP, names], capture_output=True, text=True,
                         cwd=ROOT, timeout=300)
    assert out.returncode == 0, (out.stdout[-2000:], out.stderr[-2000:])
    assert int(out.stdout.split()[-1]) >= 25
