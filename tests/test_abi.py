"""CPU checks of the boundary: libmpcd.so loads and exports every function that
include/mpcd.h declares; the binding's structures match the header's sizes.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpcd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mpcd_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_10187_gb300 import _build
    _build.build()
    import paper_1801_10187_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mpcd_create", "mpcd_set_state", "mpcd_step", "mpcd_get_state",
                 "mpcd_observables", "mpcd_profile", "mpcd_destroy", "mpcd_last_error",
                 "mpcd_batch_create", "mpcd_batch_add", "mpcd_batch_step", "mpcd_batch_remove"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def declared_arity():
    """Number of parameters of each function the header declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"\b(mpcd_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header(lib):
    """Every function the binding gives argument types to takes as many
    arguments as the header declares (a stale binding would pass garbage)."""
    arity = declared_arity()
    assert "mpcd_tune" in arity and arity["mpcd_tune"] == 7
    checked = 0
    for name, n in arity.items():
        fn = getattr(lib, name)
        if fn.argtypes is not None:
            assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
            checked += 1
    assert checked >= 20


def _c_layout(struct, fields, tmp_path):
    prog = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){",
             f'printf("size %zu\\n", sizeof({struct}));']
    for f in fields:
        lines.append(f'printf("{f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["return 0;}"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(prog)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.strip().splitlines())}


@pytest.mark.parametrize("cname,pyname", [("mpcd_params", "_Params"), ("mpcd_obs", "_Obs")])
def test_struct_layouts_match_header(lib, cname, pyname, tmp_path):
    import paper_1801_10187_gb300 as pkg
    cls = getattr(pkg, pyname)
    names = [f[0] for f in cls._fields_]
    c = _c_layout(cname, names, tmp_path)
    assert c["size"] == ctypes.sizeof(cls)
    for nm in names:
        assert c[nm] == getattr(cls, nm).offset, nm


def test_error_reporting_without_gpu_work(lib):
    import paper_1801_10187_gb300 as pkg
    # invalid parameters are rejected before any device call
    p = pkg.make_params(n=(0, 4, 4))
    ctx = ctypes.c_void_p()
    rc = lib.mpcd_create(ctypes.byref(p), None, ctypes.byref(ctx))
    assert rc == pkg.MPCD_EINVAL
    assert b"n[k]" in lib.mpcd_last_error()
    p = pkg.make_params(n=(4, 4, 4))
    p.a = 0.5
    assert lib.mpcd_create(ctypes.byref(p), None, ctypes.byref(ctx)) == pkg.MPCD_EINVAL
    assert lib.mpcd_box_footprint(ctypes.byref(pkg.make_params(n=(10, 10, 10))), 5000) > 0
    assert lib.mpcd_step(None, 1) == pkg.MPCD_EINVAL
