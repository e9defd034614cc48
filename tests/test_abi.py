"""The C-ABI library loads and exports every entry point include/lbkm.h declares,
and the ctypes structures of the binding have the header's layout. CPU only: no
call here touches a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbkm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1411_6697_gb300 import build
    build.build()
    from paper_1411_6697_gb300 import lbkm
    return lbkm.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbkm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    from paper_1411_6697_gb300 import lbkm
    assert sorted(lbkm.EXPORTED) == names


def test_struct_layout_matches_header(lib):
    from paper_1411_6697_gb300 import lbkm
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbkm.h"
#define F(s, m) printf(#m " %zu\n", offsetof(s, m));
int main(void) {
  printf("params %zu\n", sizeof(lbkm_params));
  printf("tne %zu\n", sizeof(lbkm_tne_global));
  printf("gradout %zu\n", sizeof(lbkm_grad_out));
  F(lbkm_grad_out, domega1) F(lbkm_grad_out, drho0) F(lbkm_grad_out, domega2)
  F(lbkm_params, gamma) F(lbkm_params, orbit_kind) F(lbkm_params, orbit_speed)
  F(lbkm_params, S) F(lbkm_params, Q) F(lbkm_params, T_ig) F(lbkm_params, dt)
  F(lbkm_params, bc_x) F(lbkm_params, tne_capacity) F(lbkm_params, time_scheme)
  F(lbkm_params, collision) F(lbkm_params, alloc) F(lbkm_params, free) F(lbkm_params, alloc_ctx)
  F(lbkm_tne_global, d_sum) F(lbkm_tne_global, step)
  return 0; }
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "l")
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        out = dict(line.split() for line in subprocess.check_output([exe]).decode().splitlines())
    assert int(out["params"]) == ctypes.sizeof(lbkm.Params)
    assert int(out["tne"]) == ctypes.sizeof(lbkm.TneGlobal)
    for m in ("gamma", "orbit_kind", "orbit_speed", "S", "Q", "T_ig", "dt", "bc_x",
              "tne_capacity", "time_scheme", "collision", "alloc", "free", "alloc_ctx"):
        assert int(out[m]) == getattr(lbkm.Params, m).offset, m
    assert int(out["d_sum"]) == lbkm.TneGlobal.d_sum.offset
    assert int(out["step"]) == lbkm.TneGlobal.step.offset
    assert int(out["gradout"]) == ctypes.sizeof(lbkm.GradOut)
    for m in ("domega1", "drho0", "domega2"):
        assert int(out[m]) == getattr(lbkm.GradOut, m).offset, m


def test_default_params_are_host_only(lib):
    from paper_1411_6697_gb300 import lbkm
    p = lbkm.default_params(nx=10, ny=1)
    assert p.orbit_kind[:] == [0, 1, 0, 1]
    assert list(p.orbit_speed) == [2.7, 2.2, 1.2, 1.0]
    assert p.S[5] == 1e5 and p.tne_capacity == 1 and p.precision == lbkm.F64
    assert lbkm.version() == 100


def test_missing_library_fails_loudly(monkeypatch):
    from paper_1411_6697_gb300 import lbkm
    monkeypatch.setattr(lbkm, "_lib", None)
    monkeypatch.setattr(lbkm, "LIB_PATH", "/nonexistent/libpaper_lbkm.so")
    with pytest.raises(ImportError):
        lbkm.load()


HEADER24 = os.path.join(ROOT, "include", "lbkm24.h")


def test_d2v24_symbols_and_layout(lib):
    """include/lbkm24.h (the paper's D2V24): every declared call is exported and listed by
    the binding, and lbkm24_params / lbkm24_tne_global have the ctypes layout."""
    from paper_1411_6697_gb300 import lbkm
    src = re.sub(r"/\*.*?\*/", "", open(HEADER24).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(lbkm24_[a-z_]+)\s*\(", src)))
    assert len(names) == 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbkm.EXPORTED24) == names
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbkm24.h"
#define F(s, m) printf(#m " %zu\n", offsetof(s, m));
int main(void) {
  printf("params %zu\n", sizeof(lbkm24_params));
  printf("tne %zu\n", sizeof(lbkm24_tne_global));
  F(lbkm24_params, gamma) F(lbkm24_params, v) F(lbkm24_params, eta) F(lbkm24_params, S)
  F(lbkm24_params, Q) F(lbkm24_params, dt) F(lbkm24_params, bc_x) F(lbkm24_params, tne_capacity)
  F(lbkm24_params, collision)
  F(lbkm24_tne_global, d_sum) F(lbkm24_tne_global, step)
  return 0; }
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "l")
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER24), c, "-o", exe])
        out = dict(line.split() for line in subprocess.check_output([exe]).decode().splitlines())
    assert int(out["params"]) == ctypes.sizeof(lbkm.Params24)
    assert int(out["tne"]) == ctypes.sizeof(lbkm.TneGlobal24)
    for m in ("gamma", "v", "eta", "S", "Q", "dt", "bc_x", "tne_capacity", "collision"):
        assert int(out[m]) == getattr(lbkm.Params24, m).offset, m
    assert int(out["d_sum"]) == lbkm.TneGlobal24.d_sum.offset
    assert int(out["step"]) == lbkm.TneGlobal24.step.offset
    p = lbkm.default_params24(nx=8, ny=1)
    assert list(p.v) == [2.7, 2.2, 1.2] and list(p.eta) == [5.0, 3.0, 1.1]
    assert p.S[4] == 1e4 and p.S[7] == 1e5 and p.dx == 2e-4 and p.dt == 5e-6


def test_d2v24_params_from_keywords(lib):
    """default_params24 maps the keyword forms (v, eta, S broadcast, bc, sides) onto the
    C structure; no GPU involved."""
    from paper_1411_6697_gb300 import lbkm
    sides = [(3, 1.0, 2.0, 0.0, 0.5, 0.0), (1, 1.0, 0.0, 0.0, 1.0, 0.0),
             (4, 1.0, 0.0, 0.0, 1.0, 0.0), (3, 1.25, 1.9, -0.173205, 0.56, 0.2)]
    p = lbkm.default_params24(nx=300, ny=100, v=(1.0, 2.7, 2.9), eta=(1.0, 2.9, 0.96),
                              S=1e5, bc=(5, 5), sides=sides, collision=1)
    assert list(p.v) == [1.0, 2.7, 2.9] and list(p.eta) == [1.0, 2.9, 0.96]
    assert list(p.S) == [1e5] * 24 and (p.bc_x, p.bc_y) == (5, 5) and p.collision == 1
    assert list(p.side_bc) == [3, 1, 4, 3]
    assert p.side_uy[3] == -0.173205 and p.side_lam[3] == 0.2 and p.side_T[0] == 0.5
