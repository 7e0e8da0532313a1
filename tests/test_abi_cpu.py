"""The C ABI without a GPU: the library builds and loads, exports every entry point that
include/lq.h declares, and its argument checks reject bad calls before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import formats as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lq.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|size_t|char|void)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lq_dslash_apply", "lq_dslash_adjoint", "lq_cg_solve", "lq_cg_workspace_bytes",
                 "lq_last_error", "dslash_apply", "dslash_adjoint", "cg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(lqlib):
    L = lqlib.load()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_field_bytes_match_format_definitions(lqlib):
    for dims in [(2, 2, 2, 2), (4, 6, 2, 8)]:
        for prec in ("f64", "f32", "f16s"):
            for layout in ("lex", "eo"):
                assert lqlib.field_bytes(dims, "spinor", prec, 18, layout) == F.spinor_bytes(dims, prec)
                for fmt in (18, 12, 10):
                    assert lqlib.field_bytes(dims, "gauge", prec, fmt, layout) == F.gauge_bytes(dims, prec, fmt)
    assert lqlib.field_bytes((3, 4, 4, 4), "spinor") == 0
    assert lqlib.field_bytes((4, 4, 4, 4), "gauge", "f32", 11) == 0


def test_workspace_query(lqlib):
    a = lqlib.cg_workspace_bytes((4, 4, 4, 4), "f64")
    b = lqlib.cg_workspace_bytes((8, 8, 8, 8), "f64")
    assert 0 < a < b
    assert lqlib.cg_workspace_bytes((8, 8, 8, 8), "mixed_f16") < lqlib.cg_workspace_bytes((8, 8, 8, 8), "mixed_f32")
    assert lqlib.cg_workspace_bytes((4, 4, 4, 5), "f64") == 0
    assert lqlib.cg_workspace_bytes((8, 8, 8, 8), "f64x") > lqlib.cg_workspace_bytes((8, 8, 8, 8), "f64")
    assert lqlib.load().lq_cg_workspace_bytes((ctypes.c_int32 * 4)(4, 4, 4, 4), 7) == 0


# fake device addresses: the checks below fail before any CUDA call, nothing is dereferenced
P0, P1, P2 = 0x10000, 0x20000000, 0x40000000


def _apply(L, dims, prec=0, fmt=18, layout=0, U=P0, psi=P1, out=P2, m=0.1):
    vp = ctypes.c_void_p
    return L.lq_dslash_apply((ctypes.c_int32 * 4)(*dims), m, prec, fmt, layout, vp(U), vp(psi), vp(out), None)


def test_apply_argument_checks(lqlib):
    L = lqlib.load()
    assert _apply(L, (4, 4, 4, 3)) == -2
    assert "even" in lqlib.last_error()
    assert _apply(L, (0, 4, 4, 4)) == -2
    assert _apply(L, (4096, 4096, 4096, 2)) == -2          # volume beyond 10^8 sites
    assert _apply(L, (100, 100, 100, 102)) == -2
    assert _apply(L, (4, 4, 4, 4), prec=5) == -1
    assert _apply(L, (4, 4, 4, 4), fmt=11) == -1
    assert _apply(L, (4, 4, 4, 4), layout=2) == -1
    assert _apply(L, (4, 4, 4, 4), U=0) == -1
    assert _apply(L, (4, 4, 4, 4), psi=P1 + 8) == -3          # misaligned
    assert _apply(L, (4, 4, 4, 4), out=P1) == -3              # out aliases psi
    assert _apply(L, (4, 4, 4, 4), out=P1 + 4096) == -3       # partial overlap
    assert _apply(L, (4, 4, 4, 4), m=float("nan")) == -1
    assert _apply(L, (4, 4, 4, 4), prec=3, fmt=12) == -1       # FP32-pair fields are 18-real
    assert _apply(L, (4, 4, 4, 4), prec=3, fmt=10) == -1
    assert L.lq_dslash_adjoint((ctypes.c_int32 * 4)(4, 4, 4, 3), 0.1, 0, 18, 0, None, None, None, None) == -2


def test_site_field_bound(lqlib):
    """nrhs * V <= 2^28 per call (32-bit slot indices): 64^3 x 128 takes 8 fields, not 9."""
    L = lqlib.load()
    vp = ctypes.c_void_p
    d = (ctypes.c_int32 * 4)(64, 64, 64, 128)
    apply = lambda n: L.lq_dslash_apply_multi(d, 0.1, 0, 18, 0, n, vp(0), vp(0), vp(0), None)
    assert apply(9) == -1 and "2^28" in lqlib.last_error()
    assert apply(8) == -1 and "NULL" in lqlib.last_error()          # past the bound, stopped at U
    assert lqlib.cg_workspace_bytes((64, 64, 64, 128), "mixed_f32", 4) > 0


def test_hop_and_convert_argument_checks(lqlib):
    L = lqlib.load()
    vp = ctypes.c_void_p
    d = (ctypes.c_int32 * 4)(4, 4, 4, 4)
    assert L.lq_dslash_hop(d, 2, 0, 0.0, 1.0, 0, 18, vp(P0), vp(P1), None, vp(P2), None) == -1
    assert L.lq_dslash_hop(d, 0, 0, 0.0, float("inf"), 0, 18, vp(P0), vp(P1), None, vp(P2), None) == -1
    assert L.lq_dslash_hop(d, 0, 0, 0.0, 1.0, 0, 18, vp(P0), vp(P1), vp(P2 + 16), vp(P2), None) == -3
    assert L.lq_convert_spinor(d, 0, 0, vp(P0), 1, 1, vp(P0), None) == -3
    assert L.lq_convert_gauge(d, 0, 0, vp(P0), 1, 11, 1, vp(P1), None) == -1


def test_cg_argument_checks(lqlib):
    L = lqlib.load()
    vp = ctypes.c_void_p
    d = (ctypes.c_int32 * 4)(4, 4, 4, 4)
    info = lqlib.CgInfo()
    prm = lqlib.CgParams(1e-10, 100, 0, 0.0, 0, 0)
    call = lambda mode=0, p=prm, ws=P2, wsb=1 << 30, x=P1: L.lq_cg_solve(
        d, 0.1, mode, vp(P0), vp(0x30000000), vp(x), ctypes.byref(p), vp(ws), ctypes.c_size_t(wsb),
        ctypes.byref(info), None)
    assert call(mode=9) == -1
    assert call(ws=0) == -5
    assert call(wsb=100) == -5                       # smaller than the workspace query
    assert info.status == -5
    assert call(p=lqlib.CgParams(-1.0, 100, 0, 0.0, 0, 0)) == -1
    assert call(p=lqlib.CgParams(1e-10, 0, 0, 0.0, 0, 0)) == -1
    assert call(p=lqlib.CgParams(1e-10, 10, 0, 1.5, 0, 0)) == -1
    assert call(p=lqlib.CgParams(1e-10, 10, 0, 0.0, 0, 0, -1)) == -1     # max_inner < 0
    assert call(x=0x30000000) == -3                  # x aliases eta
    assert "alias" in lqlib.last_error() or "overlap" in lqlib.last_error()


def test_version(lqlib):
    assert "sm_103a" in lqlib.version()


def _lattices(lqlib, specs):
    """Descriptors with fake, well-separated device addresses (nothing is dereferenced)."""
    arr = (lqlib.Lattice * len(specs))()
    base = 0x100000000
    for i, (dims, nrhs) in enumerate(specs):
        arr[i].dims = (ctypes.c_int32 * 4)(*dims)
        arr[i].nrhs = nrhs
        arr[i].m_q = 0.1
        arr[i].U = base + 0x30000000 * (3 * i)
        arr[i].eta = base + 0x30000000 * (3 * i + 1)
        arr[i].x = base + 0x30000000 * (3 * i + 2)
    return arr


def test_lattices_workspace_query(lqlib):
    L = lqlib.load()
    specs = [((8, 8, 8, 8), 4), ((12, 12, 12, 12), 4), ((16, 16, 16, 32), 4)]
    both = L.lq_cg_workspace_bytes_lattices(3, _lattices(lqlib, specs), 1)
    parts = [L.lq_cg_workspace_bytes_lattices(1, _lattices(lqlib, [s]), 1) for s in specs]
    assert both == sum(parts) and all(p > 0 for p in parts)
    assert L.lq_cg_workspace_bytes_lattices(0, _lattices(lqlib, specs), 1) == 0
    assert L.lq_cg_workspace_bytes_lattices(1, _lattices(lqlib, [((8, 8, 8, 8), 3)]), 1) == 0
    assert L.lq_cg_workspace_bytes_lattices(1, _lattices(lqlib, specs), 9) == 0
    # a lattice costs what the single-lattice solver needs for the same batch, or less
    assert parts[0] <= lqlib.cg_workspace_bytes((8, 8, 8, 8), "mixed_f32", 4)


def test_lattices_argument_checks(lqlib):
    L = lqlib.load()
    vp = ctypes.c_void_p
    specs = [((8, 8, 8, 8), 4), ((12, 12, 12, 12), 2)]
    info = (lqlib.CgInfo * 8)()
    ws = 0x4000000000

    def call(arr, n=None, mode=1, flags=0, wsb=64):
        prm = lqlib.CgParams(1e-10, 100, 0, 0.0, 0, flags)
        return L.lq_cg_solve_lattices(len(arr) if n is None else n, arr, mode, ctypes.byref(prm), vp(ws),
                                      ctypes.c_size_t(wsb), info, None)

    good = _lattices(lqlib, specs)
    assert call(good) == -5                          # workspace smaller than the query
    assert call(good, n=0) == -1
    assert call(good, n=9) == -1
    assert call(good, mode=7) == -1
    assert call(good, flags=lqlib.CG_PROFILE) == -1
    assert call(good, flags=lqlib.CG_NATIVE_F64) == -1
    assert call(good, flags=0x100 | 0x400) == -1     # two block sizes
    assert call(_lattices(lqlib, [((8, 8, 8, 8), 3)])) == -1
    assert call(_lattices(lqlib, [((8, 8, 7, 8), 1)])) == -2
    bad = _lattices(lqlib, specs)
    bad[1].x = bad[0].eta                            # a solution over another lattice's input
    assert call(bad) == -3
    bad = _lattices(lqlib, specs)
    bad[1].x = bad[0].x                              # two solutions in one buffer
    assert call(bad) == -3
    bad = _lattices(lqlib, specs)
    bad[0].U = 0
    assert call(bad) == -1
    bad = _lattices(lqlib, specs)
    bad[0].m_q = float("inf")
    assert call(bad) == -1


def test_noalloc_array_size_against_the_workspace_query(lqlib):
    """The fixed no-allocation scratch (64 MiB) holds a 12^4 solve in every mode and a 16^4
    solve in none, as the header states."""
    L = lqlib.load()
    L.lq_cg_noalloc_max_workspace_bytes.restype = ctypes.c_size_t
    cap = L.lq_cg_noalloc_max_workspace_bytes()
    assert cap == 64 << 20
    for mode in ("f64", "f64x", "mixed_f32", "mixed_f16", "mixed_i32"):
        assert 0 < lqlib.cg_workspace_bytes((12, 12, 12, 12), mode) <= cap, mode
        assert lqlib.cg_workspace_bytes((16, 16, 16, 16), mode) > cap, mode


def test_checked_build_exports_every_declared_symbol(lqlib):
    """The bounds-checked debug variant is the same library with checks compiled in: it
    builds (nvcc cross-compiles here) and exports the same entry points."""
    from paper_1904_08616_gb300 import build as B
    path = B.build(checked=True)
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_structs_match_the_header(tmp_path):
    """The binding's ctypes mirrors of lq_cg_params, lq_cg_info and lq_lattice have the C
    structs' size and every field's offset, as a C compiler lays them out from include/lq.h."""
    import shutil
    import subprocess
    import paper_1904_08616_gb300 as lq
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"lq_cg_params": lq.CgParams, "lq_cg_info": lq.CgInfo, "lq_lattice": lq.Lattice}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lq.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_compute_calls_refuse_host_tensors(lqlib):
    """No CPU fallback: every compute call of the binding refuses host (CPU) tensors with an
    error before anything runs, rather than computing on the host."""
    torch = pytest.importorskip("torch")
    dims = (4, 4, 4, 4)
    U = torch.zeros(lqlib.field_bytes(dims, "gauge", "f64", 18) // 8, dtype=torch.float64)
    psi = torch.zeros(lqlib.field_bytes(dims, "spinor", "f64") // 8, dtype=torch.float64)
    psi2 = torch.zeros(2 * psi.numel(), dtype=torch.float64)
    Ueo = torch.zeros(lqlib.field_bytes(dims, "gauge", "f32", 12, "eo") // 4, dtype=torch.float32)
    half = torch.zeros(lqlib.field_bytes(dims, "spinor", "f32") // 8, dtype=torch.float32)
    calls = [
        lambda: lqlib.dslash_apply(dims, 0.1, U, psi),
        lambda: lqlib.dslash_adjoint(dims, 0.1, U, psi),
        lambda: lqlib.dslash_apply_multi(dims, 0.1, 2, U, psi2),
        lambda: lqlib.dslash_adjoint_multi(dims, 0.1, 2, U, psi2),
        lambda: lqlib.dslash_hop(dims, 0, Ueo, half, prec="f32", link_fmt=12),
        lambda: lqlib.link_grad(dims, psi, psi),
        lambda: lqlib.convert_spinor(dims, psi),
        lambda: lqlib.convert_spinor_multi(dims, 2, psi2),
        lambda: lqlib.convert_gauge(dims, U),
        lambda: lqlib.cg_solve(dims, 0.1, U, psi, mode="mixed_f16"),
        lambda: lqlib.cg_solve_multi(dims, 0.1, 2, U, psi2, mode="mixed_f32"),
        lambda: lqlib.cg_solve_schur(dims, 0.1, U, psi, mode="mixed_f32"),
        lambda: lqlib.cg_solve_lattices([{"dims": dims, "m_q": 0.1, "U": U, "eta": psi}]),
    ]
    for i, call in enumerate(calls):
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()
