"""Python binding of liblq, the GB300 Wilson-Dirac library (arXiv 1904.08616).

Argument marshalling only: every operation runs in the library's CUDA kernels through the
C ABI of include/lq.h.  PyTorch provides device memory and streams.  There is no CPU
fallback: if liblq.so cannot be built or loaded, every call raises.

Fields are passed as CUDA tensors whose bytes hold the stored field (any dtype; a
complex128 tensor of shape (V, 4, 3) is exactly an F64 LEX spinor, (V, 4, 3, 3) an F64
LEX 18-real gauge field).  Precisions: "f64", "f32", "f16s", "f64x" (FP64-class values as
FP32 pairs), "i32s"; layouts: "lex", "eo"; link formats: 18, 12, 10.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

__all__ = [
    "LqError", "load", "lib_path", "PREC", "LAYOUT", "CG_MODE",
    "field_bytes", "dslash_apply", "dslash_adjoint", "dslash_apply_multi", "dslash_adjoint_multi",
    "dslash_hop", "link_grad", "convert_spinor", "convert_spinor_multi", "convert_gauge", "cg_workspace_bytes",
    "cg_solve", "cg_solve_multi", "cg_workspace_bytes_lattices", "cg_solve_lattices",
    "cg_workspace_bytes_schur", "cg_solve_schur",
    "last_error", "version", "bounds_violations", "checked",
]

PREC = {"f64": 0, "f32": 1, "f16s": 2, "f64x": 3, "i32s": 4}
LAYOUT = {"lex": 0, "eo": 1}
CG_MODE = {"f64": 0, "mixed_f32": 1, "mixed_f16": 2, "f64x": 3, "mixed_i32": 4}
CG_PROFILE, CG_NATIVE_F64, CG_LINK18, CG_AUTOTUNE, CG_NO_GRAPH, CG_LINK10 = 1, 2, 4, 8, 16, 32
CG_RHS_BLOCK_1, CG_RHS_BLOCK_2, CG_RHS_BLOCK_4 = 0x1000, 0x2000, 0x4000
CG_LATTICE_OWN_CYCLES = 0x800
STATUS = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_ARG", -2: "ERR_DIMS", -3: "ERR_ALIGN",
          -4: "ERR_CUDA", -5: "ERR_WORKSPACE", -6: "ERR_NONFINITE", -7: "ERR_BREAKDOWN"}


class LqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class CgParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("max_cycles", ctypes.c_int32),
                ("delta", ctypes.c_double), ("chunk", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("max_inner", ctypes.c_int32)]


class CgInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("high_applies", ctypes.c_int32), ("true_rel_resid", ctypes.c_double),
                ("eta_norm", ctypes.c_double), ("launches", ctypes.c_int32), ("block", ctypes.c_int32),
                ("kernel_ms", ctypes.c_double * 4), ("kernel_calls", ctypes.c_int32 * 4), ("rhs_block", ctypes.c_int32)]


class Lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("nrhs", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("m_q", ctypes.c_double), ("U", ctypes.c_void_p), ("eta", ctypes.c_void_p), ("x", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None
_Dims = ctypes.c_int32 * 4
_vp = ctypes.c_void_p


def checked() -> bool:
    """True when this process uses the bounds-checked debug library (environment variable
    LQ_LIB_VARIANT=checked): every field access of the kernels is checked against its field
    and counted (bounds_violations)."""
    return os.environ.get("LQ_LIB_VARIANT", "") == "checked"


def lib_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load(build_if_missing: bool = True):
    """Load liblq.so (compiling it with nvcc first if it is missing or stale), or the
    bounds-checked liblq_checked.so when LQ_LIB_VARIANT=checked."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if build_if_missing:
            _build.build(checked=checked())
        if not os.path.exists(path):
            raise LqError(-4, f"{path} is missing; run paper_1904_08616_gb300.build")
        L = ctypes.CDLL(path)
        i32, f64 = ctypes.c_int32, ctypes.c_double
        L.lq_field_bytes.argtypes = [_Dims, i32, i32, i32, i32]
        L.lq_field_bytes.restype = ctypes.c_size_t
        for name in ("lq_dslash_apply", "lq_dslash_adjoint"):
            fn = getattr(L, name)
            fn.argtypes = [_Dims, f64, i32, i32, i32, _vp, _vp, _vp, _vp]
            fn.restype = ctypes.c_int
        L.lq_dslash_hop.argtypes = [_Dims, i32, i32, f64, f64, i32, i32, _vp, _vp, _vp, _vp, _vp]
        L.lq_dslash_hop.restype = ctypes.c_int
        L.lq_halo_face_bytes.argtypes = [_Dims]
        L.lq_halo_face_bytes.restype = ctypes.c_size_t
        L.lq_halo_pack.argtypes = [_Dims, i32, _vp, _vp, _vp, _vp, _vp]
        L.lq_halo_pack.restype = ctypes.c_int
        L.lq_halo_dslash.argtypes = [_Dims, f64, i32, _vp, _vp, _vp, _vp, _vp, _vp]
        L.lq_halo_dslash.restype = ctypes.c_int
        L.lq_link_grad.argtypes = [_Dims, _vp, _vp, f64, i32, _vp, _vp]
        L.lq_link_grad.restype = ctypes.c_int
        L.lq_convert_spinor.argtypes = [_Dims, i32, i32, _vp, i32, i32, _vp, _vp]
        L.lq_convert_spinor.restype = ctypes.c_int
        L.lq_convert_spinor_multi.argtypes = [_Dims, i32, i32, i32, _vp, i32, i32, _vp, _vp]
        L.lq_convert_spinor_multi.restype = ctypes.c_int
        for name in ("lq_dslash_apply_multi", "lq_dslash_adjoint_multi"):
            fn = getattr(L, name)
            fn.argtypes = [_Dims, f64, i32, i32, i32, i32, _vp, _vp, _vp, _vp]
            fn.restype = ctypes.c_int
        L.lq_cg_workspace_bytes_multi.argtypes = [_Dims, i32, i32]
        L.lq_cg_workspace_bytes_multi.restype = ctypes.c_size_t
        L.lq_cg_solve_multi.argtypes = [_Dims, f64, i32, i32, _vp, _vp, _vp, ctypes.POINTER(CgParams), _vp,
                                        ctypes.c_size_t, ctypes.POINTER(CgInfo), _vp]
        L.lq_cg_solve_multi.restype = ctypes.c_int
        L.lq_cg_workspace_bytes_schur.argtypes = [_Dims, i32, i32]
        L.lq_cg_workspace_bytes_schur.restype = ctypes.c_size_t
        L.lq_cg_solve_schur.argtypes = [_Dims, f64, i32, i32, _vp, _vp, _vp, ctypes.POINTER(CgParams), _vp,
                                        ctypes.c_size_t, ctypes.POINTER(CgInfo), _vp]
        L.lq_cg_solve_schur.restype = ctypes.c_int
        L.lq_cg_workspace_bytes_lattices.argtypes = [i32, ctypes.POINTER(Lattice), i32]
        L.lq_cg_workspace_bytes_lattices.restype = ctypes.c_size_t
        L.lq_cg_solve_lattices.argtypes = [i32, ctypes.POINTER(Lattice), i32, ctypes.POINTER(CgParams), _vp,
                                           ctypes.c_size_t, ctypes.POINTER(CgInfo), _vp]
        L.lq_cg_solve_lattices.restype = ctypes.c_int
        L.lq_convert_gauge.argtypes = [_Dims, i32, i32, _vp, i32, i32, i32, _vp, _vp]
        L.lq_convert_gauge.restype = ctypes.c_int
        L.lq_cg_workspace_bytes.argtypes = [_Dims, i32]
        L.lq_cg_workspace_bytes.restype = ctypes.c_size_t
        L.lq_cg_solve.argtypes = [_Dims, f64, i32, _vp, _vp, _vp, ctypes.POINTER(CgParams), _vp,
                                  ctypes.c_size_t, ctypes.POINTER(CgInfo), _vp]
        L.lq_cg_solve.restype = ctypes.c_int
        L.lq_bounds_violations.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        L.lq_bounds_violations.restype = ctypes.c_longlong
        L.lq_last_error.restype = ctypes.c_char_p
        L.lq_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def bounds_violations():
    """(count, first slot) of the field accesses the bounds-checked library skipped since the
    last call (waits for the device); count is -1 with the normal library."""
    first = ctypes.c_ulonglong(0)
    n = int(load().lq_bounds_violations(ctypes.byref(first)))
    return n, (int(first.value) if n > 0 else None)


def last_error() -> str:
    return load().lq_last_error().decode()


def version() -> str:
    return load().lq_version().decode()


def _check(status: int):
    if status < 0:
        raise LqError(status, last_error())
    return status


def _dims(dims):
    d = [int(v) for v in dims]
    if len(d) != 4:
        raise ValueError("dims must have four extents")
    return _Dims(*d)


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def _layout(l):
    return LAYOUT[l] if isinstance(l, str) else int(l)


def _stream(stream):
    import torch
    if stream is None:
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _ptr(t, nbytes: int | None = None, name: str = "tensor"):
    """Device pointer of a CUDA tensor, checking that it is contiguous and large enough."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.is_conj() or t.is_neg():
        raise ValueError(f"{name} is a lazy conjugate/negative view: call resolve_conj()/resolve_neg() first")
    if nbytes is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{name} holds {t.numel() * t.element_size()} bytes, {nbytes} needed")
    return _vp(t.data_ptr())


def field_bytes(dims, kind: str, prec="f64", link_fmt: int = 18, layout="lex") -> int:
    k = {"spinor": 0, "gauge": 1}[kind]
    return int(load().lq_field_bytes(_dims(dims), k, _prec(prec), int(link_fmt), _layout(layout)))


def _empty_bytes(n, like):
    import torch
    return torch.empty(n, dtype=torch.uint8, device=like.device)


def _apply(fn, dims, m_q, U, psi, out, prec, link_fmt, layout, stream):
    sb = field_bytes(dims, "spinor", prec, link_fmt, layout)
    gb = field_bytes(dims, "gauge", prec, link_fmt, layout)
    if out is None:
        out = _empty_bytes(sb, psi)
    _check(fn(_dims(dims), float(m_q), _prec(prec), int(link_fmt), _layout(layout),
              _ptr(U, gb, "U"), _ptr(psi, sb, "psi"), _ptr(out, sb, "out"), _stream(stream)))
    return out


def dslash_apply(dims, m_q, U, psi, out=None, prec="f64", link_fmt=18, layout="lex", stream=None):
    """out = D psi (Eq. 1).  Returns out (a new uint8 tensor when out is None)."""
    return _apply(load().lq_dslash_apply, dims, m_q, U, psi, out, prec, link_fmt, layout, stream)


def dslash_adjoint(dims, m_q, U, psi, out=None, prec="f64", link_fmt=18, layout="lex", stream=None):
    """out = D^dag psi."""
    return _apply(load().lq_dslash_adjoint, dims, m_q, U, psi, out, prec, link_fmt, layout, stream)


def _apply_multi(fn, dims, m_q, nrhs, U, psi, out, prec, link_fmt, layout, stream):
    sb = field_bytes(dims, "spinor", prec, link_fmt, layout) * int(nrhs)
    gb = field_bytes(dims, "gauge", prec, link_fmt, layout)
    if out is None:
        out = _empty_bytes(sb, psi)
    _check(fn(_dims(dims), float(m_q), _prec(prec), int(link_fmt), _layout(layout), int(nrhs),
              _ptr(U, gb, "U"), _ptr(psi, sb, "psi"), _ptr(out, sb, "out"), _stream(stream)))
    return out


def dslash_apply_multi(dims, m_q, nrhs, U, psi, out=None, prec="f64", link_fmt=18, layout="lex", stream=None):
    """out_r = D psi_r for nrhs fields (LEX: stacked fields; EO: interleaved per site)."""
    return _apply_multi(load().lq_dslash_apply_multi, dims, m_q, nrhs, U, psi, out, prec, link_fmt, layout, stream)


def dslash_adjoint_multi(dims, m_q, nrhs, U, psi, out=None, prec="f64", link_fmt=18, layout="lex", stream=None):
    """out_r = D^dag psi_r for nrhs fields."""
    return _apply_multi(load().lq_dslash_adjoint_multi, dims, m_q, nrhs, U, psi, out, prec, link_fmt, layout,
                        stream)


def dslash_hop(dims, out_parity, U, psi_other, out=None, a=0.0, b=1.0, y=None, dagger=False,
               prec="f64", link_fmt=18, stream=None):
    """out_p = a y_p + b H_{p,1-p} psi_{1-p} on EO half fields, H = the 1/2 sum_mu of Eq. (1)."""
    hb = field_bytes(dims, "spinor", prec) // 2
    gb = field_bytes(dims, "gauge", prec, link_fmt, "eo")
    if out is None:
        out = _empty_bytes(hb, psi_other)
    _check(load().lq_dslash_hop(_dims(dims), int(out_parity), int(bool(dagger)), float(a), float(b),
                                _prec(prec), int(link_fmt), _ptr(U, gb, "U"), _ptr(psi_other, hb, "psi_other"),
                                _ptr(y, hb, "y"), _ptr(out, hb, "out"), _stream(stream)))
    return out


def link_grad(dims, g, psi, out=None, scale=1.0, accumulate=False, stream=None):
    """Gradient of Re <g, D psi> with respect to the links (F64 LEX fields; out is an F64 LEX
    18-real gauge field, written as scale * G or accumulated into)."""
    sb = field_bytes(dims, "spinor", "f64")
    gb = field_bytes(dims, "gauge", "f64", 18, "lex")
    if out is None:
        out = _empty_bytes(gb, psi)
    _check(load().lq_link_grad(_dims(dims), _ptr(g, sb, "g"), _ptr(psi, sb, "psi"), float(scale),
                               int(bool(accumulate)), _ptr(out, gb, "out"), _stream(stream)))
    return out


def convert_spinor(dims, src, src_prec="f64", src_layout="lex", dst=None, dst_prec="f32", dst_layout="eo",
                   stream=None):
    sb = field_bytes(dims, "spinor", src_prec)
    db = field_bytes(dims, "spinor", dst_prec)
    if dst is None:
        dst = _empty_bytes(db, src)
    _check(load().lq_convert_spinor(_dims(dims), _prec(src_prec), _layout(src_layout), _ptr(src, sb, "src"),
                                    _prec(dst_prec), _layout(dst_layout), _ptr(dst, db, "dst"), _stream(stream)))
    return dst


def convert_spinor_multi(dims, nrhs, src, src_prec="f64", src_layout="lex", dst=None, dst_prec="f32",
                         dst_layout="eo", stream=None):
    sb = field_bytes(dims, "spinor", src_prec) * int(nrhs)
    db = field_bytes(dims, "spinor", dst_prec) * int(nrhs)
    if dst is None:
        dst = _empty_bytes(db, src)
    _check(load().lq_convert_spinor_multi(_dims(dims), int(nrhs), _prec(src_prec), _layout(src_layout),
                                          _ptr(src, sb, "src"), _prec(dst_prec), _layout(dst_layout),
                                          _ptr(dst, db, "dst"), _stream(stream)))
    return dst


def convert_gauge(dims, src, src_prec="f64", src_layout="lex", dst=None, dst_prec="f32", dst_fmt=12,
                  dst_layout="eo", stream=None):
    sb = field_bytes(dims, "gauge", src_prec, 18)
    db = field_bytes(dims, "gauge", dst_prec, dst_fmt)
    if dst is None:
        dst = _empty_bytes(db, src)
    _check(load().lq_convert_gauge(_dims(dims), _prec(src_prec), _layout(src_layout), _ptr(src, sb, "src"),
                                   _prec(dst_prec), int(dst_fmt), _layout(dst_layout), _ptr(dst, db, "dst"),
                                   _stream(stream)))
    return dst


def cg_workspace_bytes(dims, mode="f64", nrhs=1) -> int:
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    return int(load().lq_cg_workspace_bytes_multi(_dims(dims), m, int(nrhs)))


def cg_solve(dims, m_q, U, eta, x=None, mode="f64", tol=1e-10, max_iter=100000, max_cycles=0, delta=0.0,
             chunk=0, max_inner=0, workspace=None, stream=None, profile=False, native_f64=False, link18=False, link10=False, graph=True):
    """Solve D^dag D x = eta (Algorithm 1).  U: F64 LEX 18-real links, eta / x: F64 LEX spinors.

    x (if given) is the starting guess and receives the solution.  Returns (x, info, status)
    where info is a dict of the solver statistics; raises LqError on errors (status < 0).
    mode: "f64", "f64x", "mixed_f32", "mixed_f16" or "mixed_i32"; delta <= 0 takes the mode's
    default inner reduction per cycle; max_inner caps the inner iterations of one cycle
    (0: 1000).  profile=True times the solver's kernels with CUDA
    events (host-driven cycles); graph=False drives the cycles from the host instead of
    running the whole solve's cycles in one CUDA graph launch; native_f64,
    link18 and link10 select native FP64 outer arithmetic, 18-real and 10-real inner links
    (mixed modes; link10 with the FP32-pair outer loop only).
    """
    import torch
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    sb = field_bytes(dims, "spinor", "f64")
    gb = field_bytes(dims, "gauge", "f64", 18)
    if x is None:
        x = torch.zeros_like(eta)
    wb = cg_workspace_bytes(dims, m)
    if workspace is None:
        workspace = _empty_bytes(wb, eta)
    flags = (CG_PROFILE if profile else 0) | (CG_NATIVE_F64 if native_f64 else 0) | (CG_LINK18 if link18 else 0) \
        | (CG_LINK10 if link10 else 0) | (0 if graph else CG_NO_GRAPH)
    prm = CgParams(float(tol), int(max_iter), int(max_cycles), float(delta), int(chunk), flags, int(max_inner))
    info = CgInfo()
    st = load().lq_cg_solve(_dims(dims), float(m_q), m, _ptr(U, gb, "U"), _ptr(eta, sb, "eta"),
                            _ptr(x, sb, "x"), ctypes.byref(prm), _ptr(workspace, wb, "workspace"),
                            ctypes.c_size_t(workspace.numel() * workspace.element_size()),
                            ctypes.byref(info), _stream(stream))
    _check(st)
    return x, _info_dict(info), st


def cg_solve_multi(dims, m_q, nrhs, U, eta, x=None, mode="f64", tol=1e-10, max_iter=100000, max_cycles=0,
                   delta=0.0, chunk=0, max_inner=0, workspace=None, stream=None, profile=False, native_f64=False, link18=False, link10=False,
                   graph=True, rhs_block=None, autotune=False):
    """nrhs independent solves D^dag D x_r = eta_r sharing the links (eta, x: nrhs stacked FP64
    LEX fields).  rhs_block (1, 2 or 4; None: the library's default) sets how many right-hand
    sides one thread of the inner stencil kernels serves; autotune (with rhs_block None) lets
    the library choose it by timing (info["rhs_block"] reports the choice).  Returns (x,
    [info per right-hand side], status)."""
    import torch
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    n = int(nrhs)
    sb = field_bytes(dims, "spinor", "f64") * n
    gb = field_bytes(dims, "gauge", "f64", 18)
    if x is None:
        x = torch.zeros_like(eta)
    wb = cg_workspace_bytes(dims, m, n)
    if workspace is None:
        workspace = _empty_bytes(wb, eta)
    flags = (CG_PROFILE if profile else 0) | (CG_NATIVE_F64 if native_f64 else 0) | (CG_LINK18 if link18 else 0) \
        | (CG_LINK10 if link10 else 0) | (0 if graph else CG_NO_GRAPH) | (CG_AUTOTUNE if autotune else 0)
    if rhs_block is not None:
        flags |= {1: CG_RHS_BLOCK_1, 2: CG_RHS_BLOCK_2, 4: CG_RHS_BLOCK_4}[int(rhs_block)]
    prm = CgParams(float(tol), int(max_iter), int(max_cycles), float(delta), int(chunk), flags, int(max_inner))
    infos = (CgInfo * n)()
    st = load().lq_cg_solve_multi(_dims(dims), float(m_q), m, n, _ptr(U, gb, "U"), _ptr(eta, sb, "eta"),
                                  _ptr(x, sb, "x"), ctypes.byref(prm), _ptr(workspace, wb, "workspace"),
                                  ctypes.c_size_t(workspace.numel() * workspace.element_size()), infos,
                                  _stream(stream))
    _check(st)
    return x, [_info_dict(infos[i]) for i in range(n)], st


def cg_workspace_bytes_schur(dims, mode="mixed_f32", nrhs=1) -> int:
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    return int(load().lq_cg_workspace_bytes_schur(_dims(dims), m, int(nrhs)))


def cg_solve_schur(dims, m_q, U, b, x=None, nrhs=1, mode="mixed_f32", tol=1e-10, max_iter=100000, max_cycles=0,
                   delta=0.0, chunk=0, max_inner=0, workspace=None, stream=None, profile=False, link18=False, graph=True):
    """Solve D x = b (nrhs stacked FP64 LEX fields) by the even-odd Schur complement.
    Returns (x, [info per right-hand side], status)."""
    import torch
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    n = int(nrhs)
    sb = field_bytes(dims, "spinor", "f64") * n
    gb = field_bytes(dims, "gauge", "f64", 18)
    if x is None:
        x = torch.zeros_like(b)
    wb = cg_workspace_bytes_schur(dims, m, n)
    if workspace is None:
        workspace = _empty_bytes(wb, b)
    flags = (CG_PROFILE if profile else 0) | (CG_LINK18 if link18 else 0) | (0 if graph else CG_NO_GRAPH)
    prm = CgParams(float(tol), int(max_iter), int(max_cycles), float(delta), int(chunk), flags, int(max_inner))
    infos = (CgInfo * n)()
    st = load().lq_cg_solve_schur(_dims(dims), float(m_q), m, n, _ptr(U, gb, "U"), _ptr(b, sb, "b"),
                                  _ptr(x, sb, "x"), ctypes.byref(prm), _ptr(workspace, wb, "workspace"),
                                  ctypes.c_size_t(workspace.numel() * workspace.element_size()), infos,
                                  _stream(stream))
    _check(st)
    return x, [_info_dict(infos[i]) for i in range(n)], st


def _info_dict(info) -> dict:
    d = {k: getattr(info, k) for k, _ in CgInfo._fields_}
    d["kernel_ms"] = list(d["kernel_ms"])
    d["kernel_calls"] = list(d["kernel_calls"])
    return d


def _lattice_array(problems):
    arr = (Lattice * len(problems))()
    for i, p in enumerate(problems):
        arr[i].dims = _dims(p["dims"])
        arr[i].nrhs = int(p.get("nrhs", 1))
        arr[i].pad = 0
        arr[i].m_q = float(p.get("m_q", 0.0))
    return arr


def cg_workspace_bytes_lattices(problems, mode="mixed_f32") -> int:
    """Workspace for cg_solve_lattices; problems: dicts with "dims" and "nrhs"."""
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    return int(load().lq_cg_workspace_bytes_lattices(len(problems), _lattice_array(problems), m))


def cg_solve_lattices(problems, mode="mixed_f32", tol=1e-10, max_iter=100000, max_cycles=0, delta=0.0, chunk=0, max_inner=0,
                      workspace=None, stream=None, autotune=False, graph=True, block=None, own_cycles=False):
    """Solve several lattices of different sizes together (lq_cg_solve_lattices).

    problems: list of dicts {"dims", "m_q", "U", "eta", "nrhs" (1, 2, 4 or 8), "x" (optional
    start guess)}, U an F64 LEX 18-real gauge field, eta / x nrhs stacked F64 LEX spinors.
    own_cycles=True lets each lattice take its reliable update as soon as its own inner loop
    stops, the host driving the cycles (default: the reliable updates are taken together and
    the whole batch runs as one CUDA graph launch).
    Returns ([x per lattice], [[info per right-hand side] per lattice], status).
    """
    import torch
    m = CG_MODE[mode] if isinstance(mode, str) else int(mode)
    arr = _lattice_array(problems)
    xs = []
    for i, p in enumerate(problems):
        nr = int(p.get("nrhs", 1))
        sb = field_bytes(p["dims"], "spinor", "f64") * nr
        gb = field_bytes(p["dims"], "gauge", "f64", 18)
        x = p.get("x")
        if x is None:
            x = torch.zeros_like(p["eta"])
        xs.append(x)
        arr[i].U = _ptr(p["U"], gb, "U")
        arr[i].eta = _ptr(p["eta"], sb, "eta")
        arr[i].x = _ptr(x, sb, "x")
    wb = int(load().lq_cg_workspace_bytes_lattices(len(problems), arr, m))
    if workspace is None:
        workspace = _empty_bytes(wb, problems[0]["eta"])
    flags = (CG_AUTOTUNE if autotune else 0) | (0 if graph else CG_NO_GRAPH) | (CG_LATTICE_OWN_CYCLES if own_cycles else 0)
    if block is not None:
        flags |= {64: 0x100, 128: 0x200, 256: 0x400}[int(block)]
    prm = CgParams(float(tol), int(max_iter), int(max_cycles), float(delta), int(chunk), flags, int(max_inner))
    total = sum(int(p.get("nrhs", 1)) for p in problems)
    infos = (CgInfo * total)()
    st = load().lq_cg_solve_lattices(len(problems), arr, m, ctypes.byref(prm), _ptr(workspace, wb, "workspace"),
                                     ctypes.c_size_t(workspace.numel() * workspace.element_size()), infos,
                                     _stream(stream))
    _check(st)
    out, at = [], 0
    for p in problems:
        nr = int(p.get("nrhs", 1))
        out.append([_info_dict(infos[at + j]) for j in range(nr)])
        at += nr
    return xs, out, st
