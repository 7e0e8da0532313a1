"""lq_cg_solve_noalloc: the CG solve for callers that cannot allocate device memory.

Its scratch is a fixed array inside the library instead of a caller workspace.  The test
calls it through the C ABI twice in a row (the second call reuses the array the first one
left behind) and checks each result against lq_cg_solve with a caller workspace on the
same inputs, with the solution and residual tolerances of the other CG tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu


def _entry(lqlib):
    L = lqlib.load()
    fn = L.lq_cg_solve_noalloc
    fn.argtypes = [ctypes.c_int32 * 4, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.POINTER(lqlib.CgParams), ctypes.POINTER(lqlib.CgInfo), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    L.lq_cg_noalloc_max_workspace_bytes.restype = ctypes.c_size_t
    return L, fn


@pytest.mark.parametrize("mode", ["mixed_f32", "f64", "mixed_f16"])
def test_noalloc_solver_matches_workspace_solver(lqlib, mode):
    import torch
    L, fn = _entry(lqlib)
    dims = (8, 8, 8, 8)
    m = 0.1
    U = synth.gauge_field(dims, seed=21)
    eta = synth.gaussian_spinor(dims, seed=22)
    Ud = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    ed = to_dev(F.encode_spinor(eta, dims, "f64", "lex"))
    xr, info_ref, st_ref = lqlib.cg_solve(dims, m, Ud, ed, mode=mode, tol=1e-10)
    assert st_ref == 0
    x_ref = F.decode_spinor(to_host(xr), dims)
    code = lqlib.CG_MODE[mode]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = torch.zeros_like(ed)
        prm = lqlib.CgParams(1e-10, 100000, 0, 0.0, 0, 0)
        info = lqlib.CgInfo()
        st = fn((ctypes.c_int32 * 4)(*dims), m, code, ctypes.c_void_p(Ud.data_ptr()),
                ctypes.c_void_p(ed.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.byref(prm),
                ctypes.byref(info), stream)
        assert st == 0, lqlib.last_error()
        xs = F.decode_spinor(to_host(x), dims)
        assert oracle.rel_l2(xs, x_ref) <= 1e-7
        r = eta - oracle.normal_op(dims, m, U, xs)
        assert np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10 * 1.001
        assert info.iters == info_ref["iters"]


def test_noalloc_rejects_lattices_beyond_the_array(lqlib):
    L, fn = _entry(lqlib)
    cap = L.lq_cg_noalloc_max_workspace_bytes()
    dims = (32, 32, 32, 32)
    assert lqlib.cg_workspace_bytes(dims, "mixed_f32") > cap
    info = lqlib.CgInfo()
    st = fn((ctypes.c_int32 * 4)(*dims), 0.1, 1, None, None, None, None, ctypes.byref(info), None)
    assert st == -5 and info.status == -5
    assert "no-allocation" in lqlib.last_error()
