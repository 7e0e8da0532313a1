"""GPU conjugate-gradient solves of D^dag D x = eta against the CPU oracle.

The oracle recomputes the true residual ||eta - D^dag D x|| / ||eta|| of every GPU
solution in FP64 and its own textbook CG gives the reference solution; D^dag D is
Hermitian positive definite, so the solution is unique and the two solutions can differ
only by the tolerance times the condition number.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import dense
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

RESID_SLACK = 1.001   # FP64 rounding between the GPU's and the oracle's residual evaluation


def _solve(lqlib, dims, m, U, eta, mode, x0=None, **kw):
    Ud = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    ed = to_dev(F.encode_spinor(eta, dims, "f64", "lex"))
    xd = to_dev(F.encode_spinor(x0 if x0 is not None else np.zeros_like(eta), dims, "f64", "lex"))
    x, info, status = lqlib.cg_solve(dims, m, Ud, ed, x=xd, mode=mode, **kw)
    return F.decode_spinor(to_host(x), dims, "f64", "lex"), info, status


def _true_resid(dims, m, U, eta, x):
    r = eta - oracle.normal_op(dims, m, U, x)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel())


MODES = ["f64", "f64x", "mixed_f32", "mixed_f16", "mixed_i32"]


@pytest.mark.parametrize("mode", MODES)
def test_cg_2222_against_dense_solve(lqlib, mode):
    dims = (2, 2, 2, 2)
    m = 0.1
    U = synth.gauge_field(dims, seed=1)
    eta = synth.gaussian_spinor(dims, seed=2)
    x, info, status = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10)
    assert status == 0 and info["true_rel_resid"] <= 1e-10
    Dd = dense.dense_dirac(dims, m, U)
    A = Dd.conj().T @ Dd
    xd = np.linalg.solve(A, eta.ravel())
    assert np.linalg.norm(eta.ravel() - A @ x.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10 * RESID_SLACK
    assert oracle.rel_l2(x.ravel(), xd) <= 1e-10 * np.linalg.cond(A)


@pytest.mark.parametrize("mode", MODES)
def test_cg_4444_haar_against_oracle(lqlib, mode):
    """The small FP64 configuration: 4^4 Haar links, m_q = 0.1, tolerance 1e-10."""
    dims = (4, 4, 4, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=1)
    eta = synth.gaussian_spinor(dims, seed=2)
    x, info, status = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10)
    assert status == 0
    assert info["true_rel_resid"] <= 1e-10
    assert _true_resid(dims, m, U, eta, x) <= 1e-10 * RESID_SLACK
    xo, it, rel = oracle.cg(dims, m, U, eta, tol=1e-12)
    assert oracle.rel_l2(x, xo) <= 1e-7
    if mode in ("f64", "f64x"):
        # plain CG: the same iterations as the oracle's textbook CG (up to rounding)
        _, it10, _ = oracle.cg(dims, m, U, eta, tol=1e-10)
        assert abs(info["iters"] - it10) <= 2
        assert info["cycles"] <= 2


@pytest.mark.parametrize("mode", MODES)
def test_cg_near_identity_ragged(lqlib, mode):
    """Near-free links, small mass (the ill-conditioned case) on a lattice with a ragged
    last tile."""
    dims = (6, 4, 10, 2)
    m = 0.05
    U = synth.gauge_field(dims, seed=5, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=6)
    x, info, status = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10)
    assert status == 0
    assert _true_resid(dims, m, U, eta, x) <= 1e-10 * RESID_SLACK
    if mode.startswith("mixed"):
        assert info["cycles"] >= 2


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "mixed_i32"])
@pytest.mark.parametrize("native_f64,link18", [(True, False), (False, True), (True, True)])
def test_cg_outer_arithmetic_and_link_format(lqlib, mode, native_f64, link18):
    """The solver options: native FP64 outer arithmetic instead of FP32 pairs, and 18-real
    inner links instead of 12-real."""
    dims = (4, 6, 4, 4)
    m = 0.05
    U = synth.gauge_field(dims, seed=17, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=18)
    x, info, status = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10, native_f64=native_f64, link18=link18)
    assert status == 0
    assert _true_resid(dims, m, U, eta, x) <= 1e-10 * RESID_SLACK


def test_cg_starting_guess_and_resume(lqlib):
    """A solve started from a previous solution converges at once (resume = call again)."""
    dims = (4, 4, 4, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=11)
    eta = synth.gaussian_spinor(dims, seed=12)
    x1, info1, st1 = _solve(lqlib, dims, m, U, eta, "mixed_f32", tol=1e-8)
    assert st1 == 0
    x2, info2, st2 = _solve(lqlib, dims, m, U, eta, "mixed_f32", x0=x1, tol=1e-10)
    assert st2 == 0 and info2["iters"] < info1["iters"] + 5
    assert _true_resid(dims, m, U, eta, x2) <= 1e-10 * RESID_SLACK


def test_cg_zero_rhs(lqlib):
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, seed=13)
    eta = np.zeros((synth.volume(dims), 4, 3), np.complex128)
    x0 = synth.gaussian_spinor(dims, seed=14)
    x, info, status = _solve(lqlib, dims, 0.1, U, eta, "f64", x0=x0)
    assert status == 0 and info["iters"] == 0 and np.all(x == 0)


def test_cg_max_iter_not_converged(lqlib):
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, seed=15, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=16)
    x, info, status = _solve(lqlib, dims, 0.01, U, eta, "mixed_f32", tol=1e-10, max_iter=3)
    assert status == 1
    assert info["iters"] <= 3
    assert 1e-10 < info["true_rel_resid"] < 1.0
    # the returned x is the iterate whose FP64 residual was reported
    assert abs(_true_resid(dims, 0.01, U, eta, x) - info["true_rel_resid"]) < 1e-8


def test_cg_workspace_too_small(lqlib):
    import torch
    dims = (4, 4, 4, 4)
    U = to_dev(F.encode_gauge(synth.gauge_field(dims, seed=1), dims))
    eta = to_dev(F.encode_spinor(synth.gaussian_spinor(dims, seed=2), dims))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        lqlib.cg_solve(dims, 0.1, U, eta, workspace=ws)


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "f64", "f64x", "mixed_i32"])
def test_cg_full_size_32(lqlib, mode):
    """The mixed-precision workload at full size: 32^4, links exp(0.3 i H), m_q = 0.05,
    tolerance 1e-10; the oracle recomputes the true residual in FP64."""
    dims = (32, 32, 32, 32)
    m = 0.05
    U = synth.gauge_field(dims, seed=3, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=4)
    x, info, status = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10)
    assert status == 0
    assert info["true_rel_resid"] <= 1e-10
    assert _true_resid(dims, m, U, eta, x) <= 1e-10 * RESID_SLACK


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("max_iter", [100000, 7])
def test_cg_device_loop_equals_host_loop(lqlib, mode, max_iter):
    """The solve run on the device (one CUDA graph: the cycles and each cycle's inner loop as
    conditional WHILE nodes, Algorithm 1's decisions in one-thread kernels) takes the same
    steps as the host-driven loop: the kernels, their order and the decisions are the same, so
    the solution is bit-identical, with the same iteration and cycle counts (also when
    max_iter cuts a cycle)."""
    dims = (4, 6, 4, 4)
    m = 0.05
    U = synth.gauge_field(dims, seed=19, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=20)
    xg, ig, sg = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10, max_iter=max_iter)
    xh, ih, sh = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10, max_iter=max_iter, graph=False)
    assert sg == sh
    assert ig["iters"] == ih["iters"] and ig["cycles"] == ih["cycles"]
    assert np.array_equal(xg, xh)
    assert ig["true_rel_resid"] == ih["true_rel_resid"]


@pytest.mark.parametrize("mode", ["f64", "f64x", "mixed_f16"])
def test_cg_zero_guess_starts_from_eta(lqlib, mode):
    """With x0 = 0 the first outer residual eta - D^dag D x0 is eta itself and the operator is
    not applied for it; one nonzero component (even a subnormal one) in x0 restores the apply."""
    dims = (4, 4, 4, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=21)
    eta = synth.gaussian_spinor(dims, seed=22)
    x0, info0, st0 = _solve(lqlib, dims, m, U, eta, mode, tol=1e-10)
    tiny = np.zeros_like(eta)
    tiny[5, 2, 1] = 1e-310 * 1j
    x1, info1, st1 = _solve(lqlib, dims, m, U, eta, mode, x0=tiny, tol=1e-10)
    assert st0 == st1 == 0
    assert info0["high_applies"] == info0["cycles"]
    assert info1["high_applies"] == info1["cycles"] + 1
    assert _true_resid(dims, m, U, eta, x0) <= 1e-10 * RESID_SLACK
    assert _true_resid(dims, m, U, eta, x1) <= 1e-10 * RESID_SLACK


def test_cg_scaled_fp16_keeps_the_cg_iteration_count(lqlib):
    """With the inner solution kept in FP32, the scaled-FP16 mode runs each cycle to its default
    reduction of 1e-2 without extra iterations: it needs about the iterations of plain FP64 CG
    and a handful of cycles (re-quantising psi to FP16 every iteration needed thousands of
    iterations at this reduction)."""
    dims = (8, 8, 8, 8)
    m = 0.05
    U = synth.gauge_field(dims, seed=23, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=24)
    _, i64, s64 = _solve(lqlib, dims, m, U, eta, "f64", tol=1e-10)
    x, i16, s16 = _solve(lqlib, dims, m, U, eta, "mixed_f16", tol=1e-10)
    assert s64 == s16 == 0
    assert i16["iters"] <= 1.1 * i64["iters"]
    assert i16["cycles"] <= 7
    assert _true_resid(dims, m, U, eta, x) <= 1e-10 * RESID_SLACK
