"""The solver's failure exits, driven from the host with valid memory and finite work.

Every bad value comes from the caller's inputs or parameters (a NaN or an Inf placed in a
field on the host, an operator made zero, caps that end the solve early, a tolerance
below what the arithmetic can reach); no kernel is made to fault or wait.  Each exit must
come back as its documented status (include/lq.h): LQ_ERR_NONFINITE, LQ_ERR_BREAKDOWN, or
LQ_NOT_CONVERGED with x holding the last reliable iterate and info reporting its true
residual.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
M = 0.1


def _fields(U, eta, x0=None):
    Ud = to_dev(F.encode_gauge(U, DIMS, "f64", 18, "lex"))
    ed = to_dev(F.encode_spinor(eta, DIMS, "f64", "lex"))
    xd = to_dev(F.encode_spinor(x0 if x0 is not None else np.zeros_like(eta), DIMS, "f64", "lex"))
    return Ud, ed, xd


def _true_resid(U, eta, x, m=M):
    r = eta - oracle.normal_op(DIMS, m, U, x)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel()))


@pytest.mark.parametrize("mode", ["f64", "f64x", "mixed_f32", "mixed_f16"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_right_hand_side(lqlib, mode, bad):
    U = synth.gauge_field(DIMS, seed=1)
    eta = synth.gaussian_spinor(DIMS, seed=2)
    eta[37, 2, 1] = complex(bad, 0.0)
    Ud, ed, xd = _fields(U, eta)
    with pytest.raises(lqlib.LqError) as ei:
        lqlib.cg_solve(DIMS, M, Ud, ed, x=xd, mode=mode, tol=1e-10)
    assert ei.value.status == -6


@pytest.mark.parametrize("mode", ["f64", "mixed_f32"])
def test_nonfinite_starting_guess(lqlib, mode):
    U = synth.gauge_field(DIMS, seed=1)
    eta = synth.gaussian_spinor(DIMS, seed=2)
    x0 = np.zeros_like(eta)
    x0[5, 0, 0] = complex(np.inf, 0.0)
    Ud, ed, xd = _fields(U, eta, x0)
    with pytest.raises(lqlib.LqError) as ei:
        lqlib.cg_solve(DIMS, M, Ud, ed, x=xd, mode=mode, tol=1e-10)
    assert ei.value.status == -6


@pytest.mark.parametrize("mode", ["f64", "f64x", "mixed_f32", "mixed_f16"])
def test_breakdown_on_a_zero_operator(lqlib, mode):
    """With every link zero and m_q = -4 the operator of Eq. (1) is exactly zero, so the
    first <p, D^dag D p> = ||D p||^2 is 0: the CG coefficient alpha does not exist."""
    U = np.zeros((synth.volume(DIMS), 4, 3, 3), np.complex128)
    eta = synth.gaussian_spinor(DIMS, seed=2)
    Ud, ed, xd = _fields(U, eta)
    with pytest.raises(lqlib.LqError) as ei:
        lqlib.cg_solve(DIMS, -4.0, Ud, ed, x=xd, mode=mode, tol=1e-10)
    assert ei.value.status == -7


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16"])
def test_cycle_cap_returns_the_reliable_iterate(lqlib, mode):
    """One cycle of Algorithm 1 with delta = 0.5: the solve stops not converged after that
    cycle, x is the cycle's reliable update and info reports its FP64 true residual."""
    U = synth.gauge_field(DIMS, seed=1)
    eta = synth.gaussian_spinor(DIMS, seed=2)
    Ud, ed, xd = _fields(U, eta)
    x, info, status = lqlib.cg_solve(DIMS, M, Ud, ed, x=xd, mode=mode, tol=1e-10, delta=0.5, max_cycles=1)
    assert status == 1 and info["status"] == 1
    assert info["cycles"] == 1 and info["iters"] >= 1
    xs = F.decode_spinor(to_host(x), DIMS)
    rel = _true_resid(U, eta, xs)
    assert rel <= 0.55
    assert abs(rel - info["true_rel_resid"]) <= 1e-6 * rel


def test_iteration_cap(lqlib):
    U = synth.gauge_field(DIMS, seed=1)
    eta = synth.gaussian_spinor(DIMS, seed=2)
    Ud, ed, xd = _fields(U, eta)
    x, info, status = lqlib.cg_solve(DIMS, M, Ud, ed, x=xd, mode="f64", tol=1e-10, max_iter=5)
    assert status == 1
    assert info["iters"] == 5
    xs = F.decode_spinor(to_host(x), DIMS)
    rel = _true_resid(U, eta, xs)
    assert 1e-10 < rel < 1.0
    assert abs(rel - info["true_rel_resid"]) <= 1e-9 * rel


def test_stagnation_below_the_arithmetic(lqlib):
    """A tolerance of 1e-20 lies below what the FP64-class residual can resolve: the true
    residual stops decreasing, and after five cycles without progress the solver gives up
    (long before its cycle and iteration caps) with the best accuracy it reached."""
    U = synth.gauge_field(DIMS, seed=1)
    eta = synth.gaussian_spinor(DIMS, seed=2)
    Ud, ed, xd = _fields(U, eta)
    x, info, status = lqlib.cg_solve(DIMS, M, Ud, ed, x=xd, mode="mixed_f32", tol=1e-20)
    assert status == 1
    assert info["cycles"] < 1000 and info["iters"] < 100000
    xs = F.decode_spinor(to_host(x), DIMS)
    assert _true_resid(U, eta, xs) <= 1e-12
