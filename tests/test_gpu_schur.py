"""The even-odd Schur solve of D x = b: against the oracle's solution of D x = b, the
residual of the original system, batches, a zero right-hand side, and the full 32^4 size."""
import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

MODES = ["f64x", "mixed_f32", "mixed_f16", "mixed_i32"]


def _resid_d(dims, m, U, b, x):
    r = b - oracle.dslash(dims, m, U, x)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel())


def _solve(lqlib, dims, m, U, bs, mode, tol, **kw):
    n = len(bs)
    Ud = to_dev(F.encode_gauge(U, dims))
    bd = to_dev(F.encode_spinor_multi(bs, dims, "f64", "lex"))
    x, infos, st = lqlib.cg_solve_schur(dims, m, Ud, bd, nrhs=n, mode=mode, tol=tol, **kw)
    return F.decode_spinor_multi(to_host(x), dims, n, "f64", "lex"), infos, st


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 10, 2)])
def test_schur_matches_oracle(lqlib, mode, dims):
    m = 0.1
    U = synth.gauge_field(dims, seed=81, kind="near_identity", eps=0.5)
    b = synth.gaussian_spinor(dims, seed=82)
    xs, infos, st = _solve(lqlib, dims, m, U, [b], mode, tol=1e-12)
    assert st == 0 and infos[0]["status"] == 0 and infos[0]["true_rel_resid"] <= 1e-12
    x_ref, _, _ = oracle.solve_d(dims, m, U, b, tol=1e-14)
    assert oracle.rel_l2(xs[0], x_ref) <= 1e-9
    assert _resid_d(dims, m, U, b, xs[0]) <= 1e-10


def test_schur_batches_and_zero_rhs(lqlib):
    """Three right-hand sides (batches of 2 and 1), the second one zero."""
    dims = (4, 4, 2, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=83, kind="near_identity", eps=0.5)
    bs = [synth.gaussian_spinor(dims, seed=84), np.zeros((synth.volume(dims), 4, 3), complex),
          synth.gaussian_spinor(dims, seed=85)]
    xs, infos, st = _solve(lqlib, dims, m, U, bs, "mixed_f32", tol=1e-12)
    assert st == 0
    assert np.all(xs[1] == 0) and infos[1]["status"] == 0
    for i in (0, 2):
        assert _resid_d(dims, m, U, bs[i], xs[i]) <= 1e-10


def test_schur_fewer_iterations_than_normal_equations(lqlib):
    """On the same system the even-odd operator needs fewer CG iterations than D^dag D on
    the whole lattice (its condition number is smaller)."""
    dims = (8, 8, 8, 8)
    m = 0.05
    U = synth.gauge_field(dims, seed=86, kind="near_identity", eps=0.3)
    b = synth.gaussian_spinor(dims, seed=87)
    xs, infos, st = _solve(lqlib, dims, m, U, [b], "f64x", tol=1e-10)
    assert st == 0
    Ud = to_dev(F.encode_gauge(U, dims))
    eta = lqlib.dslash_adjoint(dims, m, Ud, to_dev(F.encode_spinor(b, dims)))
    _, info_full, st2 = lqlib.cg_solve(dims, m, Ud, eta, mode="f64x", tol=1e-10)
    assert st2 == 0
    assert infos[0]["iters"] < info_full["iters"]


def test_schur_full_size_32(lqlib):
    """32^4, links exp(0.3 i H), m_q = 0.05, scaled-FP16 inner storage, tolerance 1e-10 on
    the normal equations; the oracle recomputes the residual of D x = b."""
    dims = (32, 32, 32, 32)
    m = 0.05
    U = synth.gauge_field(dims, seed=3, kind="near_identity", eps=0.3)
    b = synth.gaussian_spinor(dims, seed=4)
    xs, infos, st = _solve(lqlib, dims, m, U, [b], "mixed_f16", tol=1e-10)
    assert st == 0 and infos[0]["true_rel_resid"] <= 1e-10
    assert _resid_d(dims, m, U, b, xs[0]) <= 1e-8


def test_schur_argument_checks(lqlib):
    dims = (4, 4, 4, 4)
    U = to_dev(F.encode_gauge(synth.gauge_field(dims, seed=1), dims))
    b = to_dev(F.encode_spinor(synth.gaussian_spinor(dims, seed=2), dims))
    with pytest.raises(lqlib.LqError):
        lqlib.cg_solve_schur(dims, 0.1, U, b, mode="f64", workspace=to_dev(np.zeros(1 << 20, np.uint8)))
    assert lqlib.cg_workspace_bytes_schur(dims, "f64") == 0
    assert 0 < lqlib.cg_workspace_bytes_schur(dims, "mixed_f16") < lqlib.cg_workspace_bytes(dims, "mixed_f16")


@pytest.mark.parametrize("mode", MODES)
def test_schur_device_loop_equals_host_loop(lqlib, mode):
    """The Schur inner loop (with its extra hop kernels) run as a conditional CUDA graph and
    run from the host take the same steps: bit-identical solutions and the same counts."""
    dims = (4, 4, 2, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=86, kind="near_identity", eps=0.5)
    bs = [synth.gaussian_spinor(dims, seed=87), synth.gaussian_spinor(dims, seed=88)]
    xg, ig, sg = _solve(lqlib, dims, m, U, bs, mode, tol=1e-12)
    xh, ih, sh = _solve(lqlib, dims, m, U, bs, mode, tol=1e-12, graph=False)
    assert sg == sh == 0
    for a, b in zip(ig, ih):
        assert a["iters"] == b["iters"] and a["cycles"] == b["cycles"]
    assert np.array_equal(xg, xh)
