"""The GPU's Algorithm 1 (residual-guided mixed-precision CG, Section 1) against the
oracle's, cycle by cycle.

The oracle's Algorithm 1 is pinned on its own (tests/test_oracle_pins.py): with an FP64
inner loop its restarts continue CG exactly, so it takes the textbook CG's iterations,
and a wrong beta_0 or a dropped <r_0, p_k> projection costs iterations.  Here the library's
solver runs the same seeded systems with the same inner reduction delta and must reproduce
the oracle's number of outer cycles and (within one) its total inner iterations: the
restart is the part of the method whose mistakes would still converge, only more slowly.

With an FP64-class inner loop (native FP64, or FP32 pairs at about 2^-47) the two solvers
take the same path up to rounding, so cycles must be equal and iterations within one.  The
FP32 inner loop rounds differently from the oracle's model of it (the oracle rounds every
vector to FP32 after each operation of an FP64 computation; the kernels compute in FP32
with 12-real links in the EO layout), so there the cycles may differ by one (the last
cycle ends within rounding of the tolerance) and the iterations by a few.
"""
import functools

import numpy as np
import pytest

import oracle
import synth
from oracle import dense
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

RESID_SLACK = 1.001

# (dims, m_q, links, seeds): the small Haar configuration, and two near-identity systems
# (the ill-conditioned case) on small and ragged lattices
SYSTEMS = [
    ((4, 4, 4, 4), 0.1, "haar", (1, 2)),
    ((4, 4, 2, 4), 0.05, "near_identity", (71, 72)),
    ((6, 4, 10, 2), 0.05, "near_identity", (5, 6)),
]
IDS = ["4444-haar", "4424-near-identity", "64102-near-identity"]


def _system(dims, kind, seeds):
    U = synth.gauge_field(dims, seed=seeds[0], kind=kind, eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=seeds[1])
    return U, eta


def _gpu(lqlib, dims, m, U, eta, mode, delta):
    Ud = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    ed = to_dev(F.encode_spinor(eta, dims, "f64", "lex"))
    x, info, status = lqlib.cg_solve(dims, m, Ud, ed, mode=mode, tol=1e-10, delta=delta)
    return F.decode_spinor(to_host(x), dims, "f64", "lex"), info, status


@functools.lru_cache(maxsize=None)
def _kappa(dims, m, kind, seeds):
    """Condition number of D^dag D (dense, small lattices only)."""
    U, _ = _system(dims, kind, seeds)
    D = dense.dense_dirac(dims, m, U)
    sv = np.linalg.svd(D, compute_uv=False)
    return float((sv[0] / sv[-1]) ** 2)


@pytest.mark.parametrize("system", SYSTEMS, ids=IDS)
@pytest.mark.parametrize("mode", ["f64", "f64x"])
@pytest.mark.parametrize("delta", [1e-1, 1e-2])
def test_alg1_fp64_inner_matches_oracle(lqlib, system, mode, delta):
    dims, m, kind, seeds = system
    U, eta = _system(dims, kind, seeds)
    xo, cyc_o, it_o, rel_o = oracle.alg1(dims, m, U, eta, tol=1e-10, low="f64", delta=delta)
    assert rel_o <= 1e-10 and cyc_o >= 4
    x, info, status = _gpu(lqlib, dims, m, U, eta, mode, delta)
    assert status == 0
    assert info["cycles"] == cyc_o
    assert abs(info["iters"] - it_o) <= 1
    r = eta - oracle.normal_op(dims, m, U, x)
    assert np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10 * RESID_SLACK
    # both solutions lie within tol * kappa of the exact one
    if synth.volume(dims) <= 256:
        assert oracle.rel_l2(x, xo) <= 2e-10 * _kappa(dims, m, kind, seeds)
    else:
        assert oracle.rel_l2(x, xo) <= 1e-6


@pytest.mark.parametrize("system", SYSTEMS, ids=IDS)
@pytest.mark.parametrize("delta", [1e-3, 1e-4])
def test_alg1_fp32_inner_matches_oracle(lqlib, system, delta):
    dims, m, kind, seeds = system
    U, eta = _system(dims, kind, seeds)
    _, cyc_o, it_o, rel_o = oracle.alg1(dims, m, U, eta, tol=1e-10, low="f32", delta=delta)
    assert rel_o <= 1e-10 and cyc_o >= 3
    x, info, status = _gpu(lqlib, dims, m, U, eta, "mixed_f32", delta)
    assert status == 0
    assert abs(info["cycles"] - cyc_o) <= 1
    assert abs(info["iters"] - it_o) <= max(3, it_o // 20)
    r = eta - oracle.normal_op(dims, m, U, x)
    assert np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10 * RESID_SLACK
