"""The 10-real link form on the GPU against the oracle (Introduction and Section 2.2 of the
paper: 10 input words per link instead of 18).

The form stores row 0 and the two entries of row 1 outside column k, k being the column of
the stored row 0 with the largest max(|Re|, |Im|), the lowest on ties; both sides make that
choice on the stored values in their own exact domain (FP64, FP32, FP16 or the Q1.30
integers).  The field here mixes Haar and near-identity links with hand-built SU(3) links
that force each column, exact ties, and Q1.30 rows whose two largest components differ by
one integer step (their FP32 images coincide).  The encoder must match the oracle's byte for
byte, the operator must meet the per-precision bounds against the oracle on the rebuilt
links, and the mixed solvers must reach the FP64 tolerance with 10-real inner links.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16s": 1e-3, "i32s": 1e-6}


def _complete_su3(v, rng):
    """An SU(3) matrix whose row 0 is exactly the unit vector v (QR completion; the
    determinant's phase is taken out of row 2, so row 0 keeps its components)."""
    M = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    M[:, 0] = np.conj(v)
    Q, _ = np.linalg.qr(M)
    U = Q.conj().T
    U[0] = v                       # Q's first column is conj(v) times a phase: undo it
    U[1:] = U[1:] - np.outer(U[1:] @ np.conj(v), v)
    U[1] /= np.linalg.norm(U[1])
    U[2] -= np.vdot(U[1], U[2]) * U[1]
    U[2] /= np.linalg.norm(U[2])
    U[2] *= np.conj(np.linalg.det(U))
    return U


def _special_links(rng):
    a = np.sqrt(0.5)
    x = 0.6
    y = x + 2.0 ** -30                 # one Q1.30 step above x
    z = np.sqrt(1 - x * x - y * y)
    rows = [
        np.array([0, 0, 1], complex),                     # k = 2
        np.array([0, 1j, 0], complex),                    # k = 1
        np.array([1, 0, 0], complex),                     # k = 0
        np.array([a, 1j * a, 0]),                         # tie between 0 and 1 -> 0
        np.array([0, a, -1j * a]),                        # tie between 1 and 2 -> 1
        np.array([x, 1j * y, z]),                         # Q1.30: column 1 by one integer step
        np.array([1j * y, x, z]),                         # Q1.30: column 0 by one integer step
        np.array([1e-7, np.sqrt(0.5), np.sqrt(0.5 - 1e-14) * 1j]),
    ]
    return [_complete_su3(v / np.linalg.norm(v), rng) for v in rows]


def _field(dims, seed):
    rng = np.random.default_rng(seed)
    V = synth.volume(dims)
    U = synth.gauge_field(dims, seed=seed).reshape(V * 4, 3, 3)
    Un = synth.gauge_field(dims, seed=seed + 1, kind="near_identity", eps=0.3).reshape(V * 4, 3, 3)
    U[1::2] = Un[1::2]
    sp = _special_links(rng)
    for i in range(0, V * 4, 7):
        U[i] = sp[(i // 7) % len(sp)]
    return U.reshape(V, 4, 3, 3)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 10, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16s", "i32s"])
@pytest.mark.parametrize("layout", ["lex", "eo"])
def test_link10_encoding_bit_exact(lqlib, dims, prec, layout):
    U = _field(dims, 401)
    src = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    dst = lqlib.convert_gauge(dims, src, "f64", "lex", dst_prec=prec, dst_fmt=10, dst_layout=layout)
    assert np.array_equal(to_host(dst), F.encode_gauge(U, dims, prec, 10, layout))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 10, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16s", "i32s"])
@pytest.mark.parametrize("layout", ["lex", "eo"])
@pytest.mark.parametrize("dagger", [False, True])
def test_link10_operator_matches_oracle(lqlib, dims, prec, layout, dagger):
    U = _field(dims, 403)
    psi = synth.gaussian_spinor(dims, seed=404)
    Ub = F.encode_gauge(U, dims, prec, 10, layout)
    pb = F.encode_spinor(psi, dims, prec, layout)
    want = oracle.dslash(dims, 0.1, F.decode_gauge(Ub, dims, prec, 10, layout),
                         F.decode_spinor(pb, dims, prec, layout), dagger=dagger)
    fn = lqlib.dslash_adjoint if dagger else lqlib.dslash_apply
    out = fn(dims, 0.1, to_dev(Ub), to_dev(pb), prec=prec, link_fmt=10, layout=layout)
    assert oracle.rel_l2(F.decode_spinor(to_host(out), dims, prec, layout), want) <= TOL[prec]
    if prec == "f64":
        # and, for SU(3) links stored in FP64, the operator of the full links
        full = oracle.dslash(dims, 0.1, U, psi, dagger=dagger)
        assert oracle.rel_l2(F.decode_spinor(to_host(out), dims, prec, layout), full) <= 1e-13


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "mixed_i32"])
@pytest.mark.parametrize("dims,m,kind", [((4, 4, 4, 4), 0.1, "haar"), ((6, 4, 10, 2), 0.05, "near_identity")])
def test_link10_inner_links_in_the_solver(lqlib, mode, dims, m, kind):
    """Algorithm 1 with 10-real inner links reaches the FP64 tolerance, in about the
    iterations of the 12-real inner links."""
    U = synth.gauge_field(dims, seed=405, kind=kind, eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=406)
    Ud = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    ed = to_dev(F.encode_spinor(eta, dims, "f64", "lex"))
    x, info, st = lqlib.cg_solve(dims, m, Ud, ed, mode=mode, tol=1e-10, link10=True)
    assert st == 0
    xs = F.decode_spinor(to_host(x), dims)
    r = eta - oracle.normal_op(dims, m, U, xs)
    assert np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10 * 1.001
    _, info12, _ = lqlib.cg_solve(dims, m, Ud, ed, mode=mode, tol=1e-10)
    assert abs(info["iters"] - info12["iters"]) <= max(3, info12["iters"] // 10)


def test_link10_flag_combinations_rejected(lqlib):
    dims = (4, 4, 4, 4)
    U = to_dev(F.encode_gauge(synth.gauge_field(dims, seed=1), dims, "f64", 18, "lex"))
    eta = to_dev(F.encode_spinor(synth.gaussian_spinor(dims, seed=2), dims, "f64", "lex"))
    for kw in ({"native_f64": True}, {"link18": True}):
        with pytest.raises(lqlib.LqError) as ei:
            lqlib.cg_solve(dims, 0.1, U, eta, mode="mixed_f32", link10=True, **kw)
        assert ei.value.status == -1
