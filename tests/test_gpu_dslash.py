"""GPU parity of the operator kernels against the CPU oracle (through the C ABI).

Inputs are seeded synthetic fields encoded by the oracle's own encoders; the oracle runs
on the FP64 values of the stored (rounded) fields, so the comparison measures kernel
error only.  Bounds (relative L2 over all reals of the output field):
  F64  1e-13   (the stated FP64 bound)
  F64X 1e-13   (FP32-pair arithmetic is held to the FP64 bound)
  F32  1e-6    (the stated FP32 bound)
  F16S 1e-3    (output rounding to FP16: at most 2^-12 relative per normal component,
                about 1.4e-4 rms, plus FP32 accumulation; bound x4 above the maximum)
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import eo_embed, eo_half, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64x": 1e-13, "f32": 1e-6, "f16s": 1e-3, "i32s": 1e-6}
# 2^4 aliases n+mu and n-mu; (6, 4, 10, 2) has V = 480, a ragged last tile for 128 threads
LATTICES = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 10, 2)]


def _fields(dims, seed, kind="haar"):
    U = synth.gauge_field(dims, seed=seed, kind=kind, eps=0.3)
    psi = synth.gaussian_spinor(dims, seed=seed + 1)
    return U, psi


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("layout", ["lex", "eo"])
@pytest.mark.parametrize("fmt", [18, 12, 10])
@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16s", "i32s"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_matches_oracle(lqlib, dims, layout, fmt, prec, dagger):
    if prec == "f64x" and fmt != 18:
        pytest.skip("FP32-pair fields use 18-real links")
    m = 0.1
    U, psi = _fields(dims, 100 + sum(dims))
    Ub = F.encode_gauge(U, dims, prec, fmt, layout)
    pb = F.encode_spinor(psi, dims, prec, layout)
    want = oracle.dslash(dims, m, F.decode_gauge(Ub, dims, prec, fmt, layout),
                         F.decode_spinor(pb, dims, prec, layout), dagger=dagger)
    fn = lqlib.dslash_adjoint if dagger else lqlib.dslash_apply
    out = fn(dims, m, to_dev(Ub), to_dev(pb), prec=prec, link_fmt=fmt, layout=layout)
    got = F.decode_spinor(to_host(out), dims, prec, layout)
    assert oracle.rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 10, 2)])
@pytest.mark.parametrize("prec", ["f32", "f16s", "f64x", "i32s"])
@pytest.mark.parametrize("layout", ["lex", "eo"])
def test_convert_spinor_bit_exact(lqlib, dims, prec, layout):
    psi = synth.gaussian_spinor(dims, seed=7) * np.exp(np.linspace(-8, 8, synth.volume(dims)))[:, None, None]
    psi[1] = 0.0     # all-zero site: scale 0
    src = to_dev(F.encode_spinor(psi, dims, "f64", "lex"))
    dst = lqlib.convert_spinor(dims, src, "f64", "lex", dst_prec=prec, dst_layout=layout)
    assert np.array_equal(to_host(dst), F.encode_spinor(psi, dims, prec, layout))
    # and back to FP64 LEX: exact stored values
    back = lqlib.convert_spinor(dims, dst, prec, layout, dst_prec="f64", dst_layout="lex")
    assert np.array_equal(F.decode_spinor(to_host(back), dims, "f64", "lex"),
                          F.decode_spinor(to_host(dst), dims, prec, layout))


@pytest.mark.parametrize("layout", ["lex", "eo"])
def test_convert_pairs_bit_exact_at_the_edges(lqlib, layout):
    """FP64 -> FP32 pairs (hi = fl32(v), lo = fl32(v - hi)) for values that probe the split:
    rounding ties to even either way, a carry out of the significand, the exponent range ends
    of the fast integer route and the values outside it (zero, subnormal, tiny, near FP32
    overflow), and random doubles spread over 2^-90 .. 2^127."""
    dims = (4, 2, 2, 2)
    V = synth.volume(dims)
    rng = np.random.default_rng(9)
    edge = np.array([0.0, -0.0, 1.0, -1.0, 1 + 2.0**-24, 1 + 3 * 2.0**-24, -(1 + 2.0**-24), 2 - 2.0**-52,
                     1.5 * 2.0**-74, 2.0**-74, 1.9 * 2.0**-75, 2.0**126 * (2 - 2.0**-30), 2.0**126 * (2 - 2.0**-52),
                     3e38, 1e-30, 2.0**-1022, 5e-324, 2.0**-50 + 2.0**-80, 1 + 2.0**-24 + 2.0**-60,
                     -(2 - 2.0**-52), 7 * 2.0**-77])
    mant = rng.uniform(1.0, 2.0, 24 * V) * rng.choice([-1.0, 1.0], 24 * V)
    vals = np.ldexp(mant, rng.integers(-90, 127, 24 * V))
    bits = vals.view(np.uint64)
    tie = rng.integers(0, 3, 24 * V)
    low = np.where(tie == 0, 0x10000000, np.where(tie == 1, 0x0FFFFFFF, 0x10000001)).astype(np.uint64)
    bits[::5] = (bits[::5] & ~np.uint64(0x1FFFFFFF)) | low[::5]
    vals[:edge.size] = edge
    psi = vals.reshape(V, 4, 3, 2)
    psi = psi[..., 0] + 1j * psi[..., 1]
    src = to_dev(F.encode_spinor(psi, dims, "f64", "lex"))
    dst = lqlib.convert_spinor(dims, src, "f64", "lex", dst_prec="f64x", dst_layout=layout)
    assert np.array_equal(to_host(dst), F.encode_spinor(psi, dims, "f64x", layout))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 10, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16s", "f64x", "i32s"])
@pytest.mark.parametrize("fmt", [18, 12, 10])
@pytest.mark.parametrize("layout", ["lex", "eo"])
def test_convert_gauge_bit_exact(lqlib, dims, prec, fmt, layout):
    if prec == "f64x" and fmt != 18:
        pytest.skip("FP32-pair fields use 18-real links")
    U = synth.gauge_field(dims, seed=8)
    src = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    dst = lqlib.convert_gauge(dims, src, "f64", "lex", dst_prec=prec, dst_fmt=fmt, dst_layout=layout)
    assert np.array_equal(to_host(dst), F.encode_gauge(U, dims, prec, fmt, layout))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 10, 2)])
@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16s", "i32s"])
@pytest.mark.parametrize("fmt", [18, 12, 10])
@pytest.mark.parametrize("dagger", [False, True])
def test_hop_matches_oracle(lqlib, dims, prec, fmt, dagger):
    if prec == "f64x" and fmt != 18:
        pytest.skip("FP32-pair fields use 18-real links")
    U, psi = _fields(dims, 300)
    y = synth.gaussian_spinor(dims, seed=301)
    Ub = F.encode_gauge(U, dims, prec, fmt, "eo")
    Ud = F.decode_gauge(Ub, dims, prec, fmt, "eo")
    pb = F.encode_spinor(psi, dims, prec, "eo")
    yb = F.encode_spinor(y, dims, prec, "eo")
    pd = F.decode_spinor(pb, dims, prec, "eo")
    yd = F.decode_spinor(yb, dims, prec, "eo")
    par = oracle.parity_of_sites(dims)
    a, b = 0.7, -1.3
    for p in (0, 1):
        src = to_dev(eo_half(pb, dims, prec, 1 - p))
        yy = to_dev(eo_half(yb, dims, prec, p))
        out = lqlib.dslash_hop(dims, p, to_dev(Ub), src, a=a, b=b, y=yy, dagger=dagger, prec=prec, link_fmt=fmt)
        got = F.decode_spinor(eo_embed(to_host(out), dims, prec, p), dims, prec, "eo")[par == p]
        want = (a * yd + b * oracle.hop(dims, Ud, pd, p, dagger=dagger))[par == p]
        assert oracle.rel_l2(got, want) <= TOL[prec]
        # without y
        out = lqlib.dslash_hop(dims, p, to_dev(Ub), src, b=1.0, dagger=dagger, prec=prec, link_fmt=fmt)
        got = F.decode_spinor(eo_embed(to_host(out), dims, prec, p), dims, prec, "eo")[par == p]
        want = oracle.hop(dims, Ud, pd, p, dagger=dagger)[par == p]
        assert oracle.rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f64x", "f32"])
def test_schur_operator_from_two_hops(lqlib, prec):
    """M_ee psi_e = A psi_e - H_eo A^{-1} H_oe psi_e as two hop calls (the second in place)."""
    dims = (4, 6, 4, 4)
    m = 0.05
    U, psi = _fields(dims, 400)
    Ub = F.encode_gauge(U, dims, prec, 18, "eo")
    pb = F.encode_spinor(psi, dims, prec, "eo")
    Ud = F.decode_gauge(Ub, dims, prec, 18, "eo")
    pd = F.decode_spinor(pb, dims, prec, "eo")
    A = m + 4
    pe = to_dev(eo_half(pb, dims, prec, 0))
    t_o = lqlib.dslash_hop(dims, 1, to_dev(Ub), pe, b=1.0 / A, prec=prec)
    out = lqlib.dslash_hop(dims, 0, to_dev(Ub), t_o, a=A, b=-1.0, y=pe, prec=prec)
    par = oracle.parity_of_sites(dims)
    got = F.decode_spinor(eo_embed(to_host(out), dims, prec, 0), dims, prec, "eo")[par == 0]
    want = oracle.schur_even(dims, m, Ud, pd)[par == 0]
    assert oracle.rel_l2(got, want) <= TOL[prec]


def test_gamma5_hermiticity_on_gpu_outputs(lqlib):
    """<chi, D psi> = <D^dag chi, psi> with both sides computed by the kernels."""
    dims = (8, 4, 4, 6)
    U, psi = _fields(dims, 500)
    chi = synth.gaussian_spinor(dims, seed=502)
    Ud = to_dev(F.encode_gauge(U, dims, "f64", 18, "lex"))
    Dpsi = F.decode_spinor(to_host(lqlib.dslash_apply(dims, 0.1, Ud, to_dev(F.encode_spinor(psi, dims)))), dims)
    Ddchi = F.decode_spinor(to_host(lqlib.dslash_adjoint(dims, 0.1, Ud, to_dev(F.encode_spinor(chi, dims)))), dims)
    l = np.vdot(chi.ravel(), Dpsi.ravel())
    r = np.vdot(Ddchi.ravel(), psi.ravel())
    assert abs(l - r) / abs(l) < 1e-14


@pytest.fixture(scope="module")
def big_fields():
    dims = (32, 32, 32, 32)
    U = synth.gauge_field(dims, seed=3, kind="near_identity", eps=0.3)
    psi = synth.gaussian_spinor(dims, seed=4)
    return dims, U, psi


@pytest.mark.parametrize("prec,fmt,layout", [("f32", 12, "eo"), ("f16s", 12, "eo"), ("f64", 18, "lex"),
                                             ("f64x", 18, "eo"), ("f32", 18, "eo"), ("f16s", 18, "eo"),
                                             ("i32s", 12, "eo")])
@pytest.mark.parametrize("dagger", [False, True])
def test_full_size_sampled_sites(lqlib, big_fields, prec, fmt, layout, dagger):
    """32^4 (the mixed-precision workload), in the launch configuration of the solver's
    inner operator: 256 sampled output sites, including the lattice corners, against the
    oracle's per-site stencil."""
    dims, U, psi = big_fields
    m = 0.05
    Ub = F.encode_gauge(U, dims, prec, fmt, layout)
    pb = F.encode_spinor(psi, dims, prec, layout)
    fn = lqlib.dslash_adjoint if dagger else lqlib.dslash_apply
    out = fn(dims, m, to_dev(Ub), to_dev(pb), prec=prec, link_fmt=fmt, layout=layout)
    got = F.decode_spinor(to_host(out), dims, prec, layout)
    V = synth.volume(dims)
    rng = np.random.default_rng(9)
    sites = np.unique(np.concatenate([[0, 1, V - 1, V - 2, V // 2], rng.integers(0, V, 251)]))
    Ud = F.decode_gauge(Ub, dims, prec, fmt, layout)
    pd = F.decode_spinor(pb, dims, prec, layout)
    want = oracle.dslash_sites(dims, m, Ud, pd, sites, dagger=dagger)
    assert oracle.rel_l2(got[sites], want) <= TOL[prec]


def test_bad_arguments_raise(lqlib):
    import torch
    dims = (4, 4, 4, 4)
    buf = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqlib.LqError) as e:
        lqlib.dslash_apply((4, 4, 4, 3), 0.1, buf, buf, out=buf)
    assert e.value.status == -2
    with pytest.raises(lqlib.LqError) as e:
        lqlib.dslash_apply(dims, 0.1, buf, buf, out=buf)     # out aliases psi
    assert e.value.status == -3
    out = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqlib.LqError) as e:
        lqlib.dslash_apply(dims, 0.1, buf, buf, out=out, prec="f64x", link_fmt=12)
    assert e.value.status == -1
