"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each test ties the oracle to something other than its own formula: Clifford algebra of the
gamma basis, an independently assembled dense matrix, the closed-form free-field action
and spectrum, gamma5-hermiticity, gauge covariance, the staggered-sign identity, the
SU(3) cofactor identity, dense linear solves and the counts the paper prints.
"""
import json
import math
import os
from itertools import product

import numpy as np
import pytest

import oracle
import synth
from oracle import dense
from oracle import formats as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inner(a, b):
    return np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())


def _gamma5_apply(psi):
    g5 = dense.gamma5()
    return np.einsum("ab,nbc->nac", g5, psi)


# ----------------------------------------------------------------------------- gammas
def test_gamma_clifford_and_hermitian():
    g = [oracle.gamma(mu) for mu in range(4)]
    one = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * one * (mu == nu), atol=0)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)
    # the dense brute force builds its own copy of the basis: they must agree
    for mu in range(4):
        assert np.array_equal(g[mu], dense.gammas()[mu])


# ----------------------------------------------------------------------------- dense
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6), (4, 2, 6, 2)])
def test_stencil_equals_dense_matrix(dims):
    """Eq. (1) as a stencil equals the independently assembled (12V)x(12V) matrix."""
    U = synth.gauge_field(dims, seed=11)
    m = 0.1
    Dd = dense.dense_dirac(dims, m, U)
    V = synth.volume(dims)
    psi = synth.gaussian_spinor(dims, seed=12)
    got = oracle.dslash(dims, m, U, psi)
    assert oracle.rel_l2(got.ravel(), Dd @ psi.ravel()) < 1e-15
    # D^dag equals the conjugate transpose of the dense matrix
    gotd = oracle.dslash(dims, m, U, psi, dagger=True)
    assert oracle.rel_l2(gotd.ravel(), Dd.conj().T @ psi.ravel()) < 1e-15
    # column by column on a few basis vectors, including the wrap-around sites
    for col in (0, 5, 12 * (V - 1) + 11, 12 * (V // 2) + 7):
        e = np.zeros(12 * V, np.complex128)
        e[col] = 1.0
        got = oracle.dslash(dims, m, U, e.reshape(V, 4, 3)).ravel()
        assert np.max(np.abs(got - Dd[:, col])) < 1e-15


def test_dense_4x4x4x4_sampled_columns():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, seed=13)
    m = 0.1
    Dd = dense.dense_dirac(dims, m, U)
    psi = synth.gaussian_spinor(dims, seed=14)
    assert oracle.rel_l2(oracle.dslash(dims, m, U, psi).ravel(), Dd @ psi.ravel()) < 1e-15


# ----------------------------------------------------------------------------- free field
def test_free_field_plane_wave_closed_form():
    """U = 1, psi(n) = exp(i p.n) u:
    D psi = exp(i p.n) [ (m + 4 + sum cos p_mu) u - i sum sin p_mu gamma_mu u ],
    D^dag psi flips the sign of the gamma term."""
    dims = (4, 6, 4, 8)
    m = 0.37
    U = synth.unit_gauge_field(dims)
    V = synth.volume(dims)
    rng = np.random.default_rng(5)
    g = dense.gammas()
    lx, ly, lz, lt = dims
    n = np.arange(V)
    coords = np.stack([n % lx, (n // lx) % ly, (n // (lx * ly)) % lz, n // (lx * ly * lz)], 1)
    for _ in range(4):
        k = [rng.integers(0, L) for L in dims]
        p = np.array([2 * math.pi * k[mu] / dims[mu] for mu in range(4)])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * coords @ p)
        psi = phase[:, None, None] * u[None]
        mom = (m + 4 + np.cos(p).sum()) * u
        gs = sum(np.sin(p[mu]) * g[mu] for mu in range(4))
        want = phase[:, None, None] * (mom - 1j * gs @ u)[None]
        wantd = phase[:, None, None] * (mom + 1j * gs @ u)[None]
        assert oracle.rel_l2(oracle.dslash(dims, m, U, psi), want) < 1e-14
        assert oracle.rel_l2(oracle.dslash(dims, m, U, psi, dagger=True), wantd) < 1e-14


def test_free_field_constant_spinor():
    dims = (2, 4, 2, 4)
    m = 0.1
    U = synth.unit_gauge_field(dims)
    psi = np.ones((synth.volume(dims), 4, 3), np.complex128) * (0.3 - 0.7j)
    assert oracle.rel_l2(oracle.dslash(dims, m, U, psi), (m + 8) * psi) < 1e-15


def test_free_field_spectrum_2222():
    """On 2^4 every momentum is 0 or pi, so the spectrum is m + 8 - 2j with multiplicity
    12 * C(4, j); this needs the two hops on an extent-2 axis to add."""
    dims = (2, 2, 2, 2)
    m = 0.1
    Dd = dense.dense_dirac(dims, m, synth.unit_gauge_field(dims))
    ev = np.sort(np.linalg.eigvals(Dd).real)
    want = np.sort(np.concatenate([np.full(12 * math.comb(4, j), m + 8 - 2 * j) for j in range(5)]))
    assert np.max(np.abs(ev - want)) < 1e-12


def test_free_field_spectrum_closed_form_4444():
    dims = (4, 4, 4, 4)
    m = 0.05
    Dd = dense.dense_dirac(dims, m, synth.unit_gauge_field(dims))
    ev = np.linalg.eigvals(Dd)
    want = []
    for k in product(range(4), repeat=4):
        p = 2 * math.pi * np.array(k) / 4
        re = m + 4 + np.cos(p).sum()
        im = math.sqrt(max((np.sin(p) ** 2).sum(), 0.0))
        want += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    got = sorted(ev, key=key)
    want = sorted(want, key=key)
    assert np.max(np.abs(np.array(got) - np.array(want))) < 1e-10


# ----------------------------------------------------------------------------- symmetries
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 8)])
def test_gamma5_hermiticity(dims):
    U = synth.gauge_field(dims, seed=21)
    m = 0.1
    psi = synth.gaussian_spinor(dims, seed=22)
    chi = synth.gaussian_spinor(dims, seed=23)
    lhs = _inner(chi, oracle.dslash(dims, m, U, psi))
    g5Dg5chi = _gamma5_apply(oracle.dslash(dims, m, U, _gamma5_apply(chi)))
    rhs = _inner(g5Dg5chi, psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    # the explicit D^dag route and the gamma5 D gamma5 route agree
    assert oracle.rel_l2(oracle.dslash(dims, m, U, chi, dagger=True), g5Dg5chi) < 1e-14
    # and D^dag is the adjoint of D
    rhs2 = _inner(oracle.dslash(dims, m, U, chi, dagger=True), psi)
    assert abs(lhs - rhs2) / abs(lhs) < 1e-14


def test_gauge_covariance():
    dims = (4, 2, 4, 6)
    V = synth.volume(dims)
    U = synth.gauge_field(dims, seed=31)
    psi = synth.gaussian_spinor(dims, seed=32)
    om = synth.haar_su3(synth.make_rng(33), V)
    m = 0.2
    Up = np.empty_like(U)
    for mu in range(4):
        fwd = dense.shift_index(dims, mu, +1)
        Up[:, mu] = om @ U[:, mu] @ om[fwd].conj().transpose(0, 2, 1)
    psip = np.einsum("nab,nsb->nsa", om, psi)
    for dag in (False, True):
        lhs = oracle.dslash(dims, m, Up, psip, dagger=dag)
        rhs = np.einsum("nab,nsb->nsa", om, oracle.dslash(dims, m, U, psi, dagger=dag))
        assert oracle.rel_l2(lhs, rhs) < 1e-14


def test_staggered_sign_identity():
    """S D(m) S = 2(m+4) - D(m) with S = (-1)^(x+y+z+t): the hopping term flips sign."""
    dims = (4, 6, 2, 4)
    U = synth.gauge_field(dims, seed=41)
    psi = synth.gaussian_spinor(dims, seed=42)
    m = 0.3
    s = 1 - 2 * oracle.parity_of_sites(dims)
    lhs = s[:, None, None] * oracle.dslash(dims, m, U, s[:, None, None] * psi)
    rhs = 2 * (m + 4) * psi - oracle.dslash(dims, m, U, psi)
    assert oracle.rel_l2(lhs, rhs) < 1e-14


def test_linear_in_mass():
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, seed=43)
    psi = synth.gaussian_spinor(dims, seed=44)
    d = oracle.dslash(dims, 0.7, U, psi) - oracle.dslash(dims, -0.2, U, psi)
    assert oracle.rel_l2(d, 0.9 * psi) < 1e-14


def test_sampled_sites_match_full():
    dims = (4, 6, 4, 2)
    U = synth.gauge_field(dims, seed=45)
    psi = synth.gaussian_spinor(dims, seed=46)
    full = oracle.dslash(dims, 0.1, U, psi, dagger=True)
    sites = [0, 3, 17, synth.volume(dims) - 1]
    got = oracle.dslash_sites(dims, 0.1, U, psi, sites, dagger=True)
    assert np.array_equal(got, full[sites])


# ----------------------------------------------------------------------------- links
def test_generators_give_su3():
    for kind, eps in (("haar", 0.0), ("near_identity", 0.3)):
        U = synth.gauge_field((2, 2, 2, 4), seed=3, kind=kind, eps=eps).reshape(-1, 3, 3)
        uu = U @ U.conj().transpose(0, 2, 1)
        assert np.max(np.abs(uu - np.eye(3))) < 1e-14
        assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-14


def test_generators_deterministic():
    a = synth.gauge_field((2, 2, 2, 2), seed=9)
    b = synth.gauge_field((2, 2, 2, 2), seed=9)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.gauge_field((2, 2, 2, 2), seed=10))


def test_reconstruct12_exact_for_su3():
    U = synth.haar_su3(synth.make_rng(51), 500)
    rec = oracle.reconstruct12(U[:, :2, :])
    assert np.max(np.abs(rec - U)) < 1e-14
    # a U(3) matrix with det != 1 is not reproduced: the identity needs det = 1
    ph = np.exp(0.3j)
    rec2 = oracle.reconstruct12((U * ph)[:, :2, :])
    assert np.max(np.abs(rec2[:, 2] - (U * ph)[:, 2])) > 1e-2


def test_dslash_with_reconstructed_links():
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, seed=52)
    psi = synth.gaussian_spinor(dims, seed=53)
    rec = oracle.reconstruct12(U[:, :, :2, :])
    assert oracle.rel_l2(oracle.dslash(dims, 0.1, rec, psi), oracle.dslash(dims, 0.1, U, psi)) < 1e-14


# ----------------------------------------------------------------------------- solvers
@pytest.mark.parametrize("dims,kind", [((2, 2, 2, 2), "haar"), ((4, 4, 4, 4), "haar"),
                                       ((4, 4, 2, 2), "near_identity")])
def test_cg_against_dense_solve(dims, kind):
    m = 0.1
    U = synth.gauge_field(dims, seed=61, kind=kind, eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=62)
    x, it, rel = oracle.cg(dims, m, U, eta, tol=1e-10)
    assert rel <= 1e-10
    Dd = dense.dense_dirac(dims, m, U)
    A = Dd.conj().T @ Dd
    xd = np.linalg.solve(A, eta.ravel())
    cond = np.linalg.cond(A)
    assert oracle.rel_l2(x.ravel(), xd) < 1e-10 * cond
    # true residual recomputed here from the dense matrix
    assert np.linalg.norm(eta.ravel() - A @ x.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10


@pytest.mark.parametrize("low,delta", [("f64", 1e-2), ("f32", 1e-3), ("f32", 0.1)])
def test_alg1_converges_to_cg_solution(low, delta):
    dims = (4, 4, 2, 4)
    m = 0.05
    U = synth.gauge_field(dims, seed=71, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=72)
    x, cycles, inner, rel = oracle.alg1(dims, m, U, eta, tol=1e-10, low=low, delta=delta)
    assert rel <= 1e-10
    assert cycles >= 2 and inner > 0
    Dd = dense.dense_dirac(dims, m, U)
    A = Dd.conj().T @ Dd
    assert np.linalg.norm(eta.ravel() - A @ x.ravel()) / np.linalg.norm(eta.ravel()) <= 1e-10
    xc, _, _ = oracle.cg(dims, m, U, eta, tol=1e-12)
    assert oracle.rel_l2(x, xc) < 1e-10 * np.linalg.cond(A)


def test_alg1_single_cycle_is_cg():
    """With an FP64 inner loop and delta below the target, Algorithm 1 is plain CG: one
    cycle, and the same iterates as the textbook solver."""
    dims = (2, 2, 2, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=73)
    eta = synth.gaussian_spinor(dims, seed=74)
    x, cycles, inner, rel = oracle.alg1(dims, m, U, eta, tol=1e-10, low="f64", delta=1e-14)
    xc, itc, relc = oracle.cg(dims, m, U, eta, tol=1e-10)
    assert cycles == 1
    assert inner == itc
    assert oracle.rel_l2(x, xc) < 1e-12


# ----------------------------------------------------------------------------- even-odd
def test_hopping_connects_opposite_parity_only():
    dims = (4, 2, 4, 2)
    m = 0.4
    U = synth.gauge_field(dims, seed=81)
    psi = synth.gaussian_spinor(dims, seed=82)
    par = oracle.parity_of_sites(dims)
    for p in (0, 1):
        src = psi.copy()
        src[par != p] = 0
        out = oracle.dslash(dims, m, U, src)
        assert oracle.rel_l2(out[par == p], (m + 4) * psi[par == p]) < 1e-15


def test_schur_complement_solves_full_system():
    dims = (2, 2, 2, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=83)
    V = synth.volume(dims)
    b = synth.gaussian_spinor(dims, seed=84)
    par = oracle.parity_of_sites(dims)
    Dd = dense.dense_dirac(dims, m, U)
    x = np.linalg.solve(Dd, b.ravel()).reshape(V, 4, 3)
    a = m + 4
    # M_ee x_e = b_e - H_eo A^{-1} b_o
    b_o = b.copy()
    b_o[par == 0] = 0
    rhs = b.copy()
    rhs[par == 1] = 0
    rhs = rhs - oracle.hop(dims, U, b_o / a, 0)
    x_e = x.copy()
    x_e[par == 1] = 0
    lhs = oracle.schur_even(dims, m, U, x_e)
    assert oracle.rel_l2(lhs[par == 0], rhs[par == 0]) < 1e-13
    # x_o = A^{-1}(b_o - H_oe x_e)
    xo = (b_o - oracle.hop(dims, U, x_e, 1)) / a
    assert oracle.rel_l2(xo[par == 1], x[par == 1]) < 1e-13
    # the adjoint Schur operator is the adjoint
    y = synth.gaussian_spinor(dims, seed=85)
    y[par == 1] = 0
    l1 = _inner(y, oracle.schur_even(dims, m, U, x_e))
    l2 = _inner(oracle.schur_even(dims, m, U, y, dagger=True), x_e)
    assert abs(l1 - l2) / abs(l1) < 1e-13


# ----------------------------------------------------------------------------- formats
def test_f16s_encoding_pins():
    from oracle import formats as F
    dims = (2, 2, 2, 2)
    psi = synth.gaussian_spinor(dims, seed=91)
    psi[3] = 0.0            # an all-zero site encodes to scale 0
    buf = F.encode_spinor(psi, dims, "f16s", "lex")
    V = synth.volume(dims)
    h = buf[:48 * V].view(np.float16).reshape(V, 24)
    s = buf[48 * V:].view(np.float32)
    assert s[3] == 0 and np.all(h[3] == 0)
    # every site has one component of magnitude exactly 1 (the max-abs one)
    nz = s > 0
    assert np.all(np.max(np.abs(h[nz].astype(np.float32)), axis=1) == 1.0)
    dec = F.decode_spinor(buf, dims, "f16s", "lex")
    assert oracle.rel_l2(dec, psi) < 1e-3


def test_i32s_encoding_pins():
    """32-bit fixed point (Q1.30 with a per-site scale): zero sites encode to zero; the
    largest component of a site encodes to 2^30 up to the FP32 rounding of the scale; every
    stored value is within half a quantum (s 2^-31) of the input."""
    from oracle import formats as F
    dims = (2, 2, 2, 2)
    psi = synth.gaussian_spinor(dims, seed=94) * np.exp(np.linspace(-20, 20, 16))[:, None, None]
    psi[5] = 0.0
    buf = F.encode_spinor(psi, dims, "i32s", "lex")
    V = synth.volume(dims)
    assert buf.size == 100 * V
    q = buf[:96 * V].view(np.int32).reshape(V, 24)
    s = buf[96 * V:].view(np.float32).astype(np.float64)
    assert s[5] == 0 and np.all(q[5] == 0)
    qmax = np.max(np.abs(q.astype(np.int64)), axis=1)
    nz = s > 0
    assert np.all(np.abs(qmax[nz] - 2 ** 30) <= 2 ** 7)
    reals = np.ascontiguousarray(psi).view(np.float64).reshape(V, 24)
    dec = F.decode_spinor(buf, dims, "i32s", "lex")
    err = np.abs(np.ascontiguousarray(dec).view(np.float64).reshape(V, 24) - reals)
    assert np.all(err <= (s * 2.0 ** -31)[:, None] * (1 + 1e-9))
    # links: Q1.30 without a scale, error <= 2^-31 per entry
    U = synth.gauge_field(dims, seed=95)
    Ud = F.decode_gauge(F.encode_gauge(U, dims, "i32s", 18, "lex"), dims, "i32s", 18, "lex")
    assert np.abs(Ud - U).max() <= 2.0 ** -31 * np.sqrt(2) * (1 + 1e-9)


def test_eo_layout_roundtrip_and_parity_blocks():
    from oracle import formats as F
    dims = (4, 2, 2, 6)
    psi = synth.gaussian_spinor(dims, seed=92)
    U = synth.gauge_field(dims, seed=93)
    for prec in F.PRECS:
        b = F.encode_spinor(psi, dims, prec, "eo")
        assert np.array_equal(F.decode_spinor(b, dims, prec, "eo"),
                              F.decode_spinor(F.encode_spinor(psi, dims, prec, "lex"), dims, prec, "lex"))
        for fmt in (18, 12):
            g = F.encode_gauge(U, dims, prec, fmt, "eo")
            assert np.array_equal(F.decode_gauge(g, dims, prec, fmt, "eo"),
                                  F.decode_gauge(F.encode_gauge(U, dims, prec, fmt, "lex"), dims, prec, fmt, "lex"))
    # the first half of an f64 eo spinor holds exactly the even sites
    b = F.encode_spinor(psi, dims, "f64", "eo").view(np.float64)
    par = oracle.parity_of_sites(dims)
    V = synth.volume(dims)
    even = b[: 12 * V].reshape(12, V // 2, 2)
    assert np.array_equal(np.sort(even.ravel()), np.sort(psi[par == 0].view(np.float64).ravel()))


# ----------------------------------------------------------------------------- paper counts
def test_paper_stencil_counts():
    """360 input words per stencil = 8 links x 18 + 9 spinors x 24 (Introduction)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    words = g["links_per_stencil"] * g["words_per_link_full"] + g["spinors_per_stencil"] * 24
    assert words == g["words_per_stencil"] == 360
    assert 8 * words == g["bytes_per_stencil_f64"]
    assert sum(g["stage_cycles"]) == g["latency_cycles"]
    # stage 3: 8 directions x 2 half-spinors x 9 complex multiply-adds x 8 real operations
    assert 8 * 2 * 9 * 8 == g["stage3_ops"]


@pytest.mark.parametrize("delta", [1e-1, 1e-2])
def test_alg1_fp64_restarts_continue_cg(delta):
    """In exact arithmetic the restart p_0 = r_0 + beta_0 (p_k - <r_0,p_k> r_0) with
    beta_0 = s_l / (s_{l-1} rho_k) is the CG direction p_k rescaled into the new units, so
    with an FP64 inner loop the restarted solver takes the same iterations as plain CG.
    A wrong beta_0 or a missing projection breaks the conjugacy and costs iterations."""
    dims = (4, 4, 2, 4)
    m = 0.05
    U = synth.gauge_field(dims, seed=71, kind="near_identity", eps=0.3)
    eta = synth.gaussian_spinor(dims, seed=72)
    _, itc, _ = oracle.cg(dims, m, U, eta, tol=1e-10)
    _, cycles, inner, rel = oracle.alg1(dims, m, U, eta, tol=1e-10, low="f64", delta=delta)
    assert cycles >= 4
    assert abs(inner - itc) <= 1
    assert rel <= 1e-10


# ----------------------------------------------------------------------------- gradients
def test_link_grad_matches_finite_differences():
    """L = Re <g, D(U) psi> is linear in U, so a central difference is exact up to
    rounding; compare every component of a few links."""
    dims = (2, 4, 2, 2)
    m = 0.3
    U = synth.gauge_field(dims, seed=95)
    psi = synth.gaussian_spinor(dims, seed=96)
    g = synth.gaussian_spinor(dims, seed=97)
    G = oracle.link_grad(dims, g, psi)
    L = lambda UU: np.vdot(g.ravel(), oracle.dslash(dims, m, UU, psi).ravel()).real
    h = 1e-3
    rng = np.random.default_rng(98)
    for _ in range(12):
        n, mu, A, B = rng.integers(0, synth.volume(dims)), rng.integers(0, 4), rng.integers(0, 3), rng.integers(0, 3)
        for part in (1.0, 1j):
            Up = U.copy()
            Um = U.copy()
            Up[n, mu, A, B] += h * part
            Um[n, mu, A, B] -= h * part
            fd = (L(Up) - L(Um)) / (2 * h)
            want = G[n, mu, A, B].real if part == 1.0 else G[n, mu, A, B].imag
            assert abs(fd - want) < 1e-9 * max(1.0, abs(want))


def test_solve_grads_match_dense_finite_differences():
    """L = Re <chi, (D^dag D)^{-1} eta> on 2^4 with dense solves: the oracle's adjoint
    gradients against central differences of the dense solution."""
    dims = (2, 2, 2, 2)
    m = 0.2
    U = synth.gauge_field(dims, seed=99, kind="near_identity", eps=0.5)
    eta = synth.gaussian_spinor(dims, seed=100)
    chi = synth.gaussian_spinor(dims, seed=101)
    g_eta, g_U = oracle.solve_grads(dims, m, U, eta, chi)

    def L(UU, ee):
        Dd = dense.dense_dirac(dims, m, UU)
        x = np.linalg.solve(Dd.conj().T @ Dd, ee.ravel())
        return np.vdot(chi.ravel(), x).real

    h = 1e-6
    rng = np.random.default_rng(102)
    for _ in range(6):
        n, mu, A, B = rng.integers(0, 16), rng.integers(0, 4), rng.integers(0, 3), rng.integers(0, 3)
        for part in (1.0, 1j):
            Up, Um = U.copy(), U.copy()
            Up[n, mu, A, B] += h * part
            Um[n, mu, A, B] -= h * part
            fd = (L(Up, eta) - L(Um, eta)) / (2 * h)
            want = g_U[n, mu, A, B].real if part == 1.0 else g_U[n, mu, A, B].imag
            assert abs(fd - want) < 1e-6 * max(1.0, abs(want))
    for _ in range(4):
        n, a, A = rng.integers(0, 16), rng.integers(0, 4), rng.integers(0, 3)
        for part in (1.0, 1j):
            ep, em = eta.copy(), eta.copy()
            ep[n, a, A] += h * part
            em[n, a, A] -= h * part
            fd = (L(U, ep) - L(U, em)) / (2 * h)
            want = g_eta[n, a, A].real if part == 1.0 else g_eta[n, a, A].imag
            assert abs(fd - want) < 1e-6 * max(1.0, abs(want))


def test_solve_d_matches_dense_solve():
    """The oracle's D x = b solve (CG on D^dag D x = D^dag b) against numpy's dense solve of
    D itself on 2^4 (a mistake in the dagger or the normal-equation right-hand side fails)."""
    dims = (2, 2, 2, 2)
    m = 0.1
    U = synth.gauge_field(dims, seed=97)
    b = synth.gaussian_spinor(dims, seed=98)
    x, _, _ = oracle.solve_d(dims, m, U, b, tol=1e-14)
    Dd = dense.dense_dirac(dims, m, U)
    xd = np.linalg.solve(Dd, dense.flat(b))
    assert np.linalg.norm(dense.flat(x) - xd) / np.linalg.norm(xd) < 1e-11


def test_projected_spin_sums_reduce_to_the_upper_half():
    """For P = 1 + S gamma_mu in the chiral basis, the lower spin half of P b is S B_mu^dag times
    its upper half, so sum_s a_s conj((P b)_s) = sum_{k=0,1} (P a)_k conj((P b)_k): the identity
    the link-gradient kernel uses to sum over two spin components instead of four."""
    rng = np.random.default_rng(31)
    for mu in range(4):
        for S in (1.0, -1.0):
            P = np.eye(4) + S * oracle.gamma(mu)
            for _ in range(4):
                a = rng.normal(size=4) + 1j * rng.normal(size=4)
                b = rng.normal(size=4) + 1j * rng.normal(size=4)
                lhs = np.sum(a * np.conj(P @ b))
                rhs = np.sum((P @ a)[:2] * np.conj((P @ b)[:2]))
                assert abs(lhs - rhs) <= 1e-13 * (1 + abs(lhs))


def test_threaded_site_loops_equal_the_serial_ones():
    """Splitting the oracle's loops over output sites across host cores (used only to time
    it) changes no bit of D psi, D^dag psi or the sampled-site values."""
    dims = (4, 6, 2, 8)
    U = synth.gauge_field(dims, seed=41)
    psi = synth.gaussian_spinor(dims, seed=42)
    sites = np.random.default_rng(43).integers(0, synth.volume(dims), 97)
    oracle.set_threads(1)
    ref = [oracle.dslash(dims, 0.1, U, psi, dagger=d) for d in (False, True)]
    ref_s = oracle.dslash_sites(dims, 0.1, U, psi, sites, dagger=True)
    try:
        used = oracle.set_threads(max(2, oracle.max_threads()))
        assert 1 <= used <= oracle.max_threads()
        got = [oracle.dslash(dims, 0.1, U, psi, dagger=d) for d in (False, True)]
        got_s = oracle.dslash_sites(dims, 0.1, U, psi, sites, dagger=True)
    finally:
        oracle.set_threads(1)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert np.array_equal(got_s, ref_s)


def test_alg1_restarts_afresh_below_the_arithmetic():
    """A tolerance of 1e-20 is below what FP64 resolves: after the true residual reaches
    rounding level (~1e-16) it no longer follows the inner recurrence, and continuing the
    old direction with beta_0 ~ 1/rho_k would let each later cycle run to its cap k (1000)
    with no progress.  Starting those cycles afresh from p_0 = r_0 keeps every cycle at
    the length of a normal one and the residual at rounding level."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, seed=1)
    eta = synth.gaussian_spinor(dims, seed=2)
    _, c4, i4, r4 = oracle.alg1(dims, 0.1, U, eta, tol=1e-20, low="f32", delta=1e-4, max_cycles=4)
    assert r4 < 1e-14
    _, c12, i12, r12 = oracle.alg1(dims, 0.1, U, eta, tol=1e-20, low="f32", delta=1e-4, max_cycles=12)
    assert c12 == 12
    assert i12 - i4 <= 8 * 2 * (i4 // 4 + 1)
    assert r12 < 1e-14


# ----------------------------------------------------------------------------- 10-real links
def _su3_from_rows(M):
    """Unit-determinant test matrices built by hand (exact in binary where possible)."""
    M = np.asarray(M, dtype=np.complex128)
    assert np.allclose(M @ M.conj().T, np.eye(3), atol=1e-15)
    assert abs(np.linalg.det(M) - 1.0) < 1e-15
    return M


def test_reconstruct10_exact_for_su3():
    """Haar and near-identity SU(3) links stored in the 10-real form come back to rounding
    level, the same as from their full 18 reals."""
    rng = synth.make_rng(301)
    for U in (synth.haar_su3(rng, 4096), synth.near_identity_su3(rng, 4096, 0.3),
              synth.near_identity_su3(rng, 4096, 0.02)):
        dims = (4, 4, 8, 8)
        U = U.reshape(1024, 4, 3, 3)
        R = F.decode_gauge(F.encode_gauge(U, dims, "f64", 10, "lex"), dims, "f64", 10, "lex")
        assert np.abs(R - U).max() < 4e-15


def test_reconstruct10_column_choice_and_recovery():
    """The stored row-1 entries are the ones outside column k (largest max(|Re|,|Im|) of
    row 0, the lowest column on ties), and the missing one is recovered exactly."""
    a = np.sqrt(0.5)
    cases = [
        # row 0 = (0, 0, 1): k = 2, row 1's (u10, u11) are stored
        (_su3_from_rows([[0, 0, 1], [1, 0, 0], [0, 1, 0]]), 2),
        # row 0 = (a, i a, 0): a tie between columns 0 and 1 goes to column 0
        (_su3_from_rows([[a, 1j * a, 0], [1j * a, a, 0], [0, 0, 1]]), 0),
        # row 0 = (0, 1, 0) up to phases: k = 1
        (_su3_from_rows([[0, 1j, 0], [1j, 0, 0], [0, 0, 1]]), 1),
        # the identity: k = 0
        (np.eye(3, dtype=np.complex128), 0),
    ]
    for M, k in cases:
        U = np.broadcast_to(M, (16, 4, 3, 3)).copy()
        dims = (2, 2, 2, 2)
        buf = F.encode_gauge(U, dims, "f64", 10, "lex")
        stored = buf.view(np.complex128).reshape(16, 4, 5)
        others = [j for j in range(3) if j != k]
        assert np.array_equal(stored[0, 0, 3:], M[1, others])
        assert np.array_equal(F.link10_column(np.ascontiguousarray(M[0]).view(np.float64), "f64"), k)
        R = F.decode_gauge(buf, dims, "f64", 10, "lex")
        assert np.abs(R - U).max() < 1e-15


def test_reconstruct10_recovers_the_orthogonal_entry():
    """Brute force on the definition: for unitary links, the recovered row-1 entry makes
    rows 0 and 1 orthogonal and row 1 a unit vector; for a matrix that is not unitary the
    form does not reproduce it (the 10 stored reals do not determine a general matrix)."""
    rng = synth.make_rng(303)
    U = synth.haar_su3(rng, 64)
    R = oracle.reconstruct10(np.concatenate([U[:, 0, :], U[:, 1, 1:]], axis=-1))   # k = 0 assumed
    k = F.link10_column(np.ascontiguousarray(U[:, 0, :]).view(np.float64).reshape(64, 6), "f64")
    sel = k == 0
    assert sel.any()
    assert np.abs(R[sel] - U[sel]).max() < 4e-15
    assert np.abs(np.einsum("nj,nj->n", R[:, 1, :], R[:, 0, :].conj())).max() < 1e-14
    assert np.abs(np.linalg.norm(R[sel, 1, :], axis=-1) - 1).max() < 1e-14
    M = (rng.normal(size=(64, 3, 3)) + 1j * rng.normal(size=(64, 3, 3)))
    dims = (2, 2, 2, 2)
    Mr = F.decode_gauge(F.encode_gauge(M.reshape(16, 4, 3, 3), dims, "f64", 10, "lex"), dims, "f64", 10, "lex")
    assert np.abs(Mr - M.reshape(16, 4, 3, 3)).max() > 1e-3


def _su3_with_first_row(v, rng):
    """SU(3) matrices whose row 0 is the unit vector v up to a phase (QR completion)."""
    n = v.shape[0]
    M = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    M[:, :, 0] = v.conj()
    Q, _ = np.linalg.qr(M)
    U = Q.conj().transpose(0, 2, 1)
    return U / (np.linalg.det(U) ** (1.0 / 3.0))[:, None, None]


def test_reconstruct10_conditioning_fp32():
    """Stored in FP32 (rounding <= 2^-24 relative per real), the rebuilt entries stay within
    a fixed multiple of the storage rounding, also for rows 0 with vanishing entries: the
    division is by the chosen |u0k| >= 1/sqrt(6)."""
    rng = synth.make_rng(305)
    n = 1 << 12
    v = rng.normal(size=(n, 3)) + 1j * rng.normal(size=(n, 3))
    v[np.arange(n), rng.integers(0, 3, n)] *= 1e-7                # one entry of row 0 nearly zero
    v[: n // 2][np.arange(n // 2), rng.integers(0, 3, n // 2)] *= 1e-7   # and half of them a second one
    v /= np.linalg.norm(v, axis=1)[:, None]
    allU = np.concatenate([synth.haar_su3(rng, 1 << 14), _su3_with_first_row(v, rng)])
    m = allU.shape[0] // 4
    allU = allU.reshape(m, 4, 3, 3)
    dims = (m, 1, 1, 1)
    R = F.decode_gauge(F.encode_gauge(allU, dims, "f32", 10, "lex"), dims, "f32", 10, "lex")
    assert np.abs(R - allU).max() <= 64 * 2.0 ** -24
    row0 = np.ascontiguousarray(allU[..., 0, :]).view(np.float64).astype(np.float32)
    k = F.link10_column(row0, "f32")
    mag = np.abs(np.take_along_axis(allU[..., 0, :], k[..., None], axis=-1))
    assert mag.min() >= 1 / np.sqrt(6) - 1e-7


def test_dslash_with_10real_links():
    """D with links rebuilt from their 10 stored reals equals D with the full links."""
    dims = (4, 4, 2, 6)
    U = synth.gauge_field(dims, seed=307)
    psi = synth.gaussian_spinor(dims, seed=308)
    R = F.decode_gauge(F.encode_gauge(U, dims, "f64", 10, "eo"), dims, "f64", 10, "eo")
    for dag in (False, True):
        assert oracle.rel_l2(oracle.dslash(dims, 0.1, R, psi, dag), oracle.dslash(dims, 0.1, U, psi, dag)) < 1e-14
