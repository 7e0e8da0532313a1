"""The operator on a lattice cut into t-slabs with face exchange (virtual ranks on one GPU):
bit-identical to the single-domain kernel, equal to the oracle, and faces that hold the
projected half spinors the neighbours need."""
import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,R", [((4, 4, 4, 8), 1), ((4, 4, 4, 8), 2), ((4, 4, 4, 8), 4),
                                    ((6, 4, 2, 12), 4), ((4, 4, 2, 4), 4), ((2, 2, 2, 6), 3)])
@pytest.mark.parametrize("dagger", [False, True])
def test_virtual_ranks_equal_single_domain(lqlib, dims, R, dagger):
    from paper_1904_08616_gb300.halo import VirtualRanks
    m = 0.1
    U = synth.gauge_field(dims, seed=171)
    psi = synth.gaussian_spinor(dims, seed=172)
    Ud, pd = to_dev(F.encode_gauge(U, dims)), to_dev(F.encode_spinor(psi, dims))
    out = VirtualRanks(dims, R).apply(m, Ud, pd, dagger=dagger)
    fn = lqlib.dslash_adjoint if dagger else lqlib.dslash_apply
    single = fn(dims, m, Ud, pd)
    assert np.array_equal(to_host(out), to_host(single))
    got = F.decode_spinor(to_host(out), dims)
    assert oracle.rel_l2(got, oracle.dslash(dims, m, U, psi, dagger=dagger)) <= 1e-13


@pytest.mark.parametrize("dagger", [False, True])
def test_faces_hold_the_projected_half_spinors(lqlib, dagger):
    from paper_1904_08616_gb300.halo import halo_pack
    dims = (4, 2, 2, 3)                       # one slab, local t = 0 .. 2
    U = synth.gauge_field(dims, seed=173)
    psi = synth.gaussian_spinor(dims, seed=174)
    to_prev, to_next = halo_pack(dims, to_dev(F.encode_gauge(U, dims)), to_dev(F.encode_spinor(psi, dims)),
                                 dagger=dagger)
    S = 1.0 if dagger else -1.0
    vs = dims[0] * dims[1] * dims[2]
    g4 = oracle.gamma(3)
    one = np.eye(4)
    lo = psi[:vs]                              # t = 0
    hi = psi[-vs:]                             # t = Lt - 1
    want_prev = np.einsum("ab,nbc->nac", one + S * g4, lo)[:, :2]
    proj = np.einsum("ab,nbc->nac", one - S * g4, hi)[:, :2]
    want_next = np.einsum("nBA,nsB->nsA", np.conj(U[-vs:, 3]), proj)        # U_t^dag on colour
    got_prev = to_host(to_prev).view(np.complex128).reshape(vs, 2, 3)
    got_next = to_host(to_next).view(np.complex128).reshape(vs, 2, 3)
    assert np.abs(got_prev - want_prev).max() < 1e-14
    assert np.abs(got_next - want_next).max() < 1e-13


def test_halo_argument_checks(lqlib):
    from paper_1904_08616_gb300 import LqError
    from paper_1904_08616_gb300.halo import face_bytes, halo_pack
    assert face_bytes((4, 4, 2, 3)) == 4 * 4 * 2 * 96
    assert face_bytes((3, 4, 2, 2)) == 0                         # x must be even
    dims = (4, 4, 2, 2)
    U = to_dev(F.encode_gauge(synth.gauge_field(dims, seed=1), dims))
    psi = to_dev(F.encode_spinor(synth.gaussian_spinor(dims, seed=2), dims))
    face = to_dev(np.zeros(face_bytes(dims), np.uint8))
    with pytest.raises(LqError):
        halo_pack(dims, U, psi, to_prev=face, to_next=face)     # the two faces overlap
