"""The seeded input generators: SU(3) links that are Haar-distributed, and the chunked,
parallel draw used for large lattices (deterministic, independent chunks)."""
import numpy as np
import pytest

import synth


def _unitary_det1(u):
    eye = np.eye(3)
    uu = np.einsum("nij,nkj->nik", u, np.conj(u))
    assert np.abs(uu - eye).max() < 1e-13
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-13


def test_haar_moments():
    """Haar measure on SU(3): E[U_ij] = 0, E|U_ij|^2 = 1/3, E|tr U|^2 = 1, E|tr U|^4 = 2
    (the trivial representation occurs once in V (x) V*, twice in (V (x) V*)^2).  A QR
    without the phase fix, or a determinant fixed by the wrong root, moves these."""
    u = synth.haar_su3(synth.make_rng(11), 1 << 16)
    _unitary_det1(u)
    assert abs(u[:, 0, 0].mean()) < 0.01
    assert abs((np.abs(u) ** 2).mean() - 1 / 3) < 0.003
    tr2 = np.abs(np.trace(u, axis1=1, axis2=2)) ** 2
    assert abs(tr2.mean() - 1.0) < 0.03
    assert abs((tr2 ** 2).mean() - 2.0) < 0.12


def test_near_identity_is_close_to_one():
    u = synth.near_identity_su3(synth.make_rng(12), 4096, 0.3)
    _unitary_det1(u)
    d = np.abs(u - np.eye(3)).max(axis=(1, 2))
    assert d.max() < 1.5 and d.mean() < 0.6


@pytest.mark.parametrize("kind", ["haar", "near_identity"])
def test_chunked_draw_is_deterministic_and_independent(kind):
    dims = (4, 4, 4, 6)                     # 1536 links, chunks of 256
    a = synth.gauge_field(dims, 5, kind=kind, chunk=256, workers=1)
    b = synth.gauge_field(dims, 5, kind=kind, chunk=256, workers=3)
    assert np.array_equal(a, b)
    _unitary_det1(a.reshape(-1, 3, 3))
    flat = a.reshape(-1, 3, 3)
    # chunk 0 is the plain stream of the seed; later chunks come from jumped streams
    first = synth._links(kind, 0.3, 5, 0, 256)
    assert np.array_equal(flat[:256], first)
    for k in range(1, 6):
        assert not np.allclose(flat[256 * k:256 * (k + 1)], first)
    # a field that fits in one chunk is the one-piece draw
    c = synth.gauge_field((4, 4, 4, 4), 5, kind=kind)
    d = synth.gauge_field((4, 4, 4, 4), 5, kind=kind, chunk=1024)
    assert np.array_equal(c, d)
