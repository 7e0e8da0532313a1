"""Seeded synthetic lattice fields: gauge links and spinors.

This module only draws random numbers and shapes them into the input fields that both the
CPU oracle and the CUDA path consume. It holds none of the operator's arithmetic.

Conventions shared with every consumer (all in lexicographic site order
``n = x + Lx*(y + Ly*(z + Lz*t))``, x fastest, direction mu = 0..3 <-> x, y, z, t):

* gauge field: complex128 array ``(V, 4, 3, 3)`` = ``[site][mu][row][col]``; viewed as
  float64 it is ``[site][mu][row][col][re, im]`` (18 reals per link).
* spinor field: complex128 array ``(V, 4, 3)`` = ``[site][spin][colour]``; as float64,
  ``[site][spin][colour][re, im]`` (24 reals per site).

The paper's workloads are lattice volumes of 10^6 to 10^8 sites (Introduction) and a
12 x 8^3 on-chip lattice (Section 2.1); it uses no public dataset and no gauge ensemble,
so these seeded fields stand in for them.
"""
from __future__ import annotations

import os

import numpy as np

__all__ = [
    "volume",
    "make_rng",
    "haar_su3",
    "near_identity_su3",
    "gauge_field",
    "unit_gauge_field",
    "gaussian_spinor",
    "as_reals",
    "as_complex_gauge",
    "as_complex_spinor",
]


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def make_rng(seed: int) -> np.random.Generator:
    """NumPy PCG64 generator for a given integer seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex Gaussian with Re and Im drawn independently from N(0, 1)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-distributed SU(3) matrices, shape (n, 3, 3).

    QR of a complex Gaussian matrix, with the phases of R's diagonal moved into Q (the
    Mezzadri fix, which makes Q Haar on U(3)), then divided by the principal cube root of
    det(Q) so the determinant is exactly one up to rounding.
    """
    g = _complex_gaussian(rng, (n, 3, 3))
    q, r = np.linalg.qr(g)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / np.exp(1j * np.angle(det) / 3.0)[:, None, None]
    return q


def near_identity_su3(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """n links exp(i*eps*H), H random traceless Hermitian, shape (n, 3, 3).

    H = (G + G^dag)/2 - tr(.)/3 with G complex Gaussian; the exponential is taken through
    the eigen-decomposition of H, so U is unitary with det U = exp(i*eps*tr H) = 1.
    """
    g = _complex_gaussian(rng, (n, 3, 3))
    h = 0.5 * (g + np.conj(np.swapaxes(g, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real
    h = h - (tr / 3.0)[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("nij,nj,nkj->nik", v, ph, np.conj(v))


# Links drawn in one piece up to this many; larger fields are drawn in chunks of this size,
# chunk k from the PCG64 stream of the seed jumped k times (chunk 0 is the plain stream), so
# every field up to 32^4 sites is the one-piece draw and larger ones can be drawn in parallel.
LINK_CHUNK = 1 << 22


def _links(kind: str, eps: float, seed: int, k: int, n: int) -> np.ndarray:
    bitgen = np.random.PCG64(int(seed))
    rng = np.random.Generator(bitgen if k == 0 else bitgen.jumped(k))
    if kind == "haar":
        return haar_su3(rng, n)
    if kind == "near_identity":
        return near_identity_su3(rng, n, eps)
    raise ValueError(f"unknown gauge kind {kind!r}")


def _links_task(args):
    return args[3], _links(*args)


def gauge_field(dims, seed: int, kind: str = "haar", eps: float = 0.3, chunk: int = LINK_CHUNK,
                workers: int | None = None) -> np.ndarray:
    """A seeded gauge field, complex128 (V, 4, 3, 3).

    kind = "haar": Haar-random SU(3) on every link (maximally rough, strong coupling).
    kind = "near_identity": exp(i*eps*H) on every link (close to the free field).
    Fields of more than ``chunk`` links are drawn chunk by chunk (see LINK_CHUNK), on a pool
    of ``workers`` spawned processes (default: the CPU count, at most 16).
    """
    v = volume(dims)
    if kind not in ("haar", "near_identity"):
        raise ValueError(f"unknown gauge kind {kind!r}")
    n = 4 * v
    if n <= chunk:
        u = _links(kind, eps, seed, 0, n)
        return np.ascontiguousarray(u.reshape(v, 4, 3, 3))
    out = np.empty((n, 3, 3), dtype=np.complex128)
    nchunks = (n + chunk - 1) // chunk
    tasks = [(kind, eps, seed, k, min(chunk, n - k * chunk)) for k in range(nchunks)]
    nw = workers if workers is not None else min(16, os.cpu_count() or 1)
    if nw <= 1:
        for t in tasks:
            out[t[3] * chunk:t[3] * chunk + t[4]] = _links(*t)
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(nw) as pool:
            for k, u in pool.imap_unordered(_links_task, tasks):
                out[k * chunk:k * chunk + len(u)] = u
    return out.reshape(v, 4, 3, 3)


def unit_gauge_field(dims) -> np.ndarray:
    """The free field U = 1 on every link."""
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gaussian_spinor(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Seeded complex Gaussian spinor field(s), complex128 (V, 4, 3) or (nrhs, V, 4, 3)."""
    v = volume(dims)
    rng = make_rng(seed)
    shape = (v, 4, 3) if nrhs is None else (int(nrhs), v, 4, 3)
    return _complex_gaussian(rng, shape)


def as_reals(a: np.ndarray) -> np.ndarray:
    """View a complex128 field as its interleaved float64 [re, im] storage (no copy)."""
    a = np.ascontiguousarray(a)
    return a.view(np.float64)


def as_complex_gauge(reals: np.ndarray, dims) -> np.ndarray:
    return np.ascontiguousarray(reals, dtype=np.float64).view(np.complex128).reshape(
        volume(dims), 4, 3, 3)


def as_complex_spinor(reals: np.ndarray, dims) -> np.ndarray:
    return np.ascontiguousarray(reals, dtype=np.float64).view(np.complex128).reshape(
        volume(dims), 4, 3)
