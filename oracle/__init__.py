"""CPU oracle for the Wilson-Dirac operator (Eq. 1) and CG on D^dag D (Algorithm 1).

TEST INFRASTRUCTURE ONLY.  This package is imported by the test suite, by the smoke check
and by the benchmark's CPU-baseline / reference legs, and by nothing else.  It shares no
code with the CUDA library in ``paper_1904_08616_gb300`` and never imports it.

Everything here is FP64.  The stencil, D^dag, textbook CG and Algorithm 1 live in plain C
(``oracle.c``, built with gcc by ``oracle/build.py``); this module marshals NumPy arrays
into it.  Storage-format encoders/decoders are in ``oracle.formats``; the dense
brute-force operator is in ``oracle.dense``.

Field conventions (lexicographic sites, x fastest; mu = 0..3 <-> x, y, z, t):
  gauge  complex128 (V, 4, 3, 3) = U[n][mu][row][col]
  spinor complex128 (V, 4, 3)    = psi[n][spin][colour]
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load (building first if needed) the oracle's shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            L.lq_oracle_gamma.argtypes = [ctypes.c_int, _dp]
            L.lq_oracle_volume.argtypes = [_i32p]
            L.lq_oracle_volume.restype = ctypes.c_int64
            L.lq_oracle_dslash.argtypes = [_i32p, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int]
            L.lq_oracle_dslash_sites.argtypes = [_i32p, ctypes.c_double, _dp, _dp,
                                                 ctypes.c_int64, _i64p, _dp, ctypes.c_int]
            L.lq_oracle_normal_op.argtypes = [_i32p, ctypes.c_double, _dp, _dp, _dp]
            L.lq_oracle_cg.argtypes = [_i32p, ctypes.c_double, _dp, _dp, _dp, ctypes.c_double,
                                       ctypes.c_int32, _i32p, _dp]
            L.lq_oracle_cg.restype = ctypes.c_int
            L.lq_oracle_alg1.argtypes = [_i32p, ctypes.c_double, _dp, _dp, _dp,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _dp]
            L.lq_oracle_alg1.restype = ctypes.c_int
            L.lq_oracle_reconstruct12.argtypes = [ctypes.c_int64, _dp, _dp]
            L.lq_oracle_reconstruct10.argtypes = [ctypes.c_int64, _dp, _dp]
            L.lq_oracle_max_threads.argtypes = []
            L.lq_oracle_max_threads.restype = ctypes.c_int
            L.lq_oracle_set_threads.argtypes = [ctypes.c_int]
            L.lq_oracle_set_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def max_threads() -> int:
    """Host cores the oracle's site loops can use (1 if it was built without OpenMP)."""
    return int(lib().lq_oracle_max_threads())


def set_threads(n: int) -> int:
    """Split the loops over output sites of dslash / dslash_sites (and so of normal_op, cg and
    alg1) over n threads; 1 (the default) is serial.  Results do not depend on n.  Returns
    the thread count in use."""
    return int(lib().lq_oracle_set_threads(int(n)))


def _dims(dims):
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(4))
    if np.any(d < 1):
        raise ValueError("lattice extents must be positive")
    return d


def _cptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _as_c128(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def volume(dims) -> int:
    d = _dims(dims)
    return int(np.prod(d.astype(np.int64)))


def gamma(mu: int) -> np.ndarray:
    """gamma_{mu+1} of the chiral basis used by the oracle, complex (4, 4)."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().lq_oracle_gamma(int(mu), _cptr(out.view(np.float64), ctypes.c_double))
    return out


def dslash(dims, m_q: float, U, psi, dagger: bool = False) -> np.ndarray:
    """D psi (or D^dag psi) on the whole lattice, Eq. (1); returns complex (V, 4, 3)."""
    d = _dims(dims)
    V = volume(d)
    U = _as_c128(U, (V, 4, 3, 3))
    psi = _as_c128(psi, (V, 4, 3))
    out = np.empty((V, 4, 3), dtype=np.complex128)
    lib().lq_oracle_dslash(_cptr(d, ctypes.c_int32), float(m_q),
                           _cptr(U.view(np.float64), ctypes.c_double),
                           _cptr(psi.view(np.float64), ctypes.c_double),
                           _cptr(out.view(np.float64), ctypes.c_double), int(bool(dagger)))
    return out


def dslash_sites(dims, m_q: float, U, psi, sites, dagger: bool = False) -> np.ndarray:
    """(D psi)(n) for the lexicographic sites n in ``sites``; returns complex (k, 4, 3)."""
    d = _dims(dims)
    V = volume(d)
    U = _as_c128(U, (V, 4, 3, 3))
    psi = _as_c128(psi, (V, 4, 3))
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64).reshape(-1))
    if s.size and (s.min() < 0 or s.max() >= V):
        raise ValueError("site index out of range")
    out = np.empty((s.size, 4, 3), dtype=np.complex128)
    lib().lq_oracle_dslash_sites(_cptr(d, ctypes.c_int32), float(m_q),
                                 _cptr(U.view(np.float64), ctypes.c_double),
                                 _cptr(psi.view(np.float64), ctypes.c_double),
                                 ctypes.c_int64(s.size), _cptr(s, ctypes.c_int64),
                                 _cptr(out.view(np.float64), ctypes.c_double),
                                 int(bool(dagger)))
    return out


def normal_op(dims, m_q: float, U, psi) -> np.ndarray:
    """D^dag D psi."""
    d = _dims(dims)
    V = volume(d)
    U = _as_c128(U, (V, 4, 3, 3))
    psi = _as_c128(psi, (V, 4, 3))
    out = np.empty((V, 4, 3), dtype=np.complex128)
    lib().lq_oracle_normal_op(_cptr(d, ctypes.c_int32), float(m_q),
                              _cptr(U.view(np.float64), ctypes.c_double),
                              _cptr(psi.view(np.float64), ctypes.c_double),
                              _cptr(out.view(np.float64), ctypes.c_double))
    return out


def cg(dims, m_q: float, U, eta, x0=None, tol: float = 1e-10, max_iter: int = 100000):
    """Textbook CG on D^dag D x = eta.  Returns (x, iterations, true relative residual)."""
    d = _dims(dims)
    V = volume(d)
    U = _as_c128(U, (V, 4, 3, 3))
    eta = _as_c128(eta, (V, 4, 3))
    x = np.zeros((V, 4, 3), np.complex128) if x0 is None else _as_c128(x0, (V, 4, 3)).copy()
    it = np.zeros(1, np.int32)
    rel = np.zeros(1, np.float64)
    lib().lq_oracle_cg(_cptr(d, ctypes.c_int32), float(m_q),
                       _cptr(U.view(np.float64), ctypes.c_double),
                       _cptr(eta.view(np.float64), ctypes.c_double),
                       _cptr(x.view(np.float64), ctypes.c_double), float(tol), int(max_iter),
                       _cptr(it, ctypes.c_int32), _cptr(rel, ctypes.c_double))
    return x, int(it[0]), float(rel[0])


def alg1(dims, m_q: float, U, eta, x0=None, tol: float = 1e-10, low: str = "f32",
         delta: float = 1e-3, k_max: int = 1000, max_cycles: int = 200):
    """Algorithm 1 (residual-guided mixed-precision CG), low = "f32" or "f64".

    Returns (x, cycles, total inner iterations, true relative residual).
    """
    d = _dims(dims)
    V = volume(d)
    U = _as_c128(U, (V, 4, 3, 3))
    eta = _as_c128(eta, (V, 4, 3))
    x = np.zeros((V, 4, 3), np.complex128) if x0 is None else _as_c128(x0, (V, 4, 3)).copy()
    cyc = np.zeros(1, np.int32)
    inner = np.zeros(1, np.int32)
    rel = np.zeros(1, np.float64)
    if low not in ("f32", "f64"):
        raise ValueError("low must be 'f32' or 'f64'")
    lib().lq_oracle_alg1(_cptr(d, ctypes.c_int32), float(m_q),
                         _cptr(U.view(np.float64), ctypes.c_double),
                         _cptr(eta.view(np.float64), ctypes.c_double),
                         _cptr(x.view(np.float64), ctypes.c_double), float(tol),
                         int(low == "f32"), float(delta), int(k_max), int(max_cycles),
                         _cptr(cyc, ctypes.c_int32), _cptr(inner, ctypes.c_int32),
                         _cptr(rel, ctypes.c_double))
    return x, int(cyc[0]), int(inner[0]), float(rel[0])


def reconstruct12(rows) -> np.ndarray:
    """Full 3x3 links from their first two rows: row 2 = conj(row0 x row1).

    rows: complex (..., 2, 3); returns complex (..., 3, 3).
    """
    rows = np.ascontiguousarray(rows, dtype=np.complex128)
    lead = rows.shape[:-2]
    n = int(np.prod(lead)) if lead else 1
    flat = rows.reshape(n, 2, 3)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    lib().lq_oracle_reconstruct12(ctypes.c_int64(n), _cptr(flat.view(np.float64), ctypes.c_double),
                                  _cptr(out.view(np.float64), ctypes.c_double))
    return out.reshape(*lead, 3, 3)


def reconstruct10(stored) -> np.ndarray:
    """Full 3x3 links from their 10-real form: row 0 and the two entries of row 1 outside
    column k (k = the column of row 0 with the largest max(|Re|, |Im|), lowest on ties);
    row 1's entry k follows from row 1 being orthogonal to row 0, row 2 = conj(row0 x row1).

    stored: complex (..., 5) = (u00, u01, u02, first kept u1j, second kept u1j);
    returns complex (..., 3, 3).
    """
    stored = np.ascontiguousarray(stored, dtype=np.complex128)
    lead = stored.shape[:-1]
    n = int(np.prod(lead)) if lead else 1
    flat = stored.reshape(n, 5)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    lib().lq_oracle_reconstruct10(ctypes.c_int64(n), _cptr(flat.view(np.float64), ctypes.c_double),
                                  _cptr(out.view(np.float64), ctypes.c_double))
    return out.reshape(*lead, 3, 3)


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 over all reals of the field."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


# --------------------------------------------------------------------------------------
# Even-odd decomposition, written from its definition through the full operator:
# parity(n) = (x + y + z + t) mod 2; D = A + H with A = m_q + 4 and H the hopping term,
# which only connects sites of opposite parity.
# --------------------------------------------------------------------------------------
def parity_of_sites(dims) -> np.ndarray:
    lx, ly, lz, lt = (int(v) for v in dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


def hop(dims, U, psi_full, out_parity: int, dagger: bool = False) -> np.ndarray:
    """The hopping term H (the 1/2 sum of Eq. 1) from parity 1-p onto parity p.

    Defined as D applied to the field that keeps only the 1-p sites of psi_full, restricted
    to the p sites (the diagonal term then contributes nothing).  Returns the full-lattice
    field with zeros on parity 1-p.
    """
    par = parity_of_sites(dims)
    src = np.array(psi_full, dtype=np.complex128, copy=True)
    src[par == out_parity] = 0.0
    out = dslash(dims, 0.0, U, src, dagger=dagger)
    out[par != out_parity] = 0.0
    return out


def schur_even(dims, m_q: float, U, psi_full, dagger: bool = False) -> np.ndarray:
    """M_ee psi_e = A psi_e - H_eo A^{-1} H_oe psi_e on the even sites (odd sites zero)."""
    par = parity_of_sites(dims)
    a = m_q + 4.0
    src = np.array(psi_full, dtype=np.complex128, copy=True)
    src[par == 1] = 0.0
    t = hop(dims, U, src, 1, dagger) / a
    out = a * src - hop(dims, U, t, 0, dagger)
    out[par == 1] = 0.0
    return out


# --------------------------------------------------------------------------------------
# Gradients (PyTorch convention: grad = dL/dRe + i dL/dIm of a real loss L).
# --------------------------------------------------------------------------------------
def link_grad(dims, g, psi) -> np.ndarray:
    """Gradient with respect to the links of L = Re <g, D psi> (D of Eq. 1), complex (V,4,3,3).

    D depends on U_mu(n) through 1/2 U_mu(n) P^{-mu} psi(n+mu) in row n and, conjugated,
    through 1/2 U_mu(n)^dag P^{+mu} psi(n) in row n+mu, hence
        grad U_mu(n) = 1/2 sum_spin [ g(n) (P^{-mu} psi(n+mu))^H + (P^{+mu} psi(n)) g(n+mu)^H ].
    Written with the full 4x4 projectors and explicit index sums over spin and colour.
    """
    from . import dense
    V = volume(dims)
    g = np.asarray(g, dtype=np.complex128).reshape(V, 4, 3)
    psi = np.asarray(psi, dtype=np.complex128).reshape(V, 4, 3)
    out = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    one = np.eye(4)
    for mu in range(4):
        gm = gamma(mu)
        fwd = dense.shift_index(dims, mu, +1)
        w = np.einsum("ab,nbc->nac", one - gm, psi[fwd])      # P^{-mu} psi(n+mu)
        v = np.einsum("ab,nbc->nac", one + gm, psi)           # P^{+mu} psi(n)
        out[:, mu] = 0.5 * (np.einsum("naA,naB->nAB", g, w.conj())
                            + np.einsum("naA,naB->nAB", v, g[fwd].conj()))
    return out


def solve_grads(dims, m_q, U, eta, chi, tol=1e-13):
    """Gradients of L = Re <chi, (D^dag D)^{-1} eta>: returns (grad_eta, grad_U).

    With x = A^{-1} eta and y = A^{-1} chi (A = D^dag D is Hermitian):
        grad_eta = y,  grad_U = -[ G(D x, y) + G(D y, x) ],  G(g, psi) = link_grad(g, psi).
    """
    x, _, _ = cg(dims, m_q, U, eta, tol=tol)
    y, _, _ = cg(dims, m_q, U, chi, tol=tol)
    Dx = dslash(dims, m_q, U, x)
    Dy = dslash(dims, m_q, U, y)
    return y, -(link_grad(dims, Dx, y) + link_grad(dims, Dy, x))


def solve_d(dims, m_q, U, b, tol: float = 1e-13):
    """x with D x = b (Eq. 1), through the textbook CG on D^dag D x = D^dag b.
    Returns (x, iterations, true relative residual of the normal equations)."""
    return cg(dims, m_q, U, dslash(dims, m_q, U, b, dagger=True), tol=tol)
