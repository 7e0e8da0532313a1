"""Dense brute-force Wilson-Dirac matrix (test infrastructure only).

The operator of Eq. (1) is assembled as an explicit (12V) x (12V) complex matrix, block by
block, from Kronecker products of 4x4 spin matrices and 3x3 colour matrices:

    D = (m_q + 4) 1
        + 1/2 sum_mu sum_n [ |n><n+mu| (x) (1 - gamma_mu) (x) U_mu(n)
                           + |n><n-mu| (x) (1 + gamma_mu) (x) U_mu(n-mu)^dag ]

Row/column index of (site n, spin alpha, colour A) is 12 n + 3 alpha + A.  Blocks are
accumulated with +=, so on an extent-2 direction (where n+mu and n-mu are the same site)
both hopping terms land in the same block and add.

This code shares no loops with the stencil in oracle.c: it builds the matrix from its own
gamma matrices and index map, so the two cross-check each other.
"""
from __future__ import annotations

import numpy as np

# chiral Euclidean basis, gamma_{mu+1} for mu = 0..3
_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def gammas() -> list[np.ndarray]:
    gs = []
    for s in (_S1, _S2, _S3):
        gs.append(np.block([[_Z2, -1j * s], [1j * s, _Z2]]))
    gs.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    return gs


def gamma5() -> np.ndarray:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def _coords(dims):
    lx, ly, lz, lt = (int(v) for v in dims)
    V = lx * ly * lz * lt
    n = np.arange(V)
    x = n % lx
    y = (n // lx) % ly
    z = (n // (lx * ly)) % lz
    t = n // (lx * ly * lz)
    return np.stack([x, y, z, t], axis=1)


def _lex(dims, c):
    lx, ly, lz, _ = (int(v) for v in dims)
    return c[:, 0] + lx * (c[:, 1] + ly * (c[:, 2] + lz * c[:, 3]))


def shift_index(dims, mu: int, step: int) -> np.ndarray:
    """Index of the neighbour n + step*mu-hat for every site n (periodic)."""
    c = _coords(dims).copy()
    c[:, mu] = (c[:, mu] + step) % int(dims[mu])
    return _lex(dims, c)


def dense_dirac(dims, m_q: float, U) -> np.ndarray:
    """The full complex (12V, 12V) matrix of D."""
    lx, ly, lz, lt = (int(v) for v in dims)
    V = lx * ly * lz * lt
    U = np.asarray(U, dtype=np.complex128).reshape(V, 4, 3, 3)
    D = (m_q + 4.0) * np.eye(12 * V, dtype=np.complex128)
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    for mu in range(4):
        fwd = shift_index(dims, mu, +1)
        bwd = shift_index(dims, mu, -1)
        pm = one - g[mu]
        pp = one + g[mu]
        for n in range(V):
            m = fwd[n]
            D[12 * n:12 * n + 12, 12 * m:12 * m + 12] += 0.5 * np.kron(pm, U[n, mu])
            k = bwd[n]
            D[12 * n:12 * n + 12, 12 * k:12 * k + 12] += 0.5 * np.kron(pp, U[k, mu].conj().T)
    return D


def flat(psi) -> np.ndarray:
    return np.asarray(psi, dtype=np.complex128).reshape(-1)
