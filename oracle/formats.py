"""Storage formats of the fields, restated independently of the CUDA library.

TEST INFRASTRUCTURE ONLY.  These are the encoders that produce reduced-precision inputs
for parity tests and the decoders that turn stored fields back into the FP64 numbers the
oracle computes with.  They follow the format definitions in include/lq.h; the CUDA pack
kernels implement the same definitions in their own code.

Precisions:  "f64", "f32", "f16s", "f64x" (FP64 values as float pairs hi = fl32(v),
lo = fl32(v - hi), laid out like "f64" with every double replaced by (hi, lo)).  Link formats: 18 (full 3x3), 12 (rows 0 and 1;
row 2 is conj(row0 x row1), an exact identity for SU(3)) or 10 (row 0 and the two entries of
row 1 outside column k, where k is the column of the stored row 0 with the largest
max(|Re|, |Im|), lowest on ties; the missing entry follows from the orthogonality of rows 0
and 1, then row 2 as for 12; not for "f64x").  Layouts: "lex" (site-major,
lexicographic) and "eo" (parity-split, chunked structure of arrays).

Scaled FP16 spinors ("f16s"): per site, s = max over the 24 reals of |fl32(v)| (an FP32
number) and h = fl16(fl32(v) / s), the division in FP32 with round-to-nearest-even and the
conversion to FP16 round-to-nearest-even (h = 0 when s = 0).  The stored value of a
component is the exact product h * s.  FP16 links are fl16(fl32(v)) with no scale.

32-bit fixed-point spinors ("i32s", Q1.30): per site the same FP32 scale s and the integers
q = RN(v / s * 2^30) computed in FP64 (ties to even; q = 0 when s = 0); the stored value is
q * s * 2^-30.  Fixed-point links are q = RN(v * 2^30) with no scale.  Scaled formats keep
all elements first and the per-site scales after them.
"""
from __future__ import annotations

import numpy as np

from . import reconstruct10, reconstruct12

PRECS = ("f64", "f32", "f16s", "f64x", "i32s")
_ELEM = {"f64": np.float64, "f32": np.float32, "f16s": np.float16, "i32s": np.int32}
_SCALED = ("f16s", "i32s")
Q30 = float(2 ** 30)


def _vol(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def eo_site_map(dims):
    """(parity, checkerboard index) of every lexicographic site: p = (x+y+z+t) mod 2,
    cb = n // 2 (x is the fastest index and Lx is even, so the two sites sharing cb in an
    x-row pair have opposite parity)."""
    lx, ly, lz, lt = (int(v) for v in dims)
    n = np.arange(lx * ly * lz * lt, dtype=np.int64)
    x = n % lx
    y = (n // lx) % ly
    z = (n // (lx * ly)) % lz
    t = n // (lx * ly * lz)
    return ((x + y + z + t) % 2).astype(np.int64), n // 2


# chunk widths (number of reals per chunk) of the eo layout; f64x uses the f64 slots
def _spinor_chunk(prec):
    return {"f64": 2, "f64x": 2, "f32": 4, "f16s": 8, "i32s": 4}[prec]


def _link_chunk(prec, fmt):
    if fmt in (18, 10):
        return 2
    return {"f64": 2, "f64x": 2, "f32": 4, "f16s": 4, "i32s": 4}[prec]


def _pairs(v):
    """float64 array -> float32 array of (hi, lo) pairs, one pair per value."""
    v = np.asarray(v, dtype=np.float64)
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    return np.stack([hi, lo], axis=-1)


def _unpairs(p):
    p = np.asarray(p, dtype=np.float32)
    return p[..., 0].astype(np.float64) + p[..., 1].astype(np.float64)


def _round(v, prec):
    """fl_prec(v) for links (no scale): f16 goes through f32 first."""
    v = np.asarray(v, dtype=np.float64)
    if prec == "f64":
        return v.copy()
    if prec == "f32":
        return v.astype(np.float32)
    if prec == "i32s":
        return np.rint(v * Q30).astype(np.int32)
    return v.astype(np.float32).astype(np.float16)


# ------------------------------------------------------------------------------------
# spinors
# ------------------------------------------------------------------------------------
def spinor_bytes(dims, prec) -> int:
    V = _vol(dims)
    return {"f64": 192 * V, "f64x": 192 * V, "f32": 96 * V, "f16s": 52 * V, "i32s": 100 * V}[prec]


def _f16s_encode_sites(reals):
    """reals: float64 (V, 24) -> (halves (V, 24) float16, scales (V,) float32)."""
    v32 = np.asarray(reals, dtype=np.float64).astype(np.float32)
    s = np.max(np.abs(v32), axis=1).astype(np.float32)
    safe = np.where(s > 0, s, np.float32(1.0)).astype(np.float32)
    q = (v32 / safe[:, None]).astype(np.float32)
    h = q.astype(np.float16)
    h[s == 0] = 0
    return h, s


def _i32s_encode_sites(reals):
    """reals: float64 (V, 24) -> (integers (V, 24) int32, scales (V,) float32)."""
    v = np.asarray(reals, dtype=np.float64)
    s = np.max(np.abs(v.astype(np.float32)), axis=1).astype(np.float32)
    safe = np.where(s > 0, s, np.float32(1.0)).astype(np.float64)
    q = np.rint(v / safe[:, None] * Q30).astype(np.int32)
    q[s == 0] = 0
    return q, s


def encode_spinor(psi, dims, prec="f64", layout="lex") -> np.ndarray:
    """complex (V, 4, 3) -> the stored buffer as a flat uint8 array."""
    V = _vol(dims)
    reals = np.ascontiguousarray(psi, dtype=np.complex128).reshape(V, 12).view(np.float64)
    reals = reals.reshape(V, 24)
    if prec == "f16s":
        h, s = _f16s_encode_sites(reals)
        data = h
    elif prec == "i32s":
        data, s = _i32s_encode_sites(reals)
    elif prec == "f64x":
        data = reals
        s = None
    else:
        data = _round(reals, prec)
        s = None
    if layout == "eo":
        data = _to_eo_spinor(data, dims, _spinor_chunk(prec))
        if s is not None:
            p, cb = eo_site_map(dims)
            s2 = np.empty(V, dtype=np.float32)
            s2[p * (V // 2) + cb] = s
            s = s2
    if prec == "f64x":
        data = _pairs(data)
    out = np.ascontiguousarray(data).view(np.uint8).reshape(-1)
    if s is not None:
        out = np.concatenate([out, np.ascontiguousarray(s).view(np.uint8).reshape(-1)])
    return out


def decode_spinor(buf, dims, prec="f64", layout="lex") -> np.ndarray:
    """Stored buffer -> complex128 (V, 4, 3) holding the exact stored values."""
    V = _vol(dims)
    buf = np.ascontiguousarray(np.asarray(buf).view(np.uint8).reshape(-1))
    if buf.size != spinor_bytes(dims, prec):
        raise ValueError("spinor buffer has the wrong size")
    if prec == "f64x":
        data = _unpairs(buf.view(np.float32).reshape(-1, 2)).reshape(V, 24)
        nb = buf.size
    else:
        elem = _ELEM[prec]
        nb = V * 24 * np.dtype(elem).itemsize
        data = buf[:nb].view(elem).reshape(V, 24)
    s = buf[nb:].view(np.float32) if prec in _SCALED else None
    if layout == "eo":
        data = _from_eo_spinor(data.reshape(-1), dims, _spinor_chunk(prec))
        if s is not None:
            p, cb = eo_site_map(dims)
            s = s[p * (V // 2) + cb]
    vals = data.astype(np.float64)
    if s is not None:
        sc = s.astype(np.float64) * (1.0 / Q30 if prec == "i32s" else 1.0)
        vals = vals * sc[:, None]
    return np.ascontiguousarray(vals).view(np.complex128).reshape(V, 4, 3)


def _to_eo_spinor(data, dims, w):
    """(V, 24) site-major -> [parity][chunk][cb][w] flat."""
    V = _vol(dims)
    K = 24 // w
    p, cb = eo_site_map(dims)
    out = np.empty((2, K, V // 2, w), dtype=data.dtype)
    out[p, :, cb, :] = data.reshape(V, K, w)
    return out.reshape(-1)


def _from_eo_spinor(flat, dims, w):
    V = _vol(dims)
    K = 24 // w
    p, cb = eo_site_map(dims)
    arr = flat.reshape(2, K, V // 2, w)
    return arr[p, :, cb, :].reshape(V, 24)


# ------------------------------------------------------------------------------------
# gauge links
# ------------------------------------------------------------------------------------
def gauge_bytes(dims, prec, fmt) -> int:
    V = _vol(dims)
    per = {"f64": 8, "f64x": 8, "f32": 4, "f16s": 2, "i32s": 4}[prec]
    return V * 4 * fmt * per


def _stored_value(r, prec):
    """Stored (rounded) link reals as exact float64 numbers, in units where they compare
    like the stored elements (Q1.30 integers stay integers)."""
    return np.asarray(r).astype(np.float64)


def link10_column(row0_stored, prec):
    """k of the 10-real form for each link: the column of the stored row 0 (reals
    (..., 6)) whose larger component max(|Re|, |Im|) is largest, the lowest on ties."""
    v = np.abs(_stored_value(row0_stored, prec)).reshape(*np.shape(row0_stored)[:-1], 3, 2)
    return np.argmax(v.max(axis=-1), axis=-1)


def encode_gauge(U, dims, prec="f64", fmt=18, layout="lex") -> np.ndarray:
    """complex (V, 4, 3, 3) -> stored buffer (uint8).  fmt 12 keeps rows 0 and 1; fmt 10
    keeps row 0 and the two entries of row 1 outside column link10_column(row 0)."""
    V = _vol(dims)
    U = np.ascontiguousarray(U, dtype=np.complex128).reshape(V, 4, 3, 3)
    if fmt == 10:
        if prec == "f64x":
            raise ValueError("the 10-real link form is not defined for f64x")
        row0 = _round(np.ascontiguousarray(U[:, :, 0, :]).view(np.float64).reshape(V, 4, 6), prec)
        k = link10_column(row0, prec)
        cols = np.array([[1, 2], [0, 2], [0, 1]])[k]                        # (V, 4, 2)
        kept = np.take_along_axis(U[:, :, 1, :], cols, axis=-1)             # (V, 4, 2)
        rest = _round(np.ascontiguousarray(kept).view(np.float64).reshape(V, 4, 4), prec)
        data = np.concatenate([row0, rest], axis=-1)
        if layout == "eo":
            data = _to_eo_gauge(data, dims, fmt, _link_chunk(prec, fmt))
        return np.ascontiguousarray(data).view(np.uint8).reshape(-1)
    rows = U if fmt == 18 else U[:, :, :2, :]
    reals = np.ascontiguousarray(rows).view(np.float64).reshape(V, 4, fmt)
    data = reals if prec == "f64x" else _round(reals, prec)
    if layout == "eo":
        data = _to_eo_gauge(data, dims, fmt, _link_chunk(prec, fmt))
    if prec == "f64x":
        data = _pairs(data)
    return np.ascontiguousarray(data).view(np.uint8).reshape(-1)


def decode_gauge(buf, dims, prec="f64", fmt=18, layout="lex") -> np.ndarray:
    """Stored buffer -> complex128 (V, 4, 3, 3); 12- and 10-real links are rebuilt in FP64."""
    V = _vol(dims)
    buf = np.ascontiguousarray(np.asarray(buf).view(np.uint8).reshape(-1))
    if buf.size != gauge_bytes(dims, prec, fmt):
        raise ValueError("gauge buffer has the wrong size")
    data = _unpairs(buf.view(np.float32).reshape(-1, 2)) if prec == "f64x" else buf.view(_ELEM[prec])
    if layout == "eo":
        data = _from_eo_gauge(data, dims, fmt, _link_chunk(prec, fmt))
    vals = np.ascontiguousarray(data.reshape(V, 4, fmt).astype(np.float64))
    if prec == "i32s":
        vals = vals / Q30
    if fmt == 10:
        return np.ascontiguousarray(reconstruct10(vals.view(np.complex128).reshape(V, 4, 5)))
    c = vals.view(np.complex128).reshape(V, 4, fmt // 6, 3)
    if fmt == 12:
        c = reconstruct12(c)
    return np.ascontiguousarray(c)


def _to_eo_gauge(data, dims, fmt, w):
    """(V, 4, fmt) -> [mu][parity][chunk][cb][w] flat."""
    V = _vol(dims)
    K = fmt // w
    p, cb = eo_site_map(dims)
    out = np.empty((4, 2, K, V // 2, w), dtype=data.dtype)
    # the two index arrays are separated by a slice, so the site axis comes first
    out[:, p, :, cb, :] = data.reshape(V, 4, K, w)
    return out.reshape(-1)


def _from_eo_gauge(flat, dims, fmt, w):
    V = _vol(dims)
    K = fmt // w
    p, cb = eo_site_map(dims)
    arr = flat.reshape(4, 2, K, V // 2, w)
    d = arr[:, p, :, cb, :]          # (V, 4, K, w): advanced indices first
    return d.reshape(V, 4, fmt)


# ------------------------------------------------------------------------------------
# several fields: LEX stacks complete fields; EO interleaves the fields of each chunk slot
# ------------------------------------------------------------------------------------
def encode_spinor_multi(psis, dims, prec="f64", layout="lex") -> np.ndarray:
    """A list of complex (V, 4, 3) fields -> one multi-field buffer (uint8)."""
    n = len(psis)
    if layout == "lex":
        return np.concatenate([encode_spinor(p, dims, prec, "lex") for p in psis])
    V = _vol(dims)
    singles = [encode_spinor(p, dims, prec, "eo") for p in psis]
    if prec in _SCALED:
        nd = (48 if prec == "f16s" else 96) * V
        elems = np.stack([b[:nd].view(np.uint8).reshape(-1, 16) for b in singles], axis=1)        # slot, field, 16 B
        scales = np.stack([b[nd:].view(np.float32) for b in singles], axis=1)                    # site, field
        return np.concatenate([elems.reshape(-1), np.ascontiguousarray(scales).view(np.uint8).reshape(-1)])
    chunks = np.stack([b.reshape(-1, 16) for b in singles], axis=1)                               # slot, field, 16 B
    return np.ascontiguousarray(chunks).reshape(-1)


def decode_spinor_multi(buf, dims, n, prec="f64", layout="lex"):
    """A multi-field buffer -> list of n complex (V, 4, 3) fields."""
    buf = np.asarray(buf).view(np.uint8).reshape(-1)
    one = spinor_bytes(dims, prec)
    if layout == "lex":
        return [decode_spinor(buf[i * one:(i + 1) * one], dims, prec, "lex") for i in range(n)]
    V = _vol(dims)
    if prec in _SCALED:
        nd = (48 if prec == "f16s" else 96) * V
        elems = buf[:nd * n].reshape(-1, n, 16)
        scales = buf[nd * n:].view(np.float32).reshape(-1, n)
        return [decode_spinor(np.concatenate([np.ascontiguousarray(elems[:, i]).reshape(-1),
                                              np.ascontiguousarray(scales[:, i]).view(np.uint8).reshape(-1)]),
                              dims, prec, "eo") for i in range(n)]
    chunks = buf.reshape(-1, n, 16)
    return [decode_spinor(np.ascontiguousarray(chunks[:, i]).reshape(-1), dims, prec, "eo") for i in range(n)]
