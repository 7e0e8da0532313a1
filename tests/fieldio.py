"""Moving stored fields between NumPy (oracle side) and CUDA tensors (library side)."""
from __future__ import annotations

import numpy as np


def to_dev(buf: np.ndarray):
    import torch
    b = np.ascontiguousarray(np.asarray(buf).view(np.uint8).reshape(-1))
    return torch.from_numpy(b.copy()).cuda()


def to_host(t) -> np.ndarray:
    return t.detach().cpu().contiguous().view(-1).numpy().view(np.uint8).copy()


# bytes of the per-site elements of the scaled formats (their float scales follow)
_ELEM_BYTES = {"f16s": 48, "i32s": 96}


def eo_half(buf: np.ndarray, dims, prec: str, parity: int) -> np.ndarray:
    """The half field of one parity cut out of a full EO spinor buffer."""
    V = int(np.prod(dims))
    b = np.asarray(buf).view(np.uint8).reshape(-1)
    if prec not in _ELEM_BYTES:
        n = b.size // 2
        return b[parity * n:(parity + 1) * n].copy()
    eb = _ELEM_BYTES[prec]
    elems = b[:eb * V]
    scales = b[eb * V:]
    hn = eb * V // 2
    sn = 2 * V
    return np.concatenate([elems[parity * hn:(parity + 1) * hn], scales[parity * sn:(parity + 1) * sn]])


def eo_embed(half: np.ndarray, dims, prec: str, parity: int) -> np.ndarray:
    """A full EO spinor buffer holding ``half`` on one parity and zeros on the other."""
    V = int(np.prod(dims))
    h = np.asarray(half).view(np.uint8).reshape(-1)
    if prec not in _ELEM_BYTES:
        out = np.zeros(2 * h.size, np.uint8)
        out[parity * h.size:(parity + 1) * h.size] = h
        return out
    eb = _ELEM_BYTES[prec]
    out = np.zeros((eb + 4) * V, np.uint8)
    hn = eb * V // 2
    sn = 2 * V
    out[parity * hn:(parity + 1) * hn] = h[:hn]
    out[eb * V + parity * sn:eb * V + (parity + 1) * sn] = h[hn:]
    return out
