"""The operator on a lattice cut into t-slabs (domains), with face exchange.

The paper's Discussion (Section 3) runs large lattices on many devices that exchange
boundary data directly.  Here a lattice of dims (Lx, Ly, Lz, Lt) is cut into R slabs of
Lt / R time slices; domain r holds its own links and spinors (FP64 LEX, local dims
(Lx, Ly, Lz, Lt / R)).  One apply of D is

    pack   (lq_halo_pack): each domain fills to_prev (for domain r-1) and to_next (r+1);
    move   (a transport): from_next[r] = to_prev[r+1], from_prev[r] = to_next[r-1], periodic;
    apply  (lq_halo_dslash): each domain computes its slab of D psi.

Two transports: ``VirtualRanks`` keeps every domain on this GPU and copies the faces between
device buffers; ``exchange_faces`` moves them between processes with torch.distributed
point-to-point messages (NCCL on GPUs, any backend for the exchange itself) and turns a
neighbour that does not deliver within the timeout into an error on the host.
"""
from __future__ import annotations

import datetime

from . import _check, _dims, _ptr, _stream, load

__all__ = ["HaloError", "slab_dims", "face_bytes", "halo_pack", "halo_dslash", "VirtualRanks", "exchange_faces"]


class HaloError(RuntimeError):
    """A neighbour's face did not arrive."""


def slab_dims(dims, nranks: int):
    lx, ly, lz, lt = (int(d) for d in dims)
    if nranks < 1 or lt % nranks:
        raise ValueError(f"Lt = {lt} is not divisible by {nranks} domains")
    return (lx, ly, lz, lt // nranks)


def face_bytes(dims_local) -> int:
    return int(load().lq_halo_face_bytes(_dims(dims_local)))


def _vol(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def _empty(n, like):
    import torch
    return torch.empty(int(n), dtype=torch.uint8, device=like.device)


def halo_pack(dims_local, U, psi, to_prev=None, to_next=None, dagger=False, stream=None):
    fb = face_bytes(dims_local)
    v = _vol(dims_local)
    to_prev = _empty(fb, psi) if to_prev is None else to_prev
    to_next = _empty(fb, psi) if to_next is None else to_next
    _check(load().lq_halo_pack(_dims(dims_local), int(bool(dagger)), _ptr(U, 576 * v, "U"), _ptr(psi, 192 * v, "psi"),
                               _ptr(to_prev, fb, "to_prev"), _ptr(to_next, fb, "to_next"), _stream(stream)))
    return to_prev, to_next


def halo_dslash(dims_local, m_q, U, psi, from_next, from_prev, out=None, dagger=False, stream=None):
    fb = face_bytes(dims_local)
    n = 192 * _vol(dims_local)
    out = _empty(n, psi) if out is None else out
    _check(load().lq_halo_dslash(_dims(dims_local), float(m_q), int(bool(dagger)), _ptr(U, 3 * n, "U"),
                                 _ptr(psi, n, "psi"), _ptr(from_next, fb, "from_next"),
                                 _ptr(from_prev, fb, "from_prev"), _ptr(out, n, "out"), _stream(stream)))
    return out


class VirtualRanks:
    """R domains of one lattice on this GPU.  ``U`` and ``psi`` are the whole-lattice FP64 LEX
    fields (a t-slab is a contiguous block of them, so each domain's fields are views); the
    faces are exchanged by device copies into per-domain receive buffers."""

    def __init__(self, dims, nranks: int):
        self.dims = tuple(int(d) for d in dims)
        self.R = int(nranks)
        self.local = slab_dims(dims, nranks)
        lx, ly, lz, lt = self.local
        self.vloc = lx * ly * lz * lt

    def _slab(self, field, per_site, r):
        n = self.vloc * per_site
        return field[r * n:(r + 1) * n]

    def apply(self, m_q, U, psi, out=None, dagger=False, stream=None):
        import torch
        out = torch.empty_like(psi) if out is None else out
        fb = face_bytes(self.local)
        send = [halo_pack(self.local, self._slab(U, 576, r), self._slab(psi, 192, r), dagger=dagger, stream=stream)
                for r in range(self.R)]
        recv = [(_empty(fb, psi), _empty(fb, psi)) for _ in range(self.R)]
        for r in range(self.R):
            recv[r][0].copy_(send[(r + 1) % self.R][0])      # from_next = to_prev of r + 1
            recv[r][1].copy_(send[(r - 1) % self.R][1])      # from_prev = to_next of r - 1
        for r in range(self.R):
            halo_dslash(self.local, m_q, self._slab(U, 576, r), self._slab(psi, 192, r), recv[r][0], recv[r][1],
                        out=self._slab(out, 192, r), dagger=dagger, stream=stream)
        return out


def exchange_faces(to_prev, to_next, from_next, from_prev, group=None, timeout_s: float = 30.0):
    """Send to_prev to rank - 1 and to_next to rank + 1 (periodic), receive from_next from
    rank + 1 and from_prev from rank - 1.  Raises HaloError when a neighbour's face does not
    arrive within timeout_s seconds (a rank that failed or left)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    nxt, prv = (rank + 1) % world, (rank - 1) % world
    if world == 1:
        from_next.copy_(to_prev)
        from_prev.copy_(to_next)
        return
    # tag 1: a to_prev face (lands as the receiver's from_next); tag 2: a to_next face
    reqs = [dist.isend(to_prev, prv, group=group, tag=1), dist.isend(to_next, nxt, group=group, tag=2)]
    recvs = [(dist.irecv(from_next, nxt, group=group, tag=1), nxt), (dist.irecv(from_prev, prv, group=group, tag=2), prv)]
    limit = datetime.timedelta(seconds=timeout_s)
    for req, peer in recvs:
        try:
            ok = req.wait(limit)
        except RuntimeError as e:
            raise HaloError(f"rank {rank}: no face from rank {peer}: {e}") from e
        if ok is False:
            raise HaloError(f"rank {rank}: no face from rank {peer} within {timeout_s} s")
    for req in reqs:
        try:
            req.wait(limit)
        except RuntimeError as e:
            raise HaloError(f"rank {rank}: face to a neighbour not delivered: {e}") from e
