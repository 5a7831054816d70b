"""Host-side plan for splitting ONE volume's reconstruction over several GPUs.

Algorithm 1 (Sec. III-C) on a partitioned volume: every rank owns a rectangle
of the image (the same rectangle of every slice) and keeps u, d, w, b and the
DMD patterns of that rectangle only.

  * v-update (Eq. v-update), Tikhonov u-step and dual update are pixel-local:
    no exchange.
  * TV u-step (Eq. u-sub / u-update): T Chambolle steps of one slice.  A pixel's
    prox output depends on the prox input g within T + 1 pixels (one pixel per
    step, plus the final divergence), so a rank that holds g on its rectangle
    grown by a halo of T + 1 pixels (clipped to the image) computes the exact
    output on its own rectangle.  With the z term the slices follow one another
    (Gauss-Seidel), so the halo of g_n is exchanged once per slice and
    iteration, after each rank formed g_n on its own rectangle.  (Kernels that
    exchange the dual field p every k steps need a halo of k + 1 instead; the
    ownership and exchange rules below are the same, only the width changes.)
  * BM3D: a halo of 19 + 7 pixels (search window and patch) before matching,
    and an overlap-add of the aggregation sums at rectangle edges.

This module holds only that bookkeeping: who owns which rectangle, how far the
halo reaches, and which rows and columns go to which peer.  ``halo_exchange``
moves them with torch.distributed point-to-point calls (gloo on the CPU, NCCL
between GPUs, each rank receiving into its own memory).  It computes nothing of
the method.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass(frozen=True)
class Rect:
    """Half-open pixel rectangle [y0, y1) x [x0, x1)."""

    y0: int
    y1: int
    x0: int
    x1: int

    def intersect(self, o: "Rect") -> "Rect | None":
        y0, y1 = max(self.y0, o.y0), min(self.y1, o.y1)
        x0, x1 = max(self.x0, o.x0), min(self.x1, o.x1)
        return Rect(y0, y1, x0, x1) if y0 < y1 and x0 < x1 else None

    @property
    def shape(self) -> tuple[int, int]:
        return self.y1 - self.y0, self.x1 - self.x0


def _split(n: int, parts: int) -> list[tuple[int, int]]:
    """n items into `parts` contiguous ranges whose sizes differ by at most one."""
    if parts < 1 or parts > n:
        raise ValueError(f"cannot split {n} rows or columns into {parts} parts")
    q, r = divmod(n, parts)
    out, a = [], 0
    for i in range(parts):
        b = a + q + (1 if i < r else 0)
        out.append((a, b))
        a = b
    return out


@dataclasses.dataclass(frozen=True)
class Partition:
    """A grid of ranks_y x ranks_x rectangles over an H x W image; rank
    r = iy * ranks_x + ix owns the rectangle in grid row iy, column ix."""

    H: int
    W: int
    ranks_y: int
    ranks_x: int

    @property
    def world(self) -> int:
        return self.ranks_y * self.ranks_x

    def owned(self, rank: int) -> Rect:
        iy, ix = divmod(rank, self.ranks_x)
        (y0, y1), (x0, x1) = _split(self.H, self.ranks_y)[iy], _split(self.W, self.ranks_x)[ix]
        return Rect(y0, y1, x0, x1)

    def extended(self, rank: int, halo: int) -> Rect:
        """The owned rectangle grown by `halo` pixels on every side, clipped to
        the image (image borders keep their own boundary rule)."""
        o = self.owned(rank)
        return Rect(max(0, o.y0 - halo), min(self.H, o.y1 + halo),
                    max(0, o.x0 - halo), min(self.W, o.x1 + halo))

    def exchange_plan(self, rank: int, halo: int):
        """(sends, recvs): lists of (peer, Rect in image coordinates).  A rank
        sends the part of its owned rectangle that lies in a peer's extended
        rectangle and receives the part of each peer's owned rectangle that lies
        in its own extended rectangle; both sides list the same rectangles in
        the same (peer) order, so paired calls match."""
        mine_o, mine_e = self.owned(rank), self.extended(rank, halo)
        sends, recvs = [], []
        for peer in range(self.world):
            if peer == rank:
                continue
            s = mine_o.intersect(self.extended(peer, halo))
            if s is not None:
                sends.append((peer, s))
            r = self.owned(peer).intersect(mine_e)
            if r is not None:
                recvs.append((peer, r))
        return sends, recvs


def halo_exchange(own, part: Partition, rank: int, halo: int, group=None):
    """Returns the field on the rank's extended rectangle: `own` (a tensor whose
    last two dimensions are the owned rectangle) in the middle, the halo filled
    with the peers' owned values.  Point-to-point isend / irecv, all posted
    before any wait."""
    import torch
    import torch.distributed as dist

    o, e = part.owned(rank), part.extended(rank, halo)
    if tuple(own.shape[-2:]) != o.shape:
        raise ValueError(f"own has shape {tuple(own.shape[-2:])}, the rectangle {o.shape}")
    lead = own.shape[:-2]
    ext = torch.zeros(*lead, *e.shape, dtype=own.dtype, device=own.device)
    ext[..., o.y0 - e.y0:o.y1 - e.y0, o.x0 - e.x0:o.x1 - e.x0] = own
    sends, recvs = part.exchange_plan(rank, halo)
    reqs, bufs, pieces = [], [], []
    for peer, r in recvs:
        buf = torch.empty(*lead, *r.shape, dtype=own.dtype, device=own.device)
        bufs.append((r, buf))
        reqs.append(dist.irecv(buf, src=peer, group=group))
    for peer, s in sends:
        piece = own[..., s.y0 - o.y0:s.y1 - o.y0, s.x0 - o.x0:s.x1 - o.x0].contiguous()
        pieces.append(piece)  # kept alive until the sends complete
        reqs.append(dist.isend(piece, dst=peer, group=group))
    for q in reqs:
        q.wait()
    for r, buf in bufs:
        ext[..., r.y0 - e.y0:r.y1 - e.y0, r.x0 - e.x0:r.x1 - e.x0] = buf
    return ext
