"""The column-layout layers sharded over processes, one GPU each.

Sec. IV-A and IV-B note that the ciphertexts of the layout are independent
units: the products of a matmul split over the columns of B (one diagonal per
worker), and a convolution or dense layer over channels, kernels and
ciphertexts, meeting only in sums. This module splits each layer that way over
the ranks of a torch.distributed process group; every arithmetic step runs in
the library (he_conv2d, he_matmul_range, he_fc_partial, he_add, he_fc_finish),
and the ranks only move ciphertext words between them:

  - convolution by column slab: rank r computes the output columns
    split(w_out)[r] from the input columns stride p_lo .. stride (p_hi - 1) + k - 1,
    receiving the (k - stride)-column halo it does not hold from the ranks that
    do (one point-to-point exchange per layer);
  - convolution by output channel: every rank holds every input column and
    computes the channels split(c_out)[r]; an all-gather rebuilds the set;
  - matmul by diagonal index: rank r computes the diagonals split(p)[r] with A
    and B replicated, no exchange (an all-gather if every rank wants them all);
  - dense layer by input column: rank r sums the products of the columns it
    holds (he_fc_partial, before the rescale); the partial sums are all-gathered
    and added modulo q in rank order (a collective's integer sum would not
    reduce modulo q), then every rank finishes the layer (he_fc_finish).

Each result is word for word the one-process result: a column or channel of a
convolution depends only on its own window, and sums modulo q do not depend on
how the terms are grouped. Words move as int64 tensors: device buffers with the
NCCL backend (he_ctset_export_words / he_ctset_import_words into the tensor),
host buffers otherwise. Keys are replicated: every rank's context holds the
same keys (he_keys_export on one rank, he_keys_import on the others).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .api import CtSet, Context, PtSet


def split(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous balanced share [lo, hi) of n units for `rank` of `world` (the first n mod world
    ranks take one more)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def conv_window(p_lo: int, p_hi: int, k: int, stride: int) -> Tuple[int, int]:
    """Input columns [a, b) that output columns [p_lo, p_hi) of a k-wide, stride-`stride`
    convolution read (empty when the output range is)."""
    if p_hi <= p_lo:
        return 0, 0
    return stride * p_lo, stride * (p_hi - 1) + k


@dataclasses.dataclass
class ColumnShard:
    """Columns [lo, hi) of every channel of a channel-major column-layout set of `channels` x
    `width` ciphertexts, held by one rank; `cts` is channel-major [c][j - lo] (None if empty)."""
    cts: Optional[CtSet]
    channels: int
    lo: int
    hi: int
    width: int

    @property
    def count(self) -> int:
        return self.hi - self.lo


class Comm:
    """Ciphertext words between the ranks of a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.on_device = dist.get_backend(group) == "nccl"

    # ---- word buffers ----
    def _buffer(self, words: int):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device()) if self.on_device else torch.device("cpu")
        return torch.empty(max(words, 1), dtype=torch.int64, device=dev)

    def _pack(self, s: CtSet):
        n, limbs, _, polys = s.info4()
        buf = self._buffer(n * polys * limbs * s.ctx.N)
        s.export_words(buf)
        return buf

    def _global_rank(self, r: int) -> int:
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    # ---- collectives ----
    def all_gather_ints(self, values: Sequence[int]) -> List[List[int]]:
        """Every rank's list of len(values) integers."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device()) if self.on_device else torch.device("cpu")
        mine = torch.tensor(list(values), dtype=torch.int64, device=dev)
        out = [torch.empty_like(mine) for _ in range(self.world)]
        self.dist.all_gather(out, mine, group=self.group)
        return [[int(v) for v in t.cpu().tolist()] for t in out]

    def all_gather_sets(self, ctx: Context, local: Optional[CtSet], polys: int, limbs: int,
                        scale: float) -> List[Optional[CtSet]]:
        """Every rank's set (None where a rank has none), in rank order, on every rank."""
        counts = [c[0] for c in self.all_gather_ints([local.n if local is not None else 0])]
        words = ctx.N * polys * limbs
        mx = max(counts)
        if mx == 0:
            return [None] * self.world
        send = self._buffer(mx * words)
        if local is not None:
            local.export_words(send)
        bufs = [self._buffer(mx * words) for _ in range(self.world)]
        self.dist.all_gather(bufs, send, group=self.group)
        if self.on_device:
            import torch
            torch.cuda.current_stream().synchronize()  # the library reads them on its own stream
        out: List[Optional[CtSet]] = []
        for r in range(self.world):
            if counts[r] == 0:
                out.append(None)
            elif r == self.rank:
                out.append(local)
            else:
                out.append(ctx.import_words(bufs[r], counts[r], polys, limbs, scale))
        return out

    def exchange(self, ctx: Context, sends: Dict[int, CtSet], recv_counts: Dict[int, int], polys: int, limbs: int,
                 scale: float) -> Dict[int, CtSet]:
        """Point-to-point: sends[r] to rank r, recv_counts[r] ciphertexts from rank r."""
        dist = self.dist
        ops, keep = [], []
        inbox = {}
        words = ctx.N * polys * limbs
        for r in sorted(set(sends) | set(recv_counts)):
            if r in recv_counts and recv_counts[r] > 0:
                buf = self._buffer(recv_counts[r] * words)
                inbox[r] = buf
                ops.append(dist.P2POp(dist.irecv, buf, self._global_rank(r), group=self.group))
            if r in sends:
                buf = self._pack(sends[r])
                keep.append(buf)
                ops.append(dist.P2POp(dist.isend, buf, self._global_rank(r), group=self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if self.on_device:
            import torch
            torch.cuda.current_stream().synchronize()
        return {r: ctx.import_words(buf, recv_counts[r], polys, limbs, scale) for r, buf in inbox.items()}


def _meta(comm: Comm, s: Optional[CtSet]) -> Tuple[int, int, float]:
    """(limbs, components, scale) of the sets the ranks hold, taken from the first rank that holds
    one (every rank's sets of one layer share them)."""
    limbs, polys, scale = (0, 0, 0.0)
    if s is not None:
        _, limbs, scale, polys = s.info4()
    bits = int(np.array([scale], np.float64).view(np.int64)[0])
    for m in comm.all_gather_ints([limbs, polys, bits]):
        if m[0] > 0:
            return m[0], m[1], float(np.array([m[2]], np.int64).view(np.float64)[0])
    raise ValueError("no rank holds any ciphertext")


def _columns(ctx: Context, s: CtSet, channels: int, width: int, a: int, b: int) -> CtSet:
    """Columns [a, b) of every channel of a channel-major [channels][width] set."""
    if a == 0 and b == width:
        return s
    return ctx.concat([s.slice(c * width + a, b - a) for c in range(channels)])


def _interleave(ctx: Context, parts: Sequence[Tuple[int, CtSet, int]], channels: int) -> CtSet:
    """Channel-major set from column blocks (first column, set [channels][w], w) sorted by column."""
    parts = sorted(parts, key=lambda t: t[0])
    if len(parts) == 1:
        return parts[0][1]
    return ctx.concat([p.slice(c * w, w) for c in range(channels) for _, p, w in parts])


def conv2d_columns(ctx: Context, comm: Comm, x: ColumnShard, gap: int, W, bias, stride: int) -> ColumnShard:
    """he_conv2d sharded by output column slab; x holds this rank's input columns (disjoint
    slabs across ranks). Returns this rank's output columns split(w_out)[rank]."""
    W = np.asarray(W, dtype=np.float64)
    c_out, c_in, k, _ = W.shape
    assert c_in == x.channels
    w_out = (x.width - k) // stride + 1
    held = comm.all_gather_ints([x.lo, x.hi])
    need = [conv_window(*split(w_out, comm.world, r), k, stride) for r in range(comm.world)]
    me = comm.rank
    limbs, polys, scale = _meta(comm, x.cts)
    sends, recv = {}, {}
    for r in range(comm.world):
        if r == me:
            continue
        # columns rank r needs from my slab, and columns I need from rank r's slab
        a, b = max(need[r][0], x.lo), min(need[r][1], x.hi)
        if need[r][1] > need[r][0] and b > a:
            sends[r] = _columns(ctx, x.cts, c_in, x.count, a - x.lo, b - x.lo)
        a, b = max(need[me][0], held[r][0]), min(need[me][1], held[r][1])
        if need[me][1] > need[me][0] and b > a:
            recv[r] = c_in * (b - a)
    got = comm.exchange(ctx, sends, recv, polys, limbs, scale)
    p_lo, p_hi = split(w_out, comm.world, me)
    if p_hi <= p_lo:
        return ColumnShard(None, c_out, p_lo, p_lo, w_out)
    a, b = need[me]
    parts = []
    la, lb = max(a, x.lo), min(b, x.hi)
    if lb > la:
        parts.append((la, _columns(ctx, x.cts, c_in, x.count, la - x.lo, lb - x.lo), lb - la))
    for r, s in got.items():
        ra = max(a, held[r][0])
        parts.append((ra, s, s.n // c_in))
    slab = _interleave(ctx, parts, c_in)
    assert slab.n == c_in * (b - a), "halo exchange left a gap in the input window"
    y = ctx.conv2d(slab, c_in, gap, W, bias, stride)
    return ColumnShard(y, c_out, p_lo, p_hi, w_out)


def conv2d_channels(ctx: Context, comm: Comm, x: CtSet, c_in: int, gap: int, W, bias, stride: int) -> CtSet:
    """he_conv2d sharded by output channel: x (every input column) is replicated; rank r computes
    channels split(c_out)[r] and an all-gather rebuilds the [c_out][w_out] result on every rank."""
    W = np.asarray(W, dtype=np.float64)
    c_out = W.shape[0]
    lo, hi = split(c_out, comm.world, comm.rank)
    y = None
    if hi > lo:
        y = ctx.conv2d(x, c_in, gap, W[lo:hi], None if bias is None else np.asarray(bias)[lo:hi], stride)
    limbs, polys, scale = _meta(comm, y)
    parts = comm.all_gather_sets(ctx, y, polys, limbs, scale)
    return ctx.concat([p for p in parts if p is not None])


def matmul_diagonals(ctx: Context, comm: Comm, A: CtSet, B: CtSet, m: int, p: int,
                     gather: bool = False):
    """he_matmul sharded by diagonal index: rank r computes diagonals split(p)[r] (A, B replicated).
    Returns (lo, hi, set) of this rank, or the full p diagonals on every rank when `gather`."""
    lo, hi = split(p, comm.world, comm.rank)
    d = ctx.matmul_range(A, B, m, p, lo, hi) if hi > lo else None
    if not gather:
        return lo, hi, d
    limbs, polys, scale = _meta(comm, d)
    parts = comm.all_gather_sets(ctx, d, polys, limbs, scale)
    return 0, p, ctx.concat([s for s in parts if s is not None])


def fc_columns(ctx: Context, comm: Comm, x: ColumnShard, pts: PtSet, bias) -> CtSet:
    """he_fc_apply sharded by input column: rank r sums the products of the columns it holds
    (channel c, columns x.lo .. x.hi - 1 at input index c width + j); the partial sums are
    all-gathered and added modulo q in rank order; every rank returns the finished logits."""
    part = None
    if x.cts is not None:
        for c in range(x.channels):
            cols = x.cts.slice(c * x.count, x.count)
            z = ctx.fc_partial(cols, pts, c * x.width + x.lo)
            part = z if part is None else ctx.add(part, z)
    limbs, polys, scale = _meta(comm, part)
    total = None
    for s in comm.all_gather_sets(ctx, part, polys, limbs, scale):
        if s is not None:
            total = s if total is None else ctx.add(total, s)
    return ctx.fc_finish(total, pts, bias)
