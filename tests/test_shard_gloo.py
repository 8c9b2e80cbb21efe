"""The sharding layer's host logic on CPU (gloo, world sizes 2, 3 and 6).

The ranks run paper_2512_18646_gb300.shard against a stand-in for the
library defined here: ciphertexts are small integer arrays [n][polys][limbs][N]
modulo per-limb primes, and each operation is a linear map of the same shape
as the library's (a convolution's windowed weighted sums of rotated columns, a
dense layer's weighted column sums, diagonal products of a matmul). The test
checks that the plan, the halo exchange, the all-gathers and the modulo-q
combine put every ciphertext where the one-process evaluation of the same
stand-in puts it, word for word, including ranks that hold nothing. The
arithmetic of the real layers is checked on the GPU by the sharded-CNN test.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

PRIMES = np.array([1000003, 998244353, 65537], dtype=np.uint64)
NW = 6  # words per limb


class FakeSet:
    def __init__(self, ctx, words, scale=1.0):
        self.ctx = ctx
        self.w = np.ascontiguousarray(words, dtype=np.uint64)
        self._scale = scale

    def info4(self):
        n, polys, limbs, _ = self.w.shape
        return n, limbs, self._scale, polys

    @property
    def n(self):
        return self.w.shape[0]

    def slice(self, first, n):
        assert 0 <= first and n >= 1 and first + n <= self.n
        return FakeSet(self.ctx, self.w[first:first + n], self._scale)

    def export_words(self, buf):
        flat = self.w.reshape(-1).view(np.int64)
        assert buf.numel() >= flat.size and not buf.is_cuda
        buf.numpy()[: flat.size] = flat


class FakePts:
    def __init__(self, wt, n_in):
        self.wt = wt  # [out_dim][n_in] small integers
        self.n_in = n_in


class FakeCtx:
    N = NW

    def _mod(self, x, limbs):
        return x % PRIMES[:limbs].reshape(1, 1, limbs, 1)

    def concat(self, sets):
        assert len({s.info4()[1:] for s in sets}) == 1
        return FakeSet(self, np.concatenate([s.w for s in sets]), sets[0]._scale)

    def import_words(self, buf, n, polys, limbs, scale):
        w = buf.numpy()[: n * polys * limbs * NW].view(np.uint64).reshape(n, polys, limbs, NW)
        assert (w < PRIMES[:limbs].reshape(1, 1, limbs, 1)).all()
        return FakeSet(self, w.copy(), scale)

    def add(self, a, b):
        assert a.info4()[1:] == b.info4()[1:] and a.n == b.n
        return FakeSet(self, self._mod(a.w + b.w, a.w.shape[2]), a._scale)

    def conv2d(self, x, c_in, gap, W, bias, stride):
        W = np.asarray(W)
        c_out, _, k, _ = W.shape
        n, polys, limbs, _ = x.w.shape
        w_in = n // c_in
        w_out = (w_in - k) // stride + 1
        Wi = (np.rint(W * 1000).astype(np.int64) % 65537).astype(np.uint64)
        X = x.w.reshape(c_in, w_in, polys, limbs, NW)
        out = np.zeros((c_out, w_out, polys, limbs, NW), np.uint64)
        for o in range(c_out):
            for jp in range(w_out):
                acc = np.zeros((polys, limbs, NW), np.uint64)
                for c in range(c_in):
                    for b in range(k):
                        for a in range(k):
                            rot = np.roll(X[c, stride * jp + b], -gap * a, axis=-1)
                            acc = (acc + Wi[o, c, a, b] * rot) % PRIMES[:limbs].reshape(1, limbs, 1)
                if bias is not None:
                    acc[0] = (acc[0] + np.uint64(int(round(bias[o] * 1000)) % 65537)) % PRIMES[:limbs].reshape(limbs, 1)
                out[o, jp] = acc
        # one level down, like the library's rescale
        return FakeSet(self, out.reshape(c_out * w_out, polys, limbs, NW)[:, :, : limbs - 1], x._scale)

    def fc_partial(self, cols, pts, first):
        n, polys, limbs, _ = cols.w.shape
        assert first >= 0 and first + n <= pts.n_in
        out = np.zeros((pts.wt.shape[0], polys, limbs, NW), np.uint64)
        for o in range(pts.wt.shape[0]):
            for t in range(n):
                out[o] = (out[o] + np.uint64(pts.wt[o, first + t]) * cols.w[t]) % PRIMES[:limbs].reshape(1, limbs, 1)
        return FakeSet(self, out, cols._scale)

    def fc_finish(self, sums, pts, bias):
        limbs = sums.w.shape[2]
        z = self._mod(sums.w * np.uint64(3), limbs)[:, :2, : limbs - 1]
        if bias is not None:
            b = (np.rint(np.asarray(bias) * 1000).astype(np.int64) % 65537).astype(np.uint64)
            z[:, 0] = (z[:, 0] + b.reshape(-1, 1, 1)) % PRIMES[: limbs - 1].reshape(1, -1, 1)
        return FakeSet(self, z, sums._scale)

    def fc_apply(self, x, pts, bias):
        return self.fc_finish(self.fc_partial(x, pts, 0), pts, bias)

    def matmul_range(self, A, B, m, p, lo, hi):
        limbs = A.w.shape[2]
        out = np.zeros((hi - lo, 2, limbs, NW), np.uint64)
        for idx in range(lo, hi):
            for k in range(A.n):
                out[idx - lo] = (out[idx - lo] + A.w[k] * np.roll(B.w[k], -idx, axis=-1)) % PRIMES[:limbs].reshape(1, limbs, 1)
        return FakeSet(self, out[:, :, : limbs - 1], A._scale)


def _rand_set(ctx, rng, n, polys, limbs):
    w = np.stack([rng.integers(0, int(PRIMES[i]), size=(n, polys, NW), dtype=np.int64) for i in range(limbs)], axis=2)
    return FakeSet(ctx, w.astype(np.uint64))


def _network(seed):
    """Inputs and weights of a two-conv network on the stand-in (2 columns of halo at stride 2)."""
    rng = np.random.default_rng(seed)
    ctx = FakeCtx()
    w0 = 13
    x = _rand_set(ctx, rng, 1 * w0, 2, 3)              # one channel, 13 columns
    W1 = rng.normal(0, 0.05, (3, 1, 3, 3))
    b1 = rng.normal(0, 0.05, 3)
    W2 = rng.normal(0, 0.05, (4, 3, 2, 2))
    b2 = rng.normal(0, 0.05, 4)
    w1 = (w0 - 3) // 2 + 1                             # 6
    w2 = (w1 - 2) // 1 + 1                             # 5
    pts = FakePts(rng.integers(0, 50, size=(3, 4 * w2)), 4 * w2)
    fcb = rng.normal(0, 0.05, 3)
    A = _rand_set(ctx, rng, 3, 2, 3)
    B = _rand_set(ctx, rng, 3, 2, 3)
    return ctx, x, w0, (W1, b1, 2, 1), (W2, b2, 1, 2), pts, fcb, A, B


def _single_process(seed):
    ctx, x, w0, (W1, b1, s1, g1), (W2, b2, s2, g2), pts, fcb, A, B = _network(seed)
    y1 = ctx.conv2d(x, 1, g1, W1, b1, s1)
    y2 = ctx.conv2d(y1, 3, g2, W2, b2, s2)
    z = ctx.fc_apply(y2, pts, fcb)
    d = ctx.matmul_range(A, B, 4, 5, 0, 5)
    return y1.w, y2.w, z.w, d.w


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, seed, q):
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        from paper_2512_18646_gb300 import shard
        comm = shard.Comm()
        ctx, x, w0, (W1, b1, s1, g1), (W2, b2, s2, g2), pts, fcb, A, B = _network(seed)
        # rank r holds the input columns split(w0)[r] (disjoint slabs); the halos move
        lo, hi = shard.split(w0, world, rank)
        xs = shard.ColumnShard(x.slice(lo, hi - lo) if hi > lo else None, 1, lo, hi, w0)
        y1 = shard.conv2d_columns(ctx, comm, xs, g1, W1, b1, s1)
        y2 = shard.conv2d_columns(ctx, comm, y1, g2, W2, b2, s2)
        z = shard.fc_columns(ctx, comm, y2, pts, fcb)
        _, _, d = shard.matmul_diagonals(ctx, comm, A, B, 4, 5, gather=True)
        # the layers by output channel, on the replicated first-layer output
        yc = shard.conv2d_channels(ctx, comm, ctx.conv2d(x, 1, g1, W1, b1, s1), 3, g2, W2, b2, s2)
        q.put((rank, (y1.lo, y1.hi, None if y1.cts is None else y1.cts.w),
               (y2.lo, y2.hi, None if y2.cts is None else y2.cts.w), z.w, d.w, yc.w))
        dist.barrier()
    except Exception as e:  # reported to the test, which fails with it
        q.put((rank, "error", repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 6])
def test_sharded_layers_equal_the_one_process_result(world):
    y1_ref, y2_ref, z_ref, d_ref = _single_process(7)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, 7, q), daemon=True) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    for r in res:
        assert r[1] != "error", r[2]
    for p in procs:
        assert p.exitcode == 0
    c1, c2 = 3, 4
    w1, w2 = y1_ref.shape[0] // c1, y2_ref.shape[0] // c2
    got1 = np.zeros_like(y1_ref).reshape(c1, w1, *y1_ref.shape[1:])
    got2 = np.zeros_like(y2_ref).reshape(c2, w2, *y2_ref.shape[1:])
    seen1, seen2 = np.zeros(w1, int), np.zeros(w2, int)
    for rank, (lo1, hi1, a1), (lo2, hi2, a2), z, d, yc in res:
        if a1 is not None:
            got1[:, lo1:hi1] = a1.reshape(c1, hi1 - lo1, *a1.shape[1:])
        if a2 is not None:
            got2[:, lo2:hi2] = a2.reshape(c2, hi2 - lo2, *a2.shape[1:])
        seen1[lo1:hi1] += 1
        seen2[lo2:hi2] += 1
        np.testing.assert_array_equal(z, z_ref)     # every rank holds the finished logits
        np.testing.assert_array_equal(d, d_ref)     # the gathered diagonals
        np.testing.assert_array_equal(yc, y2_ref)   # the convolution by output channel
    assert (seen1 == 1).all() and (seen2 == 1).all()  # every output column computed once
    np.testing.assert_array_equal(got1.reshape(y1_ref.shape), y1_ref)
    np.testing.assert_array_equal(got2.reshape(y2_ref.shape), y2_ref)


def test_split_and_windows():
    from paper_2512_18646_gb300 import shard
    for n in range(0, 20):
        for world in range(1, 6):
            parts = [shard.split(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1
    # output columns 3..5 of a 5-wide stride-2 convolution read input columns 6..14
    assert shard.conv_window(3, 6, 5, 2) == (6, 15)
    assert shard.conv_window(4, 4, 5, 2) == (0, 0)
