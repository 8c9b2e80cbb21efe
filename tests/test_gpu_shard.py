"""The sharded layers on the GPU.

Single process: the split entry points (he_matmul_range, he_fc_partial +
he_add + he_fc_finish, word export/import to host and device buffers) against
the whole-layer calls, word for word. Two processes: the small CNN sharded over
two gloo ranks that share the GPU (they exchange ciphertext words through host
memory; no kernel waits on another rank), every layer's result compared with
the one-process library run and with the oracle, word for word.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from gpu_pairs import image_columns_both, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_18646_gb300 as pkg
    pkg.load()
    return pkg


def _rand_coeffs(rng, n, N):
    return rng.integers(-(1 << 40), 1 << 40, size=(n, N), dtype=np.int64)


def test_matmul_range_equals_the_diagonals_of_matmul(lib):
    from paper_2512_18646_gb300 import HeError
    from paper_2512_18646_gb300._lib import HE_E_ARG
    _, g = make_pair(10, (60, 45, 45), 2, 60, 2, 45.0, seed=5, steps=range(1, 8))
    rng = np.random.default_rng(5)
    m, n, p = 4, 3, 8
    A = g.encrypt_matrix_a(rng.uniform(-1, 1, (m, n)))
    B = g.encrypt_matrix_b(rng.uniform(-1, 1, (n, p)), 100)
    full = g.matmul(A, B, m, p).export_raw()
    for lo, hi in [(0, 3), (3, 8), (5, 6), (0, 8), (0, 1)]:
        part = g.matmul_range(A, B, m, p, lo, hi)
        assert part.n == hi - lo
        assert np.array_equal(part.export_raw(), full[lo:hi]), (lo, hi)
    for lo, hi in [(3, 3), (0, 9), (-1, 2)]:
        with pytest.raises(HeError) as e:
            g.matmul_range(A, B, m, p, lo, hi)
        assert e.value.code == HE_E_ARG


@pytest.mark.parametrize("square", [False, True])
def test_fc_partial_sums_combine_to_fc_apply(lib, square):
    from paper_2512_18646_gb300 import HeError
    from paper_2512_18646_gb300._lib import HE_E_ARG
    _, g = make_pair(10, (60, 45, 45, 45), 2, 60, 2, 45.0, seed=6, steps=[4, 8, 16])
    rng = np.random.default_rng(6)
    c_in, w_in, out_dim = 3, 4, 3
    limbs = 4 if square else 3
    x = g.encrypt_coeffs(_rand_coeffs(rng, c_in * w_in, g.N), limbs, g.scale)
    if square:
        g.square(x)  # three components, one level down
    lp = x.limbs
    pts = g.fc_prepare_coeffs(rng.integers(-(1 << 20), 1 << 20, size=(out_dim, c_in, w_in, g.N)), 4, 32, lp)
    bias = rng.normal(0, 0.1, out_dim)
    ref = g.fc_apply(x, pts, bias).export_raw()
    whole = g.fc_partial(x, pts, 0)
    assert whole.polys == x.polys and whole.n == out_dim
    assert np.array_equal(g.fc_finish(whole, pts, bias).export_raw(), ref)
    # three uneven column ranges, combined modulo q in two orders
    cuts = [(0, 5), (5, 6), (6, 12)]
    parts = [g.fc_partial(x.slice(a, b - a), pts, a) for a, b in cuts]
    s1 = g.add(g.add(parts[0], parts[1]), parts[2])
    s2 = g.add(parts[2], g.add(parts[1], parts[0]))
    assert np.array_equal(s1.export_raw(), whole.export_raw())
    assert np.array_equal(s2.export_raw(), whole.export_raw())
    assert np.array_equal(g.fc_finish(s1, pts, bias).export_raw(), ref)
    assert np.array_equal(whole.export_raw(), g.fc_partial(x, pts, 0).export_raw())  # sums not consumed
    with pytest.raises(HeError) as e:
        g.fc_partial(x.slice(0, 5), pts, 8)
    assert e.value.code == HE_E_ARG
    with pytest.raises(HeError) as e:
        g.fc_finish(parts[0].slice(0, 2), pts, bias)
    assert e.value.code == HE_E_ARG


def test_words_move_through_host_and_device_buffers(lib):
    import torch
    from paper_2512_18646_gb300 import HeError
    from paper_2512_18646_gb300._lib import HE_E_ARG
    _, g = make_pair(10, (60, 45, 45), 2, 60, 2, 45.0, seed=7, steps=())
    rng = np.random.default_rng(7)
    x = g.encrypt_coeffs(_rand_coeffs(rng, 3, g.N), 3, g.scale)
    g.square(x)
    n, limbs, scale, polys = x.info4()
    assert polys == 3
    raw = x.export_raw()
    host = np.zeros(raw.size + 5, np.uint64)
    x.export_words(host)
    assert np.array_equal(host[: raw.size], raw.reshape(-1))
    dev = torch.empty(raw.size, dtype=torch.int64, device="cuda")
    x.export_words(dev)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), raw.reshape(-1))
    for src in (dev, host):
        y = g.import_words(src, n, polys, limbs, scale)
        assert y.info4() == (n, limbs, scale, polys)
        assert np.array_equal(y.export_raw(), raw)
    for at, prime in ((g.N + 3, 1), (raw.size - 1, limbs - 1)):  # an early row; the very last word
        bad = host.copy()
        bad[at] = np.uint64(g.primes[prime])  # a residue equal to its prime
        with pytest.raises(HeError) as e:
            g.import_words(bad, n, polys, limbs, scale)
        assert e.value.code == HE_E_ARG
        with pytest.raises(HeError) as e:
            g.import_words(torch.from_numpy(bad.view(np.int64)).cuda(), n, polys, limbs, scale)
        assert e.value.code == HE_E_ARG


# ---------------------------------------------------------------------------
# the small CNN over two ranks
# ---------------------------------------------------------------------------
SIDE, H, BN = 17, 32, 3
STEPS = [1, 2, 3, 4, 8, 16]


def _cnn_inputs():
    rng = np.random.default_rng(31)
    imgs = rng.uniform(0, 1, (BN, 1, SIDE, SIDE))
    c1w, c1b = rng.normal(0, 0.2, (2, 1, 5, 5)), rng.normal(0, 0.2, 2)
    c2w, c2b = rng.normal(0, 0.2, (3, 2, 3, 3)), rng.normal(0, 0.2, 3)
    h1 = (SIDE - 5) // 2 + 1
    h2 = (h1 - 3) // 2 + 1
    fw, fb = rng.normal(0, 0.2, (4, 3 * h2 * h2)), rng.normal(0, 0.2, 4)
    return imgs, c1w, c1b, c2w, c2b, fw, fb, h1, h2


def _broadcast_words(dist, words, src, rank):
    """A flat uint64 array from rank `src` on every rank."""
    import torch
    size = torch.tensor([words.size if rank == src else 0], dtype=torch.int64)
    dist.broadcast(size, src)
    if rank == src:
        buf = torch.from_numpy(np.ascontiguousarray(words).reshape(-1).view(np.int64).copy())
    else:
        buf = torch.empty(int(size[0]), dtype=torch.int64)
    dist.broadcast(buf, src)
    return buf.numpy().view(np.uint64)


def _cnn_worker(rank, world, port, q):
    import datetime

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    # a short timeout: a rank that fails leaves its peer's next collective to end with an error
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=90))
    out = {"rank": rank}
    try:
        torch.cuda.set_device(0)
        from paper_2512_18646_gb300 import api, shard
        imgs, c1w, c1b, c2w, c2b, fw, fb, h1, h2 = _cnn_inputs()
        params = (10, (60,) + (45,) * 6, 2, 60, 2, 45.0)
        if rank == 0:
            o, g = make_pair(*params, seed=31, steps=STEPS)
            ox, gx = image_columns_both(o, g, imgs, H)
            keys = g.export_keys()
            words = gx.export_raw()
        else:
            g = api.Context(*params, seed=1000 + rank)  # its keys come from rank 0
            keys = words = np.zeros(0, np.uint64)
        keys = _broadcast_words(dist, keys, 0, rank)
        if rank != 0:
            g.import_keys(keys)
        words = _broadcast_words(dist, words, 0, rank).reshape(SIDE, 2, -1, g.N)
        # rank r holds input columns split(SIDE)[r], as a client would send them
        lo, hi = shard.split(SIDE, world, rank)
        x = shard.ColumnShard(g.import_words(words[lo:hi].copy(), hi - lo, 2, words.shape[2], g.scale),
                              1, lo, hi, SIDE)
        comm = shard.Comm()
        y1 = shard.conv2d_columns(g, comm, x, 1, c1w, c1b, 2)
        if y1.cts is not None:
            g.square(y1.cts)
        y2 = shard.conv2d_columns(g, comm, y1, 2, c2w, c2b, 2)
        if y2.cts is not None:
            g.square(y2.cts)
        lp = len(params[1]) - 4  # the dense layer's limbs: two convolutions and two squares below the top
        pts_fc = None
        if rank == 0:
            pts_fc = o.fc_plaintexts(lp, 3, h2, h2, 4, H, BN, fw, list(range(4)))
        pts_fc = _broadcast_words(dist, np.zeros(0, np.uint64) if rank else pts_fc.astype(np.int64).view(np.uint64),
                                  0, rank).view(np.int64).reshape(4, 3, h2, g.N)
        pts = g.fc_prepare_coeffs(pts_fc, 4, H, lp)
        z = shard.fc_columns(g, comm, y2, pts, fb)
        out.update(y1=(y1.lo, y1.hi, None if y1.cts is None else y1.cts.export_raw()),
                   y2=(y2.lo, y2.hi, None if y2.cts is None else y2.cts.export_raw()), z=z.export_raw())
        if rank == 0:
            # the one-process library run and the oracle on the same ciphertexts
            r1 = g.conv2d(gx, 1, 1, c1w, c1b, 2)
            g.square(r1)
            r2 = g.conv2d(r1, 2, 2, c2w, c2b, 2)
            g.square(r2)
            rz = g.fc_apply(r2, pts, fb)
            out.update(ref_y1=r1.export_raw(), ref_y2=r2.export_raw(), ref_z=rz.export_raw())
            sc = o.scale
            oy = o.square(o.conv2d(ox, 1, c1w, c1b, 2, sc))
            sc = sc * sc / o.q[o.L1 - 2]
            oy2 = o.square(o.conv2d(oy.reshape(2, h1, *oy.shape[1:]), 2, c2w, c2b, 2, sc))
            sc = sc * sc / o.q[lp]
            oz = o.fc(oy2.reshape(3, h2, *oy2.shape[1:]), 4, H, pts_fc, fb, sc, list(range(4)))
            out["oracle_equal"] = bool(np.array_equal(z.export(), oz))
        dist.barrier()
    except Exception as e:  # reported to the test, which fails with it
        out["error"] = repr(e)
    finally:
        q.put(out)
        dist.destroy_process_group()


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_cnn_sharded_over_two_ranks_equals_one_process_and_oracle(lib):
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_cnn_worker, args=(r, world, port, q), daemon=True) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted((q.get(timeout=300) for _ in procs), key=lambda d: d["rank"])
    finally:
        for p in procs:
            p.join(timeout=120)
            if p.is_alive():
                p.terminate()
    for r in res:
        assert "error" not in r, r.get("error")
    for p in procs:
        assert p.exitcode == 0
    ref = res[0]
    for key, c in (("y1", 2), ("y2", 3)):
        full = ref["ref_" + key]
        w = full.shape[0] // c
        got = np.zeros_like(full).reshape(c, w, *full.shape[1:])
        seen = np.zeros(w, int)
        for r in res:
            lo, hi, a = r[key]
            if a is not None:
                got[:, lo:hi] = a.reshape(c, hi - lo, *a.shape[1:])
            seen[lo:hi] += 1
        assert (seen == 1).all(), key
        assert np.array_equal(got.reshape(full.shape), full), key
    for r in res:
        assert np.array_equal(r["z"], ref["ref_z"])
    assert ref["oracle_equal"]
