"""Serving: slot-block packing and the continuous-batching CNN server on the GPU.

- he_pack_blocks (the server's packing step) is bit-exact against the
  oracle's ct x pt products, sums and rescale on the same integer masks;
- the server's results are the same alone and in a mix of requests of two
  image sides (within 1e-4 after decryption, CKKS noise being the only
  difference), and each matches the FP64 CNN within 1e-4;
- admission respects the device-memory budget and refuses what cannot fit.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from inputs import synthetic
from oracle import fp64_ref

from tests.gpu_pairs import encrypt_both, make_pair

pytestmark = pytest.mark.gpu

# N = 2^12 with the six levels the served network needs below the top
PRE = synthetic.small_preset(12, q_bits=(60,) + (40,) * 6)
SIDES = (16, 32)
TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_18646_gb300 as pkg
    pkg.load()
    return pkg


def test_pack_blocks_matches_oracle(lib):
    o, g = make_pair(PRE.log_n, PRE.q_bits, PRE.n_special, PRE.special_bits, PRE.alpha, PRE.log_scale, seed=61,
                     steps=())
    T, n, side = 3, 2, 32
    L = o.L1
    rng = np.random.default_rng(62)
    sets_o, sets_g, z_all = [], [], []
    for t in range(T):
        z = rng.uniform(-1, 1, size=(n, o.slots))
        m = np.stack([o.encode(v) for v in z])
        oc, gc = encrypt_both(o, g, m, ct_id_base=10 * t)
        sets_o.append(oc)
        sets_g.append(gc)
        z_all.append(z)
    q_last = float(o.q[L - 1])
    masks = []
    for t in range(T):
        v = np.zeros(o.slots)
        v[t * side:(t + 1) * side] = 1.0
        masks.append(o.encode(v, scale=q_last))
    masks = np.stack(masks)
    pts = g.fc_prepare_coeffs(masks.reshape(T, 1, 1, o.N), 1, 1, L)
    got = g.pack_blocks(sets_g, pts)
    assert got.info4() == (n, L - 1, o.scale, 2)
    ex = got.export()
    for j in range(n):
        acc = o.mul_plain(sets_o[0][j], masks[0])
        for t in range(1, T):
            acc = o.add(acc, o.mul_plain(sets_o[t][j], masks[t]))
        assert np.array_equal(ex[j], o.rescale(acc)), j
    # decrypted: block t holds set t's values, the other slots are zero
    dec = g.decrypt_slots(got)
    exp = np.zeros((n, o.slots))
    for t in range(T):
        exp[:, t * side:(t + 1) * side] = z_all[t][:, t * side:(t + 1) * side]
    assert np.abs(dec - exp).max() < 1e-6


def _request(g, img, side, ct_id_base):
    """The request words of one image: repeated in every block of stride side, top level."""
    nb = g.slots // side
    x = g.encrypt_image(np.repeat(img[None], nb, axis=0), side, ct_id_base=ct_id_base)
    return x.export_raw().reshape(-1)


def _logits(g, z, block, side):
    return g.decrypt_slots(z)[:, block * side]


@pytest.fixture(scope="module")
def served(lib):
    from paper_2512_18646_gb300 import api
    g = api.Context.from_preset(PRE, seed=71)
    g.keygen([])
    w = {s: synthetic.cnn_weights(s, seed=72) for s in SIDES}
    return g, w


def test_server_results_same_alone_and_in_the_mix(served):
    from paper_2512_18646_gb300 import api
    g, w = served
    imgs = {k: synthetic.images(1, s, s, seed=80 + k)[0] for k, s in enumerate((32, 16, 32, 16, 32))}
    side_of = {0: 32, 1: 16, 2: 32, 3: 16, 4: 32}
    reqs = {k: _request(g, imgs[k], side_of[k], 1000 * (k + 1)) for k in imgs}
    srv = api.Server(g, w, hbm_budget_bytes=16 << 30, max_blocks=8, start_paused=True)
    try:
        # request 2 alone
        rid = srv.submit(reqs[2], 32)
        srv.pause(False)
        assert srv.wait(rid, 120_000)
        z, blk, t = srv.take(rid)
        assert blk == 0 and t[0] <= t[1] <= t[2] <= t[3]
        alone = _logits(g, z, blk, 32)
        # then all five, submitted while paused so they share batches: one per side
        srv.pause(True)
        b0 = srv.stats()["batches"]
        ids = {k: srv.submit(reqs[k], side_of[k]) for k in (0, 1, 2, 3, 4)}
        st = srv.stats()
        assert st["admitted"] == 5 and st["waiting"] == 0
        srv.pause(False)
        out = {}
        for k, rid in ids.items():
            assert srv.wait(rid, 120_000)
            z, blk, t = srv.take(rid)
            out[k] = (_logits(g, z, blk, side_of[k]), blk)
        assert srv.stats()["batches"] == b0 + 2
        # blocks in submission order within each side
        assert [out[k][1] for k in (0, 2, 4)] == [0, 1, 2]
        assert [out[k][1] for k in (1, 3)] == [0, 1]
        for k in imgs:
            ref = fp64_ref.cnn(imgs[k][None], w[side_of[k]])[0]
            assert np.abs(out[k][0] - ref).max() < TOL, k
        assert np.abs(out[2][0] - alone).max() < TOL
        assert np.abs(alone - fp64_ref.cnn(imgs[2][None], w[32])[0]).max() < TOL
    finally:
        srv.close()


def test_server_admits_requests_that_arrive_while_a_batch_runs(served):
    """Continuous batching on the GPU: requests submitted while another request's batch is on the GPU
    (the server never paused) are admitted at once, while that batch still runs, and run together
    in the next batch; each late request's logits equal its alone run within 1e-4 and the FP64 CNN."""
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HE_REQ_RUNNING
    g, w = served
    imgs = synthetic.images(4, 32, 32, seed=95)
    reqs = [_request(g, imgs[k], 32, 7000 + 100 * k) for k in range(4)]
    srv = api.Server(g, {32: w[32]}, hbm_budget_bytes=16 << 30, max_blocks=8)
    try:
        alone = {}
        for k in (1, 2, 3):
            rid = srv.submit(reqs[k], 32)
            assert srv.wait(rid, 120_000)
            z, blk, _ = srv.take(rid)
            alone[k] = _logits(g, z, blk, 32)
        for attempt in range(3):
            b0 = srv.stats()["batches"]
            first = srv.submit(reqs[0], 32)
            deadline = time.monotonic() + 120
            while srv.poll(first) < HE_REQ_RUNNING:
                assert time.monotonic() < deadline
                time.sleep(0.0002)
            late = {k: srv.submit(reqs[k], 32) for k in (1, 2, 3)}
            assert srv.wait(first, 120_000)
            _, blk0, t0 = srv.take(first)
            out = {}
            for k, rid in late.items():
                assert srv.wait(rid, 120_000)
                z, blk, t = srv.take(rid)
                out[k] = (_logits(g, z, blk, 32), blk, t)
            if all(out[k][2][0] < t0[3] for k in out):
                break  # every late request arrived while the first batch was on the GPU
        else:
            pytest.fail("the first batch ended before the late requests were submitted, three times")
        assert blk0 == 0
        for k, (logit, blk, t) in out.items():
            assert t0[2] <= t[0] < t0[3], k          # submitted while the first batch ran
            assert t[1] < t0[3], k                    # admitted (device budget reserved) during it
            assert t[2] >= t0[3], k                   # run in a later batch
            assert np.abs(logit - alone[k]).max() < TOL, k
            ref = fp64_ref.cnn(imgs[k][None], w[32])[0]
            assert np.abs(logit - ref).max() < TOL, k
        # the three late requests shared one batch, in submission order
        assert sorted(out[k][1] for k in out) == [0, 1, 2]
        assert len({out[k][2][2] for k in out}) == 1
        assert srv.stats()["batches"] == b0 + 2
    finally:
        srv.close()


def test_server_admission_by_budget(served):
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HE_E_ARG, HE_E_OOM, HeError
    g, w = served
    req_bytes = 32 * 2 * g.L1 * g.N * 8
    probe = api.Server(g, {32: w[32]}, hbm_budget_bytes=16 << 30, max_blocks=8)
    reserve = probe.stats()["reserve_bytes"]
    probe.close()
    budget = reserve + int(2.5 * req_bytes)
    srv = api.Server(g, {32: w[32]}, hbm_budget_bytes=budget, max_blocks=8, start_paused=True)
    try:
        st = srv.stats()
        fit = (budget - st["reserve_bytes"]) // req_bytes
        assert 1 <= fit <= 3
        imgs = synthetic.images(4, 32, 32, seed=90)
        reqs = [_request(g, imgs[k], 32, 5000 + 100 * k) for k in range(4)]
        ids = [srv.submit(r, 32) for r in reqs]
        st = srv.stats()
        assert st["admitted"] == min(fit, 4) and st["waiting"] == 4 - min(fit, 4)
        assert st["held_bytes"] + st["reserve_bytes"] <= budget
        srv.pause(False)
        for k, rid in enumerate(ids):
            assert srv.wait(rid, 120_000)
            if k == 0:  # the host copy of the result, rebuilt as a set
                host = np.zeros(srv.result_words(), np.uint64)
                blk, _ = srv.take_host(rid, host)
                z = g.import_raw(host, g.L1 - 6, g.scale)
            else:
                z, blk, _ = srv.take(rid)
            ref = fp64_ref.cnn(imgs[k][None], w[32])[0]
            assert np.abs(_logits(g, z, blk, 32) - ref).max() < TOL
        st = srv.stats()
        assert st["max_held_bytes"] + st["reserve_bytes"] <= budget
        assert st["done"] == 4 and st["failed"] == 0
        # errors: a side not served, a wrong size
        with pytest.raises(HeError) as e:
            srv.submit(reqs[0], 16)
        assert e.value.code == HE_E_ARG
        with pytest.raises(HeError) as e:
            srv.submit(reqs[0][:-1].copy(), 32)
        assert e.value.code == HE_E_ARG
    finally:
        srv.close()
    # a budget below reserve + one request refuses every request
    tiny = api.Server(g, {32: w[32]}, hbm_budget_bytes=reserve // 2, max_blocks=2)
    try:
        with pytest.raises(HeError) as e:
            tiny.submit(reqs[0], 32)
        assert e.value.code == HE_E_OOM
    finally:
        tiny.close()


def test_server_wait_times_out_while_nothing_runs(served):
    """A request whose batch cannot start (the server is held, as a stalled producer would leave it)
    makes he_server_wait return HE_E_TIMEOUT after its limit; the request is unharmed and finishes
    once batches resume."""
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import HE_REQ_ADMITTED, HE_REQ_DONE
    g, w = served
    img = synthetic.images(1, 32, 32, seed=97)[0]
    srv = api.Server(g, {32: w[32]}, hbm_budget_bytes=16 << 30, max_blocks=4, start_paused=True)
    try:
        rid = srv.submit(_request(g, img, 32, 7500), 32)
        t0 = time.monotonic()
        assert not srv.wait(rid, 200)  # HE_E_TIMEOUT
        assert time.monotonic() - t0 >= 0.19
        assert srv.poll(rid) == HE_REQ_ADMITTED
        srv.pause(False)
        assert srv.wait(rid, 120_000) and srv.poll(rid) == HE_REQ_DONE
        z, blk, _ = srv.take(rid)
        assert np.abs(_logits(g, z, blk, 32) - fp64_ref.cnn(img[None], w[32])[0]).max() < TOL
    finally:
        srv.close()


def test_server_cancel_releases_budget_in_every_state(served):
    """he_server_cancel: a waiting request leaves the queue, an admitted one gives back its device
    budget at once (the next waiting request is admitted), a running one's share is dropped when its
    batch ends, a finished one's result share is released; a cancelled request reads
    HE_REQ_CANCELLED and he_server_take refuses it (HE_E_STATE) and forgets it. The other requests'
    results are unchanged."""
    from paper_2512_18646_gb300 import api
    from paper_2512_18646_gb300._lib import (HE_E_ARG, HE_E_STATE, HE_REQ_CANCELLED, HE_REQ_RUNNING, HE_REQ_WAITING,
                                             HeError)
    g, w = served
    req_bytes = 32 * 2 * g.L1 * g.N * 8
    probe = api.Server(g, {32: w[32]}, hbm_budget_bytes=16 << 30, max_blocks=8)
    reserve = probe.stats()["reserve_bytes"]
    probe.close()
    imgs = synthetic.images(5, 32, 32, seed=98)
    reqs = [_request(g, imgs[k], 32, 8000 + 100 * k) for k in range(5)]
    # room for two requests beside the reserve
    srv = api.Server(g, {32: w[32]}, hbm_budget_bytes=reserve + int(2.5 * req_bytes), max_blocks=8,
                     start_paused=True)
    try:
        ids = [srv.submit(reqs[k], 32) for k in range(4)]
        st = srv.stats()
        assert st["admitted"] == 2 and st["waiting"] == 2
        srv.cancel(ids[3])  # waiting
        assert srv.poll(ids[3]) == HE_REQ_CANCELLED
        st = srv.stats()
        assert st["waiting"] == 1 and st["cancelled"] == 1 and st["held_bytes"] == 2 * req_bytes
        srv.cancel(ids[1])  # admitted: its budget goes to the waiting request 2
        st = srv.stats()
        assert srv.poll(ids[1]) == HE_REQ_CANCELLED
        assert st["admitted"] == 2 and st["waiting"] == 0 and st["held_bytes"] == 2 * req_bytes
        with pytest.raises(HeError) as e:
            srv.take(ids[3])
        assert e.value.code == HE_E_STATE
        with pytest.raises(HeError) as e:
            srv.poll(ids[3])  # forgotten
        assert e.value.code == HE_E_ARG
        srv.pause(False)
        for k in (0, 2):
            assert srv.wait(ids[k], 120_000)
        # a finished request cancelled: its share of the batch result is released
        srv.cancel(ids[0])
        z, blk, _ = srv.take(ids[2])
        assert np.abs(_logits(g, z, blk, 32) - fp64_ref.cnn(imgs[2][None], w[32])[0]).max() < TOL
        assert srv.stats()["held_bytes"] == 0
        # a running request cancelled: the batch ends, the share is dropped, nothing stays held
        rid = srv.submit(reqs[4], 32)
        deadline = time.monotonic() + 120
        while srv.poll(rid) < HE_REQ_RUNNING:
            assert time.monotonic() < deadline
            time.sleep(0.0005)
        srv.cancel(rid)
        assert srv.wait(rid, 120_000) and srv.poll(rid) == HE_REQ_CANCELLED
        st = srv.stats()
        assert st["held_bytes"] == 0 and st["cancelled"] == 4
        # the server keeps serving
        rid = srv.submit(reqs[4], 32)
        assert srv.wait(rid, 120_000)
        z, blk, _ = srv.take(rid)
        assert np.abs(_logits(g, z, blk, 32) - fp64_ref.cnn(imgs[4][None], w[32])[0]).max() < TOL
        assert srv.poll(ids[1]) == HE_REQ_CANCELLED and HE_REQ_WAITING == 0
    finally:
        srv.close()


def test_server_rolls_back_a_request_whose_allocation_fails(served):
    """An admitted request whose device allocation fails (injected on the host: the next allocation
    reports out-of-memory) ends FAILED; he_server_take reports the error and forgets it, its budget
    is released, and the next request is served normally."""
    from paper_2512_18646_gb300 import api, load
    from paper_2512_18646_gb300._lib import HE_E_CUDA, HE_REQ_FAILED, HeError
    g, w = served
    imgs = synthetic.images(2, 32, 32, seed=99)
    srv = api.Server(g, {32: w[32]}, hbm_budget_bytes=16 << 30, max_blocks=4)
    try:
        words = _request(g, imgs[0], 32, 9000)  # (encryption allocates: before arming)
        g.synchronize()
        assert load().he_debug_fail_allocations(1) == 0
        rid = srv.submit(words, 32)
        assert srv.wait(rid, 120_000) and srv.poll(rid) == HE_REQ_FAILED
        assert load().he_debug_fail_allocations(0) == 0
        with pytest.raises(HeError) as e:
            srv.take(rid)
        assert e.value.code == HE_E_CUDA and "injected" in str(e.value)
        st = srv.stats()
        assert st["failed"] == 1 and st["held_bytes"] == 0
        rid = srv.submit(_request(g, imgs[1], 32, 9100), 32)
        assert srv.wait(rid, 120_000)
        z, blk, _ = srv.take(rid)
        assert np.abs(_logits(g, z, blk, 32) - fp64_ref.cnn(imgs[1][None], w[32])[0]).max() < TOL
    finally:
        load().he_debug_fail_allocations(0)
        srv.close()
