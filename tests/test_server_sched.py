"""The CNN server's request scheduler, run on a simulated GPU (he_sched_simulate).

The library's scheduler class is the one the GPU server uses. Its decisions
are checked against a separate event simulation written here from the
policy's statement (admission in arrival order within the device-memory
budget, the oldest admitted request's side batched first, up to max_blocks
requests per batch, slot blocks in arrival order) and against properties
that any run must have. No GPU is needed: the library is loaded, and this
entry point makes no CUDA call.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import pytest

from inputs import synthetic

GB = 1 << 30


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api as a
    return a


def reference_policy(arrival, side, nbytes, sides, base, per, budget, reserve, max_blocks, out_bytes):
    """The policy as stated, as a plain event loop (results claimed when their batch ends)."""
    n = len(arrival)
    sidx = {s: i for i, s in enumerate(sides)}
    waiting, ready = deque(), []
    held = 0
    max_held = 0
    res = {k: np.full(n, -1.0) for k in ("admit", "start", "done")}
    batch = np.full(n, -1, np.int64)
    block = np.full(n, -1, np.int32)
    n_batches = 0
    nxt, finished = 0, 0
    busy, busy_until, cur = False, 0.0, []

    def admit(t):
        nonlocal held, max_held
        while waiting and held + nbytes[waiting[0]] + reserve <= budget:
            r = waiting.popleft()
            held += nbytes[r]
            res["admit"][r] = t
            ready.append(r)
        max_held = max(max_held, held)

    while finished < n:
        t_arr = arrival[nxt] if nxt < n else float("inf")
        if busy and busy_until <= t_arr:
            t = busy_until
            for r in cur:
                held -= nbytes[r]
                res["done"][r] = t
            held += out_bytes
            max_held = max(max_held, held)
            held -= out_bytes
            finished += len(cur)
            busy = False
            admit(t)
        else:
            t = t_arr
            r = nxt
            nxt += 1
            if nbytes[r] + reserve > budget:
                finished += 1
            else:
                waiting.append(r)
                admit(t)
        if not busy and ready:
            s = side[ready[0]]
            cur = [r for r in ready if side[r] == s][:max_blocks]
            for b, r in enumerate(cur):
                block[r] = b
                batch[r] = n_batches
                res["start"][r] = t
            ready = [r for r in ready if r not in cur]
            n_batches += 1
            busy = True
            busy_until = t + base[sidx[s]] + per[sidx[s]] * len(cur)
    return dict(batch=batch, block=block, admit_ms=res["admit"], start_ms=res["start"], done_ms=res["done"],
                max_held=max_held)


def _trace(n, rate=20.0):
    t, side = synthetic.poisson_trace(n, rate)
    return t * 1000.0, side.astype(np.int32)


SIDES = [64, 128, 256]
BASE = [120.0, 420.0, 1100.0]   # ms per batch (independent of how many blocks are used)
PER = [0.3, 0.6, 1.2]           # ms per request (packing)


def _bytes(side):
    return np.array([int(s) * 2 * 13 * (1 << 16) * 8 for s in side], np.uint64)


def _run(api, arrival, side, budget, reserve, max_blocks, out_bytes=0):
    nb = _bytes(side)
    got = api.sched_simulate(arrival, side, nb, SIDES, BASE, PER, budget, reserve, max_blocks, out_bytes)
    ref = reference_policy(list(arrival), list(side), [int(x) for x in nb], SIDES, BASE, PER, budget, reserve,
                           max_blocks, out_bytes)
    return got, ref, nb


@pytest.mark.parametrize("max_blocks,budget_gb", [(1, 250), (64, 250), (64, 40), (3, 30)])
def test_scheduler_matches_stated_policy(api, max_blocks, budget_gb):
    arrival, side = _trace(300)
    got, ref, _ = _run(api, arrival, side, budget_gb * GB, 20 * GB, max_blocks, 70 << 20)
    for k in ("batch", "block"):
        assert np.array_equal(got[k], ref[k]), k
    for k in ("admit_ms", "start_ms", "done_ms"):
        assert np.array_equal(got[k], ref[k]), k
    assert got["max_held"] == ref["max_held"]


def test_fifo_one_at_a_time(api):
    arrival, side = _trace(120)
    got, _, _ = _run(api, arrival, side, 250 * GB, 20 * GB, 1)
    assert (got["block"] == 0).all()
    # batches are the requests in arrival order, each started when the GPU was free
    assert np.array_equal(got["batch"], np.arange(120))
    assert (np.diff(got["start_ms"]) > 0).all()
    assert (got["start_ms"] >= arrival).all()
    dur = got["done_ms"] - got["start_ms"]
    exp = np.array([BASE[SIDES.index(s)] + PER[SIDES.index(s)] for s in side])
    assert np.allclose(dur, exp)


def test_batches_are_one_side_with_blocks_in_arrival_order(api):
    arrival, side = _trace(400)
    mb = 16
    got, _, _ = _run(api, arrival, side, 250 * GB, 20 * GB, mb)
    for b in np.unique(got["batch"]):
        idx = np.nonzero(got["batch"] == b)[0]
        assert len(idx) <= mb
        assert len(set(side[idx])) == 1
        # blocks 0..T-1 given in arrival order; one start and end per batch
        assert np.array_equal(got["block"][idx], np.arange(len(idx)))
        assert len(set(got["start_ms"][idx])) == 1 and len(set(got["done_ms"][idx])) == 1
    # the GPU never runs two batches at once
    starts = np.array(sorted({(got["start_ms"][i], got["done_ms"][i]) for i in range(len(side))}))
    assert (starts[1:, 0] >= starts[:-1, 1]).all()


def test_oldest_admitted_request_picks_the_side(api):
    arrival, side = _trace(300)
    got, _, _ = _run(api, arrival, side, 250 * GB, 20 * GB, 8)
    for b in np.unique(got["batch"]):
        idx = np.nonzero(got["batch"] == b)[0]
        t0 = got["start_ms"][idx[0]]
        # admitted and not yet started at t0: the oldest of them belongs to this batch
        waiting = [i for i in range(len(side)) if got["admit_ms"][i] <= t0 and got["start_ms"][i] >= t0]
        assert min(waiting) == idx[0]


def test_budget_is_never_exceeded_and_admission_is_in_order(api):
    arrival, side = _trace(300)
    budget, reserve = 30 * GB, 12 * GB
    got, _, nb = _run(api, arrival, side, budget, reserve, 64)
    assert got["max_held"] + reserve <= budget
    ok = got["batch"] >= 0
    adm = got["admit_ms"][ok]
    assert (np.diff(adm) >= 0).all()  # admitted in arrival order
    assert (got["admit_ms"][ok] >= arrival[ok]).all()
    # with this budget some requests had to wait for memory
    assert (got["admit_ms"][ok] > arrival[ok]).any()
    # requests larger than budget - reserve are refused, every other one finishes
    too_big = nb.astype(np.float64) + reserve > budget
    assert np.array_equal(~ok, too_big)
    assert (got["done_ms"][ok] > got["start_ms"][ok]).all()


def test_requests_arriving_during_a_batch_join_the_next(api):
    # three requests of one side: the first runs alone, the two that arrive meanwhile share the next batch
    arrival = np.array([0.0, 10.0, 20.0])
    side = np.array([128, 128, 128], np.int32)
    got, _, _ = _run(api, arrival, side, 250 * GB, 20 * GB, 8)
    assert list(got["batch"]) == [0, 1, 1]
    assert list(got["block"]) == [0, 0, 1]
    assert got["start_ms"][1] == got["done_ms"][0]


def test_continuous_batching_beats_fifo_under_load(api):
    arrival, side = _trace(300)
    fifo, _, _ = _run(api, arrival, side, 250 * GB, 20 * GB, 1)
    cb, _, _ = _run(api, arrival, side, 250 * GB, 20 * GB, 128)
    lat_f = fifo["done_ms"] - arrival
    lat_c = cb["done_ms"] - arrival
    assert np.percentile(lat_c, 99) < np.percentile(lat_f, 99) / 10
    assert cb["done_ms"].max() < fifo["done_ms"].max()


def test_simulate_rejects_bad_input(api):
    from paper_2512_18646_gb300._lib import HeError
    with pytest.raises(HeError):
        api.sched_simulate([1.0, 0.0], [64, 64], [1, 1], SIDES, BASE, PER, GB, 0, 4)  # not ascending
    with pytest.raises(HeError):
        api.sched_simulate([0.0], [32], [1], SIDES, BASE, PER, GB, 0, 4)  # side not served


def test_requests_that_can_never_fit_are_refused(api):
    arrival, side = _trace(60)
    reserve = 12 * GB
    got, ref, nb = _run(api, arrival, side, reserve + 2 * GB, reserve, 8)
    refused = got["batch"] < 0
    assert np.array_equal(refused, side == 256)  # 3.5 GB requests; 64 and 128 fit in 2 GB
    assert (got["done_ms"][~refused] > 0).all()
    assert np.array_equal(got["batch"], ref["batch"])
