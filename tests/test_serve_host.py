"""Host logic of the served form (no GPU): request streams, tick planning
and the admission budget."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

S = pytest.importorskip("paper_2605_03208_gb300.serve")


def test_request_stream_is_poisson_and_seeded():
    a = S.request_stream(0, 2000, 50.0, 64)
    b = S.request_stream(0, 2000, 50.0, 64)
    assert [(r.kind, r.gid, r.t_arrival, r.n_perturb, r.seed) for r in a] == \
           [(r.kind, r.gid, r.t_arrival, r.n_perturb, r.seed) for r in b]
    t = np.array([r.t_arrival for r in a])
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0                 # mean inter-arrival 20 ms
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1                # exponential: cv = 1
    kinds = [r.kind for r in a]
    assert 0.4 < kinds.count(S.COMPARE) / len(a) < 0.6
    assert all(0 <= r.gid < 64 for r in a)
    assert all(0 <= r.n_perturb <= 64 for r in a)


def _act(rid, total, unit):
    return S.Active(S.Request(rid, S.DIGEST, 0, 0.0, 0, 0), total, unit)


def test_plan_tick_shortest_first_and_quantum():
    big = _act(0, 32768, 65536)            # 2 GiB of digest pages
    small = _act(1, 4, 65536)              # 256 KiB
    mid = _act(2, 5000, 65536)
    pieces = S.plan_tick([big, small, mid], tick_bytes=512 << 20, quantum_bytes=128 << 20)
    assert [p[0].req.rid for p in pieces] == [1, 2, 0]          # shortest remaining first
    assert pieces[0][1:] == (0, 4)                              # small finishes in this tick
    assert pieces[1][2] == 2048                                 # quantum: 128 MiB of 64 KiB pages
    assert sum(p[2] * p[0].unit_bytes for p in pieces) <= (512 << 20) + (128 << 20)


def test_plan_tick_progress_and_completion():
    a = _act(0, 10_000, 65536)
    b = _act(1, 3, 65536)
    act = [a, b]
    seen = []
    for _ in range(100):
        pieces = S.plan_tick([x for x in act if x.remaining > 0], 256 << 20, 64 << 20)
        if not pieces:
            break
        for x, first, cnt in pieces:
            assert first == x.next and cnt >= 1
            seen.append((x.req.rid, first, cnt))
            x.next += cnt
    assert a.remaining == 0 and b.remaining == 0
    # the pieces of each request tile its units exactly once, in order
    for rid, total in ((0, 10_000), (1, 3)):
        ps = [(f, c) for r, f, c in seen if r == rid]
        assert ps[0][0] == 0 and all(ps[i][0] + ps[i][1] == ps[i + 1][0] for i in range(len(ps) - 1))
        assert ps[-1][0] + ps[-1][1] == total


def test_plan_tick_always_makes_progress():
    huge = _act(0, 5, 1 << 30)             # a unit larger than the tick
    pieces = S.plan_tick([huge], tick_bytes=1 << 20, quantum_bytes=1 << 20)
    assert pieces == [(huge, 0, 1)]


def test_budget_blocks_until_release():
    b = S.Budget(100, slots=2)
    assert b.acquire(60)
    got = []

    def taker():
        got.append(b.acquire(50))
    t = threading.Thread(target=taker)
    t.start()
    time.sleep(0.1)
    assert not got                          # 60 + 50 > 100: waits
    b.release(60)
    t.join(2)
    assert got == [True] and b.used == 50 and b.waits == 1
    with pytest.raises(ValueError):
        b.acquire(101)


def test_budget_slots_and_stop():
    b = S.Budget(1000, slots=1)
    assert b.acquire(1)
    stop = threading.Event()
    stop.set()
    assert b.acquire(1, stop) is False      # no slot, and the loop is stopping


def test_budget_try_acquire():
    b = S.Budget(100, slots=2)
    assert b.try_acquire(70) and not b.try_acquire(40) and b.try_acquire(30)
    assert not b.try_acquire(0)             # no slot left
    b.release(70)
    assert b.try_acquire(10) and b.used == 40
