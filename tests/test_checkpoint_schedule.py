"""Binomial checkpointing schedule (Sec. 3.3: reverse the forward field from a
partial time history by recomputation) checked on the host.

The schedule returned by wp_checkpoint_schedule is replayed by a small
simulator: every adjoint step j = nt .. 1 must come exactly once and in that
order, with the current state equal to j; an advance must start from a slot that
really holds its start state; stores must use slots 1..c.  Its cost (forward
steps plus one per store) must equal the optimum of a brute-force dynamic
program over every split, and for c = 0 it must be the quadratic
nt(nt+1)/2 of recomputing every step from the initial state.
"""
import functools

import numpy as np
import pytest

from paper_1808_01995_gb300 import wavprop as W


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_01995_gb300 import build
    build.build()


def brute_cost(nt, c):
    @functools.lru_cache(maxsize=None)
    def T(n, k):
        if n <= 0:
            return 0
        if n == 1:
            return 1
        best = n * (n + 1) // 2
        if k == 0:
            return best
        for m in range(1, n):
            best = min(best, m + 1 + T(n - m, k - 1) + T(m, k))
        return best
    return T(nt, c)


def replay(ops, nt, c):
    slots = {0: 0}
    cur = None
    adj = []
    steps = stores = 0
    max_slot = 0
    for kind, a, b, slot in ops:
        if kind == 0:
            assert slots.get(slot) == a, (a, b, slot)
            assert b > a
            steps += b - a
            cur = b
        elif kind == 1:
            assert cur == a
            assert 1 <= slot <= c
            slots[slot] = a
            stores += 1
            max_slot = max(max_slot, slot)
        else:
            assert kind == 2
            assert cur == a, (cur, a)
            adj.append(a)
        # a stored state is never above a pending adjoint step
    assert adj == list(range(nt, 0, -1))
    return steps, stores, max_slot


@pytest.mark.parametrize("c", [0, 1, 2, 3, 5, 8])
@pytest.mark.parametrize("nt", [1, 2, 3, 7, 20, 63, 150])
def test_schedule_is_valid_and_optimal(nt, c):
    ops, fw = W.wp_checkpoint_schedule(nt, c)
    steps, stores, max_slot = replay([tuple(o) for o in ops], nt, c)
    assert steps == fw
    assert max_slot <= c
    assert steps + stores == brute_cost(nt, c)
    if c == 0:
        assert steps == nt * (nt + 1) // 2


def numpy_cost(nt, c, store=1):
    """The same recursion with every split scanned (vectorised over m)."""
    T = np.zeros((nt + 1, c + 1), dtype=np.int64)
    n = np.arange(nt + 1)
    T[:, 0] = n * (n + 1) // 2
    for k in range(1, c + 1):
        T[1, k] = 1
        for N in range(2, nt + 1):
            m = np.arange(1, N)
            T[N, k] = min(T[N, k - 1], int((m + store + T[N - m, k - 1] + T[m, k]).min()))
    return int(T[nt, c])


@pytest.mark.parametrize("c", [5, 20])
def test_large_schedule_is_valid_and_optimal(c):
    # 1500 steps (the 3D gradient workload's length): a few recomputed sweeps
    nt = 1500
    ops, fw = W.wp_checkpoint_schedule(nt, c)
    steps, stores, _ = replay([tuple(o) for o in ops], nt, c)
    assert steps == fw
    assert steps + stores == numpy_cost(nt, c)
    # charging stores never lets the step count drop below the store-free optimum
    assert steps >= numpy_cost(nt, c, store=0)
    assert steps < 8 * nt


def test_zero_steps_and_bad_arguments():
    ops, fw = W.wp_checkpoint_schedule(0, 3)
    assert len(ops) == 0 and fw == 0
    with pytest.raises(W.WpError):
        W.wp_checkpoint_schedule(-1, 2)
    with pytest.raises(W.WpError):
        W.wp_checkpoint_schedule(10, -1)


def test_memory_estimate_of_checkpointed_gradient():
    g = W.Grid((64, 64, 64), (10.0, 10.0, 10.0), (0.0, 0.0, 0.0), 8, 1e-3, 1500)
    periodic = W.wp_estimate_bytes(g, 1, 100, 1, 10)
    ck = W.wp_estimate_bytes(g, 1, 100, 2, 20)
    field = 64 * 64 * 64 * 4
    assert ck < periodic
    assert ck >= 2 * 20 * field
