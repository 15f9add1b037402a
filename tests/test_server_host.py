"""The serving runtime's admission policy, replayed on the host (sparstencil_server_simulate):
FIFO admission under a slot count and an HBM budget, checked against hand-worked cases and
against an independent event-driven restatement on random workloads."""
import heapq

import numpy as np
import pytest

from paper_2506_22969_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    from paper_2506_22969_gb300 import build
    build.build()
    return binding.load()


def test_slots_limit_concurrency(lib):
    adm, done = binding.server_simulate(1 << 30, 2, [0, 0, 0], [1.0, 1.0, 1.0], [10, 10, 10])
    np.testing.assert_array_equal(adm, [0, 0, 1])
    np.testing.assert_array_equal(done, [1, 1, 2])


def test_budget_limits_concurrency(lib):
    adm, done = binding.server_simulate(10, 8, [0, 0, 0], [1.0, 2.0, 1.0], [6, 6, 6])
    np.testing.assert_array_equal(adm, [0, 1, 3])


def test_fifo_no_overtaking(lib):
    # C fits next to A but arrives behind B, which does not: C waits for B's admission
    adm, _ = binding.server_simulate(10, 8, [0.0, 0.1, 0.2], [2.0, 1.0, 1.0], [6, 6, 1])
    np.testing.assert_array_equal(adm, [0.0, 2.0, 2.0])


def test_job_larger_than_budget_is_rejected(lib):
    adm, done = binding.server_simulate(10, 8, [0.0, 0.5], [1.0, 1.0], [11, 4])
    assert adm[0] == -1 and done[0] == -1
    assert adm[1] == 0.5 and done[1] == 1.5


def test_idle_server_admits_on_arrival(lib):
    adm, _ = binding.server_simulate(10, 2, [0.0, 5.0], [1.0, 1.0], [5, 5])
    np.testing.assert_array_equal(adm, [0.0, 5.0])


def _fifo_reference(budget, slots, arrival, duration, nbytes):
    """Independent restatement: process events in time order; the queue head is admitted as
    soon as it has arrived, a slot is free and its bytes fit."""
    order = sorted(range(len(arrival)), key=lambda i: (arrival[i], i))
    adm = [None] * len(arrival)
    done = [None] * len(arrival)
    running = []  # heap of (done, bytes)
    t, used, k = 0.0, 0, 0
    while k < len(order):
        i = order[k]
        if nbytes[i] > budget:
            adm[i] = done[i] = -1.0
            k += 1
            continue
        t = max(t, arrival[i])
        while running and running[0][0] <= t:
            used -= heapq.heappop(running)[1]
        while len(running) >= slots or used + nbytes[i] > budget:
            d, b = heapq.heappop(running)
            t = max(t, d)
            used -= b
            while running and running[0][0] <= t:
                used -= heapq.heappop(running)[1]
        adm[i] = t
        done[i] = t + duration[i]
        used += nbytes[i]
        heapq.heappush(running, (done[i], nbytes[i]))
        k += 1
    return np.array(adm), np.array(done)


@pytest.mark.parametrize("seed", range(6))
def test_policy_matches_reference_on_random_workloads(lib, seed):
    rng = np.random.default_rng(seed)
    n = 60
    arrival = np.sort(rng.exponential(0.3, n).cumsum())
    duration = rng.uniform(0.1, 2.0, n)
    nbytes = rng.integers(1, 40, n).astype(np.uint64)
    budget, slots = 64, int(rng.integers(1, 6))
    adm, done = binding.server_simulate(budget, slots, arrival, duration, nbytes)
    radm, rdone = _fifo_reference(budget, slots, list(arrival), list(duration), [int(b) for b in nbytes])
    np.testing.assert_allclose(adm, radm, rtol=0, atol=1e-12)
    np.testing.assert_allclose(done, rdone, rtol=0, atol=1e-12)
    # invariants: never over budget or slots, FIFO admission order
    ok = adm >= 0
    for t in adm[ok]:
        live = ok & (adm <= t) & (done > t)
        assert nbytes[live].sum() <= budget and live.sum() <= slots
    a = adm[ok]
    assert np.all(np.diff(a) >= 0)
