"""Pins for the red-blue pebble game simulator (oracle/pebble.py)."""
import math

import pytest

from oracle import bounds, pebble


@pytest.mark.parametrize("sliding", [False, True])
@pytest.mark.parametrize("mnk,ab", [((8, 8, 5), (4, 4)), ((12, 9, 7), (3, 3)),
                                     ((10, 7, 6), (4, 3)), ((5, 5, 9), (2, 5))])
def test_listing1_io_equals_corollary_count(sliding, mnk, ab):
    m, n, k = mnk
    a, b = ab
    S = pebble.listing1_working_set(a, b, sliding)
    res = pebble.simulate(m, n, k, S, pebble.listing1_schedule(m, n, k, a, b, sliding), sliding)
    assert res.io == pebble.tile_io(m, n, k, a, b)
    assert res.max_red == S
    assert res.computes == m * n * k
    if m % a == 0 and n % b == 0:
        assert res.io == m * n * k * (a + b) // (a * b) + m * n


@pytest.mark.parametrize("sliding", [False, True])
def test_listing1_does_not_fit_one_pebble_less(sliding):
    a, b = 4, 4
    S = pebble.listing1_working_set(a, b, sliding) - 1
    with pytest.raises(pebble.PebbleError, match="exceed"):
        pebble.simulate(8, 8, 3, S, pebble.listing1_schedule(8, 8, 3, a, b, sliding), sliding)


@pytest.mark.parametrize("S", [24, 35, 48])
def test_xs_schedule_matches_closed_form(S):
    s = pebble.xs_tile(S)
    assert s == math.sqrt(S + 1) - 1  # S + 1 a perfect square here
    m = n = 2 * s
    k = 5
    res = pebble.simulate(m, n, k, S, pebble.xs_schedule(m, n, k, S), sliding=False)
    assert res.io == pytest.approx(bounds.xs_io(m, n, k, S))


@pytest.mark.parametrize("S,mnk", [(16, (8, 8, 4)), (30, (9, 12, 5)), (64, (14, 16, 6))])
def test_valid_schedules_respect_theorem1(S, mnk):
    m, n, k = mnk
    a, b = bounds.find_seq_schedule(S)  # ab + a + 1 <= S: fits in the sliding game
    res = pebble.simulate(m, n, k, S, pebble.listing1_schedule(m, n, k, a, b, True), True)
    assert res.io >= bounds.thm1(m, n, k, S)


def test_plan_replay_split_k_counts_boundary_sums():
    m, n, k = 6, 6, 8
    units = [(0, 6, 0, 3, 0, 4), (0, 6, 0, 3, 4, 8), (0, 6, 3, 6, 0, 8)]
    S = 6 * 3 + 6 + 2
    res = pebble.simulate(m, n, k, S, pebble.plan_schedule(m, n, k, units), False)
    # tile 1: 2 segments of 4, each k(h+w) + stores; second reloads 18 sums
    seg = 4 * (6 + 3)
    assert res.io == (seg + 18) + (18 + seg + 18) + (8 * 9 + 18)


def test_rejects_load_of_non_blue():
    with pytest.raises(pebble.PebbleError, match="blue"):
        pebble.simulate(2, 2, 2, 10, [("load", ("c", 0, 0, 0))])


def test_rejects_compute_without_parent():
    moves = [("load", ("a", 0, 0)), ("compute", ("c", 0, 0, 0))]
    with pytest.raises(pebble.PebbleError, match="parent"):
        pebble.simulate(1, 1, 1, 10, moves)


def test_rejects_compute_skipping_partial_sum():
    moves = [("load", ("a", 0, 1)), ("load", ("b", 1, 0)), ("compute", ("c", 0, 0, 1))]
    with pytest.raises(pebble.PebbleError, match="parent"):
        pebble.simulate(1, 1, 2, 10, moves)


def test_rejects_missing_output():
    moves = [("load", ("a", 0, 0)), ("load", ("b", 0, 0)), ("compute", ("c", 0, 0, 0))]
    with pytest.raises(pebble.PebbleError, match="output"):
        pebble.simulate(1, 1, 1, 10, moves)


def test_minimal_complete_pebbling_1x1x1():
    moves = [("load", ("a", 0, 0)), ("load", ("b", 0, 0)), ("compute", ("c", 0, 0, 0)),
             ("store", ("c", 0, 0, 0))]
    res = pebble.simulate(1, 1, 1, 3, moves)
    assert res.io == 3 and res.max_red == 3


@pytest.mark.parametrize("sliding", [False, True])
@pytest.mark.parametrize("S", [3, 4])
def test_optimal_pebbling_2x2x2_by_exhaustive_search(sliding, S):
    """Exact least I/O of the 2x2x2 MMM CDAG: the optimal schedule replays in the
    simulator at that cost, lies above Theorem 1 and the trivial count (every
    input loaded, every output stored: 12), and below every Listing-1 tiling that
    fits in S."""
    m = n = k = 2
    io, moves = pebble.optimal_io(m, n, k, S, sliding)
    if not sliding and S == 3:
        # a compute of c(i,j,1) needs its three parents and itself red
        assert io is None
        return
    res = pebble.simulate(m, n, k, S, moves, sliding)
    assert res.io == io
    assert io >= bounds.thm1(m, n, k, S) and io >= 12
    tilings = [(a, b) for a in (1, 2) for b in (1, 2)
               if pebble.listing1_working_set(a, b, sliding) <= S]
    assert tilings
    for a, b in tilings:
        sched = pebble.listing1_schedule(m, n, k, a, b, sliding)
        assert io <= pebble.simulate(m, n, k, S, sched, sliding).io

