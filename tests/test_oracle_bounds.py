"""Pins for the paper's closed forms and searches (oracle/bounds.py)."""
import math

import pytest

from oracle import bounds


def _brute_rho(S):
    best = 0.0
    for a in range(1, S):
        for b in range(1, S):
            if a * b + a + 1 <= S:
                best = max(best, a * b / (a + b))
    return best


@pytest.mark.parametrize("S", [5, 10, 16, 37, 64, 100, 257, 1000])
def test_find_seq_schedule_is_optimal(S):
    a, b = bounds.find_seq_schedule(S)
    assert a * b + a + 1 <= S
    assert a * b / (a + b) == pytest.approx(_brute_rho(S))


@pytest.mark.parametrize("S,closed,integer", [
    (5, (1, 2), (1, 3)), (64, (7, 7), (7, 8)), (100, (9, 9), (9, 10)),
    (1000, (30, 31), (31, 31)), (4096, (63, 63), (63, 64))])
def test_closed_form_vs_integer_optimum(S, closed, integer):
    # eq. (aopt)/(bopt) are the continuous optimum floored; the integer optimum
    # of the same problem can differ by one (the reading taken in the planner).
    assert (bounds.aopt_closed(S), bounds.bopt_closed(S)) == closed
    assert bounds.find_seq_schedule(S) == integer


def test_closed_form_below_sqrt_s():
    for S in (10, 100, 1000, 10 ** 5):
        assert bounds.aopt_closed(S) < math.sqrt(S)
        assert bounds.bopt_closed(S) < math.sqrt(S)


def test_greedy_optimum_intensity():
    # eq. (seqSolution): with a = b = sqrt(S), rho = sqrt(S)/2, so Q = 2mnk/sqrt(S)
    S = 49
    a = b = 7
    assert a * b / (a + b) == pytest.approx(math.sqrt(S) / 2)
    assert bounds.corollary_factor(S, a, b) == pytest.approx(2 / math.sqrt(S) * math.sqrt(S))


def test_xs_factor_tends_to_one():
    m = n = k = 1000
    for S in (100, 10 ** 4, 10 ** 6):
        ratio = (bounds.xs_io(m, n, k, S) - m * n) / (bounds.thm1(m, n, k, S) - m * n)
        assert ratio == pytest.approx(math.sqrt(S) / (math.sqrt(S + 1) - 1))
    assert math.sqrt(1e6) / (math.sqrt(1e6 + 1) - 1) - 1 < 1.1e-3


def test_optimality_gap_words_reading():
    # "0.03% for 10MB": sqrt(S)/(sqrt(S+1)-1) - 1 ~ 1/sqrt(S) is 0.03% for S = 10^7 words
    S = 10 ** 7
    gap = math.sqrt(S) / (math.sqrt(S + 1) - 1) - 1
    assert 0.0003 < gap < 0.00035


def test_opt_tile_shape_regimes():
    S = 1000.0
    # small p: a = sqrt(S) (I/O constraint binding), b = mnk/(pS)
    a, b = bounds.opt_tile_shape(1000, 1000, 1000, 8, S)
    assert a == pytest.approx(math.sqrt(S)) and b == pytest.approx(1e9 / 8 / S)
    # large p: cubic domain
    a, b = bounds.opt_tile_shape(1000, 1000, 1000, 10 ** 6, S)
    assert a == pytest.approx(10.0) and b == pytest.approx(10.0)
    # binding threshold p = mnk / S^{3/2}
    pth = 1e9 / S ** 1.5
    a1, _ = bounds.opt_tile_shape(1000, 1000, 1000, pth * 0.99, S)
    a2, _ = bounds.opt_tile_shape(1000, 1000, 1000, pth * 1.01, S)
    assert a1 == pytest.approx(math.sqrt(S)) and a2 < math.sqrt(S)


def test_cosma_cost_vs_theorem2():
    S = 1000.0
    for p in (4, 64, 1024, 10 ** 5):
        c = bounds.cosma_cost(4096, 4096, 4096, p, S)
        assert c >= bounds.thm2(4096, 4096, 4096, p, S) - 1e-6 * c
    # in the a = sqrt(S) regime the schedule's cost is the first branch
    p = 4
    assert bounds.cosma_cost(4096, 4096, 4096, p, S) == pytest.approx(
        2 * 4096 ** 3 / (p * math.sqrt(S)) + S)


def test_step_size_and_rounds():
    # Alg. 1 with a < sqrt(S): s = floor((S - a^2)/(2a)), t = ceil(b/s)
    assert bounds.step_size(100, 8) == 2
    assert bounds.rounds(100, 8, 9) == 5
    # a = sqrt(S) leaves no room for a step (reading: reserve stages first)
    assert bounds.step_size(100, 10) == 0 and bounds.rounds(100, 10, 5) == math.inf
    assert bounds.latency(8, 9, 100) == math.ceil(144 / 36)


@pytest.mark.parametrize("e", range(9, 16))
def test_table2_tall_entry(e):
    p = 2 ** e
    assert bounds.table2_tall_general(p) == pytest.approx(bounds.table2_tall_cosma(p), rel=1e-12)
    assert bounds.table2_tall_cosma(p) == pytest.approx(0.69 * p, rel=0.01)


def test_fig6_grid_tradeoff():
    n = 4160  # divisible by 4, 5, 13 and 64
    w_513 = bounds.grid_words(n, n, n, 1, 5, 13)
    w_444 = bounds.grid_words(n, n, n, 4, 4, 4)
    assert w_444 / w_513 == pytest.approx(0.641, abs=1e-3)   # "-36% communication"
    work_65 = n ** 3 / 65
    assert bounds.grid_work(n, n, n, 4, 4, 4) / work_65 - 1 == pytest.approx(0.015625)  # "+1.5%"
    assert bounds.fit_ranks(n, n, n, 65, 0.03) == (4, 4, 4)
    # without idle processors, only factorisations of 65 remain
    assert sorted(bounds.fit_ranks(n, n, n, 65, 0.0)) == [1, 5, 13]


def test_unfavourable_processor_count_is_ignored():
    # Sec. 9: on 9217 = 13 * 709 cores the grid of 9216 cores is kept
    n = 16384
    g1 = bounds.fit_ranks(n, n, n, 9216, 0.03)
    g2 = bounds.fit_ranks(n, n, n, 9217, 0.03)
    assert g1 == g2
    assert g1[0] * g1[1] * g1[2] <= 9216
