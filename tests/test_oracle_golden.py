"""Pins of the oracle's planning and bound formulas against values the paper
prints (tests/golden/paper_printed_values.txt, each with its passage)."""
import os

import pytest

from oracle import bounds

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_printed_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, value, _ = (x.strip() for x in line.split("|", 2))
            out[key] = value
    return out


G = _golden()


def _grid(s):
    return tuple(int(x) for x in s.split("x"))


def test_fig6_grids_and_tradeoff():
    p = int(G["fig6.processors"])
    n = 4160  # square and divisible by every grid side involved
    idle = _grid(G["fig6.grid_idle"])
    full = _grid(G["fig6.grid_all"])
    assert bounds.fit_ranks(n, n, n, p, 0.03) == idle
    assert sorted(bounds.fit_ranks(n, n, n, p, 0.0)) == sorted(full)
    work = bounds.grid_work(n, n, n, *idle) / (n ** 3 / p) - 1
    assert work * 100 == pytest.approx(float(G["fig6.extra_computation_percent"]), abs=0.1)
    comm = 1 - bounds.grid_words(n, n, n, *idle) / bounds.grid_words(n, n, n, *full)
    assert comm * 100 == pytest.approx(float(G["fig6.communication_reduction_percent"]), abs=0.5)


def test_sec9_extra_core_is_not_used():
    n = int(G["sec9.mnk"])
    p1, p2 = int(G["sec9.p1"]), int(G["sec9.p2"])
    g1 = bounds.fit_ranks(n, n, n, p1, 0.03)
    g2 = bounds.fit_ranks(n, n, n, p2, 0.03)
    assert g1 == g2 and g1[0] * g1[1] * g1[2] <= p1


@pytest.mark.parametrize("e", [9, 12, 15])
def test_table2_tall_cosma_coefficient(e):
    p = 2 ** e
    assert bounds.table2_tall_cosma(p) / p == pytest.approx(float(G["table2.tall.cosma_per_p"]),
                                                           rel=0.01)
