"""The paper's closed forms and exhaustive searches (test infrastructure only).

Sequential (Sec. 5):
  thm1(m,n,k,S)           Theorem 1: Q >= 2mnk/sqrt(S) + mn.
  xs_io(m,n,k,S)          X=S schedule I/O: 2mnk/(sqrt(S+1)-1) + mn (Sec. 5.2).
  corollary_factor(S,a,b) optimal greedy I/O factor sqrt(S)(a+b)/(ab) (Corollary).
  aopt_closed(S), bopt_closed(S)   eq. (aopt), (bopt) as printed.
  find_seq_schedule(S)    brute-force integer argmax of ab/(a+b) s.t. ab+a+1 <= S
                          (Sec. 5.2 optimisation problem).  Ties: smaller ab, then a <= b.
Parallel (Sec. 6):
  opt_tile_shape(m,n,k,p,S)  eq. optTileShape: a = min(sqrt S, (mnk/p)^(1/3)),
                             b = max(mnk/(pS), (mnk/p)^(1/3)).
  thm2(m,n,k,p,S)         Theorem 2 as printed: min(2mnk/(p sqrt S) + S, 3(mnk/p)^(2/3)).
  cosma_cost(m,n,k,p,S)   the schedule's own cost 2V/a + a^2 with a from optTileShape
                          (reading: the min in Theorem 2 is a bound, not the cost).
  step_size(S,a), rounds(S,a,b)   Alg. 1: s = floor((S - a^2)/(2a)), t = ceil(b/s).
  latency(a,b,S)          ceil(2ab/(S - a^2)) (Sec. 6.3).
  table2_tall_cosma(p)    Table 2, tall case COSMA entry p(3 - 2^(1/3))/2^(4/3).
  fit_ranks(m,n,k,p,delta)   exhaustive search over grids [pm,pn,pk] (Sec. 7.1):
                          minimise the per-processor communicated words
                          ceil(m/pm)ceil(k/pk) + ceil(k/pk)ceil(n/pn) + ceil(m/pm)ceil(n/pn)
                          over grids that leave at most floor(delta p) processors idle;
                          ties: more processors, then lexicographically smaller grid.

Pins (tests/test_oracle_bounds.py): brute force vs the printed closed form, the
Fig. 6 grid trade-off (p=65: 1x5x13 vs 4x4x4, -36% words, +1.5625% work), the
9216 -> 9217 core stability of Sec. 9, the Table 2 tall entry against the
general formula, and the Theorem 2 regime switch.
"""

import math


def thm1(m, n, k, S):
    return 2.0 * m * n * k / math.sqrt(S) + m * n


def xs_io(m, n, k, S):
    return 2.0 * m * n * k / (math.sqrt(S + 1) - 1.0) + m * n


def corollary_factor(S, a, b):
    return math.sqrt(S) * (a + b) / (a * b)


def aopt_closed(S):
    r = math.sqrt((S - 1) ** 3)
    return math.floor((r - S + 1) / (S - 2))


def bopt_closed(S):
    r = math.sqrt((S - 1) ** 3)
    return math.floor(-(2 * S + r - S * S - 1) / (r - S + 1))


def find_seq_schedule(S):
    """Integer (a, b) maximising ab/(a+b) subject to ab + a + 1 <= S."""
    best = None
    for a in range(1, S):
        bmax = (S - a - 1) // a
        for b in range(1, bmax + 1):
            rho_num, rho_den = a * b, a + b
            key = (rho_num / rho_den, -(a * b), -a)
            if best is None or key > best[0]:
                best = (key, a, b)
    if best is None:
        raise ValueError("S too small for any tile")
    return best[1], best[2]


def opt_tile_shape(m, n, k, p, S):
    v = m * n * k / p
    a = min(math.sqrt(S), v ** (1.0 / 3.0))
    b = max(v / S, v ** (1.0 / 3.0))
    return a, b


def thm2(m, n, k, p, S):
    v = m * n * k / p
    return min(2.0 * v / math.sqrt(S) + S, 3.0 * v ** (2.0 / 3.0))


def cosma_cost(m, n, k, p, S):
    v = m * n * k / p
    a, _ = opt_tile_shape(m, n, k, p, S)
    return 2.0 * v / a + a * a


def step_size(S, a):
    return (S - a * a) // (2 * a)


def rounds(S, a, b):
    s = step_size(S, a)
    return math.inf if s <= 0 else -(-b // s)


def latency(a, b, S):
    return math.ceil(2 * a * b / (S - a * a))


def table2_tall_cosma(p):
    return p * (3.0 - 2.0 ** (1.0 / 3.0)) / 2.0 ** (4.0 / 3.0)


def table2_tall_general(p):
    """The general COSMA cost for the tall case m = n = sqrt(p), k = p^(3/2)/4,
    counting only words a processor does not own initially.  Reading: the
    inputs start evenly distributed ((mk + nk)/p words of A and B per
    processor) while C does not, so 3 (mnk/p)^(2/3) - (mk + nk)/p."""
    m = n = math.sqrt(p)
    k = p ** 1.5 / 4.0
    return 3.0 * (m * n * k / p) ** (2.0 / 3.0) - (m * k + n * k) / p


def _cdiv(a, b):
    return -(-a // b)


def grid_words(m, n, k, pm, pn, pk):
    lm, ln, lk = _cdiv(m, pm), _cdiv(n, pn), _cdiv(k, pk)
    return lm * lk + lk * ln + lm * ln


def grid_work(m, n, k, pm, pn, pk):
    return _cdiv(m, pm) * _cdiv(n, pn) * _cdiv(k, pk)


def fit_ranks(m, n, k, p, delta):
    """Exhaustive FitRanks over all grids pm*pn*pk in [p - floor(delta p), p]."""
    min_used = p - math.floor(delta * p)
    best = None
    for pm in range(1, min(m, p) + 1):
        for pn in range(1, min(n, p // pm) + 1):
            for pk in range(1, min(k, p // (pm * pn)) + 1):
                used = pm * pn * pk
                if used < min_used:
                    continue
                key = (grid_words(m, n, k, pm, pn, pk), -used, (pm, pn, pk))
                if best is None or key < best:
                    best = key
    return None if best is None else best[2]
