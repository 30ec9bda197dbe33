"""Red-blue pebble game simulator for the MMM CDAG (test infrastructure only).

Game (Sec. 2.2, after Hong and Kung): a vertex holding a blue pebble may get a
red one (load); a red one may get a blue one (store); a vertex whose parents all
hold red pebbles may get a red one (compute); any pebble may be removed (free).
At most S red pebbles at any time.  Initially only the inputs are blue; at the
end every output must be blue.  The I/O cost Q is the number of loads plus
stores (Sec. 2.3).

CDAG of classical MMM (Sec. 5.1): inputs ('a', i, t) and ('b', t, j); partial
sums ('c', i, j, t) for t = 0..k-1, whose parents are ('a', i, t), ('b', t, j)
and, for t > 0, ('c', i, j, t-1).  The outputs are ('c', i, j, k-1).

Reading taken (the paper counts the Listing-1 working set as ab + a + 1 words,
Sec. 5.2 attainability): that count holds when the new partial sum may take over
the red pebble of the previous one, the "sliding" move.  `sliding=False` is the
strict game, where one more pebble is needed during a compute.  Both modes are
simulated and tested.

A schedule is a sequence of moves (op, vertex) with op in
{'load', 'store', 'compute', 'free'}; the simulator checks every rule and
returns the counts.  Schedule builders below produce the paper's Listing 1
(rank-1-update, C-stationary tiling), the X=S schedule of Sec. 5.2, and the
replay of a GPU plan given as a list of work units (tile rectangle, k range).

`optimal_io` finds the least I/O of any complete pebbling by exhaustive search
(0-1 breadth-first search over (red set, blue outputs) states) for tiny
products; it returns the optimal schedule as moves, which `simulate` replays.

Pins (tests/test_oracle_pebble.py): Listing-1 I/O equals the Corollary's count
sum_tiles (k (h + w) + h w) (= mnk(1/a + 1/b) + mn when tiles divide), the X=S
schedule matches 2mnk/(sqrt(S+1)-1) + mn, every valid schedule is >= Theorem 1,
and planted rule violations (load of a non-blue vertex, exceeding S, computing
without a parent, ending without outputs) are rejected.
"""

from dataclasses import dataclass


class PebbleError(Exception):
    pass


@dataclass
class PebbleResult:
    loads: int
    stores: int
    max_red: int
    computes: int

    @property
    def io(self):
        return self.loads + self.stores


def parents(v):
    if v[0] != "c":
        return ()
    _, i, j, t = v
    ps = [("a", i, t), ("b", t, j)]
    if t > 0:
        ps.append(("c", i, j, t - 1))
    return tuple(ps)


def simulate(m, n, k, S, moves, sliding=False):
    """Replay `moves` on the MMM CDAG of an (m x k)(k x n) product with S red pebbles."""
    red = set()
    blue = set()
    for i in range(m):
        for t in range(k):
            blue.add(("a", i, t))
    for t in range(k):
        for j in range(n):
            blue.add(("b", t, j))
    loads = stores = computes = 0
    max_red = 0

    def in_cdag(v):
        if v[0] == "a":
            return 0 <= v[1] < m and 0 <= v[2] < k
        if v[0] == "b":
            return 0 <= v[1] < k and 0 <= v[2] < n
        if v[0] == "c":
            return 0 <= v[1] < m and 0 <= v[2] < n and 0 <= v[3] < k
        return False

    for step, (op, v) in enumerate(moves):
        if not in_cdag(v):
            raise PebbleError(f"step {step}: {v} is not a CDAG vertex")
        if op == "load":
            if v not in blue:
                raise PebbleError(f"step {step}: load of {v} without a blue pebble")
            if v not in red:
                red.add(v)
            loads += 1
        elif op == "store":
            if v not in red:
                raise PebbleError(f"step {step}: store of {v} without a red pebble")
            blue.add(v)
            stores += 1
        elif op == "compute":
            ps = parents(v)
            if not ps:
                raise PebbleError(f"step {step}: {v} is an input and cannot be computed")
            for p in ps:
                if p not in red:
                    raise PebbleError(f"step {step}: compute {v} but parent {p} is not red")
            if sliding and v[3] > 0:
                red.discard(("c", v[1], v[2], v[3] - 1))
            red.add(v)
            computes += 1
        elif op == "free":
            if v not in red:
                raise PebbleError(f"step {step}: free of {v} which holds no red pebble")
            red.discard(v)
        else:
            raise PebbleError(f"step {step}: unknown move {op!r}")
        if len(red) > S:
            raise PebbleError(f"step {step}: {len(red)} red pebbles exceed S={S}")
        max_red = max(max_red, len(red))

    for i in range(m):
        for j in range(n):
            if k > 0 and ("c", i, j, k - 1) not in blue:
                raise PebbleError(f"output ({i},{j}) holds no blue pebble at the end")
    return PebbleResult(loads, stores, max_red, computes)


def _tile_moves(rows, cols, k0, k1, sliding, load_c_from=None, store_c=True):
    """Moves of one C-stationary tile: rows x cols partial sums kept red while
    the k range [k0, k1) streams one A column (len(rows)) and one B element at a
    time (the rank-1 update order of Listing 1)."""
    moves = []
    if load_c_from is not None:
        for i in rows:
            for j in cols:
                moves.append(("load", ("c", i, j, load_c_from)))
    for r in range(k0, k1):
        for i in rows:
            moves.append(("load", ("a", i, r)))
        for j in cols:
            moves.append(("load", ("b", r, j)))
            for i in rows:
                moves.append(("compute", ("c", i, j, r)))
                if r > 0 and not sliding:
                    moves.append(("free", ("c", i, j, r - 1)))
            moves.append(("free", ("b", r, j)))
        for i in rows:
            moves.append(("free", ("a", i, r)))
    if k1 > k0:
        for i in rows:
            for j in cols:
                if store_c:
                    moves.append(("store", ("c", i, j, k1 - 1)))
                moves.append(("free", ("c", i, j, k1 - 1)))
    return moves


def listing1_schedule(m, n, k, a, b, sliding=False):
    """Listing 1 with 0-based half-open tiles [i1*a, min((i1+1)a, m)) x [j1*b, ...)
    (the reading of its garbled loop bounds), k loop outermost inside a tile."""
    moves = []
    for i1 in range(-(-m // a)):
        for j1 in range(-(-n // b)):
            rows = range(i1 * a, min((i1 + 1) * a, m))
            cols = range(j1 * b, min((j1 + 1) * b, n))
            moves += _tile_moves(rows, cols, 0, k, sliding)
    return moves


def listing1_working_set(a, b, sliding):
    """Red pebbles Listing 1 needs: ab partial sums + a A elements + 1 B element,
    plus one for the new partial sum in the strict game."""
    return a * b + a + 1 + (0 if sliding else 1)


def xs_tile(S):
    """Side of the X=S schedule of Sec. 5.2: vectors of length sqrt(S+1) - 1."""
    import math
    r = math.isqrt(S + 1)
    return r - 1


def xs_schedule(m, n, k, S, sliding=False):
    s = xs_tile(S)
    return listing1_schedule(m, n, k, s, s, sliding)


def plan_schedule(m, n, k, units, sliding=False):
    """Replay of a GPU plan.  `units` is a list of work units
    (r0, r1, c0, c1, k0, k1) in execution order: C rows [r0,r1) x cols [c0,c1)
    over the k range [k0, k1).  A unit that does not start at k = 0 continues
    the partial-sum chain of the unit before it in k (it loads c(i,j,k0-1));
    every unit stores its last partial sums -- the split-k reduction is modelled
    as storing and reloading the boundary partial sum of each k segment."""
    moves = []
    for (r0, r1, c0, c1, k0, k1) in units:
        rows = range(r0, r1)
        cols = range(c0, c1)
        moves += _tile_moves(rows, cols, k0, k1, sliding,
                             load_c_from=(k0 - 1) if k0 > 0 else None)
    return moves


def tile_io(m, n, k, a, b):
    """The Corollary's count for the a x b tiling: sum over tiles of
    k (h + w) + h w, h and w the tile's actual height and width."""
    q = 0
    for i1 in range(-(-m // a)):
        h = min((i1 + 1) * a, m) - i1 * a
        for j1 in range(-(-n // b)):
            w = min((j1 + 1) * b, n) - j1 * b
            q += k * (h + w) + h * w
    return q


def optimal_io(m, n, k, S, sliding=False):
    """Least I/O over all complete pebblings of the (m x k)(k x n) MMM CDAG with S
    red pebbles (exhaustive; tiny sizes only), and one optimal move sequence, or
    (None, None) when no complete pebbling exists.  Moves that never help are
    not generated (loading a red vertex, storing an input, storing a stored
    vertex); all others are, with loads and stores costing 1 and computes and
    frees 0."""
    from collections import deque
    verts = ([("a", i, t) for i in range(m) for t in range(k)] +
             [("b", t, j) for t in range(k) for j in range(n)] +
             [("c", i, j, t) for i in range(m) for j in range(n) for t in range(k)])
    index = {v: x for x, v in enumerate(verts)}
    nv = len(verts)
    first_c = m * k + k * n
    inputs = (1 << first_c) - 1
    par = [0] * nv
    pred = [0] * nv  # sliding: the red pebble a compute takes over
    for v, x in index.items():
        if v[0] == "c":
            for p in parents(v):
                par[x] |= 1 << index[p]
            if v[3] > 0:
                pred[x] = 1 << index[("c", v[1], v[2], v[3] - 1)]
    goal = 0
    for i in range(m):
        for j in range(n):
            goal |= 1 << index[("c", i, j, k - 1)]
    start = (0, 0)  # (red mask, blue mask over non-input vertices)
    dist = {start: 0}
    back = {start: None}
    dq = deque([start])
    end = None
    while dq:
        st = dq.popleft()
        d = dist[st]
        red, blue = st
        if blue & goal == goal:
            end = st
            break
        nred = bin(red).count("1")

        def relax(ns, cost, move):
            nd = d + cost
            if ns not in dist or dist[ns] > nd:
                dist[ns] = nd
                back[ns] = (st, move)
                if cost:
                    dq.append(ns)
                else:
                    dq.appendleft(ns)

        for x in range(nv):
            bit = 1 << x
            if red & bit:
                relax((red & ~bit, blue), 0, ("free", verts[x]))
                if x >= first_c and not blue & bit:
                    relax((red, blue | bit), 1, ("store", verts[x]))
                continue
            if (inputs | blue) & bit and nred < S:
                relax((red | bit, blue), 1, ("load", verts[x]))
            if x >= first_c and red & par[x] == par[x]:
                if sliding and pred[x]:
                    relax(((red & ~pred[x]) | bit, blue), 0, ("compute", verts[x]))
                elif nred < S:
                    relax((red | bit, blue), 0, ("compute", verts[x]))
    if end is None:
        return None, None
    moves = []
    st = end
    while back[st] is not None:
        st, mv = back[st]
        moves.append(mv)
    moves.reverse()
    return dist[end], moves

