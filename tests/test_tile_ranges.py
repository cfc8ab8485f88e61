"""The tile binning's per-axis tile set, restated in Python: the tiles met by the node
range [ceil(r - reach), floor(r + reach)], clipped to the lattice or wrapped on a periodic
axis, computed as one or two contiguous runs (the kernel's way) and by visiting every node
of the range (the definition). Same sets for random centres, reaches, lattice and tile
sizes, including ranges longer than a periodic axis and centres outside the lattice."""
import math

import numpy as np


def _by_nodes(r, reach, n, per, T):
    if not (-2.0 * n < r < 3.0 * n):
        return set()
    out = set()
    for q in range(math.ceil(r - reach), math.floor(r + reach) + 1):
        if per:
            out.add((q % n) // T)
        elif 0 <= q < n:
            out.add(q // T)
    return out


def _by_runs(r, reach, n, per, T):
    if not (-2.0 * n < r < 3.0 * n):
        return []
    lo, hi = math.ceil(r - reach), math.floor(r + reach)
    if lo > hi:
        return []
    nt = (n + T - 1) // T
    out = []

    def run(t0, t1):
        out.extend(range(t0, t1 + 1))

    if not per:
        lo, hi = max(lo, 0), min(hi, n - 1)
        if lo <= hi:
            run(lo // T, hi // T)
    elif hi - lo + 1 >= n:
        run(0, nt - 1)
    else:
        lw = lo % n
        hw = lw + (hi - lo)
        if hw < n:
            run(lw // T, hw // T)
        else:
            a0, b1 = lw // T, (hw - n) // T
            if b1 >= a0:
                run(0, nt - 1)
            else:
                run(a0, nt - 1)
                run(0, b1)
    return out


def test_tile_runs_equal_node_visits():
    g = np.random.default_rng(21)
    for _ in range(20000):
        n = int(g.integers(1, 200))
        T = int(g.choice([8, 16, 32]))
        per = bool(g.integers(0, 2))
        reach = float(g.uniform(0.0, 1.2 * n if g.random() < 0.1 else 12.0))
        r = float(g.uniform(-0.3 * n - 10, 1.3 * n + 10))
        runs = _by_runs(r, reach, n, per, T)
        assert len(runs) == len(set(runs))          # no tile twice
        assert set(runs) == _by_nodes(r, reach, n, per, T), (r, reach, n, per, T)
