"""The kernel's way of counting subdivision samples, restated in numpy FP32 and checked
against counting every sample with the documented predicate (Sec. 2.4 subdivision,
evaluated in FP32 with round-to-nearest in a fixed order): along a sample row the squared
normalised radius is a quadratic in the x offset, and the samples of the row where it is
below 1 - 1e-3 form an interval (counted by index arithmetic), those where it is above
1 + 1e-3 lie outside a wider one; only the samples between the two run the predicate.
The margins are far above the rounding of the set-up and of the predicate (about 1e-5),
so the counts agree exactly, for spheres and ellipsoids (the sheared suspension's
(6, 2, 2) and random shapes), at nodes near the surface where the samples straddle it
and on rows that graze it. The whole-node bounds that spare most nodes a count are
checked the same way, and so is the kernel's count for a warp's row of nodes at once (the
needing nodes' samples mapped onto one grid along x)."""
import numpy as np

f32 = np.float32
MARGIN = 1e-3


def _so(n):
    return [f32(f32(2 * i + 1 - n) / f32(2 * n)) for i in range(n)]


def _pred_ell(mm, dx, dy, dz):
    t0 = f32(f32(mm[0] * dx) + f32(mm[1] * dy))
    t1 = f32(f32(mm[3] * dx) + f32(mm[4] * dy))
    t2 = f32(f32(mm[6] * dx) + f32(mm[7] * dy))
    q0 = f32(t0 + f32(mm[2] * dz))
    q1 = f32(t1 + f32(mm[5] * dz))
    q2 = f32(t2 + f32(mm[8] * dz))
    return f32(f32(f32(q0 * q0) + f32(q1 * q1)) + f32(q2 * q2)) < f32(1)


def _pred_sph(dx, yy, zz, R2):
    return f32(f32(f32(dx * dx) + yy) + zz) < R2


def _count_all(kind, par, px, py, pz, n):
    """Every one of the n^3 samples through the predicate (the method's definition)."""
    so = _so(n)
    c = 0
    for j in range(n):
        dy = f32(py + so[j])
        for q in range(n):
            dz = f32(pz + so[q])
            for i in range(n):
                dx = f32(px + so[i])
                c += _pred_sph(dx, f32(dy * dy), f32(dz * dz), par) if kind == 0 else _pred_ell(par, dx, dy, dz)
    return c


def _count_intervals(kind, par, px, py, pz, n, stats, dt=f32):
    """The kernel's count: per sample row (fixed y, z offsets) the interval where the
    quadratic F(X) = A X^2 + 2 B X + C is below 1 - 1e-3 (shrunk by 2e-4) and the one where
    it is at most 1 + 1e-3 (grown by 2e-4); samples in the first count, samples outside the
    second do not, the rest run the predicate. Set up in `dt` arithmetic (the margins make
    the rounding of the set-up irrelevant)."""
    so = _so(n)
    if kind == 0:
        thr = dt(par)
        iA = dt(1)
    else:
        mm = [dt(v) for v in par]
        thr = dt(1)
        A = dt(mm[0] * mm[0] + mm[3] * mm[3] + mm[6] * mm[6])
        iA = dt(1) / A
    lo, hi = dt(thr * dt(1 - MARGIN)), dt(thr * dt(1 + MARGIN))
    fn, t0 = dt(n), dt(0.5 * (n - 1))
    c = 0
    for j in range(n):
        dy = f32(py + so[j])
        for q in range(n):
            dz = f32(pz + so[q])
            xc = dt(0)
            yy, zz = f32(dy * dy), f32(dz * dz)
            if kind == 0:
                Fmin = dt(dt(yy) + dt(zz))
            else:
                w = [dt(mm[1] * dt(dy) + mm[2] * dt(dz)), dt(mm[4] * dt(dy) + mm[5] * dt(dz)),
                     dt(mm[7] * dt(dy) + mm[8] * dt(dz))]
                B = dt(mm[0] * w[0] + mm[3] * w[1] + mm[6] * w[2])
                C = dt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2])
                xc = dt(-B * iA)
                Fmin = dt(C + B * xc)
            if Fmin > hi:
                continue
            ro = dt(np.sqrt(dt((hi - Fmin) * iA)) * dt(1 + 1e-5) + dt(2e-4))
            ri = dt(np.sqrt(dt((lo - Fmin) * iA)) * dt(1 - 1e-5) - dt(2e-4)) if Fmin < lo else dt(-1)
            # bounds as fractional sample indices of a node at offset 0, then of this node
            cc = dt(xc * fn + t0)
            qxn = dt(dt(px) * fn)
            oA = max(0, int(np.ceil(dt(dt(cc - ro * fn) - qxn))))
            oB = min(n - 1, int(np.floor(dt(dt(cc + ro * fn) - qxn))))
            band = list(range(oA, oB + 1))
            if ri > 0:
                ia = max(0, int(np.ceil(dt(dt(cc - ri * fn) - qxn))))
                ib = min(n - 1, int(np.floor(dt(dt(cc + ri * fn) - qxn))))
                if ia <= ib:
                    c += ib - ia + 1
                    band = [i for i in band if i < ia or i > ib]
            for i in band:
                dx = f32(px + so[i])
                stats["evaluated"] += 1
                c += _pred_sph(dx, yy, zz, f32(par)) if kind == 0 else _pred_ell(par, dx, dy, dz)
    return c


def _quick_ellipsoid(mm, px, py, pz, n):
    """The kernel's whole-node decision for an ellipsoid: with q = M p and w = M^T q, every
    sample's |M (p + c)|^2 lies within |q|^2 -/+ 2 h |w|_1 (+ G, the box's largest |M c|^2).
    Returns 0 (no sample inside), 1 (all inside) or None (count)."""
    M = np.array([[float(mm[3 * j + k]) for k in range(3)] for j in range(3)], dtype=np.float32)
    h = f32((n - 1) / (2 * n))
    p = np.array([px, py, pz], dtype=np.float32)
    q = M @ p
    s2 = f32(q @ q)
    w = M.T @ q
    l1 = f32(2 * h * np.abs(w).sum())
    G = max(float(np.sum((M.astype(np.float64) @ np.array([1.0, s1, s2_])) ** 2))
            for s1 in (1, -1) for s2_ in (1, -1)) * float(h) ** 2 * 1.0001
    slack = 1e-3 + 1e-5 * (s2 + l1)
    if s2 - l1 > 1 + slack:
        return 0
    if s2 + l1 + G < 1 - slack:
        return 1
    return None


def _ellipsoid_rows(g, semi):
    """fl32(d_j / semi_j) of a random orientation, row-major (the kernel's M)."""
    qv = g.normal(size=4)
    w, x, y, z = qv / np.linalg.norm(qv)
    Rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                    [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                    [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]).T
    return [f32(Rot[j][c] / semi[j]) for j in range(3) for c in range(3)]


def _surface_nodes(g, count):
    for t in range(count):
        if t % 3 == 0:
            yield 0, None, f32(g.uniform(2.0, 8.0) ** 2)
        else:
            semi = np.array([6.0, 2.0, 2.0]) if t % 3 == 1 else g.uniform(0.8, 6.0, 3)
            yield 1, _ellipsoid_rows(g, semi), None


def test_classified_counts_equal_full_enumeration():
    g = np.random.default_rng(11)
    stats = {"evaluated": 0}
    nodes = 0
    for kind, mm, R2 in _surface_nodes(g, 240):
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        if kind == 0:
            s = np.sqrt(float(R2)) + g.uniform(-0.8, 0.8)
            par = R2
        else:
            M = np.array([[float(mm[3 * j + c]) for c in range(3)] for j in range(3)])
            s = 1.0 / np.linalg.norm(M @ d) + g.uniform(-0.8, 0.8)
            par = mm
        px, py, pz = (f32(v) for v in d * s)
        n = 10 if nodes % 4 else int(g.integers(1, 17))
        full = _count_all(kind, par, px, py, pz, n)
        assert _count_intervals(kind, par, px, py, pz, n, stats) == full
        assert _count_intervals(kind, par, px, py, pz, n, {"evaluated": 0}, dt=np.float64) == full
        nodes += 1
    # the predicate ran on a few samples per node instead of n^3
    assert stats["evaluated"] < 5 * nodes, stats


def test_counts_at_tangent_rows():
    """Samples on the surface to a few FP32 units (a node placed so that one chosen sample
    sits on it), on rows crossing the surface and on rows that graze it (the sample at the
    row's closest point): there the set-up's rounding alone would decide wrongly, so these
    cases fail if the margins are taken out."""
    g = np.random.default_rng(12)
    n = 10
    so = [float(v) for v in _so(n)]
    for t in range(600):
        kind = 0 if t % 3 == 0 else 1
        i, j, q = (int(v) for v in g.integers(0, n, 3))
        d = g.normal(size=3)
        if t % 2:
            d[0] = 0.0   # the surface normal across the row: the row grazes the surface
        d /= np.linalg.norm(d)
        if kind == 0:
            R2 = f32(g.uniform(2.0, 8.0) ** 2)
            S = d * np.sqrt(float(R2))
            par = R2
        else:
            mm = _ellipsoid_rows(g, np.array([6.0, 2.0, 2.0]) if t % 3 == 1 else g.uniform(0.8, 6.0, 3))
            M = np.array([[float(mm[3 * a + c]) for c in range(3)] for a in range(3)])
            if t % 2:
                # a surface point whose normal M^T M S is across the row (no x component)
                S = np.linalg.solve(M.T @ M, d)
                S /= np.linalg.norm(M @ S)
            else:
                S = d / np.linalg.norm(M @ d)
            par = mm
        S = S * (1.0 + g.uniform(-4e-7, 4e-7))
        px, py, pz = f32(S[0] - so[i]), f32(S[1] - so[j]), f32(S[2] - so[q])
        assert _count_intervals(kind, par, px, py, pz, n, {"evaluated": 0}) == _count_all(kind, par, px, py, pz, n)


def test_quick_ellipsoid_decisions_are_exact():
    """Nodes the whole-node bounds decide have no sample inside (0) or every sample inside
    (1), checked by counting every sample; near the surface the bounds leave the node to
    the count."""
    g = np.random.default_rng(13)
    decided = {0: 0, 1: 0, None: 0}
    for t in range(300):
        mm = _ellipsoid_rows(g, np.array([6.0, 2.0, 2.0]) if t % 2 else g.uniform(0.8, 6.0, 3))
        M = np.array([[float(mm[3 * j + c]) for c in range(3)] for j in range(3)])
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        s = 1.0 / np.linalg.norm(M @ d) + g.uniform(-2.0, 2.0)
        px, py, pz = (f32(v) for v in d * s)
        n = 6
        r = _quick_ellipsoid(mm, px, py, pz, n)
        decided[r] += 1
        if r is not None:
            assert _count_all(1, mm, px, py, pz, n) == r * n ** 3
    assert decided[0] > 20 and decided[1] > 10 and decided[None] > 20, decided


def _row_setup(kind, par, py, pz, j, q, n, dt=f32):
    """Per-row set-up shared by a warp's nodes: the intervals as fractional sample indices
    of a node at x offset 0 (None when the row cannot reach inside)."""
    so = _so(n)
    dy, dz = f32(py + so[j]), f32(pz + so[q])
    yy, zz = f32(dy * dy), f32(dz * dz)
    fn, t0 = dt(n), dt(0.5 * (n - 1))
    if kind == 0:
        thr, iA, xc = dt(par), dt(1), dt(0)
        Fmin = dt(dt(yy) + dt(zz))
    else:
        mm = [dt(v) for v in par]
        thr = dt(1)
        iA = dt(1) / dt(mm[0] * mm[0] + mm[3] * mm[3] + mm[6] * mm[6])
        w = [dt(mm[1] * dt(dy) + mm[2] * dt(dz)), dt(mm[4] * dt(dy) + mm[5] * dt(dz)),
             dt(mm[7] * dt(dy) + mm[8] * dt(dz))]
        B = dt(mm[0] * w[0] + mm[3] * w[1] + mm[6] * w[2])
        C = dt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2])
        xc = dt(-B * iA)
        Fmin = dt(C + B * xc)
    lo, hi = dt(thr * dt(1 - MARGIN)), dt(thr * dt(1 + MARGIN))
    if Fmin > hi:
        return None
    ro = dt(np.sqrt(dt((hi - Fmin) * iA)) * dt(1 + 1e-5) + dt(2e-4))
    ri = dt(np.sqrt(dt((lo - Fmin) * iA)) * dt(1 - 1e-5) - dt(2e-4)) if Fmin < lo else dt(-1)
    cc = dt(xc * fn + t0)
    inner = (dt(cc - ri * fn), dt(cc + ri * fn)) if ri > 0 else None
    return dict(outer=(dt(cc - ro * fn), dt(cc + ro * fn)), inner=inner, dy=dy, dz=dz, yy=yy, zz=zz)


def _count_row_of_nodes(kind, par, px, need, py, pz, n):
    """The kernel's count for the needing nodes of one x-row: node L's sample i is grid
    sample (L - Lmin) n + i; each sample row's intervals are mapped onto the grid once, the
    samples between them run the predicate, the inner interval's overlap with each node's
    n grid samples is its count."""
    so = _so(n)
    L0, L1 = min(need), max(need)
    bn = f32(px[L0] * f32(n))
    S = (L1 - L0 + 1) * n
    cnt = {L: 0 for L in need}
    for j in range(n):
        for q in range(n):
            r = _row_setup(kind, par, py, pz, j, q, n)
            if r is None:
                continue
            oA = max(0, int(np.ceil(f32(r["outer"][0] - bn))))
            oB = min(S - 1, int(np.floor(f32(r["outer"][1] - bn))))
            gA, gB = 0, -1
            if r["inner"] is not None:
                gA = max(0, int(np.ceil(f32(r["inner"][0] - bn))))
                gB = min(S - 1, int(np.floor(f32(r["inner"][1] - bn))))
            for g in range(oA, oB + 1):
                if gA <= g <= gB:
                    continue
                L, i = L0 + g // n, g % n
                if L in cnt:
                    dx = f32(px[L] + so[i])
                    cnt[L] += _pred_sph(dx, r["yy"], r["zz"], f32(par)) if kind == 0 else \
                        _pred_ell(par, dx, r["dy"], r["dz"])
            for L in cnt:
                w0 = (L - L0) * n
                cnt[L] += max(0, min(gB, w0 + n - 1) - max(gA, w0) + 1)
    return cnt


def test_row_of_nodes_on_one_grid():
    """x-rows of 32 nodes (FP64 centre, offsets rounded to FP32 as the kernel does) through
    spheres and ellipsoids, the nodes whose samples straddle the surface counted at once:
    every count equals full enumeration."""
    g = np.random.default_rng(14)
    n = 10
    rows = 0
    for t in range(36):
        kind = 0 if t % 3 == 0 else 1
        if kind == 0:
            par = f32(g.uniform(2.0, 7.0) ** 2)
            reach = float(np.sqrt(float(par)))
        else:
            semi = np.array([6.0, 2.0, 2.0]) if t % 3 == 1 else g.uniform(0.8, 6.0, 3)
            par = _ellipsoid_rows(g, semi)
            reach = float(max(semi))
        p = np.array([g.uniform(100.0, 300.0), g.uniform(0.0, 200.0), g.uniform(0.0, 100.0)])
        x0 = int(np.floor(p[0])) - 16
        y = int(np.floor(p[1] + g.uniform(-0.8, 0.8) * reach))
        z = int(np.floor(p[2] + g.uniform(-0.8, 0.8) * reach))
        px = [f32(float(x0 + L) - p[0]) for L in range(32)]
        py, pz = f32(float(y) - p[1]), f32(float(z) - p[2])
        full = [_count_all(kind, par, px[L], py, pz, n) for L in range(32)]
        need = [L for L in range(32) if 0 < full[L] < n ** 3]
        if not need:
            continue
        got = _count_row_of_nodes(kind, par, px, need, py, pz, n)
        assert all(got[L] == full[L] for L in need), (t, [(L, got[L], full[L]) for L in need])
        rows += 1
    assert rows > 20


def test_row_shadow_prefilter_keeps_every_touching_row():
    """The row prefilter for ellipsoids: a row of nodes (fixed y, z offsets from the centre)
    is dropped when the smallest squared normalised radius over x, the Schur complement
    quadratic f11 dy^2 + 2 f12 dy dz + f22 dz^2 of M^T M, is at least (1 + (h sqrt(2) +
    1e-3)/s_min + 1e-3)^2 x 1.001. Rows near that bound, for the (6, 2, 2) shape and random
    shapes: a dropped row has no sample inside at any node along x (every sample of the
    nodes within reach checked with the predicate), and most rows near the shadow's rim are
    dropped where the bounding circle would keep them."""
    g = np.random.default_rng(15)
    n = 10
    so = [float(v) for v in _so(n)]
    h = (n - 1) / (2 * n)
    dropped = kept_circle = 0
    for t in range(60):
        semi = np.array([6.0, 2.0, 2.0]) if t % 2 else g.uniform(0.8, 6.0, 3)
        mm = _ellipsoid_rows(g, semi)
        M = np.array([[float(mm[3 * a + c]) for c in range(3)] for a in range(3)])
        Q = M.T @ M
        f11 = Q[1, 1] - Q[0, 1] ** 2 / Q[0, 0]
        f12 = Q[1, 2] - Q[0, 1] * Q[0, 2] / Q[0, 0]
        f22 = Q[2, 2] - Q[0, 2] ** 2 / Q[0, 0]
        grow = 1.0 + (h * np.sqrt(2.0) + 1e-3) / semi.min() + 1e-3
        bound = grow * grow * 1.001
        reach = semi.max() + 0.8661 + 1e-3
        for _ in range(40):
            ang = g.uniform(0, 2 * np.pi)
            # a row offset near the grown shadow's rim in a random direction
            e = np.array([np.cos(ang), np.sin(ang)])
            F1 = f11 * e[0] ** 2 + 2 * f12 * e[0] * e[1] + f22 * e[1] ** 2
            rho = np.sqrt(bound / F1) * g.uniform(0.9, 1.3)
            dy, dz = rho * e
            F = f11 * dy * dy + 2 * f12 * dy * dz + f22 * dz * dz
            if F < bound:
                continue
            dropped += 1
            kept_circle += dy * dy + dz * dz < reach * reach
            # every node along x within reach: no sample inside (the predicate on arrays,
            # same FP32 operations in the same order)
            px = (np.arange(-int(reach) - 1, int(reach) + 2) + g.uniform(-0.5, 0.5)).astype(np.float32)
            sx = (px[:, None] + np.asarray(so, np.float32)[None, :]).reshape(-1, 1, 1)
            sy = (f32(dy) + np.asarray(so, np.float32)).reshape(1, -1, 1)
            sz = (f32(dz) + np.asarray(so, np.float32)).reshape(1, 1, -1)
            m32 = [f32(v) for v in mm]
            q = [(m32[3 * a] * sx + m32[3 * a + 1] * sy) + m32[3 * a + 2] * sz for a in range(3)]
            r2 = (q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]
            assert r2.dtype == np.float32 and not (r2 < f32(1)).any(), (t, dy, dz)
    assert dropped > 500 and kept_circle > 0.5 * dropped, (dropped, kept_circle)
