"""The CUDA contact kernel screens ellipsoid pairs before the common-normal iteration: a
separating plane across the centre line and a Perram-Wertheim certificate. Both are exact
(a pair they reject is disjoint). The oracle decides contacts as Sec. 2.1 states the
method: bounding spheres, then the iteration alone. These tests list every pair where the
screened and the unscreened decisions differ, on random pairs and on near-tangent pairs
of the 384x384x192 ellipsoid suspension's shapes and orientations, and check that each is
a pair the iteration failed to converge on (the oracle and the kernel count those) that
the certificate proves disjoint: the screens change no decision of a converged iteration.
"""
import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W


def _plane_separated(ri, Ri, si, rj, Rj, sj):
    """Supports |diag(s) R n| of the two ellipsoids along the centre line do not reach
    across the centre distance (the kernel's test, with its 1e-12 relative margin)."""
    d = rj - ri
    dist = np.linalg.norm(d)
    n = d / dist
    h = sum(np.linalg.norm(s * (R.reshape(3, 3) @ n)) for R, s in ((Ri, si), (Rj, sj)))
    return h < dist * (1.0 - 1e-12)


def _pw_max(ri, Ri, si, rj, Rj, sj, iters=60):
    """Maximum over l of the Perram-Wertheim contact function (golden section; F is concave
    in l), in numpy: the pair overlaps iff the maximum is below 1."""
    A = [R.reshape(3, 3).T @ np.diag(np.asarray(s) ** 2) @ R.reshape(3, 3) for R, s in ((Ri, si), (Rj, sj))]
    d = rj - ri

    def F(lam):
        return lam * (1 - lam) * d @ np.linalg.solve((1 - lam) * A[0] + lam * A[1], d)

    gr = (5 ** 0.5 - 1) / 2
    lo, hi = 0.0, 1.0
    c, e = hi - gr * (hi - lo), lo + gr * (hi - lo)
    fc, fe = F(c), F(e)
    for _ in range(iters):
        if fc > fe:
            hi, e, fe = e, c, fc
            c = hi - gr * (hi - lo)
            fc = F(c)
        else:
            lo, c, fc = c, e, fe
            e = lo + gr * (hi - lo)
            fe = F(e)
    return max(fc, fe)


def _compare(oracle, pairs, max_iter=60, tol=1e-6):
    """Decisions of every pair (ri, Ri, si, rj, Rj, sj); returns the counts and the list of
    pairs where the screens change the decision, with the iteration's outcome."""
    diff, contacts, nonconv = [], 0, 0
    for k, (ri, Ri, si, rj, Rj, sj) in enumerate(pairs):
        c = oracle.ellipsoid_contact(ri, Ri, si, rj, Rj, sj, max_iter=max_iter, tol=tol)
        unscreened = c["rc"] >= 0 and c["delta"] > 0.0
        screened_out = _plane_separated(ri, Ri, si, rj, Rj, sj) or oracle.pw_separated(ri, Ri, si, rj, Rj, sj)
        contacts += unscreened
        nonconv += c["rc"] == 1
        if unscreened and screened_out:
            diff.append(dict(index=k, delta=c["delta"], rc=c["rc"], fmax=_pw_max(ri, Ri, si, rj, Rj, sj)))
    return contacts, nonconv, diff


def _check(diff):
    for d in diff:
        assert d["rc"] == 1, d          # only where the iteration did not converge
        assert d["fmax"] > 1.0, d       # and the pair is disjoint (exact criterion)


def test_screens_random_pairs(oracle):
    """300 pairs of (1.5, 0.6, 0.5) ellipsoids at centre distances 0.5-3.2, and 250 pairs of
    random semi-axes in [0.4, 2] near contact, at random orientations."""
    g = np.random.default_rng(91)
    semi = np.array([1.5, 0.6, 0.5])
    pairs = []
    for _ in range(300):
        tri = W.quaternion_to_triad(W.random_quaternions(g, 2))
        d = g.normal(size=3)
        d *= g.uniform(0.5, 3.2) / np.linalg.norm(d)
        pairs.append((np.zeros(3), tri[0], semi, d, tri[1], semi))
    g = np.random.default_rng(95)
    for _ in range(250):
        si, sj = g.uniform(0.4, 2.0, 3), g.uniform(0.4, 2.0, 3)
        tri = W.quaternion_to_triad(W.random_quaternions(g, 2))
        d = g.normal(size=3)
        d *= g.uniform(0.3, 1.2) * (si.max() + sj.max()) / np.linalg.norm(d)
        pairs.append((np.zeros(3), tri[0], si, d, tri[1], sj))
    contacts, nonconv, diff = _compare(oracle, pairs)
    print(f"random pairs: {len(pairs)}, contacts {contacts}, not converged {nonconv}, "
          f"screens change {len(diff)}: {[(d['index'], round(d['delta'], 4)) for d in diff]}")
    assert contacts > 100
    _check(diff)


@pytest.mark.slow
def test_screens_ellipsoid_suspension_near_tangency(oracle):
    """A 192x192x96 crop of the sheared ellipsoid suspension (2500 prolate (6, 2, 2)
    ellipsoids at uniformly random orientations, the workload's density). Every pair whose
    bounding spheres overlap is moved along its centre line to 1 -/+ 1e-3 and 1e-2 of the
    tangent separation (from the exact criterion) and tested as placed."""
    w = W.ellipsoid_shear(nx=192, ny=192, nz=96, n_particles=2500)
    L = np.array([192.0, 192.0, 96.0])
    d = w.pos[None, :, :] - w.pos[:, None, :]
    d[:, :, :2] -= L[:2] * np.round(d[:, :, :2] / L[:2])
    ii, jj = np.nonzero(np.triu(np.linalg.norm(d, axis=2) < 12.0, 1))
    sel = np.random.default_rng(7).permutation(len(ii))[:1500]
    rows = []
    for k in sel:
        i, j = ii[k], jj[k]
        ri, dv = w.pos[i], d[i, j]
        args = (w.triad[i], w.semi[i], w.triad[j], w.semi[j])
        # F_max(s d) = s^2 F_max(d): tangent at s* = F_max(d)^(-1/2)
        s_star = 1.0 / np.sqrt(_pw_max(ri, args[0], args[1], ri + dv, args[2], args[3]))
        for eps in (None, -1e-2, -1e-3, 1e-3, 1e-2):
            rj = ri + dv * (1.0 if eps is None else s_star * (1.0 + eps))
            rows.append((ri, args[0], args[1], rj, args[2], args[3]))
    contacts, nonconv, diff = _compare(oracle, rows)
    print(f"suspension pairs: {len(rows)}, contacts {contacts}, not converged {nonconv}, "
          f"screens change {len(diff)}, largest iteration overlap among them "
          f"{max([x['delta'] for x in diff], default=0.0):.3f}")
    assert len(sel) == 1500 and contacts > 2500
    _check(diff)
    assert len(diff) < 0.01 * len(rows)
