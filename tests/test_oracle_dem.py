"""Pins of the oracle's DEM part (Secs. 2.1, 2.2, 3.2.1, 3.2.2, App. A).

Brute force on small inputs for the integer work (cell keys, contact sets), closed forms
for the contact laws (linear restitution, Hertz energy, the friction Psi-law of Sec. 4.3),
conservation laws, exact free-flight and free-rotation solutions, and closed forms of
the ellipsoid contact geometry.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_dem_cases.json")))


def dem(oracle, n, params, lo=(-5, -5, -5), hi=(5, 5, 5), periodic=(1, 1, 1), u_wall=None):
    return oracle.Sim(0, 0, 0, periodic=periodic, params=params, box_lo=lo, box_hi=hi,
                      max_particles=n, u_wall=u_wall)


def _random_packing(seed, n, L, periodic):
    g = W.rng(seed)
    radii = g.uniform(0.8, 1.2, n)
    pos = g.uniform(0, L, (n, 3))
    return radii, pos


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_cell_keys_and_sort_bruteforce(oracle, periodic):
    """Cell keys floor((r - lo)/h) with h = L/floor(L/h_req), clamped, and the (key, id)
    lexicographic order (Sec. 3.2.1), checked bit for bit against numpy."""
    n, L = 500, 20.0
    radii, pos = _random_packing(300, n, L, periodic)
    p = oracle.default_params(dem_h=2.6)
    s = dem(oracle, n, p, lo=(0, 0, 0), hi=(L, L, L), periodic=periodic)
    s.set_particles([0] * n, radii, np.tile(radii[:, None], (1, 3)), np.ones(n), pos)
    keys, ids, gn = s.cell_keys()
    gn_ref = np.floor(L / 2.6).astype(int)
    h = L / gn_ref
    k = np.clip(np.floor((pos - 0.0) / h), 0, gn_ref - 1).astype(np.int64)
    ref = k[:, 0] + gn_ref * (k[:, 1] + gn_ref * k[:, 2])
    assert gn == (gn_ref,) * 3
    assert np.array_equal(keys, ref.astype(np.uint32))
    assert np.array_equal(ids, np.lexsort((np.arange(n), ref)))


def _bruteforce_contacts(pos, radii, L, periodic):
    n = len(pos)
    out = []
    for i in range(n):
        d = pos[i] - pos[i + 1:]
        for a in range(3):
            if periodic[a]:
                d[:, a] = np.where(d[:, a] > 0.5 * L, d[:, a] - L,
                                   np.where(d[:, a] < -0.5 * L, d[:, a] + L, d[:, a]))
        dist = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
        delta = (radii[i] + radii[i + 1:]) - dist
        for j in np.nonzero(delta > 0.0)[0]:
            out.append((i << 32) | (i + 1 + int(j)))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 0, 1), (1, 1, 1)])
def test_contact_set_bruteforce(oracle, periodic):
    """Sorted unique contact pairs (i < j, overlap > 0) from the grid = O(N^2) brute force."""
    n, L = 1500, 24.0
    radii, pos = _random_packing(301, n, L, periodic)
    s = dem(oracle, n, oracle.default_params(dem_h=2.4), lo=(0, 0, 0), hi=(L, L, L),
            periodic=periodic)
    s.set_particles([0] * n, radii, np.tile(radii[:, None], (1, 3)), np.ones(n), pos)
    got = s.contacts()
    ref = _bruteforce_contacts(pos, radii, L, periodic)
    assert len(ref) > 100
    assert np.array_equal(got, ref)


def _linear_pair(oracle, eps, tc_steps):
    R, rho = 1.0, 1.0
    v = 1.0 / tc_steps      # keeps the peak overlap near 0.6 % of the radius
    ms = 4.0 / 3.0 * math.pi / 2
    beta = math.log(eps) / math.sqrt(math.log(eps) ** 2 + math.pi ** 2)
    # damped contact time pi / sqrt(k/m* - (gamma/2m*)^2) = tc_steps
    kn = ms * (math.pi / tc_steps) ** 2 / (1 - beta ** 2)
    p = oracle.default_params(law=0, k_n=kn, k_t=kn * 2 / 7, restitution=eps, friction=0.0,
                              rho_f=0.0, dem_h=2.5)
    s = dem(oracle, 2, p, lo=(-100, -3, -3), hi=(100, 3, 3))
    s.set_particles([0, 0], [R, R], [[R] * 3] * 2, [rho, rho], [[-1.005, 0, 0], [1.005, 0, 0]],
                    vel=[[v, 0, 0], [-v, 0, 0]])
    s.step(int(4 * tc_steps))
    _, vel, _, _ = s.particles()
    return (vel[1, 0] - vel[0, 0]) / (2 * v)


@pytest.mark.parametrize("eps", [0.5, 0.7, 0.9])
def test_linear_restitution(oracle, eps):
    """Linear spring-dashpot with gamma = -2 beta sqrt(k m*), beta = ln e/sqrt(ln^2 e + pi^2):
    the restitution of a head-on collision is e exactly in the continuum limit; the
    velocity-Verlet error is O(dt/t_c)."""
    e100 = _linear_pair(oracle, eps, 100)
    e200 = _linear_pair(oracle, eps, 200)
    # the error depends on where the last substep falls in the contact, so it is bounded
    # by O(dt/t_c) rather than monotone in dt
    assert abs(e100 - eps) < 6e-3
    assert abs(e200 - eps) < 6e-3


def test_hertz_head_on_energy(oracle):
    """Head-on elastic collision with the parameters of Sec. 4.1 (time unit 1e-4 s): the
    total energy E_k + 8/15 Y* sqrt(R*) delta^(5/2) (Eq. enel) is conserved, momentum stays
    zero and the velocities are exactly reversed afterwards."""
    c = GOLDEN["head_on_spheres"]
    R, m, nu = c["radius_m"], c["mass_kg"], c["poisson"]
    T = c["dt_s"]
    E = c["young_pa"] * T * T
    rho = m / (4.0 / 3.0 * math.pi * R ** 3)
    p = oracle.default_params(law=1, young=E, poisson=nu, restitution=1.0, friction=0.0,
                              rho_f=0.0, dem_h=0.5)
    s = dem(oracle, 2, p)
    v = c["speed_m_s"] * T
    gap = c["gap_m"]
    s.set_particles([0, 0], [R, R], [[R] * 3] * 2, [rho, rho],
                    [[-R - gap / 2, 0, 0], [R + gap / 2, 0, 0]], vel=[[v, 0, 0], [-v, 0, 0]])
    Ys = E / (2 * (1 - nu * nu))
    E0 = m * v * v
    worst, max_overlap = 0.0, 0.0
    for _ in range(c["iterations"]):
        s.step(1)
        pos, vel, _, _ = s.particles()
        d = max(2 * R - (pos[1, 0] - pos[0, 0]), 0.0)
        max_overlap = max(max_overlap, d)
        e = 0.5 * m * (vel ** 2).sum() + 8.0 / 15.0 * Ys * math.sqrt(R / 2) * d ** 2.5
        worst = max(worst, abs(e - E0) / E0)
        assert abs(vel[:, 0].sum()) < 1e-18
    assert max_overlap > 1e-4          # a real collision happened
    assert worst < 1e-4
    assert np.allclose(vel[:, 0], [-v, v], rtol=1e-6)


@pytest.mark.parametrize("mu", [0.1, 0.3])
def test_friction_psi_law(oracle, mu):
    """Sphere hitting a wall obliquely with restitution 1 (Sec. 4.3): in the sliding
    regime Psi_in >= 5 mu the contact-point ratio obeys Psi_out = Psi_in - 7 mu; below it
    the collision partly sticks and Psi_out lies above that line."""
    law = GOLDEN["friction_wall"]
    R, rho = 0.1, 1.0
    m = rho * 4.0 / 3.0 * math.pi * R ** 3
    kn = m * (math.pi / 200.0) ** 2
    vz = -1e-4
    for psi_in in (0.5, 1.0, 2.0, 3.0):
        p = oracle.default_params(law=0, k_n=kn, k_t=kn * 2 / 7, restitution=1.0, friction=mu,
                                  rho_f=0.0, dem_h=0.5)
        s = dem(oracle, 1, p, lo=(-5, -5, 0), hi=(5, 5, 5), periodic=(1, 1, 0))
        s.set_particles([0], [R], [[R] * 3], [rho], [[0, 0, R + 1e-4]],
                        vel=[[psi_in * (-vz), 0, vz]])
        s.step(600)
        _, vel, omg, _ = s.particles()
        psi_out = -(vel[0, 0] - omg[0, 1] * R) / vz
        theory = psi_in + law["slope"] * mu
        if psi_in >= law["sliding_threshold"] * mu:
            assert abs(psi_out - theory) < 0.02 * max(1.0, abs(theory))
        else:
            assert psi_out > theory + 0.05
        assert abs(vel[0, 2] / vz + 1.0) < 1e-5


def test_momentum_conserved_many_body(oracle):
    """Periodic box, no walls, no gravity: pair forces are equal and opposite
    (Sec. 3.2.2), so total momentum is invariant."""
    g = W.rng(302)
    side, sp = 7, 2.05
    L = side * sp
    grid = (np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
            + 0.5) * sp
    n = len(grid)
    radii = g.uniform(0.8, 1.0, n)
    pos = grid + g.uniform(-0.02, 0.02, (n, 3))
    vel = g.normal(0, 0.01, (n, 3))
    p = oracle.default_params(k_n=5.0, k_t=5.0 * 2 / 7, rho_f=0.0, dem_h=2.4)
    s = dem(oracle, n, p, lo=(0, 0, 0), hi=(L, L, L), periodic=(1, 1, 1))
    s.set_particles([0] * n, radii, np.tile(radii[:, None], (1, 3)), np.ones(n), pos, vel=vel)
    m = 4.0 / 3.0 * math.pi * radii ** 3
    P0 = (m[:, None] * vel).sum(0)
    assert s.status()["ncontacts"] == 0
    s.step(50)
    _, v1, _, _ = s.particles()
    assert s.status()["ncontacts"] > 20
    assert np.allclose((m[:, None] * v1).sum(0), P0, atol=1e-14)


def test_free_fall_with_buoyancy(oracle):
    """Velocity Verlet is exact for constant acceleration: z = z0 + 1/2 g (1 - rho_f/rho_p) t^2
    (buoyancy imposed analytically, Sec. 4.6)."""
    g_ = -1e-3
    p = oracle.default_params(gravity=(0, 0, g_), rho_f=1.0, dem_h=2.5, n_sub=4)
    s = dem(oracle, 1, p, lo=(-50, -50, -50), hi=(50, 50, 50), periodic=(1, 1, 1))
    s.set_particles([0], [1.0], [[1.0] * 3], [2.5], [[0, 0, 10.0]], vel=[[0.01, 0, 0]])
    s.step(100)  # t = 100
    pos, vel, _, _ = s.particles()
    gb = g_ * (1 - 1 / 2.5)
    assert pos[0, 2] == pytest.approx(10.0 + 0.5 * gb * 100 ** 2, rel=1e-12)
    assert vel[0, 2] == pytest.approx(gb * 100, rel=1e-12)
    assert pos[0, 0] == pytest.approx(1.0, rel=1e-12)


def _rodrigues(axis, ang):
    k = np.asarray(axis, dtype=float)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_free_rotation_triad(oracle):
    """A torque-free sphere spinning at w: the triad turns by |w| t about w (Rodrigues),
    with the second-order error of the midpoint triad update."""
    errs = []
    for nsub in (1, 2):
        p = oracle.default_params(rho_f=0.0, dem_h=2.5, n_sub=nsub)
        s = dem(oracle, 1, p, lo=(-50, -50, -50), hi=(50, 50, 50))
        w = np.array([0.01, -0.02, 0.015])
        s.set_particles([0], [1.0], [[1.0] * 3], [1.0], [[0, 0, 0]], omg=[w])
        T = 100
        s.step(T)
        _, _, omg, tri = s.particles()
        Rw = _rodrigues(w, np.linalg.norm(w) * T)
        d = tri[0].reshape(3, 3)          # rows are the body axes in world components
        errs.append(np.abs(d - Rw.T).max())
        assert np.allclose(omg[0], w, atol=1e-16)
    assert errs[0] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0   # second order in dt


def test_torque_free_ellipsoid_angular_momentum(oracle):
    """Torque-free asymmetric rigid body (Euler's equations, body frame): the world-frame
    angular momentum R^T I R w and the energy are invariants. The scheme of Eq.
    (advance-omega) with the triad update at w(t) conserves them to first order in dt; a
    wrong sign of the gyroscopic term would make the momentum drift by O(1)."""
    semi = np.array([3.0, 2.0, 1.0])
    m = 4.0 / 3.0 * math.pi * semi.prod()
    I = m / 5 * np.array([semi[1] ** 2 + semi[2] ** 2, semi[0] ** 2 + semi[2] ** 2,
                          semi[0] ** 2 + semi[1] ** 2])
    drifts = []
    for nsub in (10, 20):
        p = oracle.default_params(rho_f=0.0, dem_h=7.0, n_sub=nsub)
        s = dem(oracle, 1, p, lo=(-50, -50, -50), hi=(50, 50, 50))
        w0 = np.array([0.01, 0.002, 0.012])
        s.set_particles([1], [3.0], [semi], [1.0], [[0, 0, 0]], omg=[w0])

        def invariants():
            _, _, omg, tri = s.particles()
            d = tri[0].reshape(3, 3)
            wb = d @ omg[0]
            return d.T @ (I * wb), 0.5 * (I * wb * wb).sum()

        L0, E0 = invariants()
        drift = 0.0
        for _ in range(20):
            s.step(50)
            L1, E1 = invariants()
            drift = max(drift, np.linalg.norm(L1 - L0) / np.linalg.norm(L0), abs(E1 - E0) / E0)
        drifts.append(drift)
    assert drifts[0] < 3e-3
    assert 1.7 < drifts[0] / drifts[1] < 2.3   # first order in dt


def test_ellipsoid_contact_sphere_limit(oracle):
    """a = b = c: the common-normal construction returns the sphere overlap R_i + R_j - d
    and the centre-to-centre normal."""
    g = W.rng(303)
    for _ in range(20):
        ri = g.uniform(-1, 1, 3)
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        Ri_, Rj_ = g.uniform(0.5, 1.5, 2)
        d = (Ri_ + Rj_) * g.uniform(0.9, 0.999)
        rj = ri + d * u
        tri = W.quaternion_to_triad(W.random_quaternions(g, 2))
        res = oracle.ellipsoid_contact(ri, tri[0], [Ri_] * 3, rj, tri[1], [Rj_] * 3)
        assert res["rc"] == 0
        assert res["delta"] == pytest.approx(Ri_ + Rj_ - d, abs=1e-12)
        assert np.allclose(res["en"], -u, atol=1e-12)
        assert res["rho_i"] == pytest.approx(Ri_, rel=1e-12)


def test_ellipsoid_contact_principal_axes(oracle):
    """Axis-aligned ellipsoids touching tip to tip along x: overlap a_i + a_j - d exactly,
    curvature radii b c / a at the tips (Eq. local-curvature)."""
    si, sj = np.array([3.0, 1.0, 2.0]), np.array([2.0, 1.5, 0.5])
    eye = np.eye(3).reshape(9)
    d = 4.9
    res = oracle.ellipsoid_contact([0, 0, 0], eye, si, [d, 0, 0], eye, sj)
    assert res["rc"] == 0
    assert res["delta"] == pytest.approx(si[0] + sj[0] - d, abs=1e-12)
    assert res["rho_i"] == pytest.approx(si[1] * si[2] / si[0], rel=1e-12)
    assert res["rho_j"] == pytest.approx(sj[1] * sj[2] / sj[0], rel=1e-12)
    assert np.allclose(res["en"], [-1, 0, 0], atol=1e-14)


def test_ellipsoid_separated_common_normal_bruteforce(oracle):
    """Separated convex bodies: at convergence the normals at both points are opposite and
    parallel to the connecting segment, and the gap equals the surface distance found by
    brute-force sampling of both surfaces."""
    g = W.rng(304)
    si, sj = np.array([1.5, 0.6, 0.5]), np.array([1.2, 0.5, 0.7])
    checked = 0
    for _ in range(6):
        tri = W.quaternion_to_triad(W.random_quaternions(g, 2))
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        rj = 2.4 * u
        res = oracle.ellipsoid_contact([0, 0, 0], tri[0], si, rj, tri[1], sj, max_iter=400,
                                       tol=1e-10)
        if res["rc"] != 0:
            continue
        checked += 1
        # brute-force surface distance
        th = np.linspace(0, np.pi, 181)
        ph = np.linspace(0, 2 * np.pi, 361)
        T, P = np.meshgrid(th, ph, indexing="ij")
        unit = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
        Pi = (unit * si) @ tri[0].reshape(3, 3)
        Pj = (unit * sj) @ tri[1].reshape(3, 3) + rj
        from scipy.spatial import cKDTree
        dmin = cKDTree(Pj).query(Pi)[0].min()
        assert -res["delta"] == pytest.approx(dmin, abs=0.02)
        assert res["delta"] < 0
    assert checked >= 3


def test_eccentric_ellipsoids_energy(oracle):
    """Sec. 4.2 with the paper's parameters (time unit 1e-5 s): the off-centre collision
    spins the bodies up, and the total energy changes by a small amount set by the
    curvature approximation, of the order of the paper's 0.15 % and insensitive to dt."""
    c = GOLDEN["eccentric_ellipsoids"]
    nu = GOLDEN["head_on_spheres"]["poisson"]
    m = c["mass"]
    V = 4.0 / 3.0 * math.pi * np.prod(c["semi_i"])
    rho = m / V
    out = []
    for scale in (1, 2):
        T = c["dt_s"] / scale
        E = GOLDEN["head_on_spheres"]["young_pa"] * T * T
        p = oracle.default_params(law=1, young=E, poisson=nu, restitution=1.0, friction=0.0,
                                  rho_f=0.0, dem_h=1.0)
        s = dem(oracle, 2, p)
        v = c["speed"] * T
        s.set_particles([1, 1], [0.45, 0.45], [c["semi_i"], c["semi_j"]], [rho, rho],
                        [c["pos_i"], c["pos_j"]], vel=[[v, 0, 0], [-v, 0, 0]],
                        triad=W.identity_triads(2))
        Ii = m / 5 * np.array([0.15 ** 2 + 0.15 ** 2, 0.45 ** 2 + 0.15 ** 2, 0.45 ** 2 + 0.15 ** 2])
        Ij = m / 5 * np.array([0.45 ** 2 + 0.15 ** 2, 0.15 ** 2 + 0.15 ** 2, 0.45 ** 2 + 0.15 ** 2])

        def energy():
            _, vel, omg, tri = s.particles()
            e = 0.5 * m * (vel ** 2).sum()
            for k, I in ((0, Ii), (1, Ij)):
                wb = tri[k].reshape(3, 3) @ omg[k]
                e += 0.5 * (I * wb * wb).sum()
            return e, omg

        E0, _ = energy()
        s.step(c["iterations"] * scale)
        E1, omg = energy()
        assert s.status()["ncontacts"] == 0        # separated again
        assert np.abs(omg).max() > 0.1 * v         # rotation was induced
        out.append(abs(E1 - E0) / E0)
    assert 0.3 * c["energy_change_reported"] < out[0] < 5 * c["energy_change_reported"]
    assert abs(out[1] / out[0] - 1.0) < 0.1


def test_ellipsoid_contact_decision_matches_perram_wertheim(oracle):
    """The contact decision for ellipsoid pairs (bounding spheres, then the common-normal
    iteration) agrees with the exact Perram-Wertheim
    overlap criterion on random pairs at random orientations; pairs within 2 % of
    tangency (contact function within [0.98, 1.02]) are left out."""
    g = np.random.default_rng(91)
    semi = np.array([1.5, 0.6, 0.5])
    agree = checked = contacts = 0
    for _ in range(300):
        q = W.random_quaternions(g, 2)
        tri = W.quaternion_to_triad(q)
        d = g.normal(size=3)
        d *= g.uniform(0.5, 3.2) / np.linalg.norm(d)
        pos = np.array([[5.0, 5.0, 5.0], 5.0 + d])
        # Perram-Wertheim contact function maximum by dense scan (independent of the oracle)
        R = tri.reshape(2, 3, 3)
        Ainv = [Rk.T @ np.diag(semi ** 2) @ Rk for Rk in R]
        lam = np.linspace(1e-4, 1 - 1e-4, 4001)
        Fmax = max(l * (1 - l) * d @ np.linalg.solve((1 - l) * Ainv[0] + l * Ainv[1], d) for l in lam)
        if 0.98 < Fmax < 1.02:
            continue
        p = oracle.default_params(law=oracle.LAW_HERTZ, young=10.0, rho_f=0.0, dem_h=3.2,
                                  ell_max_iter=400, ell_tol=1e-10)
        s = oracle.Sim(params=p, box_lo=(0, 0, 0), box_hi=(10, 10, 10), periodic=(1, 1, 1),
                       max_particles=2)
        s.set_particles(np.ones(2, dtype=np.int32), np.full(2, semi.max()), np.tile(semi, (2, 1)),
                        np.ones(2), pos, triad=tri)
        c = s.contacts()
        checked += 1
        contacts += len(c) > 0
        agree += (len(c) > 0) == (Fmax < 1.0)
    assert checked > 150 and contacts > 30
    assert agree == checked


def _hamilton(a, b):
    a0, av, b0, bv = a[0], np.asarray(a[1:]), b[0], np.asarray(b[1:])
    return np.concatenate([[a0 * b0 - av @ bv], a0 * bv + b0 * av + np.cross(av, bv)])


def _shoemake(g, n):
    u = g.uniform(size=(n, 3))
    return np.stack([np.sqrt(1 - u[:, 0]) * np.sin(2 * np.pi * u[:, 1]),
                     np.sqrt(1 - u[:, 0]) * np.cos(2 * np.pi * u[:, 1]),
                     np.sqrt(u[:, 0]) * np.sin(2 * np.pi * u[:, 2]),
                     np.sqrt(u[:, 0]) * np.cos(2 * np.pi * u[:, 2])], axis=1)


def test_quaternion_triad_conversions(oracle):
    """Triad of a unit quaternion = the body axes e_i turned by the sandwich product
    q (0, e_i) q*, and = Rodrigues' matrix of the quaternion's axis and angle; the
    triad-to-quaternion conversion returns +-q, including half turns (w = 0), where
    the trace branch cannot be used, and the identity."""
    g = W.rng(411)
    qs = list(_shoemake(g, 200))
    for axis in np.eye(3):
        qs.append(np.concatenate([[0.0], axis]))                          # half turns
        qs.append(np.concatenate([[1e-9], axis]) / math.hypot(1e-9, 1.0))
    qs.append(np.array([1.0, 0.0, 0.0, 0.0]))
    for q in qs:
        d = oracle.triad_from_quat(q)
        qc = np.concatenate([[q[0]], -q[1:]])
        for i in range(3):
            e = np.concatenate([[0.0], np.eye(3)[i]])
            assert np.allclose(d[i], _hamilton(_hamilton(q, e), qc)[1:], atol=1e-15)
        if abs(q[0]) < 1.0:
            ang = 2 * math.acos(max(-1.0, min(1.0, q[0])))
            assert np.allclose(d, _rodrigues(q[1:], ang).T, atol=1e-14)
        back = oracle.quat_from_triad(d.ravel())
        assert min(np.abs(back - q).max(), np.abs(back + q).max()) < 1e-14


@pytest.mark.parametrize("nsub", [1, 3])
def test_free_rotation_quaternion_exact(oracle, nsub):
    """With the quaternion orientation option a torque-free sphere spinning at w turns
    by exactly |w| t about the world axis w, whatever dt (the triad update carries an
    O(dt^2) error here), from any initial orientation: the rotation acts on the left
    (world frame), so d_i(t) = Rod(w, |w| t) d_i(0)."""
    g = W.rng(412)
    q0 = _shoemake(g, 1)[0]
    d0 = oracle.triad_from_quat(q0)
    p = oracle.default_params(rho_f=0.0, dem_h=2.5, n_sub=nsub, orient=oracle.ORIENT_QUAT)
    s = dem(oracle, 1, p, lo=(-50, -50, -50), hi=(50, 50, 50))
    w = np.array([0.01, -0.02, 0.015])
    s.set_particles([0], [1.0], [[1.0] * 3], [1.0], [[0, 0, 0]], omg=[w], triad=[d0.ravel()])
    T = 100
    s.step(T)
    _, _, omg, tri = s.particles()
    Rw = _rodrigues(w, np.linalg.norm(w) * T)
    assert np.abs(tri[0].reshape(3, 3) - d0 @ Rw.T).max() < 1e-13
    assert np.allclose(omg[0], w, atol=1e-16)


def test_quaternion_and_triad_updates_agree_to_second_order(oracle):
    """Torque-free asymmetric ellipsoid (gyroscopic term active): the quaternion and the
    triad orientation updates differ by O(dt^3) per step, so the orientations after a
    fixed time differ by O(dt^2): a quarter when dt halves."""
    semi = [3.0, 2.0, 1.0]
    diffs = []
    for nsub in (10, 20):
        tris = []
        for orient in (oracle.ORIENT_TRIAD, oracle.ORIENT_QUAT):
            p = oracle.default_params(rho_f=0.0, dem_h=7.0, n_sub=nsub, orient=orient)
            s = dem(oracle, 1, p, lo=(-50, -50, -50), hi=(50, 50, 50))
            s.set_particles([1], [3.0], [semi], [1.0], [[0, 0, 0]], omg=[[0.01, 0.002, 0.012]])
            s.step(400)
            tris.append(s.particles()[3][0])
        diffs.append(np.abs(tris[0] - tris[1]).max())
    assert 1e-9 < diffs[0] < 1e-4
    assert 3.3 < diffs[0] / diffs[1] < 4.7


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pw_certificate_spheres_closed_form(oracle, seed):
    """Two spheres: the Perram-Wertheim function peaks at D^2/(R_i + R_j)^2 (at
    l = R_i/(R_i + R_j)), so a certificate exists just beyond touching and never before."""
    g = np.random.default_rng(seed)
    for _ in range(50):
        Ri, Rj = g.uniform(0.5, 8.0, 2)
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        tri = W.quaternion_to_triad(W.random_quaternions(g, 2)).reshape(2, 9)
        for f, expect in ((1.0 + 1e-4, True), (1.0 - 1e-4, False), (0.5, False), (2.0, True)):
            rj = u * (Ri + Rj) * f
            got = oracle.pw_separated(np.zeros(3), tri[0], [Ri] * 3, rj, tri[1], [Rj] * 3)
            assert got == expect, (Ri, Rj, f)


def _ellipsoid_points(center, R, s, n, g):
    """Surface points of an ellipsoid (body axes = rows of R)."""
    v = g.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return center + (v * s) @ R


def test_pw_certificate_is_sound_bruteforce(oracle):
    """Random ellipsoid pairs near contact: whenever the certificate is given, no sampled
    surface point of either ellipsoid lies inside the other and the common-normal
    iteration finds a gap; pairs whose surfaces are found to interpenetrate by sampling
    never get a certificate. Both outcomes occur."""
    g = np.random.default_rng(95)
    sep = ovl = 0
    for _ in range(250):
        si = g.uniform(0.4, 2.0, 3)
        sj = g.uniform(0.4, 2.0, 3)
        tri = W.quaternion_to_triad(W.random_quaternions(g, 2)).reshape(2, 3, 3)
        d = g.normal(size=3)
        d *= g.uniform(0.3, 1.2) * (si.max() + sj.max()) / np.linalg.norm(d)
        ri, rj = np.zeros(3), d
        cert = oracle.pw_separated(ri, tri[0].ravel(), si, rj, tri[1].ravel(), sj)
        pi = _ellipsoid_points(ri, tri[0], si, 20000, g)
        pj = _ellipsoid_points(rj, tri[1], sj, 20000, g)
        # inside test x^T A x < 1 with A = R^T diag(1/s^2) R
        bi = ((pj - ri) @ tri[0].T) / si
        bj = ((pi - rj) @ tri[1].T) / sj
        inside = (np.einsum("ij,ij->i", bi, bi) < 1.0).any() or (np.einsum("ij,ij->i", bj, bj) < 1.0).any()
        if cert:
            sep += 1
            assert not inside
            c = oracle.ellipsoid_contact(ri, tri[0].ravel(), si, rj, tri[1].ravel(), sj, max_iter=400, tol=1e-10)
            if c["rc"] == 0:
                assert c["delta"] < 0.0
        if inside:
            ovl += 1
            assert not cert
    assert sep > 50 and ovl > 50


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_ellipsoid_wall_contact_closed_form(oracle, seed):
    """An ellipsoid pressed into the bottom wall by delta, at a random orientation: with the
    linear law the wall pushes with k_n delta along the wall normal, at the ellipsoid's
    support point towards the wall, r - E n/sqrt(n.E n) with E = R^T diag(s^2) R (here
    built as a matrix), moved half the overlap back towards the wall; the torque is that
    point's arm crossed with the force. Sliding along x adds a friction force against the
    motion, whose torque needs the contact point exactly (also the half-overlap shift)."""
    g = np.random.default_rng(seed)
    semi = g.uniform(0.6, 2.0, 3)
    R = W.quaternion_to_triad(W.random_quaternions(g, 1)).reshape(3, 3)
    E = R.T @ np.diag(semi ** 2) @ R
    n = np.array([0.0, 0.0, 1.0])               # inward normal of the bottom wall z = -5
    h = np.sqrt(n @ E @ n)
    delta = 0.05
    r = np.array([0.3, -0.2, -5.0 + h - delta])
    kn = 1000.0
    p = oracle.default_params(rho_f=0.0, dem_h=4.5, k_n=kn, k_t=kn * 2 / 7, friction=0.4)
    s = dem(oracle, 1, p, periodic=(1, 1, 0))
    s.set_particles([1], [semi.max()], [semi], [1.0], [r], triad=[R.ravel()])
    s.contact_forces(0.1)
    _, _, Fc, Mc = s.forces()
    F = kn * delta * n
    assert np.allclose(Fc[0], F, rtol=1e-12, atol=1e-12)
    pc = r - E @ n / h + 0.5 * delta * n
    assert np.allclose(Mc[0], np.cross(pc - r, F), rtol=1e-10, atol=1e-12)
    s = dem(oracle, 1, p, periodic=(1, 1, 0))
    s.set_particles([1], [semi.max()], [semi], [1.0], [r], vel=[[0.02, 0.0, 0.0]], triad=[R.ravel()])
    s.contact_forces(0.1)
    _, _, Fc, Mc = s.forces()
    assert Fc[0][2] == pytest.approx(kn * delta, rel=1e-12)
    assert Fc[0][0] < 0.0 and abs(Fc[0][0]) > 1e-4 * kn * delta      # friction against the motion
    assert np.allclose(Mc[0], np.cross(pc - r, Fc[0]), rtol=1e-10, atol=1e-12)
