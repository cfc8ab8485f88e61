"""Pins of the oracle's PSM coupling and solid fractions (Sec. 2.4).

Each test checks a fact the method fixes independently of how the oracle codes it:
limits of Eq. (lbePS), conservation of mass and of momentum between fluid and solid,
exact sample counts in special geometries, solid volumes, Stokes drag, and the sign of
the hydrodynamic torque on a rotating sphere.
"""
import math

import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W


def _random_cell(g, oracle):
    rho = 1.0 + 0.02 * g.uniform(-1, 1)
    u = 0.05 * g.uniform(-1, 1, 3)
    return oracle.equilibrium(rho, u) + 1e-3 * g.uniform(-1, 1, 19)


@pytest.mark.parametrize("collision", [0, 1])
def test_psm_zero_weight_is_bgk(oracle, collision):
    """B = 0: the PSM operator reverts to the plain collision (Sec. 2.4), BGK or TRT."""
    g = W.rng(200)
    f = _random_cell(g, oracle)
    plain, _, _ = oracle.cell_collide(f, 0.8, collision=collision)
    blended, F, M = oracle.cell_collide(f, 0.8, B=[0.0], uk=[[0.01, 0.02, 0.0]], arm=[[1, 0, 0]],
                                        collision=collision)
    assert np.array_equal(plain, blended)
    assert np.all(F == 0) and np.all(M == 0)


@pytest.mark.parametrize("collision", [0, 1])
def test_psm_full_solid_limit(oracle, collision):
    """B = 1: f*_i = f_ibar - f^eq_ibar(rho,u) + f^eq_i(rho,u_k), whatever tau is and
    whichever fluid collision (BGK or TRT: its weight 1 - B_tot vanishes)."""
    g = W.rng(201)
    f = _random_cell(g, oracle)
    c, _, opp = oracle.lattice_tables()
    rho = f.sum()
    u = (f @ c) / rho
    uk = np.array([0.02, -0.01, 0.03])
    expect = f[opp] - oracle.equilibrium(rho, u)[opp] + oracle.equilibrium(rho, uk)
    for tau in (0.6, 0.8, 1.5):
        got, _, _ = oracle.cell_collide(f, tau, B=[1.0], uk=[uk], arm=[[0, 0, 0]], collision=collision)
        assert np.allclose(got, expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("collision", [0, 1])
def test_psm_conserves_mass_and_momentum(oracle, collision):
    """Sum f* = sum f, and the momentum the fluid gains is exactly minus the force on the
    solids of Eq. (forceSF) (action-reaction between fluid and particles), BGK or TRT."""
    g = W.rng(202)
    c, _, _ = oracle.lattice_tables()
    for _ in range(20):
        f = _random_cell(g, oracle)
        B = g.uniform(0, 1, 2)
        uk = 0.05 * g.uniform(-1, 1, (2, 3))
        arm = g.uniform(-3, 3, (2, 3))
        fs, F, M = oracle.cell_collide(f, g.uniform(0.55, 1.5), B=B, uk=uk, arm=arm, collision=collision)
        assert abs(fs.sum() - f.sum()) < 1e-15
        dp = (fs - f) @ c
        assert np.allclose(dp + F.sum(0), 0.0, atol=1e-16)
        # torque is the arm times each solid's force
        for k in range(2):
            assert np.allclose(M[k], np.cross(arm[k], F[k]), atol=1e-16)


def test_subdivision_plane_and_extremes(oracle):
    """Subdivision (n = 10): a node on the surface of a huge sphere sees half of its
    samples inside (the surface is a plane at that scale); a node deep inside sees all,
    a node far outside none; the count is symmetric under rel -> -rel."""
    R = 1.0e4
    assert oracle.subdiv_count([-R, 0.0, 0.0], 0, R) == 500
    assert oracle.subdiv_count([0.0, R, 0.0], 0, R) == 500
    assert oracle.subdiv_count([0.3, 0.2, -0.1], 0, 4.0) == 1000
    assert oracle.subdiv_count([7.0, 0.0, 0.0], 0, 4.0) == 0
    g = W.rng(203)
    for _ in range(50):
        rel = g.uniform(-5, 5, 3)
        assert oracle.subdiv_count(rel, 0, 4.0) == oracle.subdiv_count(-rel, 0, 4.0)


def test_distance_method_values(oracle):
    """Eq. (naiveSolidFrac): beta = 1/2 at a node on the surface, 1 at depth >= R_c,
    0 beyond R_c outside, linear in between."""
    Rc = (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    R = 5.0
    assert oracle.beta_distance([R, 0, 0], R) == pytest.approx(0.5, abs=1e-15)
    assert oracle.beta_distance([R - Rc - 1e-9, 0, 0], R) == 1.0
    assert oracle.beta_distance([R + Rc + 1e-9, 0, 0], R) == 0.0
    assert oracle.beta_distance([0, R - Rc / 2, 0], R) == pytest.approx(0.75, abs=1e-14)


@pytest.mark.parametrize("method,R,tol", [(1, 4.0, 2e-3), (1, 6.0, 1e-3), (0, 4.0, 3e-2),
                                          (0, 6.0, 1.5e-2)])
def test_sphere_volume(oracle, method, R, tol):
    """Summed solid fractions approach the sphere volume 4/3 pi R^3."""
    n = int(2 * R + 6)
    s = oracle.Sim(n, n, n, periodic=(1, 1, 1), params=oracle.default_params(voxel=method))
    c = n / 2 - 0.5
    s.set_particles([0], [R], [[R, R, R]], [1.0], [[c + 0.23, c - 0.11, c + 0.07]])
    beta, ids, ns = s.voxelize()
    assert abs(beta[:, 0].sum() / (4.0 / 3.0 * math.pi * R ** 3) - 1.0) < tol
    assert np.all((beta >= 0) & (beta <= 1))


def test_ellipsoid_volume_any_orientation(oracle):
    """Subdivision of a rotated prolate ellipsoid (6,2,2): volume 4/3 pi a b c."""
    g = W.rng(204)
    tri = W.quaternion_to_triad(W.random_quaternions(g, 3))
    n = 20
    for k in range(3):
        s = oracle.Sim(n, n, n, periodic=(1, 1, 1), params=oracle.default_params(voxel=1))
        s.set_particles([1], [6.0], [[6, 2, 2]], [1.0], [[9.6, 9.3, 9.8]], triad=tri[k:k + 1])
        beta, _, _ = s.voxelize()
        assert abs(beta[:, 0].sum() / (4.0 / 3.0 * math.pi * 24.0) - 1.0) < 3e-3


def test_two_solids_per_cell(oracle):
    """At most two solids per cell (Sec. 3.2.3); with three touching a cell the two with
    the largest solid fraction are kept and the total is reported."""
    n = 12
    s = oracle.Sim(n, n, n, periodic=(1, 1, 1), params=oracle.default_params(voxel=0),
                   max_particles=3)
    node = np.array([6.0, 6.0, 6.0])
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    R = 2.0
    dist = [R + 0.1, R - 0.2, R + 0.3]     # betas ordered: 2nd > 1st > 3rd
    pos = node - dirs * np.array(dist)[:, None]
    s.set_particles([0, 0, 0], [R] * 3, [[R] * 3] * 3, [1.0] * 3, pos)
    beta, ids, ns = s.voxelize()
    cell = 6 + n * (6 + n * 6)
    assert ns[cell] == 3
    assert list(ids[cell]) == [1, 0]
    assert beta[cell, 0] > beta[cell, 1] > 0


def test_stokes_drag_periodic_array(oracle):
    """A fixed sphere in a periodic box with the fluid driven by a body force. At steady
    state the drag equals the total force on the fluid (momentum balance), and it is
    within the low-resolution PSM effective-radius deficit of Stokes drag corrected for a
    periodic array (Hasimoto 1959: K = 1/(1 - 1.7601 c^(1/3) + c - 1.5593 c^2))."""
    N, R, tau, f = 16, 2.5, 1.0, 1e-6
    nu = (tau - 0.5) / 3
    s = oracle.Sim(N, N, N, periodic=(1, 1, 1),
                   params=oracle.default_params(tau=tau, voxel=0, fluid_force=(f, 0, 0)))
    c = N / 2 - 0.5
    s.set_particles([0], [R], [[R] * 3], [1.0], [[c, c, c]])
    for _ in range(3000):
        s.lbm_psm_step()
    Fh, _, _, _ = s.forces()
    _, u = s.moments()
    beta, _, _ = s.voxelize()
    B = beta[:, 0] * (tau - 0.5) / ((1 - beta[:, 0]) + (tau - 0.5))
    ftot = f * (1.0 - np.minimum(B, 1.0)).sum()
    assert abs(Fh[0, 0] / ftot - 1.0) < 0.01
    phi = 4.0 / 3.0 * math.pi * R ** 3 / N ** 3
    K = 1.0 / (1 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2)
    ratio = Fh[0, 0] / (6 * math.pi * nu * R * u[0].mean() * K)
    assert 0.75 < ratio < 1.05
    assert abs(Fh[0, 1]) < 1e-12 and abs(Fh[0, 2]) < 1e-12


def test_rotating_sphere_torque(oracle):
    """A sphere spinning at fixed omega feels a torque opposing the spin, of the order of
    the Stokes value 8 pi mu R^3 omega. (With the sign of u_k as printed in Sec. 2.4 the
    torque would drive the spin instead.)"""
    N, R, tau, w = 16, 2.5, 1.0, 1e-3
    nu = (tau - 0.5) / 3
    s = oracle.Sim(N, N, N, periodic=(1, 1, 1), params=oracle.default_params(tau=tau, voxel=1))
    c = N / 2 - 0.5
    s.set_particles([0], [R], [[R] * 3], [1.0], [[c, c, c]], omg=[[0, 0, w]])
    for _ in range(800):
        s.lbm_psm_step()
    _, Mh, _, _ = s.forces()
    ratio = Mh[0, 2] / (-8 * math.pi * nu * R ** 3 * w)
    assert 0.6 < ratio < 1.1
    assert abs(Mh[0, 0]) < 1e-10 * abs(Mh[0, 2]) + 1e-15


def test_coupled_step_momentum_budget(oracle):
    """The flowchart order (Sec. 3.2) couples fluid and particles through the same force:
    the collision removes F_h(n) from the fluid, while the velocity-Verlet corrector gives
    the particle (F_h(n-1) + F_h(n))/2. In a periodic box without walls or gravity the sum
    p_fluid + p_particles + F_h(last)/2 is therefore exactly conserved (contacts cancel)."""
    N = 24
    g = W.rng(205)
    p = oracle.default_params(tau=0.9, voxel=0, n_sub=1, rho_f=1.0, k_n=5.0, k_t=5.0 * 2 / 7,
                              dem_h=7.5)
    s = oracle.Sim(N, N, N, periodic=(1, 1, 1), params=p, max_particles=3)
    rho, u = W.random_fields(g, N, N, N, amp_u=0.01)
    s.init_equilibrium(rho, u)
    pos = np.array([[5.0, 6.0, 7.0], [12.0, 12.5, 11.0], [18.0, 5.0, 17.0]])
    vel = np.array([[0.01, -0.005, 0.002], [-0.004, 0.003, 0.0], [0.0, 0.006, -0.008]])
    s.set_particles([0, 0, 0], [3.0] * 3, [[3.0] * 3] * 3, [1.5, 1.2, 2.0], pos, vel=vel)
    c, _, _ = oracle.lattice_tables()
    m = np.array([1.5, 1.2, 2.0]) * 4.0 / 3.0 * math.pi * 27.0

    def budget():
        f = s.populations()
        pf = (f.T @ c).sum(0)
        _, v, _, _ = s.particles()
        Fh, _, _, _ = s.forces()
        return pf + (m[:, None] * v).sum(0) + 0.5 * Fh.sum(0)

    b0 = budget()
    s.step(40)
    b1 = budget()
    _, v1, _, _ = s.particles()
    assert np.abs(v1 - vel).max() > 1e-4          # the particles did exchange momentum
    assert np.allclose(b1, b0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("angle", [math.pi / 2, 0.0])
def test_jeffery_rotation_rate(oracle, angle):
    """A prolate ellipsoid (a = 6, b = 3, aspect ratio r = 2) in shear rotates about the
    vorticity axis at Jeffery's rate shear (r^2 sin^2 phi + cos^2 phi)/(r^2 + 1), phi the
    angle of the major axis from the flow direction: checked after 300 steps (the rate at the
    orientation then reached) with the major axis started along the gradient (fastest) and
    along the flow (slowest), within 8 %. The wrong sign of the solid surface velocity
    (the printed u_k = v_k - w_k x r) would reverse the torque feedback and fail this."""
    from _helpers import oracle_from_workload
    w = W.jeffery_ellipsoid(a=6.0, b=3.0, box=(32, 24, 32), angle=angle, u_wall=0.02, steps=300)
    o = oracle_from_workload(oracle, w)
    o.step(w.steps)
    _, _, omg, tri = o.particles()
    d1 = tri[0][:3]
    phi = math.atan2(d1[2], d1[0])
    shear, r = 0.04 / 32, 2.0
    jeffery = shear * (r * r * math.sin(phi) ** 2 + math.cos(phi) ** 2) / (r * r + 1.0)
    assert omg[0][1] > 0.0
    assert abs(omg[0][1] / jeffery - 1.0) < 0.08, (omg[0][1], jeffery)


@pytest.mark.parametrize("voxel,periodic", [("distance", (1, 1, 0)), ("subdiv", (1, 0, 1))])
def test_solids_at_matches_lattice_voxelisation(oracle, voxel, periodic):
    """The oracle's one-node voxelisation (used for spot checks of lattices too large to
    voxelise whole) gives, node by node, exactly the whole-lattice result: the same two
    solids, fractions and counts, with spheres and ellipsoids across periodic faces."""
    g = W.rng(5)
    n = 12
    w = W.Workload(name="t", nx=30, ny=22, nz=26, periodic=periodic)
    w.params = W.base_params(voxel=voxel, dem_h=0.0)
    w.shape = (np.arange(n) % 3 == 0).astype(np.int32)
    w.radius = g.uniform(2, 4, n)
    w.semi = np.stack([w.radius * 1.4, w.radius * 0.8, w.radius * 0.7], 1)
    w.semi[w.shape == 0] = np.stack([w.radius] * 3, 1)[w.shape == 0]
    w.density = np.ones(n)
    w.pos = g.uniform(0, 1, (n, 3)) * [30, 22, 26]
    w.vel = np.zeros((n, 3))
    w.omg = np.zeros((n, 3))
    w.triad = W.quaternion_to_triad(W.random_quaternions(g, n))
    o = oracle.from_workload(w)
    b, ids, ns = o.voxelize()
    assert (ns > 1).sum() > 25 and (ns > 0).sum() > 2000
    for c in range(w.ncell):
        x, y, z = c % 30, (c // 30) % 22, c // (30 * 22)
        i2, b2, t = o.solids_at(x, y, z)
        assert np.array_equal(i2, ids[c]) and np.array_equal(b2, b[c]) and t == ns[c], (c, i2, ids[c])
