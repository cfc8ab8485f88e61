"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle on seeded inputs.

Tolerances (stated per test): FP32 storage <= 1e-5 normwise on fields and trajectories;
integer work (cell keys, sorted ids, contact pairs, subdivision counts) bit-exact.
Sizes span several 32x8x4 tiles with ragged tails in x, y and z.
"""
import math

import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W

from _helpers import gpu_from_workload, normwise, oracle_from_workload, random_populations

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lattice_workload(nx, ny, nz, periodic, tau=0.8, **kw):
    w = W.Workload(name="lattice", nx=nx, ny=ny, nz=nz, periodic=periodic)
    w.params = W.base_params(tau=tau, **kw)
    return w


# ------------------------------------------------------------------------------------
# lattice only
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("collision", ["bgk", "trt"])
@pytest.mark.parametrize("periodic,walls", [((1, 1, 1), None), ((1, 1, 0), "z"), ((0, 0, 0), "all")])
def test_lattice_populations_and_fields(oracle, periodic, walls, collision):
    """Pull streaming, periodic wrap, halfway and moving-wall bounce-back (edges and
    corners included) and the BGK or TRT collision, on off-equilibrium random populations."""
    nx, ny, nz = 37, 19, 11     # 2 tiles in x, 3 in y, 3 in z, all ragged
    g = W.rng(500)
    f0 = random_populations(oracle, g, nx, ny, nz)
    w = lattice_workload(nx, ny, nz, periodic, tau=0.7, collision=collision)
    if walls == "z":
        w.u_wall[2, 0] = [-0.03, 0.01, 0.0]
        w.u_wall[2, 1] = [0.04, 0.0, 0.0]
    elif walls == "all":
        w.u_wall[0, 1] = [0.0, 0.02, -0.01]
        w.u_wall[1, 0] = [0.01, 0.0, 0.015]
        w.u_wall[2, 1] = [0.05, -0.02, 0.0]
    o = oracle_from_workload(oracle, w, populations=f0)
    s = gpu_from_workload(w, populations=f0)
    # the first pull returns exactly the populations that were set
    assert normwise(s.populations().cpu().numpy(), f0) < 1e-7
    o.step(40)
    s.step(40)
    fo = o.populations()
    fg = s.populations().cpu().numpy()
    err_f = np.abs(fg - fo).max()
    rho_o, u_o = o.moments()
    rho_g, u_g = (x.cpu().numpy() for x in s.fields())
    err_u = normwise(u_g, u_o)
    # rho is read out in FP32 around 1 (resolution 6e-8); the populations above carry
    # the strict check of mass transport
    err_rho = np.abs(rho_g - rho_o).max()
    assert err_f < 2e-7, err_f
    assert err_u < FP32_TOL, err_u
    assert err_rho < 1e-6, err_rho


@pytest.mark.parametrize("collision,tau", [("bgk", 0.5 + math.sqrt(3) / 4), ("trt", 0.8), ("trt", 1.4)])
def test_guo_forcing_channel(oracle, collision, tau):
    """Body-force-driven channel (Guo forcing) between no-slip walls, BGK at its exact tau
    and TRT at any tau; after the flow has developed, also against the exact parabola."""
    H, F = 12, 1e-5
    w = lattice_workload(3, 5, H, (1, 1, 0), tau=tau, fluid_force=(F, 0, 0), collision=collision)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(300)
    s.step(300)
    _, u_o = o.moments()
    _, u_g = s.fields()
    assert normwise(u_g.cpu().numpy(), u_o) < FP32_TOL
    nu = (tau - 0.5) / 3.0
    s.step(int(40 * H * H / nu))
    _, u_g = s.fields()
    z = np.arange(H) + 0.5
    ex = F / (2 * nu) * z * (H - z)
    ux = u_g[0].cpu().numpy().reshape(H, 5, 3)
    assert np.abs(ux - ex[:, None, None]).max() / ex.max() < 1e-4   # FP32 steady state


def test_graph_and_eager_paths_agree(oracle):
    """Graph replay (1- and 2-step graphs, both parities) equals eager profiled launches."""
    nx, ny, nz = 33, 9, 6
    g = W.rng(501)
    f0 = random_populations(oracle, g, nx, ny, nz)
    w = lattice_workload(nx, ny, nz, (1, 0, 1), tau=0.9)
    w.u_wall[1, 1] = [0.02, 0, 0]
    a = gpu_from_workload(w, populations=f0)
    b = gpu_from_workload(w, populations=f0)
    a.step(1)
    a.step(4)
    a.step(3)
    b.set_profiling(True)
    b.step(8)
    assert np.array_equal(a.populations().cpu().numpy(), b.populations().cpu().numpy())


# ------------------------------------------------------------------------------------
# solid fractions
# ------------------------------------------------------------------------------------
def _particles_workload(nx, ny, nz, periodic, voxel, seed, shapes, radius=3.2, clear=False,
                        semi=(4.5, 2.0, 1.6)):
    g = W.rng(seed)
    w = lattice_workload(nx, ny, nz, periodic, voxel=voxel, dem_h=2 * max(max(semi), radius) + 0.5)
    n = len(shapes)
    w.shape = np.array(shapes, dtype=np.int32)
    w.semi = np.where(w.shape[:, None] == 1, np.array(semi, dtype=float), radius)
    w.radius = np.where(w.shape == 1, max(semi), radius)
    w.density = np.full(n, 1.3)
    if clear:
        # non-overlapping, one lattice unit away from the walls
        lo = [-0.5 if periodic[a] else 0.5 for a in range(3)]
        hi = [(nx, ny, nz)[a] - 0.5 - (0 if periodic[a] else 1.0) for a in range(3)]
        w.pos = W.rsa_spheres(g, n, w.radius.astype(float), lo, hi, periodic, gap=0.3)
    else:
        w.pos = g.random((n, 3)) * (np.array([nx, ny, nz]) - 1.0)
    w.vel = g.normal(0, 0.01, (n, 3))
    w.omg = g.normal(0, 0.002, (n, 3))
    w.triad = W.quaternion_to_triad(W.random_quaternions(g, n))
    return w


@pytest.mark.parametrize("voxel,semi", [("subdiv", (4.5, 2.0, 1.6)), ("subdiv", (6.0, 2.0, 2.0)),
                                        ("distance", None)])
def test_voxelize_parity(oracle, voxel, semi):
    """Top-two solid fractions per node. Subdivision counts are bit-exact (both sides use
    the same FP32 predicate); distance fractions agree to FP32 rounding. The ellipsoids
    take semi-axes (4.5, 2, 1.6) and the sheared suspension's (6, 2, 2), at random
    orientations and positions (some across the periodic faces)."""
    shapes = [0] * 10 + ([1] * 6 if voxel == "subdiv" else [])
    if semi == (6.0, 2.0, 2.0):
        w = _particles_workload(54, 40, 26, (1, 1, 0), voxel, 503, shapes, semi=semi)
    else:
        w = _particles_workload(45, 30, 21, (1, 1, 0), voxel, 502, shapes)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    b_o, id_o, ns_o = o.voxelize()
    b_g, id_g, ns_g = (x.cpu().numpy() for x in s.voxelize())
    assert np.array_equal(ns_g, ns_o)
    amb = ns_o > 2          # with three or more solids near-equal fractions may tie
    assert np.array_equal(id_g[~amb], id_o[~amb])
    if voxel == "subdiv":
        assert np.array_equal(np.rint(b_g * 1000).astype(int), np.rint(b_o * 1000).astype(int))
    else:
        assert np.abs(b_g - b_o).max() < 2e-5
    assert (b_o[:, 0] > 0).sum() > 1000


# ------------------------------------------------------------------------------------
# coupled steps
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("voxel,n_sub,collision", [("distance", 1, "bgk"), ("subdiv", 3, "bgk"),
                                                    ("distance", 2, "trt")])
def test_coupled_small(oracle, voxel, n_sub, collision):
    """Several spheres and ellipsoids in a sheared box: fields, forces and trajectories
    after 30 coupled steps (PSM + hydrodynamic force + DEM substeps + walls). The
    hydrodynamic force and torque of a particle are sums of node terms that largely
    cancel, so their bound is relative to the sum of the terms' magnitudes (the condition
    of the sum, as at full size): 2e-5 of it per particle; the angular velocity integrates
    such torques over the 30 steps, so its bound adds 30 dt times 2e-5 of that magnitude
    over the particle's smallest moment of inertia."""
    shapes = [0] * 5 + ([1] * 2 if voxel == "subdiv" else [])
    w = _particles_workload(40, 26, 24, (1, 1, 0), voxel, 503, shapes, radius=3.0, clear=True)
    w.params.update(n_sub=n_sub, k_n=20.0, k_t=20.0 * 2 / 7, gravity=(0, 0, -2e-5), collision=collision)
    w.u_wall[2, 1] = [0.03, 0.0, 0.0]
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(29)
    s.step(29)
    f_pre = o.populations()          # pre-collision populations of the last step
    o.step(1)
    s.step(1)
    _, u_o = o.moments()
    _, u_g = s.fields()
    assert normwise(u_g.cpu().numpy(), u_o) < FP32_TOL
    po, vo, wo, to = o.particles()
    pg, vg, wg, tg = s.particles()
    assert np.abs(pg - po).max() < 1e-6
    assert normwise(vg, vo) < FP32_TOL
    Fh_o, Mh_o, Fc_o, Mc_o = o.forces()
    Fh_g, Mh_g, Fc_g, Mc_g = s.forces()
    # magnitudes of the node terms of the last step's sums (the oracle's collision of every
    # solid node, at the positions the step used)
    beta, ids, _ = o.voxelize()
    n = w.n
    Fabs, Mabs = np.zeros((n, 3)), np.zeros((n, 3))
    tau = w.params["tau"]
    for c in np.nonzero(beta[:, 0] > 0)[0]:
        x, y, z = c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)
        B, uk, arm, kk = [], [], [], []
        for m in range(2):
            k = int(ids[c, m])
            if k < 0 or not beta[c, m] > 0:
                continue
            a = np.array([x, y, z], float) - po[k]
            a[0] -= w.nx * round(a[0] / w.nx)
            a[1] -= w.ny * round(a[1] / w.ny)
            B.append(oracle.bk(beta[c, m], tau))
            uk.append(vo[k] + np.cross(wo[k], a))
            arm.append(a)
            kk.append(k)
        _, Fk, Mk = oracle.cell_collide(f_pre[:, c], tau, B, uk, arm, force=w.params["fluid_force"],
                                        collision={"bgk": 0, "trt": 1}[collision])
        for m, k in enumerate(kk):
            Fabs[k] += np.abs(Fk[m])
            Mabs[k] += np.abs(Mk[m])
    assert np.all(np.abs(Fh_g - Fh_o) <= 2e-5 * Fabs + 1e-12), np.abs(Fh_g - Fh_o) / (Fabs + 1e-30)
    assert np.all(np.abs(Mh_g - Mh_o) <= 2e-5 * Mabs + 1e-12), np.abs(Mh_g - Mh_o) / (Mabs + 1e-30)
    m = w.density * np.where(w.shape == 1, 4.0 / 3.0 * np.pi * w.semi.prod(1), 4.0 / 3.0 * np.pi * w.radius ** 3)
    s2 = w.semi ** 2
    Imin = 0.2 * m * np.min(np.stack([s2[:, 1] + s2[:, 2], s2[:, 0] + s2[:, 2], s2[:, 0] + s2[:, 1]]), axis=0)
    wtol = 1e-5 * np.abs(wo).max() + 30 * 2e-5 * Mabs.max(1) / Imin
    assert np.all(np.abs(wg - wo).max(1) <= wtol), (np.abs(wg - wo).max(1), wtol)
    st = s.status()
    assert st["rc"] == 0 and st["skin_violation"] == 0, st


def test_settling_sphere_full_length(oracle):
    """The single-sphere settling workload (32x32x64, tau 0.8, R 4, density ratio 2.5,
    subdivision fractions) over its full 2000 steps: fields and trajectory <= 1e-5."""
    w = W.settling_sphere(steps=2000)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(w.steps)
    s.step(w.steps)
    _, u_o = o.moments()
    _, u_g = s.fields()
    err_u = normwise(u_g.cpu().numpy(), u_o)
    po, vo, _, _ = o.particles()
    pg, vg, _, _ = s.particles()
    err_v = normwise(vg, vo)
    err_z = abs(pg[0, 2] - po[0, 2]) / abs(po[0, 2] - w.pos[0, 2])
    assert vo[0, 2] < 0                      # the sphere settles
    assert err_u < FP32_TOL, err_u
    assert err_v < FP32_TOL, err_v
    assert err_z < FP32_TOL, err_z


# ------------------------------------------------------------------------------------
# DEM only
# ------------------------------------------------------------------------------------
def _granular(n=3000, box=(36.0, 36.0, 48.0), seed=2):
    w = W.granular_box(n_particles=n, box=box, seed_index=seed)
    # shake it so that contacts form quickly
    g = W.rng(600 + seed)
    w.vel = g.normal(0, 0.02, (n, 3))
    w.params.update(gravity=(0, 0, -1e-4))
    return w


# DEM tolerances per contact arithmetic: FP64 everywhere agrees with the oracle to FP64
# rounding; FP32 forces (summed in FP64, integrated in FP64) to FP32 rounding of a force,
# about 1e-7 relative, bounded here by the 1e-5 relative tolerance of FP32 results.
DEM_TOL = {0: dict(force=1e-9, pos=1e-9, vel=1e-8), 1: dict(force=1e-5, pos=1e-6, vel=1e-5)}


@pytest.mark.parametrize("fp32", [0, 1])
def test_dem_keys_and_pairs_bitexact(oracle, fp32):
    """Cell keys, the (key, id)-sorted order and the contact set are integers: bit-exact
    after the same number of steps from the same uploaded state (the contact predicate is
    FP64 in both contact-arithmetic modes)."""
    w = _granular()
    w.params["force_fp32"] = fp32
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    for steps in (1, 25):
        o.step(steps)
        s.step(steps)
        pg, _, _, _ = s.particles()
        po, _, _, _ = o.particles()
        assert np.abs(pg - po).max() < DEM_TOL[fp32]["pos"]
        kg, idg, gng = s.cell_keys()
        # the GPU keys are those of the last rebuild (start of the last step): compare
        # with the oracle keys recomputed at the positions before that step
        pairs_g = s.pairs()
        pairs_o = o.contacts()
        assert np.array_equal(pairs_g, pairs_o)
    assert len(pairs_o) > 200
    ko, ido, gno = o.cell_keys()
    assert gng == gno


def test_dem_cell_keys_at_rebuild(oracle):
    """Keys of the rebuild at the start of a step equal the oracle's keys at the same
    positions, and the sorted ids match np.lexsort."""
    w = _granular(n=2500, seed=3)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    s.step(1)   # rebuild happened at the uploaded positions
    kg, idg, gn = s.cell_keys()
    ko, ido, gno = o.cell_keys()
    assert gn == gno
    assert np.array_equal(kg, ko)
    assert np.array_equal(idg, ido)


@pytest.mark.parametrize("fp32", [0, 1])
def test_dem_forces_and_trajectories(oracle, fp32):
    """Contact forces and the trajectories of a many-body pile over 50 steps: FP64 rounding
    (1e-9) with FP64 contact arithmetic, 1e-5 relative with FP32 contact arithmetic."""
    w = _granular(n=2000, seed=4)
    w.params["force_fp32"] = fp32
    tol = DEM_TOL[fp32]
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(50)
    s.step(50)
    _, _, Fc_o, Mc_o = o.forces()
    _, _, Fc_g, Mc_g = s.forces()
    assert normwise(Fc_g, Fc_o) < tol["force"]
    assert normwise(Mc_g, Mc_o) < tol["force"]
    po, vo, wo, _ = o.particles()
    pg, vg, wg, _ = s.particles()
    assert np.abs(pg - po).max() < tol["pos"]
    assert normwise(vg, vo) < tol["vel"]
    assert np.abs(vo).max() > 1e-3             # the pile is moving


def _ellipsoid_pile(fp32, orient, screen):
    g = W.rng(604)
    n = 500
    box = (30.0, 30.0, 30.0)
    w = W.Workload(name="ell", box_lo=(0, 0, 0), box_hi=box, periodic=(1, 0, 0))
    w.params = W.base_params(law="hertz", young=5.0, poisson=0.3, restitution=0.8, friction=0.3,
                             rho_f=0.0, gravity=(0, 0, -1e-3), dem_h=2 * 1.5 + 0.3, skin=0.3,
                             force_fp32=fp32, orient=orient, ell_screen=screen)
    semi = np.array([1.5, 0.8, 0.6])
    w.shape = np.ones(n, dtype=np.int32)
    w.semi = np.tile(semi, (n, 1))
    w.radius = np.full(n, 1.5)
    w.density = np.ones(n)
    w.pos = W.rsa_spheres(g, n, np.full(n, 1.5), (0, 0, 0), box, (1, 0, 0), gap=-0.4)
    w.vel = g.normal(0, 0.02, (n, 3))
    w.omg = g.normal(0, 0.01, (n, 3))
    w.triad = W.quaternion_to_triad(W.random_quaternions(g, n))
    return w


def _pairs_of(keys):
    return {(int(k) >> 32, int(k) & 0xffffffff) for k in keys}


def test_dem_ellipsoid_screens_from_identical_state(oracle):
    """The kernel's default decision (exact disjointness screens, then the iteration)
    against the oracle's (the iteration alone, Sec. 2.1) at identical states: snapshots of
    a GPU run of a dense ellipsoid pile, uploaded into the oracle. Every pair the oracle
    finds and the kernel does not is one where the oracle's iteration did not converge and
    the pair is proven disjoint; the kernel finds no pair the oracle does not."""
    w = _ellipsoid_pile(0, "triad", 1)
    s = gpu_from_workload(w)
    semi = w.semi[0]
    listed = []
    common = 0
    for snap in range(4):
        s.step(20)
        pg = _pairs_of(s.pairs())
        pos, vel, omg, tri = s.particles()
        o = oracle_from_workload(oracle, w)
        o.set_particles(w.shape, w.radius, w.semi, w.density, pos, vel, omg, tri)
        o.contact_forces(1.0)
        po = _pairs_of(o.contacts())
        assert pg <= po, pg - po
        common += len(pg)
        for i, j in sorted(po - pg):
            d = pos[j] - pos[i]
            d[0] -= 30.0 * np.round(d[0] / 30.0)
            c = oracle.ellipsoid_contact(pos[i], tri[i], semi, pos[i] + d, tri[j], semi,
                                         max_iter=w.params["ell_max_iter"], tol=w.params["ell_tol"])
            assert c["rc"] == 1, (i, j, c)                       # not converged
            assert oracle.pw_separated(pos[i], tri[i], semi, pos[i] + d, tri[j], semi) or \
                _plane_separated(pos[i], tri[i], semi, pos[i] + d, tri[j], semi), (i, j)
            listed.append((snap, i, j, round(c["delta"], 4)))
    print(f"pairs in both: {common}; oracle-only (iteration not converged, proven disjoint): {listed}")
    assert common > 20


def _plane_separated(ri, Ri, si, rj, Rj, sj):
    d = rj - ri
    dist = np.linalg.norm(d)
    n = d / dist
    h = sum(np.linalg.norm(sv * (np.reshape(R, (3, 3)) @ n)) for R, sv in ((Ri, si), (Rj, sj)))
    return h < dist * (1.0 - 1e-12)


@pytest.mark.parametrize("fp32,orient", [(0, "triad"), (1, "triad"), (0, "quat"), (1, "quat")])
def test_dem_ellipsoids_hertz(oracle, fp32, orient):
    """Ellipsoid contacts (common-normal iteration, FP64 in both modes) with the Hertz law
    and walls; orientations integrated by the triad update or by the quaternion option. The
    kernel's screens are off (ell_screen 0), so both sides decide contacts by the iteration
    alone and follow the same trajectory."""
    w = _ellipsoid_pile(fp32, orient, 0)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(80)
    s.step(80)
    pairs_o = o.contacts()
    pairs_g = s.pairs()
    assert len(pairs_o) > 5
    assert np.array_equal(pairs_g, pairs_o)
    _, _, Fc_o, Mc_o = o.forces()
    _, _, Fc_g, Mc_g = s.forces()
    assert np.abs(Fc_o).max() > 0
    ftol = 1e-8 if fp32 == 0 else 1e-5
    assert normwise(Fc_g, Fc_o) < ftol
    assert normwise(Mc_g, Mc_o) < ftol
    po, vo, wo, to = o.particles()
    pg, vg, wg, tg = s.particles()
    assert np.abs(vo).max() < 0.2          # a well-conditioned run
    # FP32 contact arithmetic: 1e-5 of the largest semi-axis (1.5) after 80 steps
    assert np.abs(pg - po).max() < (1e-8 if fp32 == 0 else 1.5e-5)
    assert np.abs(tg - to).max() < (1e-8 if fp32 == 0 else 1e-4)
    assert np.abs(wo).max() > 1e-3         # the orientations do change


def test_quaternion_free_rotation_exact():
    """Quaternion orientation option on the GPU, a property that holds at any size: 3000
    torque-free spheres, far apart, each spinning at its own w from its own orientation,
    turn by exactly |w| t about w (Rodrigues), to FP64 rounding, after 300 steps."""
    g = W.rng(613)
    n = 3000
    box = (400.0, 400.0, 400.0)
    w = W.Workload(name="spin", box_lo=(0, 0, 0), box_hi=box, periodic=(1, 1, 1))
    w.params = W.base_params(rho_f=0.0, dem_h=2.5, skin=0.3, orient="quat", n_sub=2)
    w.shape = np.zeros(n, dtype=np.int32)
    w.radius = np.ones(n)
    w.semi = np.ones((n, 3))
    w.density = np.ones(n)
    w.pos = W.rsa_spheres(g, n, np.ones(n), (0, 0, 0), box, (1, 1, 1), gap=1.0)
    w.vel = np.zeros((n, 3))
    w.omg = g.normal(0, 0.02, (n, 3))
    q0 = W.random_quaternions(g, n)
    w.triad = W.quaternion_to_triad(q0)
    s = gpu_from_workload(w)
    T = 300
    s.step(T)
    _, _, omg, tri = s.particles()
    assert np.abs(omg - w.omg).max() < 1e-15   # the gyroscopic term of a sphere vanishes
    d0 = w.triad.reshape(n, 3, 3)
    err = 0.0
    for k in range(n):
        wk = w.omg[k]
        ang = np.linalg.norm(wk) * T
        kx = wk / np.linalg.norm(wk)
        K = np.array([[0, -kx[2], kx[1]], [kx[2], 0, -kx[0]], [-kx[1], kx[0], 0]])
        Rw = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
        err = max(err, np.abs(tri[k].reshape(3, 3) - d0[k] @ Rw.T).max())
    assert err < 1e-12


def test_fluidised_bed_small(oracle):
    """The fluidised-bed workload shape (periodic x and z, walls on y, gravity along -y on
    particles of density ratio 1.1, distance fractions, 10 DEM substeps, tau for Re = 1)
    scaled to 66 x 48 x 66 with spheres of diameter 10 at solid fraction 0.3, 20 coupled
    steps: fields, trajectories and hydrodynamic forces at the parity tolerances."""
    w = W.fluidised_bed(0.3, nx=66, ny=48, nz=66, diameter=10.0)
    assert w.n > 40
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(20)
    s.step(20)
    _, u_o = o.moments()
    _, u_g = s.fields()
    assert normwise(u_g.cpu().numpy(), u_o) < FP32_TOL
    po, vo, _, _ = o.particles()
    pg, vg, _, _ = s.particles()
    assert np.abs(pg - po).max() < 1e-6
    assert normwise(vg, vo) < FP32_TOL
    assert normwise(s.forces()[0], o.forces()[0]) < 1e-4
    assert np.abs(vo[:, 1]).max() > 1e-7            # the spheres have started to settle (7e-7)
    st = s.status()
    assert st["rc"] == 0 and st["skin_violation"] == 0, st
