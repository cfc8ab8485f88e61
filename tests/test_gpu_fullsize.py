"""Parity at the full size of the main benchmark, in the launch configuration the benchmark
times: the 256^3 Couette suspension (4000 spheres R 6, FP32, n_sub 10, graph replay), one
coupled step from its initial state. The oracle cannot step 16.7 M cells in a test, so it
checks sampled outputs one by one:

- sampled nodes (fluid and solid): the oracle voxelises each node itself (its two largest
  solid fractions among all 4000 spheres, at the positions the PSM stage used) and the
  kernel's solids there must be the same; the stored post-collision populations are
  checked against the oracle's collision of the node (Eqs. psm1, lbePS) from the
  pre-collision populations read before the step, with the oracle's solids;
- sampled particles: the hydrodynamic force and torque against the oracle's sum of the
  node forces (Eqs. forceSF, torqueSF) over every node where the oracle finds the
  particle among the node's solids;
- every node: its collision conserves mass;
- after 40 coupled steps (contacts active): the DEM part from the state read back there,
  stepped by the kernel and by the oracle from identical positions, velocities and
  orientations: contact forces and torques, velocities and the contact sets.

In the first step after the particles are set, no sphere touches another (placement gap
0.1, relative speeds below 0.005 per step) and no force acts during the DEM substeps, so
the PSM stage sees each particle at its initial velocity and at the position read back
after the step (the final velocity update does not move particles).
"""
import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W

from _helpers import gpu_from_workload, normwise, oracle_from_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_solids_sim(oracle, w, pos):
    o = oracle.Sim(w.nx, w.ny, w.nz, periodic=w.periodic, u_wall=w.u_wall,
                   params=oracle.default_params(tau=w.params["tau"], voxel=0),
                   max_particles=w.n)
    o.set_particles(w.shape, w.radius, w.semi, w.density, pos, w.vel, w.omg, w.triad)
    return o


@pytest.fixture(scope="module")
def full_step():
    import torch
    from paper_2512_04997_gb300 import ledds
    w = W.couette_suspension()          # the main benchmark workload
    s = ledds.from_workload(w)
    f_pre = s.populations(0)            # pre-collision populations of the first step
    s.step(1)
    f_post = s.populations(1)           # post-collision populations it stored
    pos, _, _, _ = s.particles()
    Fh, Mh, Fc, _ = s.forces()
    beta, ids, nsol = s.voxelize()
    st = s.status()
    out = dict(w=w, f_pre=f_pre, f_post=f_post, pos=pos, Fh=Fh, Mh=Mh, Fc=Fc, beta=beta, ids=ids,
               nsol=nsol, status=st)
    yield out
    s.close()
    del s
    torch.cuda.empty_cache()


def _arm(w, x, y, z, p):
    """Node minus centre, minimum image on the periodic axes."""
    d = np.array([x, y, z], dtype=np.float64) - p
    L = (w.nx, w.ny, w.nz)
    for a in range(3):
        if w.periodic[a]:
            d[a] -= L[a] * round(d[a] / L[a])
    return d


def _node_collide(oracle, w, pos, fpre, beta, ids, cell):
    """Oracle collision of one node with the given solids there (centres `pos`, the
    initial velocities); returns f*, node forces [ns, 3] and torques, and the solid ids."""
    nx, ny = w.nx, w.ny
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    B, uk, arm, kk = [], [], [], []
    for m in range(2):
        b, k = float(beta[m]), int(ids[m])
        if k < 0 or not b > 0.0:
            continue
        B.append(oracle.bk(b, w.params["tau"]))
        a = _arm(w, x, y, z, pos[k])
        # first step: omega = 0, velocity = initial
        uk.append(w.vel[k] + np.cross(w.omg[k], a))
        arm.append(a)
        kk.append(k)
    fstar, Fk, Mk = oracle.cell_collide(fpre, w.params["tau"], B, uk, arm, force=w.params["fluid_force"])
    return fstar, Fk, Mk, kk


def _xyz(w, c):
    return c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)


def test_status_and_no_contacts(full_step):
    st = full_step["status"]
    assert st["rc"] == 0 and st["tile_overflow"] == 0 and st["cand_overflow"] == 0, st
    assert np.abs(full_step["Fc"]).max() == 0.0      # no sphere touched another in the step
    assert st["solids_overflow"] == 0


def test_sampled_nodes_post_collision(oracle, full_step):
    import torch
    w, pos = full_step["w"], full_step["pos"]
    N = w.ncell
    o = _oracle_solids_sim(oracle, w, pos)
    g = np.random.default_rng(2024)
    nsol = full_step["nsol"]
    solid_cells = (nsol > 0).nonzero().flatten()
    dev = full_step["f_pre"].device
    fluid = g.integers(0, N, 1500)
    pick = torch.as_tensor(g.integers(0, solid_cells.numel(), 1500), device=dev)
    solid = solid_cells[pick].cpu().numpy()
    cells = np.concatenate([fluid, solid])
    ci = torch.as_tensor(cells, device=dev)
    fpre = full_step["f_pre"][:, ci].cpu().numpy().astype(np.float64)
    fpost = full_step["f_post"][:, ci].cpu().numpy().astype(np.float64)
    beta_k = full_step["beta"][ci].cpu().numpy()
    ids_k = full_step["ids"][ci].cpu().numpy()
    nsol_k = nsol[ci].cpu().numpy()
    err = 0.0
    nsolid_seen = 0
    for j, c in enumerate(cells):
        ids_o, beta_o, tot_o = o.solids_at(*_xyz(w, int(c)))
        # the kernel found the same solids (distance fractions: FP32 against FP64)
        assert tot_o == nsol_k[j], (c, tot_o, nsol_k[j])
        assert np.array_equal(ids_o, ids_k[j]), (c, ids_o, ids_k[j])
        assert np.abs(beta_o - beta_k[j]).max() < 2e-5, (c, beta_o, beta_k[j])
        fstar, _, _, kk = _node_collide(oracle, w, pos, fpre[:, j], beta_o, ids_o, int(c))
        nsolid_seen += len(kk) > 0
        err = max(err, np.abs(fstar - fpost[:, j]).max())
    assert nsolid_seen >= 1500
    # FP32 collision of FP32 inputs against FP64 (and FP32 against FP64 solid fractions):
    # a few units in the last place of values <= 0.4
    assert err < 5e-7, err


def test_sampled_particles_hydrodynamic_force(oracle, full_step):
    w, pos = full_step["w"], full_step["pos"]
    f_pre = full_step["f_pre"]
    o = _oracle_solids_sim(oracle, w, pos)
    g = np.random.default_rng(77)
    ks = g.choice(w.n, 12, replace=False)
    Fh, Mh = full_step["Fh"], full_step["Mh"]
    import torch
    for k in ks:
        # every node where the oracle finds particle k among the node's solids: its
        # bounding box (one lattice unit of margin), periodic images on x and y
        r = pos[k]
        e = w.radius[k] + 1.0
        box = [np.arange(int(np.ceil(r[a] - e)), int(np.floor(r[a] + e)) + 1) for a in range(3)]
        cells, betas, idss = [], [], []
        for zz in box[2]:
            if zz < 0 or zz >= w.nz:
                continue
            for yy in box[1]:
                for xx in box[0]:
                    x, y = xx % w.nx, yy % w.ny
                    ids_o, beta_o, _ = o.solids_at(x, y, zz)
                    if int(k) in ids_o:
                        cells.append(x + w.nx * (y + w.ny * zz))
                        betas.append(beta_o)
                        idss.append(ids_o)
        assert len(cells) > 500          # a sphere of radius 6 covers ~900 nodes
        ci = torch.as_tensor(np.array(cells), device=f_pre.device)
        fpre = f_pre[:, ci].cpu().numpy().astype(np.float64)
        F, M = np.zeros(3), np.zeros(3)
        Fabs, Mabs = np.zeros(3), np.zeros(3)
        for j, c in enumerate(cells):
            _, Fk, Mk, kk = _node_collide(oracle, w, pos, fpre[:, j], betas[j], idss[j], int(c))
            m = kk.index(int(k))
            F += Fk[m]
            M += Mk[m]
            Fabs += np.abs(Fk[m])
            Mabs += np.abs(Mk[m])
        # In the shear flow the node forces of a particle cancel to about 1e-3 of their
        # absolute sum, so the bound is relative to that sum (the condition of the sum):
        # FP32 moments and node forces (unit roundoff 6e-8) over ~900 nodes stay within
        # 2e-5 of it; a wrong or missing node term is of the order of the sum itself.
        assert np.all(np.abs(Fh[k] - F) <= 2e-5 * Fabs + 1e-12), (k, Fh[k], F, Fabs)
        assert np.all(np.abs(Mh[k] - M) <= 2e-5 * Mabs + 1e-12), (k, Mh[k], M, Mabs)


def test_mass_conserved_per_node(full_step):
    """Every node's collision (fluid or solid) conserves its mass: sum_i f*_i = sum_i f_i."""
    d = (full_step["f_post"].double().sum(0) - full_step["f_pre"].double().sum(0)).abs().max().item()
    assert d < 2e-6, d


def test_dem_from_state_after_40_steps(oracle):
    """The main workload after 40 coupled steps: its particle state (positions, velocities,
    angular velocities, orientations) is read back and the DEM part is stepped from it by
    the kernel and by the oracle (no fluid: the box's walls at the lattice's halfway planes
    with their velocities, tangential histories starting at zero on both sides), with
    random velocities added so that many spheres touch, two fluid steps of 10 substeps.
    Contact sets are identical; the kernel's FP32 contact arithmetic keeps forces and
    velocities within 1e-5 of the oracle's."""
    import torch
    from paper_2512_04997_gb300 import ledds
    w = W.couette_suspension()
    s = ledds.from_workload(w)
    s.step(40)
    pos, vel, omg, tri = s.particles()
    assert s.status()["rc"] == 0
    s.close()
    del s
    torch.cuda.empty_cache()
    d = W.Workload(name="dem", box_lo=(-0.5, -0.5, -0.5), box_hi=(w.nx - 0.5, w.ny - 0.5, w.nz - 0.5),
                   periodic=w.periodic)
    d.u_wall = w.u_wall.copy()
    d.params = dict(w.params)
    d.shape, d.radius, d.semi, d.density = w.shape, w.radius, w.semi, w.density
    # the suspension's lubricated spheres rarely touch in a few steps: random velocities
    # of 0.05 per step (a gap of 0.1 closes in two) bring many into contact
    d.pos, d.vel, d.omg, d.triad = pos, vel + W.rng(41).normal(0.0, 0.05, vel.shape), omg, tri
    o = oracle_from_workload(oracle, d)
    g = gpu_from_workload(d)
    o.step(2)
    g.step(2)
    pairs_o, pairs_g = o.contacts(), g.pairs()
    assert len(pairs_o) > 20, len(pairs_o)      # contacts are active
    assert np.array_equal(pairs_g, pairs_o)
    _, _, Fc_o, Mc_o = o.forces()
    _, _, Fc_g, Mc_g = g.forces()
    assert normwise(Fc_g, Fc_o) < 1e-5 and normwise(Mc_g, Mc_o) < 1e-5
    po, vo, wo, _ = o.particles()
    pg, vg, wg, _ = g.particles()
    assert normwise(vg, vo) < 1e-5 and normwise(wg, wo) < 1e-5
    assert np.abs(pg - po).max() < 1e-6
