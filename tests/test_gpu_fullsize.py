"""Parity at the full size of the main benchmark, in the launch configuration the benchmark
times: the 256^3 Couette suspension (4000 spheres R 6, FP32, n_sub 10, graph replay), one
coupled step from its initial state. The oracle cannot step 16.7 M cells in a test, so it
checks sampled outputs one by one:

- sampled nodes (fluid and solid): the stored post-collision populations against the
  oracle's collision of the same node (Eqs. psm1, lbePS) from the pre-collision
  populations read before the step, with the solids the kernel found there (two largest
  solid fractions, from ledds_voxelize at the positions the PSM stage used);
- sampled particles: the hydrodynamic force and torque against the oracle's sum of the
  node forces (Eqs. forceSF, torqueSF) over every node where the particle is a solid;
- every node: its collision conserves mass.

In the first step after the particles are set, no sphere touches another (placement gap
0.1, relative speeds below 0.005 per step) and no force acts during the DEM substeps, so
the PSM stage sees each particle at its initial velocity and at the position read back
after the step (the final velocity update does not move particles).
"""
import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


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
    """Oracle collision of one node with the kernel's solids there (centres `pos`, the
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


def test_status_and_no_contacts(full_step):
    st = full_step["status"]
    assert st["rc"] == 0 and st["tile_overflow"] == 0 and st["cand_overflow"] == 0, st
    assert np.abs(full_step["Fc"]).max() == 0.0      # no sphere touched another in the step
    assert st["solids_overflow"] == 0


def test_sampled_nodes_post_collision(oracle, full_step):
    import torch
    w, pos = full_step["w"], full_step["pos"]
    N = w.ncell
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
    beta = full_step["beta"][ci].cpu().numpy()
    ids = full_step["ids"][ci].cpu().numpy()
    err = 0.0
    nsolid_seen = 0
    for j, c in enumerate(cells):
        fstar, _, _, kk = _node_collide(oracle, w, pos, fpre[:, j], beta[j], ids[j], int(c))
        nsolid_seen += len(kk) > 0
        err = max(err, np.abs(fstar - fpost[:, j]).max())
    assert nsolid_seen >= 1500
    # FP32 collision of FP32 inputs against FP64: a few units in the last place of values <= 0.4
    assert err < 5e-7, err


def test_sampled_particles_hydrodynamic_force(oracle, full_step):
    w, pos = full_step["w"], full_step["pos"]
    ids_all = full_step["ids"]
    beta_all = full_step["beta"]
    f_pre = full_step["f_pre"]
    g = np.random.default_rng(77)
    ks = g.choice(w.n, 12, replace=False)
    Fh, Mh = full_step["Fh"], full_step["Mh"]
    for k in ks:
        cells = ((ids_all[:, 0] == int(k)) | (ids_all[:, 1] == int(k))).nonzero().flatten()
        assert cells.numel() > 500          # a sphere of radius 6 covers ~900 nodes
        fpre = f_pre[:, cells].cpu().numpy().astype(np.float64)
        beta = beta_all[cells].cpu().numpy()
        ids = ids_all[cells].cpu().numpy()
        F, M = np.zeros(3), np.zeros(3)
        Fabs, Mabs = np.zeros(3), np.zeros(3)
        for j, c in enumerate(cells.cpu().numpy()):
            _, Fk, Mk, kk = _node_collide(oracle, w, pos, fpre[:, j], beta[j], ids[j], int(c))
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
