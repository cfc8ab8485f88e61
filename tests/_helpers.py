"""Helpers shared by the GPU parity tests: build the oracle and the CUDA simulation from the
same seeded workload, and the error norms the tolerances are stated in."""
import numpy as np

from paper_2512_04997_gb300 import workloads as W

VOX = {"distance": 0, "subdiv": 1}
LAWS = {"linear": 0, "hertz": 1}


def oracle_from_workload(O, w, populations=None):
    p = dict(w.params)
    op = O.default_params(tau=p["tau"], fluid_force=p["fluid_force"], voxel=VOX[p["voxel"]],
                          subdiv_n=p["subdiv_n"], law=LAWS[p["law"]], n_sub=p["n_sub"],
                          rho_f=p["rho_f"], gravity=p["gravity"], k_n=p["k_n"], k_t=p["k_t"],
                          young=p["young"], poisson=p["poisson"], restitution=p["restitution"],
                          friction=p["friction"], dem_h=p["dem_h"],
                          ell_max_iter=p["ell_max_iter"], ell_tol=p["ell_tol"],
                          collision={"bgk": 0, "trt": 1}[p.get("collision", "bgk")],
                          orient={"triad": 0, "quat": 1}[p.get("orient", "triad")])
    s = O.Sim(w.nx, w.ny, w.nz, periodic=w.periodic, u_wall=w.u_wall, params=op,
              box_lo=w.box_lo, box_hi=w.box_hi, max_particles=max(w.n, 1))
    if w.ncell:
        if populations is not None:
            s.set_populations(populations)
        elif w.init_u is not None:
            s.init_equilibrium(None, w.init_u)
    if w.n:
        s.set_particles(w.shape, w.radius, w.semi, w.density, w.pos, w.vel, w.omg, w.triad)
    return s


def gpu_from_workload(w, populations=None, **over):
    from paper_2512_04997_gb300 import ledds
    s = ledds.from_workload(w, **over)
    if populations is not None:
        s.init_populations(populations)
    return s


def normwise(a, ref):
    """||a - ref||_inf / ||ref||_inf (the field error norm of the parity tolerances)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max()
    return float(np.abs(a - ref).max() / (den if den > 0 else 1.0))


def random_populations(O, g, nx, ny, nz, amp_u=0.02, noise=2e-4):
    """Off-equilibrium populations [19][cells]: equilibrium of smooth random fields plus
    uniform noise (the equilibrium is the oracle's; the CUDA side only receives f)."""
    rho, u = W.random_fields(g, nx, ny, nz, amp_u=amp_u)
    n = nx * ny * nz
    tmp = O.Sim(nx, ny, nz, periodic=(1, 1, 1))
    tmp.init_equilibrium(rho, u)
    return tmp.populations() + W.population_noise(g, n, noise)
