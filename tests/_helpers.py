"""Helpers shared by the GPU parity tests: build the oracle and the CUDA simulation from the
same seeded workload, and the error norms the tolerances are stated in."""
import numpy as np

from paper_2512_04997_gb300 import workloads as W


def oracle_from_workload(O, w, populations=None):
    """The oracle simulation of workload w (O: the oracle module)."""
    return O.from_workload(w, populations=populations)


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
