"""Seeded synthetic workloads shaped like the paper's runs.

This module only draws inputs: particle placements, orientations, random initial fields
and the parameter sets of the standard workloads. It contains none of the method's
arithmetic (no equilibrium, collision, solid fraction or contact law), so the CUDA path
and the FP64 oracle can both be fed from it without sharing any computation.

Conventions: lattice nodes sit at integer coordinates 0..n-1, walls lie halfway at -1/2
and n-1/2. Particle arrays are per particle with xyz contiguous; the orientation triad is
``(n, 9)`` = d1, d2, d3 (unit body axes in world components).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 12345


def rng(index: int) -> np.random.Generator:
    """PCG64 generator for workload ``index`` (seed 12345 + index)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(index)))


def random_quaternions(g: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly random unit quaternions (w, x, y, z), Shoemake's method."""
    u1, u2, u3 = g.random(n), g.random(n), g.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)
    return q[:, [3, 0, 1, 2]]


def quaternion_to_triad(q: np.ndarray) -> np.ndarray:
    """Rows d1, d2, d3 of the rotation that maps world components to body components.

    The body axis d_m, expressed in world coordinates, is column m of the usual
    body-to-world rotation matrix of the quaternion.
    """
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    M = np.empty((len(q), 3, 3))
    M[:, 0, 0] = 1 - 2 * (y * y + z * z)
    M[:, 0, 1] = 2 * (x * y - w * z)
    M[:, 0, 2] = 2 * (x * z + w * y)
    M[:, 1, 0] = 2 * (x * y + w * z)
    M[:, 1, 1] = 1 - 2 * (x * x + z * z)
    M[:, 1, 2] = 2 * (y * z - w * x)
    M[:, 2, 0] = 2 * (x * z - w * y)
    M[:, 2, 1] = 2 * (y * z + w * x)
    M[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return np.ascontiguousarray(np.transpose(M, (0, 2, 1)).reshape(len(q), 9))


def identity_triads(n: int) -> np.ndarray:
    return np.tile(np.eye(3).reshape(1, 9), (n, 1))


def rsa_spheres(g: np.random.Generator, n: int, radii: np.ndarray, lo, hi, periodic,
                gap: float = 0.0, max_tries: int = 200000) -> np.ndarray:
    """Random sequential addition of non-overlapping spheres.

    Centres are drawn uniformly in [lo + R, hi - R] on wall axes and in [lo, hi) on
    periodic axes; a draw is kept if it is at least R_i + R_j + gap from every kept
    sphere (minimum image on periodic axes). Raises if ``max_tries`` is exhausted.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    rmax = float(np.max(radii)) if n else 1.0
    h = 2 * rmax + gap
    gn = np.maximum(1, np.floor(L / h)).astype(int)
    gh = L / gn
    cells: dict = {}
    pos = np.zeros((n, 3))
    tries = 0
    for k in range(n):
        R = radii[k]
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError(f"RSA jammed after placing {k} of {n} spheres")
            p = np.empty(3)
            for a in range(3):
                if periodic[a]:
                    p[a] = lo[a] + g.random() * L[a]
                else:
                    p[a] = lo[a] + R + g.random() * (L[a] - 2 * R)
            c = np.minimum(np.floor((p - lo) / gh).astype(int), gn - 1)
            ok = True
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        q = c + np.array([dx, dy, dz])
                        skip = False
                        for a in range(3):
                            if q[a] < 0 or q[a] >= gn[a]:
                                if periodic[a]:
                                    q[a] %= gn[a]
                                else:
                                    skip = True
                        if skip:
                            continue
                        for j in cells.get(tuple(q), ()):
                            d = p - pos[j]
                            for a in range(3):
                                if periodic[a]:
                                    d[a] -= L[a] * np.round(d[a] / L[a])
                            if d @ d < (R + radii[j] + gap) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[k] = p
                cells.setdefault(tuple(c), []).append(k)
                break
    return pos


@dataclass
class Workload:
    """A lattice/particle problem with its parameters (lattice units)."""
    name: str
    nx: int = 0
    ny: int = 0
    nz: int = 0
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (1, 1, 1)
    u_wall: np.ndarray = field(default_factory=lambda: np.zeros((3, 2, 3)))
    params: dict = field(default_factory=dict)
    shape: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    radius: np.ndarray = field(default_factory=lambda: np.zeros(0))
    semi: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    density: np.ndarray = field(default_factory=lambda: np.zeros(0))
    pos: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    vel: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    omg: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    triad: np.ndarray = field(default_factory=lambda: np.zeros((0, 9)))
    init_u: np.ndarray | None = None      # (3, ncell) initial velocity field or None
    steps: int = 1
    notes: str = ""

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return len(self.shape)


def base_params(**kw) -> dict:
    """Default parameter set (lattice units); keys mirror the C-ABI parameter struct."""
    p = dict(tau=0.8, fluid_force=(0.0, 0.0, 0.0), storage="f32", voxel="distance",
             subdiv_n=10, law="linear", n_sub=1, rho_f=1.0, gravity=(0.0, 0.0, 0.0),
             k_n=1000.0, k_t=1000.0 * 2.0 / 7.0, young=1.0e4, poisson=0.3, restitution=0.7,
             friction=0.4, skin=0.5, dem_h=0.0, ell_max_iter=60, ell_tol=1e-6,
             force_fp32=1, collision="bgk", orient="triad", pattern="ab")
    p.update(kw)
    return p


def settling_sphere(steps: int = 2000) -> Workload:
    """Single sphere settling in a closed box (32x32x64, tau 0.8, R 4, density ratio 2.5,
    gravity 1e-5 on the particle with analytic buoyancy, subdivision solid fractions)."""
    w = Workload(name="settling_sphere_32x32x64", nx=32, ny=32, nz=64, periodic=(0, 0, 0))
    R, rho_p = 4.0, 2.5
    m = rho_p * 4.0 / 3.0 * math.pi * R ** 3
    # Linear wall contact lasting at least 20 steps: k_n <= m (pi/20)^2.
    kn = 0.6 * m * (math.pi / 20.0) ** 2
    w.params = base_params(tau=0.8, voxel="subdiv", gravity=(0.0, 0.0, -1e-5), k_n=kn,
                           k_t=kn * 2.0 / 7.0, skin=0.5, dem_h=2 * R + 0.5)
    w.shape = np.zeros(1, dtype=np.int32)
    w.radius = np.array([R])
    w.semi = np.array([[R, R, R]])
    w.density = np.array([rho_p])
    w.pos = np.array([[16.0, 16.0, 48.0]])
    w.vel = np.zeros((1, 3))
    w.omg = np.zeros((1, 3))
    w.triad = identity_triads(1)
    w.steps = steps
    return w


def couette_suspension(nx: int = 256, ny: int = 256, nz: int = 256, n_particles: int = 4000,
                       radius: float = 6.0, u_wall: float = 0.05, steps: int = 5000,
                       seed_index: int = 3, storage: str = "f32") -> Workload:
    """Particle-laden Couette flow: walls at z moving at -/+ u_wall along x, periodic x
    and y, RSA spheres of equal density with the fluid (no gravity), distance-based solid
    fractions, 10 DEM substeps, linear contacts lasting >= 20 substeps."""
    g = rng(seed_index)
    w = Workload(name=f"couette_suspension_{nx}x{ny}x{nz}_{n_particles}spheres",
                 nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0))
    uw = np.zeros((3, 2, 3))
    uw[2, 0, 0] = -u_wall
    uw[2, 1, 0] = +u_wall
    w.u_wall = uw
    m = 4.0 / 3.0 * math.pi * radius ** 3
    n_sub = 10
    kn = 0.45 * (m / 2) * (math.pi / (20.0 / n_sub)) ** 2
    w.params = base_params(tau=0.8, voxel="distance", n_sub=n_sub, rho_f=1.0, k_n=kn,
                           k_t=kn * 2.0 / 7.0, skin=0.5, dem_h=2 * radius + 0.5,
                           storage=storage)
    radii = np.full(n_particles, radius)
    lo = (-0.5, -0.5, -0.5 + 1.0)
    hi = (nx - 0.5, ny - 0.5, nz - 0.5 - 1.0)
    w.pos = rsa_spheres(g, n_particles, radii, lo, hi, (1, 1, 0), gap=0.1)
    w.shape = np.zeros(n_particles, dtype=np.int32)
    w.radius = radii
    w.semi = np.tile(radii[:, None], (1, 3))
    w.density = np.ones(n_particles)
    # Fluid and particles start on the linear wall-driven profile.
    zc = w.pos[:, 2]
    w.vel = np.zeros((n_particles, 3))
    w.vel[:, 0] = -u_wall + 2 * u_wall * (zc + 0.5) / nz
    w.omg = np.zeros((n_particles, 3))
    w.triad = identity_triads(n_particles)
    z = np.arange(nz, dtype=np.float64)
    prof = -u_wall + 2 * u_wall * (z + 0.5) / nz
    u = np.zeros((3, nz, ny, nx))
    u[0] = prof[:, None, None]
    w.init_u = u.reshape(3, -1)
    w.steps = steps
    return w


def granular_box(n_particles: int = 100000, box=(120.0, 120.0, 240.0), seed_index: int = 2,
                 steps: int = 10000) -> Workload:
    """DEM-only granular box: radii U[0.8, 1.2], jittered cubic lattice of spacing 2.5
    (sites chosen by a seeded shuffle), walls on all faces, linear law, mu 0.4,
    restitution 0.7, cell size 2.4 plus skin, gravity along -z.

    The box of the workload description (60x60x120) cannot hold 1e5 such spheres
    (their volume exceeds the box); it is read as 120x120x240.
    """
    g = rng(seed_index)
    w = Workload(name=f"granular_box_{n_particles}spheres", box_lo=(0.0, 0.0, 0.0),
                 box_hi=tuple(box), periodic=(0, 0, 0))
    radii = g.uniform(0.8, 1.2, n_particles)
    sp = 2.5
    ns = [int((box[a] - 2 * 1.2) // sp) for a in range(3)]
    sites = np.stack(np.meshgrid(*[1.2 + sp / 2 + sp * np.arange(ns[a]) for a in range(3)],
                                 indexing="ij"), axis=-1).reshape(-1, 3)
    if len(sites) < n_particles:
        raise ValueError("box too small for the requested particle count")
    sel = g.permutation(len(sites))[:n_particles]
    pos = sites[sel] + g.uniform(-0.04, 0.04, (n_particles, 3))
    rho_p = 1.0
    m_min = rho_p * 4.0 / 3.0 * math.pi * 0.8 ** 3
    kn = 0.9 * (m_min / 2) * (math.pi / 20.0) ** 2
    w.params = base_params(tau=0.8, rho_f=0.0, gravity=(0.0, 0.0, -2e-6), k_n=kn,
                           k_t=kn * 2.0 / 7.0, restitution=0.7, friction=0.4, skin=0.2,
                           dem_h=2.4 + 0.2, n_sub=1)
    w.shape = np.zeros(n_particles, dtype=np.int32)
    w.radius = radii
    w.semi = np.tile(radii[:, None], (1, 3))
    w.density = np.full(n_particles, rho_p)
    w.pos = pos
    w.vel = np.zeros((n_particles, 3))
    w.omg = np.zeros((n_particles, 3))
    w.triad = identity_triads(n_particles)
    w.steps = steps
    return w


def random_fields(g: np.random.Generator, nx: int, ny: int, nz: int, amp_u: float = 0.02,
                  amp_rho: float = 0.01, modes: int = 3):
    """Smooth random density and velocity fields: a few random Fourier modes."""
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    rho = np.ones((nx, ny, nz))
    u = np.zeros((3, nx, ny, nz))
    for _ in range(modes):
        k = g.integers(1, 3, 3)
        ph = g.random(4) * 2 * np.pi
        arg = 2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz)
        rho += amp_rho * g.uniform(-1, 1) * np.cos(arg + ph[0])
        for a in range(3):
            u[a] += amp_u * g.uniform(-1, 1) * np.cos(arg + ph[1 + a])
    # to [component][cell] with cell = x + nx*(y + ny*z)
    rho = np.ascontiguousarray(np.transpose(rho, (2, 1, 0)).reshape(-1))
    u = np.ascontiguousarray(np.transpose(u, (0, 3, 2, 1)).reshape(3, -1))
    return rho, u


def population_noise(g: np.random.Generator, ncell: int, amp: float = 1e-3) -> np.ndarray:
    """Uniform noise of shape (19, ncell) used to push populations off equilibrium."""
    return g.uniform(-amp, amp, (19, ncell))


def _place_greedy(g: np.random.Generator, radii: np.ndarray, lo, hi, periodic, gap: float,
                  draws: int = 256):
    """Random sequential addition with a bounded number of draws per sphere: each sphere
    takes the first uniform candidate (drawn in batches of 64, 512, then ``draws``) that
    clears every kept sphere by ``gap`` (minimum image on periodic axes), or is dropped.
    Returns (positions, radii)."""
    L = hi - lo
    per = np.array([bool(x) for x in periodic])
    keep_p, keep_r = [], []
    P = np.zeros((0, 3))
    Rk = np.zeros(0)
    for R in radii:
        lo_c = np.where(per, lo, lo + R)
        span = np.where(per, L, L - 2 * R)
        placed = False
        for batch in (64, 512, draws):   # small batches first: most spheres fit at once
            cand = lo_c + g.random((batch, 3)) * span
            if len(P):
                d = cand[:, None, :] - P[None, :, :]
                d = np.where(per, d - L * np.round(d / L), d)
                ok = ((d ** 2).sum(-1) >= (R + Rk + gap) ** 2).all(1)
            else:
                ok = np.ones(batch, dtype=bool)
            idx = np.flatnonzero(ok)
            if idx.size:
                keep_p.append(cand[idx[0]])
                keep_r.append(R)
                P = np.array(keep_p)
                Rk = np.array(keep_r)
                placed = True
                break
            if batch >= draws:
                break
        if not placed:
            continue
    return np.array(keep_p).reshape(-1, 3), np.array(keep_r)


def batched_ensemble(nsim: int = 64, seed_index: int = 5, steps: int = 1000,
                     storage: str = "f16") -> list:
    """Ensemble of independent simulations for one batched launch: lattice edges drawn
    independently from U{24..96}, tau ~ U[0.6, 1.2], 1-64 spheres with radii U[3, 8],
    alternately settling (closed box, gravity 1e-5 on particles of density ratio 2.5) and
    sheared (z walls at -/+0.05, periodic x and y, neutrally buoyant), distance-based solid
    fractions, one DEM substep.

    Placement: random sequential addition at solid fraction <= 0.3 and one lattice unit
    from the walls; a sphere that finds no room after a bounded number of draws is left
    out, and the largest radius is capped where a small periodic box or lattice could not
    hold it (a periodic edge must exceed twice the contact range, as the minimum-image
    convention needs)."""
    g = rng(seed_index)
    out = []
    skin = 0.5
    for i in range(nsim):
        n3 = [int(g.integers(24, 97)) for _ in range(3)]
        tau = float(g.uniform(0.6, 1.2))
        settling = i % 2 == 0
        periodic = (0, 0, 0) if settling else (1, 1, 0)
        w = Workload(name=f"ensemble_{i}", nx=n3[0], ny=n3[1], nz=n3[2], periodic=periodic)
        if not settling:
            w.u_wall[2, 0, 0] = -0.05
            w.u_wall[2, 1, 0] = +0.05
        rmax = min(8.0, (min(n3) - 4) / 2.0)
        per_edges = [n3[a] for a in range(3) if periodic[a]]
        if per_edges:
            rmax = min(rmax, (min(per_edges) / 2.0 - skin) / 2.0 - 0.25)
        rmax = max(rmax, 3.0)
        n_target = int(g.integers(1, 65))
        radii = g.uniform(3.0, rmax, n_target)
        vol = float(np.prod(n3))
        while len(radii) > 1 and (4.0 / 3.0 * math.pi * radii ** 3).sum() > 0.3 * vol:
            radii = radii[:-1]
        lo = np.array([-0.5 if periodic[a] else 0.5 for a in range(3)])
        hi = np.array([n3[a] - 0.5 - (0 if periodic[a] else 1.0) for a in range(3)])
        pos, radii = _place_greedy(g, radii, lo, hi, periodic, gap=0.2)
        n = len(radii)
        rho_p = 2.5 if settling else 1.0
        m_min = rho_p * 4.0 / 3.0 * math.pi * radii.min() ** 3
        kn = 0.5 * (m_min / 2) * (math.pi / 20.0) ** 2
        w.params = base_params(tau=tau, storage=storage, voxel="distance", n_sub=1, rho_f=1.0,
                               gravity=(0.0, 0.0, -1e-5) if settling else (0.0, 0.0, 0.0),
                               k_n=kn, k_t=kn * 2.0 / 7.0, skin=skin, dem_h=2 * rmax + skin)
        w.shape = np.zeros(n, dtype=np.int32)
        w.radius = radii
        w.semi = np.tile(radii[:, None], (1, 3))
        w.density = np.full(n, rho_p)
        w.pos = pos
        w.vel = np.zeros((n, 3))
        w.omg = np.zeros((n, 3))
        w.triad = identity_triads(n)
        if not settling:
            w.vel[:, 0] = -0.05 + 0.1 * (pos[:, 2] + 0.5) / n3[2]
            z = np.arange(n3[2], dtype=np.float64)
            u = np.zeros((3, n3[2], n3[1], n3[0]))
            u[0] = (-0.05 + 0.1 * (z + 0.5) / n3[2])[:, None, None]
            w.init_u = u.reshape(3, -1)
        w.steps = steps
        out.append(w)
    return out


def _pw_overlap(ra, Ainv, rb, Binv, iters: int = 40) -> np.ndarray:
    """Perram-Wertheim test for pairs of ellipsoids (rows): they overlap iff
    max_{l in [0,1]} l (1 - l) r^T [(1 - l) A^-1 + l B^-1]^-1 r < 1, r = r_b - r_a, with
    A^-1 = R^T diag(a^2) R the inverse shape matrix. The function is concave in l; its
    maximum is found by golden-section search."""
    r = rb - ra

    def F(lam):
        C = (1.0 - lam)[:, None, None] * Ainv + lam[:, None, None] * Binv
        x = np.linalg.solve(C, r[:, :, None])[:, :, 0]
        return lam * (1.0 - lam) * (r * x).sum(1)

    lo = np.zeros(len(r))
    hi = np.ones(len(r))
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    x1 = hi - gr * (hi - lo)
    x2 = lo + gr * (hi - lo)
    f1, f2 = F(x1), F(x2)
    for _ in range(iters):
        left = f1 < f2            # the maximum lies in [x1, hi]
        lo = np.where(left, x1, lo)
        hi = np.where(left, hi, x2)
        nx1 = hi - gr * (hi - lo)
        nx2 = lo + gr * (hi - lo)
        x1, x2 = np.where(left, x2, nx1), np.where(left, nx2, x1)
        f1n, f2n = np.where(left, f2, F(nx1)), np.where(left, F(nx2), f1)
        f1, f2 = f1n, f2n
    return np.maximum(f1, f2) < 1.0


def ellipsoid_shear(nx: int = 384, ny: int = 384, nz: int = 192, n_particles: int = 20000,
                    semi=(6.0, 2.0, 2.0), shear_rate: float = 1e-4, steps: int = 3000,
                    seed_index: int = 4, storage: str = "f32", gap: float = 0.2) -> Workload:
    """Prolate ellipsoids in simple shear: walls at z moving at -/+ shear_rate nz/2 along x,
    periodic x and y, uniformly random orientations (Shoemake quaternions), subdivision
    solid fractions, common-normal contacts, 10 DEM substeps, neutrally buoyant.

    Placement: centres uniform in the box (one semi-axis plus a lattice unit from the
    walls); every pair closer than the sum of the largest semi-axes is tested exactly
    (Perram-Wertheim, with the semi-axes grown by gap/2), and one member of each
    overlapping pair is redrawn, until no pair overlaps."""
    g = rng(seed_index)
    a = np.asarray(semi, dtype=np.float64)
    n = n_particles
    w = Workload(name=f"ellipsoid_shear_{nx}x{ny}x{nz}_{n}ellipsoids", nx=nx, ny=ny, nz=nz,
                 periodic=(1, 1, 0))
    U = shear_rate * nz / 2.0
    w.u_wall[2, 0, 0] = -U
    w.u_wall[2, 1, 0] = +U
    L = np.array([nx, ny, nz], dtype=np.float64)
    lo = np.array([-0.5, -0.5, 0.5 + a.max()])
    span = np.array([nx, ny, nz - 2.0 - 2.0 * a.max()])
    grown = a + gap / 2.0
    pos = lo + g.random((n, 3)) * span
    quat = random_quaternions(g, n)
    triad = quaternion_to_triad(quat)
    reach = 2.0 * grown.max()
    for _ in range(200):
        # candidate pairs by a uniform grid of cell size >= reach (minimum image in x, y)
        gn = np.maximum(1, np.floor(L / reach)).astype(int)
        cell = np.minimum(np.floor((pos - np.array([-0.5, -0.5, -0.5])) / (L / gn)).astype(int), gn - 1)
        key = cell[:, 0] + gn[0] * (cell[:, 1] + gn[1] * cell[:, 2])
        order = np.argsort(key, kind="stable")
        sk = key[order]
        starts = np.searchsorted(sk, np.arange(gn.prod() + 1))
        pairs_i, pairs_j = [], []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    c2 = cell + np.array([dx, dy, dz])
                    c2[:, 0] %= gn[0]
                    c2[:, 1] %= gn[1]
                    ok = (c2[:, 2] >= 0) & (c2[:, 2] < gn[2])
                    k2 = c2[:, 0] + gn[0] * (c2[:, 1] + gn[1] * np.clip(c2[:, 2], 0, gn[2] - 1))
                    s0, s1 = starts[k2], starts[k2 + 1]
                    cnt = np.where(ok, s1 - s0, 0)
                    idx_i = np.repeat(np.arange(n), cnt)
                    off = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                    idx_j = order[np.repeat(s0, cnt) + off]
                    keep = idx_i < idx_j
                    pairs_i.append(idx_i[keep])
                    pairs_j.append(idx_j[keep])
        pi = np.concatenate(pairs_i)
        pj = np.concatenate(pairs_j)
        uniq = np.unique(pi.astype(np.int64) * n + pj)
        pi, pj = uniq // n, uniq % n
        d = pos[pj] - pos[pi]
        d[:, :2] -= L[:2] * np.round(d[:, :2] / L[:2])
        close = (d * d).sum(1) < reach * reach
        pi, pj = pi[close], pj[close]
        if len(pi) == 0:
            break
        R = triad.reshape(n, 3, 3)            # rows d1, d2, d3 (body axes in world components)
        inv = np.einsum("nki,k,nkj->nij", R, grown ** 2, R)
        rb = pos[pi] + d[close]
        hit = _pw_overlap(pos[pi], inv[pi], rb, inv[pj])
        bad = np.unique(pj[hit])
        if len(bad) == 0:
            break
        pos[bad] = lo + g.random((len(bad), 3)) * span
        q = random_quaternions(g, len(bad))
        triad[bad] = quaternion_to_triad(q)
    else:
        raise RuntimeError("ellipsoid placement did not converge")
    rho_p = 1.0
    vol = 4.0 / 3.0 * math.pi * a.prod()
    m = rho_p * vol
    kn = 0.5 * (m / 2) * (math.pi / 20.0 * 10) ** 2   # contact >= 20 substeps (dt_p = 1/10)
    w.params = base_params(tau=0.8, storage=storage, voxel="subdiv", subdiv_n=10, n_sub=10,
                           rho_f=1.0, law="linear", k_n=kn, k_t=kn * 2.0 / 7.0, skin=0.5,
                           dem_h=2.0 * a.max() + 0.5)
    w.shape = np.ones(n, dtype=np.int32)
    w.radius = np.full(n, a.max())
    w.semi = np.tile(a, (n, 1))
    w.density = np.full(n, rho_p)
    w.pos = pos
    zc = pos[:, 2]
    w.vel = np.zeros((n, 3))
    w.vel[:, 0] = -U + 2.0 * U * (zc + 0.5) / nz
    w.omg = np.zeros((n, 3))
    w.triad = triad
    z = np.arange(nz, dtype=np.float64)
    u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    u[0] = (-U + 2.0 * U * (z + 0.5) / nz)[:, None, None]
    w.init_u = u.reshape(3, -1)
    w.steps = steps
    return w


def fluidised_bed(phi: float, nx: int = 500, ny: int = 200, nz: int = 800, diameter: float = 20.0,
                  steps: int = 100, seed_index: int = 6, storage: str = "f32") -> Workload:
    """The paper's performance workload shape: 500 x 200 x 800 lattice, periodic x and z,
    walls on y, gravity along -y on the particles, density ratio 1.1, spheres of diameter
    20 lattice units, 10 DEM substeps, distance-based solid fractions, tau for Re = 1.

    Placement: a jittered simple-cubic lattice of spacing 1.05 diameters (sites one radius
    plus a lattice unit from the walls) holds solid fraction up to about 0.43; a seeded
    random subset of its sites gives the requested fraction (clamped to what it holds;
    0.41 for the default box)."""
    g = rng(seed_index)
    R = diameter / 2.0
    sp = 1.05 * diameter
    w = Workload(name=f"fluidised_bed_{nx}x{ny}x{nz}_phi{phi:.2f}", nx=nx, ny=ny, nz=nz,
                 periodic=(1, 0, 1))
    lo = np.array([-0.5, 0.5 + R, -0.5])
    hi = np.array([nx - 0.5, ny - 1.5 - R, nz - 0.5])
    ns = [int(nx // sp), int((hi[1] - lo[1]) // sp) + 1, int(nz // sp)]
    axes = [lo[a] + sp / 2 + sp * np.arange(ns[a]) if a != 1 else
            np.linspace(lo[1], hi[1], ns[1]) for a in range(3)]
    sites = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    vol = 4.0 / 3.0 * math.pi * R ** 3
    n = min(len(sites), int(round(phi * nx * ny * nz / vol)))
    sel = g.permutation(len(sites))[:n]
    jit = 0.4 * (sp - diameter)
    pos = sites[sel] + g.uniform(-jit, jit, (n, 3))
    rho_p = 1.1
    m = rho_p * vol
    kn = 0.5 * (m / 2) * (math.pi / 2.0) ** 2      # contact >= 20 substeps of 1/10
    u_ref = 0.01
    nu = u_ref * diameter / 1.0                     # Re = u d / nu = 1
    tau = 0.5 + 3.0 * nu
    w.params = base_params(tau=tau, storage=storage, voxel="distance", n_sub=10, rho_f=1.0,
                           gravity=(0.0, -1e-6, 0.0), law="linear", k_n=kn, k_t=kn * 2.0 / 7.0,
                           skin=0.5, dem_h=diameter + 0.5)
    w.shape = np.zeros(n, dtype=np.int32)
    w.radius = np.full(n, R)
    w.semi = np.full((n, 3), R)
    w.density = np.full(n, rho_p)
    w.pos = pos
    w.vel = np.zeros((n, 3))
    w.omg = np.zeros((n, 3))
    w.triad = identity_triads(n)
    w.steps = steps
    return w


def rheology_suspension(phi: float, n: int = 96, radius: float = 5.0, u_wall: float = 0.05,
                        seed_index: int = 7, storage: str = "f32") -> Workload:
    """Sheared suspension for the effective viscosity (Sec. 4.8 setup at reduced size):
    n^3 lattice, walls at z moving at -/+ u_wall along x, periodic x and y, neutrally
    buoyant spheres of radius 5 (10 cells per diameter, as in the paper) at solid fraction
    phi placed at random (bounded draws; the fraction reached is n_spheres * volume / n^3),
    fluid and particles on the linear profile, 10 DEM substeps, linear law lasting 20
    substeps, friction 0.45, restitution 0.95, distance-based solid fractions."""
    g = rng(seed_index)
    w = Workload(name=f"rheology_{n}^3_phi{phi:.2f}", nx=n, ny=n, nz=n, periodic=(1, 1, 0))
    w.u_wall[2, 0, 0] = -u_wall
    w.u_wall[2, 1, 0] = +u_wall
    vol = 4.0 / 3.0 * math.pi * radius ** 3
    target = int(round(phi * n ** 3 / vol))
    lo = np.array([-0.5, -0.5, 0.5])
    hi = np.array([n - 0.5, n - 0.5, n - 1.5])
    pos, radii = _place_greedy(g, np.full(target, radius), lo, hi, (1, 1, 0), gap=0.2, draws=2048)
    k = len(radii)
    m = vol
    kn = 0.5 * (m / 2) * (math.pi / 2.0) ** 2   # contact >= 20 substeps of 1/10
    w.params = base_params(tau=0.8, storage=storage, voxel="distance", n_sub=10, rho_f=1.0,
                           law="linear", k_n=kn, k_t=kn * 2.0 / 7.0, restitution=0.95, friction=0.45,
                           skin=0.5, dem_h=2 * radius + 0.5)
    w.shape = np.zeros(k, dtype=np.int32)
    w.radius = radii
    w.semi = np.tile(radii[:, None], (1, 3))
    w.density = np.ones(k)
    w.pos = pos
    w.vel = np.zeros((k, 3))
    w.vel[:, 0] = -u_wall + 2.0 * u_wall * (pos[:, 2] + 0.5) / n
    w.omg = np.zeros((k, 3))
    w.omg[:, 1] = u_wall / n      # the rotation of the undisturbed shear flow (du/dz / 2)
    w.triad = identity_triads(k)
    z = np.arange(n, dtype=np.float64)
    u = np.zeros((3, n, n, n), dtype=np.float32)
    u[0] = (-u_wall + 2.0 * u_wall * (z + 0.5) / n)[:, None, None]
    w.init_u = u.reshape(3, -1)
    w.steps = 20000
    return w


def wall_shear_rate(ux_profile: np.ndarray, u_wall: float) -> float:
    """Shear rate at the walls of a z-profile of u_x between halfway walls at -1/2 (moving at
    -u_wall) and nz - 1/2 (+u_wall): slope at the wall of the parabola through the wall value
    and the first two fluid nodes (Sec. 4.8), averaged over both walls."""
    u = np.asarray(ux_profile, dtype=np.float64)
    bottom = -8.0 / 3.0 * (-u_wall) + 3.0 * u[0] - u[1] / 3.0
    top = -8.0 / 3.0 * u_wall + 3.0 * u[-1] - u[-2] / 3.0
    return 0.5 * (bottom - top)


def jeffery_ellipsoid(a: float = 12.0, b: float = 6.0, box=(96, 64, 96), u_wall: float = 0.05,
                      angle: float = 0.0, tau: float = 0.8, steps: int = 9000) -> Workload:
    """One neutrally buoyant prolate ellipsoid (semi-axes a, b, b) at the centre of a
    sheared box (walls at z moving at -/+ u_wall along x, periodic x and y), its major axis
    in the flow-gradient (x-z) plane at `angle` from the flow direction, started with the
    fluid's rotation rate; subdivision solid fractions. Jeffery: the major axis turns by pi
    in pi (a^2 + b^2) / (a b shear_rate)."""
    nx, ny, nz = box
    w = Workload(name=f"jeffery_{a:g}x{b:g}_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0))
    w.u_wall[2, 0, 0] = -u_wall
    w.u_wall[2, 1, 0] = +u_wall
    shear = 2.0 * u_wall / nz
    c, s = math.cos(angle), math.sin(angle)
    d1 = np.array([c, 0.0, s])
    d2 = np.array([0.0, 1.0, 0.0])
    d3 = np.cross(d1, d2)
    vol = 4.0 / 3.0 * math.pi * a * b * b
    kn = 0.5 * vol * (math.pi / 2.0) ** 2
    w.params = base_params(tau=tau, voxel="subdiv", subdiv_n=10, n_sub=10, rho_f=1.0, law="linear",
                           k_n=kn, k_t=kn * 2.0 / 7.0, skin=0.5, dem_h=2.0 * a + 0.5)
    w.shape = np.ones(1, dtype=np.int32)
    w.radius = np.array([a])
    w.semi = np.array([[a, b, b]])
    w.density = np.ones(1)
    w.pos = np.array([[nx / 2.0 - 0.5, ny / 2.0 - 0.5, nz / 2.0 - 0.5]])
    w.vel = np.zeros((1, 3))
    w.omg = np.array([[0.0, shear / 2.0, 0.0]])
    w.triad = np.concatenate([d1, d2, d3])[None, :]
    z = np.arange(nz, dtype=np.float64)
    u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    u[0] = (-u_wall + 2.0 * u_wall * (z + 0.5) / nz)[:, None, None]
    w.init_u = u.reshape(3, -1)
    w.steps = steps
    return w
