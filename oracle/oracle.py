"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use this
module. It marshals numpy arrays into ``ledds_oracle.c``; all arithmetic is in C.
Particle arrays here are per particle with xyz contiguous (shape ``(n, 3)``), the triad
is ``(n, 9)`` = d1, d2, d3, and fields are ``[component][cell]`` with the cell index
``x + nx*(y + ny*z)``.
"""
import ctypes as C
import numpy as np

from . import build as _build

SPHERE, ELLIPSOID = 0, 1
VOXEL_DISTANCE, VOXEL_SUBDIV = 0, 1
LAW_LINEAR, LAW_HERTZ = 0, 1
COLLIDE_BGK, COLLIDE_TRT = 0, 1
ORIENT_TRIAD, ORIENT_QUAT = 0, 1


class Params(C.Structure):
    _fields_ = [
        ("tau", C.c_double),
        ("fluid_force", C.c_double * 3),
        ("voxel", C.c_int),
        ("subdiv_n", C.c_int),
        ("law", C.c_int),
        ("n_sub", C.c_int),
        ("rho_f", C.c_double),
        ("gravity", C.c_double * 3),
        ("k_n", C.c_double),
        ("k_t", C.c_double),
        ("young", C.c_double),
        ("poisson", C.c_double),
        ("restitution", C.c_double),
        ("friction", C.c_double),
        ("dem_h", C.c_double),
        ("ell_max_iter", C.c_int),
        ("ell_tol", C.c_double),
        ("collision", C.c_int),
        ("orient", C.c_int),
    ]


_libs = {}


def lib(parallel=False):
    """The parity build (serial, in order), or with parallel=True the OpenMP build that
    times the CPU baseline."""
    if parallel not in _libs:
        path = _build.build(parallel=parallel)
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, ip, dp, C.POINTER(Params), C.c_int]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_init_equilibrium.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_set_populations.argtypes = [C.c_void_p, dp]
        L.or_get_populations.argtypes = [C.c_void_p, dp]
        L.or_moments.argtypes = [C.c_void_p, dp, dp]
        L.or_equilibrium.argtypes = [C.c_double, dp, dp]
        L.or_lattice_tables.argtypes = [ip, dp, ip]
        L.or_set_particles.restype = C.c_int
        L.or_set_particles.argtypes = [C.c_void_p, C.c_int, ip, dp, dp, dp, dp, dp, dp, dp]
        L.or_get_particles.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.or_get_forces.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.or_get_accel.argtypes = [C.c_void_p, dp, dp]
        L.or_quat_from_triad.argtypes = [dp, dp]
        L.or_bk.restype = C.c_double
        L.or_bk.argtypes = [C.c_double, C.c_double]
        L.or_triad_from_quat.argtypes = [dp, dp]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_voxelize.argtypes = [C.c_void_p, dp, ip, ip]
        L.or_lbm_psm_step.argtypes = [C.c_void_p]
        L.or_cell_keys.restype = C.c_int
        L.or_cell_keys.argtypes = [C.c_void_p, up, ip, ip]
        L.or_contacts.restype = C.c_int
        L.or_contacts.argtypes = [C.c_void_p, lp, C.c_int]
        L.or_contact_forces.argtypes = [C.c_void_p, C.c_double]
        L.or_subdiv_count.restype = C.c_int
        L.or_subdiv_count.argtypes = [dp, C.c_int, C.c_double, dp, dp, C.c_int]
        L.or_beta_distance.restype = C.c_double
        L.or_beta_distance.argtypes = [dp, C.c_double]
        L.or_cell_collide.argtypes = [dp, C.c_double, C.c_int, dp, C.c_int, dp, dp, dp, dp, dp, dp]
        L.or_pw_separated.restype = C.c_int
        L.or_pw_separated.argtypes = [dp, dp, dp, dp, dp, dp]
        L.or_ellipsoid_contact.restype = C.c_int
        L.or_ellipsoid_contact.argtypes = [dp, dp, dp, dp, dp, dp, C.c_int, C.c_double,
                                           dp, dp, dp, dp, dp, ip]
        L.or_status.argtypes = [C.c_void_p, lp]
        L.or_solids_at.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, ip, dp, ip]
        L.or_threads.restype = C.c_int
        L.or_threads.argtypes = []
        _libs[parallel] = L
    return _libs[parallel]


def threads(parallel=False):
    """Threads the oracle's lattice update uses in that build."""
    return int(lib(parallel).or_threads())


def default_params(**kw) -> Params:
    p = Params()
    p.tau = 0.8
    p.voxel = VOXEL_DISTANCE
    p.subdiv_n = 10
    p.law = LAW_LINEAR
    p.n_sub = 1
    p.rho_f = 1.0
    p.k_n = 1000.0
    p.k_t = 1000.0 * 2.0 / 7.0
    p.young = 1.0e4
    p.poisson = 0.3
    p.restitution = 0.7
    p.friction = 0.4
    p.dem_h = 1.0
    p.ell_max_iter = 60
    p.ell_tol = 1e-6
    p.collision = COLLIDE_BGK
    p.orient = ORIENT_TRIAD
    for k, v in kw.items():
        if k in ("fluid_force", "gravity"):
            getattr(p, k)[:] = list(v)
        else:
            setattr(p, k, v)
    return p


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


class Sim:
    """One oracle simulation (lattice and/or particles)."""

    def __init__(self, nx=0, ny=0, nz=0, periodic=(1, 1, 1), u_wall=None, params=None,
                 box_lo=(0, 0, 0), box_hi=(1, 1, 1), max_particles=1, parallel=False):
        self._L = L = lib(parallel)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.ncell = nx * ny * nz
        self.params = params if params is not None else default_params()
        uw = np.zeros(18) if u_wall is None else _d(u_wall).reshape(18)
        self._h = L.or_create(nx, ny, nz, _d(box_lo, 3), _d(box_hi, 3),
                              np.ascontiguousarray(periodic, dtype=np.int32), uw,
                              C.byref(self.params), int(max_particles))
        self.n = 0

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.or_destroy(self._h)
            self._h = None

    # fluid -------------------------------------------------------------------------
    def init_equilibrium(self, rho=None, u=None):
        r = None if rho is None else _d(rho, self.ncell)
        v = None if u is None else _d(u, 3 * self.ncell)
        self._L.or_init_equilibrium(self._h, None if r is None else r.ctypes.data,
                                  None if v is None else v.ctypes.data)
        self._keep = (r, v)

    def set_populations(self, f):
        self._L.or_set_populations(self._h, _d(f, 19 * self.ncell))

    def populations(self):
        out = np.zeros(19 * self.ncell)
        self._L.or_get_populations(self._h, out)
        return out.reshape(19, self.ncell)

    def moments(self):
        rho = np.zeros(self.ncell)
        u = np.zeros(3 * self.ncell)
        self._L.or_moments(self._h, rho, u)
        return rho, u.reshape(3, self.ncell)

    # particles ---------------------------------------------------------------------
    def set_particles(self, shape, radius, semi, density, pos, vel=None, omg=None, triad=None):
        n = len(shape)
        z3 = np.zeros((n, 3))
        if triad is None:
            triad = np.tile(np.eye(3).reshape(1, 9), (n, 1))
        rc = self._L.or_set_particles(self._h, n, np.ascontiguousarray(shape, dtype=np.int32),
                                    _d(radius, n), _d(semi, 3 * n), _d(density, n),
                                    _d(pos, 3 * n), _d(z3 if vel is None else vel, 3 * n),
                                    _d(z3 if omg is None else omg, 3 * n), _d(triad, 9 * n))
        if rc != 0:
            raise ValueError("too many particles for this oracle simulation")
        self.n = n

    def particles(self):
        n = self.n
        pos, vel, omg, tri = np.zeros(3 * n), np.zeros(3 * n), np.zeros(3 * n), np.zeros(9 * n)
        self._L.or_get_particles(self._h, pos, vel, omg, tri)
        return pos.reshape(n, 3), vel.reshape(n, 3), omg.reshape(n, 3), tri.reshape(n, 9)

    def forces(self):
        n = self.n
        a = [np.zeros(3 * n) for _ in range(4)]
        self._L.or_get_forces(self._h, *a)
        return tuple(x.reshape(n, 3) for x in a)  # Fh, Mh, Fc, Mc

    def accel(self):
        n = self.n
        a, b = np.zeros(3 * n), np.zeros(3 * n)
        self._L.or_get_accel(self._h, a, b)
        return a.reshape(n, 3), b.reshape(n, 3)

    # stepping ----------------------------------------------------------------------
    def step(self, nsteps=1):
        self._L.or_step(self._h, int(nsteps))

    def lbm_psm_step(self):
        self._L.or_lbm_psm_step(self._h)

    def contact_forces(self, dt):
        self._L.or_contact_forces(self._h, float(dt))

    def solids_at(self, x, y, z):
        """(ids[2], betas[2], total) of node (x, y, z): the voxelisation of one node."""
        ids = np.zeros(2, dtype=np.int32)
        b = np.zeros(2)
        t = np.zeros(1, dtype=np.int32)
        self._L.or_solids_at(self._h, int(x), int(y), int(z), ids, b, t)
        return ids, b, int(t[0])

    def voxelize(self):
        beta = np.zeros(2 * self.ncell)
        ids = np.zeros(2 * self.ncell, dtype=np.int32)
        ns = np.zeros(self.ncell, dtype=np.int32)
        self._L.or_voxelize(self._h, beta, ids, ns)
        return beta.reshape(self.ncell, 2), ids.reshape(self.ncell, 2), ns

    def cell_keys(self):
        keys = np.zeros(max(self.n, 1), dtype=np.uint32)
        ids = np.zeros(max(self.n, 1), dtype=np.int32)
        g = np.zeros(3, dtype=np.int32)
        self._L.or_cell_keys(self._h, keys, ids, g)
        return keys[: self.n], ids[: self.n], tuple(int(x) for x in g)

    def contacts(self):
        cap = max(16, 16 * self.n)
        while True:
            out = np.zeros(cap, dtype=np.int64)
            nc = self._L.or_contacts(self._h, out, cap)
            if nc <= cap:
                return out[:nc]
            cap = nc

    def status(self):
        out = np.zeros(4, dtype=np.int64)
        self._L.or_status(self._h, out)
        return {"solids_overflow": int(out[0]), "ell_nonconverged": int(out[1]),
                "steps": int(out[2]), "ncontacts": int(out[3])}


# free functions ----------------------------------------------------------------------

def lattice_tables():
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    lib().or_lattice_tables(c, w, opp)
    return c.reshape(19, 3), w, opp


def equilibrium(rho, u):
    out = np.zeros(19)
    lib().or_equilibrium(float(rho), _d(u, 3), out)
    return out


def subdiv_count(rel, shape, radius, semi=(1, 1, 1), triad=None, n=10):
    tri = np.eye(3).reshape(9) if triad is None else _d(triad, 9)
    return lib().or_subdiv_count(_d(rel, 3), int(shape), float(radius), _d(semi, 3), tri, int(n))


def beta_distance(rel, radius):
    return lib().or_beta_distance(_d(rel, 3), float(radius))


def bk(beta, tau):
    """Solid weight B_k of solid fraction beta, Eq. (bk)."""
    return lib().or_bk(float(beta), float(tau))


def quat_from_triad(triad):
    """Unit quaternion (w, x, y, z) of the body-to-world rotation whose columns are the
    triad rows d1, d2, d3 (Shepperd's method)."""
    q = np.zeros(4)
    lib().or_quat_from_triad(_d(triad, 9), q)
    return q


def triad_from_quat(q):
    """Triad d1, d2, d3 (3x3, rows) of a unit quaternion (w, x, y, z)."""
    d = np.zeros(9)
    lib().or_triad_from_quat(_d(q, 4), d)
    return d.reshape(3, 3)


def cell_collide(f, tau, B=(), uk=(), arm=(), force=(0, 0, 0), collision=0):
    ns = len(B)
    fstar = np.zeros(19)
    Fk = np.zeros(6)
    Mk = np.zeros(6)
    Bb = np.zeros(2)
    Bb[:ns] = B
    ukb = np.zeros(6)
    armb = np.zeros(6)
    if ns:
        ukb[: 3 * ns] = np.asarray(uk, dtype=np.float64).reshape(-1)
        armb[: 3 * ns] = np.asarray(arm, dtype=np.float64).reshape(-1)
    lib().or_cell_collide(_d(f, 19), float(tau), int(collision), _d(force, 3), ns, Bb, ukb, armb, fstar, Fk, Mk)
    return fstar, Fk.reshape(2, 3)[:ns], Mk.reshape(2, 3)[:ns]


def pw_separated(ri, Ri, si, rj, Rj, sj):
    """True if a Perram-Wertheim certificate proves the two ellipsoids disjoint."""
    return bool(lib().or_pw_separated(_d(ri, 3), _d(Ri, 9), _d(si, 3), _d(rj, 3), _d(Rj, 9), _d(sj, 3)))


def ellipsoid_contact(ri, Ri, si, rj, Rj, sj, max_iter=60, tol=1e-6):
    delta = np.zeros(1)
    en = np.zeros(3)
    cp = np.zeros(3)
    rho_i = np.zeros(1)
    rho_j = np.zeros(1)
    it = np.zeros(1, dtype=np.int32)
    rc = lib().or_ellipsoid_contact(_d(ri, 3), _d(Ri, 9), _d(si, 3), _d(rj, 3), _d(Rj, 9),
                                    _d(sj, 3), int(max_iter), float(tol), delta, en, cp,
                                    rho_i, rho_j, it)
    return {"rc": rc, "delta": float(delta[0]), "en": en, "cp": cp,
            "rho_i": float(rho_i[0]), "rho_j": float(rho_j[0]), "iters": int(it[0])}


_VOX = {"distance": 0, "subdiv": 1}
_LAWS = {"linear": 0, "hertz": 1}


def from_workload(w, populations=None, parallel=False):
    """Oracle simulation of a seeded workload description (``workloads.Workload``: lattice,
    walls, parameters and particles), the same inputs the CUDA path receives. parallel:
    the OpenMP timing build."""
    p = dict(w.params)
    op = default_params(tau=p["tau"], fluid_force=p["fluid_force"], voxel=_VOX[p["voxel"]],
                        subdiv_n=p["subdiv_n"], law=_LAWS[p["law"]], n_sub=p["n_sub"],
                        rho_f=p["rho_f"], gravity=p["gravity"], k_n=p["k_n"], k_t=p["k_t"],
                        young=p["young"], poisson=p["poisson"], restitution=p["restitution"],
                        friction=p["friction"], dem_h=p["dem_h"],
                        ell_max_iter=p["ell_max_iter"], ell_tol=p["ell_tol"],
                        collision={"bgk": 0, "trt": 1}[p.get("collision", "bgk")],
                        orient={"triad": 0, "quat": 1}[p.get("orient", "triad")])
    s = Sim(w.nx, w.ny, w.nz, periodic=w.periodic, u_wall=w.u_wall, params=op,
            box_lo=w.box_lo, box_hi=w.box_hi, max_particles=max(w.n, 1), parallel=parallel)
    if w.ncell:
        if populations is not None:
            s.set_populations(populations)
        elif w.init_u is not None:
            s.init_equilibrium(None, w.init_u)
    if w.n:
        s.set_particles(w.shape, w.radius, w.semi, w.density, w.pos, w.vel, w.omg, w.triad)
    return s
