"""ctypes binding of the C-ABI library ``libledds.so`` (include/ledds.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of the
library. The module-level functions carry the C names; ``Sim`` is a convenience wrapper
that allocates the device workspace and output buffers as torch tensors and passes
their pointers and the current torch stream. Loading fails loudly if the library is not
built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LEDDS_OK = 0
LEDDS_ERR_CAPACITY, LEDDS_ERR_STATE = -2, -6
MAX_CAP = 64        # largest candidate and tile capacity of the library
ERRORS = {-1: "invalid argument", -2: "capacity exceeded", -3: "non-finite values detected",
          -4: "device wait timed out", -5: "CUDA runtime error", -6: "invalid state"}
STORE = {"f32": 0, "f16": 1, "bf16": 2}
VOXEL = {"distance": 0, "subdiv": 1}
LAW = {"linear": 0, "hertz": 1}
COLLIDE = {"bgk": 0, "trt": 1}
ORIENT = {"triad": 0, "quat": 1}
PATTERN = {"ab": 0, "aa": 1}
SPHERE, ELLIPSOID = 0, 1


class ledds_dims(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("periodic", C.c_int * 3), ("max_particles", C.c_int),
                ("cand_cap", C.c_int), ("tile_cap", C.c_int)]


class ledds_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("fluid_force", C.c_double * 3), ("storage", C.c_int),
                ("storage_scale_log2", C.c_int), ("voxel", C.c_int), ("subdiv_n", C.c_int),
                ("law", C.c_int), ("n_sub", C.c_int), ("rho_f", C.c_double),
                ("gravity", C.c_double * 3), ("k_n", C.c_double), ("k_t", C.c_double),
                ("young", C.c_double), ("poisson", C.c_double), ("restitution", C.c_double),
                ("friction", C.c_double), ("skin", C.c_double), ("dem_h", C.c_double),
                ("ell_max_iter", C.c_int), ("ell_tol", C.c_double),
                ("force_fp32", C.c_int), ("collision", C.c_int), ("orient", C.c_int),
                ("pattern", C.c_int), ("index64", C.c_int), ("psm_route", C.c_int),
                ("ell_screen", C.c_int)]


class ledds_particle(C.Structure):
    _fields_ = [("shape", C.c_int), ("radius", C.c_double), ("semi", C.c_double * 3),
                ("density", C.c_double), ("pos", C.c_double * 3), ("vel", C.c_double * 3),
                ("omg", C.c_double * 3), ("triad", C.c_double * 9)]


class ledds_status(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("tile_overflow", C.c_int), ("cand_overflow", C.c_int),
                ("solids_overflow", C.c_int), ("skin_violation", C.c_int),
                ("ell_nonconverged", C.c_int), ("nan_detected", C.c_int),
                ("n_particles", C.c_int), ("launches_per_step", C.c_int), ("wait_timeout", C.c_int),
                ("psm_staged", C.c_int)]


VP = C.c_void_p
_SIGS = {
    "ledds_version": (C.c_int, []),
    "ledds_strerror": (C.c_char_p, [C.c_int]),
    "ledds_params_default": (C.c_int, [C.POINTER(ledds_params)]),
    "ledds_workspace_size": (C.c_int, [C.POINTER(ledds_dims), C.POINTER(ledds_params), C.POINTER(C.c_size_t)]),
    "ledds_create": (C.c_int, [C.POINTER(ledds_dims), C.POINTER(ledds_params), VP, C.c_size_t, VP, C.POINTER(VP)]),
    "ledds_destroy": (C.c_int, [VP]),
    "ledds_set_wall_velocity": (C.c_int, [VP, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "ledds_set_forcing": (C.c_int, [VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ledds_init_fluid": (C.c_int, [VP, VP, VP]),
    "ledds_init_populations": (C.c_int, [VP, VP]),
    "ledds_set_particles": (C.c_int, [VP, C.c_int, C.POINTER(ledds_particle)]),
    "ledds_write_kinematics": (C.c_int, [VP, VP, C.c_int]),
    "ledds_step": (C.c_int, [VP, C.c_int]),
    "ledds_sync": (C.c_int, [VP]),
    "ledds_get_status": (C.c_int, [VP, C.POINTER(ledds_status)]),
    "ledds_read_fields": (C.c_int, [VP, VP, VP]),
    "ledds_read_populations": (C.c_int, [VP, VP, C.c_int]),
    "ledds_read_particles": (C.c_int, [VP, VP, C.c_int]),
    "ledds_read_forces": (C.c_int, [VP, VP, VP, VP, VP]),
    "ledds_read_pairs": (C.c_int, [VP, VP, C.c_int, C.POINTER(C.c_int)]),
    "ledds_read_cell_keys": (C.c_int, [VP, VP, VP, C.POINTER(C.c_int)]),
    "ledds_voxelize": (C.c_int, [VP, VP, VP, VP]),
    "ledds_set_profiling": (C.c_int, [VP, C.c_int]),
    "ledds_read_profile": (C.c_int, [VP, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "ledds_save": (C.c_int, [VP, VP, C.POINTER(C.c_size_t)]),
    "ledds_load": (C.c_int, [VP, VP, C.c_size_t]),
    "ledds_cell_list_noalloc": (C.c_int, [VP, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.c_double, VP, VP, C.POINTER(C.c_int), VP]),
    "ledds_batch_workspace_size": (C.c_int, [C.c_int, VP, VP, C.POINTER(C.c_size_t)]),
    "ledds_batch_create": (C.c_int, [C.c_int, VP, VP, VP, C.c_size_t, VP, C.POINTER(VP)]),
    "ledds_batch_sim": (C.c_int, [VP, C.c_int, C.POINTER(VP)]),
    "ledds_batch_step": (C.c_int, [VP, C.c_int]),
    "ledds_batch_destroy": (C.c_int, [VP]),
    "ledds_batch_configure": (C.c_int, [VP, C.c_int, C.c_int, C.c_int]),
    "ledds_batch_get_config": (C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ledds_batch_autotune": (C.c_int, [VP, C.c_int, C.POINTER(C.c_int)]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libledds.so (building it first if the sources are newer). Raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libledds.so is not built; run paper_2512_04997_gb300/build.py")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LeddsError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)} ({code})")
        self.code = code


def check(fn, code):
    if code != LEDDS_OK:
        raise LeddsError(fn, code)
    return code


def _dbl3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def make_params(**kw) -> ledds_params:
    """ledds_params from keyword values (strings accepted for storage, voxel and law)."""
    p = ledds_params()
    check("ledds_params_default", lib().ledds_params_default(C.byref(p)))
    for k, v in kw.items():
        if k == "storage":
            v = STORE[v] if isinstance(v, str) else v
        elif k == "voxel":
            v = VOXEL[v] if isinstance(v, str) else v
        elif k == "law":
            v = LAW[v] if isinstance(v, str) else v
        elif k == "collision":
            v = COLLIDE[v] if isinstance(v, str) else v
        elif k == "orient":
            v = ORIENT[v] if isinstance(v, str) else v
        elif k == "pattern":
            v = PATTERN[v] if isinstance(v, str) else v
        if k in ("fluid_force", "gravity"):
            getattr(p, k)[:] = [float(x) for x in v]
        else:
            setattr(p, k, v)
    return p


def make_dims(nx=0, ny=0, nz=0, periodic=(1, 1, 1), max_particles=0, box_lo=(0, 0, 0),
              box_hi=(1, 1, 1), cand_cap=0, tile_cap=0) -> ledds_dims:
    d = ledds_dims()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.box_lo[:] = [float(x) for x in box_lo]
    d.box_hi[:] = [float(x) for x in box_hi]
    d.periodic[:] = [int(x) for x in periodic]
    d.max_particles = int(max_particles)
    d.cand_cap = int(cand_cap)
    d.tile_cap = int(tile_cap)
    return d


def particles_array(shape, radius, semi, density, pos, vel=None, omg=None, triad=None):
    n = len(shape)
    arr = (ledds_particle * max(n, 1))()
    z3 = np.zeros((n, 3))
    vel = z3 if vel is None else np.asarray(vel, dtype=np.float64).reshape(n, 3)
    omg = z3 if omg is None else np.asarray(omg, dtype=np.float64).reshape(n, 3)
    tri = np.tile(np.eye(3).reshape(1, 9), (n, 1)) if triad is None else np.asarray(triad).reshape(n, 9)
    semi = np.asarray(semi, dtype=np.float64).reshape(n, 3)
    pos = np.asarray(pos, dtype=np.float64).reshape(n, 3)
    for k in range(n):
        q = arr[k]
        q.shape = int(shape[k])
        q.radius = float(radius[k])
        q.semi[:] = semi[k].tolist()
        q.density = float(density[k])
        q.pos[:] = pos[k].tolist()
        q.vel[:] = vel[k].tolist()
        q.omg[:] = omg[k].tolist()
        q.triad[:] = tri[k].tolist()
    return arr


class Sim:
    """A simulation whose workspace is a torch uint8 tensor on ``device``."""

    @classmethod
    def _member(cls, handle, dims, params, device, stream, owner):
        obj = cls.__new__(cls)
        import torch
        obj.torch = torch
        obj.device = torch.device(device)
        obj.dims, obj.params = dims, params
        obj.stream = stream
        obj.h = handle
        obj.ncell = dims.nx * dims.ny * dims.nz
        obj.n = 0
        obj._owner = owner          # the batch keeps the workspace alive
        return obj

    def __init__(self, dims: ledds_dims, params: ledds_params, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        L = lib()
        self.dims, self.params = dims, params
        nbytes = C.c_size_t(0)
        check("ledds_workspace_size", L.ledds_workspace_size(C.byref(dims), C.byref(params), C.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = VP()
        check("ledds_create", L.ledds_create(C.byref(dims), C.byref(params), self.workspace.data_ptr(),
                                             nbytes.value, VP(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.ncell = dims.nx * dims.ny * dims.nz
        self.n = 0

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self.h = None           # members are released by their batch
            return
        if getattr(self, "h", None):
            lib().ledds_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # configuration ------------------------------------------------------------------
    def set_wall_velocity(self, axis, side, u):
        check("ledds_set_wall_velocity", lib().ledds_set_wall_velocity(self.h, axis, side, _dbl3(u)))

    def set_forcing(self, gravity=None, fluid_force=None):
        check("ledds_set_forcing", lib().ledds_set_forcing(
            self.h, None if gravity is None else _dbl3(gravity), None if fluid_force is None else _dbl3(fluid_force)))

    def init_fluid(self, rho=None, u=None):
        t = self.torch
        r = None if rho is None else t.as_tensor(np.asarray(rho, dtype=np.float32), device=self.device).contiguous()
        v = None if u is None else t.as_tensor(np.asarray(u, dtype=np.float32), device=self.device).contiguous()
        check("ledds_init_fluid", lib().ledds_init_fluid(self.h, None if r is None else r.data_ptr(),
                                                         None if v is None else v.data_ptr()))
        self.sync()

    def init_populations(self, f):
        f = self.torch.as_tensor(np.asarray(f, dtype=np.float32), device=self.device).contiguous()
        check("ledds_init_populations", lib().ledds_init_populations(self.h, f.data_ptr()))
        self.sync()

    def set_particles(self, shape, radius, semi, density, pos, vel=None, omg=None, triad=None):
        arr = particles_array(shape, radius, semi, density, pos, vel, omg, triad)
        check("ledds_set_particles", lib().ledds_set_particles(self.h, len(shape), arr))
        self.n = len(shape)

    def write_kinematics(self, state, on_device=None):
        if on_device is None:
            on_device = hasattr(state, "data_ptr") and state.is_cuda
        ptr = state.data_ptr() if hasattr(state, "data_ptr") else state.ctypes.data
        check("ledds_write_kinematics", lib().ledds_write_kinematics(self.h, ptr, int(bool(on_device))))

    # stepping -----------------------------------------------------------------------
    def step(self, n=1, regrow=False, chunk=100):
        """Advance n fluid steps (asynchronous). With regrow, the steps run in chunks of
        `chunk`, each after a checkpoint; a chunk that overflows the candidate or tile
        capacity is replayed from that checkpoint in a simulation with doubled capacities
        (up to the library's maximum, 64), which then replaces this one's handle and
        workspace. LeddsError(CAPACITY) if the maximum does not suffice."""
        if not regrow:
            check("ledds_step", lib().ledds_step(self.h, int(n)))
            return
        if getattr(self, "_owner", None) is not None:
            raise LeddsError("ledds_step", LEDDS_ERR_STATE)   # batch members cannot be replaced
        left = int(n)
        while left > 0:
            k = min(left, int(chunk))
            snap = self.save()
            check("ledds_step", lib().ledds_step(self.h, k))
            st = self.status()
            while st["tile_overflow"] or st["cand_overflow"]:
                self._regrow(snap, st["tile_overflow"] > 0, st["cand_overflow"] > 0)
                check("ledds_step", lib().ledds_step(self.h, k))
                st = self.status()
            left -= k

    def _regrow(self, snap, tiles, cands):
        """Replace this simulation by one with doubled tile and/or candidate capacity,
        loaded from checkpoint `snap` (taken with the current, smaller capacities)."""
        d = ledds_dims()
        C.memmove(C.byref(d), C.byref(self.dims), C.sizeof(d))
        cur_t = d.tile_cap if d.tile_cap > 0 else 64
        cur_c = d.cand_cap if d.cand_cap > 0 else 32
        if (tiles and cur_t >= MAX_CAP) or (cands and cur_c >= MAX_CAP):
            raise LeddsError("ledds_step", LEDDS_ERR_CAPACITY)
        if tiles:
            d.tile_cap = min(MAX_CAP, 2 * cur_t)
        if cands:
            d.cand_cap = min(MAX_CAP, 2 * cur_c)
        new = Sim(d, self.params, self.device, self.stream)
        new.load(snap)
        new.n = self.n
        lib().ledds_destroy(self.h)
        self.h, self.workspace, self.dims = new.h, new.workspace, new.dims
        new.h = None

    def sync(self):
        check("ledds_sync", lib().ledds_sync(self.h))

    def status(self, raise_on_error=False):
        st = ledds_status()
        rc = lib().ledds_get_status(self.h, C.byref(st))
        if raise_on_error:
            check("ledds_get_status", rc)
        return {f: getattr(st, f) for f, _ in ledds_status._fields_} | {"rc": rc}

    # outputs ------------------------------------------------------------------------
    def fields(self):
        t = self.torch
        rho = t.empty(self.ncell, dtype=t.float32, device=self.device)
        u = t.empty(3 * self.ncell, dtype=t.float32, device=self.device)
        check("ledds_read_fields", lib().ledds_read_fields(self.h, rho.data_ptr(), u.data_ptr()))
        self.sync()
        return rho, u.view(3, self.ncell)

    def populations(self, which=0):
        t = self.torch
        f = t.empty(19 * self.ncell, dtype=t.float32, device=self.device)
        check("ledds_read_populations", lib().ledds_read_populations(self.h, f.data_ptr(), int(which)))
        self.sync()
        return f.view(19, self.ncell)

    def particles(self):
        out = np.zeros(18 * max(self.n, 1))
        check("ledds_read_particles", lib().ledds_read_particles(self.h, out.ctypes.data, 0))
        st = out[: 18 * self.n].reshape(18, self.n)
        return st[0:3].T.copy(), st[3:6].T.copy(), st[6:9].T.copy(), st[9:18].T.copy()

    def forces(self):
        t = self.torch
        bufs = [t.zeros(3 * max(self.n, 1), dtype=t.float64, device=self.device) for _ in range(4)]
        check("ledds_read_forces", lib().ledds_read_forces(self.h, *[b.data_ptr() for b in bufs]))
        self.sync()
        return tuple(b[: 3 * self.n].view(3, self.n).T.cpu().numpy() for b in bufs)

    def pairs(self):
        t = self.torch
        cap = max(16, 16 * self.n)
        while True:
            keys = t.zeros(cap, dtype=t.int64, device=self.device)
            n = C.c_int(0)
            check("ledds_read_pairs", lib().ledds_read_pairs(self.h, keys.data_ptr(), cap, C.byref(n)))
            if n.value <= cap:
                return keys[: n.value].cpu().numpy()
            cap = n.value

    def cell_keys(self):
        t = self.torch
        k = t.zeros(max(self.n, 1), dtype=t.int32, device=self.device)
        ids = t.zeros(max(self.n, 1), dtype=t.int32, device=self.device)
        g = (C.c_int * 3)()
        check("ledds_read_cell_keys", lib().ledds_read_cell_keys(self.h, k.data_ptr(), ids.data_ptr(), g))
        return (k[: self.n].cpu().numpy().view(np.uint32), ids[: self.n].cpu().numpy(), tuple(g))

    def voxelize(self):
        t = self.torch
        beta = t.zeros(2 * self.ncell, dtype=t.float32, device=self.device)
        ids = t.zeros(2 * self.ncell, dtype=t.int32, device=self.device)
        ns = t.zeros(self.ncell, dtype=t.int32, device=self.device)
        check("ledds_voxelize", lib().ledds_voxelize(self.h, beta.data_ptr(), ids.data_ptr(), ns.data_ptr()))
        self.sync()
        return beta.view(self.ncell, 2), ids.view(self.ncell, 2), ns

    def set_profiling(self, on=True):
        check("ledds_set_profiling", lib().ledds_set_profiling(self.h, int(bool(on))))

    def read_profile(self):
        ms = (C.c_double * 5)()
        steps = C.c_longlong(0)
        launches = C.c_longlong(0)
        check("ledds_read_profile", lib().ledds_read_profile(self.h, ms, C.byref(steps), C.byref(launches)))
        return list(ms), steps.value, launches.value

    def save(self) -> bytes:
        n = C.c_size_t(0)
        check("ledds_save", lib().ledds_save(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        check("ledds_save", lib().ledds_save(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def load(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        check("ledds_load", lib().ledds_load(self.h, buf, len(data)))


def from_workload(w, device="cuda:0", **over) -> Sim:
    """Create a simulation of a ``workloads.Workload`` (fluid initial state and particles)."""
    prm = dict(w.params)
    prm.update(over)
    keys = {f for f, _ in ledds_params._fields_}
    p = make_params(**{k: v for k, v in prm.items() if k in keys})
    d = make_dims(w.nx, w.ny, w.nz, w.periodic, w.n, w.box_lo, w.box_hi,
                  cand_cap=prm.get("cand_cap", 0), tile_cap=prm.get("tile_cap", 0))
    s = Sim(d, p, device)
    for a in range(3):
        if not w.periodic[a]:
            for side in range(2):
                s.set_wall_velocity(a, side, w.u_wall[a, side])
    if w.ncell and w.init_u is not None:
        s.init_fluid(None, w.init_u)
    if w.n:
        s.set_particles(w.shape, w.radius, w.semi, w.density, w.pos, w.vel, w.omg, w.triad)
    return s


class Batch:
    """Many simulations advanced together (ledds_batch_*); members are ``Sim`` objects."""

    def __init__(self, dims_list, params_list, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        L = lib()
        n = len(dims_list)
        self.dims = (ledds_dims * n)(*dims_list)
        self.params = (ledds_params * n)(*params_list)
        nbytes = C.c_size_t(0)
        check("ledds_batch_workspace_size", L.ledds_batch_workspace_size(n, self.dims, self.params, C.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=torch.device(device))
        self.stream = stream if stream is not None else torch.cuda.current_stream(torch.device(device))
        h = VP()
        check("ledds_batch_create", L.ledds_batch_create(n, self.dims, self.params, self.workspace.data_ptr(),
                                                         nbytes.value, VP(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.members = []
        for i in range(n):
            mh = VP()
            check("ledds_batch_sim", L.ledds_batch_sim(h, i, C.byref(mh)))
            self.members.append(Sim._member(mh, dims_list[i], params_list[i], device, self.stream, self))

    def step(self, n=1):
        check("ledds_batch_step", lib().ledds_batch_step(self.h, int(n)))

    def sync(self):
        self.torch.cuda.synchronize()

    def configure(self, tile_depth=16, ctas_per_sm=None, order=0):
        if ctas_per_sm is None:
            ctas_per_sm = self.config()["ctas_per_sm"]
        check("ledds_batch_configure", lib().ledds_batch_configure(self.h, int(tile_depth), int(ctas_per_sm),
                                                                   int(order)))

    def config(self):
        d, c, o = C.c_int(0), C.c_int(0), C.c_int(0)
        check("ledds_batch_get_config", lib().ledds_batch_get_config(self.h, C.byref(d), C.byref(c), C.byref(o)))
        return {"tile_depth": d.value, "ctas_per_sm": c.value, "order": o.value}

    def autotune(self, steps_per_trial=4):
        """Choose the persistent launch shape and work order by timing (advances the members)."""
        c = C.c_int(-1)
        check("ledds_batch_autotune", lib().ledds_batch_autotune(self.h, int(steps_per_trial), C.byref(c)))
        return c.value

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None          # member handles die with the batch
            lib().ledds_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_from_workloads(ws, device="cuda:0", **over):
    """A batch whose members are the given workloads (fluid initial state and particles)."""
    keys = {f for f, _ in ledds_params._fields_}
    dims, params = [], []
    for w in ws:
        prm = dict(w.params)
        prm.update(over)
        params.append(make_params(**{k: v for k, v in prm.items() if k in keys}))
        dims.append(make_dims(w.nx, w.ny, w.nz, w.periodic, w.n, w.box_lo, w.box_hi,
                              cand_cap=prm.get("cand_cap", 0), tile_cap=prm.get("tile_cap", 0)))
    b = Batch(dims, params, device)
    for w, s in zip(ws, b.members):
        for a in range(3):
            if not w.periodic[a]:
                for side in range(2):
                    s.set_wall_velocity(a, side, w.u_wall[a, side])
        if w.init_u is not None:
            s.init_fluid(None, w.init_u)
        if w.n:
            s.set_particles(w.shape, w.radius, w.semi, w.density, w.pos, w.vel, w.omg, w.triad)
    return b
