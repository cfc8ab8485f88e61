"""Longer GPU parity runs and checkpoint resume: a c3-shaped 64^3 crop in the default mode
(50-step trajectories and 1000-step statistics), the particle-free crop at 1000 steps, the
reduced-precision bounds (fields 2e-3, drag 0.5 %) on the settling sphere and on crops
of the two benchmark workloads against the oracle, the rheology workload on a 48^3 crop,
and bit-identical resume from a checkpoint."""
import math

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


def _profiles(w, u, pos):
    """Mean streamwise velocity per z-layer, and the solid fraction per 8-layer slab: each
    sphere's volume split exactly between the slabs its extent crosses (a smooth function
    of the centres, so nearby trajectories give nearby profiles)."""
    ux = np.asarray(u)[0].reshape(w.nz, w.ny, w.nx).mean(axis=(1, 2))
    edges = np.arange(0, w.nz + 8, 8) - 0.5
    R = w.radius[:, None]
    zc = pos[:, 2][:, None]

    def cap(zz):   # volume of the sphere below height zz
        t = np.clip(zz - zc, -R, R)
        return math.pi * (R ** 2 * t - t ** 3 / 3.0 + 2.0 * R ** 3 / 3.0)

    vol = cap(edges[None, 1:]) - cap(edges[None, :-1])
    phi = vol.sum(0) / (8.0 * w.nx * w.ny)
    return ux, phi


def test_couette_crop_1000_steps(oracle):
    """The Couette suspension shrunk to 64^3 (62 spheres R 6, same solid fraction, walls at
    -/+0.05, n_sub 10), in the product's default mode (FP32 storage, FP32 contact
    arithmetic), against the FP64 oracle. The sheared suspension is chaotic: FP32 and FP64
    particle trajectories part exponentially, and the field difference follows them. So,
    as the tolerance definitions for many-body runs state: (iii) fields and trajectories
    after 50 steps within 1e-5, and (iv) statistics over 1000 steps: the mean velocity
    profile within 1e-4 of its maximum, the solid-fraction profile (8-layer bins) within
    1e-3, and the particles' kinetic energy within 1e-3. The pointwise field difference at
    1000 steps is printed as a diagnostic."""
    w = W.couette_suspension(nx=64, ny=64, nz=64, n_particles=62, steps=1000)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(50)
    s.step(50)
    _, u_o = o.moments()
    _, u_g = s.fields()
    po, vo, _, _ = o.particles()
    pg, vg, _, _ = s.particles()
    e50 = normwise(u_g.cpu().numpy(), u_o)
    assert e50 < 1e-5, e50
    assert normwise(vg, vo) < 1e-5
    assert np.abs(pg - po).max() < 1e-5
    ux_sum_o = ux_sum_g = 0.0
    phi_o = phi_g = 0.0
    ke = []
    for _ in range(19):                 # steps 50 .. 1000, statistics sampled every 50 steps
        o.step(50)
        s.step(50)
        _, u_o = o.moments()
        _, u_g = s.fields()
        po, vo, _, _ = o.particles()
        pg, vg, _, _ = s.particles()
        a, b = _profiles(w, u_o, po)
        c, d = _profiles(w, u_g.cpu().numpy(), pg)
        ux_sum_o, phi_o = ux_sum_o + a, phi_o + b
        ux_sum_g, phi_g = ux_sum_g + c, phi_g + d
        m = w.density * 4.0 / 3.0 * math.pi * w.radius ** 3
        ke.append((0.5 * (m[:, None] * vo ** 2).sum(), 0.5 * (m[:, None] * vg ** 2).sum()))
    prof = np.abs(ux_sum_g - ux_sum_o).max() / np.abs(ux_sum_o).max()
    phid = np.abs(phi_g - phi_o).max() / 19.0
    ke = np.array(ke)
    ked = np.abs(ke[:, 1] - ke[:, 0]).max() / ke[:, 0].max()
    e1000 = normwise(u_g.cpu().numpy(), u_o)
    print(f"fields at 50 steps {e50:.2e}; over 1000 steps: mean profile {prof:.2e}, "
          f"solid-fraction profile {phid:.2e}, kinetic energy {ked:.2e}; "
          f"pointwise field difference at 1000 steps {e1000:.2e} (diagnostic)")
    assert prof < 1e-4, prof
    assert phid < 1e-3, phid
    assert ked < 1e-3, ked
    st = s.status()
    assert st["rc"] == 0 and st["skin_violation"] == 0 and st["nan_detected"] == 0, st


def test_couette_lattice_1000_steps(oracle):
    """The same 64^3 box without particles, started from rest: after 1000 steps the FP32
    velocity field is within 1e-5 of the FP64 oracle."""
    w = W.couette_suspension(nx=64, ny=64, nz=64, n_particles=0, steps=1000)
    w.init_u = None
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(w.steps)
    s.step(w.steps)
    _, u_o = o.moments()
    _, u_g = s.fields()
    assert normwise(u_g.cpu().numpy(), u_o) < 1e-5


@pytest.mark.parametrize("storage", [
    "f16",
    pytest.param("bf16", marks=pytest.mark.xfail(
        reason="BF16 keeps 8 significand bits; its measured field error is above 2e-3 "
               "(the bound is not loosened)", strict=False)),
])
def test_settling_sphere_reduced_precision(oracle, storage):
    """16-bit storage of f_i - t_i on the settling sphere (500 steps): fields within 2e-3 of
    the FP64 oracle and the hydrodynamic drag within 0.5 %."""
    w = W.settling_sphere(steps=500)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w, storage=storage)
    o.step(w.steps)
    s.step(w.steps)
    _, u_o = o.moments()
    _, u_g = s.fields()
    err_u = normwise(u_g.cpu().numpy(), u_o)
    Fh_o = o.forces()[0][0]
    Fh_g = s.forces()[0][0]
    drag_err = abs(Fh_g[2] - Fh_o[2]) / abs(Fh_o[2])
    print(f"{storage}: field error {err_u:.3e}, drag error {drag_err:.3e}")
    assert err_u < 2e-3, err_u
    assert drag_err < 5e-3, drag_err


@pytest.mark.parametrize("storage", [
    "f16",
    pytest.param("bf16", marks=pytest.mark.xfail(
        reason="BF16 keeps 8 significand bits; its field error against the FP64 oracle is above "
               "2e-3 (the bound is not loosened)", strict=False)),
])
@pytest.mark.parametrize("case", ["couette_crop", "ellipsoid_crop"])
def test_reduced_precision_crops_vs_oracle(oracle, storage, case):
    """16-bit population storage against the FP64 oracle (not against FP32) on crops of the
    two benchmark workloads: the 256^3 Couette suspension shrunk to 64^3 (62 spheres, 100
    steps) and the sheared ellipsoid suspension shrunk to 48x48x32 (its density of (6, 2, 2)
    ellipsoids, subdivision fractions, 20 steps: the oracle counts every sample). Fields
    within 2e-3; the FP32 run's error is printed beside it."""
    if case == "couette_crop":
        w = W.couette_suspension(nx=64, ny=64, nz=64, n_particles=62, storage=storage)
        steps = 100
    else:
        w = W.ellipsoid_shear(nx=48, ny=48, nz=32, n_particles=52, storage=storage)
        steps = 20
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    r = gpu_from_workload(w, storage="f32")
    o.step(steps)
    s.step(steps)
    r.step(steps)
    _, u_o = o.moments()
    e16 = normwise(s.fields()[1].cpu().numpy(), u_o)
    e32 = normwise(r.fields()[1].cpu().numpy(), u_o)
    print(f"{case} {storage}: field error against the oracle {e16:.2e} (FP32 storage {e32:.2e})")
    assert e32 < 1e-5
    assert e16 < 2e-3, e16


def test_rheology_crop_vs_oracle(oracle):
    """The rheology workload (spheres of diameter 10, walls at -/+0.05, solid fraction 0.2,
    friction 0.45, restitution 0.95, n_sub 10) on a 48^3 crop for 300 steps against the
    oracle: fields, particle velocities, the mean velocity profile and the wall shear rate
    the viscosity estimate uses."""
    w = W.rheology_suspension(0.2, n=48)
    o = oracle_from_workload(oracle, w)
    s = gpu_from_workload(w)
    o.step(300)
    s.step(300)
    _, u_o = o.moments()
    _, u_g = s.fields()
    u_g = u_g.cpu().numpy()
    assert normwise(u_g, u_o) < 1e-5
    _, vo, _, _ = o.particles()
    _, vg, _, _ = s.particles()
    assert normwise(vg, vo) < 1e-5
    # the wall shear rate is a short difference of near-wall mean velocities (about 0.05)
    # that cancels to about 0.003: its error is bounded against the size of the terms it
    # differences, not against its own value
    n, U = w.nz, w.u_wall[2, 1, 0]
    po = np.asarray(u_o)[0].reshape(n, -1).mean(1)
    pg = u_g[0].reshape(n, -1).mean(1)
    assert normwise(pg, po) < 1e-5
    go, gg = W.wall_shear_rate(po, U), W.wall_shear_rate(pg, U)
    scale = 0.5 * (3.0 * abs(po[0]) + abs(po[1]) / 3.0 + 3.0 * abs(po[-1]) + abs(po[-2]) / 3.0)
    print(f"wall shear rate {gg:.6e} against {go:.6e} (terms {scale:.3e})")
    assert abs(gg - go) < 1e-5 * scale, (gg, go, scale)
    assert w.n > 30


def _resume_case(w, steps_a, steps_b):
    a = gpu_from_workload(w)
    a.step(steps_a)
    blob = a.save()
    a.step(steps_b)
    b = gpu_from_workload(w)
    b.load(blob)
    b.step(steps_b)
    return a, b


def test_checkpoint_resume_lattice_bitwise():
    """Lattice with moving walls: save after 7 steps, resume in a fresh simulation, 9 more
    steps: populations identical bit for bit (odd counts exercise both buffer parities)."""
    w = W.Workload(name="lattice", nx=40, ny=12, nz=20, periodic=(1, 1, 0))
    w.params = W.base_params(tau=0.7)
    w.u_wall[2, 1] = [0.04, 0.0, 0.0]
    a, b = _resume_case(w, 7, 9)
    assert np.array_equal(a.populations().cpu().numpy(), b.populations().cpu().numpy())


def test_checkpoint_resume_dem_bitwise():
    """DEM only (contact histories in flight): resume gives identical particle states."""
    w = W.granular_box(n_particles=2000, box=(36.0, 36.0, 48.0), seed_index=2)
    g = W.rng(600 + 2)
    w.vel = g.normal(0, 0.02, (w.n, 3))
    w.params.update(gravity=(0, 0, -1e-4))
    a, b = _resume_case(w, 13, 11)
    for x, y in zip(a.particles(), b.particles()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.pairs(), b.pairs())


def test_checkpoint_resume_coupled():
    """Coupled step: resume agrees to FP64 accumulation-order rounding (hydrodynamic sums use
    atomics, whose order varies between runs)."""
    w = W.couette_suspension(nx=48, ny=32, nz=32, n_particles=12, steps=20)
    a, b = _resume_case(w, 5, 6)
    _, ua = a.fields()
    _, ub = b.fields()
    assert normwise(ub.cpu().numpy(), ua.cpu().numpy()) < 1e-6
    pa, va, _, _ = a.particles()
    pb, vb, _, _ = b.particles()
    assert np.abs(pa - pb).max() < 1e-7


def _eta_rel(w, steps=8000, every=250):
    from paper_2512_04997_gb300 import ledds
    torch = pytest.importorskip("torch")
    n, U = w.nz, w.u_wall[2, 1, 0]
    s = ledds.from_workload(w)
    s.step(steps // 2)
    prof = torch.zeros(n, dtype=torch.float64, device="cuda")
    k = 0
    for _ in range(steps // 2 // every):
        s.step(every)
        _, u = s.fields()
        prof += u[0].view(n, -1).double().mean(1)
        k += 1
    return W.wall_shear_rate((prof / k).cpu().numpy(), U) / (2.0 * U / n)


def test_effective_viscosity_method():
    """The wall-stress estimate of the effective viscosity (Sec. 4.8): exactly 1 for the
    particle-free sheared box (a linear profile), and above 1, of the order of the
    Krieger-Dougherty value (1.31), at solid fraction 0.1 on a short run."""
    w0 = W.rheology_suspension(0.0, n=64)
    assert abs(_eta_rel(w0, steps=2000) - 1.0) < 1e-3
    w1 = W.rheology_suspension(0.1, n=64)
    eta = _eta_rel(w1, steps=8000)
    print(f"eta/eta0 at phi 0.1 (64^3, 8000 steps): {eta:.3f}")
    assert 1.05 < eta < 1.8, eta


def test_jeffery_orbit_period():
    """A prolate ellipsoid (a = 12, b = 6: 12 cells across the minor axis) in shear: the
    major axis turns by pi in pi (a^2 + b^2)/(a b shear_rate) (Jeffery); within 5 %. The
    time is taken between the crossings of the flow direction (angle 0 and pi), where the
    rotation is slowest and the crossing time sharpest."""
    from paper_2512_04997_gb300 import ledds
    a, b = 12.0, 6.0
    w = W.jeffery_ellipsoid(a, b, angle=0.3)
    s = ledds.from_workload(w)
    shear = 2.0 * 0.05 / w.nz
    T = math.pi * (a * a + b * b) / (a * b * shear)
    every = 20
    angles, times = [], []
    prev = None
    turn = 0.0
    for k in range(int(1.6 * T / every)):
        s.step(every)
        d1 = s.particles()[3][0][:3]
        ang = math.atan2(d1[2], d1[0])          # angle of the major axis in the x-z plane
        if prev is not None:
            da = ang - prev
            da -= math.pi * round(da / math.pi)  # the axis is a line: unwrap modulo pi
            turn += da
        prev = ang
        angles.append(turn)
        times.append((k + 1) * every)
    angles = np.array(angles)
    times = np.array(times)
    sense = np.sign(angles[-1])
    psi = np.maximum.accumulate(np.abs(angles))   # angle turned so far
    # the axis starts 0.3 rad from the flow direction and crosses it (slowest rotation)
    # after turning 0.3 (clockwise seen along +y) or pi - 0.3, and again pi later
    first = 0.3 if sense < 0 else math.pi - 0.3
    t1 = np.interp(first, psi, times)
    t2 = np.interp(first + math.pi, psi, times)
    assert psi[-1] > first + math.pi, psi[-1]
    T_meas = t2 - t1
    print(f"Jeffery half period: measured {T_meas:.0f} steps, theory {T:.0f}")
    assert abs(T_meas / T - 1.0) < 0.05, (T_meas, T)
    st = s.status()
    assert st["rc"] == 0 and st["nan_detected"] == 0, st


def test_capacity_regrow_and_replay():
    """Too small candidate and tile capacities: stepping with regrow replays every chunk that
    overflowed from its checkpoint in a simulation with doubled capacities, and ends where a
    simulation created with ample capacities ends (to the accumulation-order rounding of
    the hydrodynamic sums), with no overflow left in its counters."""
    w = W.couette_suspension(nx=64, ny=64, nz=64, n_particles=62, steps=40)
    w.params["tile_cap"] = 4        # a 32x8x16 tile meets more spheres than that
    w.params["cand_cap"] = 2        # and a sphere more candidates
    ref = gpu_from_workload(w, tile_cap=64, cand_cap=32)
    s = gpu_from_workload(w)
    assert (s.dims.tile_cap, s.dims.cand_cap) == (4, 2)
    ref.step(30)
    s.step(30, regrow=True, chunk=10)
    st = s.status()
    assert st["rc"] == 0 and st["tile_overflow"] == 0 and st["cand_overflow"] == 0, st
    assert s.dims.tile_cap > 4 and s.dims.cand_cap > 2
    _, ur = ref.fields()
    _, us = s.fields()
    assert normwise(us.cpu().numpy(), ur.cpu().numpy()) < 1e-6
    pr, vr, _, _ = ref.particles()
    ps, vs, _, _ = s.particles()
    assert np.abs(ps - pr).max() < 1e-7
    assert normwise(vs, vr) < 1e-6
    # without regrow the same capacities overflow
    t = gpu_from_workload(w)
    t.step(10)
    assert t.status()["tile_overflow"] > 0
