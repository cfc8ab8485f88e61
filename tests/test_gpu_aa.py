"""The in-place AA pattern (one population array, alternating in-place and streaming
steps) against the two-lattice pull and the oracle. Per node the arithmetic of the two
patterns is the same, so with FP32 storage their populations and fields agree bit for bit
after any number of steps. Rounding differences remain only where a moving-wall term is
added and taken off again: the two-lattice initialisation stores f - term so that the
first pull returns f (to rounding) where the AA pattern stores f itself; the AA read-back
of the last post-collision values across a wall; and 16-bit storage, where the AA pattern
rounds f* plus the wall term and the pull rounds f* alone."""
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


# 37 x 19 x 11: ragged tiles in x, y and z, odd nx (16-bit values share words across
# rows); 104 x 19 x 11: even nx, three full x-tiles and a ragged one.
SIZES = [(37, 19, 11), (104, 19, 11)]


def _lattice(periodic, walls, size=(37, 19, 11), **kw):
    nx, ny, nz = size
    w = W.Workload(name="lattice", nx=nx, ny=ny, nz=nz, periodic=periodic)
    w.params = W.base_params(tau=0.7, **kw)
    if walls == "z":
        w.u_wall[2, 0] = [-0.03, 0.01, 0.0]
        w.u_wall[2, 1] = [0.04, 0.0, 0.0]
    elif walls == "all":   # walls on every face; three of them move
        w.u_wall[0, 1] = [0.0, 0.02, -0.01]
        w.u_wall[1, 0] = [0.01, 0.0, 0.015]
        w.u_wall[2, 1] = [0.05, -0.02, 0.0]
    return w


def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("collision", ["bgk", "trt"])
@pytest.mark.parametrize("periodic,walls", [((1, 1, 1), None), ((0, 0, 0), "resting"), ((1, 1, 0), "z"),
                                            ((0, 0, 0), "all")])
def test_aa_lattice_matches_ab_and_oracle(oracle, periodic, walls, collision, size):
    """Lattice only (forced, off-equilibrium start): bit-exact without moving walls (periodic
    box; resting walls on every face); with moving walls the patterns start one rounding
    apart at the wall links and stay within a few units in the last place."""
    g = W.rng(510)
    w = _lattice(periodic, walls, size, collision=collision, fluid_force=(2e-6, -1e-6, 0.0))
    f0 = random_populations(oracle, g, w.nx, w.ny, w.nz)
    o = oracle_from_workload(oracle, w, populations=f0)
    ab = gpu_from_workload(w, populations=f0)
    aa = gpu_from_workload(w, populations=f0, pattern="aa")
    assert np.array_equal(_np(aa.populations()), _np(ab.populations()))
    done = 0
    for n in (1, 1, 5, 6):          # odd and even totals: 1, 2, 7, 13
        o.step(n)
        ab.step(n)
        aa.step(n)
        done += n
        f_ab, f_aa = _np(ab.populations()), _np(aa.populations())
        r_ab, u_ab = ab.fields()
        r_aa, u_aa = aa.fields()
        s_ab, s_aa = _np(ab.populations(1)), _np(aa.populations(1))
        if walls in (None, "resting"):
            assert np.array_equal(f_aa, f_ab), (done, np.abs(f_aa - f_ab).max())
            assert np.array_equal(_np(r_aa), _np(r_ab)) and np.array_equal(_np(u_aa), _np(u_ab))
            assert np.array_equal(s_aa, s_ab)
        else:
            assert np.abs(f_aa - f_ab).max() < 2e-7, (done, np.abs(f_aa - f_ab).max())
            assert normwise(_np(u_aa), _np(u_ab)) < 1e-6
            assert np.abs(s_aa - s_ab).max() < 2e-7
        assert np.abs(f_aa - o.populations()).max() < 2e-7
    _, u_o = o.moments()
    assert normwise(_np(u_aa), u_o) < FP32_TOL


@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_aa_16bit_storage(oracle, storage, size):
    """16-bit storage: bit-exact without walls; with walls the AA pattern rounds f* plus the
    wall term where the pull rounds f* alone, a difference of one rounding of the format."""
    g = W.rng(511)
    for periodic, walls, tol in (((1, 1, 1), None, 0.0), ((0, 0, 0), "all", 2e-3 if storage == "bf16" else 2e-4)):
        w = _lattice(periodic, walls, size, storage=storage)
        f0 = random_populations(oracle, g, w.nx, w.ny, w.nz)
        ab = gpu_from_workload(w, populations=f0)
        aa = gpu_from_workload(w, populations=f0, pattern="aa")
        for n in (3, 4):
            ab.step(n)
            aa.step(n)
            d = np.abs(_np(aa.populations()) - _np(ab.populations())).max()
            assert d <= tol, (walls, n, d)


def _coupled(seed=520):
    w = W.couette_suspension(nx=104, ny=48, nz=40, n_particles=64, radius=4.0, seed_index=seed)
    return w


def test_aa_coupled_matches_ab_and_oracle(oracle):
    """Particles in a sheared box between moving walls: the patterns start one rounding apart
    at the wall links and the force sums use atomics (order-dependent rounding), so they
    agree to rounding: fields 1e-6; the hydrodynamic forces, sums over a particle's surface
    nodes with strong cancellation, within twice the oracle parity tolerance of the coupled
    tests (each pattern is within 1e-4 of the oracle, so the two within 2e-4; measured
    1.05e-4 on this machine), and through them velocities 1e-5 and positions 1e-7 (measured
    3e-9 after 11 steps). Both against the oracle at the parity tolerances."""
    w = _coupled()
    o = oracle_from_workload(oracle, w)
    ab = gpu_from_workload(w)
    aa = gpu_from_workload(w, pattern="aa")
    for n in (5, 6):
        o.step(n)
        ab.step(n)
        aa.step(n)
        _, u_ab = ab.fields()
        _, u_aa = aa.fields()
        assert normwise(_np(u_aa), _np(u_ab)) < 1e-6
        p_ab, v_ab, _, _ = ab.particles()
        p_aa, v_aa, _, _ = aa.particles()
        assert np.abs(p_aa - p_ab).max() < 1e-7
        assert normwise(v_aa, v_ab) < FP32_TOL
        Fh_ab = ab.forces()[0]
        Fh_aa = aa.forces()[0]
        assert normwise(Fh_aa, Fh_ab) < 2e-4
    _, u_o = o.moments()
    assert normwise(_np(u_aa), u_o) < FP32_TOL
    po, vo, _, _ = o.particles()
    assert np.abs(p_aa - po).max() < 1e-6
    assert normwise(v_aa, vo) < FP32_TOL
    assert normwise(Fh_aa, o.forces()[0]) < 1e-4
    assert aa.status()["rc"] == 0


def test_aa_checkpoint_rebase_and_reinit(oracle):
    """Host operations at both array states of the AA pattern: a checkpoint taken after an
    odd step count resumes bit for bit; re-initialising the populations after an odd count
    matches the two-lattice pull; a wall velocity change at either state keeps the current
    populations (to rounding of the pull's rebase)."""
    g = W.rng(512)
    w = _lattice((1, 1, 0), "z")
    f0 = random_populations(oracle, g, w.nx, w.ny, w.nz)
    f1 = random_populations(oracle, g, w.nx, w.ny, w.nz)
    aa = gpu_from_workload(w, populations=f0, pattern="aa")
    ab = gpu_from_workload(w, populations=f0)
    aa.step(3)
    ab.step(3)
    blob = aa.save()
    aa.step(4)
    ref = _np(aa.populations())
    aa.load(blob)
    aa.step(4)
    assert np.array_equal(_np(aa.populations()), ref)
    # re-initialise at the post-collision state (odd count), then step on
    for s in (aa, ab):
        s.init_populations(f1)
    assert np.array_equal(_np(aa.populations()), _np(ab.populations()))
    aa.step(1)
    ab.step(1)
    assert np.array_equal(_np(aa.populations()), _np(ab.populations()))
    # wall velocity changes at the natural state (even count) and the post-collision state
    for k in range(2):
        for s in (aa, ab):
            before = _np(s.populations())
            s.set_wall_velocity(2, 1, [0.02 * (k + 1), 0.01, 0.0])
            assert np.abs(_np(s.populations()) - before).max() < 1e-7
        aa.step(3)
        ab.step(3)
        assert np.abs(_np(aa.populations()) - _np(ab.populations())).max() < 1e-6


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_64bit_offsets_identical(oracle, pattern, storage):
    """The PSM kernel with 64-bit population offsets (used automatically beyond 19 N = 2^31
    elements, requested here on small lattices) gives the same populations in every step
    form, with walls and with periodic wraps: bit for bit in FP32; with 16-bit storage the
    two instantiations may fuse the scaling of decoded values into different FMAs, which
    shifts a stored value by one rounding of the format now and then (seen: 2e-7 to 2e-6
    on a few of 1.5e5 values after 3 to 6 steps), so the bound there is 1e-5."""
    g = W.rng(530)
    for periodic, walls in (((1, 1, 1), None), ((1, 1, 0), "z"), ((0, 0, 0), "all")):
        w = _lattice(periodic, walls, (37, 19, 11), storage=storage, fluid_force=(1e-6, 0.0, 0.0))
        f0 = random_populations(oracle, g, w.nx, w.ny, w.nz)
        a = gpu_from_workload(w, populations=f0, pattern=pattern)
        b = gpu_from_workload(w, populations=f0, pattern=pattern, index64=1)
        for n in (1, 2, 3):
            a.step(n)
            b.step(n)
            d = np.abs(_np(a.populations()) - _np(b.populations())).max()
            assert d <= (0.0 if storage == "f32" else 1e-5), (walls, n, d)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_lattice_beyond_32bit_offsets(oracle, pattern):
    """A lattice of 512 x 512 x 432 nodes (1.13e8; 19 N > 2^31 population elements), walls
    on z moving in x, one step in each form of the pattern: sampled nodes, many in the top
    planes where the element offsets pass 2^31, against the oracle's collision of the
    node's pre-collision populations."""
    import torch
    from paper_2512_04997_gb300 import ledds
    nx, ny, nz = 512, 512, 432
    assert 19 * nx * ny * nz > 2 ** 31
    w = W.Workload(name="big", nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0))
    w.params = W.base_params(tau=0.8, pattern=pattern)
    w.u_wall[2, 0] = [-0.05, 0.0, 0.0]
    w.u_wall[2, 1] = [0.05, 0.0, 0.0]
    z = np.arange(nz, dtype=np.float64)
    u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    u[0] = (-0.05 + 0.1 * (z + 0.5) / nz)[:, None, None]
    u[1] = 0.01 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, None, :]
    s = ledds.from_workload(w)
    s.init_fluid(None, u.reshape(3, -1))
    del u
    g = np.random.default_rng(77)
    N = nx * ny * nz
    cells = np.concatenate([g.integers(0, N, 400), g.integers(N - 3 * nx * ny, N, 400)])
    ci = torch.as_tensor(cells, device="cuda")
    for step in range(2):   # both step forms of the AA pattern
        f_pre = s.populations(0)[:, ci].cpu().numpy().astype(np.float64)
        s.step(1)
        f_post = s.populations(1)[:, ci].cpu().numpy().astype(np.float64)
        err = 0.0
        for j in range(len(cells)):
            fstar, _, _ = oracle.cell_collide(f_pre[:, j], 0.8)
            err = max(err, np.abs(fstar - f_post[:, j]).max())
        assert err < 5e-7, (step, err)
    st = s.status()
    assert st["rc"] == 0
    s.close()
    torch.cuda.empty_cache()
