"""Pins of the oracle's lattice Boltzmann part (Sec. 2.3) against closed forms.

None of these re-types the oracle's formulas: each checks a fact that the mathematics of
the D3Q19 BGK scheme fixes (lattice moments, conservation, exact steady solutions, the
viscosity relation of Eq. (tau)).
"""
import math

import numpy as np
import pytest

from paper_2512_04997_gb300 import workloads as W


def test_lattice_moments(oracle):
    """D3Q19 isotropy: sum w = 1, sum w c = 0, sum w c c = I/3,
    sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9, c_opp = -c."""
    c, w, opp = oracle.lattice_tables()
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose((w[:, None] * c).sum(0), 0.0, atol=1e-15)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, np.eye(3) / 3.0, atol=1e-15)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(fourth, iso, atol=1e-15)
    assert np.array_equal(c[opp], -c)
    assert len({tuple(v) for v in c}) == 19


@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.03, (0.05, -0.02, 0.01)),
                                   (0.97, (-0.1, 0.07, 0.03))])
def test_equilibrium_moments(oracle, rho, u):
    """Eq. (equilibrium) reproduces rho, rho u and the second moment rho (u u + I/3)."""
    c, _, _ = oracle.lattice_tables()
    f = oracle.equilibrium(rho, u)
    u = np.array(u)
    assert np.isclose(f.sum(), rho, rtol=1e-14)
    assert np.allclose(f @ c, rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.allclose(P, rho * (np.outer(u, u) + np.eye(3) / 3.0), atol=1e-14)


def test_mass_momentum_conserved_periodic(oracle):
    """Periodic box, off-equilibrium start: mass and momentum are invariants of BGK."""
    g = W.rng(100)
    nx, ny, nz = 6, 5, 4
    s = oracle.Sim(nx, ny, nz, periodic=(1, 1, 1), params=oracle.default_params(tau=0.7))
    rho, u = W.random_fields(g, nx, ny, nz)
    s.init_equilibrium(rho, u)
    f0 = s.populations() + W.population_noise(g, s.ncell, 1e-3)
    s.set_populations(f0)
    c, _, _ = oracle.lattice_tables()
    m0, p0 = f0.sum(), (f0.T @ c).sum(0)
    s.step(25)
    f1 = s.populations()
    assert abs(f1.sum() - m0) <= 1e-12 * m0
    assert np.allclose((f1.T @ c).sum(0), p0, atol=1e-13)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_shear_wave_viscosity(oracle, tau):
    """A sinusoidal shear wave decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3, Eq. (tau).
    The residual is the O(k^2) lattice dispersion (below 1 % at 32 nodes a wavelength)."""
    N, A, T = 32, 1e-3, 200
    s = oracle.Sim(1, 1, N, periodic=(1, 1, 1), params=oracle.default_params(tau=tau))
    z = np.arange(N)
    u = np.zeros((3, N))
    u[0] = A * np.sin(2 * np.pi * z / N)
    s.init_equilibrium(None, u)
    s.step(T)
    _, uu = s.moments()
    amp = (uu[0] * np.sin(2 * np.pi * z / N)).sum() * 2 / N
    k = 2 * np.pi / N
    expect = math.exp(-(tau - 0.5) / 3.0 * k * k * T)
    assert abs(amp / A / expect - 1.0) < 0.01
    # a wrong relation (e.g. nu = tau/3 or nu = (tau-1/2)/6) would be off by far more
    assert abs(math.exp(-tau / 3.0 * k * k * T) / expect - 1.0) > 0.05


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_couette_is_steady(oracle, tau):
    """Halfway moving-wall bounce-back (Sec. 2.3, Ladd): the linear Couette profile with
    the walls at -1/2 and nz-1/2 is an exact steady state for any tau."""
    nz, U = 16, 0.05
    uw = np.zeros((3, 2, 3))
    uw[2, 0, 0], uw[2, 1, 0] = -U, U
    s = oracle.Sim(2, 2, nz, periodic=(1, 1, 0), u_wall=uw, params=oracle.default_params(tau=tau))
    z = np.arange(nz)
    prof = -U + 2 * U * (z + 0.5) / nz
    u = np.zeros((3, nz, 2, 2))
    u[0] = prof[:, None, None]
    s.init_equilibrium(None, u.reshape(3, -1))
    s.step(200)
    rho, uu = s.moments()
    ux = uu[0].reshape(nz, 2, 2)
    assert np.abs(ux - prof[:, None, None]).max() < 1e-12 * U / U
    assert np.abs(rho - 1.0).max() < 1e-12
    assert np.abs(uu[1:]).max() < 1e-14


def test_couette_develops_from_rest(oracle):
    """Started from rest, the flow converges to the same linear profile."""
    nz, U = 16, 0.05
    uw = np.zeros((3, 2, 3))
    uw[2, 0, 0], uw[2, 1, 0] = -U, U
    s = oracle.Sim(1, 1, nz, periodic=(1, 1, 0), u_wall=uw, params=oracle.default_params(tau=0.8))
    s.step(6000)
    _, uu = s.moments()
    prof = -U + 2 * U * (np.arange(nz) + 0.5) / nz
    assert np.abs(uu[0] - prof).max() < 1e-9


def test_poiseuille_exact_at_magic_tau(oracle):
    """Body-force-driven channel between no-slip walls. With BGK, tau = 1/2 + sqrt(3)/4
    makes (tau - 1/2)^2 = 3/16, the magic combination for which the halfway-wall
    parabola u = F/(2 nu) (z+1/2)(H - z - 1/2) is the exact discrete solution; the same
    run at tau = 0.8 is off by the known O((tau-1/2)^2 - 3/16) slip error."""
    H, F = 8, 1e-6
    z = np.arange(H) + 0.5
    tau = 0.5 + math.sqrt(3) / 4
    s = oracle.Sim(1, 1, H, periodic=(1, 1, 0),
                   params=oracle.default_params(tau=tau, fluid_force=(F, 0, 0)))
    s.step(20000)
    _, uu = s.moments()
    ex = F / (2 * (tau - 0.5) / 3.0) * z * (H - z)
    assert np.abs(uu[0] - ex).max() / ex.max() < 1e-10
    s2 = oracle.Sim(1, 1, H, periodic=(1, 1, 0),
                    params=oracle.default_params(tau=0.8, fluid_force=(F, 0, 0)))
    s2.step(20000)
    _, u2 = s2.moments()
    ex2 = F / (2 * 0.1) * z * (H - z)
    err = np.abs(u2[0] - ex2).max() / ex2.max()
    assert 1e-3 < err < 3e-2


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2, 2.0])
def test_trt_poiseuille_exact_for_any_tau(oracle, tau):
    """TRT (Eq. TRT) with the paper's 1/tau- = 8 (2 - 1/tau+)/(8 - 1/tau+), i.e. the
    combination (tau+ - 1/2)(tau- - 1/2) = 3/16: the halfway-wall Poiseuille parabola is the
    exact discrete steady state for every tau (BGK reaches it only at one tau)."""
    H, F = 8, 1e-6
    z = np.arange(H) + 0.5
    s = oracle.Sim(1, 1, H, periodic=(1, 1, 0),
                   params=oracle.default_params(tau=tau, fluid_force=(F, 0, 0),
                                                collision=oracle.COLLIDE_TRT))
    nu = (tau - 0.5) / 3.0
    s.step(int(40 * H * H / nu) + 2000)
    _, uu = s.moments()
    ex = F / (2 * nu) * z * (H - z)
    assert np.abs(uu[0] - ex).max() / ex.max() < 1e-9


def test_trt_reduces_to_bgk_when_rates_coincide(oracle):
    """1/tau- = 1/tau+ where w^2 - 16 w + 16 = 0, w = 8 - 4 sqrt(3): there TRT is BGK
    (checked on random off-equilibrium cells, with and without solids and forcing)."""
    g = np.random.default_rng(77)
    tau = 1.0 / (8.0 - 4.0 * math.sqrt(3.0))
    for trial in range(20):
        f = oracle.lattice_tables()[1] * (1.0 + 0.05 * g.standard_normal(19))
        B = list(g.uniform(0, 0.6, trial % 3))
        uk = g.normal(0, 0.02, (len(B), 3))
        arm = g.normal(0, 2, (len(B), 3))
        force = g.normal(0, 1e-4, 3) if trial % 2 else (0, 0, 0)
        a = oracle.cell_collide(f, tau, B, uk, arm, force, collision=oracle.COLLIDE_BGK)
        b = oracle.cell_collide(f, tau, B, uk, arm, force, collision=oracle.COLLIDE_TRT)
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=0, atol=1e-15)


def test_trt_conserves_mass_and_momentum(oracle):
    """The TRT operator changes neither the density nor the momentum of a fluid cell, and
    relaxes the symmetric and antisymmetric non-equilibrium parts at 1/tau+ and 1/tau-."""
    g = np.random.default_rng(78)
    c, t, opp = oracle.lattice_tables()
    for tau in (0.55, 0.8, 1.5):
        f = t * (1.0 + 0.05 * g.standard_normal(19))
        fs, _, _ = oracle.cell_collide(f, tau, collision=oracle.COLLIDE_TRT)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.abs(c.T @ fs - c.T @ f).max() < 1e-15
        rho = f.sum()
        u = (c.T @ f) / rho
        feq = oracle.equilibrium(rho, u)
        wp = 1.0 / tau
        wm = 8.0 * (2.0 - wp) / (8.0 - wp)
        neq, neq_out = f - feq, fs - feq
        sym_in, asym_in = 0.5 * (neq + neq[opp]), 0.5 * (neq - neq[opp])
        sym_out, asym_out = 0.5 * (neq_out + neq_out[opp]), 0.5 * (neq_out - neq_out[opp])
        assert np.allclose(sym_out, (1 - wp) * sym_in, rtol=0, atol=1e-15)
        assert np.allclose(asym_out, (1 - wm) * asym_in, rtol=0, atol=1e-15)
