"""Pins of the oracle's closure formulas (Section 2.1) by limits, special
cases and closed forms that a dropped term, wrong sign or wrong index would
break."""
import numpy as np
import pytest

from oracle import model
from oracle.geometry import Geometry, U, V, W, cell_gradient
from paper_2603_21869_gb300 import cases

NU = 1.5e-5


def test_alpha_star_limits():
    # Eq. a_star: alpha* -> alpha*_0 = beta_i/3 as Re_t -> 0, -> alpha*_inf = 1 as Re_t -> inf
    assert model.alpha_star(np.array(0.0), np.array(1.0), NU) == pytest.approx(0.072 / 3, rel=1e-15)
    assert model.alpha_star(np.array(1e12), np.array(1.0), NU) == pytest.approx(1.0, rel=1e-9)
    # at Re_t = R_k the blend is halfway in the sense (a0 + 1) / 2
    k = 6.0 * NU * 2.0
    assert model.alpha_star(np.array(k), np.array(2.0), NU) == pytest.approx((0.024 + 1) / 2, rel=1e-14)


def test_beta_star_limits():
    # Eq. beta_star: beta*_inf * 4/15 at Re_t = 0, beta*_inf as Re_t -> inf
    assert model.beta_star(np.array(0.0), np.array(1.0), NU) == pytest.approx(0.09 * 4 / 15, rel=1e-15)
    assert model.beta_star(np.array(1e6), np.array(1e-3), NU) == pytest.approx(0.09, rel=1e-12)
    k = 8.0 * NU * 3.0     # Re_t = R_beta -> (4/15 + 1) / 2
    assert model.beta_star(np.array(k), np.array(3.0), NU) == pytest.approx(0.09 * (4 / 15 + 1) / 2, rel=1e-14)


def test_alpha_limits():
    # Eq. a: alpha * alpha* -> alpha_inf alpha_0 at Re_t = 0 and -> alpha_inf as Re_t -> inf
    z = np.array(0.0)
    a0 = model.alpha_coef(z, np.array(1.0), NU) * model.alpha_star(z, np.array(1.0), NU)
    assert a0 == pytest.approx(0.52 / 9, rel=1e-14)
    big = np.array(1e12)
    assert model.alpha_coef(big, np.array(1.0), NU) == pytest.approx(0.52, rel=1e-9)


def test_f_beta_star_branches_and_continuity():
    chi = np.array([-1.0, 0.0, 1e-9, 1e9])
    f = model.f_beta_star(chi)
    assert f[0] == 1.0 and f[1] == 1.0
    assert f[2] == pytest.approx(1.0, abs=1e-12)        # continuous at chi_k = 0
    assert f[3] == pytest.approx(680 / 400, rel=1e-12)  # large-chi limit 1.7


def test_f_beta_limits():
    assert model.f_beta(np.array(0.0)) == 1.0
    assert model.f_beta(np.array(1e12)) == pytest.approx(70 / 80, rel=1e-9)


def test_inlet_turbulence_matches_k_epsilon_viscosity():
    # k0/omega0 must equal the k-epsilon eddy viscosity C_mu k0^2 / eps0 = C_mu sqrt(k0) l0
    for U_, I, l0 in [(0.455, 0.04, 0.3), (1.0, 0.05, 0.07), (2.0, 0.1, 0.0448)]:
        k0, om0 = model.inlet_turbulence(U_, I, l0)
        assert k0 == pytest.approx(1.5 * (I * U_) ** 2, rel=1e-15)
        assert k0 / om0 == pytest.approx(0.09 * np.sqrt(k0) * l0, rel=1e-13)


def test_omega_wall_scaling():
    # omega_wall = 6 nu / (beta_i d^2): inverse-square in d, linear in nu
    assert model.omega_wall(1.0, 1.0) == pytest.approx(6 / 0.072)
    assert model.omega_wall(NU, 0.5e-3) / model.omega_wall(NU, 1e-3) == pytest.approx(4.0)


def _box_spec(n=8):
    faces = [cases.Patch(cases.OUTLET) for _ in range(6)]
    return cases.CaseSpec(nx=n, ny=n, nz=n, Lx=1.0, Ly=1.0, Lz=1.0, faces=faces, mg_levels=2)


def test_cell_gradient_exact_on_linear_field_and_strain_invariants():
    """Central L*D*BC(phi) recovers a linear velocity field's gradient exactly
    in the interior; S, S^2 and the vortex-stretching invariant then follow."""
    geo = Geometry(_box_spec())
    h = geo.h[0]
    x = (np.arange(8) + 0.5) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    rng = np.random.default_rng(1)
    G = rng.normal(size=(3, 3))
    vel = [G[i, 0] * X + G[i, 1] * Y + G[i, 2] * Z for i in range(3)]
    grad = [cell_gradient(geo, vel[i], f) for i, f in enumerate((U, V, W))]
    inner = (slice(1, -1),) * 3
    for i in range(3):
        for j in range(3):
            assert np.allclose(grad[i][j][inner], G[i, j], rtol=0, atol=1e-12)
    S, O = model.strain_rotation(grad)
    S2 = model.strain_magnitude_sq(S)
    Sm = 0.5 * (G + G.T)
    assert np.allclose(S2[inner], 2.0 * np.sum(Sm * Sm), rtol=1e-12)


def test_chi_omega_vortex_stretching_closed_form():
    """Rotation a about z with axial strain s (S = diag(-s/2, -s/2, s)):
    Omega_ij Omega_jk S_ki = a^2 s, so chi_omega = |a^2 s| / (beta*_inf omega)^3."""
    a, s, om = 0.7, 0.3, 2.0
    z = np.zeros(())
    grad = [[z - s / 2, z + a, z], [z - a, z - s / 2, z], [z, z, z + s]]
    S, O = model.strain_rotation(grad)
    chi = model.chi_omega(S, O, np.array(om))
    assert chi == pytest.approx(a * a * s / (0.09 * om) ** 3, rel=1e-14)
    # pure rotation and pure strain give zero
    rot = [[z, z + a, z], [z - a, z, z], [z, z, z]]
    assert model.chi_omega(*model.strain_rotation(rot), np.array(om)) == 0.0
    strain = [[z + s, z, z], [z, z - s, z], [z, z, z]]
    assert model.chi_omega(*model.strain_rotation(strain), np.array(om)) == 0.0


def test_chi_omega_vanishes_in_2d_for_trace_free_strain():
    """2D: Omega^2 = -a^2 I on the plane, so the invariant is -a^2 tr(S) = 0
    when the (cell) velocity field is divergence free."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        p, q, r = rng.normal(size=3)
        z = np.zeros(())
        grad = [[z + p, z + q, z], [z + r, z - p, z], [z, z, z]]
        S, O = model.strain_rotation(grad)
        assert abs(float(model.chi_omega(S, O, np.array(1.3)))) < 1e-15


def test_production_simple_shear():
    """u = gamma y: S = |gamma|, G_k = nu_t gamma^2 (Eq. k_gen with Eq. strain_rate_magnitude)."""
    g = 2.5
    z = np.zeros(())
    grad = [[z, z + g, z], [z, z, z], [z, z, z]]
    S, _ = model.strain_rotation(grad)
    S2 = model.strain_magnitude_sq(S)
    assert S2 == pytest.approx(g * g, rel=1e-15)
    k, om = np.array(0.01), np.array(3.0)
    assert model.production_k(k, om, NU, S2) == pytest.approx(model.nu_t(k, om, NU) * g * g, rel=1e-15)
    # G_omega = alpha alpha* S^2 identically
    Gw = model.production_omega(k, om, NU, S2)
    assert Gw == pytest.approx(model.alpha_coef(k, om, NU) * model.alpha_star(k, om, NU) * g * g, rel=1e-13)
