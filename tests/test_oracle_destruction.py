"""Pins of the semi-implicit destruction (Eqs. k_des_step, o_des_step,
Algorithm 4) and the Strang splitting (Section 2.6): homogeneous decay in
closed form, exact discrete recurrences, positivity, gradient branches."""
import numpy as np
import pytest

from oracle import model
from oracle.destruction import destruction_step
from oracle.geometry import Geometry
from oracle.step import OracleCase
from paper_2603_21869_gb300 import cases


def _homogeneous(n=4, nu=1e-10, dt=0.01, k0=1.0, om0=2.0):
    faces = [cases.Patch(cases.OUTLET) for _ in range(6)]
    spec = cases.CaseSpec(nx=n, ny=n, nz=n, Lx=1.0, Ly=1.0, Lz=1.0, nu=nu, faces=faces,
                          dt=dt, dt_adapt=0, mg_levels=2, init_k=k0, init_omega=om0, init_T=1.0)
    return spec


def test_homogeneous_omega_decay_closed_form():
    """Without gradients 1/omega grows by beta dt/2 per half step, so after n
    steps omega_n = omega0 / (1 + n beta omega0 dt): the exact solution of
    d omega/dt = -beta omega^2."""
    spec = _homogeneous()
    c = OracleCase(spec)
    for n in range(1, 41):
        c.step()
        exact = 2.0 / (1.0 + n * 0.072 * 2.0 * 0.01)
        assert np.allclose(c.state[5], exact, rtol=1e-13, atol=0)
    assert np.all(c.state[0] == 0.0) and np.all(c.p == 0.0)


def test_homogeneous_k_recurrence_and_first_order_convergence():
    """At Re_t >> R_beta beta* = beta*_inf; k follows
    k <- k / (1 + dt/2 beta*_inf omega) with the pre-update omega, exactly,
    and tends to the ODE solution k0 (1 + beta omega0 t)^(-beta*_inf/beta)
    at first order in dt."""
    t_end = 0.8
    errs = []
    for dt in (0.02, 0.01):
        c = OracleCase(_homogeneous(dt=dt))
        k, om = 1.0, 2.0
        nsteps = int(round(t_end / dt))
        for _ in range(nsteps):
            c.step()
            for _half in range(2):
                k, om = k / (1 + dt / 2 * 0.09 * om), om / (1 + dt / 2 * 0.072 * om)
        assert np.allclose(c.state[4], k, rtol=1e-12, atol=0)
        k_ode = (1 + 0.072 * 2.0 * t_end) ** (-0.09 / 0.072)
        errs.append(abs(c.state[4][0, 0, 0] - k_ode))
    assert 1.8 < errs[0] / errs[1] < 2.2


def test_low_reynolds_beta_star():
    """Re_t -> 0 gives beta* = beta*_inf 4/15 in the k update."""
    spec = _homogeneous(nu=1e6)
    geo = Geometry(spec)
    z = np.zeros(geo.shape)
    k = np.full(geo.shape, 0.5)
    om = np.full(geo.shape, 3.0)
    dt = 0.1
    k1, om1 = destruction_step(geo, z, z, z, k, om, dt)
    assert np.allclose(k1, 0.5 / (1 + dt * 0.09 * 4 / 15 * 3.0), rtol=1e-12)
    assert np.allclose(om1, 3.0 / (1 + dt * 0.072 * 3.0), rtol=1e-15)


def test_positivity_for_huge_time_step():
    """The semi-implicit update keeps k, omega positive for any dt (Section 2.5)."""
    spec = cases.heated_channel_3d(16, 8, 8, mg_levels=2, init_perturb=0.3)
    c = OracleCase(spec)
    u, v, w, T, k, om = c.state
    for dt in (1e3, 1e9):
        k1, om1 = destruction_step(c.geo, u, v, w, k, om, dt)
        assert np.all(k1 > 0) and np.all(om1 > 0) and np.all(np.isfinite(k1))
        assert np.all(k1 <= k) and np.all(om1 <= om)


def test_chi_k_branch_on_aligned_gradients():
    """k = 1 + a x, omega = 2 + b x with a b > 0: chi_k = a b / omega^3 > 0
    and f_beta* = (1 + 680 chi^2)/(1 + 400 chi^2) raises the destruction of k;
    with opposed gradients f_beta* = 1 (Eq. k_des)."""
    n = 8
    spec = _homogeneous(n=n, nu=1e-10)
    geo = Geometry(spec)
    x = (np.arange(n) + 0.5) / n
    z = np.zeros(geo.shape)
    dt = 0.05
    for a, b in ((0.8, 1.5), (0.8, -1.5)):
        k = np.broadcast_to((1 + a * x)[:, None, None], geo.shape).copy()
        om = np.broadcast_to((2 + b * x)[:, None, None], geo.shape).copy()
        k1, _ = destruction_step(geo, z, z, z, k, om, dt)
        chi = a * b / om ** 3
        f = np.where(chi > 0, (1 + 680 * chi ** 2) / (1 + 400 * chi ** 2), 1.0)
        exp = k / (1 + dt * 0.09 * f * om)
        assert np.allclose(k1[1:-1], exp[1:-1], rtol=1e-12)
        if a * b > 0:
            assert np.all(f[1:-1] > 1.0)


def test_omega_destruction_uses_vortex_stretching():
    """A 3D velocity field with rotation about z and axial strain gives
    chi_omega = a^2 s / (beta*_inf omega)^3 and f_beta = (1+70 chi)/(1+80 chi)."""
    n = 8
    spec = _homogeneous(n=n, nu=1e-10)
    geo = Geometry(spec)
    c = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    a, s = 0.6, 0.4
    u = -s / 2 * X + a * Y
    v = -a * X - s / 2 * Y
    w = s * Z
    om = np.full(geo.shape, 1.2)
    k = np.full(geo.shape, 0.3)
    dt = 0.1
    _, om1 = destruction_step(geo, u, v, w, k, om, dt)
    chi = a * a * s / (0.09 * 1.2) ** 3
    fb = (1 + 70 * chi) / (1 + 80 * chi)
    inner = (slice(1, -1),) * 3
    assert np.allclose(om1[inner], 1.2 / (1 + dt * 0.072 * fb * 1.2), rtol=1e-12)


def test_explicit_stage_is_zero_for_homogeneous_state():
    """No gradients and no walls: the explicit stage leaves the state unchanged."""
    spec = _homogeneous(n=4)
    c = OracleCase(spec)
    before = [s.copy() for s in c.state]
    c.explicit()
    for b, a in zip(before, c.state):
        assert np.array_equal(b, a)
