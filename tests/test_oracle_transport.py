"""Pins of the oracle's explicit stage (Sections 2.3, A.2-A.4) and the full
step: exact upwind shifts, exact discrete eigen-decay of diffusion, exact
steady states, closed-form sources, wall treatment, symmetry."""
import numpy as np
import pytest

from oracle import model, transport
from oracle.geometry import Geometry
from oracle.step import OracleCase
from paper_2603_21869_gb300 import cases

P_ = cases.Patch


def _faces(x=(cases.OUTLET, cases.OUTLET), y=(cases.OUTLET, cases.OUTLET), z=(cases.EMPTY, cases.EMPTY)):
    return [P_(x[0]), P_(x[1]), P_(y[0]), P_(y[1]), P_(z[0]), P_(z[1])]


def _state(spec, u=0.0, v=0.0, w=0.0, T=0.0, k=1e-14, om=1e4):
    shape = (spec.nx, spec.ny, spec.nz)
    return [np.broadcast_to(np.asarray(a, dtype=float), shape).copy() for a in (u, v, w, T, k, om)]


@pytest.mark.parametrize("direction", [+1, -1])
def test_upwind_cfl_one_is_exact_shift(direction):
    """First-order upwind at CFL 1 moves a step profile exactly one cell per
    step, downstream; the branch I[u_face >= 0] vs I[u_face < 0] decides the
    direction (Eq. upwind_x)."""
    n = 16
    faces = _faces()
    inlet_face = 0 if direction > 0 else 1
    faces[inlet_face] = P_(cases.INLET, u_normal=1.0, T_in=1.0, k_value=1e-14, omega_value=1.0)
    spec = cases.CaseSpec(nx=n, ny=4, nz=1, Lx=1.0, Ly=0.25, Lz=1.0 / 16, nu=1e-30, faces=faces,
                          dt=1.0 / 16, dt_adapt=0, mg_levels=2)
    T0 = np.zeros((n, 4, 1))
    if direction > 0:
        T0[:4] = 1.0
    else:
        T0[-4:] = 1.0
    c = OracleCase(spec, state=_state(spec, u=float(direction), T=T0, om=1.0))
    for s in range(1, 6):
        c.step()
        T = c.state[3]
        exp = np.zeros_like(T)
        if direction > 0:
            exp[:4 + s] = 1.0
        else:
            exp[-(4 + s):] = 1.0
        assert np.max(np.abs(T - exp)) < 1e-11
        assert np.allclose(c.state[0], float(direction), atol=1e-12)
        assert np.max(np.abs(c.p)) == 0.0


@pytest.mark.parametrize("thermal,mode", [(cases.ADIABATIC, "cos"), (cases.FIXED_T, "sin")])
def test_temperature_diffusion_exact_discrete_decay(thermal, mode):
    """T = cos (zero-gradient walls) or sin (T_w = 0 walls) modes of the
    discrete Laplacian decay by exactly (1 - dt alpha lambda_m) per step."""
    ny, m, nu = 16, 3, 0.01
    faces = _faces(y=(cases.WALL, cases.WALL))
    faces[2] = P_(cases.WALL, thermal=thermal, T_value=0.0)
    faces[3] = P_(cases.WALL, thermal=thermal, T_value=0.0)
    spec = cases.CaseSpec(nx=4, ny=ny, nz=1, Lx=0.25, Ly=1.0, Lz=1.0 / 16, nu=nu, Pr=0.7,
                          faces=faces, dt_adapt=0, mg_levels=2)
    h = 1.0 / ny
    alpha = nu / 0.7
    spec = spec.replace(dt=0.2 * h * h / alpha)
    j = np.arange(ny) + 0.5
    prof = np.cos(m * np.pi * j / ny) if mode == "cos" else np.sin(m * np.pi * j / ny)
    T0 = np.broadcast_to(prof[None, :, None], (4, ny, 1))
    c = OracleCase(spec, state=_state(spec, T=T0))
    lam = (2 - 2 * np.cos(m * np.pi / ny)) / h ** 2
    g = 1.0 - spec.dt * alpha * lam
    c.step(10)
    assert np.allclose(c.state[3], T0 * g ** 10, rtol=0, atol=1e-12)


def test_velocity_diffusion_between_no_slip_walls():
    """u = sin mode across no-slip walls (ghost -u_P) decays by (1 - dt nu lambda_m)."""
    ny, m, nu = 16, 1, 0.01
    faces = _faces(y=(cases.WALL, cases.WALL))
    spec = cases.CaseSpec(nx=4, ny=ny, nz=1, Lx=0.25, Ly=1.0, Lz=1.0 / 16, nu=nu,
                          faces=faces, dt_adapt=0, mg_levels=2)
    h = 1.0 / ny
    spec = spec.replace(dt=0.2 * h * h / nu)
    j = np.arange(ny) + 0.5
    u0 = np.broadcast_to(np.sin(m * np.pi * j / ny)[None, :, None], (4, ny, 1))
    c = OracleCase(spec, state=_state(spec, u=u0))
    c.step(10)
    g = 1.0 - spec.dt * nu * (2 - 2 * np.cos(m * np.pi / ny)) / h ** 2
    assert np.allclose(c.state[0], u0 * g ** 10, rtol=0, atol=1e-12)
    assert np.max(np.abs(c.state[1])) < 1e-12


def _body_force_poiseuille(ny, nu=0.01, F=0.5, H=1.0):
    faces = _faces(y=(cases.WALL, cases.WALL))
    spec = cases.CaseSpec(nx=4, ny=ny, nz=1, Lx=4 * H / ny, Ly=H, Lz=H / ny, nu=nu, faces=faces,
                          buoyancy=1, gravity=(-1.0, 0.0, 0.0), beta_T=1.0, T_ref=0.0,
                          dt_adapt=0, mg_levels=2)
    h = H / ny
    spec = spec.replace(dt=0.2 * h * h / nu)
    # discrete steady state: nu (u_{j+1} - 2u_j + u_{j-1}) / h^2 + F = 0, mirror ghosts at walls
    M = np.zeros((ny, ny))
    for j in range(ny):
        M[j, j] = -2.0
        if j > 0:
            M[j, j - 1] = 1.0
        if j < ny - 1:
            M[j, j + 1] = 1.0
    M[0, 0] -= 1.0
    M[-1, -1] -= 1.0
    u = np.linalg.solve(nu * M / h ** 2, -F * np.ones(ny))
    y = (np.arange(ny) + 0.5) * h
    return spec, u, F / (2 * nu) * y * (H - y)


def test_body_force_poiseuille_is_a_fixed_point():
    """Laminar channel driven by a uniform body force: the discrete steady
    profile is left unchanged by full steps (walls, viscous term, force,
    projection), and it converges to the closed form u = F y (H - y) / (2 nu)
    at second order."""
    spec, u_disc, _ = _body_force_poiseuille(16)
    u0 = np.broadcast_to(u_disc[None, :, None], (4, 16, 1))
    c = OracleCase(spec, state=_state(spec, u=u0, T=0.5))
    c.step(5)
    assert np.max(np.abs(c.state[0] - u0)) < 1e-12 * np.max(u_disc)
    errs = []
    for ny in (16, 32):
        _, ud, uex = _body_force_poiseuille(ny)
        errs.append(np.max(np.abs(ud - uex)))
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("where", ["wall", "box"])
def test_heat_flux_and_fixed_temperature_linear_steady_state(where):
    """Heat flux q entering through a wall or an obstacle face and leaving
    through a fixed-temperature wall: the linear profile with slope
    q / (rho cp alpha) is an exact fixed point."""
    ny, nu, q, Tw = 8, 1.5e-5, 50.0, 20.0
    faces = _faces(y=(cases.WALL, cases.WALL))
    boxes = []
    if where == "wall":
        faces[2] = P_(cases.WALL, thermal=cases.FIXED_T, T_value=Tw)
        faces[3] = P_(cases.WALL, thermal=cases.HEAT_FLUX, T_value=q)
    else:
        faces[2] = P_(cases.WALL)
        faces[3] = P_(cases.WALL, thermal=cases.FIXED_T, T_value=Tw)
        boxes = [cases.Box(0, 4, 0, 2, 0, 1, thermal=cases.HEAT_FLUX, T_value=q)]
    spec = cases.CaseSpec(nx=4, ny=ny, nz=1, Lx=0.5, Ly=1.0, Lz=1.0 / ny, nu=nu, Pr=0.71,
                          faces=faces, boxes=boxes, dt=1.0, dt_adapt=0, mg_levels=2)
    alpha = nu / 0.71
    s = q / (spec.rho * spec.cp * alpha)
    y = (np.arange(ny) + 0.5) / ny
    T = Tw + s * y if where == "wall" else Tw + s * (1.0 - y)
    T = np.broadcast_to(T[None, :, None], (4, ny, 1)).copy()
    geo = Geometry(spec)
    T[geo.solid] = 0.0
    c = OracleCase(spec, state=_state(spec, T=T))
    c.step(3)
    fl = geo.fluid
    assert np.max(np.abs(c.state[3][fl] - T[fl])) < 1e-9 * np.max(np.abs(T))


def test_two_thirds_k_gradient_in_momentum():
    """With u = 0 and k linear in x the u-momentum rate is -(2/3) dk/dx (Eq. ko_mom)."""
    n = 8
    spec = cases.CaseSpec(nx=n, ny=n, nz=n, Lx=1.0, Ly=1.0, Lz=1.0, faces=_faces(z=(cases.OUTLET,) * 2))
    geo = Geometry(spec)
    x = (np.arange(n) + 0.5) / n
    k = np.broadcast_to((1.0 + 0.5 * x)[:, None, None], (n, n, n)).copy()
    rhs = transport.explicit_rhs(geo, _state(spec, k=k, om=1.0))
    assert np.allclose(rhs[0][1:-1], -(2.0 / 3.0) * 0.5, rtol=1e-12)
    assert np.allclose(rhs[1], 0.0, atol=1e-14) and np.allclose(rhs[2], 0.0, atol=1e-14)


def test_buoyancy_source_sign_and_size():
    """Warm fluid (T > T_ref) accelerates against gravity: dw/dt = g beta (T - T_ref)."""
    spec = cases.CaseSpec(nx=4, ny=4, nz=4, Lx=1.0, Ly=1.0, Lz=1.0, faces=_faces(z=(cases.OUTLET,) * 2),
                          buoyancy=1, gravity=(0.0, 0.0, -9.81), beta_T=1 / 295.15, T_ref=22.0)
    rhs = transport.explicit_rhs(Geometry(spec), _state(spec, T=27.0, om=1.0))
    assert np.allclose(rhs[2], 9.81 / 295.15 * 5.0, rtol=1e-13)
    assert np.allclose(rhs[0], 0.0, atol=1e-15)


def test_shear_production_in_k_equation():
    """u = gamma y with uniform k and omega: dk/dt = nu_t gamma^2 away from walls (Eq. k_gen)."""
    n, g = 8, 3.0
    spec = cases.CaseSpec(nx=n, ny=n, nz=n, Lx=1.0, Ly=1.0, Lz=1.0, faces=_faces(z=(cases.OUTLET,) * 2))
    geo = Geometry(spec)
    y = (np.arange(n) + 0.5) / n
    u = np.broadcast_to((g * y)[None, :, None], (n, n, n))
    k, om = 0.02, 5.0
    rhs = transport.explicit_rhs(geo, _state(spec, u=u, k=k, om=om))
    nut = float(model.nu_t(np.array(k), np.array(om), spec.nu))
    assert np.allclose(rhs[4][:, 1:-1, :], nut * g * g, rtol=1e-12)


def test_wall_omega_uses_nearest_wall():
    """omega in wall-adjacent cells = 6 nu/(beta_i d^2), d = half the normal
    width; corners take the larger value; obstacle faces count as walls."""
    faces = _faces(y=(cases.WALL, cases.WALL), z=(cases.WALL, cases.OUTLET))
    spec = cases.CaseSpec(nx=8, ny=8, nz=8, Lx=1.0, Ly=1.0, Lz=0.5, faces=faces,
                          boxes=[cases.Box(3, 5, 3, 5, 3, 5)])
    geo = Geometry(spec)
    ow = transport.wall_omega(geo)
    wy = model.omega_wall(spec.nu, 0.5 / 8)
    wz = model.omega_wall(spec.nu, 0.25 / 8)
    assert ow[4, 0, 4] == pytest.approx(wy) and ow[4, 7, 6] == pytest.approx(wy)
    assert ow[4, 4, 0] == pytest.approx(wz) and ow[4, 0, 0] == pytest.approx(wz)
    assert ow[2, 4, 4] == pytest.approx(model.omega_wall(spec.nu, 1 / 16))   # x face of the box
    assert ow[4, 4, 2] == pytest.approx(wz)                                  # z face of the box
    assert ow[0, 4, 4] == 0.0 and ow[4, 4, 7] == 0.0 and ow[4, 4, 4] == 0.0


def test_channel_stays_symmetric():
    """A y-symmetric 2D channel stays mirror-symmetric: u, k, omega, T even
    and v odd about the centre line (pins y indexing and signs)."""
    spec = cases.channel_2d(32, 16, 3, init_perturb=0.0)
    c = OracleCase(spec).step(8)
    u, v, w, T, k, om = c.state
    for f in (u, k, om, T, c.p):
        assert np.max(np.abs(f - f[:, ::-1, :])) <= 1e-11 * max(1.0, np.max(np.abs(f)))
    assert np.max(np.abs(v + v[:, ::-1, :])) <= 1e-11


def test_mass_balance_after_projection():
    """Inflow through the inlet equals the outflow of the corrected fluxes to
    solver tolerance (Eq. ko_cont enforced by the projection)."""
    spec = cases.heated_channel_3d(32, 8, 8, mg_levels=3, mg_rel_tol=1e-11,
                                   boxes=[cases.Box(8, 12, 2, 6, 0, 5)])
    c = OracleCase(spec).step(3)
    div = c.divergence_after_projection()
    assert np.max(np.abs(div)) < 1e-9 * 2.0 / c.geo.h[0]
    assert c.last_rel <= 1e-11


@pytest.mark.parametrize("stages", [1, 2, 3])
@pytest.mark.parametrize("z", [0.1, 0.45])
def test_runge_kutta_stability_polynomial_on_a_diffusion_eigenmode(stages, z):
    """On an eigenmode of the discrete Laplacian the explicit operator is the
    scalar -alpha lambda_m, so an s-stage scheme of order s multiplies the mode
    by its stability polynomial R(-z) = sum_{j<=s} (-z)^j / j! per step,
    z = dt alpha lambda_m (the strong-stability-preserving schemes of order
    2 and 3 have exactly these polynomials).  m = 8 of 16 keeps the largest
    eigenvalue of the 2D operator at 4 lambda_m, inside the stability
    interval for both z (rounding does not seed a growing mode)."""
    ny, m, nu = 16, 8, 0.01
    faces = _faces(y=(cases.WALL, cases.WALL))
    faces[2] = P_(cases.WALL, thermal=cases.ADIABATIC)
    faces[3] = P_(cases.WALL, thermal=cases.ADIABATIC)
    spec = cases.CaseSpec(nx=4, ny=ny, nz=1, Lx=0.25, Ly=1.0, Lz=1.0 / 16, nu=nu, Pr=0.7,
                          faces=faces, dt_adapt=0, mg_levels=2, rk_stages=stages)
    h = 1.0 / ny
    alpha = nu / 0.7
    lam = (2 - 2 * np.cos(m * np.pi / ny)) / h ** 2
    spec = spec.replace(dt=z / (alpha * lam))
    j = np.arange(ny) + 0.5
    T0 = np.broadcast_to(np.cos(m * np.pi * j / ny)[None, :, None], (4, ny, 1))
    c = OracleCase(spec, state=_state(spec, T=T0))
    R = sum((-z) ** q / np.prod(range(1, q + 1)) for q in range(stages + 1))
    c.step(6)
    assert np.allclose(c.state[3], T0 * R ** 6, rtol=0, atol=1e-12)


@pytest.mark.parametrize("stages", [2, 3])
def test_strong_stability_keeps_an_advected_step_within_bounds(stages):
    """At CFL 1 each forward-Euler upwind stage is a shift, so the convex
    combinations of the strong-stability-preserving schemes keep a step
    profile inside [0, 1] (a classical midpoint RK2 would not)."""
    n = 32
    faces = _faces()
    faces[0] = P_(cases.INLET, u_normal=1.0, T_in=1.0, k_value=1e-14, omega_value=1.0)
    spec = cases.CaseSpec(nx=n, ny=4, nz=1, Lx=1.0, Ly=0.125, Lz=1.0 / 32, nu=1e-30, faces=faces,
                          dt=1.0 / 32, dt_adapt=0, mg_levels=2, rk_stages=stages)
    T0 = np.zeros((n, 4, 1))
    T0[:6] = 1.0
    c = OracleCase(spec, state=_state(spec, u=1.0, T=T0, om=1.0))
    for _ in range(12):
        c.step()
        T = c.state[3]
        assert T.min() >= -1e-14 and T.max() <= 1.0 + 1e-14
    assert 0.0 < T[10, 0, 0] < 1.0          # a smeared front (not the exact shift of forward Euler)


def test_runge_kutta_temporal_order_on_smooth_nonlinear_transport():
    """Nonlinear advection and diffusion of a smooth velocity and temperature
    field (turbulence negligible: k at its floor) over a fixed time: the error
    against a fine-step reference falls by 2^s when dt halves, s = the
    scheme's order (1, 2, 3)."""
    n, h = (16, 8, 8), 0.01
    faces = [P_(cases.OUTLET) for _ in range(6)]
    spec = cases.CaseSpec(nx=n[0], ny=n[1], nz=n[2], Lx=n[0] * h, Ly=n[1] * h, Lz=n[2] * h, nu=1e-4, Pr=0.7,
                          faces=faces, dt=0.002, dt_adapt=0, mg_levels=2)
    geo = Geometry(spec)
    X, Y, Z = np.meshgrid(*[(np.arange(m) + 0.5) * h for m in n], indexing="ij")
    Lx, Ly, Lz = (m * h for m in n)
    s0 = [1.0 + 0.3 * np.sin(2 * np.pi * Y / Ly) * np.cos(2 * np.pi * Z / Lz),
          0.2 * np.sin(2 * np.pi * X / Lx),
          0.1 * np.cos(2 * np.pi * X / Lx) * np.sin(2 * np.pi * Y / Ly),
          20.0 + np.cos(2 * np.pi * X / Lx) * np.cos(2 * np.pi * Y / Ly),
          np.full(X.shape, 1e-14), np.ones(X.shape)]
    t_end = 0.008

    def run(stages, nsteps):
        st = [x.copy() for x in s0]
        for _ in range(nsteps):
            st = transport.explicit_stage_rk(geo, st, t_end / nsteps, stages)
        return st[:4]

    ref = run(3, 1024)
    for stages in (1, 2, 3):
        errs = [max(float(np.max(np.abs(a - b))) for a, b in zip(run(stages, m), ref)) for m in (4, 8, 16)]
        for r in (errs[0] / errs[1], errs[1] / errs[2]):
            assert 0.75 * 2 ** stages < r < 1.25 * 2 ** stages, (stages, errs)


def test_one_stage_is_forward_euler_and_bad_stage_count_rejected():
    spec = cases.heated_channel_3d(16, 8, 8, mg_levels=2, init_perturb=0.2)
    geo = Geometry(spec)
    s0 = OracleCase(spec).state
    a = transport.explicit_stage(geo, s0, 1e-3)
    b = transport.explicit_stage_rk(geo, s0, 1e-3, 1)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    with pytest.raises(ValueError):
        transport.explicit_stage_rk(geo, s0, 1e-3, 4)
