"""Explicit stage: convection, diffusion and production (Sections 2.3, A.2-A.4).

For each transported phi in {u, v, w, T, k, omega}, along each axis:
  * face velocity u_face = L * BC(u)                      (Algorithm 2)
  * upwind value: W+ * BC(phi) where u_face >= 0, else W- * BC(phi)
                                                          (Eq. upwind_x)
  * convective flux (u phi)_face = phi_upwind u_face
  * diffusive flux Gamma_face D * BC(phi) with Gamma = nu + nu_t
    (momentum), nu + nu_t/sigma_k (k), nu + nu_t/sigma_omega (omega),
    alpha + nu_t/Pr_t (T)                                 (Eqs. ko_mom - ko_temp)
  * the momentum component along the axis also carries -(2/3) k_face
    (the -2/3 k delta_ij term of Eq. ko_mom, placed like the face pressure
    of Algorithm 3)
  * d phi / dt = sum_j D_j * f_j                          (Eq. divergence_theorem)
Sources: G_k (Eq. k_gen), G_omega (Eq. o_gen), and, when enabled, Boussinesq
buoyancy -g_i beta_T (T - T_ref).  The pressure gradient is not part of the
predictor (the projection of Section 2.4 supplies it).

Face eddy viscosity: the mean of the two cells; zero on wall faces (domain
walls and obstacle faces); the interior cell's value on inlet, outlet and
empty faces.

After the forward-Euler update k and omega are clamped positive (Section
A.4) and omega in every cell next to a wall is set to 6 nu / (beta_i d^2)
with d = half the cell width normal to that wall (Section 2.7).

Section 2.6 leaves the explicit Runge-Kutta scheme for these terms
unnamed.  Forward Euler is the default; the
strong-stability-preserving schemes of Shu and Osher (J. Comput. Phys. 77,
1988) of order 2 and 3 are the alternatives: each stage is the forward-Euler
update above (clamps and wall omega included) from the previous stage, and
the stages are convex combinations with the state at the start:
  RK2: u1 = E(u0);  u = 1/2 u0 + 1/2 E(u1)
  RK3: u1 = E(u0);  u2 = 3/4 u0 + 1/4 E(u1);  u = 1/3 u0 + 2/3 E(u2)
with omega set to its wall value again after each combination.
"""
import numpy as np

from . import model
from .geometry import (U, V, W, T, K, OM, FK_WALL, FK_SOLID, D_op, cell_gradient)

TRANSPORTED = (U, V, W, T, K, OM)


def _nut_faces(nut, axis, kind):
    pad = [(0, 0)] * 3
    pad[axis] = (1, 1)
    e = np.pad(nut, pad, mode="edge")
    n = e.shape[axis]
    L = np.take(e, range(0, n - 1), axis=axis)
    R = np.take(e, range(1, n), axis=axis)
    f = 0.5 * (L + R)
    f[(kind == FK_WALL) | (kind == FK_SOLID)] = 0.0
    return f


def explicit_rhs(geo, state):
    """d phi / dt for phi in (u, v, w, T, k, omega) without the destruction terms."""
    s = geo.spec
    nu = s.nu
    phis = dict(zip(TRANSPORTED, state))
    k, om = phis[K], phis[OM]
    nut = np.where(geo.fluid, model.nu_t(k, om, nu), 0.0)
    gam_mol = {U: nu, V: nu, W: nu, T: geo.alpha, K: nu, OM: nu}
    sigma = {U: 1.0, V: 1.0, W: 1.0, T: s.Prt, K: s.sigma_k, OM: s.sigma_w}
    rhs = {f: np.zeros(geo.shape, dtype=np.result_type(*state)) for f in TRANSPORTED}
    vel = (phis[U], phis[V], phis[W])
    for axis in range(3):
        if geo.shape[axis] == 1:
            continue            # empty direction of a 2D case: every flux across it cancels
        h = geo.h[axis]
        UL, UR, kind = geo.face_states(vel[axis], axis, axis)
        u_face = 0.5 * (UL + UR)                             # L * BC(u)
        nut_f = _nut_faces(nut, axis, kind)
        kL, kR, _ = geo.face_states(k, K, axis)
        for f in TRANSPORTED:
            pL, pR, _ = geo.face_states(phis[f], f, axis)
            up = np.where(np.real(u_face) >= 0.0, pL, pR)    # I[u_face >= 0] selects W+
            flux = -(up * u_face) + (gam_mol[f] + nut_f / sigma[f]) * (pR - pL) / h
            if f == axis:
                flux = flux - (2.0 / 3.0) * 0.5 * (kL + kR)
            flux[kind == FK_SOLID] = 0.0
            rhs[f] += D_op(flux, axis, h)
    grads = [cell_gradient(geo, phis[f], f) for f in (U, V, W)]
    S, _ = model.strain_rotation(grads)
    S2 = model.strain_magnitude_sq(S)
    with np.errstate(divide="ignore", invalid="ignore"):   # k = 0 in solid cells, masked below
        rhs[K] += model.production_k(k, om, nu, S2)
        rhs[OM] += model.production_omega(k, om, nu, S2)
    if s.buoyancy:
        for i, f in enumerate((U, V, W)):
            if s.gravity[i] != 0.0:
                rhs[f] += -s.gravity[i] * s.beta_T * (phis[T] - s.T_ref)
    for f in TRANSPORTED:
        rhs[f][geo.solid] = 0.0
    return [rhs[f] for f in TRANSPORTED]


def wall_omega(geo):
    """Per fluid cell, the wall value 6 nu / (beta_i d^2) for the nearest
    wall face (d = half the cell width normal to it), or 0 if none."""
    out = np.zeros(geo.shape)
    for axis in range(3):
        if geo.shape[axis] == 1:
            continue
        _, _, kind = geo.face_states(np.zeros(geo.shape), U, axis)
        n = kind.shape[axis]
        west = np.take(kind, range(0, n - 1), axis=axis) == FK_WALL
        east = np.take(kind, range(1, n), axis=axis) == FK_WALL
        val = model.omega_wall(geo.spec.nu, 0.5 * geo.h[axis])
        out = np.where(west | east, np.maximum(out, val), out)
    out[geo.solid] = 0.0
    return out


def explicit_stage(geo, state, dt):
    """Forward-Euler update of (u, v, w, T, k, omega) by the explicit terms."""
    rhs = explicit_rhs(geo, state)
    new = [np.where(geo.fluid, phi + dt * r, phi) for phi, r in zip(state, rhs)]
    u, v, w, T_, k, om = new
    # (decisions on the real part: the same values for real fields, and one branch
    # for the complex-step derivatives of the adjoint)
    k = np.where(geo.fluid, np.where(np.real(k) > model.K_MIN, k, model.K_MIN), k)
    om = np.where(geo.fluid, np.where(np.real(om) > model.OMEGA_MIN, om, model.OMEGA_MIN), om)
    ow = wall_omega(geo)
    om = np.where(ow > 0.0, ow, om)
    return [u, v, w, T_, k, om]


def _combine(geo, a, x0, b, y):
    """a x0 + b y in fluid cells (solid cells keep x0), wall omega set again."""
    out = [np.where(geo.fluid, a * p + b * q, p) for p, q in zip(x0, y)]
    ow = wall_omega(geo)
    out[5] = np.where(ow > 0.0, ow, out[5])
    return out


def explicit_stage_rk(geo, state, dt, stages=1):
    """The explicit terms over dt by forward Euler (stages = 1) or the
    strong-stability-preserving Runge-Kutta scheme of order 2 or 3 (Shu and
    Osher) built from forward-Euler stages."""
    if stages == 1:
        return explicit_stage(geo, state, dt)
    u1 = explicit_stage(geo, state, dt)
    if stages == 2:
        return _combine(geo, 0.5, state, 0.5, explicit_stage(geo, u1, dt))
    if stages == 3:
        u2 = _combine(geo, 0.75, state, 0.25, explicit_stage(geo, u1, dt))
        return _combine(geo, 1.0 / 3.0, state, 2.0 / 3.0, explicit_stage(geo, u2, dt))
    raise ValueError("stages must be 1, 2 or 3")
