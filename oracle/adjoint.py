"""Adjoints (vector-Jacobian products) of the stages of the step, for a
differentiable step: the pressure projection u* -> (u^{n+1}, p), the
semi-implicit destruction step and the explicit stage.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The map (Section 2.4, Algorithm 1, with the projection reading of the step):
    b = -div(u*) / dt          (face velocities L * BC(u*), Eq. pc_residual)
    A p = b                    (solved exactly here, not to a tolerance)
    u^{n+1} = u* - dt G p      (G the cell gradient L * D * BC(p))
is affine in u*: inlet ghosts add constants, everything else is linear.  Its
Jacobian J is therefore one fixed matrix, and the vector-Jacobian product of
a cotangent (ubar, vbar, wbar, pbar) is J^T applied to it.

J is built from the forward oracle functions by the definition.  The three
local pieces (b(u*), the gradient term of the projection, A) reach only the
cells within one index of a cell along each axis, so evaluating each piece
on 27 probe fields -- all cells with (i mod 3, j mod 3, k mod 3) equal to one
colour set to 1 -- recovers every matrix entry exactly: an output cell sees
exactly one probed cell within its reach (Curtis, Powell and Reid, 1974).
A^{-1} is a sparse direct solve on the fluid cells (solid cells hold p = 0).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .poisson import apply_A, poisson_rhs, project


def local_jacobian(apply, n_in, shape, reach=1):
    """Matrix of the affine map `apply` (a list of n_in arrays of `shape` -> a
    list of output arrays) whose output entry q depends only on inputs within
    `reach` indices of q along each axis (probes with period 2 reach + 1 per
    axis).  An output may have one more entry than `shape` along an axis (face
    values: face q lies between cells q - 1 and q).  Rows and columns are
    array-major, each array in numpy C order.  The matrix is checked against the
    map on a random input."""
    N = int(np.prod(shape))
    P = 2 * reach + 1
    zero = [np.zeros(shape) for _ in range(n_in)]
    y0 = apply(zero)
    n_out = len(y0)
    out_sizes = [int(np.prod(y.shape)) for y in y0]
    out_off = np.concatenate([[0], np.cumsum(out_sizes)])
    idx = np.indices(shape)
    rows, cols, vals = [], [], []
    for fi in range(n_in):
        for colour in np.ndindex(P, P, P):
            mask = np.ones(shape, dtype=bool)
            for a in range(3):
                mask &= (idx[a] % P) == colour[a]
            if not mask.any():
                continue
            x = [np.zeros(shape) for _ in range(n_in)]
            x[fi][mask] = 1.0
            y = apply(x)
            for fo in range(n_out):
                # for every output entry, the probed cell within its reach: along each
                # axis the index among q - reach .. q + reach with the colour's residue
                oidx = np.indices(y0[fo].shape)
                src = []
                ok = np.ones(y0[fo].shape, dtype=bool)
                for a in range(3):
                    q = oidx[a]
                    s = q - reach + ((colour[a] - (q - reach)) % P)
                    ok &= (s >= 0) & (s < shape[a])
                    src.append(np.clip(s, 0, shape[a] - 1))
                src_flat = np.ravel_multi_index(src, shape)
                d = y[fo] - y0[fo]
                nz = (d != 0.0)
                assert not (nz & ~ok).any(), "output outside the reach of its probe"
                r = np.flatnonzero(nz)
                rows.append(out_off[fo] + r)
                cols.append(fi * N + src_flat.ravel()[r])
                vals.append(d.ravel()[r])
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(int(out_off[-1]), n_in * N))
    rng = np.random.default_rng(12345)
    x = [rng.standard_normal(shape) for _ in range(n_in)]
    want = np.concatenate([(a - b).ravel() for a, b in zip(apply(x), y0)])
    got = J @ np.concatenate([a.ravel() for a in x])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want))), "Jacobian check"
    return J


class ProjectionAdjoint:
    """J^T of u* -> (u^{n+1}, v^{n+1}, w^{n+1}, p) on one case's level-0 grid."""

    def __init__(self, geo, lev0, dt):
        shape = geo.shape
        self.shape = shape
        self.N = N = int(np.prod(shape))
        self.JB = local_jacobian(lambda x: [poisson_rhs(geo, x[0], x[1], x[2], dt)], 3, shape)
        z = np.zeros(shape)
        self.JPp = local_jacobian(lambda x: project(geo, lev0, z, z, z, x[0], dt), 1, shape)
        self.JPu = local_jacobian(lambda x: project(geo, lev0, x[0], x[1], x[2], z, dt), 3, shape)
        A = local_jacobian(lambda x: [apply_A(lev0, x[0])], 1, shape)
        self.fluid = np.flatnonzero(lev0.fluid.ravel())
        self.AFF = A[self.fluid][:, self.fluid].tocsc()
        self._luT = spla.splu(self.AFF.T.tocsc())
        self._lu = spla.splu(self.AFF)

    def _solve(self, b, transpose=False):
        out = np.zeros(self.N)
        lu = self._luT if transpose else self._lu
        out[self.fluid] = lu.solve(b[self.fluid])
        return out

    def forward_linear(self, du, dv, dw):
        """J applied to a velocity perturbation: (du', dv', dw', dp)."""
        x = np.concatenate([a.ravel() for a in (du, dv, dw)])
        dp = self._solve(self.JB @ x)
        y = self.JPu @ x + self.JPp @ dp
        N = self.N
        return [y[i * N:(i + 1) * N].reshape(self.shape) for i in range(3)] + [dp.reshape(self.shape)]

    def vjp(self, ubar, vbar, wbar, pbar=None):
        """J^T (ubar, vbar, wbar, pbar): the cotangent of u*, v*, w*."""
        ybar = np.concatenate([a.ravel() for a in (ubar, vbar, wbar)])
        q = self.JPp.T @ ybar
        if pbar is not None:
            q = q + pbar.ravel()
        xbar = self.JPu.T @ ybar + self.JB.T @ self._solve(q, transpose=True)
        N = self.N
        return [xbar[i * N:(i + 1) * N].reshape(self.shape) for i in range(3)]


class DestructionAdjoint:
    """J^T of the semi-implicit destruction step (u, v, w, k, omega) -> (k', omega')
    over dt (Section 2.5, Algorithm 4), linearised at a given state.

    Per fluid cell the step is a function of k, omega and the cell gradients
    G = grad(u, v, w), grad k, grad omega; those gradients are affine stencil
    maps of the fields (their Jacobians come from local_jacobian on
    geometry.cell_gradient).  The partial derivatives of the pointwise part
    are written out below from the forward formulas of oracle/model.py:
      omega_s = max(omega, eps), Re_t = k / (nu omega_s), x = Re_t / R_beta,
      beta* = beta*_inf (4/15 + x^4) / (1 + x^4),
      chi_k = (grad k . grad omega) / omega_s^3,
      f_beta* = 1 (chi_k <= 0) or (1 + 680 chi_k^2) / (1 + 400 chi_k^2),
      k' = k / (1 + dt beta* f_beta* omega),
      chi_w = |tr(Omega Omega S)| / (beta*_inf omega_s)^3,
      f_beta = (1 + 70 chi_w) / (1 + 80 chi_w),
      omega' = omega / (1 + dt beta f_beta omega).
    Solid cells keep k and omega (identity)."""

    def __init__(self, geo, dt, state):
        from .geometry import U, V, W, K, OM, cell_gradient
        self.geo, self.dt = geo, dt
        shape = geo.shape
        self.shape = shape
        self.N = int(np.prod(shape))
        fields = (U, V, W, K, OM)
        self.Jg = [local_jacobian(lambda x, f=f: cell_gradient(geo, x[0], f), 1, shape) for f in fields]
        u, v, w, k, om = [np.asarray(a, dtype=np.float64) for a in state]
        grads = [cell_gradient(geo, phi, f) for phi, f in zip((u, v, w, k, om), fields)]
        self.G = np.stack([np.stack(grads[i], axis=0) for i in range(3)], axis=0)    # (3, 3, ...)
        self.gk = np.stack(grads[3], axis=0)
        self.gw = np.stack(grads[4], axis=0)
        self.k, self.om = k, om

    def _partials(self):
        from . import model as m
        nu, dt = self.geo.spec.nu, self.dt
        k, om, G, gk, gw = self.k, self.om, self.G, self.gk, self.gw
        oms = np.maximum(om, m.EPS_OMEGA)
        doms = (om > m.EPS_OMEGA).astype(np.float64)                # d omega_s / d omega
        # k' = k / Dk
        re = k / (nu * oms)
        dre_dk = 1.0 / (nu * oms)
        dre_dom = -re / oms * doms
        x = re / m.R_BETA
        x4 = x ** 4
        bs = m.BETA_STAR_INF * (4.0 / 15.0 + x4) / (1.0 + x4)
        dbs_dre = m.BETA_STAR_INF * (11.0 / 15.0) / (1.0 + x4) ** 2 * 4.0 * x ** 3 / m.R_BETA
        dot = np.sum(gk * gw, axis=0)
        chik = dot / oms ** 3
        pos = chik > 0.0
        fbs = np.where(pos, (1.0 + 680.0 * chik ** 2) / (1.0 + 400.0 * chik ** 2), 1.0)
        dfbs = np.where(pos, 560.0 * chik / (1.0 + 400.0 * chik ** 2) ** 2, 0.0)
        Dk = 1.0 + dt * bs * fbs * om
        c = -k / Dk ** 2 * dt                                       # d k' / d (beta* f_beta* omega)
        dk_dk = 1.0 / Dk + c * fbs * om * dbs_dre * dre_dk
        dk_dom = c * (fbs * om * dbs_dre * dre_dom + bs * om * dfbs * (-3.0 * chik / oms * doms) + bs * fbs)
        dk_dgk = c * bs * om * dfbs * gw / oms ** 3
        dk_dgw = c * bs * om * dfbs * gk / oms ** 3
        # omega' = omega / Dw
        S = 0.5 * (G + np.swapaxes(G, 0, 1))
        O = 0.5 * (G - np.swapaxes(G, 0, 1))
        OO = np.einsum("ij...,jk...->ik...", O, O)
        T = np.einsum("ik...,ki...->...", OO, S)
        dT_dS = OO                                                  # d tr(O O S) / d S_ab = (O O)_ba = (O O)_ab
        dT_dO = -(np.einsum("ij...,jk...->ik...", S, O) + np.einsum("ij...,jk...->ik...", O, S))
        # chain to G: dS_ab/dG = (delta + transpose)/2, dO_ab/dG = (delta - transpose)/2
        dT_dG = 0.5 * (dT_dS + np.swapaxes(dT_dS, 0, 1)) + 0.5 * (dT_dO - np.swapaxes(dT_dO, 0, 1))
        den = (m.BETA_STAR_INF * oms) ** 3
        chiw = np.abs(T) / den
        dchiw_dG = np.sign(T) / den * dT_dG
        dchiw_dom = -3.0 * chiw / oms * doms
        fb = (1.0 + 70.0 * chiw) / (1.0 + 80.0 * chiw)
        dfb = -10.0 / (1.0 + 80.0 * chiw) ** 2
        Dw = 1.0 + dt * m.BETA * fb * om
        cw = -om / Dw ** 2 * dt * m.BETA                            # d omega' / d (f_beta omega)
        dw_dom = 1.0 / Dw + cw * (fb + om * dfb * dchiw_dom)
        dw_dG = cw * om * dfb * dchiw_dG
        return dk_dk, dk_dom, dk_dgk, dk_dgw, dw_dom, dw_dG

    def vjp(self, kbar, ombar):
        """Cotangents of (u, v, w, k, omega) for cotangents (kbar, ombar) of (k', omega')."""
        fluid = self.geo.fluid
        kb = np.where(fluid, kbar, 0.0)
        wb = np.where(fluid, ombar, 0.0)
        dk_dk, dk_dom, dk_dgk, dk_dgw, dw_dom, dw_dG = self._partials()
        out_k = kb * dk_dk + np.where(fluid, 0.0, kbar)
        out_om = kb * dk_dom + wb * dw_dom + np.where(fluid, 0.0, ombar)
        Gbar = wb * dw_dG                                           # (3, 3, ...)
        gkbar = kb * dk_dgk
        gwbar = kb * dk_dgw

        def back(J, gbar):   # gbar: (3, ...) cotangent of a gradient -> cotangent of its field
            return (J.T @ np.concatenate([gbar[a].ravel() for a in range(3)])).reshape(self.shape)

        ub = back(self.Jg[0], Gbar[0])
        vb = back(self.Jg[1], Gbar[1])
        wbv = back(self.Jg[2], Gbar[2])
        out_k = out_k + back(self.Jg[3], gkbar)
        out_om = out_om + back(self.Jg[4], gwbar)
        return ub, vb, wbv, out_k, out_om


class ExplicitAdjoint:
    """J^T of the explicit stage (u, v, w, T, k, omega) -> its update over dt
    (forward Euler, or the Runge-Kutta schemes of rk_stages 2 and 3),
    linearised at a given state.

    The Jacobian is taken from the forward oracle itself by complex-step
    differentiation (Squire and Trapp, SIAM Review 40, 1998): for a real
    direction d, Im F(x + i h d) / h with h = 1e-30 is the directional
    derivative J d to rounding, with no subtractive cancellation.  The forward
    functions are complex-safe: branch decisions (the upwind switch, the
    clamps, max(omega, eps)) compare real parts, as numpy orders complex
    numbers by their real part first.  A forward-Euler stage reaches one cell
    along each axis and s stages reach s cells, so colour probes of period
    2 s + 1 recover every entry of J.  Clamped values and wall omega get zero
    derivatives, as the forward sets them to constants."""

    H = 1e-30

    def __init__(self, geo, dt, state, stages=1):
        from .transport import explicit_stage_rk
        self.shape = geo.shape
        self.N = int(np.prod(geo.shape))
        x = [np.asarray(a, dtype=np.float64) for a in state]

        def jvp(d):
            y = explicit_stage_rk(geo, [a + 1j * self.H * b for a, b in zip(x, d)], dt, stages)
            return [np.imag(v) / self.H for v in y]

        self.J = local_jacobian(jvp, 6, self.shape, reach=stages)

    def jvp(self, *d):
        y = self.J @ np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in d])
        return [y[i * self.N:(i + 1) * self.N].reshape(self.shape) for i in range(6)]

    def vjp(self, *ybar):
        """Cotangents of (u, v, w, T, k, omega) for cotangents of the updated fields."""
        x = self.J.T @ np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in ybar])
        return [x[i * self.N:(i + 1) * self.N].reshape(self.shape) for i in range(6)]


class StepAdjoint:
    """J^T of one whole time step (Section 2.6) at a given state, with the
    pressure solve exact and dt fixed:
        s1 = D(x0), s2 = E(s1), s3 = D(s2)     (destruction dt/2, explicit dt,
                                                 destruction dt/2; D changes k and
                                                 omega only)
        (u, v, w, p) = Pi(u, v, w of s3)       (right-hand side, solve, projection)
    with T, k and omega of s3 passing to the output.  The cotangent of the
    output (u, v, w, p, T, k, omega) runs back through the stage adjoints
    above in reverse order."""

    def __init__(self, geo, dt, state, stages=1):
        from .destruction import destruction_step
        from .transport import explicit_stage_rk
        self.geo = geo
        x0 = [np.asarray(a, dtype=np.float64) for a in state]
        u, v, w, T, k, om = x0
        self.D1 = DestructionAdjoint(geo, 0.5 * dt, [u, v, w, k, om])
        k, om = destruction_step(geo, u, v, w, k, om, 0.5 * dt)
        s1 = [u, v, w, T, k, om]
        self.E = ExplicitAdjoint(geo, dt, s1, stages)
        u, v, w, T, k, om = explicit_stage_rk(geo, s1, dt, stages)
        self.D2 = DestructionAdjoint(geo, 0.5 * dt, [u, v, w, k, om])
        self.P = ProjectionAdjoint(geo, geo.level0, dt)

    @staticmethod
    def _through_destruction(D, bar):
        """bar = cotangents of (u, v, w, T, k, omega) after D -> before D."""
        u, v, w, T, k, om = bar
        du, dv, dw, dk, dom = D.vjp(k, om)
        return [u + du, v + dv, w + dw, T, dk, dom]

    def vjp(self, ubar, vbar, wbar, pbar, Tbar, kbar, ombar):
        """Cotangents of (u, v, w, T, k, omega) at the start of the step."""
        bu, bv, bw = self.P.vjp(ubar, vbar, wbar, pbar)
        bar = [bu, bv, bw, Tbar, kbar, ombar]
        bar = self._through_destruction(self.D2, bar)
        bar = self.E.vjp(*bar)
        return self._through_destruction(self.D1, bar)


def _face_diff_T(rbar, axis, h):
    """Transpose of D_op along `axis`: cell cotangents -> face cotangents."""
    shape = list(rbar.shape)
    shape[axis] += 1
    fb = np.zeros(shape)
    hi = [slice(None)] * 3
    lo = [slice(None)] * 3
    hi[axis] = slice(1, None)
    lo[axis] = slice(0, -1)
    fb[tuple(hi)] += rbar / h
    fb[tuple(lo)] -= rbar / h
    return fb


def explicit_vjp_by_hand(geo, state, dt, ybar):
    """J^T ybar of one forward-Euler explicit stage with every partial derivative
    written out: an independent derivation of ExplicitAdjoint(stages=1), and the
    arithmetic a GPU kernel of the adjoint follows.

    Per face along axis a, with u_f = (U_L + U_R)/2, phi_up = phi_L if u_f >= 0 else
    phi_R and Gamma = gamma + nu_t,f / sigma, the flux -phi_up u_f + Gamma (phi_R -
    phi_L)/h (- (k_L + k_R)/3 for the momentum component along a) has the partials
    d/d phi_up = -u_f, d/d u_f = -phi_up, d/d phi_R = -d/d phi_L = Gamma / h,
    d/d nu_t,f = (phi_R - phi_L) / (sigma h), d/d k_L = d/d k_R = -1/3.  The face
    states (ghosts of Section 2.7) and the face eddy viscosity are affine maps of the
    cell values, transposed by colour probing.  Sources: G_k = nu_t S^2 (dS^2/dG_ab =
    4 S_ab), G_omega = alpha (omega / k) G_k, buoyancy -g_i beta_T (T - T_ref).  The
    update phi + dt rhs passes nothing from clamped k, omega or the wall omega."""
    from . import model as m
    from .geometry import U, V, W, T, K, OM, FK_SOLID, cell_gradient
    from .transport import TRANSPORTED, _nut_faces, explicit_rhs, wall_omega
    s = geo.spec
    nu = s.nu
    shape = geo.shape
    x = [np.asarray(a, dtype=np.float64) for a in state]
    phis = dict(zip(TRANSPORTED, x))
    pos = {f: i for i, f in enumerate(TRANSPORTED)}              # field id -> state slot
    k, om = phis[K], phis[OM]
    fluid = geo.fluid
    gam_mol = {U: nu, V: nu, W: nu, T: geo.alpha, K: nu, OM: nu}
    sigma = {U: 1.0, V: 1.0, W: 1.0, T: s.Prt, K: s.sigma_k, OM: s.sigma_w}
    # the update: which cells pass a derivative
    rhs = explicit_rhs(geo, x)
    live_k = fluid & (k + dt * rhs[4] > m.K_MIN)
    live_o = fluid & (om + dt * rhs[5] > m.OMEGA_MIN) & ~(wall_omega(geo) > 0.0)
    live = [fluid, fluid, fluid, fluid, live_k, live_o]
    xbar = [np.where(fluid, 0.0, yb) + np.where(lv, yb, 0.0) for yb, lv in zip(ybar, live)]
    rbar = [np.where(lv, dt * yb, 0.0) for yb, lv in zip(ybar, live)]
    nut = np.where(fluid, m.nu_t(k, om, nu), 0.0)
    nutbar = np.zeros(shape)

    def fs_T(field, axis, Lb, Rb):
        J = local_jacobian(lambda z: list(geo.face_states(z[0], field, axis)[:2]), 1, shape)
        return (J.T @ np.concatenate([Lb.ravel(), Rb.ravel()])).reshape(shape)

    for axis in range(3):
        if shape[axis] == 1:
            continue
        h = geo.h[axis]
        UL, UR, kind = geo.face_states(x[axis], axis, axis)
        u_face = 0.5 * (UL + UR)
        nut_f = _nut_faces(nut, axis, kind)
        solid_f = kind == FK_SOLID
        ufb = np.zeros(u_face.shape)
        nfb = np.zeros(u_face.shape)
        kLb = np.zeros(u_face.shape)
        kRb = np.zeros(u_face.shape)
        upL = u_face >= 0.0
        for f in TRANSPORTED:
            pL, pR, _ = geo.face_states(phis[f], f, axis)
            up = np.where(upL, pL, pR)
            fb = _face_diff_T(rbar[pos[f]], axis, h)
            fb[solid_f] = 0.0
            gam = gam_mol[f] + nut_f / sigma[f]
            pLb = np.where(upL, -u_face * fb, 0.0) - gam / h * fb
            pRb = np.where(upL, 0.0, -u_face * fb) + gam / h * fb
            xbar[pos[f]] = xbar[pos[f]] + fs_T(f, axis, pLb, pRb)
            ufb += -up * fb
            nfb += (pR - pL) / (h * sigma[f]) * fb
            if f == axis:
                kLb += -fb / 3.0
                kRb += -fb / 3.0
        xbar[axis] = xbar[axis] + fs_T(axis, axis, 0.5 * ufb, 0.5 * ufb)
        xbar[pos[K]] = xbar[pos[K]] + fs_T(K, axis, kLb, kRb)
        JN = local_jacobian(lambda z: [_nut_faces(z[0], axis, kind)], 1, shape)
        nutbar += (JN.T @ nfb.ravel()).reshape(shape)
    # sources
    G = np.stack([np.stack(cell_gradient(geo, x[i], f), axis=0) for i, f in enumerate((U, V, W))], axis=0)
    S = 0.5 * (G + np.swapaxes(G, 0, 1))
    S2 = 2.0 * np.sum(S * S, axis=(0, 1))
    oms = np.where(om > m.EPS_OMEGA, om, m.EPS_OMEGA)
    doms = (om > m.EPS_OMEGA).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        re = k / (nu * oms)
        dre_dk = 1.0 / (nu * oms)
        dre_dom = -re / oms * doms
        r = re / m.R_K
        ast = m.ALPHA_STAR_INF * (m.ALPHA_STAR_0 + r) / (1.0 + r)
        dast = m.ALPHA_STAR_INF * (1.0 - m.ALPHA_STAR_0) / (m.R_K * (1.0 + r) ** 2)
        nut_c = ast * k / oms
        dnut_dk = ast / oms + k / oms * dast * dre_dk
        dnut_dom = -ast * k / oms ** 2 * doms + k / oms * dast * dre_dom
        rw = re / m.R_OMEGA
        A = (m.ALPHA_0 + rw) / (1.0 + rw)
        dA = (1.0 - m.ALPHA_0) / (m.R_OMEGA * (1.0 + rw) ** 2)
        ac = m.ALPHA_INF * A / ast
        dac = m.ALPHA_INF * (dA / ast - A * dast / ast ** 2)
        Gk = nut_c * S2
        q = ac * om / k                                             # G_omega = q G_k
        dq_dk = dac * dre_dk * om / k - ac * om / k ** 2
        dq_dom = dac * dre_dom * om / k + ac / k
    rk, ro = rbar[4], rbar[5]
    Gkb = np.where(fluid, rk + ro * q, 0.0)
    xbar[4] = xbar[4] + np.where(fluid, ro * Gk * dq_dk, 0.0)
    xbar[5] = xbar[5] + np.where(fluid, ro * Gk * dq_dom, 0.0)
    nutbar = nutbar + np.where(fluid, Gkb * S2, 0.0)
    S2b = np.where(fluid, Gkb * nut_c, 0.0)
    Gbar = 4.0 * S * S2b
    xbar[4] = xbar[4] + np.where(fluid, nutbar * dnut_dk, 0.0)
    xbar[5] = xbar[5] + np.where(fluid, nutbar * dnut_dom, 0.0)
    for i, f in enumerate((U, V, W)):
        J = local_jacobian(lambda z, f=f: cell_gradient(geo, z[0], f), 1, shape)
        xbar[i] = xbar[i] + (J.T @ np.concatenate([Gbar[i, a].ravel() for a in range(3)])).reshape(shape)
    if s.buoyancy:
        for i in range(3):
            if s.gravity[i] != 0.0:
                xbar[3] = xbar[3] + np.where(fluid, -s.gravity[i] * s.beta_T * rbar[i], 0.0)
    return xbar
