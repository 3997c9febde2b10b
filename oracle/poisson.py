"""Pressure Poisson equation, multigrid and projection (Section 2.4, Algorithm 1).

  b        = -(1/dt) (D_x * L_x * BC_x(u*) + D_y * ... + D_z * ...)   (Eq. pc_residual)
  A p      = -Laplacian_h p with one ghost layer (Eq. neg_lap_discretize
             and the printed 3x3x3 kernel)
  smoother   p <- p + w_J D^{-1} (b - A p), D = sum_d 2 / h_d^2 scalar
             (Eq. jacobi_pc; weighted); smoother 1 (an addition): one weight
             per sweep, the reciprocals of the Chebyshev roots on [1/4, 2]
  RES        mean of the 2x2x2 children (Eq. restriction)
  PROL       cell-centred trilinear interpolation, 3/4 parent + 1/4
             neighbour per axis (Eq. prolongation); beyond a domain face
             the neighbour is the coarse level's ghost (Section 2.7 rules:
             the cell itself, negated across a zero-value face)
  V-cycle    pre-smooth, restrict the residual, recurse, prolong and
             correct, post-smooth; exact dense solve on the coarsest level;
             coarse_sweeps > 0 sets both sweep counts on the levels below
             the finest (a tuning choice, not in the paper)
  krylov 1   flexible CG with one kept direction around V-cycles (each
             V-cycle from zero on A z = r gives a direction, A-orthogonalised
             against the previous one, and the step minimising the A-norm of
             the error along it)
  Algorithm 1 (mg_variant 1): the fine residual restricted straight down,
             one unweighted Jacobi per coarse level on the way up (A and D
             with the fine spacing), nearest upsampling, a final unweighted
             Jacobi sweep on p
  projection u = u* - dt G p, G the cell-centred gradient L * D * BC(p)

Solid cells hold zero pressure and are excluded from every norm.
"""
import copy

import numpy as np

from .geometry import U, V, W, FK_SOLID, D_op, L_op, pressure_face_states


# ------------------------------------------------------------------ level 0
def poisson_rhs(geo, u, v, w, dt):
    """b = -div(u*) / dt with face velocities L * BC(u*) (the right-hand side of Algorithm 1; Eq. pc_residual)."""
    div = np.zeros(geo.shape)
    for axis, (phi, f) in enumerate(((u, U), (v, V), (w, W))):
        if geo.shape[axis] == 1:
            continue
        L, R, kind = geo.face_states(phi, f, axis)
        uf = 0.5 * (L + R)
        uf[kind == FK_SOLID] = 0.0
        div += D_op(uf, axis, geo.h[axis])
    b = -div / dt
    b[geo.solid] = 0.0
    return b


def pressure_gradient(lev, p):
    """Cell-centred gradient L_j * D_j * BC_j(p) with the pressure ghosts."""
    g = []
    for axis in range(3):
        if lev.shape[axis] == 1:
            g.append(np.zeros(lev.shape))
            continue
        L, R = pressure_face_states(p, lev, axis)
        g.append(L_op((R - L) / lev.h[axis], axis))
    return g


def project(geo, lev0, u, v, w, p, dt):
    """u = u* - dt grad p on fluid cells (projection step of Section 2.4)."""
    g = pressure_gradient(lev0, p)
    out = []
    for phi, gg in zip((u, v, w), g):
        out.append(np.where(geo.fluid, phi - dt * gg, phi))
    return out


def face_divergence(geo, lev0, u, v, w, p, dt):
    """Divergence of the face fluxes u*_f - dt (p_R - p_L)/h: equals dt (A p - b)."""
    div = np.zeros(geo.shape)
    for axis, (phi, f) in enumerate(((u, U), (v, V), (w, W))):
        if geo.shape[axis] == 1:
            continue
        L, R, kind = geo.face_states(phi, f, axis)
        pL, pR = pressure_face_states(p, lev0, axis)
        uf = 0.5 * (L + R) - dt * (pR - pL) / geo.h[axis]
        uf[kind == FK_SOLID] = 0.0
        div += D_op(uf, axis, geo.h[axis])
    div[geo.solid] = 0.0
    return div


# ------------------------------------------------------------------ operators
def apply_A(lev, p):
    """A p = -sum_d D_d * (D_d * BC_d(p)) on fluid cells."""
    out = np.zeros(lev.shape)
    for axis in range(3):
        if lev.shape[axis] == 1:
            continue
        L, R = pressure_face_states(p, lev, axis)
        out -= D_op((R - L) / lev.h[axis], axis, lev.h[axis])
    out[lev.solid] = 0.0
    return out


def residual(lev, p, b):
    r = b - apply_A(lev, p)
    r[lev.solid] = 0.0
    return r


def jacobi_weight(lev, spec):
    if spec.jacobi_weight > 0:
        return spec.jacobi_weight
    return 6.0 / 7.0 if all(lev.active) else 4.0 / 5.0


def chebyshev_weights(n, lo=0.25, hi=2.0):
    """Weights of n Jacobi sweeps whose error polynomial prod_i (1 - w_i x) in x = lambda(D^-1 A)
    is the degree-n Chebyshev polynomial of the interval [lo, hi], scaled to 1 at x = 0: w_i is
    the reciprocal of its i-th root, (hi + lo)/2 + (hi - lo)/2 cos((2i - 1) pi / (2n)), largest
    root first.  hi = 2 bounds the spectrum of D^-1 A (Gershgorin, with the scalar D of Eq.
    jacobi_pc); lo = 1/4 lies below the high-frequency band of full coarsening (1/3 in 3D, 1/2 in
    2D), so the sweeps damp that band by 1 / T_n((hi + lo)/(hi - lo)) at least."""
    i = np.arange(1, n + 1)
    roots = (hi + lo) / 2 + (hi - lo) / 2 * np.cos((2 * i - 1) * np.pi / (2 * n))
    return list(1.0 / roots)


def sweep_weights(lev, spec, n, post):
    """The weights of n smoothing sweeps: the constant w_J (smoother 0), or (smoother 1, an
    addition to the paper's fixed weight) the Chebyshev weights, in reverse order after the
    coarse correction so that the post-smoother mirrors the pre-smoother."""
    if getattr(spec, "smoother", 0) == 1:
        w = chebyshev_weights(n)
        return w[::-1] if post else w
    return [jacobi_weight(lev, spec)] * n


def smooth(lev, p, b, sweeps, wJ):
    """Weighted Jacobi: p <- p + w_J (b - A p) / D (Eq. jacobi_pc); wJ is one weight for every
    sweep or a list of one weight per sweep."""
    D = lev.diag()
    ws = list(wJ) if np.ndim(wJ) else [wJ] * sweeps
    assert len(ws) == sweeps
    for w in ws:
        p = np.where(lev.fluid, p + w * residual(lev, p, b) / D, 0.0)
    return p


def restrict(lev, r):
    """RES: mean of the children (2 per active axis)."""
    f = tuple(2 if a else 1 for a in lev.active)
    c = tuple(n // ff for n, ff in zip(lev.shape, f))
    return r.reshape(c[0], f[0], c[1], f[1], c[2], f[2]).mean(axis=(1, 3, 5))


def ghost_pad(lev, e):
    """The coarse field with one ghost layer on each side of every active axis,
    by the pressure rules of Section 2.7 applied on the level: the cell's own
    value across a zero-gradient face, its negative across a zero-value
    (outlet) face.  Axes are padded in turn, so an edge or corner ghost carries
    the signs of all its faces (the face masks extend into the ghost layers of
    the axes padded before by their edge values)."""
    g = e
    for axis in range(3):
        if not lev.active[axis]:
            continue
        n = g.shape[axis]
        lo = np.take(g, [0], axis=axis)
        hi = np.take(g, [n - 1], axis=axis)
        masks = []
        for face in (2 * axis, 2 * axis + 1):
            m = lev.dirichlet[face]
            # the mask's two axes are the tangential axes in increasing order
            tang = [a for a in range(3) if a != axis]
            pad = [(1, 1) if (lev.active[a] and a < axis) else (0, 0) for a in tang]
            m = np.pad(m, pad, mode="edge")
            masks.append(np.expand_dims(m, axis))
        g = np.concatenate([np.where(masks[0], -lo, lo), g, np.where(masks[1], -hi, hi)], axis=axis)
    return g


def prolong(coarse_lev, coarse, fine_shape):
    """PROL: cell-centred trilinear interpolation (Eq. prolongation): per
    active axis, fine cell = 3/4 parent + 1/4 the parent's neighbour on the
    fine cell's side.  A neighbour beyond a domain face is the coarse level's
    ghost (ghost_pad)."""
    e = ghost_pad(coarse_lev, coarse)
    for axis in range(3):
        if not coarse_lev.active[axis]:
            continue
        nf = fine_shape[axis]
        i_f = np.arange(nf)
        parent = i_f // 2 + 1                                   # +1: the ghost layer
        nb = parent + np.where(i_f % 2 == 0, -1, 1)
        e = 0.75 * np.take(e, parent, axis=axis) + 0.25 * np.take(e, nb, axis=axis)
    return e


def prolong_nearest(coarse, fine_shape):
    """PROL of the paper's scheme (Algorithm 1, an upsampling layer): every fine
    cell takes its parent's value."""
    e = coarse
    for axis in range(3):
        if fine_shape[axis] != e.shape[axis]:
            e = np.repeat(e, 2, axis=axis)
    return e


def dense_operator(lev):
    """The matrix of A on a level, built column by column from unit vectors.
    Rows and columns of solid cells are the identity."""
    n = int(np.prod(lev.shape))
    M = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = apply_A(lev, e.reshape(lev.shape)).ravel()
    solid = lev.solid.ravel()
    M[solid, :] = 0.0
    M[:, solid] = 0.0
    M[solid, solid] = 1.0
    return M


def direct_solve(lev, b):
    """Exact discrete solution of A p = b (dense LU through numpy)."""
    M = dense_operator(lev)
    rhs = np.where(lev.solid, 0.0, b).ravel()
    return np.linalg.solve(M, rhs).reshape(lev.shape)


# ------------------------------------------------------------------ V-cycle
class Multigrid:
    def __init__(self, geo, n_levels):
        self.spec = geo.spec
        self.levels = geo.levels(n_levels)
        self._coarse_M = dense_operator(self.levels[-1])

    def coarse_solve(self, b):
        lev = self.levels[-1]
        rhs = np.where(lev.solid, 0.0, b).ravel()
        return np.linalg.solve(self._coarse_M, rhs).reshape(lev.shape)

    def sweeps(self, l):
        """(pre, post) smoothing sweeps on level l: the spec's on the finest level;
        coarse_sweeps, when set, on both sides of every coarser level."""
        k = getattr(self.spec, "coarse_sweeps", 0)
        if l > 0 and k > 0:
            return k, k
        return self.spec.pre_sweeps, self.spec.post_sweeps

    def vcycle(self, p, b, l=0):
        lev = self.levels[l]
        if l == len(self.levels) - 1:
            return self.coarse_solve(b)
        pre, post = self.sweeps(l)
        p = smooth(lev, p, b, pre, sweep_weights(lev, self.spec, pre, False))
        bc = restrict(lev, residual(lev, p, b))
        ec = self.vcycle(np.zeros(self.levels[l + 1].shape), bc, l + 1)
        p = np.where(lev.fluid, p + prolong(self.levels[l + 1], ec, lev.shape), 0.0)
        p = smooth(lev, p, b, post, sweep_weights(lev, self.spec, post, True))
        return p

    def paper_cycle(self, p, b):
        """One iteration of Algorithm 1, in this module's sign convention
        (r = b - A p, so the correction is added; the paper writes
        r0 = A p - b and subtracts it).  The fine residual is restricted
        straight down through every level.  On the way up, each coarse level
        gets one unweighted Jacobi iteration on the correction, starting from
        the upsampled coarser correction (zero on the coarsest level), then
        upsampling (nearest).  The upsampled level-1 correction is added to p,
        and one unweighted Jacobi sweep on p ends the iteration.  The residual
        is recomputed each iteration.  A and D keep the fine grid's spacing on
        every level (the paper applies one convolution kernel and one scalar
        D = 6/dx^2 at all levels)."""
        levs = self.levels
        r = [residual(levs[0], p, b)]
        for l in range(1, len(levs)):
            r.append(restrict(levs[l - 1], r[l - 1]))
        w = np.zeros(levs[-1].shape)
        for l in range(len(levs) - 1, 0, -1):
            lev = copy.copy(levs[l])
            lev.h = levs[0].h
            w = np.where(lev.fluid, w + residual(lev, w, r[l]) / lev.diag(), 0.0)
            w = prolong_nearest(w, levs[l - 1].shape)
        lev0 = levs[0]
        p = np.where(lev0.fluid, p + w, 0.0)
        return np.where(lev0.fluid, p + residual(lev0, p, b) / lev0.diag(), 0.0)

    def cycle(self, p, b):
        """One iteration of the configured scheme (mg_variant 0: V-cycle, 1: Algorithm 1)."""
        if getattr(self.spec, "mg_variant", 0) == 1:
            return self.paper_cycle(p, b)
        return self.vcycle(p, b)

    def fcg_solve(self, p, b, cycles_cap, tol, fixed):
        """Flexible conjugate gradients with one kept direction, one V-cycle
        from zero on A z = r as the preconditioner (the outer acceleration of
        krylov = 1).  A is symmetric positive definite on the fluid cells, so
        a step along any direction d with alpha = (r, d) / (d, A d) cannot
        raise the A-norm of the error.  Each iteration: z = V(r), made
        A-orthogonal to the previous direction (beta = (z, A d_prev) /
        (d_prev, A d_prev), d = z - beta d_prev), then that step,
        p += alpha d; r = b - A p is recomputed from p.  With a fixed
        symmetric positive definite preconditioner in place of the V-cycle
        this is preconditioned CG.  Inner products over fluid cells.  Should
        (d, A d) come out <= 0 (by rounding only) the step restarts along z
        alone."""
        lev = self.levels[0]
        fl = lev.fluid

        def dot(a, c):
            return float(np.sum(a[fl] * c[fl]))

        dp = qp = None
        n = 0
        rel = self.rel_residual(p, b)
        while (n < fixed) if fixed > 0 else (rel > tol and n < cycles_cap):
            r = residual(lev, p, b)
            d = self.vcycle(np.zeros(lev.shape), r)
            q = apply_A(lev, d)
            z, qz = d, q
            if dp is not None and dot(dp, qp) > 0.0:
                beta = dot(d, qp) / dot(dp, qp)
                d = d - beta * dp
                q = q - beta * qp
            dq = dot(d, q)
            if not dq > 0.0:   # (d, A d) <= 0 only by rounding: restart along z alone
                d, q = z, qz
                dq = dot(d, q)
            alpha = dot(r, d) / dq if dq > 0.0 else 0.0
            p = np.where(fl, p + alpha * d, 0.0)
            dp, qp = d, q
            n += 1
            rel = self.rel_residual(p, b)
        return p, n, rel

    def rel_residual(self, p, b):
        lev = self.levels[0]
        nb = np.linalg.norm(b[lev.fluid])
        if nb == 0.0:
            return 0.0
        return float(np.linalg.norm(residual(lev, p, b)[lev.fluid]) / nb)

    def solve(self, p, b):
        """V-cycles from warm start p: exactly fixed_vcycles of them if set,
        else until the relative residual is <= mg_rel_tol or max_vcycles ran.
        Returns (p, cycles, final relative residual)."""
        s = self.spec
        if getattr(s, "krylov", 0) == 1:
            return self.fcg_solve(p, b, s.max_vcycles, s.mg_rel_tol, s.fixed_vcycles)
        if s.fixed_vcycles > 0:
            for _ in range(s.fixed_vcycles):
                p = self.cycle(p, b)
            return p, s.fixed_vcycles, self.rel_residual(p, b)
        n = 0
        rel = self.rel_residual(p, b)
        while rel > s.mg_rel_tol and n < s.max_vcycles:
            p = self.cycle(p, b)
            n += 1
            rel = self.rel_residual(p, b)
        return p, n, rel
