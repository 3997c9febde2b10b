"""Grid levels, boundary patches and ghost cells (Section 2.7).

External boundaries: BC_x pads a field with one ghost layer on each side
along x (Eq. bc_x); BC_y, BC_z likewise (Eqs. bc_y, bc_z).  Internal
boundaries (solid boxes): where a face separates a fluid and a solid cell,
the solid cell's value is replaced by the ghost value built from the
neighbouring fluid cell, the mask-based treatment of Section 2.7.

Ghost values (one rule for external and internal walls):

  field      WALL / obstacle          INLET                 OUTLET     EMPTY
  u, v, w    -phi_P (no slip)         2 u_in - phi_P        phi_P      phi_P
  p          phi_P                    phi_P                 -phi_P     phi_P
  k, omega   phi_P (dk/dn = 0)        2 k0 - phi_P, ...     phi_P      phi_P
  T          2 T_w - T_P (fixed),     2 T_in - T_P          T_P        T_P
             T_P (adiabatic),
             T_P + q h / (rho cp alpha) (heat flux)

Mirror ghosts place the prescribed value on the face itself (face value =
mean of the two sides).  EMPTY is the degenerate z direction of a 2D case
(nz = 1): every term across it vanishes.
"""
import numpy as np

from . import model

WALL, INLET, OUTLET, EMPTY = 0, 1, 2, 3
ADIABATIC, FIXED_T, HEAT_FLUX = 0, 1, 2
U, V, W, P, T, K, OM = range(7)

# face kinds returned by face_states
FK_INTERIOR, FK_WALL, FK_INLET, FK_OUTLET, FK_EMPTY, FK_SOLID = 0, 1, 2, 3, 4, 5
_PATCH_TO_FK = {WALL: FK_WALL, INLET: FK_INLET, OUTLET: FK_OUTLET, EMPTY: FK_EMPTY}


def face_shape(shape, face):
    axis = face // 2
    return tuple(n for a, n in enumerate(shape) if a != axis)


class Level:
    """One grid level: shape, spacing, solid mask, pressure-Dirichlet faces."""

    def __init__(self, shape, h, solid, dirichlet):
        self.shape = tuple(shape)
        self.h = tuple(h)
        self.solid = solid
        self.fluid = ~solid
        self.dirichlet = dirichlet          # 6 bool arrays (outlet faces)
        self.active = tuple(n > 1 for n in self.shape)

    def diag(self):
        """Scalar Jacobi diagonal D = sum_d 2 / h_d^2 (Eq. jacobi_pc: 6/dx^2 when isotropic)."""
        return sum(2.0 / self.h[a] ** 2 for a in range(3) if self.active[a])

    def coarsen(self):
        f = tuple(2 if a else 1 for a in self.active)
        shape = tuple(n // ff for n, ff in zip(self.shape, f))
        h = tuple(hh * ff for hh, ff in zip(self.h, f))
        s = self.solid.reshape(shape[0], f[0], shape[1], f[1], shape[2], f[2])
        solid = s.all(axis=(1, 3, 5))                      # coarse cell solid iff all children solid
        dirichlet = []
        for face in range(6):
            ff = tuple(x for a, x in enumerate(f) if a != face // 2)
            d = self.dirichlet[face]
            fs = face_shape(shape, face)
            dirichlet.append(d.reshape(fs[0], ff[0], fs[1], ff[1]).any(axis=(1, 3)))
        return Level(shape, h, solid, dirichlet)


class Geometry:
    """Level-0 geometry of a case: patches per boundary cell and box ids."""

    def __init__(self, spec):
        self.spec = spec
        shape = (spec.nx, spec.ny, spec.nz)
        self.shape = shape
        self.h = (spec.Lx / spec.nx, spec.Ly / spec.ny, spec.Lz / spec.nz)
        self.patches = list(spec.faces) + [v.bc for v in spec.vents]
        self.face_patch = []
        for face in range(6):
            fp = np.full(face_shape(shape, face), face, dtype=np.int64)
            self.face_patch.append(fp)
        for n, v in enumerate(spec.vents):
            self.face_patch[v.face][v.a0:v.a1, v.b0:v.b1] = 6 + n
        self.box_id = np.zeros(shape, dtype=np.int64)      # 0 fluid, b + 1 for box b
        for b, bx in enumerate(spec.boxes):
            self.box_id[bx.i0:bx.i1, bx.j0:bx.j1, bx.k0:bx.k1] = b + 1
        self.solid = self.box_id > 0
        self.fluid = ~self.solid
        dirichlet = [np.vectorize(lambda pid: self.patches[pid].kind == OUTLET, otypes=[bool])(fp)
                     for fp in self.face_patch]
        self.level0 = Level(shape, self.h, self.solid, dirichlet)
        self.alpha = spec.nu / spec.Pr
        self.inlet_kw = {}
        for pid, pt in enumerate(self.patches):
            if pt.kind == INLET:
                k0, om0 = model.inlet_turbulence(pt.u_normal, pt.intensity, pt.length_scale) \
                    if pt.intensity > 0 else (0.0, 0.0)
                if pt.k_value > 0:
                    k0 = pt.k_value
                if pt.omega_value > 0:
                    om0 = pt.omega_value
                self.inlet_kw[pid] = (k0, om0)

    def levels(self, n):
        """n grid levels; every active axis must keep at least 2 cells."""
        lv = [self.level0]
        for _ in range(n - 1):
            lv.append(lv[-1].coarsen())
        for a in range(3):
            if self.shape[a] > 1:
                assert lv[-1].shape[a] >= 2 and lv[-1].shape[a] * 2 ** (n - 1) == self.shape[a], \
                    "active axes must halve evenly down to >= 2 cells"
        return lv

    # ---------------------------------------------------------------- ghosts
    def _patch_ghost(self, field, Pv, patch, pid, face):
        axis = face // 2
        hn = self.h[axis]
        kind = patch.kind
        if kind == EMPTY:
            return Pv.copy()
        if kind == WALL:
            if field in (U, V, W):
                return -Pv
            if field == T:
                return self._thermal_ghost(Pv, patch.thermal, patch.T_value, hn)
            return Pv.copy()
        if kind == INLET:
            if field == P:
                return Pv.copy()
            if field in (U, V, W):
                inward = 1.0 if face % 2 == 0 else -1.0
                val = inward * patch.u_normal if field == axis else 0.0
            elif field == T:
                val = patch.T_in
            elif field == K:
                val = self.inlet_kw[pid][0]
            else:
                val = self.inlet_kw[pid][1]
            return 2.0 * val - Pv
        # OUTLET
        if field == P:
            return -Pv
        return Pv.copy()

    def _thermal_ghost(self, Pv, thermal, value, hn):
        if thermal == FIXED_T:
            return 2.0 * value - Pv
        if thermal == HEAT_FLUX:
            s = self.spec
            return Pv + value * hn / (s.rho * s.cp * self.alpha)
        return Pv.copy()

    def boundary_ghost(self, field, Pv, face):
        """Ghost layer of `field` outside boundary face `face` from the adjacent interior layer Pv."""
        out = np.empty_like(Pv)
        fp = self.face_patch[face]
        for pid in np.unique(fp):
            m = fp == pid
            out[m] = self._patch_ghost(field, Pv[m], self.patches[pid], int(pid), face)
        return out

    def obstacle_ghost(self, field, Pv, box_ids, axis):
        """Ghost replacing a solid neighbour (internal wall of box box_ids - 1)."""
        if field in (U, V, W):
            return -Pv
        if field != T:
            return Pv.copy()
        out = Pv.copy()
        for b in np.unique(box_ids):
            bx = self.spec.boxes[int(b) - 1]
            m = box_ids == b
            out[m] = self._thermal_ghost(Pv[m], bx.thermal, bx.T_value, self.h[axis])
        return out

    def boundary_kind(self, face):
        fp = self.face_patch[face]
        kinds = np.array([_PATCH_TO_FK[p.kind] for p in self.patches])
        return kinds[fp]

    def face_states(self, phi, field, axis):
        """Left/right states on the n+1 faces along `axis`: BC_axis(phi)
        sliced into its lower (W+) and upper (W-) neighbours, with solid
        neighbours replaced by wall ghosts.  Also returns the face kinds."""
        lo = np.take(phi, [0], axis=axis)
        hi = np.take(phi, [phi.shape[axis] - 1], axis=axis)
        g_lo = np.expand_dims(self.boundary_ghost(field, np.squeeze(lo, axis), 2 * axis), axis)
        g_hi = np.expand_dims(self.boundary_ghost(field, np.squeeze(hi, axis), 2 * axis + 1), axis)
        pad = np.concatenate([g_lo, phi, g_hi], axis=axis)        # BC_axis(phi)
        n = pad.shape[axis]
        L = np.take(pad, range(0, n - 1), axis=axis).copy()       # W+ * BC(phi)
        R = np.take(pad, range(1, n), axis=axis).copy()           # W- * BC(phi)
        kind = np.zeros(L.shape, dtype=np.int64)
        kl = np.expand_dims(self.boundary_kind(2 * axis), axis)
        kh = np.expand_dims(self.boundary_kind(2 * axis + 1), axis)
        idx_lo = [slice(None)] * 3
        idx_lo[axis] = slice(0, 1)
        idx_hi = [slice(None)] * 3
        idx_hi[axis] = slice(n - 2, n - 1)
        kind[tuple(idx_lo)] = kl
        kind[tuple(idx_hi)] = kh
        # internal walls; the ghost layer outside the domain is tagged -1
        outside = np.full_like(np.take(self.box_id, [0], axis=axis), -1)
        bid = np.concatenate([outside, self.box_id, outside], axis=axis)
        bL = np.take(bid, range(0, n - 1), axis=axis)
        bR = np.take(bid, range(1, n), axis=axis)
        mL = (bL > 0) & (bR == 0)
        mR = (bR > 0) & (bL == 0)
        both = ((bL > 0) | (bR > 0)) & ~mL & ~mR
        if mL.any():
            L[mL] = self.obstacle_ghost(field, R[mL], bL[mL], axis)
            kind[mL] = FK_WALL
        if mR.any():
            R[mR] = self.obstacle_ghost(field, L[mR], bR[mR], axis)
            kind[mR] = FK_WALL
        # a face between two solids, or a boundary face next to a solid cell
        kind[both] = FK_SOLID
        return L, R, kind


def pressure_face_states(e, lev, axis):
    """Faces of a pressure-like field on a multigrid level: Neumann ghosts
    (ghost = interior) at walls, inlets and solid neighbours, homogeneous
    Dirichlet (ghost = -interior) on outlet faces (p = 0 on the face)."""
    n = e.shape[axis]
    lo = np.squeeze(np.take(e, [0], axis=axis), axis)
    hi = np.squeeze(np.take(e, [n - 1], axis=axis), axis)
    g_lo = np.where(lev.dirichlet[2 * axis], -lo, lo)
    g_hi = np.where(lev.dirichlet[2 * axis + 1], -hi, hi)
    pad = np.concatenate([np.expand_dims(g_lo, axis), e, np.expand_dims(g_hi, axis)], axis=axis)
    L = np.take(pad, range(0, n + 1), axis=axis).copy()
    R = np.take(pad, range(1, n + 2), axis=axis).copy()
    zero = np.zeros_like(np.take(lev.solid, [0], axis=axis))
    s = np.concatenate([zero, lev.solid, zero], axis=axis)
    sL = np.take(s, range(0, n + 1), axis=axis)
    sR = np.take(s, range(1, n + 2), axis=axis)
    mL = sL & ~sR
    mR = sR & ~sL
    L[mL] = R[mL]
    R[mR] = L[mR]
    return L, R


def D_op(F, axis, h):
    """D_x * F: face values (n+1) -> cell differences (n), divided by h (Eq. Dx_Lx)."""
    n = F.shape[axis]
    return (np.take(F, range(1, n), axis=axis) - np.take(F, range(0, n - 1), axis=axis)) / h


def L_op(F, axis):
    """L_x * F: two neighbours averaged (kernel [1/2, 1/2], Eq. Dx_Lx)."""
    n = F.shape[axis]
    return 0.5 * (np.take(F, range(1, n), axis=axis) + np.take(F, range(0, n - 1), axis=axis))


def cell_gradient(geo, phi, field):
    """d phi / d x_j at cell centres: L_j * (D_j * BC_j(phi)) (Algorithm 4)."""
    g = []
    for axis in range(3):
        L, R, kind = geo.face_states(phi, field, axis)
        fg = (R - L) / geo.h[axis]                  # D_axis * BC_axis(phi) on faces
        fg[kind == FK_SOLID] = 0.0
        g.append(L_op(fg, axis))                    # back to cells
    return g
