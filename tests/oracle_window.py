"""The oracle's local stages on a window of a large grid.

Every stage of a step except the pressure solve is local: a cell's update reads
the state within one cell of it (face states, cell gradients and the pointwise
eddy viscosity of the two cells beside a face), and an explicit stage of s
Runge-Kutta substeps within s cells; a whole step, given its pressure, within
three (forward Euler).  So the oracle can give the exact result
of a stage at sampled cells of a grid too large for it to step whole: cut a
window of the state with a margin of MARGIN cells, build the window as a case
of its own (the same cell size, the domain faces and vents it touches, the
boxes clipped to it) and run the stage there; the window's cells at least
MARGIN cells inside its cut faces hold the full grid's values.  The cut faces
take the domain face's boundary condition of the same side, which changes only
the margin.  tests/test_oracle_window.py checks this against whole-grid oracle
stages."""
import dataclasses

import numpy as np

from oracle.destruction import destruction_step
from oracle.geometry import Geometry
from oracle.poisson import poisson_rhs, project
from oracle.transport import explicit_stage_rk

MARGIN = 3   # the reach of a whole step's local part, and of a three-stage explicit stage
STATE = ("u", "v", "w", "T", "k", "omega")


def clip_window(spec, center, size):
    """The window of `size` cells per axis around `center`, widened by MARGIN on each
    side and clipped to the grid: (lo, hi) cell bounds of the cut and (ilo, ihi) of
    the cells whose values are exact (the cut minus MARGIN on every cut face)."""
    n = (spec.nx, spec.ny, spec.nz)
    lo, hi, ilo, ihi = [], [], [], []
    for a in range(3):
        s = min(size[a], n[a])
        c0 = min(max(center[a] - s // 2, 0), n[a] - s)
        c1 = c0 + s
        l, h = max(c0 - MARGIN, 0), min(c1 + MARGIN, n[a])
        lo.append(l)
        hi.append(h)
        ilo.append(c0 if l > 0 else 0)
        ihi.append(c1 if h < n[a] else n[a])
    return tuple(lo), tuple(hi), tuple(ilo), tuple(ihi)


def window_spec(spec, lo, hi):
    """The cut [lo, hi) as a case of its own."""
    n = (spec.nx, spec.ny, spec.nz)
    h = (spec.Lx / spec.nx, spec.Ly / spec.ny, spec.Lz / spec.nz)
    m = tuple(hi[a] - lo[a] for a in range(3))
    boxes = []
    for b in spec.boxes:
        r = [(max(b0, lo[a]) - lo[a], min(b1, hi[a]) - lo[a])
             for a, (b0, b1) in enumerate(((b.i0, b.i1), (b.j0, b.j1), (b.k0, b.k1)))]
        if all(x0 < x1 for x0, x1 in r):
            boxes.append(dataclasses.replace(b, i0=r[0][0], i1=r[0][1], j0=r[1][0], j1=r[1][1],
                                             k0=r[2][0], k1=r[2][1]))
    vents = []
    for v in spec.vents:
        axis, side = v.face // 2, v.face % 2
        if (side == 0 and lo[axis] != 0) or (side == 1 and hi[axis] != n[axis]):
            continue   # the window does not reach this face
        ta, tb = [a for a in range(3) if a != axis]
        a0, a1 = max(v.a0, lo[ta]) - lo[ta], min(v.a1, hi[ta]) - lo[ta]
        b0, b1 = max(v.b0, lo[tb]) - lo[tb], min(v.b1, hi[tb]) - lo[tb]
        if a0 < a1 and b0 < b1:
            vents.append(dataclasses.replace(v, a0=a0, a1=a1, b0=b0, b1=b1))
    return spec.replace(nx=m[0], ny=m[1], nz=m[2], Lx=m[0] * h[0], Ly=m[1] * h[1], Lz=m[2] * h[2],
                        boxes=boxes, vents=vents, mg_levels=1)


class Window:
    """The cut [lo, hi) of a case with the oracle's stages on it; `inner` indexes the
    exact cells within the cut, `full` the same cells within the whole grid."""

    def __init__(self, spec, center, size):
        self.lo, self.hi, ilo, ihi = clip_window(spec, center, size)
        self.geo = Geometry(window_spec(spec, self.lo, self.hi))
        self.inner = tuple(slice(ilo[a] - self.lo[a], ihi[a] - self.lo[a]) for a in range(3))
        self.full = tuple(slice(ilo[a], ihi[a]) for a in range(3))
        self.cut = tuple(slice(self.lo[a], self.hi[a]) for a in range(3))

    def take(self, arrays):
        return [np.array(x[self.cut], dtype=np.float64) for x in arrays]

    def destruction_half(self, state, dt):
        u, v, w, T_, k, om = self.take(state)
        k, om = destruction_step(self.geo, u, v, w, k, om, 0.5 * dt)
        return {"k": k[self.inner], "omega": om[self.inner]}

    def explicit(self, state, dt, stages=1):
        new = explicit_stage_rk(self.geo, self.take(state), dt, stages)
        return {f: x[self.inner] for f, x in zip(STATE, new)}

    def rhs(self, state, dt):
        u, v, w = self.take(state[:3])
        return poisson_rhs(self.geo, u, v, w, dt)[self.inner]

    def project(self, state, p, dt):
        u, v, w = self.take(state[:3])
        (pp,) = self.take([p])
        out = project(self.geo, self.geo.level0, u, v, w, pp, dt)
        return {f: x[self.inner] for f, x in zip(("u", "v", "w"), out)}

    def step(self, state, p, dt, stages=1):
        """One whole step from `state` with the step's pressure p (the solve's result, which
        a window cannot form): the destruction half step, the explicit stage, the second half
        step, the right-hand side b and the projection (Section 2.6).  The velocity after the
        explicit stage reaches two cells (one, through the first half step's k and omega, one
        more); b and the second half step's k and omega three.  Returns (fields, b) at the
        exact cells."""
        u, v, w, T_, k, om = self.take(state)
        k, om = destruction_step(self.geo, u, v, w, k, om, 0.5 * dt)
        u, v, w, T_, k, om = explicit_stage_rk(self.geo, [u, v, w, T_, k, om], dt, stages)
        k, om = destruction_step(self.geo, u, v, w, k, om, 0.5 * dt)
        b = poisson_rhs(self.geo, u, v, w, dt)
        (pp,) = self.take([p])
        u, v, w = project(self.geo, self.geo.level0, u, v, w, pp, dt)
        out = dict(zip(STATE, (u, v, w, T_, k, om)))
        return {f: x[self.inner] for f, x in out.items()}, b[self.inner]
