"""One time step of the k-omega solver (Section 2.6) and the initial state.

Strang splitting (Section 2.6): a half step dt/2 of the semi-implicit
destruction (Algorithm 4), one full explicit step of the remaining terms
(forward Euler, Section A.4), a second half step of destruction; the
resulting intermediate velocity u* is then projected (Section 2.4,
Algorithm 1): b = -div(u*)/dt, V-cycles on A p = b warm-started from the
previous pressure, u = u* - dt grad p.

Time step: dt0 as given, else dt0 = CFL min_d h_d / U_ref with U_ref the
largest inlet speed.  With dt_adapt set, every step starts by capping it
with the forward-Euler stability limit of the explicit stage:
dt = min(dt0, CFL / max over fluid cells of sum_d (|u_d|/h_d + 2 Gamma/h_d^2)),
Gamma = max(nu + nu_t, alpha + nu_t/Pr_t), from the state at the step's start.

Initial state: the uniform state (init_vel, init_T, init_k, init_omega;
k and omega default to the first inlet's k0 and omega0), each of u, v, w,
T, k, omega multiplied by (1 + eps xi) with xi uniform in [-1, 1) drawn from
SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): draw number
n = field * N + (k ny + j) nx + i of the generator seeded with `seed`.
"""
import numpy as np

from . import model
from .destruction import destruction_step
from .geometry import Geometry, INLET, U, V, W, T, K, OM
from .poisson import Multigrid, poisson_rhs, project, face_divergence
from .transport import explicit_stage_rk

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def splitmix64(seed, n):
    """Output number n (0-based, numpy uint64 array) of SplitMix64 seeded with `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (n.astype(np.uint64) + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed, field, shape):
    """xi in [-1, 1) for every cell of `shape` = (nx, ny, nz), field id `field`."""
    nx, ny, nz = shape
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    idx = (k * ny + j) * nx + i + field * (nx * ny * nz)
    bits = splitmix64(seed, idx.astype(np.uint64))
    return (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def time_step(spec):
    if spec.dt > 0:
        return spec.dt
    geo_h = (spec.Lx / spec.nx, spec.Ly / spec.ny, spec.Lz / spec.nz)
    n = (spec.nx, spec.ny, spec.nz)
    hmin = min(h for h, nn in zip(geo_h, n) if nn > 1)
    speeds = [p.u_normal for p in list(spec.faces) + [v.bc for v in spec.vents] if p.kind == INLET]
    U_ref = max(speeds) if speeds else max(abs(x) for x in spec.init_vel)
    if U_ref <= 0:
        U_ref = 1.0
    return spec.cfl * hmin / U_ref


def stable_dt(geo, state, dt0):
    """dt0 capped by CFL / max_cells sum_d (|u_d|/h_d + 2 Gamma/h_d^2)."""
    spec = geo.spec
    u, v, w, T_, k, om = state
    nut = model.nu_t(k, om, spec.nu)
    gam = np.maximum(spec.nu + nut, geo.alpha + nut / spec.Prt)
    lam = np.zeros(geo.shape)
    for axis, phi in enumerate((u, v, w)):
        if geo.shape[axis] == 1:
            continue
        lam = lam + np.abs(phi) / geo.h[axis] + 2.0 * gam / geo.h[axis] ** 2
    lam_max = float(np.max(lam[geo.fluid])) if geo.fluid.any() else 0.0
    if lam_max <= 0.0:
        return dt0
    return min(dt0, spec.cfl / lam_max)


def initial_state(geo):
    spec = geo.spec
    k0, om0 = spec.init_k, spec.init_omega
    inlets = [pid for pid, p in enumerate(geo.patches) if p.kind == INLET]
    if (k0 <= 0 or om0 <= 0) and inlets:
        ik, iw = geo.inlet_kw[inlets[0]]
        k0 = ik if k0 <= 0 else k0
        om0 = iw if om0 <= 0 else om0
    base = {U: spec.init_vel[0], V: spec.init_vel[1], W: spec.init_vel[2],
            T: spec.init_T, K: k0, OM: om0}
    state = []
    for f in (U, V, W, T, K, OM):
        phi = np.full(geo.shape, float(base[f]))
        if spec.init_perturb != 0.0:
            phi = phi * (1.0 + spec.init_perturb * uniform_pm1(spec.seed, f, geo.shape))
        state.append(np.where(geo.fluid, phi, 0.0))
    return state


class OracleCase:
    """State of one case: fields u, v, w, T, k, omega, p (shape (nx, ny, nz))."""

    def __init__(self, spec, state=None, p=None):
        self.spec = spec
        self.geo = Geometry(spec)
        self.mg = Multigrid(self.geo, spec.mg_levels)
        self.dt0 = time_step(spec)
        self.dt = self.dt0
        self.state = initial_state(self.geo) if state is None else [np.array(s, dtype=np.float64) for s in state]
        self.p = np.zeros(self.geo.shape) if p is None else np.array(p, dtype=np.float64)
        self.b = np.zeros(self.geo.shape)
        self.last_vcycles = 0
        self.last_rel = 0.0

    def fields(self):
        u, v, w, T_, k, om = self.state
        return {"u": u, "v": v, "w": w, "p": self.p, "T": T_, "k": k, "omega": om}

    # the stages of one step, exposed one by one
    def destruction_half(self):
        u, v, w, T_, k, om = self.state
        k, om = destruction_step(self.geo, u, v, w, k, om, 0.5 * self.dt)
        self.state = [u, v, w, T_, k, om]

    def explicit(self):
        self.state = explicit_stage_rk(self.geo, self.state, self.dt, getattr(self.spec, "rk_stages", 1))

    def rhs(self):
        u, v, w = self.state[:3]
        self.b = poisson_rhs(self.geo, u, v, w, self.dt)

    def solve(self):
        self.p, self.last_vcycles, self.last_rel = self.mg.solve(self.p, self.b)

    def project(self):
        u, v, w = self.state[:3]
        u, v, w = project(self.geo, self.mg.levels[0], u, v, w, self.p, self.dt)
        self.state = [u, v, w] + self.state[3:]

    def update_dt(self):
        self.dt = stable_dt(self.geo, self.state, self.dt0) if self.spec.dt_adapt else self.dt0

    def step(self, n=1):
        for _ in range(n):
            self.update_dt()
            self.destruction_half()
            self.explicit()
            self.destruction_half()
            self.rhs()
            u_star = [x.copy() for x in self.state[:3]]
            self.solve()
            self.project()
            self._u_star = u_star
        return self

    def divergence_after_projection(self):
        """Face divergence of the last projection's corrected fluxes."""
        u, v, w = self._u_star
        return face_divergence(self.geo, self.mg.levels[0], u, v, w, self.p, self.dt)
