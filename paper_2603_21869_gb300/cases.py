"""Case descriptions and seeded synthetic workloads.

This module holds plain data only: grid sizes, physical constants, boundary
patches, obstacle boxes and the seeded draws that place vents and boxes.  It
contains none of the solver's arithmetic (no turbulence closure, no inlet
turbulence formula, no time-step rule); the CUDA library and the CPU oracle
each derive those from a :class:`CaseSpec` on their own.

Geometry conventions (shared vocabulary, not arithmetic):

* cells are indexed (i, j, k) along (x, y, z); z is vertical;
* boundary faces are numbered 0..5 = x-, x+, y-, y+, z-, z+;
* a vent is a rectangle of boundary cells on one face, given as half-open
  ranges [a0, a1) x [b0, b1) along the face's two tangential axes in
  increasing axis order (x faces: y then z; y faces: x then z; z faces: x
  then y);
* a box is a half-open cell range [i0, i1) x [j0, j1) x [k0, k1) of solid.

The workloads follow the problem statements of the paper's verification
cases (Section 3.1: 2.56 x 0.64 x 0.64 m channel at 1 cm; Section 3.2.4:
room inlet u0 = 0.455 m/s, I0 = 0.04, l0 = h/10).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# face kinds
WALL, INLET, OUTLET, EMPTY = 0, 1, 2, 3
# wall thermal conditions
ADIABATIC, FIXED_T, HEAT_FLUX = 0, 1, 2
# precision modes
FP64, FP32, BF16_MIXED = 0, 1, 2
PRECISION_NAMES = {FP64: "f64", FP32: "f32", BF16_MIXED: "bf16"}

FIELDS = ("u", "v", "w", "p", "T", "k", "omega")
FIELD_INDEX = {n: i for i, n in enumerate(FIELDS)}


@dataclass
class Patch:
    """Boundary condition on a whole face or on a vent."""
    kind: int = WALL
    thermal: int = ADIABATIC
    T_value: float = 0.0        # wall temperature (FIXED_T) or heat flux W/m^2 (HEAT_FLUX)
    u_normal: float = 0.0       # inlet: speed into the domain, m/s
    intensity: float = 0.0      # inlet: turbulence intensity I0
    length_scale: float = 0.0   # inlet: turbulence length scale l0, m
    T_in: float = 0.0           # inlet temperature
    k_value: float = 0.0        # inlet: explicit k (used when > 0)
    omega_value: float = 0.0    # inlet: explicit omega (used when > 0)


@dataclass
class Vent:
    face: int
    a0: int
    a1: int
    b0: int
    b1: int
    bc: Patch = field(default_factory=Patch)


@dataclass
class Box:
    i0: int
    i1: int
    j0: int
    j1: int
    k0: int
    k1: int
    thermal: int = ADIABATIC
    T_value: float = 0.0


@dataclass
class CaseSpec:
    nx: int
    ny: int
    nz: int
    Lx: float
    Ly: float
    Lz: float
    nu: float = 1.5e-5
    Pr: float = 0.71
    Prt: float = 0.85
    sigma_k: float = 2.0
    sigma_w: float = 2.0
    rho: float = 1.2
    cp: float = 1005.0
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.81)
    beta_T: float = 0.0
    T_ref: float = 0.0
    buoyancy: int = 0
    dt: float = 0.0
    cfl: float = 0.5
    dt_adapt: int = 1            # 1: cap dt every step by the explicit stability limit
    faces: List[Patch] = field(default_factory=lambda: [Patch() for _ in range(6)])
    vents: List[Vent] = field(default_factory=list)
    boxes: List[Box] = field(default_factory=list)
    precision: int = FP64
    mg_levels: int = 4
    pre_sweeps: int = 3
    post_sweeps: int = 3
    max_vcycles: int = 50
    fixed_vcycles: int = 0
    inner_cycles: int = 0        # V-cycles per FP64 outer residual (0: 1 for FP64, 2 otherwise)
    sweep_planes: int = 0        # z planes per block of the four-cell level kernels (0: built-in rule)
    mg_variant: int = 0          # 0: V-cycles; 1: the paper's scheme (Algorithm 1)
    krylov: int = 0              # 1: flexible CG with one kept direction around the V-cycles
    coarse_sweeps: int = 0       # pre- and post-sweeps on the levels below the finest (0: as the finest)
    rk_stages: int = 1           # explicit stage: 1 forward Euler, 2 / 3 strong-stability-preserving RK
    mg_rel_tol: float = 1e-8
    jacobi_weight: float = 0.0   # 0 -> 6/7 in 3D, 4/5 in 2D
    smoother: int = 0            # 0: that weight on every sweep; 1: Chebyshev weights on [1/4, 2] per sweep
    seed: int = 0
    init_perturb: float = 0.0
    init_vel: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    init_T: float = 0.0
    init_k: float = 0.0          # <= 0 -> the first inlet's k0
    init_omega: float = 0.0      # <= 0 -> the first inlet's omega0

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "CaseSpec":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def channel_2d(nx: int = 128, ny: int = 32, steps_levels: int = 5, **kw) -> CaseSpec:
    """2D turbulent channel: L = 4 m, H = 1 m, u_in = 1 m/s, I = 5%,
    l0 = 0.07 H, nu = 1.5e-5, no-slip walls, zero-gradient outlet, CFL 0.5,
    5-level multigrid to a 1e-8 relative residual, seed 0."""
    inlet = Patch(kind=INLET, u_normal=1.0, intensity=0.05, length_scale=0.07, T_in=20.0)
    faces = [inlet, Patch(kind=OUTLET), Patch(WALL), Patch(WALL), Patch(EMPTY), Patch(EMPTY)]
    spec = CaseSpec(nx=nx, ny=ny, nz=1, Lx=4.0, Ly=1.0, Lz=1.0 / ny, nu=1.5e-5,
                    cfl=0.5, faces=faces, mg_levels=steps_levels, init_vel=(1.0, 0.0, 0.0),
                    init_T=20.0, seed=0)
    return spec.replace(**kw) if kw else spec


def heated_channel_3d(nx: int = 256, ny: int = 64, nz: int = 64, mg_levels: int = 6,
                      precision: int = FP64, **kw) -> CaseSpec:
    """3D heated channel at the paper's 1 cm verification geometry
    (2.56 x 0.64 x 0.64 m): inlet u = 2 m/s, I = 5 %, l0 = 0.07 H, Pr = 0.71,
    Prt = 0.85, bottom wall 10 K above the inlet temperature, other walls
    adiabatic, fields initialised from a seeded +-1 % perturbation."""
    h = 0.01 * 256 / nx
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    T_in = 25.0
    inlet = Patch(kind=INLET, u_normal=2.0, intensity=0.05, length_scale=0.07 * Lz, T_in=T_in)
    faces = [inlet, Patch(kind=OUTLET), Patch(WALL), Patch(WALL),
             Patch(WALL, thermal=FIXED_T, T_value=T_in + 10.0), Patch(WALL)]
    spec = CaseSpec(nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz, nu=1.5e-5, Pr=0.71, Prt=0.85,
                    cfl=0.5, faces=faces, mg_levels=mg_levels, precision=precision,
                    init_vel=(2.0, 0.0, 0.0), init_T=T_in, seed=0, init_perturb=0.01)
    return spec.replace(**kw) if kw else spec


def _draw_room_geometry(rng: np.random.Generator, nx: int, ny: int, nz: int, Lz: float,
                        vent_cells: int, outlet_cells: int, box_range: Tuple[int, int],
                        n_vents: Tuple[int, int], n_boxes: Tuple[int, int]):
    vents: List[Vent] = []
    taken = []
    nv = int(rng.integers(n_vents[0], n_vents[1] + 1))
    tries = 0
    while len(vents) < nv and tries < 1000:
        tries += 1
        a0 = int(rng.integers(1, nx - vent_cells - 1))
        b0 = int(rng.integers(1, ny - vent_cells - 1))
        r = (a0, a0 + vent_cells, b0, b0 + vent_cells)
        if any(not (r[1] <= t[0] or t[1] <= r[0] or r[3] <= t[2] or t[3] <= r[2]) for t in taken):
            continue
        taken.append(r)
        vents.append(Vent(face=5, a0=r[0], a1=r[1], b0=r[2], b1=r[3],
                          bc=Patch(kind=INLET, u_normal=0.455, intensity=0.04,
                                   length_scale=Lz / 10.0, T_in=18.0)))
    a0 = int(rng.integers(1, nx - outlet_cells - 1))
    b0 = int(rng.integers(1, ny - outlet_cells - 1))
    vents.append(Vent(face=4, a0=a0, a1=a0 + outlet_cells, b0=b0, b1=b0 + outlet_cells,
                      bc=Patch(kind=OUTLET)))
    boxes: List[Box] = []
    nb = int(rng.integers(n_boxes[0], n_boxes[1] + 1))
    tries = 0
    floor_out = (a0, a0 + outlet_cells, b0, b0 + outlet_cells)
    while len(boxes) < nb and tries < 2000:
        tries += 1
        sx, sy = (int(rng.integers(box_range[0], box_range[1] + 1)) for _ in range(2))
        sz = int(rng.integers(box_range[0], min(box_range[1], nz // 2) + 1))
        sx, sy = min(sx, nx // 3), min(sy, ny // 3)
        i0 = int(rng.integers(2, nx - sx - 2))
        j0 = int(rng.integers(2, ny - sy - 2))
        k0 = 0 if rng.random() < 0.5 else int(rng.integers(1, max(2, nz - sz - 2)))
        b = Box(i0, i0 + sx, j0, j0 + sy, k0, k0 + sz, thermal=HEAT_FLUX,
                T_value=float(rng.uniform(50.0, 200.0)))
        clash = any(not (b.i1 + 1 <= o.i0 or o.i1 + 1 <= b.i0 or b.j1 + 1 <= o.j0 or
                         o.j1 + 1 <= b.j0 or b.k1 + 1 <= o.k0 or o.k1 + 1 <= b.k0) for o in boxes)
        over_outlet = b.k0 == 0 and not (b.i1 <= floor_out[0] or floor_out[1] <= b.i0 or
                                         b.j1 <= floor_out[2] or floor_out[3] <= b.j0)
        if clash or over_outlet:
            continue
        boxes.append(b)
    return vents, boxes


def room_3d(nx: int = 512, ny: int = 256, nz: int = 128, seed: int = 0, mg_levels: int = 7,
            precision: int = BF16_MIXED, h: float = 0.02, **kw) -> CaseSpec:
    """Indoor room: 2-4 ceiling inlet vents (8 x 8 cells, downward
    u0 = 0.455 m/s, I0 = 0.04, l0 = h/10), one 16 x 16 floor outlet and 3-6
    heated box obstacles (50-200 W/m^2), Boussinesq buoyancy, all placed by a
    seeded draw."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    vent_cells = max(2, min(8, nx // 8, ny // 8))
    outlet_cells = max(2, min(16, nx // 4, ny // 4))
    box_lo = max(2, min(8, nz // 8))
    box_hi = max(box_lo, min(48, nz // 2))
    vents, boxes = _draw_room_geometry(rng, nx, ny, nz, Lz, vent_cells, outlet_cells,
                                       (box_lo, box_hi), (2, 4), (3, 6))
    T_ref = 22.0
    spec = CaseSpec(nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz, nu=1.5e-5, Pr=0.71, Prt=0.85,
                    gravity=(0.0, 0.0, -9.81), beta_T=1.0 / (T_ref + 273.15), T_ref=T_ref,
                    buoyancy=1, cfl=0.5, faces=[Patch(WALL) for _ in range(6)], vents=vents,
                    boxes=boxes, mg_levels=mg_levels, precision=precision,
                    init_vel=(0.0, 0.0, 0.0), init_T=T_ref, seed=seed, init_perturb=0.0)
    return spec.replace(**kw) if kw else spec


def batched_channels(n_cases: int = 64, seed: int = 0, precision: int = FP32,
                     mg_levels: int = 5) -> List[CaseSpec]:
    """Uneven 3D channel cases: nx in {64, 96, ..., 192}, ny = nz in {64, 96},
    inlet speed U(0.5, 3) m/s, intensity U(1 %, 10 %)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cases):
        nx = int(rng.choice([64, 96, 128, 160, 192]))
        nyz = int(rng.choice([64, 96]))
        U = float(rng.uniform(0.5, 3.0))
        I = float(rng.uniform(0.01, 0.10))
        s = heated_channel_3d(nx, nyz, nyz, mg_levels=mg_levels, precision=precision,
                              seed=seed * 100003 + c)
        faces = list(s.faces)
        faces[0] = dataclasses.replace(faces[0], u_normal=U, intensity=I)
        out.append(s.replace(faces=faces, init_vel=(U, 0.0, 0.0)))
    return out


def served_rooms(n_requests: int = 2000, seed: int = 0, rate: float = 20.0, channel_share: float = 0.2,
                 precision: int = BF16_MIXED):
    """Poisson arrivals (rate per second) of room cases sized 64^3 to
    256 x 128 x 128 (multiples of 32), with seeded vents, obstacles and heat
    loads; a share of the requests are heated channels of the same sizes.
    Rooms run the flexible-CG acceleration (their small outlet makes plain
    V-cycles slow) with V(2,2) and two V-cycles per outer residual, channels
    V(3,3) with three and no acceleration, both with the constant sweep
    weight: over 600 requests of 300 steps this choice converged every solve,
    where one V-cycle per outer residual left a room whose one-direction step
    stalls (the flexible-CG step on a non-symmetric V-cycle).  Returns
    (arrival_times, specs)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    specs = []
    for r in range(n_requests):
        nx = int(rng.choice([64, 96, 128, 160, 192, 224, 256]))
        ny = int(rng.choice([64, 96, 128]))
        nz = int(rng.choice([64, 96, 128]))
        if rng.uniform() < channel_share:
            specs.append(heated_channel_3d(nx, ny, nz, mg_levels=5, precision=precision,
                                           seed=seed * 1000003 + r, inner_cycles=3))
        else:
            specs.append(room_3d(nx, ny, nz, seed=seed * 1000003 + r, mg_levels=5, h=0.04, precision=precision,
                                 krylov=1, pre_sweeps=2, post_sweeps=2, inner_cycles=2))
    return t, specs
