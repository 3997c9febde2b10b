"""Pins of the oracle's per-step time-step cap (``oracle.step.stable_dt``).

The cap is dt = min(dt0, CFL / max over fluid cells of
sum_d (|u_d| / h_d + 2 Gamma / h_d^2)), Gamma = max(nu + nu_t, alpha + nu_t / Pr_t):
the forward-Euler stability limit of first-order upwind convection plus
central diffusion, summed over the active axes.  Every expected value below
is worked out by hand from the printed closure constants (Section 2.1:
alpha*_0 = beta_i / 3 = 0.024, R_k = 6, alpha*_inf = 1) and written as a
literal, so that a dropped factor 2, Gamma taken as nu + nu_t alone, the
wrong spacing per axis, solid cells in the maximum or a collapsed axis that
still contributes each fail one of them.
"""
import numpy as np
import pytest

from oracle.geometry import Geometry
from oracle.step import stable_dt
from paper_2603_21869_gb300 import cases


def _box(nx, ny, nz, Lx, Ly, Lz, **kw):
    faces = [cases.Patch() for _ in range(6)]
    if nz == 1:
        faces[4] = cases.Patch(kind=cases.EMPTY)
        faces[5] = cases.Patch(kind=cases.EMPTY)
    return cases.CaseSpec(nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz, faces=faces, mg_levels=2, **kw)


def _state(geo, u, v, w, k, om):
    return [np.full(geo.shape, float(x)) for x in (u, v, w, 0.0, k, om)]


def test_laminar_cap_uses_twice_the_larger_diffusivity_per_axis():
    # h = (0.1, 0.2, 0.4); nu = 0.01, Pr = 0.71 -> alpha = 0.01 / 0.71 > nu; k = 0 -> nu_t = 0
    spec = _box(8, 4, 4, 0.8, 0.8, 1.6, nu=0.01, Pr=0.71, cfl=0.5)
    geo = Geometry(spec)
    st = _state(geo, 1.0, -2.0, 0.5, 0.0, 3.0)
    # convection 1/0.1 + 2/0.2 + 0.5/0.4 = 21.25
    # diffusion 2 * (0.01 / 0.71) * (100 + 25 + 6.25) = 3.6971830985915493
    lam = 21.25 + 3.6971830985915493
    assert stable_dt(geo, st, 1.0) == pytest.approx(0.5 / lam, rel=1e-14)
    # Pr = 2: alpha = 0.005 < nu, so Gamma = nu: diffusion 2 * 0.01 * 131.25 = 2.625
    spec2 = spec.replace(Pr=2.0)
    assert stable_dt(Geometry(spec2), st, 1.0) == pytest.approx(0.5 / (21.25 + 2.625), rel=1e-14)
    # a cap above dt0 leaves dt0
    assert stable_dt(geo, st, 1e-3) == 1e-3


def test_eddy_viscosity_enters_both_diffusivities():
    # nu = 0.01, k = 6, omega = 100: Re_t = k / (nu omega) = 6 = R_k, so
    # alpha* = (0.024 + 1) / (1 + 1) = 0.512 and nu_t = 0.512 * 6 / 100 = 0.03072
    nut = 0.03072
    spec = _box(8, 4, 4, 0.8, 0.8, 1.6, nu=0.01, Pr=0.71, Prt=0.85, cfl=0.5)
    geo = Geometry(spec)
    st = _state(geo, 0.0, 0.0, 0.0, 6.0, 100.0)
    inv_h2 = 100.0 + 25.0 + 6.25
    # Pr_t = 0.85: alpha + nu_t / Pr_t = 0.014084507042253521 + 0.036141176470588235 > nu + nu_t = 0.04072
    g_T = 0.01 / 0.71 + nut / 0.85
    assert g_T > 0.01 + nut
    assert stable_dt(geo, st, 1.0) == pytest.approx(0.5 / (2.0 * g_T * inv_h2), rel=1e-13)
    # Pr_t = 2: alpha + nu_t / 2 = 0.029444507... < nu + nu_t = 0.04072, the momentum diffusivity wins
    spec2 = spec.replace(Prt=2.0)
    assert 0.01 / 0.71 + nut / 2.0 < 0.01 + nut
    assert stable_dt(Geometry(spec2), st, 1.0) == pytest.approx(0.5 / (2.0 * (0.01 + nut) * inv_h2), rel=1e-13)


def test_solid_cells_do_not_lower_the_step():
    box = cases.Box(2, 4, 1, 3, 1, 3)
    spec = _box(8, 4, 4, 0.8, 0.8, 1.6, nu=0.01, Pr=2.0, cfl=0.5, boxes=[box])
    geo = Geometry(spec)
    st = _state(geo, 1.0, 0.0, 0.0, 0.0, 3.0)
    for f in (0, 1, 2):
        st[f][2:4, 1:3, 1:3] = 1e6    # a huge velocity inside the obstacle
    st[4][2:4, 1:3, 1:3] = 1e6        # and a huge k there
    lam = 1.0 / 0.1 + 2.0 * 0.01 * (100.0 + 25.0 + 6.25)
    assert stable_dt(geo, st, 1.0) == pytest.approx(0.5 / lam, rel=1e-14)


def test_collapsed_axis_contributes_nothing():
    # 2D: nz = 1 with Lz = 1e-3 (h_z would dominate if the empty axis were counted)
    spec = _box(8, 4, 1, 0.8, 0.8, 1e-3, nu=0.01, Pr=2.0, cfl=0.5)
    geo = Geometry(spec)
    st = _state(geo, 1.0, 1.0, 50.0, 0.0, 3.0)
    lam = 1.0 / 0.1 + 1.0 / 0.2 + 2.0 * 0.01 * (100.0 + 25.0)
    assert stable_dt(geo, st, 1.0) == pytest.approx(0.5 / lam, rel=1e-14)


def test_maximum_is_taken_over_cells_not_averaged():
    spec = _box(8, 4, 4, 0.8, 0.8, 1.6, nu=0.01, Pr=2.0, cfl=0.5)
    geo = Geometry(spec)
    st = _state(geo, 0.0, 0.0, 0.0, 0.0, 3.0)
    st[0][5, 2, 1] = -4.0             # one fast cell, speed |u| = 4
    lam = 4.0 / 0.1 + 2.0 * 0.01 * 131.25
    assert stable_dt(geo, st, 1.0) == pytest.approx(0.5 / lam, rel=1e-14)
