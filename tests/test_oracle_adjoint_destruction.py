"""Pins of the destruction adjoint (oracle/adjoint.py, DestructionAdjoint):
for random directions d and cotangents ybar, the central difference
<F(x + h d) - F(x - h d), ybar> / (2 h) of the forward destruction step must
approach <d, J^T ybar> at second order in h (a wrong or missing derivative
term leaves a gap that does not shrink with h), on states that reach every
branch: chi_k of both signs, inlet and obstacle ghosts, a vent.  The rough
states make the curvature of omega' in the velocity gradient large, so the
step is small (1e-6) and the gap is measured against sum |d_i xbar_i| (the
size of the terms of the inner product, not of their sum)."""
import numpy as np
import pytest

from oracle.adjoint import DestructionAdjoint
from oracle.destruction import destruction_step
from oracle.geometry import Geometry
from oracle.step import OracleCase
from paper_2603_21869_gb300 import cases


def _state(spec, seed):
    c = OracleCase(spec)
    u, v, w, T, k, om = c.state
    rng = np.random.default_rng(seed)
    fl = c.geo.fluid
    # strong, rough perturbations so that the gradients (and chi_k's sign) vary
    u = u + np.where(fl, 0.5 * rng.standard_normal(u.shape), 0.0)
    v = v + np.where(fl, 0.5 * rng.standard_normal(u.shape), 0.0)
    w = w + np.where(fl, 0.5 * rng.standard_normal(u.shape), 0.0)
    k = k * np.where(fl, np.exp(0.5 * rng.standard_normal(u.shape)), 1.0)
    om = om * np.where(fl, np.exp(0.5 * rng.standard_normal(u.shape)), 1.0)
    return [u, v, w, k, om]


SPECS = {
    "channel_box_vent": lambda: cases.heated_channel_3d(
        16, 8, 8, mg_levels=2, boxes=[cases.Box(5, 9, 0, 3, 2, 5, thermal=cases.ADIABATIC)],
        vents=[cases.Vent(face=5, a0=8, a1=12, b0=2, b1=6,
                          bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1, length_scale=0.02, T_in=15.0))]),
    "channel2d": lambda: cases.channel_2d(16, 8, 2),
    "room": lambda: cases.room_3d(16, 8, 8, seed=2, mg_levels=2, h=0.32),
}


@pytest.mark.parametrize("name", list(SPECS))
def test_destruction_vjp_matches_central_differences(name):
    spec = SPECS[name]()
    geo = Geometry(spec)
    dt = 0.05
    x = _state(spec, 1)
    adj = DestructionAdjoint(geo, dt, x)
    dot = np.sum(adj.gk * adj.gw, axis=0)[geo.fluid]
    assert np.any(dot > 0) and np.any(dot < 0)      # both branches of f_beta*
    rng = np.random.default_rng(2)
    d = [np.where(geo.fluid, rng.standard_normal(geo.shape), 0.0) for _ in range(5)]
    d[3] = d[3] * x[3] * 0.1      # relative perturbations of k and omega keep them positive
    d[4] = d[4] * x[4] * 0.1
    ybar = [rng.standard_normal(geo.shape) for _ in range(2)]
    xbar = adj.vjp(*ybar)
    rhs = sum(float(np.sum(a * b)) for a, b in zip(d, xbar))
    scale = sum(float(np.sum(np.abs(a * b))) for a, b in zip(d, xbar))

    def F(s):
        u, v, w, k, om = [a + s * b for a, b in zip(x, d)]
        return destruction_step(geo, u, v, w, k, om, dt)

    h = 1e-6
    kp, op = F(h)
    km, omm = F(-h)
    lhs = (float(np.sum((kp - km) * ybar[0])) + float(np.sum((op - omm) * ybar[1]))) / (2 * h)
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs, scale)


def test_destruction_vjp_each_input_separately():
    """Directions in one input at a time (u, v, w, k, omega): each term of
    the chain rule is checked on its own."""
    spec = SPECS["channel_box_vent"]()
    geo = Geometry(spec)
    dt = 0.05
    x = _state(spec, 3)
    adj = DestructionAdjoint(geo, dt, x)
    rng = np.random.default_rng(4)
    ybar = [rng.standard_normal(geo.shape) for _ in range(2)]
    xbar = adj.vjp(*ybar)
    for i in range(5):
        d = [np.zeros(geo.shape) for _ in range(5)]
        d[i] = np.where(geo.fluid, rng.standard_normal(geo.shape), 0.0) * (x[i] * 0.1 if i >= 3 else 1.0)
        rhs = float(np.sum(d[i] * xbar[i]))
        scale = float(np.sum(np.abs(d[i] * xbar[i])))
        h = 1e-6

        def F(s):
            u, v, w, k, om = [a + s * b for a, b in zip(x, d)]
            return destruction_step(geo, u, v, w, k, om, dt)

        kp, op = F(h)
        km, omm = F(-h)
        lhs = (float(np.sum((kp - km) * ybar[0])) + float(np.sum((op - omm) * ybar[1]))) / (2 * h)
        assert abs(lhs - rhs) <= 1e-6 * scale, (i, lhs, rhs, scale)


def test_solid_cells_are_identity():
    spec = SPECS["channel_box_vent"]()
    geo = Geometry(spec)
    adj = DestructionAdjoint(geo, 0.05, _state(spec, 5))
    rng = np.random.default_rng(6)
    kb = np.where(geo.solid, rng.standard_normal(geo.shape), 0.0)
    ob = np.where(geo.solid, rng.standard_normal(geo.shape), 0.0)
    ub, vb, wb, kk, oo = adj.vjp(kb, ob)
    assert np.array_equal(kk, kb) and np.array_equal(oo, ob)
    assert all(np.all(a == 0.0) for a in (ub, vb, wb))
