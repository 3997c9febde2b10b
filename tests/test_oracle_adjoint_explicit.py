"""Pins of the explicit-stage adjoint (oracle/adjoint.py, ExplicitAdjoint):
the complex-step directional derivatives agree with central differences of
the forward stage; the colour-probed Jacobian equals the dense Jacobian built
one unit vector at a time (brute force on a tiny grid); the
vector-Jacobian product satisfies <J d, ybar> = <d, J^T ybar> against a
complex-step derivative taken directly along d; and the hand-derived
forward-Euler adjoint (explicit_vjp_by_hand) equals it to rounding."""
import numpy as np
import pytest

from oracle import transport
from oracle.adjoint import ExplicitAdjoint, explicit_vjp_by_hand
from oracle.step import OracleCase
from paper_2603_21869_gb300 import cases


def _box_vent(nx=16, ny=8, nz=8, **kw):
    return cases.heated_channel_3d(
        nx, ny, nz, mg_levels=2, init_perturb=0.1,
        boxes=[cases.Box(nx // 4, nx // 4 + 3, 0, 3, 2, 5, thermal=cases.HEAT_FLUX, T_value=100.0)],
        vents=[cases.Vent(face=5, a0=nx // 2, a1=nx // 2 + 4, b0=2, b1=6,
                          bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1, length_scale=0.02, T_in=15.0))],
        **kw)


SPECS = {
    "channel_box_vent": lambda: _box_vent(),
    "channel2d": lambda: cases.channel_2d(16, 8, 2, init_perturb=0.1),
    "room_buoyant": lambda: cases.room_3d(16, 8, 8, seed=2, mg_levels=2, h=0.32, init_perturb=0.1),
}


def _state(spec, seed):
    c = OracleCase(spec)
    rng = np.random.default_rng(seed)
    x = [np.array(a) for a in c.state]
    fl = c.geo.fluid
    for i in range(3):   # cross-flow so that the upwind switch flips inside the grid
        x[i] = x[i] + np.where(fl, 0.3 * rng.standard_normal(x[i].shape), 0.0)
    return c.geo, x, c.dt0


def _direction(geo, x, rng):
    return [np.where(geo.fluid, rng.standard_normal(geo.shape), 0.0) * 0.01 * max(float(np.max(np.abs(a))), 1e-3)
            for a in x]


def _cs(geo, x, d, dt, stages):
    y = transport.explicit_stage_rk(geo, [a + 1j * 1e-30 * b for a, b in zip(x, d)], dt, stages)
    return [np.imag(v) / 1e-30 for v in y]


@pytest.mark.parametrize("name,stages", [(n, 1) for n in SPECS] + [("channel_box_vent", 2), ("channel2d", 3)])
def test_complex_step_matches_central_differences(name, stages):
    geo, x, dt = _state(SPECS[name](), 1)
    rng = np.random.default_rng(2)
    d = _direction(geo, x, rng)
    cs = _cs(geo, x, d, dt, stages)
    h = 1e-5
    yp = transport.explicit_stage_rk(geo, [a + h * b for a, b in zip(x, d)], dt, stages)
    ym = transport.explicit_stage_rk(geo, [a - h * b for a, b in zip(x, d)], dt, stages)
    for a, p, m in zip(cs, yp, ym):
        fd = (p - m) / (2 * h)
        assert np.max(np.abs(a - fd)) <= 1e-6 * max(float(np.max(np.abs(a))), 1e-300)


@pytest.mark.parametrize("stages", [1, 2])
def test_probed_jacobian_equals_dense_jacobian(stages):
    spec = _box_vent(8, 4, 4)
    geo, x, dt = _state(spec, 3)
    adj = ExplicitAdjoint(geo, dt, x, stages)
    N = int(np.prod(geo.shape))
    dense = np.zeros((6 * N, 6 * N))
    for j in range(6 * N):
        e = np.zeros(6 * N)
        e[j] = 1.0
        col = _cs(geo, x, [e[i * N:(i + 1) * N].reshape(geo.shape) for i in range(6)], dt, stages)
        dense[:, j] = np.concatenate([a.ravel() for a in col])
    J = adj.J.toarray()
    assert np.max(np.abs(J - dense)) <= 1e-13 * np.max(np.abs(dense))


@pytest.mark.parametrize("name,stages", [(n, 1) for n in SPECS] + [("channel_box_vent", 2), ("channel2d", 3)])
def test_vjp_adjoint_identity(name, stages):
    geo, x, dt = _state(SPECS[name](), 4)
    adj = ExplicitAdjoint(geo, dt, x, stages)
    rng = np.random.default_rng(5)
    d = _direction(geo, x, rng)
    ybar = [rng.standard_normal(geo.shape) for _ in range(6)]
    jd = _cs(geo, x, d, dt, stages)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(jd, ybar))
    xbar = adj.vjp(*ybar)
    rhs = sum(float(np.sum(a * b)) for a, b in zip(d, xbar))
    scale = sum(float(np.sum(np.abs(a * b))) for a, b in zip(d, xbar))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_wall_omega_cells_have_no_derivative():
    """omega next to a wall is set to a constant after the stage, so no input
    moves it: its cotangent reaches nothing."""
    geo, x, dt = _state(SPECS["channel_box_vent"](), 6)
    adj = ExplicitAdjoint(geo, dt, x, 1)
    ow = transport.wall_omega(geo) > 0
    assert ow.any()
    rng = np.random.default_rng(7)
    ybar = [np.zeros(geo.shape) for _ in range(6)]
    ybar[5] = np.where(ow, rng.standard_normal(geo.shape), 0.0)
    assert all(np.max(np.abs(a)) == 0.0 for a in adj.vjp(*ybar))


@pytest.mark.parametrize("name", list(SPECS))
def test_hand_derived_adjoint_equals_complex_step_adjoint(name):
    geo, x, dt = _state(SPECS[name](), 8)
    adj = ExplicitAdjoint(geo, dt, x, 1)
    rng = np.random.default_rng(9)
    ybar = [rng.standard_normal(geo.shape) for _ in range(6)]
    for a, b in zip(adj.vjp(*ybar), explicit_vjp_by_hand(geo, x, dt, ybar)):
        assert np.max(np.abs(a - b)) <= 1e-13 * max(float(np.max(np.abs(a))), 1e-300)
