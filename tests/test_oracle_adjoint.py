"""Pins of the projection adjoint (oracle/adjoint.py): the transpose of the
Jacobian of u* -> (u^{n+1}, p) must equal, on tiny grids, the transpose of
the dense Jacobian built column by column from the forward oracle with an
exact dense solve (brute force), and on larger grids it must satisfy the
adjoint identity <Pi(u + d) - Pi(u), ybar> = <d, J^T ybar>, exact for an
affine map."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.adjoint import ProjectionAdjoint, local_jacobian
from oracle.geometry import Geometry
from oracle.poisson import dense_operator, poisson_rhs, project
from paper_2603_21869_gb300 import cases


def _channel_box(nx=8, ny=4, nz=4):
    spec = cases.heated_channel_3d(nx, ny, nz, mg_levels=2, init_perturb=0.1,
                                   boxes=[cases.Box(3, 5, 0, 2, 1, 3, thermal=cases.ADIABATIC)])
    return spec


def _specs():
    return {
        "channel_box": _channel_box(),
        "channel2d": cases.channel_2d(12, 6, 2),
        "room": cases.room_3d(16, 8, 8, seed=2, mg_levels=2, h=0.32),
    }


class Forward:
    """Pi(u*) = (u', v', w', p) with the exact dense solve of A (dense_operator:
    solid rows and columns the identity), factorised once."""

    def __init__(self, geo, lev0, dt):
        self.geo, self.lev0, self.dt = geo, lev0, dt
        self.lu = sla.lu_factor(dense_operator(lev0))

    def __call__(self, u, v, w):
        b = poisson_rhs(self.geo, u, v, w, self.dt)
        rhs = np.where(self.lev0.solid, 0.0, b).ravel()
        p = sla.lu_solve(self.lu, rhs).reshape(self.lev0.shape)
        p = np.where(self.lev0.solid, 0.0, p)
        return list(project(self.geo, self.lev0, u, v, w, p, self.dt)) + [p]


@pytest.mark.parametrize("name", list(_specs()))
def test_vjp_equals_dense_jacobian_transpose(name):
    spec = _specs()[name]
    geo = Geometry(spec)
    lev0 = geo.level0
    dt = 0.05
    shape = geo.shape
    N = int(np.prod(shape))
    forward = Forward(geo, lev0, dt)
    zero = [np.zeros(shape)] * 3
    y0 = np.concatenate([a.ravel() for a in forward(*zero)])
    J = np.zeros((4 * N, 3 * N))
    for j in range(3 * N):
        x = np.zeros(3 * N)
        x[j] = 1.0
        parts = [x[i * N:(i + 1) * N].reshape(shape) for i in range(3)]
        J[:, j] = np.concatenate([a.ravel() for a in forward(*parts)]) - y0
    adj = ProjectionAdjoint(geo, lev0, dt)
    rng = np.random.default_rng(7)
    ybar = rng.standard_normal(4 * N)
    want = J.T @ ybar
    got = adj.vjp(*[ybar[i * N:(i + 1) * N].reshape(shape) for i in range(4)])
    got = np.concatenate([a.ravel() for a in got])
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))
    d = rng.standard_normal(3 * N)
    lin = adj.forward_linear(*[d[i * N:(i + 1) * N].reshape(shape) for i in range(3)])
    lin = np.concatenate([a.ravel() for a in lin])
    assert np.max(np.abs(lin - J @ d)) <= 1e-11 * np.max(np.abs(J @ d))


def test_adjoint_identity_on_a_larger_room():
    spec = cases.room_3d(24, 12, 12, seed=4, mg_levels=2, h=0.2)
    geo = Geometry(spec)
    lev0 = geo.level0
    dt = 0.02
    shape = geo.shape
    rng = np.random.default_rng(8)
    u = [rng.standard_normal(shape) for _ in range(3)]
    d = [rng.standard_normal(shape) for _ in range(3)]
    ybar = [rng.standard_normal(shape) for _ in range(4)]
    forward = Forward(geo, lev0, dt)
    a = forward(*[x + y for x, y in zip(u, d)])
    b = forward(*u)
    lhs = sum(float(np.sum((p - q) * yb)) for p, q, yb in zip(a, b, ybar))
    xbar = ProjectionAdjoint(geo, lev0, dt).vjp(*ybar)
    rhs = sum(float(np.sum(x * y)) for x, y in zip(d, xbar))
    assert rhs == pytest.approx(lhs, rel=1e-10)


def test_solid_cells_pass_through_and_pressure_cotangent():
    """Solid-cell velocities are copied by the projection, so their cotangent
    passes through unchanged; a pressure cotangent alone reaches u* only
    through b(u*)."""
    spec = _channel_box()
    geo = Geometry(spec)
    adj = ProjectionAdjoint(geo, geo.level0, 0.05)
    rng = np.random.default_rng(9)
    yb = [np.where(geo.solid, rng.standard_normal(geo.shape), 0.0) for _ in range(3)]
    xb = adj.vjp(*yb)
    for x, y in zip(xb, yb):
        assert np.array_equal(x[geo.solid], y[geo.solid])
        assert np.max(np.abs(x[geo.fluid])) == 0.0
    pb = rng.standard_normal(geo.shape)
    z = np.zeros(geo.shape)
    xp = adj.vjp(z, z, z, pb)
    assert all(np.all(x[geo.solid] == 0.0) for x in xp)
    assert max(float(np.max(np.abs(x))) for x in xp) > 0.0


def test_local_jacobian_rejects_a_wider_stencil():
    """The colour probing is exact only for maps that reach one index per
    axis; a two-cell shift is detected."""
    with pytest.raises(AssertionError):
        local_jacobian(lambda x: [np.roll(x[0], 2, axis=0)], 1, (9, 3, 3))
