"""Pin of the whole-step adjoint (oracle/adjoint.py, StepAdjoint): against
central differences of the forward step (destruction dt/2, explicit stage,
destruction dt/2, right-hand side, exact pressure solve, projection) built
here from the oracle's stage functions, <J d, ybar> = <d, J^T ybar> to the
accuracy of the differences, for forward Euler and the Runge-Kutta stage."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.adjoint import StepAdjoint
from oracle.destruction import destruction_step
from oracle.poisson import dense_operator, poisson_rhs, project
from oracle.step import OracleCase
from oracle.transport import explicit_stage_rk
from paper_2603_21869_gb300 import cases


class ForwardStep:
    def __init__(self, geo, dt, stages):
        self.geo, self.dt, self.stages = geo, dt, stages
        self.lu = sla.lu_factor(dense_operator(geo.level0))

    def __call__(self, x):
        geo, dt = self.geo, self.dt
        u, v, w, T, k, om = x
        k, om = destruction_step(geo, u, v, w, k, om, 0.5 * dt)
        u, v, w, T, k, om = explicit_stage_rk(geo, [u, v, w, T, k, om], dt, self.stages)
        k, om = destruction_step(geo, u, v, w, k, om, 0.5 * dt)
        b = poisson_rhs(geo, u, v, w, dt)
        p = sla.lu_solve(self.lu, np.where(geo.solid, 0.0, b).ravel()).reshape(geo.shape)
        p = np.where(geo.solid, 0.0, p)
        u, v, w = project(geo, geo.level0, u, v, w, p, dt)
        return [u, v, w, p, T, k, om]


SPECS = {
    "channel_box_vent": lambda: cases.heated_channel_3d(
        16, 8, 8, mg_levels=2, init_perturb=0.1,
        boxes=[cases.Box(4, 7, 0, 3, 2, 5, thermal=cases.HEAT_FLUX, T_value=100.0)],
        vents=[cases.Vent(face=5, a0=8, a1=12, b0=2, b1=6,
                          bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1, length_scale=0.02, T_in=15.0))]),
    "room_buoyant": lambda: cases.room_3d(16, 8, 8, seed=2, mg_levels=2, h=0.32, init_perturb=0.1),
}


@pytest.mark.parametrize("name,stages", [("channel_box_vent", 1), ("room_buoyant", 1), ("channel_box_vent", 2)])
def test_step_vjp_matches_central_differences(name, stages):
    spec = SPECS[name]()
    c = OracleCase(spec)
    geo, dt = c.geo, c.dt0
    rng = np.random.default_rng(11)
    x = [np.array(a) for a in c.state]
    for i in range(3):
        x[i] = x[i] + np.where(geo.fluid, 0.3 * rng.standard_normal(geo.shape), 0.0)
    d = [np.where(geo.fluid, rng.standard_normal(geo.shape), 0.0) * 0.01 * max(float(np.max(np.abs(a))), 1e-3)
         for a in x]
    ybar = [rng.standard_normal(geo.shape) for _ in range(7)]
    xbar = StepAdjoint(geo, dt, x, stages).vjp(*ybar)
    rhs = sum(float(np.sum(a * b)) for a, b in zip(d, xbar))
    scale = sum(float(np.sum(np.abs(a * b))) for a, b in zip(d, xbar))
    F = ForwardStep(geo, dt, stages)
    h = 1e-6
    yp = F([a + h * b for a, b in zip(x, d)])
    ym = F([a - h * b for a, b in zip(x, d)])
    lhs = sum(float(np.sum((p - m) * yb)) for p, m, yb in zip(yp, ym, ybar)) / (2 * h)
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs, scale)
