"""The step's adjoint kernels (FP64) against the oracle's adjoints on the same
state and cotangents: fvm_destruction_vjp against DestructionAdjoint (partial
derivatives written out, gradient stencils transposed by colour probing),
fvm_explicit_vjp against ExplicitAdjoint (complex-step Jacobian of the forward
oracle) and fvm_step_vjp against StepAdjoint (the whole step, exact solve).

The destruction and explicit products involve no solve: FP64 agreement to
1e-10 of each field's largest cotangent.  The step product contains the
adjoint pressure solve, which the GPU runs to a relative residual of 1e-13
where the oracle solves exactly: 1e-8 (the projection adjoint's bound)."""
import numpy as np
import pytest

from oracle.adjoint import DestructionAdjoint, ExplicitAdjoint, StepAdjoint
from oracle.geometry import Geometry
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

STATE = ("u", "v", "w", "T", "k", "omega")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def channel_box(**kw):
    spec = cases.heated_channel_3d(24, 8, 8, mg_levels=3, init_perturb=0.05,
                                   boxes=[cases.Box(6, 10, 2, 5, 0, 4, thermal=cases.HEAT_FLUX, T_value=150.0),
                                          cases.Box(14, 17, 4, 8, 3, 6, thermal=cases.FIXED_T, T_value=40.0)],
                                   vents=[cases.Vent(face=5, a0=10, a1=14, b0=2, b1=6,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(**kw)


SPECS = {
    "channel3d_boxes_vent": lambda: channel_box(fixed_vcycles=3),
    "room_buoyant": lambda: cases.room_3d(16, 16, 8, seed=3, mg_levels=2, h=0.16, precision=cases.FP64,
                                          fixed_vcycles=3),
    "channel2d": lambda: cases.channel_2d(24, 12, 2, fixed_vcycles=3, init_perturb=0.05),
}


def rel_err(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / scale if scale > 0 else float(np.max(np.abs(a)))


def stepped_state(spec, steps=2):
    """The case after a few steps (nonzero gradients and eddy viscosity everywhere)."""
    c = binding.Case(spec)
    c.step(steps)
    f = c.read()
    return c, [f[n] for n in STATE], c.info()["dt"]


@pytest.mark.parametrize("name", list(SPECS))
def test_destruction_vjp_matches_oracle(name):
    spec = SPECS[name]()
    c, x, dt = stepped_state(spec)
    try:
        geo = Geometry(spec)
        rng = np.random.default_rng(5)
        ybar = [rng.standard_normal(geo.shape) for _ in range(5)]
        got = c.destruction_vjp(0.5 * dt, *ybar)
        after = c.read()
    finally:
        c.close()
    u, v, w, T, k, om = x
    D = DestructionAdjoint(geo, 0.5 * dt, [u, v, w, k, om])
    du, dv, dw, dk, dom = D.vjp(ybar[3], ybar[4])
    want = [ybar[0] + du, ybar[1] + dv, ybar[2] + dw, dk, dom]
    for n, g, r in zip(("u", "v", "w", "k", "omega"), got, want):
        assert rel_err(g, r) <= 1e-10, (name, n, rel_err(g, r))
    for n, a in zip(STATE, x):   # the call leaves the case alone
        assert np.array_equal(after[n], a), n


@pytest.mark.parametrize("name", list(SPECS))
def test_explicit_vjp_matches_oracle(name):
    spec = SPECS[name]()
    c, x, dt = stepped_state(spec)
    try:
        geo = Geometry(spec)
        rng = np.random.default_rng(6)
        ybar = [rng.standard_normal(geo.shape) for _ in range(6)]
        got = c.explicit_vjp(dt, *ybar)
    finally:
        c.close()
    want = ExplicitAdjoint(geo, dt, x).vjp(*ybar)
    for n, g, r in zip(STATE, got, want):
        assert rel_err(g, r) <= 1e-10, (name, n, rel_err(g, r))


@pytest.mark.parametrize("name", list(SPECS))
def test_step_vjp_matches_oracle(name):
    spec = SPECS[name]()
    c, x, dt = stepped_state(spec)
    try:
        geo = Geometry(spec)
        rng = np.random.default_rng(7)
        ybar = [rng.standard_normal(geo.shape) for _ in range(7)]   # u, v, w, p, T, k, omega
        before = c.read()
        rhs_before = c.read_rhs()
        got, rel = c.step_vjp(dt, *ybar)
        after = c.read()
        rhs_after = c.read_rhs()
    finally:
        c.close()
    assert rel <= 1e-13
    want = StepAdjoint(geo, dt, x).vjp(*ybar)
    for n, g, r in zip(STATE, got, want):
        assert rel_err(g, r) <= 1e-8, (name, n, rel_err(g, r))
    for n in cases.FIELDS:   # fields, p and b restored
        assert np.array_equal(after[n], before[n]), n
    assert np.array_equal(rhs_after, rhs_before)


def test_vjp_calls_reject_bad_arguments():
    spec = SPECS["channel2d"]()
    with binding.Case(spec.replace(precision=cases.FP32)) as c:
        z = [np.zeros((spec.nx, spec.ny, spec.nz))] * 7
        with pytest.raises(binding.FvmError) as e:
            c.destruction_vjp(0.01, *z[:5])
        assert e.value.status == binding.ERR_INVALID
    with binding.Case(spec.replace(rk_stages=3)) as c:
        with pytest.raises(binding.FvmError) as e:
            c.explicit_vjp(0.01, *z[:6])
        assert e.value.status == binding.ERR_INVALID
    with binding.Case(spec) as c:
        with pytest.raises(binding.FvmError) as e:
            c.step_vjp(-1.0, *z)
        assert e.value.status == binding.ERR_INVALID
