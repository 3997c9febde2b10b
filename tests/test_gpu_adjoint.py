"""fvm_projection_vjp against the oracle's projection adjoint on the same
cotangents (FP64 cases).

The GPU solves A lambda = q with V-cycles to a relative residual of 1e-13
where the oracle solves exactly; the error in lambda is then at most
cond(A) * 1e-13 relative, and cond(A) of these grids is below 1e4, so the
solve's part of xbar (xbar - ybar) must agree to 1e-8 of its magnitude."""
import numpy as np
import pytest

from oracle.adjoint import ProjectionAdjoint
from oracle.geometry import Geometry
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def channel_box(**kw):
    spec = cases.heated_channel_3d(48, 16, 16, mg_levels=3, init_perturb=0.02,
                                   boxes=[cases.Box(10, 16, 4, 10, 0, 7, thermal=cases.HEAT_FLUX, T_value=150.0)],
                                   vents=[cases.Vent(face=5, a0=20, a1=28, b0=4, b1=12,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(**kw)


SPECS = {
    "channel3d_box_vent": lambda: channel_box(fixed_vcycles=2),
    "room_buoyant": lambda: cases.room_3d(32, 16, 16, seed=3, mg_levels=3, h=0.16, precision=cases.FP64,
                                          fixed_vcycles=2),
    "channel2d_ragged": lambda: cases.channel_2d(48, 20, 3, fixed_vcycles=2, init_perturb=0.05),
    "room_krylov": lambda: cases.room_3d(32, 16, 16, seed=5, mg_levels=3, h=0.16, precision=cases.FP64,
                                         fixed_vcycles=2, krylov=1),
}


@pytest.mark.parametrize("name", list(SPECS))
def test_projection_vjp_matches_oracle(name):
    spec = SPECS[name]()
    dt = 0.01
    geo = Geometry(spec)
    rng = np.random.default_rng(21)
    ybar = [rng.standard_normal(geo.shape) for _ in range(4)]
    with binding.Case(spec) as c:
        c.step(1)
        before = c.read()
        rhs_before = c.read_rhs()
        (xu, xv, xw), rel = c.projection_vjp(dt, *ybar)
        after = c.read()
        rhs_after = c.read_rhs()
    assert rel <= 1e-13
    for f in cases.FIELDS:
        assert np.array_equal(before[f], after[f]), f
    assert np.array_equal(rhs_before, rhs_after)
    want = ProjectionAdjoint(geo, geo.level0, dt).vjp(*ybar)
    scale = max(float(np.max(np.abs(ref - yb))) for ref, yb in zip(want, ybar[:3]))
    assert scale > 0.0
    for got, ref, yb in zip((xu, xv, xw), want, ybar[:3]):
        assert np.max(np.abs(got - ref)) <= TOL * scale
        assert np.array_equal(got[geo.solid], yb[geo.solid])


def test_projection_vjp_zero_and_linear():
    """A zero cotangent gives zero; the map is linear in the cotangent."""
    spec = SPECS["channel3d_box_vent"]()
    geo = Geometry(spec)
    rng = np.random.default_rng(22)
    y1 = [rng.standard_normal(geo.shape) for _ in range(4)]
    y2 = [rng.standard_normal(geo.shape) for _ in range(4)]
    z = np.zeros(geo.shape)
    with binding.Case(spec) as c:
        (a, b, w), rel = c.projection_vjp(0.02, z, z, z, z)
        assert all(np.all(x == 0.0) for x in (a, b, w))
        x1, _ = c.projection_vjp(0.02, *y1)
        x2, _ = c.projection_vjp(0.02, *y2)
        x12, _ = c.projection_vjp(0.02, *[p + 2.0 * q for p, q in zip(y1, y2)])
    for p, q, r in zip(x1, x2, x12):
        assert np.max(np.abs(r - (p + 2.0 * q))) <= 1e-8 * np.max(np.abs(r))


def test_projection_vjp_rejects_bad_calls():
    spec = channel_box(fixed_vcycles=2, precision=cases.FP32)
    geo = Geometry(spec)
    z = np.zeros(geo.shape)
    with binding.Case(spec) as c:
        with pytest.raises(binding.FvmError) as ei:
            c.projection_vjp(0.01, z, z, z)
        assert ei.value.status == binding.ERR_INVALID
    with binding.Case(channel_box(fixed_vcycles=2)) as c:
        with pytest.raises(binding.FvmError):
            c.projection_vjp(-1.0, z, z, z)
        (xu, _, _), rel = c.projection_vjp(0.01, z + 1.0, z, z, max_vcycles=4, rel_tol=1e-30,
                                           allow_not_converged=True)
        assert rel > 1e-30 and np.all(np.isfinite(xu))
