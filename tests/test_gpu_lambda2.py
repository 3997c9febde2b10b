"""The lambda_2 vortex criterion (fvm_lambda2, Section 3.2.3) against the
oracle on the same velocity fields.

The error bound follows from the arithmetic: M = S^2 + Omega^2 =
(G G + G^T G^T) / 2 for the cell gradient G, so |M| <= |G|_F^2, and the
eigenvalues of a symmetric matrix move by at most the perturbation of the
matrix (Weyl).  The kernel's rounding in G and in the Jacobi rotations is a
few eps |G|_F^2, so the difference is bounded by tol * max over cells of
|G|_F^2: 1e-10 for FP64, 1e-4 for the FP32 fields."""
import numpy as np
import pytest

from oracle.diagnostics import lambda2 as oracle_lambda2
from oracle.geometry import U, V, W, Geometry, cell_gradient
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

TOL = {cases.FP64: 1e-10, cases.FP32: 1e-4, cases.BF16_MIXED: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def grad_scale(geo, u, v, w):
    """max over cells of |G|_F^2."""
    acc = np.zeros(geo.shape)
    for phi, f in ((u, U), (v, V), (w, W)):
        for g in cell_gradient(geo, phi, f):
            acc += g * g
    return float(np.max(acc))


def check_case(spec, steps, tol):
    with binding.Case(spec) as c:
        if steps:
            c.step(steps)
        vel = c.read(("u", "v", "w"))
        before = c.read()
        got = c.lambda2()
        after = c.read()
    for f in cases.FIELDS:
        assert np.array_equal(before[f], after[f]), f"fvm_lambda2 changed {f}"
    geo = Geometry(spec)
    ref = oracle_lambda2(geo, vel["u"], vel["v"], vel["w"])
    scale = grad_scale(geo, vel["u"], vel["v"], vel["w"])
    assert scale > 0.0
    err = float(np.max(np.abs(got - ref)))
    assert err <= tol * scale, (err / scale, tol)
    assert np.all(got[~geo.fluid] == 0.0)
    # the sign decides where vortex cores are: it agrees wherever lambda_2 is
    # clear of the error bound
    clear = np.abs(ref) > 10 * tol * scale
    assert np.array_equal(np.sign(got[clear]), np.sign(ref[clear]))
    return got, ref


def room_small(precision=cases.FP64, **kw):
    return cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=precision, **kw)


def channel_box(precision=cases.FP64, **kw):
    spec = cases.heated_channel_3d(48, 16, 16, mg_levels=3, precision=precision, init_perturb=0.05,
                                   boxes=[cases.Box(10, 16, 4, 10, 0, 7, thermal=cases.HEAT_FLUX, T_value=150.0)],
                                   vents=[cases.Vent(face=5, a0=20, a1=28, b0=4, b1=12,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(**kw)


SPECS = {
    "channel2d_ragged": lambda p: cases.channel_2d(48, 20, 3, fixed_vcycles=3, init_perturb=0.05, precision=p),
    "channel3d_box_vent": lambda p: channel_box(precision=p, fixed_vcycles=3),
    "room_buoyant": lambda p: room_small(precision=p, fixed_vcycles=3),
    "tiny_3d": lambda p: cases.heated_channel_3d(8, 4, 4, mg_levels=2, fixed_vcycles=2, init_perturb=0.1, precision=p),
}


@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32, cases.BF16_MIXED], ids=["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", list(SPECS))
def test_lambda2_matches_oracle(name, prec):
    check_case(SPECS[name](prec), 3, TOL[prec])


def test_lambda2_initial_state_and_mid_size_room_fp32():
    """A 256 x 128 x 64 room (2 M cells, thousands of blocks, vents and
    heated boxes) after two FP32 steps, and a channel's seeded initial state."""
    check_case(cases.room_3d(256, 128, 64, seed=5, mg_levels=5, h=0.04, precision=cases.FP32,
                             fixed_vcycles=4), 2, 1e-4)
    check_case(cases.heated_channel_3d(64, 16, 16, mg_levels=3, init_perturb=0.3), 0, 1e-10)


@pytest.mark.slow
@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32], ids=["fp64", "fp32"])
def test_lambda2_full_size_heated_channel(prec):
    """The 256 x 64 x 64 channel after two steps, every cell."""
    check_case(cases.heated_channel_3d(precision=prec, fixed_vcycles=3), 2, TOL[prec])


def _box_spec(prec, n=(16, 12, 8)):
    faces = [cases.Patch(cases.OUTLET) for _ in range(6)]
    return cases.CaseSpec(nx=n[0], ny=n[1], nz=n[2], Lx=1.0, Ly=0.75, Lz=0.5, nu=1e-5, faces=faces,
                          dt=0.01, dt_adapt=0, mg_levels=2, init_k=1e-3, init_omega=1.0, precision=prec)


def _centres(spec):
    geo = Geometry(spec)
    axes = [(np.arange(n) + 0.5) * h for n, h in zip(geo.shape, geo.h)]
    return np.meshgrid(*axes, indexing="ij")


@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32], ids=["fp64", "fp32"])
def test_closed_forms_on_the_gpu(prec):
    """Written linear fields: rigid rotation gives -W^2, pure strain +a^2,
    simple shear 0, a stretched vortex a^2/4 - W^2 (interior cells, where the
    central gradient is exact); a fluid at rest gives 0 everywhere."""
    spec = _box_spec(prec)
    X = _centres(spec)
    W_, a = 1.7, 0.9
    fields = {
        "rotation": ([-W_ * (X[1] - 0.4), W_ * (X[0] - 0.5), 0 * X[0]], -W_ * W_),
        "strain": ([a * X[0], -a * X[1], 0 * X[0]], a * a),
        "shear": ([2.3 * X[1], 0 * X[0], 0 * X[0]], 0.0),
        "stretched": ([-a / 2 * X[0] - W_ * X[1], W_ * X[0] - a / 2 * X[1], a * X[2]], a * a / 4 - W_ * W_),
        "rest": ([0 * X[0], 0 * X[0], 0 * X[0]], 0.0),
    }
    rtol = 1e-12 if prec == cases.FP64 else 1e-5
    with binding.Case(spec) as c:
        for name, (uvw, expect) in fields.items():
            c.write(dict(zip(("u", "v", "w"), uvw)))
            lam = c.lambda2()
            inner = lam[1:-1, 1:-1, 1:-1]
            assert np.allclose(inner, expect, rtol=rtol, atol=rtol * 6.0), name
            if name == "rest":
                assert np.all(lam == 0.0)


def test_lambda2_leaves_the_step_unchanged():
    """The diagnostic uses only scratch memory: steps taken after it are
    bitwise those taken without it."""
    spec = channel_box(fixed_vcycles=0, mg_rel_tol=1e-8, max_vcycles=40)
    out = []
    for call in (False, True):
        with binding.Case(spec) as c:
            c.step(1)
            if call:
                c.lambda2()
            c.step(2)
            out.append(c.read())
    for f in cases.FIELDS:
        assert np.array_equal(out[0][f], out[1][f]), f


def test_lambda2_profiled_and_invalid_calls():
    spec = room_small(precision=cases.FP32, fixed_vcycles=2)
    with binding.Case(spec) as c:
        c.step(1)
        c.profile(True)
        c.lambda2()
        stats = c.profile_read()
        c.profile(False)
        assert "lambda2" in stats and stats["lambda2"]["launches"] == 1
        assert stats["lambda2"]["bytes"] == pytest.approx(c.N * (3 * 4 + 1 + 8))
        with pytest.raises(binding.FvmError):
            c.lambda2(out=np.empty(c.N - 1))
