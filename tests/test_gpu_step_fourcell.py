"""The FP32-field step kernels (the projection four cells per thread where
nx % 4 = 0, every other stage and other nx one cell per thread) stage by
stage against the oracle's FP64 stage on
the same state: the GPU's FP32 state after a few steps, read back exactly, is
the oracle's input, and each stage's output must agree to 1e-5 of each field's
largest magnitude, the velocity components' of the largest component (FP32
rounding of differences and quotients; a stage involves no solve).  The cases mix regular groups with groups holding walls,
obstacles, vents and outlets, x extents whose row segments are 16, 64 and 128
cells (nx = 20 leaves most lanes of its segment outside the grid), a
collapsed z axis, nx % 4 != 0 (the one-cell form) and the Runge-Kutta
stages."""
import numpy as np
import pytest

from oracle.step import OracleCase
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

TOL = 1e-5
STATE = ("u", "v", "w", "T", "k", "omega")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def rel_err(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / scale if scale > 0 else float(np.max(np.abs(a)))


def box_channel(nx, ny, nz, mg_levels, precision=cases.FP32, **kw):
    spec = cases.heated_channel_3d(nx, ny, nz, mg_levels=mg_levels, precision=precision, init_perturb=0.05,
                                   boxes=[cases.Box(nx // 4, nx // 4 + 3, 2, 5, 0, nz // 2, thermal=cases.HEAT_FLUX,
                                                    T_value=150.0),
                                          cases.Box(nx // 2, nx // 2 + 2, ny - 4, ny, 2, 5, thermal=cases.FIXED_T,
                                                    T_value=40.0)],
                                   vents=[cases.Vent(face=5, a0=nx // 2 - 4, a1=nx // 2, b0=2, b1=6,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(fixed_vcycles=3, **kw)


SPECS = {
    "room_64x32x32": lambda: cases.room_3d(64, 32, 32, seed=3, mg_levels=3, h=0.08, precision=cases.FP32,
                                           fixed_vcycles=3),
    "room_bf16": lambda: cases.room_3d(64, 32, 32, seed=5, mg_levels=3, h=0.08, precision=cases.BF16_MIXED,
                                       fixed_vcycles=3),
    "channel_48x16x16": lambda: box_channel(48, 16, 16, 3),
    "channel_128x12x8": lambda: box_channel(128, 12, 8, 3),
    "channel_20x12x8": lambda: box_channel(20, 12, 8, 2),
    "channel_50x12x8_onecell": lambda: box_channel(50, 12, 8, 2),
    "channel2d_48x20": lambda: cases.channel_2d(48, 20, 3, fixed_vcycles=3, init_perturb=0.05,
                                                precision=cases.FP32),
}


def gpu_state(c):
    f = c.read()
    return [f[n] for n in STATE], f["p"]


def check(got, want, names, label):
    # velocity components against the largest speed component (a component that stays at
    # rounding level, such as w of a 2D case in FP32 at 1e-10, has no scale of its own)
    vscale = max(float(np.max(np.abs(want[n]))) for n in ("u", "v", "w"))
    errs = {n: (float(np.max(np.abs(got[n] - want[n]))) / vscale if n in ("u", "v", "w") else rel_err(got[n], want[n]))
            for n in names}
    bad = {n: e for n, e in errs.items() if not e <= TOL}
    assert not bad, f"{label}: {bad} (all {errs})"


@pytest.mark.parametrize("name", list(SPECS))
def test_stages_match_oracle_on_the_same_state(name):
    spec = SPECS[name]()
    with binding.Case(spec) as c:
        c.step(3)
        c.run_stage(binding.STAGE_DT)
        dt = c.info()["dt"]
        # destruction half step (writes nu_t for the explicit stage)
        x, p = gpu_state(c)
        c.run_stage(binding.STAGE_DESTRUCTION)
        o = OracleCase(spec, state=x, p=p)
        o.dt = dt
        o.destruction_half()
        check(c.read(STATE), o.fields(), ("k", "omega"), f"{name} destruction")
        # explicit stage
        x, p = gpu_state(c)
        c.run_stage(binding.STAGE_EXPLICIT)
        o = OracleCase(spec, state=x, p=p)
        o.dt = dt
        o.explicit()
        check(c.read(STATE), o.fields(), STATE, f"{name} explicit")
        # the second half step fused with the right-hand side runs inside step(); run the stages here
        x, p = gpu_state(c)
        c.run_stage(binding.STAGE_DESTRUCTION)
        c.run_stage(binding.STAGE_RHS)
        o = OracleCase(spec, state=x, p=p)
        o.dt = dt
        o.destruction_half()
        o.rhs()
        check(c.read(STATE), o.fields(), ("k", "omega"), f"{name} destruction 2")
        assert rel_err(c.read_rhs(), o.b) <= TOL, f"{name} rhs"
        c.run_stage(binding.STAGE_SOLVE)
        # projection
        x, p = gpu_state(c)
        c.run_stage(binding.STAGE_PROJECT)
        o = OracleCase(spec, state=x, p=p)
        o.dt = dt
        o.project()
        check(c.read(STATE), o.fields(), ("u", "v", "w"), f"{name} project")


@pytest.mark.parametrize("name", ["channel_48x16x16", "room_64x32x32"])
def test_steps_fuse_the_second_half_step_with_the_rhs(name):
    """step() runs the second destruction half step and the right-hand side as one pass; the
    same steps through the separate stages give the same fields to FP32 rounding."""
    spec = SPECS[name]()
    with binding.Case(spec) as a, binding.Case(spec) as b:
        a.step(2)
        for _ in range(2):
            for st in (binding.STAGE_DT, binding.STAGE_DESTRUCTION, binding.STAGE_EXPLICIT,
                       binding.STAGE_DESTRUCTION, binding.STAGE_RHS, binding.STAGE_SOLVE, binding.STAGE_PROJECT):
                b.run_stage(st)
        fa, fb = a.read(), b.read()
    for n in cases.FIELDS:
        assert rel_err(fa[n], fb[n]) <= 1e-6, n


@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("name", ["channel_48x16x16", "room_64x32x32", "channel_20x12x8"])
def test_runge_kutta_stages_match_oracle(name, rk):
    spec = SPECS[name]().replace(rk_stages=rk)
    with binding.Case(spec) as c:
        c.step(2)
        c.run_stage(binding.STAGE_DT)
        dt = c.info()["dt"]
        x, p = gpu_state(c)
        c.run_stage(binding.STAGE_EXPLICIT)
        o = OracleCase(spec, state=x, p=p)
        o.dt = dt
        o.explicit()
        check(c.read(STATE), o.fields(), STATE, f"{name} rk{rk}")
