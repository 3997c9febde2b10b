"""The Chebyshev sweep weights (smoother 1: sweep i of n on a side takes the
reciprocal of a root of the degree-n Chebyshev polynomial of [1/4, 2]) against
the oracle's: FP64 steps and V-cycles within 1e-10, with the fused first
sweeps of the residual and restriction kernels, the coarse single-CTA levels,
per-level sweep counts, the flexible-CG acceleration, several V-cycles per
outer residual and a batch; the reduced-precision paths within 1e-4 of the
FP64 oracle; argument checks."""
import numpy as np
import pytest

from oracle.poisson import direct_solve
from oracle.step import OracleCase
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
STATE = ("u", "v", "w", "T", "k", "omega")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def rel_err(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / scale if scale > 0 else float(np.max(np.abs(a)))


def channel_box(**kw):
    spec = cases.heated_channel_3d(48, 16, 16, mg_levels=3, init_perturb=0.02,
                                   boxes=[cases.Box(10, 16, 4, 10, 0, 7, thermal=cases.HEAT_FLUX, T_value=150.0)],
                                   vents=[cases.Vent(face=5, a0=20, a1=28, b0=4, b1=12,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(**{"smoother": 1, **kw})


SPECS = {
    "channel3d_box_vent": lambda: channel_box(fixed_vcycles=3),
    "room_buoyant_v22_krylov": lambda: cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=cases.FP64,
                                                     fixed_vcycles=3, pre_sweeps=2, post_sweeps=2, krylov=1,
                                                     smoother=1),
    "channel2d_v41_coarse2": lambda: cases.channel_2d(48, 20, 3, fixed_vcycles=3, init_perturb=0.05, pre_sweeps=4,
                                                      post_sweeps=1, coarse_sweeps=2, smoother=1),
}


@pytest.mark.parametrize("name", list(SPECS))
def test_steps_match_oracle(name):
    spec = SPECS[name]()
    with binding.Case(spec) as c:
        st = c.step(3)
        got = c.read()
    o = OracleCase(spec).step(3)
    assert st["vcycles_total"] == 3 * spec.fixed_vcycles
    for f in cases.FIELDS:
        assert rel_err(got[f], o.fields()[f]) <= TOL64, (name, f, rel_err(got[f], o.fields()[f]))


def test_vcycles_match_oracle_and_reach_the_dense_solution():
    spec = channel_box(fixed_vcycles=1)
    o = OracleCase(spec)
    lev = o.mg.levels[0]
    b = np.where(lev.fluid, np.random.default_rng(11).normal(size=lev.shape), 0.0)
    p = np.zeros(lev.shape)
    with binding.Case(spec) as c:
        c.set_rhs(b)
        c.write({"p": p})
        for n in (1, 2, 4):
            rel = c.vcycle(n)
            for _ in range(n):
                p = o.mg.vcycle(p, b)
            assert rel_err(c.read(("p",))["p"], p) <= TOL64
            assert rel == pytest.approx(o.mg.rel_residual(p, b), rel=1e-6)
        c.vcycle(40)
        got = c.read(("p",))["p"]
    assert rel_err(got, direct_solve(lev, b)) <= 1e-9


@pytest.mark.parametrize("prec", [cases.FP32, cases.BF16_MIXED], ids=["fp32", "bf16"])
def test_reduced_precision_within_1e4_of_fp64_oracle(prec):
    """Several V-cycles per FP64 outer residual (inner_cycles 2: the level-0 pre-sweeps of the
    second cycle start from the first cycle's correction) and the flexible-CG step."""
    spec = cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=prec, mg_rel_tol=1e-8,
                         max_vcycles=40, pre_sweeps=2, post_sweeps=2, inner_cycles=2, krylov=1, smoother=1)
    with binding.Case(spec) as c:
        st = c.step(6)
        got = c.read()
    assert st["rel_residual"] <= 1e-8
    o = OracleCase(spec.replace(precision=cases.FP64)).step(6)
    for f in STATE:
        assert rel_err(got[f], o.fields()[f]) <= 1e-4, f


def test_batch_equals_each_case_alone():
    specs = [channel_box(fixed_vcycles=3), SPECS["room_buoyant_v22_krylov"](),
             channel_box(fixed_vcycles=3, smoother=0)]
    alone = []
    for s in specs:
        with binding.Case(s) as c:
            c.step(2)
            alone.append(c.read())
    cs = [binding.Case(s) for s in specs]
    try:
        with binding.Batch(cs) as b:
            b.step(2)
        got = [c.read() for c in cs]
    finally:
        for c in cs:
            c.close()
    for g, a in zip(got, alone):
        for f in cases.FIELDS:
            assert rel_err(g[f], a[f]) <= 1e-12, f


def test_fewer_cycles_than_the_constant_weight_on_a_room():
    """To the same tolerance, V(2,2) with the flexible-CG step needs fewer cycles per step with
    the Chebyshev weights than with the constant 6/7 (the oracle shows the same on this room)."""
    base = cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=cases.FP64, mg_rel_tol=1e-8,
                         max_vcycles=60, pre_sweeps=2, post_sweeps=2, krylov=1)
    total = {}
    for sm in (0, 1):
        with binding.Case(base.replace(smoother=sm)) as c:
            total[sm] = c.step(4)["vcycles_total"]
    assert total[1] < total[0], total


def test_arguments_are_checked():
    bad = [channel_box(smoother=2), channel_box(mg_variant=1), channel_box(pre_sweeps=17),
           channel_box(coarse_sweeps=17)]
    for spec in bad:
        with pytest.raises(binding.FvmError) as e:
            binding.Case(spec)
        assert e.value.status == binding.ERR_INVALID
