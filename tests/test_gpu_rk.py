"""The strong-stability-preserving Runge-Kutta explicit stage (rk_stages = 2
and 3; Section 2.6 leaves the explicit scheme open) against the oracle's:
FP64 within 1e-10 stage by stage and over full steps, graph and launch paths
bitwise, reduced precision within 1e-4 of the FP64 oracle, and batches
mixing schemes equal to each case stepped alone."""
import numpy as np
import pytest

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
    scale = np.max(np.abs(b))
    if scale == 0.0:
        return float(np.max(np.abs(a)))
    return float(np.max(np.abs(a - b)) / scale)


def room_small(precision=cases.FP64, **kw):
    return cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=precision, **kw)


def channel_box(precision=cases.FP64, **kw):
    spec = cases.heated_channel_3d(48, 16, 16, mg_levels=3, precision=precision, init_perturb=0.02,
                                   boxes=[cases.Box(10, 16, 4, 10, 0, 7, thermal=cases.HEAT_FLUX, T_value=150.0)],
                                   vents=[cases.Vent(face=5, a0=20, a1=28, b0=4, b1=12,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(**kw)


SPECS = {
    "channel3d_box_vent": lambda rk: channel_box(fixed_vcycles=3, rk_stages=rk),
    "room_buoyant": lambda rk: room_small(fixed_vcycles=3, rk_stages=rk),
    "channel2d_ragged": lambda rk: cases.channel_2d(48, 20, 3, fixed_vcycles=3, init_perturb=0.05, rk_stages=rk),
}


@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("name", list(SPECS))
def test_rk_explicit_stage_and_steps_match_oracle(name, rk):
    spec = SPECS[name](rk)
    o = OracleCase(spec)
    with binding.Case(spec) as c:
        c.run_stage(binding.STAGE_DT)
        o.update_dt()
        c.run_stage(binding.STAGE_DESTRUCTION)
        o.destruction_half()
        c.run_stage(binding.STAGE_EXPLICIT)
        o.explicit()
        got = c.read(STATE)
        for f in STATE:
            assert rel_err(got[f], o.fields()[f]) <= TOL64, (f, "explicit stage")
    # full steps
    with binding.Case(spec) as c:
        st = c.step(3)
        got = c.read()
    o = OracleCase(spec).step(3)
    assert st["rel_residual"] == pytest.approx(o.last_rel, rel=1e-6)
    for f in cases.FIELDS:
        assert rel_err(got[f], o.fields()[f]) <= TOL64, f


def test_rk_schemes_differ_from_forward_euler():
    """The three schemes give different fields (the switch reaches the kernels)."""
    outs = []
    for rk in (1, 2, 3):
        with binding.Case(SPECS["channel3d_box_vent"](rk)) as c:
            c.step(2)
            outs.append(c.read(STATE))
    for a, b in ((0, 1), (1, 2), (0, 2)):
        assert max(rel_err(outs[a][f], outs[b][f]) for f in STATE) > 1e-8, (a, b)


@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32])
def test_rk_graph_and_launch_paths_agree_bitwise(prec, rk):
    spec = channel_box(precision=prec, fixed_vcycles=0, mg_rel_tol=1e-8, max_vcycles=40, rk_stages=rk)
    out = []
    for graph in (True, False):
        with binding.Case(spec) as c:
            c.set_graph(graph)
            st = c.step(4)
            out.append((st, c.read(), c.info()["kernel_launches"]))
    (s1, f1, l1), (s2, f2, l2) = out
    assert s1["vcycles_total"] == s2["vcycles_total"] and s1["rel_residual"] == s2["rel_residual"]
    assert l1 == l2
    for f in cases.FIELDS:
        assert np.array_equal(f1[f], f2[f]), f


@pytest.mark.parametrize("prec", [cases.FP32, cases.BF16_MIXED], ids=["fp32", "bf16"])
def test_rk3_reduced_precision_within_1e4_of_fp64_oracle(prec):
    spec = room_small(precision=prec, mg_rel_tol=1e-8, max_vcycles=40, rk_stages=3)
    with binding.Case(spec) as c:
        st = c.step(6)
        got = c.read()
    assert st["rel_residual"] <= 1e-8
    o = OracleCase(spec.replace(precision=cases.FP64)).step(6)
    for f in STATE:
        assert rel_err(got[f], o.fields()[f]) <= 1e-4, f


def test_batch_mixing_schemes_equals_each_alone():
    specs = [channel_box(mg_rel_tol=1e-8, max_vcycles=40, rk_stages=rk) for rk in (1, 2, 3)]
    specs.append(room_small(mg_rel_tol=1e-8, max_vcycles=40, rk_stages=3, krylov=1))
    alone, alone_st = [], []
    for s in specs:
        with binding.Case(s) as c:
            alone_st.append(c.step(3))
            alone.append(c.read())
    cs = [binding.Case(s) for s in specs]
    try:
        with binding.Batch(cs) as b:
            st = b.step(3)
        got = [c.read() for c in cs]
    finally:
        for c in cs:
            c.close()
    for i in range(len(specs)):
        assert st[i]["vcycles_total"] == alone_st[i]["vcycles_total"], i
        for f in cases.FIELDS:
            assert rel_err(got[i][f], alone[i][f]) <= 1e-12, (i, f)
