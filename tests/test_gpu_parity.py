"""GPU-vs-oracle parity through the C-ABI (FP64 path: 1e-10 relative to each
field's largest magnitude; FP32 path: 1e-4), stage by stage, over full
steps, for the V-cycle alone, at edge cases and at full workload size."""
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
    scale = np.max(np.abs(b))
    if scale == 0.0:
        return float(np.max(np.abs(a)))
    return float(np.max(np.abs(a - b)) / scale)


def assert_fields(got, ref, tol, fields, label=""):
    errs = {f: rel_err(got[f], ref[f]) for f in fields}
    bad = {f: e for f, e in errs.items() if not e <= tol}
    assert not bad, f"{label}: relative errors above {tol}: {bad} (all: {errs})"
    return errs


def room_small(precision=cases.FP64, seed=3, **kw):
    return cases.room_3d(64, 32, 32, seed=seed, mg_levels=4, h=0.08, precision=precision, **kw)


def channel_box(precision=cases.FP64, **kw):
    spec = cases.heated_channel_3d(48, 16, 16, mg_levels=3, precision=precision, init_perturb=0.02,
                                   boxes=[cases.Box(10, 16, 4, 10, 0, 7, thermal=cases.HEAT_FLUX, T_value=150.0),
                                          cases.Box(30, 34, 8, 16, 6, 12, thermal=cases.FIXED_T, T_value=40.0)],
                                   vents=[cases.Vent(face=5, a0=20, a1=28, b0=4, b1=12,
                                                     bc=cases.Patch(cases.INLET, u_normal=0.8, intensity=0.1,
                                                                    length_scale=0.02, T_in=15.0))])
    return spec.replace(**kw)


SPECS = {
    "channel2d_full": lambda: cases.channel_2d(fixed_vcycles=4),
    "channel2d_ragged": lambda: cases.channel_2d(48, 20, 3, fixed_vcycles=3, init_perturb=0.05),
    "channel3d_box_vent": lambda: channel_box(fixed_vcycles=3),
    "room_buoyant": lambda: room_small(fixed_vcycles=3),
    "tiny_3d": lambda: cases.heated_channel_3d(8, 4, 4, mg_levels=2, fixed_vcycles=2, init_perturb=0.1),
}


@pytest.mark.parametrize("name", list(SPECS))
def test_initial_state_matches(name):
    spec = SPECS[name]()
    with binding.Case(spec) as c:
        got = c.read()
    ref = OracleCase(spec).fields()
    assert_fields(got, ref, 1e-15, cases.FIELDS, name)


@pytest.mark.parametrize("name", ["channel3d_box_vent", "room_buoyant", "channel2d_ragged"])
def test_each_stage_matches_oracle(name):
    spec = SPECS[name]()
    o = OracleCase(spec)
    with binding.Case(spec) as c:
        for s in range(2):
            c.run_stage(binding.STAGE_DT)
            o.update_dt()
            assert c.info()["dt"] == pytest.approx(o.dt, rel=1e-13)
            c.run_stage(binding.STAGE_DESTRUCTION)
            o.destruction_half()
            assert_fields(c.read(STATE), o.fields(), TOL64, ("k", "omega"), f"{name} step {s} destruction 1")
            c.run_stage(binding.STAGE_EXPLICIT)
            o.explicit()
            assert_fields(c.read(STATE), o.fields(), TOL64, STATE, f"{name} step {s} explicit")
            c.run_stage(binding.STAGE_DESTRUCTION)
            o.destruction_half()
            assert_fields(c.read(STATE), o.fields(), TOL64, ("k", "omega"), f"{name} step {s} destruction 2")
            c.run_stage(binding.STAGE_RHS)
            o.rhs()
            assert rel_err(c.read_rhs(), o.b) <= TOL64, f"{name} rhs"
            c.run_stage(binding.STAGE_SOLVE)
            o.solve()
            assert_fields(c.read(("p",)), o.fields(), TOL64, ("p",), f"{name} step {s} solve")
            c.run_stage(binding.STAGE_PROJECT)
            o.project()
            assert_fields(c.read(), o.fields(), TOL64, cases.FIELDS, f"{name} step {s} project")


@pytest.mark.parametrize("name", list(SPECS))
def test_steps_match_oracle(name):
    spec = SPECS[name]()
    nsteps = 3
    with binding.Case(spec) as c:
        st = c.step(nsteps)
        got = c.read()
    o = OracleCase(spec).step(nsteps)
    assert st["vcycles_total"] == nsteps * spec.fixed_vcycles
    assert st["dt_last"] == pytest.approx(o.dt, rel=1e-12)
    assert st["rel_residual"] == pytest.approx(o.last_rel, rel=1e-6)
    assert_fields(got, o.fields(), TOL64, cases.FIELDS, name)


def test_vcycle_alone_matches_oracle_and_reaches_dense_solution():
    spec = channel_box(fixed_vcycles=1)
    o = OracleCase(spec)
    lev = o.mg.levels[0]
    rng = np.random.default_rng(11)
    b = rng.normal(size=lev.shape)
    b[lev.solid] = 0.0
    p = np.zeros(lev.shape)
    with binding.Case(spec) as c:
        c.set_rhs(b)
        c.write({"p": p})
        for n in (1, 2, 5):
            rel = c.vcycle(n)
            for _ in range(n):
                p = o.mg.vcycle(p, b)
            got = c.read(("p",))["p"]
            assert rel_err(got, p) <= TOL64
            assert rel == pytest.approx(o.mg.rel_residual(p, b), rel=1e-6)
        c.vcycle(40)
        got = c.read(("p",))["p"]
    pd = direct_solve(lev, b)
    assert rel_err(got, pd) <= 1e-9


def test_adaptive_solve_tracks_oracle():
    spec = cases.heated_channel_3d(64, 16, 16, mg_levels=4, mg_rel_tol=1e-8, max_vcycles=40)
    with binding.Case(spec) as c:
        cyc = []
        for _ in range(4):
            cyc.append(c.step(1)["vcycles_last"])
        got = c.read()
    o = OracleCase(spec)
    ocyc = []
    for _ in range(4):
        o.step()
        ocyc.append(o.last_vcycles)
    assert all(abs(a - b) <= 1 for a, b in zip(cyc, ocyc)), (cyc, ocyc)
    assert o.last_rel <= 1e-8
    assert_fields(got, o.fields(), 1e-7, cases.FIELDS, "adaptive")


@pytest.mark.parametrize("prec", [cases.FP32, cases.BF16_MIXED], ids=["fp32", "bf16"])
@pytest.mark.parametrize("make", [lambda p: channel_box(precision=p, fixed_vcycles=0, mg_rel_tol=1e-8, max_vcycles=40),
                                  lambda p: room_small(precision=p, mg_rel_tol=1e-8, max_vcycles=40)],
                         ids=["channel_box", "room"])
def test_reduced_precision_within_1e4_of_fp64_oracle(make, prec):
    """FP32 field storage; FP32 or BF16 (FP32 accumulation) multigrid
    corrections inside the FP64 defect-correction solve: u, v, w, T, k, omega
    within 1e-4 (relative to each field's magnitude)."""
    spec = make(prec)
    nsteps = 10
    with binding.Case(spec) as c:
        st = c.step(nsteps)
        got = c.read()
    assert st["rel_residual"] <= 1e-8
    o = OracleCase(spec.replace(precision=cases.FP64)).step(nsteps)
    assert_fields(got, o.fields(), 1e-4, STATE, f"precision {prec}")


def test_checkpoint_resume_is_exact():
    spec = channel_box(fixed_vcycles=2)
    with binding.Case(spec) as a:
        a.step(2)
        snap = a.read()
        a.step(2)
        ref = a.read()
    with binding.Case(spec) as b:
        b.write(snap)
        b.step(2)
        got = b.read()
    # dt depends on the state only, so resuming reproduces the run bit for bit
    for f in cases.FIELDS:
        assert np.array_equal(got[f], ref[f]), f


@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32])
def test_flat_buffers_match_the_field_dict(prec):
    """read_flat / write_flat move the same values as read / write, in the
    library's layout (field after field, x fastest), with no reshaping."""
    spec = channel_box(precision=prec, fixed_vcycles=2)
    with binding.Case(spec) as c:
        c.step(1)
        ref = c.read()
        flat = np.empty(7 * c.N)
        c.read_flat(flat)
        for i, f in enumerate(cases.FIELDS):
            assert np.array_equal(flat[i * c.N:(i + 1) * c.N], ref[f].transpose(2, 1, 0).ravel()), f
        flat2 = flat.copy()
        flat2[3 * c.N:4 * c.N] *= 2.0   # p
        c.write_flat(flat2)
        got = c.read()
    assert np.array_equal(got["p"], 2.0 * ref["p"])
    for f in ("u", "v", "w", "T", "k", "omega"):
        assert np.array_equal(got[f], ref[f]), f


@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32, cases.BF16_MIXED], ids=["fp64", "fp32", "bf16"])
def test_flat_float32_buffers(prec):
    """read_flat / write_flat with float32 buffers (fvm_read_fields_f32 / fvm_write_fields_f32):
    every field reads as its FP64 read rounded to FP32 (for an FP32-field case the state is
    the stored value itself, p the double-float pair rounded once); written FP32 values read
    back exactly, p included, in either storage."""
    spec = channel_box(precision=prec, fixed_vcycles=2)
    with binding.Case(spec) as c:
        c.step(1)
        ref = c.read()
        flat = np.empty(7 * c.N, dtype=np.float32)
        c.read_flat(flat)
        for i, f in enumerate(cases.FIELDS):
            want = ref[f].transpose(2, 1, 0).ravel().astype(np.float32)
            assert np.array_equal(flat[i * c.N:(i + 1) * c.N], want), f
        rng = np.random.default_rng(3)
        new = (flat * (1.0 + 0.01 * rng.standard_normal(flat.size))).astype(np.float32)
        c.write_flat(new)
        got = c.read()
        back = np.empty_like(new)
        c.read_flat(back)
        # a subset of fields: the others stay
        c.write_flat(np.zeros(c.N, dtype=np.float32), fields=("T",))
        after = c.read()
    for i, f in enumerate(cases.FIELDS):
        assert np.array_equal(got[f].transpose(2, 1, 0).ravel(), new[i * c.N:(i + 1) * c.N].astype(np.float64)), f
    assert np.array_equal(back, new)
    assert not after["T"].any()
    for f in ("u", "v", "w", "p", "k", "omega"):
        assert np.array_equal(after[f], got[f]), f
    with binding.Case(spec) as c:
        with pytest.raises(binding.FvmError):
            c.read_flat(np.empty(7 * c.N - 1, dtype=np.float32))


def test_zero_rhs_needs_no_cycles():
    """Uniform through-flow is discretely divergence free: b = 0, no V-cycle runs."""
    spec = cases.heated_channel_3d(32, 8, 8, mg_levels=3, init_perturb=0.0)
    faces = list(spec.faces)
    faces[2:] = [cases.Patch(cases.OUTLET)] * 4
    spec = spec.replace(faces=faces)
    with binding.Case(spec) as c:
        c.run_stage(binding.STAGE_DT)
        c.run_stage(binding.STAGE_RHS)
        assert np.max(np.abs(c.read_rhs())) == 0.0


def test_not_converged_status_is_reported():
    spec = cases.heated_channel_3d(32, 8, 8, mg_levels=3, mg_rel_tol=1e-15, max_vcycles=1)
    with binding.Case(spec) as c:
        st = c.step(1, allow_not_converged=True)
        assert st["status"] == binding.ERR_NOT_CONVERGED
        f = c.read()
    assert all(np.all(np.isfinite(v)) for v in f.values())


def test_nan_injection_reports_diverged():
    """Host-side fault injection: a NaN written into u is reported as
    FVM_ERR_DIVERGED by the next step; the device stays usable."""
    spec = cases.heated_channel_3d(32, 8, 8, mg_levels=3)
    with binding.Case(spec) as c:
        u = c.read(("u",))["u"].copy()
        u[5, 3, 3] = np.nan
        c.write({"u": u})
        with pytest.raises(binding.FvmError) as ei:
            c.step(1)
        assert ei.value.status == binding.ERR_DIVERGED
    with binding.Case(spec) as c2:
        c2.step(1)


@pytest.mark.parametrize("prec", [cases.FP64, cases.FP32])
def test_graph_and_launch_paths_agree_bitwise(prec):
    """The CUDA-graph step (device-side V-cycle loop) and the launch-by-launch
    step run the same kernels in the same order: identical fields and counts."""
    spec = channel_box(precision=prec, fixed_vcycles=0, mg_rel_tol=1e-8, max_vcycles=40)
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


@pytest.mark.parametrize("name", ["channel3d_box_vent", "room_buoyant", "channel2d_ragged"])
def test_paper_multigrid_scheme_matches_oracle(name):
    """mg_variant 1 (Algorithm 1: straight restriction, one unweighted Jacobi
    per coarse level, nearest upsampling, a final Jacobi on p), a fixed
    number of iterations per step: FP64 fields within 1e-10 of the oracle."""
    spec = SPECS[name]().replace(mg_variant=1, fixed_vcycles=5)
    with binding.Case(spec) as c:
        c.step(2)
        got = c.read()
    o = OracleCase(spec).step(2)
    assert_fields(got, o.fields(), TOL64, cases.FIELDS, f"{name}, Algorithm 1")


@pytest.mark.parametrize("name", ["channel3d_box_vent", "room_buoyant", "channel2d_ragged"])
def test_coarse_level_sweep_counts_match_oracle(name):
    """One sweep on each side of every level below the finest (coarse_sweeps = 1),
    the finest level keeping its own: FP64 fields within 1e-10 of the oracle."""
    spec = SPECS[name]().replace(coarse_sweeps=1)
    with binding.Case(spec) as c:
        c.step(2)
        got = c.read()
    o = OracleCase(spec).step(2)
    assert_fields(got, o.fields(), TOL64, cases.FIELDS, f"{name}, coarse_sweeps 1")


def test_paper_scheme_iterations_track_the_oracle_and_converge_slower():
    spec = cases.heated_channel_3d(32, 16, 16, mg_levels=3, fixed_vcycles=1)
    o = OracleCase(spec)
    lev = o.mg.levels[0]
    b = np.where(lev.fluid, np.random.default_rng(7).normal(size=lev.shape), 0.0)
    res = {}
    for variant in (0, 1):
        s = spec.replace(mg_variant=variant)
        mg = OracleCase(s).mg
        p = np.zeros(lev.shape)
        with binding.Case(s) as c:
            c.set_rhs(b)
            c.write({"p": p})
            rels = []
            for _ in range(6):
                rels.append(c.vcycle(1))
                p = mg.cycle(p, b)
            assert rel_err(c.read(("p",))["p"], p) <= 1e-10
        res[variant] = rels
    assert res[1][-1] > res[0][-1]   # the paper's scheme converges more slowly per iteration


@pytest.mark.slow
def test_full_size_heated_channel_one_step():
    """The 256 x 64 x 64 channel (the benchmark workload) in FP64, one step
    with a fixed cycle count, against the oracle everywhere."""
    spec = cases.heated_channel_3d(fixed_vcycles=2)
    with binding.Case(spec) as c:
        c.step(1)
        got = c.read()
    o = OracleCase(spec).step(1)
    assert_fields(got, o.fields(), TOL64, cases.FIELDS, "full size")
