"""Oracle parity of the reduced-precision path at the sizes that select its
four-cell kernels.

Single-case FP32 / BF16 levels of 2^20 cells or more with nx % 4 == 0 run
the four-cells-per-thread multigrid kernels (the sweep, the residual and
restriction, the prolongation, the flexible-CG passes) and the double-float
level-0 residual and projection; batched launches use them at every size.
Each test here runs one of those configurations through the C-ABI and
compares the fields, element by element, with the FP64 oracle stepped from
the same seeded state: within 1e-4 of each field's largest magnitude on u,
v, w, T, k and omega (the reduced-precision bound), both solves at the same
1e-8 relative residual (Algorithm 1's solve wrapped in FP64 defect
correction; Eq. jacobi_pc for the smoother)."""
import numpy as np
import pytest

from oracle.step import OracleCase
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

TOL = 1e-4
STATE = ("u", "v", "w", "T", "k", "omega")
FOUR_CELL_MIN = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def rel_err(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / scale if scale > 0.0 else float(np.max(np.abs(a)))


def check(got, ref, label, tol=TOL):
    errs = {f: rel_err(got[f], ref[f]) for f in STATE}
    bad = {f: e for f, e in errs.items() if not e <= tol}
    assert not bad, f"{label}: relative errors above {tol}: {bad} (all: {errs})"
    return errs


def oracle_fields(spec, steps):
    o = OracleCase(spec.replace(precision=cases.FP64)).step(steps)
    assert o.last_rel <= spec.mg_rel_tol
    return o.fields()


def test_channel_256x64x64_fp32_matches_oracle():
    """The 1 M-cell heated channel, FP32 fields and corrections, V(3,3), three steps."""
    spec = cases.heated_channel_3d(256, 64, 64, mg_levels=6, precision=cases.FP32, mg_rel_tol=1e-8,
                                   max_vcycles=60)
    assert spec.cells >= FOUR_CELL_MIN and spec.nx % 4 == 0
    with binding.Case(spec) as c:
        st = c.step(3)
        got = c.read()
    assert st["rel_residual"] <= 1e-8
    check(got, oracle_fields(spec, 3), "channel fp32")


def test_room_256x128x32_bf16_krylov_matches_oracle():
    """A 1 M-cell room (vents, outlet, heated boxes, buoyancy), FP32 fields with BF16
    corrections, the flexible-CG acceleration, V(2,2), two cycles per outer residual."""
    spec = cases.room_3d(256, 128, 32, seed=0, mg_levels=5, precision=cases.BF16_MIXED, mg_rel_tol=1e-8,
                         max_vcycles=80, krylov=1, pre_sweeps=2, post_sweeps=2, inner_cycles=2)
    assert spec.cells >= FOUR_CELL_MIN and spec.nx % 4 == 0
    with binding.Case(spec) as c:
        st = c.step(3)
        got = c.read()
    assert st["rel_residual"] <= 1e-8
    check(got, oracle_fields(spec, 3), "room bf16 krylov")


def test_batched_cases_match_oracle():
    """Uneven channels stepped as one batch (four-cell kernels at every size), each case
    against its own oracle run."""
    specs = []
    for n, (nx, nyz, U) in enumerate([(64, 32, 1.2), (96, 32, 2.5), (128, 64, 0.7)]):
        s = cases.heated_channel_3d(nx, nyz, nyz, mg_levels=4, precision=cases.FP32, seed=40 + n,
                                    init_perturb=0.02, mg_rel_tol=1e-8, max_vcycles=60)
        faces = list(s.faces)
        faces[0] = cases.Patch(cases.INLET, u_normal=U, intensity=0.05, length_scale=0.07 * s.Lz,
                               T_in=s.faces[0].T_in)
        specs.append(s.replace(faces=faces, init_vel=(U, 0.0, 0.0)))
    cs = [binding.Case(s) for s in specs]
    try:
        with binding.Batch(cs) as b:
            st = b.step(3)
        got = [c.read() for c in cs]
    finally:
        for c in cs:
            c.close()
    for s, g, x in zip(specs, got, st):
        assert x["rel_residual"] <= 1e-8
        check(g, oracle_fields(s, 3), f"batched {s.nx}x{s.ny}x{s.nz}")


def test_served_request_matches_oracle():
    """One room request served next to another (continuous batching), against the oracle."""
    r1 = cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=cases.BF16_MIXED, max_vcycles=60)
    r2 = cases.room_3d(96, 64, 32, seed=5, mg_levels=4, h=0.06, precision=cases.BF16_MIXED, max_vcycles=60)
    with binding.Server(budget_bytes=8 << 30, keep_results=True) as srv:
        ids = [srv.submit(r1, 4), srv.submit(r2, 3)]
        done = []
        for _ in range(20):
            if len(done) == 2:
                break
            done += srv.poll(chunk=2)
        got = {i: srv.read(i) for i in ids}
    assert len(done) == 2 and all(d["status"] == binding.OK for d in done)
    check(got[ids[0]], oracle_fields(r1, 4), "served room 64x32x32")
    check(got[ids[1]], oracle_fields(r2, 3), "served room 96x64x32")
