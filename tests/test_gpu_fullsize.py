"""The timed workloads at full size against the oracle on sampled outputs: the
512 x 256 x 128 room (16.8 M cells: vents, outlet, heated boxes, buoyancy)
with the multigrid parameters the autotuner picks for it (V(2,2), one V-cycle
per outer residual, the flexible-CG step, Chebyshev sweep weights), BF16 and
FP32 corrections; the 64 uneven channels (57.5 M cells) stepped as one
batch with theirs (V(3,3), two V-cycles per outer residual, the flexible-CG
step, Chebyshev weights), FP32; and the served stream's largest room
(256 x 128 x 128) served in a mix, BF16 corrections.

The oracle cannot step these grids in a test's time, so the local part of the
path is checked on windows of the GPU's own state (tests/oracle_window.py: the
exact oracle result at every cell of a window, at box corners, vent, inlet and
outlet edges, face centres, domain corners, the centre and seeded positions):
each stage alone to 1e-5 of each field's largest magnitude (the velocity
components' of the largest component), the bound of an FP32 stage against FP64
on the same input, and whole graph-mode steps, as timed, given the pressure
they solved for, to 1e-4 (the reduced-precision bound).  The pressure solve,
which is global, is checked by the oracle's FP64 residual of the GPU's pressure
against the GPU's right-hand side: at most the 1e-8 tolerance, and equal to the
residual the GPU reports for the step."""
import numpy as np
import pytest

from oracle.geometry import Geometry
from oracle.poisson import residual
from oracle.step import stable_dt, time_step
from paper_2603_21869_gb300 import binding, build, cases

import oracle_window as ow

pytestmark = pytest.mark.gpu

TOL = 1e-5        # one stage, FP32 against FP64 on the same input
TOL_STEP = 1e-4   # a whole step
STATE = ow.STATE
WIN = (16, 16, 16)
BATCH_CELLS = 57_000_000   # the 64 channels hold 57.5 M cells
SERVED_BIG = (256, 128, 128)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def room(precision):
    return cases.room_3d(512, 256, 128, seed=0, mg_levels=7, precision=precision, mg_rel_tol=1e-8,
                         max_vcycles=60, pre_sweeps=2, post_sweeps=2, inner_cycles=1, krylov=1, smoother=1)


def centers(spec, seed=7):
    n = (spec.nx, spec.ny, spec.nz)
    out = [tuple(x // 2 for x in n), (0, 0, 0), tuple(x - 1 for x in n), (n[0] - 1, 0, n[2] - 1)]
    for face in range(6):   # each face's centre
        c = [x // 2 for x in n]
        c[face // 2] = 0 if face % 2 == 0 else n[face // 2] - 1
        out.append(tuple(c))
    for b in spec.boxes:
        out += [(b.i0, b.j0, b.k1), (b.i1, b.j1, b.k0)]
    for v in spec.vents:
        axis, side = v.face // 2, v.face % 2
        ta, tb = [a for a in range(3) if a != axis]
        c = [0, 0, 0]
        c[axis] = 0 if side == 0 else n[axis] - 1
        c[ta], c[tb] = v.a0, v.b1
        out.append(tuple(c))
    rng = np.random.default_rng(seed)
    out += [tuple(int(rng.integers(0, x)) for x in n) for _ in range(4)]
    return out


def rel_residual(lev0, p, b):
    """||b - A p|| / ||b|| over the fluid cells, in FP64."""
    return float(np.linalg.norm(residual(lev0, p, b)[lev0.fluid]) / np.linalg.norm(b[lev0.fluid]))


def fields(c, names=STATE):
    f = c.read(names)
    return [f[n] for n in names]


def scales(arrays, names):
    """Largest magnitude per field; the velocity components share the largest one."""
    s = {n: float(np.max(np.abs(a))) for n, a in zip(names, arrays)}
    vs = max(s.get(n, 0.0) for n in ("u", "v", "w"))
    return {n: (vs if n in ("u", "v", "w") else s[n]) for n in names}


def check(wins, want_of, got, names, label, tol=TOL):
    sc = scales([got[n] for n in names], names)
    worst = {n: 0.0 for n in names}
    for win in wins:
        want = want_of(win)
        for n in names:
            e = float(np.max(np.abs(got[n][win.full] - want[n]))) / sc[n]
            worst[n] = max(worst[n], e)
    bad = {n: e for n, e in worst.items() if not e <= tol}
    assert not bad, f"{label}: {bad} (all {worst})"
    print(f"{label}: largest error over {len(wins)} windows", {n: f"{e:.2e}" for n, e in worst.items()})
    return worst


@pytest.mark.parametrize("precision", [cases.BF16_MIXED, cases.FP32], ids=["bf16", "fp32"])
def test_room_full_size_stages_on_sampled_windows(precision):
    spec = room(precision)
    wins = [ow.Window(spec, c, WIN) for c in centers(spec)]
    lev0 = Geometry(spec).level0
    with binding.Case(spec) as c:
        st = c.step(2)   # graph mode, as timed
        b = c.read_rhs()
        p = c.read(("p",))["p"]
        rel = rel_residual(lev0, p, b)
        assert st["rel_residual"] <= 1e-8 and rel <= 1.001e-8
        assert rel == pytest.approx(st["rel_residual"], rel=1e-4)

        c.run_stage(binding.STAGE_DT)
        dt = c.info()["dt"]
        x = fields(c)
        c.run_stage(binding.STAGE_DESTRUCTION)
        y = dict(zip(STATE, fields(c)))
        for n in ("u", "v", "w", "T"):
            assert np.array_equal(y[n], x[STATE.index(n)]), n
        check(wins, lambda w: w.destruction_half(x, dt), y, ("k", "omega"), "destruction")

        x = [y[n] for n in STATE]
        c.run_stage(binding.STAGE_EXPLICIT)
        y = dict(zip(STATE, fields(c)))
        check(wins, lambda w: w.explicit(x, dt), y, STATE, "explicit")

        x = [y[n] for n in STATE]
        c.run_stage(binding.STAGE_DESTRUCTION)
        c.run_stage(binding.STAGE_RHS)
        y = dict(zip(STATE, fields(c)))
        check(wins, lambda w: w.destruction_half(x, dt), y, ("k", "omega"), "destruction 2")
        x = [y[n] for n in STATE]
        b = c.read_rhs()
        check(wins, lambda w: {"b": w.rhs(x, dt)}, {"b": b}, ("b",), "rhs")

        c.run_stage(binding.STAGE_SOLVE)
        p = c.read(("p",))["p"]
        rel = rel_residual(lev0, p, b)
        assert rel <= 1.001e-8, rel
        print(f"solve: FP64 relative residual {rel:.3e}")

        c.run_stage(binding.STAGE_PROJECT)
        y = dict(zip(("u", "v", "w"), fields(c, ("u", "v", "w"))))
        check(wins, lambda w: w.project(x, p, dt), y, ("u", "v", "w"), "project")


def check_step(spec, wins, lev0, x0, x1, p, b, st, label):
    """A whole step from x0 to x1 (given its pressure p and right-hand side b) on the windows,
    and its solve by the FP64 residual."""
    rel = rel_residual(lev0, p, b)
    assert st["rel_residual"] <= spec.mg_rel_tol and rel <= 1.001 * spec.mg_rel_tol, (label, rel, st)
    assert rel == pytest.approx(st["rel_residual"], rel=1e-4), label
    dt = st["dt_last"]
    want = {id(w): w.step(x0, p, dt) for w in wins}
    check(wins, lambda w: want[id(w)][0], x1, STATE, f"{label} step", TOL_STEP)
    check(wins, lambda w: {"b": want[id(w)][1]}, {"b": b}, ("b",), f"{label} step rhs", TOL_STEP)
    print(f"{label}: FP64 relative residual {rel:.3e} (reported {st['rel_residual']:.3e})")


@pytest.mark.parametrize("precision", [cases.BF16_MIXED, cases.FP32], ids=["bf16", "fp32"])
def test_room_full_size_graph_step_on_sampled_windows(precision):
    spec = room(precision)
    wins = [ow.Window(spec, c, WIN) for c in centers(spec, seed=11)]
    lev0 = Geometry(spec).level0
    with binding.Case(spec) as c:
        c.step(2)
        x0 = fields(c)
        st = c.step(1)   # graph mode, as timed: the second half step fused with the right-hand side
        x1 = dict(zip(STATE, fields(c)))
        p = c.read(("p",))["p"]
        b = c.read_rhs()
    check_step(spec, wins, lev0, x0, x1, p, b, st, "room")


def test_batched_channels_full_size_graph_step_on_sampled_windows():
    specs = [sp.replace(pre_sweeps=3, post_sweeps=3, inner_cycles=2, krylov=1, smoother=1)
             for sp in cases.batched_channels(64, seed=0, precision=cases.FP32, mg_levels=5)]
    assert sum(sp.cells for sp in specs) >= BATCH_CELLS
    rng = np.random.default_rng(5)
    sizes = [sp.cells for sp in specs]
    picked = sorted({int(np.argmax(sizes)), int(np.argmin(sizes))} | {int(i) for i in rng.choice(64, 4, replace=False)})
    cs = [binding.Case(sp) for sp in specs]
    try:
        with binding.Batch(cs) as batch:
            batch.step(2)
            x0 = {i: fields(cs[i]) for i in picked}
            st = batch.step(1)
            for i in picked:
                spec = specs[i]
                c = cs[i]
                x1 = dict(zip(STATE, fields(c)))
                p = c.read(("p",))["p"]
                b = c.read_rhs()
                wins = [ow.Window(spec, ctr, WIN) for ctr in centers(spec, seed=i)]
                check_step(spec, wins, Geometry(spec).level0, x0[i], x1, p, b, st[i],
                           f"case {i} ({spec.nx}x{spec.ny}x{spec.nz})")
    finally:
        for c in cs:
            c.close()


def test_served_largest_room_alone_in_the_mix_and_on_oracle_windows():
    """The served stream's largest room (256 x 128 x 128) admitted with a mid-size room, a
    channel and a second copy of itself stepped one step less: every result equal alone and in
    the mix (the reduced-precision bound), and the room's last step, from the copy's state and
    given the pressure it solved for, against the oracle on windows."""
    _, specs = cases.served_rooms(400, seed=0)
    rooms = [sp for sp in specs if sp.buoyancy]
    big = max(rooms, key=lambda sp: sp.cells)
    mid = next(sp for sp in rooms if sp.nx == 160)
    chan = next(sp for sp in specs if not sp.buoyancy)
    assert (big.nx, big.ny, big.nz) == SERVED_BIG
    reqs = [(big, 3), (mid, 3), (big, 2), (chan, 2)]
    alone = []
    for spec, n in reqs:
        with binding.Case(spec) as c:
            c.step(n)
            alone.append(c.read())
    with binding.Server(budget_bytes=40 << 30, keep_results=True) as srv:
        ids = [srv.submit(*reqs[0])]
        done = srv.poll(chunk=1)
        for spec, n in reqs[1:]:   # admitted while the first runs
            ids.append(srv.submit(spec, n))
            done += srv.poll(chunk=1)
        for _ in range(20):
            if len(done) == len(reqs):
                break
            done += srv.poll(chunk=1)
        got = {i: srv.read(i) for i in ids}
    res = {d["id"]: d for d in done}
    assert len(done) == len(reqs)
    for i, (spec, n), a in zip(ids, reqs, alone):
        assert res[i]["status"] == binding.OK and res[i]["steps"] == n
        for f in cases.FIELDS:
            e = float(np.max(np.abs(got[i][f] - a[f]))) / max(float(np.max(np.abs(a[f]))), 1e-300)
            assert e <= TOL_STEP, (i, f, e)
    x0 = [got[ids[2]][f] for f in STATE]
    x1 = {f: got[ids[0]][f] for f in STATE}
    dt = stable_dt(Geometry(big), x0, time_step(big)) if big.dt_adapt else time_step(big)
    wins = [ow.Window(big, c, WIN) for c in centers(big, seed=3)]
    want = {id(w): w.step(x0, got[ids[0]]["p"], dt) for w in wins}
    check(wins, lambda w: want[id(w)][0], x1, STATE, "served room step", TOL_STEP)
