"""The windowed oracle stages (tests/oracle_window.py) against the same stages on
the whole grid: on a room whose windows hold box edges and corners, a ceiling
inlet vent, the floor outlet, domain edges and corners and plain interior, the
exact cells of every window equal the whole-grid result bit for bit, for the
destruction half step, the explicit stage (forward Euler and the three-stage
Runge-Kutta form), the right-hand side, the projection and a whole step given
its pressure.  A margin one cell short of the reach changes a cell of the
three-stage Runge-Kutta stage and of a step's right-hand side and k, so the
check can fail."""
import numpy as np
import pytest

from oracle.destruction import destruction_step
from oracle.poisson import poisson_rhs, project
from oracle.step import OracleCase
from oracle.transport import explicit_stage_rk
from paper_2603_21869_gb300 import cases

import oracle_window as ow


@pytest.fixture(scope="module")
def room():
    spec = cases.room_3d(64, 32, 32, seed=3, mg_levels=3, h=0.08, precision=cases.FP64, fixed_vcycles=4)
    o = OracleCase(spec).step(3)   # a developed state: nonzero velocity, k and omega
    return spec, o


def centers(spec):
    out = [(spec.nx // 2, spec.ny // 2, spec.nz // 2), (0, 0, 0), (spec.nx - 1, spec.ny - 1, spec.nz - 1)]
    for b in spec.boxes:
        out.append((b.i0, b.j0, b.k1))      # a box corner
    for v in spec.vents:
        axis, side = v.face // 2, v.face % 2
        ta, tb = [a for a in range(3) if a != axis]
        c = [0, 0, 0]
        c[axis] = 0 if side == 0 else (spec.nx, spec.ny, spec.nz)[axis] - 1
        c[ta], c[tb] = v.a0, v.b1            # a vent edge
        out.append(tuple(c))
    return out


def test_windows_cover_boxes_and_vents(room):
    spec, _ = room
    assert len(spec.boxes) >= 3 and any(v.bc.kind == cases.OUTLET for v in spec.vents)
    assert any(v.bc.kind == cases.INLET for v in spec.vents)


def test_windowed_stages_equal_whole_grid_stages(room):
    spec, o = room
    state = [x.copy() for x in o.state]
    dt = 0.7 * o.dt
    u, v, w, T_, k, om = state
    kd, omd = destruction_step(o.geo, u, v, w, k, om, 0.5 * dt)
    ex1 = dict(zip(ow.STATE, explicit_stage_rk(o.geo, state, dt, 1)))
    ex3 = dict(zip(ow.STATE, explicit_stage_rk(o.geo, state, dt, 3)))
    b = poisson_rhs(o.geo, u, v, w, dt)
    pu = dict(zip(("u", "v", "w"), project(o.geo, o.mg.levels[0], u, v, w, o.p, dt)))
    for c in centers(spec):
        win = ow.Window(spec, c, (12, 10, 8))
        d = win.destruction_half(state, dt)
        assert np.array_equal(d["k"], kd[win.full]) and np.array_equal(d["omega"], omd[win.full]), c
        e = win.explicit(state, dt)
        e3 = win.explicit(state, dt, 3)
        for f in ow.STATE:
            assert np.array_equal(e[f], ex1[f][win.full]), (c, f)
            assert np.array_equal(e3[f], ex3[f][win.full]), (c, f, "rk3")
        assert np.array_equal(win.rhs(state, dt), b[win.full]), c
        pr = win.project(state, o.p, dt)
        for f in ("u", "v", "w"):
            assert np.array_equal(pr[f], pu[f][win.full]), (c, f)


def test_windowed_step_equals_whole_grid_step(room):
    """A whole oracle step (its dt and pressure taken as given) on the windows."""
    spec, o = room
    state = [x.copy() for x in o.state]
    o2 = OracleCase(spec, state=state, p=o.p).step(1)
    want = o2.fields()
    for c in centers(spec):
        win = ow.Window(spec, c, (12, 10, 8))
        got, b = win.step(state, o2.p, o2.dt)
        assert np.array_equal(b, o2.b[win.full]), c
        for f in ow.STATE:
            assert np.array_equal(got[f], want[f][win.full]), (c, f)


def test_a_margin_short_of_the_reach_is_detected(room, monkeypatch):
    spec, o = room
    state = [x.copy() for x in o.state]
    ex3 = dict(zip(ow.STATE, explicit_stage_rk(o.geo, state, o.dt, 3)))
    o2 = OracleCase(spec, state=state, p=o.p).step(1)
    monkeypatch.setattr(ow, "MARGIN", 2)
    win = ow.Window(spec, (spec.nx // 2, spec.ny // 2, spec.nz // 2), (12, 10, 8))
    e3 = win.explicit(state, o.dt, 3)
    assert any(not np.array_equal(e3[f], ex3[f][win.full]) for f in ow.STATE)
    got, b = win.step(state, o2.p, o2.dt)
    assert not np.array_equal(b, o2.b[win.full])
    assert not np.array_equal(got["k"], o2.fields()["k"][win.full])
