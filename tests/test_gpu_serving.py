"""Serving (fvm_server): requests admitted by device-memory budget while
others run, stepped together, retired.  Each result must be the same alone
and in the mix."""
import numpy as np
import pytest

from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the reduced-precision bound (BF16 corrections, FP32 fields)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def mix():
    """Two small rooms and a channel, mixed precision, different sizes."""
    r1 = cases.room_3d(64, 32, 32, seed=3, mg_levels=4, h=0.08, precision=cases.BF16_MIXED, max_vcycles=40)
    r2 = cases.room_3d(96, 64, 32, seed=5, mg_levels=4, h=0.06, precision=cases.BF16_MIXED, max_vcycles=40)
    ch = cases.heated_channel_3d(64, 32, 32, mg_levels=4, precision=cases.BF16_MIXED, init_perturb=0.02)
    return [(r1, 6), (r2, 5), (ch, 4)]


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = mix()
    alone = []
    for spec, n in reqs:
        with binding.Case(spec) as c:
            c.step(n, allow_not_converged=True)
            alone.append(c.read())
    with binding.Server(budget_bytes=8 << 30, keep_results=True) as srv:   # each round: steps, then admissions
        ids = [srv.submit(reqs[0][0], reqs[0][1])]
        done = srv.poll(chunk=2)            # the first request is admitted
        ids.append(srv.submit(reqs[1][0], reqs[1][1]))
        done += srv.poll(chunk=2)           # it runs alone for two steps while the second is admitted
        ids.append(srv.submit(reqs[2][0], reqs[2][1]))
        for _ in range(20):
            if len(done) == len(reqs):
                break
            done += srv.poll(chunk=2)
        info = srv.info()
        res = {d["id"]: d for d in done}
        got = {i: srv.read(i) for i in ids}
    assert len(done) == len(reqs) and info["done"] == len(reqs) and info["running"] == 0
    assert info["batch_rebuilds"] >= 3          # membership changed with each admission / retirement
    # the later requests were admitted while the first was still running
    assert res[ids[1]]["t_admit"] < res[ids[0]]["t_done"]
    assert res[ids[2]]["t_admit"] < res[ids[0]]["t_done"]
    for i, (spec, n) in zip(ids, reqs):
        assert res[i]["status"] == binding.OK and res[i]["steps"] == n
        assert res[i]["t_arrive"] <= res[i]["t_admit"] <= res[i]["t_done"]
        for f in cases.FIELDS:
            assert rel(got[i][f], alone[ids.index(i)][f]) <= TOL, (i, f)


def test_budget_admission_waits_for_memory():
    reqs = mix()
    sizes = [binding.case_bytes(s) for s, _ in reqs]
    budget = int(max(sizes) * 1.2)               # room for one case at a time
    with binding.Server(budget_bytes=budget) as srv:
        ids = [srv.submit(s, n, t_arrive=0.0) for s, n in reqs]
        done = []
        peak = 0
        for _ in range(40):
            done += srv.poll(chunk=3)
            inf = srv.info()
            peak = max(peak, inf["bytes_in_use"])
            if len(done) == len(reqs):
                break
    assert len(done) == len(reqs) and all(d["status"] == binding.OK for d in done)
    assert peak <= budget
    order = sorted(done, key=lambda d: d["t_admit"])
    for a, b in zip(order, order[1:]):
        assert b["t_admit"] >= a["t_done"]   # one resident case at a time
    assert [d["id"] for d in order] == ids   # first come, first served


def test_request_larger_than_the_budget_is_refused():
    spec, n = mix()[1]
    with binding.Server(budget_bytes=binding.case_bytes(spec) // 2) as srv:
        with pytest.raises(binding.FvmError) as e:
            srv.submit(spec, n)
        assert e.value.status == binding.ERR_BUDGET
