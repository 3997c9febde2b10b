"""Pins of the oracle's time step plumbing: the random draw, the time-step
rule, the initial state and a short run of the 2D channel workload."""
import os

import numpy as np
import pytest

from oracle import model
from oracle.step import OracleCase, splitmix64, time_step, uniform_pm1
from paper_2603_21869_gb300 import cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_vector():
    exp = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
           if l.strip() and not l.startswith("#")]
    got = [int(x) for x in splitmix64(1234567, np.arange(5, dtype=np.uint64))]
    assert got == exp


def test_uniform_draw_range_and_moments():
    xi = uniform_pm1(0, 4, (64, 32, 16))
    assert xi.min() >= -1.0 and xi.max() < 1.0
    assert abs(xi.mean()) < 0.01 and abs(xi.var() - 1 / 3) < 0.01
    assert not np.array_equal(xi, uniform_pm1(0, 5, (64, 32, 16)))


def test_cfl_time_step():
    # 2D channel: h = 4/128 = 1/32, u_in = 1, CFL 0.5 -> dt0 = 1/64
    assert time_step(cases.channel_2d()) == 0.015625
    # 3D channel at 1 cm, u_in = 2: dt0 = 0.5 * 0.01 / 2
    assert time_step(cases.heated_channel_3d()) == pytest.approx(0.0025, rel=1e-15)


def test_initial_state_from_inlet():
    spec = cases.channel_2d(32, 16, 3)
    c = OracleCase(spec)
    k0, om0 = model.inlet_turbulence(1.0, 0.05, 0.07)
    assert np.all(c.state[4] == k0) and np.all(c.state[5] == om0)
    assert om0 == pytest.approx(9.72, rel=1e-3)
    spec = cases.heated_channel_3d(32, 8, 8, mg_levels=3)
    c = OracleCase(spec)
    u = c.state[0]
    assert np.all(np.abs(u / 2.0 - 1.0) <= 0.01) and u.std() > 0.001


def test_channel_2d_short_run_is_finite_and_positive():
    c = OracleCase(cases.channel_2d()).step(10)
    for f in c.state:
        assert np.all(np.isfinite(f))
    assert np.all(c.state[4] > 0) and np.all(c.state[5] > 0)
    assert c.last_rel <= 1e-8
    assert c.dt <= c.dt0
