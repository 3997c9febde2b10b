"""The level-0 residual of the reduced-precision modes on large grids:
r = b - A p with p in FP64, evaluated in float-float arithmetic (no FP64
pipe), against the same residual in FP64 on the host (the oracle's A)."""
import numpy as np
import pytest

from oracle.poisson import apply_A
from oracle.step import OracleCase
from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.ensure_built()
    binding.lib()


@pytest.mark.parametrize("prec,tol", [(cases.FP32, 1e-5), (cases.BF16_MIXED, 2e-2)], ids=["fp32", "bf16"])
def test_float_float_residual_matches_fp64(prec, tol):
    """A smooth p with a large offset and a right-hand side that it nearly
    solves (relative residual about 1e-6): an FP32 stencil would be off by
    orders of magnitude, the float-float one agrees with FP64 to the
    rounding of r to the inner precision.  2^20 cells, a solid box
    (irregular cells)."""
    spec = cases.heated_channel_3d(256, 64, 64, mg_levels=6, precision=prec,
                                   boxes=[cases.Box(60, 80, 10, 30, 0, 20, thermal=cases.HEAT_FLUX, T_value=100.0)])
    lev = OracleCase(spec).mg.levels[0]
    fl = lev.fluid
    nx, ny, nz = lev.shape
    x, y, z = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny, np.arange(nz) / nz, indexing="ij")
    p = np.where(fl, 40.0 + 3.0 * np.sin(2.0 * x + 1.0) * np.cos(3.0 * y) + 0.5 * z * z, 0.0)
    b = apply_A(lev, p)
    b = np.where(fl, b + 1e-6 * np.std(b[fl]) * np.random.default_rng(3).normal(size=b.shape), 0.0)
    with binding.Case(spec) as c:
        c.set_rhs(b)
        c.write({"p": p})
        rel = c.vcycle(0)
        bf = c.read_rhs()
    r = np.where(fl, bf - apply_A(lev, p), 0.0)
    rel_ref = float(np.linalg.norm(r[fl]) / np.linalg.norm(bf[fl]))
    assert 1e-8 < rel_ref < 1e-4
    assert rel == pytest.approx(rel_ref, rel=tol)
