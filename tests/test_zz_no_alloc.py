"""The allocation-free pressure residual (fvm_poisson_residual_static),
called through the C-ABI on device buffers the caller owns.

It serves callers that cannot allocate device memory themselves: memory
owned by a pooling allocator, loops that must not take an allocation's
latency or implicit synchronisation, plug-ins with a fixed device
footprint.  Its scratch is a static device array shared by every call, so
this file is collected last and must pass alone too.  The results are
compared with the library's own residual (two calls in a row) and, element
by element, with the CPU oracle's r = b - A p on boxes with other
zero-value faces, a 2D grid and grids that are not multiples of the block."""
import ctypes as ct

import numpy as np
import pytest

from oracle.geometry import Level
from oracle.poisson import residual
from paper_2603_21869_gb300 import binding, build, cases


def _flat(a):
    """(nx, ny, nz) array -> the library's x-fastest float64 buffer."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).transpose(2, 1, 0)).ravel()


def _unflat(v, shape):
    nx, ny, nz = shape
    return np.asarray(v).reshape(nz, ny, nx).transpose(2, 1, 0)


def _call(L, p, b, shape, h, mask, r, norms):
    nx, ny, nz = shape
    hh = (ct.c_double * 3)(*h)
    dirichlet = (ct.c_int32 * 6)(*mask)
    return L.fvm_poisson_residual_static(ct.c_void_p(p.data_ptr()), ct.c_void_p(b.data_ptr()), nx, ny, nz, hh,
                                         dirichlet, ct.c_void_p(r.data_ptr()), ct.c_void_p(norms.data_ptr()), None)


@pytest.mark.gpu
def test_static_residual_matches_case_residual_twice():
    torch = pytest.importorskip("torch")
    build.ensure_built()
    L = binding.lib()
    spec = cases.heated_channel_3d(64, 16, 16, mg_levels=4, fixed_vcycles=2)
    shape = (spec.nx, spec.ny, spec.nz)
    h = (spec.Lx / spec.nx, spec.Ly / spec.ny, spec.Lz / spec.nz)
    mask = [1 if f.kind == cases.OUTLET else 0 for f in spec.faces]
    dev = torch.device("cuda", 0)
    with binding.Case(spec) as c:
        for call in range(2):
            c.step(1)
            rel_case = c.vcycle(0)          # the library's own residual of the current p, b
            p = torch.from_numpy(_flat(c.read(("p",))["p"])).to(dev)
            b = torch.from_numpy(_flat(c.read_rhs())).to(dev)
            r = torch.empty_like(p)
            norms = torch.zeros(2, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            st = _call(L, p, b, shape, h, mask, r, norms)
            assert st == binding.OK, binding.last_error()
            torch.cuda.synchronize()
            r2, b2 = norms.cpu().numpy()
            rel_static = float(np.sqrt(r2 / b2))
            assert rel_case > 0.0
            assert rel_static == pytest.approx(rel_case, rel=1e-10), (call, rel_static, rel_case)
            # the residual field itself: its norm is the reported one
            assert float(torch.sum(r * r)) == pytest.approx(r2, rel=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("shape,mask", [((64, 16, 16), (0, 1, 0, 0, 0, 0)),
                                        ((33, 7, 3), (1, 0, 1, 0, 0, 1)),
                                        ((37, 5, 1), (1, 0, 1, 0, 0, 0)),
                                        ((35, 9, 5), (0, 0, 0, 1, 1, 0))],
                         ids=["channel", "ragged3d", "ragged2d", "yz_faces"])
def test_static_residual_matches_oracle_elementwise(shape, mask):
    """r and both norms against the oracle's r = b - A p, two calls in a row on the shared scratch."""
    torch = pytest.importorskip("torch")
    build.ensure_built()
    L = binding.lib()
    h = (0.05, 0.07, 0.11)
    rng = np.random.default_rng(sum(shape) + 7 * sum(mask))
    solid = np.zeros(shape, dtype=bool)
    faces = []
    for f in range(6):
        fs = tuple(n for a, n in enumerate(shape) if a != f // 2)
        faces.append(np.full(fs, bool(mask[f])))
    lev = Level(shape, h, solid, faces)
    dev = torch.device("cuda", 0)
    for call in range(2):
        p_h = rng.standard_normal(shape)
        b_h = rng.standard_normal(shape)
        ref = residual(lev, p_h, b_h)
        p = torch.from_numpy(_flat(p_h)).to(dev)
        b = torch.from_numpy(_flat(b_h)).to(dev)
        r = torch.full_like(p, np.nan)
        norms = torch.full((2,), np.nan, dtype=torch.float64, device=dev)
        st = _call(L, p, b, shape, h, mask, r, norms)
        assert st == binding.OK, binding.last_error()
        torch.cuda.synchronize()
        got = _unflat(r.cpu().numpy(), shape)
        scale = float(np.max(np.abs(ref)))
        assert float(np.max(np.abs(got - ref))) <= 1e-12 * scale, call
        r2, b2 = norms.cpu().numpy()
        assert r2 == pytest.approx(float(np.sum(ref * ref)), rel=1e-12)
        assert b2 == pytest.approx(float(np.sum(b_h * b_h)), rel=1e-12)


@pytest.mark.parametrize("dims", [(4096, 4096, 4096), (32, 4, 131072), (32, 262144, 2), (2 ** 31 - 1, 1, 1)],
                         ids=["total", "grid_z", "grid_y", "wide_x"])
def test_static_residual_rejects_grids_above_capacity(dims):
    """Rejected before any device work (no GPU needed): the pointers are never touched."""
    build.ensure_built()
    L = binding.lib()
    h = (ct.c_double * 3)(1.0, 1.0, 1.0)
    dirichlet = (ct.c_int32 * 6)(0, 1, 0, 0, 0, 0)
    st = L.fvm_poisson_residual_static(ct.c_void_p(16), ct.c_void_p(16), *dims, h, dirichlet,
                                       ct.c_void_p(16), ct.c_void_p(16), None)
    assert st == binding.ERR_INVALID
    assert "static scratch" in binding.last_error()
