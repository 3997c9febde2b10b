"""The allocation-free pressure residual, called through the C-ABI on device
buffers that the caller owns, agrees with the library's own residual (the
relative residual fvm_vcycle reports with zero cycles) on two calls in a row.

It serves callers that cannot allocate device memory themselves (memory
owned by a pooling allocator, loops that must not take an allocation's
latency, plug-ins with a fixed device footprint); its scratch is a static
device array, so this file is collected last and must pass alone too."""
import ctypes as ct

import numpy as np
import pytest

from paper_2603_21869_gb300 import binding, build, cases

pytestmark = pytest.mark.gpu


def _flat(a):
    """(nx, ny, nz) array -> the library's x-fastest float64 buffer."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).transpose(2, 1, 0)).ravel()


def test_static_residual_matches_case_residual_twice():
    torch = pytest.importorskip("torch")
    build.ensure_built()
    L = binding.lib()
    spec = cases.heated_channel_3d(64, 16, 16, mg_levels=4, fixed_vcycles=2)
    nx, ny, nz = spec.nx, spec.ny, spec.nz
    h = (ct.c_double * 3)(spec.Lx / nx, spec.Ly / ny, spec.Lz / nz)
    dirichlet = (ct.c_int32 * 6)(*[1 if f.kind == cases.OUTLET else 0 for f in spec.faces])
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
            st = L.fvm_poisson_residual_static(ct.c_void_p(p.data_ptr()), ct.c_void_p(b.data_ptr()), nx, ny, nz,
                                               h, dirichlet, ct.c_void_p(r.data_ptr()),
                                               ct.c_void_p(norms.data_ptr()), None)
            assert st == binding.OK, binding.last_error()
            torch.cuda.synchronize()
            r2, b2 = norms.cpu().numpy()
            rel_static = float(np.sqrt(r2 / b2))
            assert rel_case > 0.0
            assert rel_static == pytest.approx(rel_case, rel=1e-10), (call, rel_static, rel_case)
            # the residual field itself: its norm is the reported one
            assert float(torch.sum(r * r)) == pytest.approx(r2, rel=1e-12)


def test_static_residual_rejects_grids_above_capacity():
    build.ensure_built()
    L = binding.lib()
    h = (ct.c_double * 3)(1.0, 1.0, 1.0)
    dirichlet = (ct.c_int32 * 6)(0, 1, 0, 0, 0, 0)
    st = L.fvm_poisson_residual_static(ct.c_void_p(16), ct.c_void_p(16), 4096, 4096, 4096, h, dirichlet,
                                       ct.c_void_p(16), ct.c_void_p(16), None)
    assert st == binding.ERR_INVALID
    assert "static scratch" in binding.last_error()
