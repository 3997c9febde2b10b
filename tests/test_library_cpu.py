"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every symbol include/fvm.h declares, its structs match the binding, and
descriptor validation and memory accounting work."""
import os
import re

import pytest

from paper_2603_21869_gb300 import binding, cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_21869_gb300 import build
    build.ensure_built()
    return binding.lib()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "fvm.h")).read()
    declared = set(re.findall(r"\b(fvm_[a-z_0-9]+)\s*\(", hdr))
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTS)


def test_struct_layout_matches_binding(lib):
    import ctypes as ct
    sizes = binding.struct_sizes()
    ours = [ct.sizeof(t) for t in (binding.Patch, binding.Vent, binding.Box, binding.CaseDesc,
                                   binding.StepStats, binding.CaseInfo, binding.KernelStat, binding.BatchInfo,
                                   binding.RequestResult, binding.ServerInfo, binding.Tuning)]
    assert sizes == ours


def test_batch_create_rejects_bad_arguments_without_a_gpu(lib):
    import ctypes as ct
    h = ct.c_void_p()
    assert lib.fvm_batch_create(None, 0, None, ct.byref(h)) == binding.ERR_INVALID
    arr = (ct.c_void_p * 2)(None, None)
    assert lib.fvm_batch_create(arr, 2, None, ct.byref(h)) == binding.ERR_INVALID
    assert "null case" in binding.last_error()
    assert not h.value
    assert lib.fvm_batch_step(None, 1, None) == binding.ERR_INVALID
    assert lib.fvm_batch_launch(None, 1) == binding.ERR_INVALID
    assert lib.fvm_batch_wait(None, None) == binding.ERR_INVALID


def test_lambda2_rejects_bad_arguments_without_a_gpu(lib):
    import ctypes as ct
    buf = (ct.c_double * 4)()
    assert lib.fvm_lambda2(None, buf, 4) == binding.ERR_INVALID
    assert "null case" in binding.last_error()


def test_autotune_rejects_bad_arguments_without_a_gpu(lib):
    import ctypes as ct
    t = binding.Tuning()
    assert lib.fvm_autotune(None, 3, ct.byref(t)) == binding.ERR_INVALID
    d = binding._Desc(cases.heated_channel_3d(32, 16, 16, mg_levels=3))
    assert lib.fvm_autotune(ct.byref(d.desc), 0, ct.byref(t)) == binding.ERR_INVALID
    bad = binding._Desc(cases.heated_channel_3d(30, 16, 16, mg_levels=3))   # 30 does not halve twice
    assert lib.fvm_autotune(ct.byref(bad.desc), 3, ct.byref(t)) == binding.ERR_INVALID


def test_server_rejects_bad_arguments_without_a_gpu(lib):
    import ctypes as ct
    h = ct.c_void_p()
    assert lib.fvm_server_create(0, 0, None, 0, ct.byref(h)) == binding.ERR_INVALID
    assert lib.fvm_server_create(1 << 30, -1, None, 0, ct.byref(h)) == binding.ERR_INVALID
    assert not h.value
    assert lib.fvm_server_poll(None, 1, None, 0, None) == binding.ERR_INVALID
    assert lib.fvm_server_submit(None, None, 1, 0.0, None) == binding.ERR_INVALID


def test_case_bytes_scale_with_precision(lib):
    s64 = cases.heated_channel_3d(64, 16, 16, mg_levels=4)
    s32 = s64.replace(precision=cases.FP32)
    b64, b32 = binding.case_bytes(s64), binding.case_bytes(s32)
    N = 64 * 16 * 16
    assert b64 > 100 * N and b32 < b64
    # full 3D channel workload (1M cells) in FP32 stays well under 200 MB
    assert binding.case_bytes(cases.heated_channel_3d(precision=cases.FP32)) < 200e6
    # flexible CG keeps one more level-0 vector in the inner precision
    assert binding.case_bytes(s32.replace(krylov=1)) >= b32 + 4 * N


@pytest.mark.parametrize("bad", [
    dict(nx=0),
    dict(mg_levels=9),
    dict(mg_levels=1),
    dict(pre_sweeps=0),
    dict(nu=0.0),
    dict(boxes=[cases.Box(0, 100, 0, 4, 0, 4)]),
    dict(vents=[cases.Vent(face=2, a0=0, a1=200, b0=0, b1=2, bc=cases.Patch(cases.OUTLET))]),
    dict(faces=[cases.Patch(cases.INLET, u_normal=1.0, intensity=0.05, length_scale=0.1)] + [cases.Patch()] * 5),
    dict(nz=1),
    dict(krylov=2),
    dict(krylov=1, mg_variant=1),
    dict(mg_variant=2),
    dict(coarse_sweeps=-1),
    dict(coarse_sweeps=1, mg_variant=1),
    dict(rk_stages=-1),
    dict(boxes=[cases.Box(0, 32, 0, 16, 0, 8), cases.Box(0, 32, 0, 16, 8, 16)]),
])
def test_invalid_descriptors_are_rejected_without_a_gpu(lib, bad):
    spec = cases.heated_channel_3d(32, 16, 16, mg_levels=3).replace(**bad)
    assert binding.case_bytes(spec) == 0
    with pytest.raises(binding.FvmError) as ei:
        binding.Case(spec)
    assert ei.value.status == binding.ERR_INVALID
    assert binding.last_error()


def test_rk_stages_validation_and_bytes_without_a_gpu(lib):
    """rk_stages 3 holds one more copy of the six state fields; 4 is refused."""
    spec = cases.heated_channel_3d(32, 16, 16, mg_levels=3, precision=cases.FP32)
    b1 = binding.case_bytes(spec)
    assert binding.case_bytes(spec.replace(rk_stages=2)) == b1
    assert binding.case_bytes(spec.replace(rk_stages=3)) - b1 == 6 * spec.cells * 4
    assert binding.case_bytes(spec.replace(rk_stages=4)) == 0
    assert "rk_stages" in binding.last_error()


def test_projection_vjp_rejects_bad_arguments_without_a_gpu(lib):
    import ctypes as ct
    buf = (ct.c_double * 8)()
    assert lib.fvm_projection_vjp(None, 0.01, buf, buf, 8, 1e-12, 10, None) == binding.ERR_INVALID
    assert "null case" in binding.last_error()


def test_step_adjoints_reject_bad_arguments_without_a_gpu(lib):
    """The new vector-Jacobian products validate their arguments before any device work."""
    import ctypes as ct
    dp = ct.POINTER(ct.c_double)
    for name in ("fvm_destruction_vjp", "fvm_explicit_vjp"):
        st = getattr(lib, name)(None, 0.01, dp(), dp(), 0)
        assert st == binding.ERR_INVALID, name
        assert "null" in binding.last_error()
    st = lib.fvm_step_vjp(None, 0.01, dp(), dp(), 0, 1e-10, 10, None)
    assert st == binding.ERR_INVALID and "null" in binding.last_error()
