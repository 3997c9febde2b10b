"""ctypes binding of libfvm.so (the C-ABI declared in include/fvm.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  The library must have been built (``build.build()``); if it
is missing this module raises instead of falling back to anything else.

Field arrays cross the boundary as float64 host buffers in the library's
layout (x fastest); this module returns and accepts numpy arrays shaped
(nx, ny, nz), the transposed view of that buffer.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import cases

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfvm.so")

OK, ERR_INVALID, ERR_OOM, ERR_BUDGET, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_CUDA = 0, -1, -2, -3, -4, -5, -6
STAGE_DT, STAGE_DESTRUCTION, STAGE_EXPLICIT, STAGE_RHS, STAGE_SOLVE, STAGE_PROJECT = range(6)
OPT_GRAPH = 1


class FvmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fvm status {status}: {msg}")
        self.status = status


class Patch(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("thermal", ct.c_int32), ("T_value", ct.c_double),
                ("u_normal", ct.c_double), ("intensity", ct.c_double), ("length_scale", ct.c_double),
                ("T_in", ct.c_double), ("k_value", ct.c_double), ("omega_value", ct.c_double)]


class Vent(ct.Structure):
    _fields_ = [("face", ct.c_int32), ("a0", ct.c_int32), ("a1", ct.c_int32), ("b0", ct.c_int32),
                ("b1", ct.c_int32), ("reserved", ct.c_int32), ("bc", Patch)]


class Box(ct.Structure):
    _fields_ = [("i0", ct.c_int32), ("i1", ct.c_int32), ("j0", ct.c_int32), ("j1", ct.c_int32),
                ("k0", ct.c_int32), ("k1", ct.c_int32), ("thermal", ct.c_int32), ("reserved", ct.c_int32),
                ("T_value", ct.c_double)]


class CaseDesc(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("precision", ct.c_int32),
                ("Lx", ct.c_double), ("Ly", ct.c_double), ("Lz", ct.c_double),
                ("nu", ct.c_double), ("Pr", ct.c_double), ("Prt", ct.c_double),
                ("sigma_k", ct.c_double), ("sigma_w", ct.c_double), ("rho", ct.c_double), ("cp", ct.c_double),
                ("gravity", ct.c_double * 3), ("beta_T", ct.c_double), ("T_ref", ct.c_double),
                ("buoyancy", ct.c_int32), ("dt_adapt", ct.c_int32), ("dt", ct.c_double), ("cfl", ct.c_double),
                ("faces", Patch * 6),
                ("vents", ct.POINTER(Vent)), ("n_vents", ct.c_int32), ("reserved0", ct.c_int32),
                ("boxes", ct.POINTER(Box)), ("n_boxes", ct.c_int32), ("reserved1", ct.c_int32),
                ("mg_levels", ct.c_int32), ("pre_sweeps", ct.c_int32), ("post_sweeps", ct.c_int32),
                ("max_vcycles", ct.c_int32), ("fixed_vcycles", ct.c_int32), ("inner_cycles", ct.c_int32),
                ("sweep_planes", ct.c_int32), ("mg_variant", ct.c_int32), ("krylov", ct.c_int32),
                ("coarse_sweeps", ct.c_int32), ("rk_stages", ct.c_int32), ("smoother", ct.c_int32),
                ("mg_rel_tol", ct.c_double), ("jacobi_weight", ct.c_double), ("seed", ct.c_uint64),
                ("init_perturb", ct.c_double), ("init_vel", ct.c_double * 3), ("init_T", ct.c_double),
                ("init_k", ct.c_double), ("init_omega", ct.c_double), ("stream", ct.c_void_p)]


class StepStats(ct.Structure):
    _fields_ = [("steps", ct.c_int32), ("vcycles_total", ct.c_int32), ("vcycles_last", ct.c_int32),
                ("reserved", ct.c_int32), ("rel_residual", ct.c_double), ("dt_last", ct.c_double),
                ("sim_time", ct.c_double)]


class CaseInfo(ct.Structure):
    _fields_ = [("cells", ct.c_int64), ("levels", ct.c_int32), ("precision", ct.c_int32),
                ("dt0", ct.c_double), ("dt", ct.c_double), ("sim_time", ct.c_double),
                ("device_bytes", ct.c_int64), ("steps", ct.c_int64), ("kernel_launches", ct.c_int64)]


class KernelStat(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int64), ("ms", ct.c_double), ("bytes", ct.c_double)]


class RequestResult(ct.Structure):
    _fields_ = [("id", ct.c_int64), ("status", ct.c_int32), ("steps", ct.c_int32), ("cells", ct.c_int64),
                ("device_bytes", ct.c_int64), ("vcycles_total", ct.c_int32), ("reserved", ct.c_int32),
                ("rel_residual", ct.c_double), ("t_arrive", ct.c_double), ("t_admit", ct.c_double),
                ("t_done", ct.c_double)]


class ServerInfo(ct.Structure):
    _fields_ = [("queued", ct.c_int64), ("running", ct.c_int64), ("done", ct.c_int64), ("bytes_in_use", ct.c_int64),
                ("rounds", ct.c_int64), ("batch_rebuilds", ct.c_int64), ("cell_steps", ct.c_int64),
                ("t_admit_s", ct.c_double), ("t_rebuild_s", ct.c_double), ("t_step_s", ct.c_double)]


class Tuning(ct.Structure):
    _fields_ = [("pre_sweeps", ct.c_int32), ("post_sweeps", ct.c_int32), ("inner_cycles", ct.c_int32),
                ("sweep_planes", ct.c_int32), ("ms_per_step", ct.c_double), ("candidates", ct.c_int32),
                ("krylov", ct.c_int32), ("coarse_sweeps", ct.c_int32), ("smoother", ct.c_int32)]


class BatchInfo(ct.Structure):
    _fields_ = [("n_cases", ct.c_int32), ("graphs", ct.c_int32), ("steps", ct.c_int64),
                ("kernel_launches", ct.c_int64), ("cells", ct.c_int64), ("launches_per_step", ct.c_int64),
                ("launches_per_outer", ct.c_int64)]


EXPORTS = ["fvm_case_bytes", "fvm_create_case", "fvm_destroy_case", "fvm_step", "fvm_run_stage", "fvm_vcycle",
           "fvm_read_fields", "fvm_write_fields", "fvm_read_fields_f32", "fvm_write_fields_f32",
           "fvm_set_poisson_rhs", "fvm_read_poisson_rhs", "fvm_lambda2",
           "fvm_projection_vjp", "fvm_destruction_vjp", "fvm_explicit_vjp", "fvm_step_vjp", "fvm_step_batch",
           "fvm_case_get_info", "fvm_set_option", "fvm_profile_enable",
           "fvm_profile_read", "fvm_struct_sizes", "fvm_last_error", "fvm_poisson_residual_static",
           "fvm_batch_create", "fvm_batch_step", "fvm_batch_launch", "fvm_batch_wait", "fvm_batch_get_info",
           "fvm_batch_destroy", "fvm_batch_profile", "fvm_server_create", "fvm_server_now", "fvm_server_submit",
           "fvm_server_poll", "fvm_server_get_info", "fvm_server_read_fields", "fvm_server_release",
           "fvm_server_destroy", "fvm_autotune"]

_lib = None


def lib():
    """Load libfvm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2603_21869_gb300.build.build()")
    L = ct.CDLL(LIB_PATH)
    CP = ct.c_void_p
    L.fvm_case_bytes.argtypes = [ct.POINTER(CaseDesc)]
    L.fvm_case_bytes.restype = ct.c_size_t
    L.fvm_create_case.argtypes = [ct.POINTER(CaseDesc), ct.POINTER(CP)]
    L.fvm_destroy_case.argtypes = [CP]
    L.fvm_destroy_case.restype = None
    L.fvm_step.argtypes = [CP, ct.c_int, ct.POINTER(StepStats)]
    L.fvm_run_stage.argtypes = [CP, ct.c_int]
    L.fvm_vcycle.argtypes = [CP, ct.c_int, ct.POINTER(ct.c_double)]
    L.fvm_read_fields.argtypes = [CP, ct.c_uint, ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_write_fields.argtypes = [CP, ct.c_uint, ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_read_fields_f32.argtypes = [CP, ct.c_uint, ct.POINTER(ct.c_float), ct.c_size_t]
    L.fvm_write_fields_f32.argtypes = [CP, ct.c_uint, ct.POINTER(ct.c_float), ct.c_size_t]
    L.fvm_set_poisson_rhs.argtypes = [CP, ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_read_poisson_rhs.argtypes = [CP, ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_lambda2.argtypes = [CP, ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_projection_vjp.argtypes = [CP, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_size_t,
                                     ct.c_double, ct.c_int32, ct.POINTER(ct.c_double)]
    L.fvm_destruction_vjp.argtypes = [CP, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                      ct.c_size_t]
    L.fvm_explicit_vjp.argtypes = [CP, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_step_vjp.argtypes = [CP, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_size_t,
                               ct.c_double, ct.c_int32, ct.POINTER(ct.c_double)]
    L.fvm_step_batch.argtypes = [ct.POINTER(CP), ct.c_int, ct.c_int, ct.POINTER(StepStats)]
    L.fvm_case_get_info.argtypes = [CP, ct.POINTER(CaseInfo)]
    L.fvm_set_option.argtypes = [CP, ct.c_int, ct.c_int64]
    L.fvm_profile_enable.argtypes = [CP, ct.c_int]
    L.fvm_profile_read.argtypes = [CP, ct.POINTER(KernelStat), ct.c_int, ct.POINTER(ct.c_int)]
    L.fvm_poisson_residual_static.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32,
                                              ct.POINTER(ct.c_double), ct.POINTER(ct.c_int32), ct.c_void_p,
                                              ct.c_void_p, ct.c_void_p]
    L.fvm_poisson_residual_static.restype = ct.c_int
    L.fvm_batch_create.argtypes = [ct.POINTER(CP), ct.c_int32, CP, ct.POINTER(CP)]
    L.fvm_batch_step.argtypes = [CP, ct.c_int32, ct.POINTER(StepStats)]
    L.fvm_batch_launch.argtypes = [CP, ct.c_int32]
    L.fvm_batch_wait.argtypes = [CP, ct.POINTER(StepStats)]
    L.fvm_batch_get_info.argtypes = [CP, ct.POINTER(BatchInfo)]
    L.fvm_batch_profile.argtypes = [CP, ct.c_int32, ct.POINTER(KernelStat), ct.c_int32, ct.POINTER(ct.c_int32)]
    L.fvm_autotune.argtypes = [ct.POINTER(CaseDesc), ct.c_int32, ct.POINTER(Tuning)]
    L.fvm_server_create.argtypes = [ct.c_int64, ct.c_int32, CP, ct.c_int32, ct.POINTER(CP)]
    L.fvm_server_now.argtypes = [CP]
    L.fvm_server_now.restype = ct.c_double
    L.fvm_server_submit.argtypes = [CP, ct.POINTER(CaseDesc), ct.c_int32, ct.c_double, ct.POINTER(ct.c_int64)]
    L.fvm_server_poll.argtypes = [CP, ct.c_int32, ct.POINTER(RequestResult), ct.c_int32, ct.POINTER(ct.c_int32)]
    L.fvm_server_get_info.argtypes = [CP, ct.POINTER(ServerInfo)]
    L.fvm_server_read_fields.argtypes = [CP, ct.c_int64, ct.c_uint, ct.POINTER(ct.c_double), ct.c_size_t]
    L.fvm_server_release.argtypes = [CP, ct.c_int64]
    L.fvm_server_destroy.argtypes = [CP]
    L.fvm_server_destroy.restype = None
    L.fvm_batch_destroy.argtypes = [CP]
    L.fvm_batch_destroy.restype = None
    L.fvm_struct_sizes.argtypes = [ct.POINTER(ct.c_size_t)]
    L.fvm_struct_sizes.restype = None
    L.fvm_last_error.restype = ct.c_char_p
    for name in ["fvm_create_case", "fvm_step", "fvm_run_stage", "fvm_vcycle", "fvm_read_fields",
                 "fvm_write_fields", "fvm_read_fields_f32", "fvm_write_fields_f32", "fvm_set_poisson_rhs",
                 "fvm_read_poisson_rhs", "fvm_lambda2",
                 "fvm_projection_vjp", "fvm_destruction_vjp", "fvm_explicit_vjp", "fvm_step_vjp",
                 "fvm_step_batch",
                 "fvm_case_get_info", "fvm_set_option", "fvm_profile_enable", "fvm_profile_read",
                 "fvm_batch_create", "fvm_batch_step", "fvm_batch_launch", "fvm_batch_wait", "fvm_batch_get_info",
                 "fvm_batch_profile",
                 "fvm_server_create", "fvm_server_submit", "fvm_server_poll", "fvm_server_get_info",
                 "fvm_server_read_fields", "fvm_server_release", "fvm_autotune"]:
        getattr(L, name).restype = ct.c_int
    _lib = L
    return L


def last_error() -> str:
    return lib().fvm_last_error().decode()


def _check(status, allow=()):
    if status != OK and status not in allow:
        raise FvmError(status, last_error())
    return status


def _patch(p: cases.Patch) -> Patch:
    return Patch(p.kind, p.thermal, p.T_value, p.u_normal, p.intensity, p.length_scale, p.T_in,
                 p.k_value, p.omega_value)


class _Desc:
    """A CaseDesc plus the vent and box arrays it points to (kept alive together)."""

    def __init__(self, spec: cases.CaseSpec, stream=None):
        self.vents = (Vent * max(1, len(spec.vents)))()
        for n, v in enumerate(spec.vents):
            self.vents[n] = Vent(v.face, v.a0, v.a1, v.b0, v.b1, 0, _patch(v.bc))
        self.boxes = (Box * max(1, len(spec.boxes)))()
        for n, b in enumerate(spec.boxes):
            self.boxes[n] = Box(b.i0, b.i1, b.j0, b.j1, b.k0, b.k1, b.thermal, 0, b.T_value)
        d = CaseDesc()
        d.nx, d.ny, d.nz, d.precision = spec.nx, spec.ny, spec.nz, spec.precision
        d.Lx, d.Ly, d.Lz = spec.Lx, spec.Ly, spec.Lz
        d.nu, d.Pr, d.Prt, d.sigma_k, d.sigma_w = spec.nu, spec.Pr, spec.Prt, spec.sigma_k, spec.sigma_w
        d.rho, d.cp = spec.rho, spec.cp
        d.gravity[:] = list(spec.gravity)
        d.beta_T, d.T_ref, d.buoyancy, d.dt_adapt = spec.beta_T, spec.T_ref, spec.buoyancy, spec.dt_adapt
        d.dt, d.cfl = spec.dt, spec.cfl
        for f in range(6):
            d.faces[f] = _patch(spec.faces[f])
        d.vents = ct.cast(self.vents, ct.POINTER(Vent))
        d.n_vents = len(spec.vents)
        d.boxes = ct.cast(self.boxes, ct.POINTER(Box))
        d.n_boxes = len(spec.boxes)
        d.mg_levels, d.pre_sweeps, d.post_sweeps = spec.mg_levels, spec.pre_sweeps, spec.post_sweeps
        d.max_vcycles, d.fixed_vcycles, d.inner_cycles = spec.max_vcycles, spec.fixed_vcycles, spec.inner_cycles
        d.sweep_planes = spec.sweep_planes
        d.mg_variant = spec.mg_variant
        d.krylov = spec.krylov
        d.coarse_sweeps = spec.coarse_sweeps
        d.rk_stages = spec.rk_stages
        d.smoother = spec.smoother
        d.mg_rel_tol, d.jacobi_weight = spec.mg_rel_tol, spec.jacobi_weight
        d.seed = spec.seed & ((1 << 64) - 1)
        d.init_perturb = spec.init_perturb
        d.init_vel[:] = list(spec.init_vel)
        d.init_T, d.init_k, d.init_omega = spec.init_T, spec.init_k, spec.init_omega
        d.stream = stream
        self.desc = d


def case_bytes(spec: cases.CaseSpec) -> int:
    """Device bytes fvm_create_case would allocate for spec (0 if invalid)."""
    d = _Desc(spec)
    return int(lib().fvm_case_bytes(ct.byref(d.desc)))


def struct_sizes():
    out = (ct.c_size_t * 11)()
    lib().fvm_struct_sizes(out)
    return list(out)


def _mask(fields):
    m = 0
    for f in fields:
        m |= 1 << cases.FIELD_INDEX[f]
    return m


class Case:
    """One case held by the library (device memory owned by libfvm)."""

    def __init__(self, spec: cases.CaseSpec, stream=None):
        self.spec = spec
        self.shape = (spec.nx, spec.ny, spec.nz)
        self.N = spec.nx * spec.ny * spec.nz
        d = _Desc(spec, stream)
        h = ct.c_void_p()
        _check(lib().fvm_create_case(ct.byref(d.desc), ct.byref(h)))
        self._h = h
        self._desc = d

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().fvm_destroy_case(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n=1, allow_not_converged=False):
        st = StepStats()
        status = lib().fvm_step(self._h, n, ct.byref(st))
        _check(status, allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return {"steps": st.steps, "vcycles_total": st.vcycles_total, "vcycles_last": st.vcycles_last,
                "rel_residual": st.rel_residual, "dt_last": st.dt_last, "sim_time": st.sim_time,
                "status": status}

    def run_stage(self, stage):
        _check(lib().fvm_run_stage(self._h, stage))

    def vcycle(self, n=1):
        rel = ct.c_double()
        _check(lib().fvm_vcycle(self._h, n, ct.byref(rel)))
        return rel.value

    def read(self, fields=cases.FIELDS, out=None):
        fields = [f for f in cases.FIELDS if f in fields]
        buf = out if out is not None else np.empty(len(fields) * self.N, dtype=np.float64)
        _check(lib().fvm_read_fields(self._h, _mask(fields), buf.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))
        nx, ny, nz = self.shape
        return {f: buf[i * self.N:(i + 1) * self.N].reshape(nz, ny, nx).transpose(2, 1, 0)
                for i, f in enumerate(fields)}

    def write(self, values: dict):
        fields = [f for f in cases.FIELDS if f in values]
        buf = np.empty(len(fields) * self.N, dtype=np.float64)
        for i, f in enumerate(fields):
            buf[i * self.N:(i + 1) * self.N] = np.asarray(values[f], dtype=np.float64).transpose(2, 1, 0).ravel()
        _check(lib().fvm_write_fields(self._h, _mask(fields), buf.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))

    def read_flat(self, out, fields=cases.FIELDS):
        """The fields into a flat float64 or float32 buffer in the library's layout
        (field after field in FIELDS order, x fastest), no host-side reshaping; a
        pinned buffer gives the full transfer rate.  float32 (fvm_read_fields_f32)
        moves an FP32-field case's state as stored and p rounded to FP32."""
        fields = [f for f in cases.FIELDS if f in fields]
        if out.dtype == np.float32:
            _check(lib().fvm_read_fields_f32(self._h, _mask(fields), out.ctypes.data_as(ct.POINTER(ct.c_float)),
                                             out.size))
        elif out.dtype == np.float64:
            _check(lib().fvm_read_fields(self._h, _mask(fields), out.ctypes.data_as(ct.POINTER(ct.c_double)),
                                         out.size))
        else:
            raise TypeError("read_flat wants a float64 or float32 buffer")
        return out

    def write_flat(self, buf, fields=cases.FIELDS):
        """The fields from a flat float64 or float32 buffer in the library's layout (see read_flat)."""
        fields = [f for f in cases.FIELDS if f in fields]
        if buf.dtype == np.float32:
            _check(lib().fvm_write_fields_f32(self._h, _mask(fields), buf.ctypes.data_as(ct.POINTER(ct.c_float)),
                                              buf.size))
        elif buf.dtype == np.float64:
            _check(lib().fvm_write_fields(self._h, _mask(fields), buf.ctypes.data_as(ct.POINTER(ct.c_double)),
                                          buf.size))
        else:
            raise TypeError("write_flat wants a float64 or float32 buffer")

    def set_rhs(self, b):
        buf = np.ascontiguousarray(np.asarray(b, dtype=np.float64).transpose(2, 1, 0).ravel())
        _check(lib().fvm_set_poisson_rhs(self._h, buf.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))

    def read_rhs(self):
        buf = np.empty(self.N, dtype=np.float64)
        _check(lib().fvm_read_poisson_rhs(self._h, buf.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))
        nx, ny, nz = self.shape
        return buf.reshape(nz, ny, nx).transpose(2, 1, 0)

    def lambda2(self, out=None):
        """lambda_2 vortex criterion of the current velocity (fvm_lambda2),
        shape (nx, ny, nz); `out` (N float64, optional) receives the flat
        x-fastest values."""
        buf = out if out is not None else np.empty(self.N, dtype=np.float64)
        _check(lib().fvm_lambda2(self._h, buf.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))
        nx, ny, nz = self.shape
        return buf.reshape(nz, ny, nx).transpose(2, 1, 0)

    def projection_vjp(self, dt, ubar, vbar, wbar, pbar=None, rel_tol=1e-13, max_vcycles=400,
                       allow_not_converged=False):
        """J^T (ubar, vbar, wbar, pbar) for the projection u* -> (u^{n+1}, p)
        (fvm_projection_vjp); arrays of shape (nx, ny, nz).  Returns
        ((xbar_u, xbar_v, xbar_w), final relative residual of the solve)."""
        nx, ny, nz = self.shape
        z = np.zeros((nx, ny, nz))
        parts = [ubar, vbar, wbar, z if pbar is None else pbar]
        buf = np.ascontiguousarray(np.concatenate(
            [np.asarray(a, dtype=np.float64).transpose(2, 1, 0).ravel() for a in parts]))
        out = np.empty(3 * self.N, dtype=np.float64)
        rel = ct.c_double()
        status = lib().fvm_projection_vjp(self._h, dt, buf.ctypes.data_as(ct.POINTER(ct.c_double)),
                                          out.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size, rel_tol,
                                          max_vcycles, ct.byref(rel))
        _check(status, allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        xs = tuple(out[i * self.N:(i + 1) * self.N].reshape(nz, ny, nx).transpose(2, 1, 0) for i in range(3))
        return xs, rel.value

    def _fields_in(self, arrays):
        return np.ascontiguousarray(np.concatenate(
            [np.asarray(a, dtype=np.float64).transpose(2, 1, 0).ravel() for a in arrays]))

    def _fields_out(self, buf, n):
        nx, ny, nz = self.shape
        return tuple(buf[i * self.N:(i + 1) * self.N].reshape(nz, ny, nx).transpose(2, 1, 0) for i in range(n))

    def destruction_vjp(self, dt, ubar, vbar, wbar, kbar, ombar):
        """Cotangents of (u, v, w, k, omega) before one destruction step over dt from
        cotangents of its output (fvm_destruction_vjp), at the current state."""
        buf = self._fields_in([ubar, vbar, wbar, kbar, ombar])
        out = np.empty(5 * self.N, dtype=np.float64)
        _check(lib().fvm_destruction_vjp(self._h, dt, buf.ctypes.data_as(ct.POINTER(ct.c_double)),
                                         out.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))
        return self._fields_out(out, 5)

    def explicit_vjp(self, dt, *ybar):
        """Cotangents of (u, v, w, T, k, omega) before the forward-Euler explicit stage over dt
        from cotangents of its output (fvm_explicit_vjp), at the current state."""
        buf = self._fields_in(ybar)
        out = np.empty(6 * self.N, dtype=np.float64)
        _check(lib().fvm_explicit_vjp(self._h, dt, buf.ctypes.data_as(ct.POINTER(ct.c_double)),
                                      out.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size))
        return self._fields_out(out, 6)

    def step_vjp(self, dt, ubar, vbar, wbar, pbar, Tbar, kbar, ombar, rel_tol=1e-13, max_vcycles=400,
                 allow_not_converged=False):
        """Cotangents of (u, v, w, T, k, omega) at the start of one time step over dt from
        cotangents of its output (fvm_step_vjp).  Returns (six arrays, relative residual of the
        adjoint pressure solve)."""
        buf = self._fields_in([ubar, vbar, wbar, pbar, Tbar, kbar, ombar])
        out = np.empty(6 * self.N, dtype=np.float64)
        rel = ct.c_double()
        status = lib().fvm_step_vjp(self._h, dt, buf.ctypes.data_as(ct.POINTER(ct.c_double)),
                                    out.ctypes.data_as(ct.POINTER(ct.c_double)), buf.size, rel_tol, max_vcycles,
                                    ct.byref(rel))
        _check(status, allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return self._fields_out(out, 6), rel.value

    def set_graph(self, enable=True):
        _check(lib().fvm_set_option(self._h, OPT_GRAPH, 1 if enable else 0))

    def profile(self, enable=True):
        _check(lib().fvm_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        cap = 256
        arr = (KernelStat * cap)()
        n = ct.c_int()
        _check(lib().fvm_profile_read(self._h, arr, cap, ct.byref(n)))
        return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
                for i in range(min(n.value, cap))}

    def info(self):
        inf = CaseInfo()
        _check(lib().fvm_case_get_info(self._h, ct.byref(inf)))
        return {k: getattr(inf, k) for k, _ in CaseInfo._fields_}


def autotune(spec: cases.CaseSpec, steps=5):
    """Measured choice of V(nu, nu), V-cycles per outer residual, the Krylov
    acceleration, the sweep weights, planes per block and the coarser levels'
    sweeps (fvm_autotune).  Returns (tuned spec, details)."""
    d = _Desc(spec)
    t = Tuning()
    _check(lib().fvm_autotune(ct.byref(d.desc), int(steps), ct.byref(t)))
    info = {k: getattr(t, k) for k, _ in Tuning._fields_}
    return spec.replace(pre_sweeps=t.pre_sweeps, post_sweeps=t.post_sweeps, inner_cycles=t.inner_cycles,
                        sweep_planes=t.sweep_planes, krylov=t.krylov, coarse_sweeps=t.coarse_sweeps,
                        smoother=t.smoother), info


def _stats(s: StepStats, status=OK):
    return {"steps": s.steps, "vcycles_total": s.vcycles_total, "vcycles_last": s.vcycles_last,
            "rel_residual": s.rel_residual, "dt_last": s.dt_last, "sim_time": s.sim_time, "status": status}


def step_batch(cs, nsteps, allow_not_converged=False):
    """One-shot batched step of the cases (a temporary fvm_batch)."""
    arr = (ct.c_void_p * len(cs))(*[c.handle.value for c in cs])
    stats = (StepStats * len(cs))()
    status = lib().fvm_step_batch(arr, len(cs), nsteps, stats)
    _check(status, allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return [_stats(s, status) for s in stats]


class Batch:
    """Cases stepped together by one CUDA graph per step (fvm_batch).  The
    cases stay owned by the caller and must outlive the batch."""

    def __init__(self, cs, stream=None):
        self.cases = list(cs)
        arr = (ct.c_void_p * len(self.cases))(*[c.handle.value for c in self.cases])
        h = ct.c_void_p()
        _check(lib().fvm_batch_create(arr, len(self.cases), stream, ct.byref(h)))
        self._h = h

    def step(self, n=1, allow_not_converged=False):
        stats = (StepStats * len(self.cases))()
        status = lib().fvm_batch_step(self._h, n, stats)
        _check(status, allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return [_stats(s, status) for s in stats]

    def launch(self, n=1):
        """Enqueue n steps and return (fvm_batch_launch); wait() collects them."""
        _check(lib().fvm_batch_launch(self._h, n))

    def wait(self, allow_not_converged=False):
        stats = (StepStats * len(self.cases))()
        status = lib().fvm_batch_wait(self._h, stats)
        _check(status, allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return [_stats(s, status) for s in stats]

    def profile(self, n=1):
        """n steps launch by launch with CUDA events around every batched launch."""
        cap = 512
        arr = (KernelStat * cap)()
        m = ct.c_int32()
        _check(lib().fvm_batch_profile(self._h, n, arr, cap, ct.byref(m)))
        return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
                for i in range(min(m.value, cap))}

    def info(self):
        inf = BatchInfo()
        _check(lib().fvm_batch_get_info(self._h, ct.byref(inf)))
        return {k: getattr(inf, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if self._h:
            lib().fvm_batch_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Request loop with continuous batching (fvm_server): requests are
    admitted by device-memory budget, stepped together, and retired."""

    def __init__(self, budget_bytes, max_cases=0, stream=None, keep_results=False):
        h = ct.c_void_p()
        _check(lib().fvm_server_create(int(budget_bytes), int(max_cases), stream, 1 if keep_results else 0,
                                       ct.byref(h)))
        self._h = h
        self._shapes = {}
        self._descs = []   # keep the submitted descriptors' arrays alive until submit copied them

    def now(self):
        return lib().fvm_server_now(self._h)

    def submit(self, spec: cases.CaseSpec, nsteps, t_arrive=None):
        d = _Desc(spec)
        rid = ct.c_int64()
        t = self.now() if t_arrive is None else float(t_arrive)
        _check(lib().fvm_server_submit(self._h, ct.byref(d.desc), int(nsteps), t, ct.byref(rid)))
        self._shapes[rid.value] = (spec.nx, spec.ny, spec.nz)
        return rid.value

    def poll(self, chunk=10, cap=1024):
        arr = (RequestResult * cap)()
        n = ct.c_int32()
        _check(lib().fvm_server_poll(self._h, int(chunk), arr, cap, ct.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in RequestResult._fields_} for i in range(min(n.value, cap))]

    def info(self):
        inf = ServerInfo()
        _check(lib().fvm_server_get_info(self._h, ct.byref(inf)))
        return {k: getattr(inf, k) for k, _ in ServerInfo._fields_}

    def read(self, rid, fields=cases.FIELDS):
        fields = [f for f in cases.FIELDS if f in fields]
        nx, ny, nz = self._shapes[rid]
        N = nx * ny * nz
        buf = np.empty(len(fields) * N, dtype=np.float64)
        _check(lib().fvm_server_read_fields(self._h, rid, _mask(fields), buf.ctypes.data_as(ct.POINTER(ct.c_double)),
                                            buf.size))
        return {f: buf[i * N:(i + 1) * N].reshape(nz, ny, nx).transpose(2, 1, 0) for i, f in enumerate(fields)}

    def release(self, rid):
        _check(lib().fvm_server_release(self._h, rid))

    def close(self):
        if self._h:
            lib().fvm_server_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
