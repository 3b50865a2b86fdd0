"""Python binding of the B300 pressure-Poisson library (libcans.so, C ABI in include/cans.h).

The functions named ``cans_*`` mirror the C entry points one to one and only marshal arguments:
device pointers (ints), sizes and the CUDA stream handle.  ``PoissonSolver`` is a small torch
convenience wrapper that owns a plan and its workspace.  Every step of a solve runs in the CUDA
library; there is no CPU fallback, and loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcans.so")

CANS_BC_P, CANS_BC_NN, CANS_BC_DD = 0, 1, 2
CANS_FP64, CANS_MIXED = 0, 1
CANS_OK = 0
CANS_ERR_ARG, CANS_ERR_UNSUPPORTED, CANS_ERR_CUDA, CANS_ERR_WORKSPACE = -1, -2, -3, -4
STATUS_NAMES = {0: "CANS_OK", -1: "CANS_ERR_ARG", -2: "CANS_ERR_UNSUPPORTED", -3: "CANS_ERR_CUDA",
                -4: "CANS_ERR_WORKSPACE", -5: "CANS_ERR_INCOMPATIBLE", -6: "CANS_ERR_NOT_CONVERGED",
                -7: "CANS_ERR_TIMEOUT"}


class CansError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({cans_status_string(status)})")


class cans_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("tol", ctypes.c_double),
                ("fp64_mode_fraction", ctypes.c_double), ("autotune", ctypes.c_int), ("shift", ctypes.c_double),
                ("z_grid", ctypes.c_int), ("verify", ctypes.c_int)]


class cans_rk3_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("cfl", ctypes.c_double), ("ubulk", ctypes.c_double),
                ("dt", ctypes.c_double), ("forcing", ctypes.c_int)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libcans.so (built in-tree by build_lib.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2001_05234_b300.build_lib.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        L.cans_opts_default.argtypes = [ctypes.POINTER(cans_opts)]
        L.cans_opts_default.restype = None
        L.cans_status_string.argtypes = [ctypes.c_int]
        L.cans_status_string.restype = ctypes.c_char_p
        L.cans_poisson_plan.argtypes = [ip, dp, ip, dp, ctypes.POINTER(cans_opts), ctypes.POINTER(vp)]
        L.cans_poisson_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_poisson_solve.argtypes = [vp, vp, vp, vp, vp, dp]
        L.cans_poisson_solve_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cans_helmholtz_solve.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, dp]
        L.cans_plan_destroy.argtypes = [vp]
        L.cans_plan_status.argtypes = [vp, ip]
        L.cans_check_bounded_wait.argtypes = [vp, ctypes.c_uint, ctypes.c_int, vp]
        L.cans_fp64_fma_probe.argtypes = [vp, ctypes.c_size_t, ctypes.c_uint, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_zslab_create.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        L.cans_zslab_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t)]
        L.cans_zslab_eliminate.argtypes = [vp, vp, vp, vp, vp, vp]
        L.cans_zslab_finish.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp]
        L.cans_zslab_destroy.argtypes = [vp]
        L.cans_poisson_solve_divergence.argtypes = [vp, vp, vp, vp, ctypes.c_double, vp, ctypes.c_double, vp, vp,
                                                    vp, vp, dp]
        L.cans_poisson_adjoint_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_poisson_solve_adjoint.argtypes = [vp, vp, vp, vp, vp]
        L.cans_transform_xy.argtypes = [vp, vp, ctypes.c_int, vp]
        L.cans_transform_xy_f32.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.cans_zsolve.argtypes = [vp, vp, vp]
        L.cans_plan_eigenvalues.argtypes = [vp, dp, dp]
        L.cans_plan_profile.argtypes = [vp, ctypes.c_int]
        L.cans_poisson_solve_noalloc.argtypes = [vp, vp, vp, vp, dp]
        L.cans_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
        L.cans_batch_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
        L.cans_batch_destroy.argtypes = [vp]
        L.cans_poisson_batched_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(vp),
                                                           ctypes.POINTER(ctypes.c_size_t)]
        L.cans_poisson_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                 ctypes.POINTER(vp), vp, vp, vp]
        L.cans_rk3_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_rk3_step.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(cans_rk3_params), vp, vp, vp]
        L.cans_rk3_implicit_workspace_size.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_box_rk3_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_box_rk3_step.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(cans_rk3_params), ctypes.c_double, vp,
                                        vp, vp]
        L.cans_rk3_step_implicit.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(cans_rk3_params), vp, vp, vp]
        L.cans_project_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cans_project.argtypes = [vp, vp, vp, vp, vp, vp]
        L.cans_project_adjoint.argtypes = [vp, vp, vp, vp, vp, vp]
        L.cans_noalloc_scratch_bytes.argtypes = []
        L.cans_noalloc_scratch_bytes.restype = ctypes.c_size_t
        L.cans_plan_profile_read.argtypes = [vp, ctypes.c_int, dp, ip]
        L.cans_split_f64.argtypes = [vp, ctypes.c_size_t, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _check(status: int, where: str) -> int:
    if status != CANS_OK:
        raise CansError(status, where)
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- one-to-one C entry points ----------------------------------------------------------------
def cans_status_string(status: int) -> str:
    return lib().cans_status_string(int(status)).decode()


def cans_opts_default() -> cans_opts:
    o = cans_opts()
    lib().cans_opts_default(ctypes.byref(o))
    return o


def cans_poisson_plan(n, len_xy, bc, dzf=None, opts: cans_opts | None = None, check: bool = True):
    """Returns (status, plan handle)."""
    n_a = (ctypes.c_int * 3)(*[int(v) for v in n])
    l_a = (ctypes.c_double * 2)(*[float(v) for v in len_xy])
    b_a = (ctypes.c_int * 3)(*[int(v) for v in bc])
    dz = None
    if dzf is not None:
        dz = np.ascontiguousarray(dzf, dtype=np.float64)
        if dz.shape != (int(n[2]),):
            raise ValueError("dzf must hold n[2] cell widths")
    h = ctypes.c_void_p()
    st = lib().cans_poisson_plan(n_a, l_a, b_a, _dptr(dz) if dz is not None else None,
                                 ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    if check:
        _check(st, "cans_poisson_plan")
    return st, h


def cans_poisson_workspace_size(plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().cans_poisson_workspace_size(plan, ctypes.byref(b)), "cans_poisson_workspace_size")
    return int(b.value)


def cans_poisson_solve(plan, f_ptr: int, p_ptr: int, workspace_ptr: int, stream_ptr: int, info=None) -> int:
    """Returns the status; info (numpy float64 array of max_sweeps+2) is filled when given."""
    return lib().cans_poisson_solve(plan, f_ptr, p_ptr, workspace_ptr or None, stream_ptr or None,
                                    _dptr(info) if info is not None else None)


def cans_helmholtz_solve(plan, f_ptr: int, p_ptr: int, shift: float, workspace_ptr: int, stream_ptr: int,
                         info=None) -> int:
    """(L_h + shift) p = f; returns the status (info as cans_poisson_solve)."""
    return lib().cans_helmholtz_solve(plan, f_ptr, p_ptr, float(shift), workspace_ptr or None, stream_ptr or None,
                                      _dptr(info) if info is not None else None)


def cans_poisson_solve_noalloc(plan, f_ptr: int, p_ptr: int, stream_ptr: int, info=None) -> int:
    """cans_poisson_solve without a caller workspace: the library's fixed scratch array is used
    (for callers that cannot allocate device memory).  Calls that overlap on the GPU race."""
    return lib().cans_poisson_solve_noalloc(plan, f_ptr, p_ptr, stream_ptr or None,
                                            _dptr(info) if info is not None else None)


def cans_rk3_workspace_size(plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().cans_rk3_workspace_size(plan, ctypes.byref(b)), "cans_rk3_workspace_size")
    return int(b.value)


def cans_rk3_implicit_workspace_size(plan, uv_plan, w_plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().cans_rk3_implicit_workspace_size(plan, uv_plan, w_plan, ctypes.byref(b)),
           "cans_rk3_implicit_workspace_size")
    return int(b.value)


def cans_rk3_step_implicit(plan, uv_plan, w_plan, u_ptr: int, v_ptr: int, w_ptr: int, p_ptr: int,
                           params: cans_rk3_params, dt_dev_ptr: int, workspace_ptr: int, stream_ptr: int) -> int:
    return lib().cans_rk3_step_implicit(plan, uv_plan, w_plan, u_ptr, v_ptr, w_ptr, p_ptr, ctypes.byref(params),
                                        dt_dev_ptr or None, workspace_ptr, stream_ptr or None)


def cans_rk3_step(plan, u_ptr: int, v_ptr: int, w_ptr: int, p_ptr: int, params: cans_rk3_params, dt_dev_ptr: int,
                  workspace_ptr: int, stream_ptr: int) -> int:
    return lib().cans_rk3_step(plan, u_ptr, v_ptr, w_ptr, p_ptr, ctypes.byref(params), dt_dev_ptr or None,
                               workspace_ptr, stream_ptr or None)


def cans_project_workspace_size(plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().cans_project_workspace_size(plan, ctypes.byref(b)), "cans_project_workspace_size")
    return int(b.value)


def cans_project(plan, u_ptr: int, v_ptr: int, w_ptr: int, workspace_ptr: int, stream_ptr: int) -> int:
    return lib().cans_project(plan, u_ptr, v_ptr, w_ptr, workspace_ptr, stream_ptr or None)


def cans_project_adjoint(plan, u_ptr: int, v_ptr: int, w_ptr: int, workspace_ptr: int, stream_ptr: int) -> int:
    return lib().cans_project_adjoint(plan, u_ptr, v_ptr, w_ptr, workspace_ptr, stream_ptr or None)


def cans_batch_create(plans, nstreams: int = 8):
    arr = (ctypes.c_void_p * len(plans))(*[p.value if hasattr(p, "value") else p for p in plans])
    h = ctypes.c_void_p()
    _check(lib().cans_batch_create(len(plans), arr, int(nstreams), ctypes.byref(h)), "cans_batch_create")
    return h


def cans_batch_workspace_size(batch) -> int:
    b = ctypes.c_size_t()
    _check(lib().cans_batch_workspace_size(batch, ctypes.byref(b)), "cans_batch_workspace_size")
    return int(b.value)


def cans_batch_solve(batch, f_ptrs, p_ptrs, workspace_ptr: int, stream_ptr: int) -> int:
    fa = (ctypes.c_void_p * len(f_ptrs))(*f_ptrs)
    pa = (ctypes.c_void_p * len(p_ptrs))(*p_ptrs)
    return lib().cans_batch_solve(batch, fa, pa, workspace_ptr or None, stream_ptr or None)


def cans_batch_destroy(batch) -> int:
    return lib().cans_batch_destroy(batch)


def cans_poisson_batched_workspace_size(plans) -> int:
    arr = (ctypes.c_void_p * len(plans))(*[p.value if hasattr(p, "value") else p for p in plans])
    b = ctypes.c_size_t()
    _check(lib().cans_poisson_batched_workspace_size(len(plans), arr, ctypes.byref(b)),
           "cans_poisson_batched_workspace_size")
    return int(b.value)


def cans_poisson_solve_batched(plans, f_ptrs, p_ptrs, workspace_ptr: int, stream_ptr: int, status_ptr: int = 0) -> int:
    arr = (ctypes.c_void_p * len(plans))(*[p.value if hasattr(p, "value") else p for p in plans])
    fa = (ctypes.c_void_p * len(f_ptrs))(*f_ptrs)
    pa = (ctypes.c_void_p * len(p_ptrs))(*p_ptrs)
    return lib().cans_poisson_solve_batched(len(plans), arr, fa, pa, workspace_ptr or None, stream_ptr or None,
                                            status_ptr or None)


def cans_noalloc_scratch_bytes() -> int:
    return int(lib().cans_noalloc_scratch_bytes())


def cans_plan_destroy(plan) -> int:
    return lib().cans_plan_destroy(plan)


def cans_poisson_solve_divergence(plan, u: int, v: int, w: int, scale: float, dt_ptr: int, gamma: float, f_ptr: int,
                                  p_ptr: int, workspace_ptr: int, stream_ptr: int, info=None) -> int:
    """cans_poisson_solve_divergence: p solves L_h p = scale / (gamma dt) D(u, v, w) (dt on the device;
    dt_ptr 0: scale D(u, v, w)); f_ptr (0 allowed where the solve does not re-read f) receives f."""
    return lib().cans_poisson_solve_divergence(plan, u, v, w, float(scale), dt_ptr or None, float(gamma), f_ptr or None,
                                               p_ptr, workspace_ptr or None, stream_ptr or None,
                                               _dptr(info) if info is not None else None)


def cans_zslab_create(plan, z0: int, z1: int):
    h = ctypes.c_void_p()
    _check(lib().cans_zslab_create(plan, int(z0), int(z1), ctypes.byref(h)), "cans_zslab_create")
    return h


def cans_zslab_sizes(slab):
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().cans_zslab_sizes(slab, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "cans_zslab_sizes")
    return int(a.value), int(b.value), int(c.value)


def cans_zslab_eliminate(slab, field: int, iface: int, col00: int, workspace: int, stream_ptr: int) -> int:
    return lib().cans_zslab_eliminate(slab, field, iface, col00, workspace, stream_ptr or None)


def cans_zslab_finish(slab, field: int, iface_all: int, col00_all: int, nranks: int, rank: int, scale: float,
                      workspace: int, stream_ptr: int) -> int:
    return lib().cans_zslab_finish(slab, field, iface_all, col00_all or None, int(nranks), int(rank), float(scale),
                                   workspace, stream_ptr or None)


def cans_zslab_destroy(slab) -> int:
    return lib().cans_zslab_destroy(slab)


def cans_check_bounded_wait(plan, polls: int, complete: bool, stream=None) -> None:
    """Run the bounded device-side wait on a barrier that completes (complete) or never does
    (cans_check_bounded_wait): a wait that runs out records CANS_ERR_TIMEOUT in the plan's status word."""
    _check(lib().cans_check_bounded_wait(plan, int(polls), 1 if complete else 0, _stream_ptr(stream) or None),
           "cans_check_bounded_wait")


def fp64_fma_tflops(iters: int = 20000, reps: int = 3) -> float:
    """The GPU's FP64 FMA rate in TFLOP/s (cans_fp64_fma_probe timed with CUDA events, best of reps)."""
    import torch

    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    out = torch.empty(props.multi_processor_count * 2048, dtype=torch.float64, device="cuda")
    flops = ctypes.c_size_t(0)
    st = torch.cuda.current_stream()
    best = 0.0
    for _ in range(reps + 1):  # the first launch warms up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(lib().cans_fp64_fma_probe(out.data_ptr(), out.numel(), int(iters), _stream_ptr(st),
                                         ctypes.byref(flops)), "cans_fp64_fma_probe")
        e1.record(st)
        e1.synchronize()
        best = max(best, flops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def cans_plan_status(plan) -> int:
    """The plan's device status word (synchronises the device, then clears the word)."""
    word = ctypes.c_int(0)
    _check(lib().cans_plan_status(plan, ctypes.byref(word)), "cans_plan_status")
    return int(word.value)


def cans_poisson_adjoint_workspace_size(plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().cans_poisson_adjoint_workspace_size(plan, ctypes.byref(b)), "cans_poisson_adjoint_workspace_size")
    return int(b.value)


def cans_poisson_solve_adjoint(plan, g_ptr: int, q_ptr: int, workspace_ptr: int, stream_ptr: int) -> int:
    return lib().cans_poisson_solve_adjoint(plan, g_ptr, q_ptr, workspace_ptr or None, stream_ptr or None)


def cans_transform_xy(plan, field_ptr: int, direction: int, stream_ptr: int) -> int:
    return lib().cans_transform_xy(plan, field_ptr, int(direction), stream_ptr or None)


def cans_transform_xy_f32(plan, field_ptr: int, work_ptr: int, direction: int, stream_ptr: int) -> int:
    return lib().cans_transform_xy_f32(plan, field_ptr, work_ptr, int(direction), stream_ptr or None)


def cans_zsolve(plan, field_ptr: int, stream_ptr: int) -> int:
    return lib().cans_zsolve(plan, field_ptr, stream_ptr or None)


def cans_plan_eigenvalues(plan, nx: int, ny: int):
    mx, my = np.empty(nx), np.empty(ny)
    _check(lib().cans_plan_eigenvalues(plan, _dptr(mx), _dptr(my)), "cans_plan_eigenvalues")
    return mx, my


def cans_split_f64(x_ptr: int, n: int, rn_ptr: int = 0, hi_ptr: int = 0, lo_ptr: int = 0, back_ptr: int = 0,
                   stream_ptr: int = 0) -> int:
    """Element-wise double -> float conversions of the mixed path (device pointers; 0 = not wanted)."""
    return lib().cans_split_f64(x_ptr or None, int(n), rn_ptr or None, hi_ptr or None, lo_ptr or None,
                                back_ptr or None, stream_ptr or None)


CANS_PASS_NAMES = ("x_forward", "y_forward", "z_solve", "y_inverse", "x_inverse", "x_forward_residual",
                   "x_inverse_update", "residual_stencil", "z_solve_double_columns", "momentum", "divergence",
                   "correction", "chkdt", "forcing")


def cans_plan_profile(plan, enable: bool) -> int:
    return lib().cans_plan_profile(plan, 1 if enable else 0)


def cans_plan_profile_read(plan, pass_kind: int):
    """(total milliseconds, launches) of one pass kind since profiling was enabled."""
    ms = ctypes.c_double()
    n = ctypes.c_int()
    _check(lib().cans_plan_profile_read(plan, int(pass_kind), ctypes.byref(ms), ctypes.byref(n)),
           "cans_plan_profile_read")
    return float(ms.value), int(n.value)


# ---- torch convenience -------------------------------------------------------------------------
def _stream_ptr(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class PoissonSolver:
    """Owns a plan and its device workspace.  f, p: torch float64 CUDA tensors of shape (Nz, Ny, Nx).
    shift: the plan's Helmholtz shift (solves (L_h + shift) p = f); z_grid 1: unknowns on the interior
    z-faces (a staggered w; the solve uses the first Nz - 1 planes)."""

    def __init__(self, n, bc, length_xy=(1.0, 1.0), dzf=None, prec=CANS_FP64, sweeps=2, tol=1e-12,
                 fp64_fraction=0.01, autotune=False, shift=0.0, z_grid=0, verify=False):
        import torch

        self.n = tuple(int(v) for v in n)
        self.bc = tuple(int(v) for v in bc)
        o = cans_opts_default()
        o.prec = int(prec)
        o.max_sweeps = int(sweeps)
        o.tol = float(tol)
        o.fp64_mode_fraction = float(fp64_fraction)
        o.autotune = 1 if autotune else 0
        o.shift = float(shift)
        o.z_grid = int(z_grid)
        o.verify = 1 if verify else 0
        self.opts = o
        _, self.plan = cans_poisson_plan(self.n, length_xy, self.bc, dzf, o)
        nbytes = cans_poisson_workspace_size(self.plan)
        self.workspace = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device="cuda")
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = self.workspace.data_ptr() + off if nbytes else 0

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def solve(self, f, out=None, stream=None, info: bool = False, shift=None):
        """p = (L_h + shift)^-1 f; shift None = the plan's own (cans_poisson_solve), else a per-call
        Helmholtz shift (cans_helmholtz_solve)."""
        import torch

        assert f.dtype == torch.float64 and f.is_cuda and f.is_contiguous() and tuple(f.shape) == self.shape
        if out is None:
            out = torch.empty_like(f)
        buf = np.zeros(self.opts.max_sweeps + 2) if info else None
        if shift is None:
            st = cans_poisson_solve(self.plan, f.data_ptr(), out.data_ptr(), self._ws_ptr, _stream_ptr(stream), buf)
        else:
            st = cans_helmholtz_solve(self.plan, f.data_ptr(), out.data_ptr(), shift, self._ws_ptr,
                                      _stream_ptr(stream), buf)
        if st != CANS_OK and not (info and st in (-5, -6)):
            raise CansError(st, "cans_helmholtz_solve" if shift is not None else "cans_poisson_solve")
        return (out, buf, st) if info else out

    def solve_host(self, f_host, p_host, f_dev, p_dev, copy_in=None, compute=None, copy_out=None):
        """cans_poisson_solve_host: upload f_host into f_dev on copy_in, solve into p_dev on compute,
        download into p_host on copy_out (torch streams; None = the current stream), all asynchronous."""
        import torch

        for t, dev in ((f_host, False), (p_host, False), (f_dev, True), (p_dev, True)):
            assert t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == self.shape
            assert t.is_cuda == dev
        _check(lib().cans_poisson_solve_host(self.plan, f_host.data_ptr(), p_host.data_ptr(), f_dev.data_ptr(),
                                             p_dev.data_ptr(), self._ws_ptr, _stream_ptr(copy_in),
                                             _stream_ptr(compute), _stream_ptr(copy_out)),
               "cans_poisson_solve_host")
        return p_host

    def status(self) -> int:
        """The plan's device status word since the last read (cans_plan_status; synchronises)."""
        return cans_plan_status(self.plan)

    def solve_adjoint(self, g, out=None, stream=None):
        """q = S^T g (cans_poisson_solve_adjoint); the adjoint workspace is allocated on first use."""
        import torch

        assert g.dtype == torch.float64 and g.is_cuda and g.is_contiguous() and tuple(g.shape) == self.shape
        if out is None:
            out = torch.empty_like(g)
        if getattr(self, "_adj_ws", None) is None:
            self._adj_ws, self._adj_ptr = _aligned_workspace(cans_poisson_adjoint_workspace_size(self.plan))
        _check(cans_poisson_solve_adjoint(self.plan, g.data_ptr(), out.data_ptr(), self._adj_ptr, _stream_ptr(stream)),
               "cans_poisson_solve_adjoint")
        return out

    def close(self):
        if getattr(self, "plan", None):
            cans_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _poisson_function():
    import torch

    class PoissonSolve(torch.autograd.Function):
        """f -> p = S f (the solver's plan); backward applies S^T through cans_poisson_solve_adjoint."""

        @staticmethod
        def forward(ctx, solver, f):
            ctx.solver = solver
            return solver.solve(f.detach().contiguous())

        @staticmethod
        def backward(ctx, gp):
            return None, ctx.solver.solve_adjoint(gp.contiguous())

    return PoissonSolve


_Poisson = None


def poisson_solve(solver, f):
    """Differentiable Poisson solve: returns S f; gradients flow through the adjoint solve."""
    global _Poisson
    if _Poisson is None:
        _Poisson = _poisson_function()
    return _Poisson.apply(solver, f)


def _aligned_workspace(nbytes: int):
    import torch

    buf = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device="cuda")
    return buf, (buf.data_ptr() + 255) // 256 * 256


class Channel:
    """Channel flow (x, y periodic, no-slip walls in z) on one GPU: plan + workspaces for the RK3 step
    and the projection.  Velocities u, v, w and pressure p are float64 CUDA tensors (Nz, Ny, Nx)."""

    def __init__(self, n, length_xy, dzf, prec=CANS_FP64, sweeps=2, implicit=False):
        self.n = tuple(int(v) for v in n)
        o = cans_opts_default()
        o.prec = int(prec)
        o.max_sweeps = int(sweeps)
        _, self.plan = cans_poisson_plan(self.n, length_xy, (CANS_BC_P, CANS_BC_P, CANS_BC_NN), dzf, o)
        self._rk_buf, self._rk_ws = _aligned_workspace(cans_rk3_workspace_size(self.plan))
        self._pj_buf, self._pj_ws = _aligned_workspace(cans_project_workspace_size(self.plan))
        self.uv_plan = self.w_plan = None
        if implicit:  # the velocity Helmholtz plans of the Crank-Nicolson step
            vel = (CANS_BC_P, CANS_BC_P, CANS_BC_DD)
            _, self.uv_plan = cans_poisson_plan(self.n, length_xy, vel, dzf, o)
            ow = cans_opts_default()
            ow.prec, ow.max_sweeps, ow.z_grid = int(prec), int(sweeps), 1
            _, self.w_plan = cans_poisson_plan(self.n, length_xy, vel, dzf, ow)
            self._im_buf, self._im_ws = _aligned_workspace(
                cans_rk3_implicit_workspace_size(self.plan, self.uv_plan, self.w_plan))

    def rk3_step_implicit(self, u, v, w, p, nu, dt, ubulk=1.0, forcing=True, dt_out=None, stream=None):
        """One RK3 step with Crank-Nicolson diffusion (cans_rk3_step_implicit); dt fixed (> 0)."""
        prm = cans_rk3_params(float(nu), 1.0, float(ubulk), float(dt), 1 if forcing else 0)
        st = cans_rk3_step_implicit(self.plan, self.uv_plan, self.w_plan, u.data_ptr(), v.data_ptr(), w.data_ptr(),
                                    p.data_ptr(), prm, dt_out.data_ptr() if dt_out is not None else 0, self._im_ws,
                                    _stream_ptr(stream))
        _check(st, "cans_rk3_step_implicit")

    def rk3_step(self, u, v, w, p, nu, cfl=0.9, ubulk=1.0, dt=0.0, forcing=True, dt_out=None, stream=None):
        prm = cans_rk3_params(float(nu), float(cfl), float(ubulk), float(dt), 1 if forcing else 0)
        st = cans_rk3_step(self.plan, u.data_ptr(), v.data_ptr(), w.data_ptr(), p.data_ptr(), prm,
                           dt_out.data_ptr() if dt_out is not None else 0, self._rk_ws, _stream_ptr(stream))
        _check(st, "cans_rk3_step")

    def project_(self, u, v, w, adjoint=False, stream=None):
        fn = cans_project_adjoint if adjoint else cans_project
        _check(fn(self.plan, u.data_ptr(), v.data_ptr(), w.data_ptr(), self._pj_ws, _stream_ptr(stream)),
               "cans_project")
        return u, v, w

    def close(self):
        for name in ("plan", "uv_plan", "w_plan"):
            if getattr(self, name, None):
                cans_plan_destroy(getattr(self, name))
                setattr(self, name, None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Box:
    """Fractional-step flow in a box: each direction periodic (False) or bounded by no-slip walls (True),
    an optional lid (the top z wall moving along x).  u, v, w, p: float64 CUDA tensors (Nz, Ny, Nx)."""

    def __init__(self, n, length_xy, dzf, walls, prec=CANS_FP64, sweeps=2):
        self.n = tuple(int(v) for v in n)
        self.walls = tuple(bool(x) for x in walls)
        o = cans_opts_default()
        o.prec, o.max_sweeps = int(prec), int(sweeps)
        bc = tuple(CANS_BC_NN if wl else CANS_BC_P for wl in self.walls)
        _, self.plan = cans_poisson_plan(self.n, length_xy, bc, dzf, o)
        b = ctypes.c_size_t()
        _check(lib().cans_box_rk3_workspace_size(self.plan, ctypes.byref(b)), "cans_box_rk3_workspace_size")
        self._buf, self._ws = _aligned_workspace(int(b.value))

    def rk3_step(self, u, v, w, p, nu, cfl=0.5, ubulk=0.0, dt=0.0, forcing=False, lid=0.0, dt_out=None, stream=None):
        prm = cans_rk3_params(float(nu), float(cfl), float(ubulk), float(dt), 1 if forcing else 0)
        st = lib().cans_box_rk3_step(self.plan, u.data_ptr(), v.data_ptr(), w.data_ptr(), p.data_ptr(),
                                     ctypes.byref(prm), float(lid), dt_out.data_ptr() if dt_out is not None else None,
                                     self._ws, _stream_ptr(stream) or None)
        _check(st, "cans_box_rk3_step")

    def close(self):
        if getattr(self, "plan", None):
            cans_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _projection_function():
    import torch

    class Projection(torch.autograd.Function):
        """u* -> P u* (divergence-free part); backward applies P^T through cans_project_adjoint."""

        @staticmethod
        def forward(ctx, chan, u, v, w):
            ctx.chan = chan
            uo, vo, wo = u.detach().clone(), v.detach().clone(), w.detach().clone()
            chan.project_(uo, vo, wo)
            return uo, vo, wo

        @staticmethod
        def backward(ctx, gu, gv, gw):
            gu, gv, gw = gu.contiguous().clone(), gv.contiguous().clone(), gw.contiguous().clone()
            ctx.chan.project_(gu, gv, gw, adjoint=True)
            return None, gu, gv, gw

    return Projection


_Projection = None


def projection(chan, u, v, w):
    """Differentiable projection: returns P(u, v, w); gradients flow through the adjoint kernel."""
    global _Projection
    if _Projection is None:
        _Projection = _projection_function()
    return _Projection.apply(chan, u, v, w)


class Batch:
    """Many independent Poisson problems solved in one asynchronous call (cans_batch_*).
    cases: objects with .n, .bc, .length_xy, .dzf (e.g. inputs.PoissonCase)."""

    def __init__(self, cases, prec=CANS_MIXED, sweeps=2, nstreams=8, autotune=False):
        self.cases = list(cases)
        self.plans = []
        for c in self.cases:
            o = cans_opts_default()
            o.prec, o.max_sweeps = int(prec), int(sweeps)
            o.autotune = 1 if autotune else 0
            self.plans.append(cans_poisson_plan(c.n, c.length_xy, c.bc, c.dzf, o)[1])
        self.batch = cans_batch_create(self.plans, nstreams)
        self._ws_buf, self._ws = _aligned_workspace(cans_batch_workspace_size(self.batch))

    def solve(self, fs, ps, stream=None):
        _check(cans_batch_solve(self.batch, [t.data_ptr() for t in fs], [t.data_ptr() for t in ps], self._ws,
                                _stream_ptr(stream)), "cans_batch_solve")
        return ps

    def close(self):
        if getattr(self, "batch", None):
            cans_batch_destroy(self.batch)
            self.batch = None
        for p in getattr(self, "plans", []):
            cans_plan_destroy(p)
        self.plans = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
