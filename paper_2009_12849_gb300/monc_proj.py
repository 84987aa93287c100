"""Python binding of the C ABI in ``include/monc_proj.h`` (argument marshalling only).

PyTorch supplies device memory and streams; every step of the projection runs
in the CUDA kernels of ``libmonc_proj.so``.  There is no fallback: if the
library is missing, every call raises.

The functions keep the C names (``monc_proj_plan``, ``monc_proj_solve``, ...);
``Projector`` wraps one plan with its workspace for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmonc_proj.so")

MONC_PROJ_OK = 0
MONC_PROJ_EINVAL = 1
MONC_PROJ_EUNSUPPORTED = 2
MONC_PROJ_ENOMEM = 3
MONC_PROJ_ECUDA = 4
MONC_PROJ_ETIMEOUT = 5
MONC_PROJ_EDEVICE = 6
MONC_PROJ_ESCRATCH = 7
MONC_PROJ_ENOCONV = 8
MONC_PROJ_EBREAKDOWN = 9
MONC_PROJ_PC_NONE = 0
MONC_PROJ_PC_LINE = 1
PRECONDITIONERS = {"none": MONC_PROJ_PC_NONE, "line": MONC_PROJ_PC_LINE}
MONC_PROJ_NOALLOC_SCRATCH_BYTES = 32 << 20
MONC_PROJ_FP64 = 0
MONC_PROJ_MIXED = 1
MONC_PROJ_REFINED = 2
MONC_PROJ_MIXED_Z64 = 3

PRECISIONS = {"fp64": MONC_PROJ_FP64, "mixed": MONC_PROJ_MIXED, "refined": MONC_PROJ_REFINED,
              "mixed_z64": MONC_PROJ_MIXED_Z64}
DTYPES = {MONC_PROJ_FP64: torch.float64, MONC_PROJ_MIXED: torch.float32, MONC_PROJ_REFINED: torch.float64,
          MONC_PROJ_MIXED_Z64: torch.float32}

EXPORTS = [
    "monc_proj_plan", "monc_proj_workspace_size", "monc_proj_solve",
    "monc_proj_batch_workspace_size", "monc_proj_solve_batch", "monc_proj_sync_status",
    "monc_proj_destroy", "monc_proj_status_string", "monc_proj_plan_info",
    "monc_proj_profile", "monc_proj_profile_read", "monc_proj_phase_name",
    "monc_proj_solve_noalloc", "monc_proj_autotune", "monc_proj_host_staging_size", "monc_proj_solve_host",
    "monc_proj_krylov_workspace_size", "monc_proj_solve_krylov", "monc_proj_set_allocator",
    "monc_proj_spectral_pitch", "monc_proj_forward_slab", "monc_proj_vertical_pencil", "monc_proj_inverse_slab",
    "monc_proj_pack_pencils", "monc_proj_unpack_pencils", "monc_proj_solve_batch_grouped",
    "monc_proj_plan_schedule", "monc_proj_set_schedule",
]

# Allocator hooks of plan tables (monc_proj_set_allocator)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class ProjError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {monc_proj_status_string(status)} (status {status})")


class Fields(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("u_out", ctypes.c_void_p), ("v_out", ctypes.c_void_p), ("w_out", ctypes.c_void_p),
                ("phi_out", ctypes.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmonc_proj.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    L.monc_proj_plan.argtypes = [ctypes.POINTER(vp), i, i, i, d, d, dp, dp, dp, i, vp]
    L.monc_proj_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.monc_proj_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.monc_proj_batch_workspace_size.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(sz)]
    L.monc_proj_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Fields), i, vp, sz, vp]
    L.monc_proj_solve_batch_grouped.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Fields), i, vp, sz, vp]
    L.monc_proj_set_schedule.argtypes = [vp, i, i, i]
    L.monc_proj_sync_status.argtypes = [vp, vp]
    L.monc_proj_destroy.argtypes = [vp]
    L.monc_proj_status_string.argtypes = [i]
    L.monc_proj_status_string.restype = ctypes.c_char_p
    ll = ctypes.POINTER(ctypes.c_longlong)
    ip = ctypes.POINTER(ctypes.c_int)
    L.monc_proj_plan_info.argtypes = [vp, ip, ip, ip, ip, ll, ll]
    L.monc_proj_profile.argtypes = [vp, i]
    L.monc_proj_profile_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), ip, ip]
    L.monc_proj_phase_name.argtypes = [i]
    L.monc_proj_phase_name.restype = ctypes.c_char_p
    L.monc_proj_solve_noalloc.argtypes = [i, i, i, d, d, dp, dp, dp, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.monc_proj_autotune.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i, vp, ip, ip]
    L.monc_proj_host_staging_size.argtypes = [vp, i, ctypes.POINTER(sz)]
    L.monc_proj_solve_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp, vp]
    L.monc_proj_krylov_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.monc_proj_solve_krylov.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, d, i, i, ip, dp, vp]
    L.monc_proj_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    L.monc_proj_spectral_pitch.argtypes = [vp, ip]
    L.monc_proj_forward_slab.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp]
    L.monc_proj_vertical_pencil.argtypes = [vp, i, i, vp, vp, vp, vp]
    L.monc_proj_plan_schedule.argtypes = [vp, ip, ip, ip, ip]
    L.monc_proj_inverse_slab.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.monc_proj_pack_pencils.argtypes = [vp, i, i, vp, vp, vp]
    L.monc_proj_unpack_pencils.argtypes = [vp, i, i, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("monc_proj_status_string", "monc_proj_phase_name"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != MONC_PROJ_OK:
        raise ProjError(rc, where)


def _dbl(a) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return (ctypes.c_double * a.size)(*a.tolist())


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ----------------------------------------------------------------- C names

def monc_proj_status_string(status: int) -> str:
    return load_library().monc_proj_status_string(int(status)).decode()


def monc_proj_plan(nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision="fp64", stream=None) -> int:
    """Create a plan; returns the opaque handle (an int)."""
    L = load_library()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    h = ctypes.c_void_p()
    if len(dz) != nz or len(rho_c) != nz or len(rho_f) != nz + 1:
        raise ProjError(MONC_PROJ_EINVAL, "monc_proj_plan")
    rc = L.monc_proj_plan(ctypes.byref(h), int(nx), int(ny), int(nz), float(dx), float(dy),
                          _dbl(dz), _dbl(rho_c), _dbl(rho_f), prec,
                          ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_plan")
    return h.value


def monc_proj_workspace_size(plan: int) -> int:
    n = ctypes.c_size_t()
    _check(load_library().monc_proj_workspace_size(ctypes.c_void_p(plan), ctypes.byref(n)),
           "monc_proj_workspace_size")
    return n.value


def monc_proj_solve(plan: int, u, v, w, u_out, v_out, w_out, phi_out, workspace, stream=None):
    """Enqueue one projection; tensors are passed by their device pointers."""
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
    rc = load_library().monc_proj_solve(ctypes.c_void_p(plan), ptr(u), ptr(v), ptr(w), ptr(u_out),
                                        ptr(v_out), ptr(w_out), ptr(phi_out), ptr(workspace),
                                        ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_solve")


def monc_proj_autotune(plan: int, u, v, w, u_out, v_out, w_out, workspace, reps=3, stream=None):
    """Time the plan's candidate task shapes on these fields and keep the
    fastest; returns (row_threads, col_threads)."""
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rt, ct = ctypes.c_int(), ctypes.c_int()
    _check(load_library().monc_proj_autotune(ctypes.c_void_p(plan), ptr(u), ptr(v), ptr(w), ptr(u_out),
                                             ptr(v_out), ptr(w_out), ptr(workspace), int(reps),
                                             ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(rt),
                                             ctypes.byref(ct)), "monc_proj_autotune")
    return rt.value, ct.value


def monc_proj_host_staging_size(plan: int, with_phi=False) -> int:
    n = ctypes.c_size_t()
    _check(load_library().monc_proj_host_staging_size(ctypes.c_void_p(plan), int(bool(with_phi)), ctypes.byref(n)),
           "monc_proj_host_staging_size")
    return n.value


def monc_proj_solve_host(plan: int, u, v, w, u_out, v_out, w_out, phi_out, staging, workspace, stream=None):
    """Enqueue one projection of host tensors (page-locked for asynchronous
    copies) through a device staging buffer."""
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
    rc = load_library().monc_proj_solve_host(ctypes.c_void_p(plan), ptr(u), ptr(v), ptr(w), ptr(u_out), ptr(v_out),
                                             ptr(w_out), ptr(phi_out), ptr(staging),
                                             ctypes.c_size_t(staging.numel() * staging.element_size()),
                                             ptr(workspace), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_solve_host")


def monc_proj_krylov_workspace_size(plan: int) -> int:
    n = ctypes.c_size_t()
    _check(load_library().monc_proj_krylov_workspace_size(ctypes.c_void_p(plan), ctypes.byref(n)),
           "monc_proj_krylov_workspace_size")
    return n.value


def monc_proj_solve_krylov(plan: int, u, v, w, u_out, v_out, w_out, phi_out, workspace, tol, max_iter,
                           precond="line", stream=None):
    """BiCGStab projection of the plan's field type; returns (status, iterations,
    relative residual).  Status OK, MONC_PROJ_ENOCONV or MONC_PROJ_EBREAKDOWN
    is returned (the outputs are written in all three cases); any other
    status raises."""
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
    pc = PRECONDITIONERS[precond] if isinstance(precond, str) else int(precond)
    it, rr = ctypes.c_int(), ctypes.c_double()
    rc = load_library().monc_proj_solve_krylov(ctypes.c_void_p(plan), ptr(u), ptr(v), ptr(w), ptr(u_out),
                                               ptr(v_out), ptr(w_out), ptr(phi_out), ptr(workspace),
                                               float(tol), int(max_iter), pc, ctypes.byref(it), ctypes.byref(rr),
                                               ctypes.c_void_p(_stream_handle(stream)))
    if rc not in (MONC_PROJ_OK, MONC_PROJ_ENOCONV, MONC_PROJ_EBREAKDOWN):
        raise ProjError(rc, "monc_proj_solve_krylov")
    return rc, it.value, rr.value


def monc_proj_batch_workspace_size(plans) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    n = ctypes.c_size_t()
    _check(load_library().monc_proj_batch_workspace_size(arr, len(plans), ctypes.byref(n)),
           "monc_proj_batch_workspace_size")
    return n.value


def _batch_call(name, plans, fields, workspace, stream):
    n = len(plans)
    arr = (ctypes.c_void_p * n)(*plans)
    fa = (Fields * n)()
    for i, f in enumerate(fields):
        fa[i] = Fields(*[None if t is None else t.data_ptr() for t in f])
    rc = getattr(load_library(), name)(arr, fa, n, ctypes.c_void_p(workspace.data_ptr()),
                                       workspace.numel() * workspace.element_size(),
                                       ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, name)


def monc_proj_solve_batch(plans, fields, workspace, stream=None):
    """fields: list of (u, v, w, u_out, v_out, w_out, phi_out-or-None) tensors."""
    _batch_call("monc_proj_solve_batch", plans, fields, workspace, stream)


def monc_proj_solve_batch_grouped(plans, fields, workspace, stream=None):
    """As monc_proj_solve_batch, one launch per phase and group of instances."""
    _batch_call("monc_proj_solve_batch_grouped", plans, fields, workspace, stream)


def monc_proj_sync_status(plan: int, stream=None) -> int:
    return load_library().monc_proj_sync_status(ctypes.c_void_p(plan),
                                                ctypes.c_void_p(_stream_handle(stream)))


def monc_proj_destroy(plan: int):
    _check(load_library().monc_proj_destroy(ctypes.c_void_p(plan)), "monc_proj_destroy")


def monc_proj_plan_info(plan: int) -> dict:
    ints = [ctypes.c_int() for _ in range(4)]
    lls = [ctypes.c_longlong() for _ in range(2)]
    _check(load_library().monc_proj_plan_info(ctypes.c_void_p(plan), *[ctypes.byref(x) for x in ints],
                                              *[ctypes.byref(x) for x in lls]), "monc_proj_plan_info")
    return {"nx": ints[0].value, "ny": ints[1].value, "nz": ints[2].value,
            "precision": ints[3].value, "fp64_columns": lls[0].value, "total_columns": lls[1].value}


def monc_proj_plan_schedule(plan: int) -> dict:
    """Elements per thread (radix schedule) of the row and column plans and
    the task shapes."""
    vals = [ctypes.c_int() for _ in range(4)]
    _check(load_library().monc_proj_plan_schedule(ctypes.c_void_p(plan), *[ctypes.byref(v) for v in vals]),
           "monc_proj_plan_schedule")
    return dict(zip(("row_elems", "col_elems", "row_threads", "col_threads"), (v.value for v in vals)))


def monc_proj_set_schedule(plan: int, row_threads: int, col_threads: int, col_elems: int):
    """Set the task shapes and column radix schedule of an FP32 mixed plan."""
    _check(load_library().monc_proj_set_schedule(ctypes.c_void_p(plan), int(row_threads), int(col_threads),
                                                 int(col_elems)), "monc_proj_set_schedule")


def monc_proj_profile(plan: int, enable: bool):
    _check(load_library().monc_proj_profile(ctypes.c_void_p(plan), int(bool(enable))), "monc_proj_profile")


def monc_proj_phase_name(phase: int):
    r = load_library().monc_proj_phase_name(int(phase))
    return None if r is None else r.decode()


def monc_proj_profile_read(plan: int) -> dict:
    """Per-phase summed device time [ms] of the solves recorded since profiling began."""
    buf = (ctypes.c_double * 32)()
    nph = ctypes.c_int()
    ns = ctypes.c_int()
    _check(load_library().monc_proj_profile_read(ctypes.c_void_p(plan), 32, buf, ctypes.byref(nph),
                                                 ctypes.byref(ns)), "monc_proj_profile_read")
    return {"solves": ns.value,
            "phases": {monc_proj_phase_name(i): buf[i] for i in range(nph.value)}}


def monc_proj_solve_noalloc(nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision, u, v, w,
                            u_out, v_out, w_out, phi_out=None, stream=None):
    """One projection that allocates no device memory (static scratch in the library).

    For callers that cannot allocate device memory themselves or let a library
    do so; see the header for the size limit and the sharing rules."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
    rc = load_library().monc_proj_solve_noalloc(
        int(nx), int(ny), int(nz), float(dx), float(dy), _dbl(dz), _dbl(rho_c), _dbl(rho_f), prec,
        ptr(u), ptr(v), ptr(w), ptr(u_out), ptr(v_out), ptr(w_out), ptr(phi_out),
        ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_solve_noalloc")


_allocator_refs = None


def monc_proj_spectral_pitch(plan: int) -> int:
    """Row pitch (complex values) of the plan's spectral arrays."""
    n = ctypes.c_int()
    _check(load_library().monc_proj_spectral_pitch(ctypes.c_void_p(plan), ctypes.byref(n)),
           "monc_proj_spectral_pitch")
    return n.value


def _ptr(t):
    return ctypes.c_void_p(None if t is None else t.data_ptr())


def monc_proj_forward_slab(plan: int, k0, k1, u, v, w, dhat, workspace, stream=None):
    """Enqueue a1-a2 on levels [k0, k1): dhat receives the slab's spectrum."""
    rc = load_library().monc_proj_forward_slab(ctypes.c_void_p(plan), int(k0), int(k1), _ptr(u), _ptr(v),
                                               _ptr(w), _ptr(dhat), _ptr(workspace),
                                               ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_forward_slab")


def monc_proj_vertical_pencil(plan: int, j0, j1, spec, gz, workspace, stream=None):
    """Enqueue a3 on spectral rows [j0, j1): spec D^ -> p^ in place, gz^ out."""
    rc = load_library().monc_proj_vertical_pencil(ctypes.c_void_p(plan), int(j0), int(j1), _ptr(spec), _ptr(gz),
                                                  _ptr(workspace), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_vertical_pencil")


def monc_proj_inverse_slab(plan: int, k0, k1, phat, gz, u, v, w, u_out, v_out, w_out, workspace, stream=None):
    """Enqueue a4-a5 on levels [k0, k1)."""
    rc = load_library().monc_proj_inverse_slab(ctypes.c_void_p(plan), int(k0), int(k1), _ptr(phat), _ptr(gz),
                                               _ptr(u), _ptr(v), _ptr(w), _ptr(u_out), _ptr(v_out), _ptr(w_out),
                                               _ptr(workspace), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_inverse_slab")


def monc_proj_pack_pencils(plan: int, nzl, parts, slab, packed, stream=None):
    """Enqueue slab [nzl][ny][nxp] -> per-part row blocks (all-to-all send buffer)."""
    rc = load_library().monc_proj_pack_pencils(ctypes.c_void_p(plan), int(nzl), int(parts), _ptr(slab),
                                               _ptr(packed), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_pack_pencils")


def monc_proj_unpack_pencils(plan: int, nzl, parts, packed, slab, stream=None):
    """Enqueue per-part row blocks (all-to-all receive buffer) -> slab [nzl][ny][nxp]."""
    rc = load_library().monc_proj_unpack_pencils(ctypes.c_void_p(plan), int(nzl), int(parts), _ptr(packed),
                                                 _ptr(slab), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "monc_proj_unpack_pencils")


def monc_proj_set_allocator(alloc=None, release=None):
    """Install Python callables alloc(bytes) -> device pointer (int, 0 on
    failure) and release(ptr) as the allocator of plan tables; no arguments
    restore cudaMalloc / cudaFree.  The callbacks are kept alive here."""
    global _allocator_refs
    if alloc is None and release is None:
        rc = load_library().monc_proj_set_allocator(ALLOC_FN(), FREE_FN(), None)
        _allocator_refs = None
        _check(rc, "monc_proj_set_allocator")
        return
    a = ALLOC_FN(lambda n, user: int(alloc(int(n)) or 0))
    r = FREE_FN(lambda ptr, user: release(int(ptr or 0)))
    rc = load_library().monc_proj_set_allocator(a, r, None)
    _check(rc, "monc_proj_set_allocator")
    _allocator_refs = (a, r)


# ----------------------------------------------------------------- convenience

class Projector:
    """One plan plus its workspace on the current CUDA device."""

    def __init__(self, nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision="fp64", device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.plan = monc_proj_plan(nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision)
            self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
            self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
            self.dtype = DTYPES[self.precision]
            self.workspace_bytes = monc_proj_workspace_size(self.plan)
            self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=self.device)

    @classmethod
    def from_grid(cls, grid, precision="fp64", device=None):
        return cls(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.rho_c, grid.rho_f,
                   precision, device)

    def _check_field(self, t, shape, name):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype \
                or tuple(t.shape) != shape or not t.is_contiguous():
            raise ProjError(MONC_PROJ_EINVAL, f"field {name}: need contiguous {self.dtype} "
                                              f"{shape} on {self.device}")

    def solve(self, u, v, w, out=None, phi=False, stream=None):
        """Project (u, v, w); returns (u_out, v_out, w_out) or (..., phi)."""
        c = (self.nz, self.ny, self.nx)
        f = (self.nz + 1, self.ny, self.nx)
        self._check_field(u, c, "u")
        self._check_field(v, c, "v")
        self._check_field(w, f, "w")
        if out is None:
            out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        for t, s, n in zip(out, (c, c, f), ("u_out", "v_out", "w_out")):
            self._check_field(t, s, n)
        p = torch.empty(c, dtype=self.dtype, device=self.device) if phi is True else (phi or None)
        if p is not None:
            self._check_field(p, c, "phi")
        monc_proj_solve(self.plan, u, v, w, out[0], out[1], out[2], p, self.workspace, stream)
        return (*out, p) if p is not None else tuple(out)

    def solve_host(self, u, v, w, out, staging=None, workspace=None, stream=None):
        """Project host tensors (page-locked for asynchronous copies) into the
        host tensors `out` through a device staging buffer (allocated here
        if not given); returns out.  Enqueued on `stream`."""
        if staging is None:
            staging = torch.empty(max(monc_proj_host_staging_size(self.plan), 256), dtype=torch.uint8,
                                  device=self.device)
        ws = self.workspace if workspace is None else workspace
        monc_proj_solve_host(self.plan, u, v, w, out[0], out[1], out[2], None, staging, ws, stream)
        return out

    def solve_krylov(self, u, v, w, tol=1e-4, max_iter=1000, precond="line", out=None, phi=False,
                     workspace=None, stream=None):
        """Project (u, v, w) with the BiCGStab pressure solver (FP32 vectors
        for mixed plans, FP64 otherwise); returns (u_out, v_out, w_out, phi or None, status, iterations,
        relative residual).  The Krylov workspace is allocated here unless
        given."""
        c = (self.nz, self.ny, self.nx)
        f = (self.nz + 1, self.ny, self.nx)
        self._check_field(u, c, "u")
        self._check_field(v, c, "v")
        self._check_field(w, f, "w")
        if out is None:
            out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        for t, s, n in zip(out, (c, c, f), ("u_out", "v_out", "w_out")):
            self._check_field(t, s, n)
        p = torch.empty(c, dtype=self.dtype, device=self.device) if phi is True else (phi or None)
        if p is not None:
            self._check_field(p, c, "phi")
        if workspace is None:
            workspace = torch.empty(max(monc_proj_krylov_workspace_size(self.plan), 256), dtype=torch.uint8,
                                    device=self.device)
        st, it, rr = monc_proj_solve_krylov(self.plan, u, v, w, out[0], out[1], out[2], p, workspace, tol,
                                            max_iter, precond, stream)
        return (*out, p, st, it, rr)

    def autotune(self, u, v, w, reps=3, stream=None):
        """Pick the plan's task shapes by timing them on (u, v, w), which
        are left unchanged; returns (row_threads, col_threads)."""
        out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        return monc_proj_autotune(self.plan, u, v, w, *out, self.workspace, reps, stream)

    def sync_status(self, stream=None) -> int:
        return monc_proj_sync_status(self.plan, stream)

    def info(self) -> dict:
        return monc_proj_plan_info(self.plan)

    def close(self):
        if getattr(self, "plan", None):
            monc_proj_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A plan handle without a workspace (for batched and served solves)."""

    def __init__(self, grid, precision="mixed", device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.handle = monc_proj_plan(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.rho_c,
                                         grid.rho_f, precision)
        self.grid = grid
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dtype = DTYPES[self.precision]
        self.workspace_bytes = monc_proj_workspace_size(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            monc_proj_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchProjector:
    """Uneven batch of independent projections, solved together by
    monc_proj_solve_batch (the instances run concurrently on the device)."""

    def __init__(self, grids, precision="mixed", device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.plans = [Plan(g, precision, self.device) for g in grids]
            self.workspace_bytes = monc_proj_batch_workspace_size([p.handle for p in self.plans])
            self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=self.device)

    def solve(self, fields, stream=None, grouped=False):
        """fields: list of (u, v, w, u_out, v_out, w_out) or (..., phi_out)
        tensors.  grouped: one launch per phase and group of instances
        (monc_proj_solve_batch_grouped) instead of per-instance launches."""
        if len(fields) != len(self.plans):
            raise ProjError(MONC_PROJ_EINVAL, "BatchProjector.solve")
        full = [tuple(f) + (None,) * (7 - len(f)) for f in fields]
        fn = monc_proj_solve_batch_grouped if grouped else monc_proj_solve_batch
        fn([p.handle for p in self.plans], full, self.workspace, stream)

    def autotune(self, fields, reps=3, stream=None):
        """Tune each instance's plan alone on its fields (inputs left
        unchanged); returns the (row_threads, col_threads) kept per plan."""
        out = []
        for p, f in zip(self.plans, fields):
            u, v, w = f[0], f[1], f[2]
            tmp = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
            out.append(monc_proj_autotune(p.handle, u, v, w, *tmp, self.workspace, reps, stream))
        return out

    def close(self):
        for p in self.plans:
            p.close()
