"""GB300 (sm_103a) solver for the variable-density pressure Poisson equation div((1/rho) grad p) = f
on a triply periodic staggered grid (Sec. 3.4 of Pouransari, Mortazavi & Mani, arXiv:1601.05448).

This package is a thin ctypes binding over ``libvdp.so`` (built from ``csrc/`` by ``build.py``);
the functions keep the C names of ``include/vdp.h`` and only marshal arguments.  Every step of
the solve runs in the library's CUDA kernels; there is no Python or CPU fallback -- importing
works without the library, but any call raises ``VdpUnavailable`` if ``libvdp.so`` is missing.

Arrays are float64, contiguous, shape (nz, ny, nx) (x fastest): torch CUDA tensors (device
pointers), or torch CPU tensors / numpy arrays (host pointers, staged by the library).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvdp.so")

VDP_OK, VDP_EINVAL, VDP_ENOMEM, VDP_EDENSITY, VDP_ENOTCONV, VDP_EBREAKDOWN, VDP_ETIMEOUT, VDP_ECUDA = range(8)
VDP_FP64, VDP_MIXED, VDP_MIXED_BF16 = 0, 1, 2
VDP_PRECOND_JACOBI, VDP_PRECOND_CHEB, VDP_PRECOND_SPECTRAL, VDP_PRECOND_MG = 0, 1, 2, 3
VDP_METHOD_CG, VDP_METHOD_FIXED_POINT = 0, 1
VDP_BC_PERIODIC, VDP_BC_DUCT = 0, 1
PRECISIONS = {"fp64": VDP_FP64, "mixed": VDP_MIXED, "mixed_bf16": VDP_MIXED_BF16}
# grid sizes (per direction) the spectral preconditioner's FFT passes support
SPECTRAL_SIZES = (32, 48, 64, 96, 128, 192, 256, 512)


def spectral_supported(nx: int, ny: int, nz: int) -> bool:
    return all(n in SPECTRAL_SIZES for n in (nx, ny, nz))


def spectral_extra_bytes(nx: int, ny: int, nz: int) -> int:
    """Device memory the spectral passes add to a context: z (8 B/cell), the weights (4 B/cell,
    4 more for the fixed-point iteration's density weight) and the half spectrum (8 B per
    complex value, rows padded to 8 values)."""
    nxp = ((nx // 2 + 1 + 7) // 8) * 8
    return 16 * nx * ny * nz + 8 * nxp * ny * nz


class VdpUnavailable(RuntimeError):
    """libvdp.so is not built (run __graft_entry__.build() or paper_1601_05448_gb300.build)."""


class VdpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {vdp_strerror(status)}"
        if status == VDP_ECUDA:
            msg += f" ({vdp_last_cuda_error()})"
        super().__init__(msg)


class vdp_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("precond", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("use_guess", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("stencil", ctypes.c_int), ("tile_y", ctypes.c_int), ("units", ctypes.c_int),
                ("stages", ctypes.c_int), ("threads", ctypes.c_int), ("steps_per_sync", ctypes.c_int),
                ("method", ctypes.c_int), ("damping", ctypes.c_double), ("spec_slab", ctypes.c_int)]


class vdp_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("rhs_mean", ctypes.c_double), ("ms", ctypes.c_double),
                ("sweeps", ctypes.c_int), ("launches", ctypes.c_int)]


(VDP_SWEEP_RES64, VDP_SWEEP_STENCIL, VDP_SWEEP_CHEB, VDP_SWEEP_UPDATE, VDP_SWEEP_OTHER, VDP_SWEEP_SPEC_X,
 VDP_SWEEP_SPEC_Y, VDP_SWEEP_SPEC_Z, VDP_SWEEP_MG, VDP_SWEEP_KINDS) = range(10)
SWEEP_NAMES = ("res64", "stencil", "cheb", "update", "other", "spec_x", "spec_y", "spec_z", "mg")


class vdp_sweep_times(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int * VDP_SWEEP_KINDS), ("ms", ctypes.c_double * VDP_SWEEP_KINDS),
                ("ms_min", ctypes.c_double * VDP_SWEEP_KINDS)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes) of every entry point declared in include/vdp.h
_P = ctypes.c_void_p
_SIGS = {
    "vdp_default_options": (None, [ctypes.POINTER(vdp_opts)]),
    "vdp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "vdp_set_options": (ctypes.c_int, [_P, ctypes.POINTER(vdp_opts)]),
    "vdp_get_options": (ctypes.c_int, [_P, ctypes.POINTER(vdp_opts)]),
    "vdp_create_bc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "vdp_set_density": (ctypes.c_int, [_P, _P]),
    "vdp_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "vdp_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(vdp_stats)]),
    "vdp_destroy": (None, [_P]),
    "vdp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vdp_last_cuda_error": (ctypes.c_char_p, []),
    "vdp_version": (ctypes.c_int, []),
    "vdp_apply": (ctypes.c_int, [_P, _P, _P]),
    "vdp_inverse_laplacian": (ctypes.c_int, [_P, _P, _P]),
    "vdp_mg_levels": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "vdp_mg_apply": (ctypes.c_int, [_P, _P, _P]),
    "vdp_projection_rhs": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double, _P]),
    "vdp_projection_correct": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P]),
    "vdp_project": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double, _P]),
    "vdp_project_timed": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double, _P,
                                         ctypes.POINTER(ctypes.c_float)]),
    "vdp_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "vdp_batch_destroy": (None, [_P]),
    "vdp_batch_add": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double]),
    "vdp_batch_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "vdp_batch_done": (ctypes.c_int, [_P, _P]),
    "vdp_batch_remove": (ctypes.c_int, [_P, _P]),
    "vdp_batch_size": (ctypes.c_int, [_P]),
    "vdp_batch_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_double]),
    "vdp_batch_inject_lost_arrival": (ctypes.c_int, [_P]),
    "vdp_solve_timed": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.POINTER(vdp_sweep_times)]),
    "vdp_spectral_slabs": (ctypes.c_int, [_P]),
    "vdp_probe_fp64": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "vdp_solve_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P,
                                         ctypes.c_double, ctypes.c_int, _P, ctypes.POINTER(vdp_stats)]),
}
VDP_NOALLOC_MAX_CELLS = 65536


def exported_symbols():
    """Names of the C entry points this binding expects (those declared in include/vdp.h)."""
    return list(_SIGS)


def load(path: str = LIB_PATH):
    """Load libvdp.so (no build); raises VdpUnavailable when it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise VdpUnavailable(f"{path} not found: build it with paper_1601_05448_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


# ---- the C entry points, same names -------------------------------------------------------------

def vdp_default_options() -> vdp_opts:
    o = vdp_opts()
    load().vdp_default_options(ctypes.byref(o))
    return o


def vdp_create(nx: int, ny: int, nz: int, L: float) -> int:
    h = ctypes.c_void_p()
    st = load().vdp_create(int(nx), int(ny), int(nz), float(L), ctypes.byref(h))
    if st != VDP_OK:
        raise VdpError(st, "vdp_create")
    return h.value


def vdp_create_bc(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float, bc_x: int) -> int:
    h = ctypes.c_void_p()
    st = load().vdp_create_bc(int(nx), int(ny), int(nz), float(Lx), float(Ly), float(Lz), int(bc_x),
                              ctypes.byref(h))
    if st != VDP_OK:
        raise VdpError(st, "vdp_create_bc")
    return h.value


def vdp_set_options(ctx: int, opts: vdp_opts) -> int:
    return load().vdp_set_options(ctx, ctypes.byref(opts))


def vdp_get_options(ctx: int) -> vdp_opts:
    o = vdp_opts()
    st = load().vdp_get_options(ctx, ctypes.byref(o))
    if st != VDP_OK:
        raise VdpError(st, "vdp_get_options")
    return o


def vdp_set_density(ctx: int, rho) -> int:
    return load().vdp_set_density(ctx, _ptr(rho))


def vdp_solve(ctx: int, rhs, p, tol: float) -> int:
    return load().vdp_solve(ctx, _ptr(rhs), _ptr(p, writable=True), float(tol))


def vdp_get_stats(ctx: int) -> vdp_stats:
    s = vdp_stats()
    load().vdp_get_stats(ctx, ctypes.byref(s))
    return s


def vdp_destroy(ctx) -> None:
    if ctx:
        load().vdp_destroy(ctx)


def vdp_strerror(status: int) -> str:
    return load().vdp_strerror(int(status)).decode()


def vdp_last_cuda_error() -> str:
    return load().vdp_last_cuda_error().decode()


def vdp_version() -> int:
    return load().vdp_version()


def vdp_apply(ctx: int, p, out) -> int:
    return load().vdp_apply(ctx, _ptr(p), _ptr(out, writable=True))


def vdp_inverse_laplacian(ctx: int, g, out) -> int:
    return load().vdp_inverse_laplacian(ctx, _ptr(g), _ptr(out, writable=True))


def vdp_mg_levels(nx: int, ny: int, nz: int) -> int:
    return load().vdp_mg_levels(nx, ny, nz)


def vdp_mg_apply(ctx: int, g, out) -> int:
    return load().vdp_mg_apply(ctx, _ptr(g), _ptr(out, writable=True))


def _opt_ptr(a):
    return None if a is None else _ptr(a)


def vdp_projection_rhs(ctx: int, mx, my, mz, rhs_div, c: float, f) -> int:
    return load().vdp_projection_rhs(ctx, _ptr(mx), _ptr(my), _ptr(mz), _opt_ptr(rhs_div), float(c),
                                     _ptr(f, writable=True))


def vdp_projection_correct(ctx: int, p, c: float, mx, my, mz) -> int:
    return load().vdp_projection_correct(ctx, _ptr(p), float(c), _ptr(mx, writable=True),
                                         _ptr(my, writable=True), _ptr(mz, writable=True))


def vdp_project(ctx: int, mx, my, mz, rhs_div, c: float, tol: float, p) -> int:
    return load().vdp_project(ctx, _ptr(mx, writable=True), _ptr(my, writable=True), _ptr(mz, writable=True),
                              _opt_ptr(rhs_div), float(c), float(tol), _ptr(p, writable=True))


def vdp_project_timed(ctx: int, mx, my, mz, rhs_div, c: float, tol: float, p):
    """vdp_project with its kernels timed; returns (status, (rhs_ms, solve_ms, correct_ms))."""
    ms = (ctypes.c_float * 3)()
    st = load().vdp_project_timed(ctx, _ptr(mx, writable=True), _ptr(my, writable=True),
                                  _ptr(mz, writable=True), _opt_ptr(rhs_div), float(c), float(tol),
                                  _ptr(p, writable=True), ms)
    return st, (ms[0], ms[1], ms[2])


def vdp_solve_timed(ctx: int, rhs, p, tol: float):
    """vdp_solve with each kernel launch timed alone; returns (status, vdp_sweep_times)."""
    t = vdp_sweep_times()
    st = load().vdp_solve_timed(ctx, _ptr(rhs), _ptr(p, writable=True), float(tol), ctypes.byref(t))
    return st, t


def vdp_solve_noalloc(nx: int, ny: int, nz: int, L: float, rho, rhs, p, tol: float, precision: int = VDP_FP64,
                      stream=None):
    """Solve without any device allocation (device tensors of the current device only,
    nx*ny*nz <= VDP_NOALLOC_MAX_CELLS).

    For callers that cannot allocate device memory: hosts whose GPU memory is reserved by a pool
    or budget manager that forbids side allocations, and latency-critical loops that cannot take
    the device-wide synchronisation of cudaMalloc/cudaFree.  Intermediates live in a fixed device
    array owned by the library; calls share it, so do not run two at once.  Returns (status,
    stats); arrays of the wrong size raise ValueError before the C call."""
    n = int(nx) * int(ny) * int(nz)
    for a, name in ((rho, "rho"), (rhs, "rhs"), (p, "p")):
        if _numel(a) != n:
            raise ValueError(f"{name}: expected {n} elements, got {_numel(a)}")
    s = vdp_stats()
    st = load().vdp_solve_noalloc(int(nx), int(ny), int(nz), float(L), _ptr(rho), _ptr(rhs),
                                  _ptr(p, writable=True), float(tol), int(precision),
                                  stream if (stream is None or isinstance(stream, int)) else stream.cuda_stream,
                                  ctypes.byref(s))
    return st, s


def vdp_spectral_slabs(ctx: int) -> int:
    return load().vdp_spectral_slabs(ctx)


def vdp_probe_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s (see include/vdp.h)."""
    t = ctypes.c_double(0.0)
    st = load().vdp_probe_fp64(_stream(stream), ctypes.byref(t))
    if st != VDP_OK:
        raise VdpError(st, "vdp_probe_fp64")
    return t.value


def vdp_batch_create(precision: int = VDP_MIXED, persistent: int = 1, stream=None) -> int:
    h = ctypes.c_void_p()
    st = load().vdp_batch_create(int(precision), int(persistent), _stream(stream), ctypes.byref(h))
    if st != VDP_OK:
        raise VdpError(st, "vdp_batch_create")
    return h.value


def vdp_batch_destroy(batch) -> None:
    if batch:
        load().vdp_batch_destroy(batch)


def vdp_batch_add(batch: int, ctx: int, rhs, p, tol: float) -> int:
    return load().vdp_batch_add(batch, ctx, _ptr(rhs), _ptr(p, writable=True), float(tol))


def vdp_batch_run(batch: int, max_pairs: int):
    active = ctypes.c_int(0)
    st = load().vdp_batch_run(batch, int(max_pairs), ctypes.byref(active))
    return st, active.value


def vdp_batch_done(batch: int, ctx: int) -> int:
    return load().vdp_batch_done(batch, ctx)


def vdp_batch_remove(batch: int, ctx: int) -> int:
    return load().vdp_batch_remove(batch, ctx)


def vdp_batch_size(batch: int) -> int:
    return load().vdp_batch_size(batch)


def vdp_batch_set_wait_limit(batch: int, seconds: float) -> int:
    return load().vdp_batch_set_wait_limit(batch, float(seconds))


def vdp_batch_inject_lost_arrival(batch: int) -> int:
    return load().vdp_batch_inject_lost_arrival(batch)


def _stream(stream):
    if stream is None or isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- marshalling ------------------------------------------------------------------------------

def _ptr(a, writable: bool = False) -> int:
    """Data pointer of a contiguous float64 torch tensor (CUDA or CPU) or numpy array."""
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a contiguous float64 numpy array")
    if writable and not a.flags["WRITEABLE"]:
        raise TypeError("output array is read-only")
    return a.ctypes.data


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


@dataclass
class Stats:
    status: int
    iters: int
    outer_iters: int
    rel_res: float
    rhs_mean: float
    ms: float
    sweeps: int
    launches: int

    @property
    def ok(self) -> bool:
        return self.status == VDP_OK


class Solver:
    """Owns one vdp context: ``Solver(nx, ny, nz, L, precision="fp64")``; ``set_density(rho)``;
    ``solve(rhs, p, tol) -> Stats``.  Raises VdpError on any status other than OK (and, for
    solve, other than ENOTCONV/EBREAKDOWN when ``check=False``)."""

    def __init__(self, nx: int, ny: int, nz: int, L: float, precision: str = "fp64", stream=None,
                 lengths=None, bc_x: int = VDP_BC_PERIODIC, **opts):
        """L: side of the cube; lengths = (Lx, Ly, Lz) instead, and bc_x = VDP_BC_DUCT for the
        inflow-outflow duct (no pressure flux through the x ends)."""
        self.shape = (nz, ny, nx)
        self.L = float(L)
        if lengths is None and bc_x == VDP_BC_PERIODIC:
            self.ctx = vdp_create(nx, ny, nz, L)
        else:
            Lx, Ly, Lz = lengths if lengths is not None else (L, L, L)
            self.ctx = vdp_create_bc(nx, ny, nz, Lx, Ly, Lz, bc_x)
        o = vdp_default_options()
        o.precision = PRECISIONS[precision]
        if stream is not None:
            o.stream = stream if isinstance(stream, int) else stream.cuda_stream
        for k, v in opts.items():
            setattr(o, k, v)
        st = vdp_set_options(self.ctx, o)
        if st != VDP_OK:
            self.close()
            raise VdpError(st, "vdp_set_options")

    @property
    def n(self) -> int:
        nz, ny, nx = self.shape
        return nx * ny * nz

    def options(self) -> vdp_opts:
        return vdp_get_options(self.ctx)

    def set_options(self, **kw) -> None:
        o = vdp_get_options(self.ctx)
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            setattr(o, k, v)
        st = vdp_set_options(self.ctx, o)
        if st != VDP_OK:
            raise VdpError(st, "vdp_set_options")

    def _check(self, a, name):
        if _numel(a) != self.n:
            raise ValueError(f"{name}: expected {self.n} elements, got {_numel(a)}")

    def set_density(self, rho) -> None:
        self._check(rho, "rho")
        st = vdp_set_density(self.ctx, rho)
        if st != VDP_OK:
            raise VdpError(st, "vdp_set_density")

    def stats(self) -> Stats:
        s = vdp_get_stats(self.ctx)
        return Stats(s.status, s.iters, s.outer_iters, s.rel_res, s.rhs_mean, s.ms, s.sweeps, s.launches)

    def solve(self, rhs, p, tol: float, check: bool = True) -> Stats:
        self._check(rhs, "rhs")
        self._check(p, "p")
        st = vdp_solve(self.ctx, rhs, p, tol)
        s = vdp_get_stats(self.ctx)
        out = Stats(s.status, s.iters, s.outer_iters, s.rel_res, s.rhs_mean, s.ms, s.sweeps, s.launches)
        if st != VDP_OK and (check or st not in (VDP_ENOTCONV, VDP_EBREAKDOWN)):
            raise VdpError(st, "vdp_solve")
        return out

    def solve_timed(self, rhs, p, tol: float, check: bool = True):
        """The solve with every kernel launch timed on its own (device tensors).  Returns
        (Stats, {kind: {"launches", "ms", "ms_min", "ms_mean"}}) with kind in SWEEP_NAMES."""
        self._check(rhs, "rhs")
        self._check(p, "p")
        st, t = vdp_solve_timed(self.ctx, rhs, p, tol)
        s = vdp_get_stats(self.ctx)
        out = Stats(s.status, s.iters, s.outer_iters, s.rel_res, s.rhs_mean, s.ms, s.sweeps, s.launches)
        if st != VDP_OK and (check or st not in (VDP_ENOTCONV, VDP_EBREAKDOWN)):
            raise VdpError(st, "vdp_solve_timed")
        kinds = {}
        for i, name in enumerate(SWEEP_NAMES):
            n = t.launches[i]
            kinds[name] = {"launches": n, "ms": t.ms[i], "ms_min": t.ms_min[i],
                           "ms_mean": t.ms[i] / n if n else 0.0}
        return out, kinds

    def spectral_slabs(self) -> int:
        """Slabs the spectral passes run in (1: the whole grid at once; 0: no spectral passes)."""
        return vdp_spectral_slabs(self.ctx)

    def inverse_laplacian(self, g, out) -> None:
        """out = L_h^-1 g, the constant-coefficient periodic solve (device tensors)."""
        self._check(g, "g")
        self._check(out, "out")
        st = vdp_inverse_laplacian(self.ctx, g, out)
        if st != VDP_OK:
            raise VdpError(st, "vdp_inverse_laplacian")

    def mg_apply(self, g, out) -> None:
        """out = one multigrid V-cycle applied to g (approximately (-A)^-1 g; device tensors)."""
        self._check(g, "g")
        self._check(out, "out")
        st = vdp_mg_apply(self.ctx, g, out)
        if st != VDP_OK:
            raise VdpError(st, "vdp_mg_apply")

    def projection_rhs(self, m, rhs_div, c: float, f) -> None:
        """f = (div(m / rho_face) - rhs_div) / c (App. A); m = (mx, my, mz) face momenta on the
        low faces, rhs_div may be None (device tensors)."""
        for a, name in zip((*m, f), ("mx", "my", "mz", "f")):
            self._check(a, name)
        if rhs_div is not None:
            self._check(rhs_div, "rhs_div")
        st = vdp_projection_rhs(self.ctx, *m, rhs_div, c, f)
        if st != VDP_OK:
            raise VdpError(st, "vdp_projection_rhs")

    def projection_correct(self, p, c: float, m) -> None:
        """Eq. (mom): m -= c grad p on the low faces, in place (device tensors)."""
        for a, name in zip((p, *m), ("p", "mx", "my", "mz")):
            self._check(a, name)
        st = vdp_projection_correct(self.ctx, p, c, *m)
        if st != VDP_OK:
            raise VdpError(st, "vdp_projection_correct")

    def project(self, m, rhs_div, c: float, tol: float, p, check: bool = True) -> Stats:
        """One projection (App. A): right side, solve into p, momentum correction of m in place."""
        for a, name in zip((p, *m), ("p", "mx", "my", "mz")):
            self._check(a, name)
        if rhs_div is not None:
            self._check(rhs_div, "rhs_div")
        st = vdp_project(self.ctx, *m, rhs_div, c, tol, p)
        s = vdp_get_stats(self.ctx)
        out = Stats(s.status, s.iters, s.outer_iters, s.rel_res, s.rhs_mean, s.ms, s.sweeps, s.launches)
        if st != VDP_OK and (check or st not in (VDP_ENOTCONV, VDP_EBREAKDOWN)):
            raise VdpError(st, "vdp_project")
        return out

    def project_timed(self, m, rhs_div, c: float, tol: float, p, check: bool = True):
        """project() with its kernels timed: (Stats, {"rhs_ms", "solve_ms", "correct_ms"})."""
        for a, name in zip((p, *m), ("p", "mx", "my", "mz")):
            self._check(a, name)
        if rhs_div is not None:
            self._check(rhs_div, "rhs_div")
        st, ms = vdp_project_timed(self.ctx, *m, rhs_div, c, tol, p)
        s = vdp_get_stats(self.ctx)
        out = Stats(s.status, s.iters, s.outer_iters, s.rel_res, s.rhs_mean, s.ms, s.sweeps, s.launches)
        if st != VDP_OK and (check or st not in (VDP_ENOTCONV, VDP_EBREAKDOWN)):
            raise VdpError(st, "vdp_project_timed")
        return out, {"rhs_ms": ms[0], "solve_ms": ms[1], "correct_ms": ms[2]}

    def apply(self, p, out) -> None:
        self._check(p, "p")
        self._check(out, "out")
        st = vdp_apply(self.ctx, p, out)
        if st != VDP_OK:
            raise VdpError(st, "vdp_apply")

    def close(self) -> None:
        if getattr(self, "ctx", None):
            vdp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Continuous batch of solves: ``add(solver, rhs, p, tol)``; ``run(max_pairs) -> active``;
    ``done(solver)``; ``remove(solver)``.  All member solvers must use the batch's precision."""

    def __init__(self, precision: str = "mixed", persistent: bool = True, stream=None):
        self.precision = PRECISIONS[precision]
        self.handle = vdp_batch_create(self.precision, 1 if persistent else 0, stream)
        self._keep = {}

    def add(self, solver: "Solver", rhs, p, tol: float) -> None:
        solver._check(rhs, "rhs")
        solver._check(p, "p")
        st = vdp_batch_add(self.handle, solver.ctx, rhs, p, tol)
        if st != VDP_OK:
            raise VdpError(st, "vdp_batch_add")
        self._keep[solver.ctx] = (solver, rhs, p)

    def run(self, max_pairs: int = 64) -> int:
        st, active = vdp_batch_run(self.handle, max_pairs)
        if st != VDP_OK:
            raise VdpError(st, "vdp_batch_run")
        return active

    def done(self, solver: "Solver") -> bool:
        r = vdp_batch_done(self.handle, solver.ctx)
        if r < 0:
            raise VdpError(-r, "vdp_batch_done")
        return r == 1

    def remove(self, solver: "Solver") -> None:
        st = vdp_batch_remove(self.handle, solver.ctx)
        if st != VDP_OK:
            raise VdpError(st, "vdp_batch_remove")
        self._keep.pop(solver.ctx, None)

    def __len__(self):
        return vdp_batch_size(self.handle)

    def set_wait_limit(self, seconds: float) -> None:
        """Bound on each grid-barrier wait of the persistent kernel (an expired wait raises
        VdpError(VDP_ETIMEOUT) from run(); the members stay usable)."""
        st = vdp_batch_set_wait_limit(self.handle, seconds)
        if st != VDP_OK:
            raise VdpError(st, "vdp_batch_set_wait_limit")

    def inject_lost_arrival(self) -> None:
        """Failure injection for tests: the next persistent run waits for a block that never
        arrives, so its bounded grid-barrier wait expires."""
        st = vdp_batch_inject_lost_arrival(self.handle)
        if st != VDP_OK:
            raise VdpError(st, "vdp_batch_inject_lost_arrival")

    def run_to_completion(self, max_pairs: int = 64, max_runs: int = 100000) -> None:
        for _ in range(max_runs):
            if self.run(max_pairs) == 0:
                return
        raise VdpError(VDP_ENOTCONV, "Batch.run_to_completion")

    def close(self) -> None:
        if getattr(self, "handle", None):
            vdp_batch_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
