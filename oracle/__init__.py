"""CPU oracle for the variable-coefficient pressure Poisson solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It wraps ``vdp_oracle.c`` (plain FP64 C + OpenMP, built here with gcc into
``liboracle.so``) with numpy arrays.  It shares no code with the GPU library and never calls it.

What it computes (Pouransari, Mortazavi & Mani, arXiv:1601.05448):
  * ``face_coefficients``: 1/rho on every cell face from the arithmetic mean of the two adjacent
    cell-centre densities (the averaging App. B uses), times 1/h^2 (Sec. 3.1 staggered grid).
  * ``apply``: the conservative 7-point discretisation of div((1/rho) grad p) (Sec. 3.4).
  * ``solve_cg``: the discrete problem A p = f - <f>, <p> = 0 (compatibility constant chi' of
    App. A), by Jacobi-preconditioned conjugate gradients, stopped on the recomputed true
    residual.
  * ``solve_fixed_point``: the paper's own iteration of Eq. (Pois) (Sec. 3.4), with the
    constant-coefficient inverse applied through a plain DFT; an independent second solver.
  * ``geom=(Lx, Ly, Lz, bc_x)`` on the functions above: per-direction box lengths and, with
    bc_x = 1, the inflow-outflow duct of Sec. 3.2 (periodic y, z; no pressure flux through the x
    ends -- a reading, the paper does not state the pressure condition), whose constant-
    coefficient inverse uses a plain cosine transform along x.

  * ``projection_rhs`` / ``projection_correct`` / ``project``: the steps either side of the solve
    in App. A -- the Poisson right side (div((rho u)~ / rho_new) - RHS^div) / (C_pre dt) and the
    momentum correction (rho u)_new = (rho u)~ - C_pre dt grad p of Eq. (mom) -- on face momenta
    stored on the low face of each cell; ``divergence`` and ``face_velocity`` are their parts.

Arrays are numpy float64 of shape (nz, ny, nx) (C order, x fastest).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vdp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "einval", 2: "enomem", 3: "edensity", 4: "enotconv", 5: "ebreakdown"}


def build(force: bool = False) -> str:
    """Compile vdp_oracle.c into liboracle.so (gcc, FP64, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d = ctypes.c_double
            i = ctypes.c_int
            pd = ctypes.POINTER(ctypes.c_double)
            lib.vdpo_sum.argtypes = [i, i, i, pd]
            lib.vdpo_sum.restype = d
            lib.vdpo_dot.argtypes = [i, i, i, pd, pd]
            lib.vdpo_dot.restype = d
            lib.vdpo_mean.argtypes = [i, i, i, pd]
            lib.vdpo_mean.restype = d
            lib.vdpo_face_coefficients.argtypes = [i, i, i, d, pd, pd, pd, pd]
            lib.vdpo_face_coefficients.restype = i
            lib.vdpo_apply.argtypes = [i, i, i, pd, pd, pd, pd, pd]
            lib.vdpo_apply.restype = None
            lib.vdpo_relative_residual.argtypes = [i, i, i, d, pd, pd, pd]
            lib.vdpo_relative_residual.restype = d
            lib.vdpo_solve_cg.argtypes = [i, i, i, d, pd, pd, pd, d, i, pd]
            lib.vdpo_solve_cg.restype = i
            lib.vdpo_inverse_laplacian.argtypes = [i, i, i, d, pd, pd]
            lib.vdpo_inverse_laplacian.restype = None
            lib.vdpo_solve_fixed_point.argtypes = [i, i, i, d, pd, pd, pd, d, i, d, pd]
            lib.vdpo_solve_fixed_point.restype = i
            lib.vdpo_face_coefficients_g.argtypes = [i, i, i, d, d, d, i, pd, pd, pd, pd]
            lib.vdpo_face_coefficients_g.restype = i
            lib.vdpo_relative_residual_g.argtypes = [i, i, i, d, d, d, i, pd, pd, pd]
            lib.vdpo_relative_residual_g.restype = d
            lib.vdpo_solve_cg_g.argtypes = [i, i, i, d, d, d, i, pd, pd, pd, d, i, pd]
            lib.vdpo_solve_cg_g.restype = i
            lib.vdpo_inverse_laplacian_g.argtypes = [i, i, i, d, d, d, i, pd, pd]
            lib.vdpo_inverse_laplacian_g.restype = None
            lib.vdpo_solve_fixed_point_g.argtypes = [i, i, i, d, d, d, i, pd, pd, pd, d, i, d, pd]
            lib.vdpo_solve_fixed_point_g.restype = i
            lib.vdpo_divergence.argtypes = [i, i, i, d, pd, pd, pd, pd]
            lib.vdpo_divergence.restype = None
            lib.vdpo_face_velocity.argtypes = [i, i, i, pd, pd, pd, pd, pd, pd, pd]
            lib.vdpo_face_velocity.restype = i
            lib.vdpo_projection_rhs.argtypes = [i, i, i, d, pd, pd, pd, pd, pd, d, pd]
            lib.vdpo_projection_rhs.restype = i
            lib.vdpo_projection_correct.argtypes = [i, i, i, d, pd, d, pd, pd, pd, pd, pd, pd]
            lib.vdpo_projection_correct.restype = i
            lib.vdpo_num_threads.argtypes = []
            lib.vdpo_num_threads.restype = i
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(a: np.ndarray):
    nz, ny, nx = a.shape
    return nx, ny, nz


def num_threads() -> int:
    return _load().vdpo_num_threads()


def mean(x) -> float:
    x = _f64(x)
    return _load().vdpo_mean(*_dims(x), _ptr(x))


def dot(x, y) -> float:
    x, y = _f64(x), _f64(y)
    return _load().vdpo_dot(*_dims(x), _ptr(x), _ptr(y))


def _geom(L, geom):
    """(Lx, Ly, Lz, bc_x): the cube of side L (periodic) unless geom is given."""
    if geom is None:
        return float(L), float(L), float(L), 0
    Lx, Ly, Lz, bc_x = geom
    return float(Lx), float(Ly), float(Lz), int(bc_x)


def face_coefficients(rho, L: float, geom=None):
    """(bx, by, bz): coefficient of the low face of every cell, 1/rho_face/h^2.  geom = (Lx, Ly,
    Lz, bc_x) selects per-direction lengths and, with bc_x = 1, the inflow-outflow duct (no flux
    through the x ends: bx = 0 on the faces of cells i = 0)."""
    rho = _f64(rho)
    bx, by, bz = (np.empty_like(rho) for _ in range(3))
    st = _load().vdpo_face_coefficients_g(*_dims(rho), *_geom(L, geom), _ptr(rho), _ptr(bx), _ptr(by), _ptr(bz))
    if st != 0:
        raise ValueError(f"face_coefficients: {STATUS.get(st, st)}")
    return bx, by, bz


def apply(b, p) -> np.ndarray:
    """A p for face coefficients b = (bx, by, bz)."""
    bx, by, bz = (_f64(x) for x in b)
    p = _f64(p)
    out = np.empty_like(p)
    _load().vdpo_apply(*_dims(p), _ptr(bx), _ptr(by), _ptr(bz), _ptr(p), _ptr(out))
    return out


def apply_rho(rho, L: float, p, geom=None) -> np.ndarray:
    return apply(face_coefficients(rho, L, geom), p)


def relative_residual(rho, L: float, f, p, geom=None) -> float:
    """||(f - <f>) - A p||_2 / ||f - <f>||_2 evaluated with the oracle's operator."""
    rho, f, p = _f64(rho), _f64(f), _f64(p)
    return _load().vdpo_relative_residual_g(*_dims(rho), *_geom(L, geom), _ptr(rho), _ptr(f), _ptr(p))


def solve_cg(rho, f, L: float, tol: float = 1e-13, maxit: int = 100000, geom=None):
    """Zero-mean p with A p = f - <f>; returns (p, info) with info keys iters, rel_res, rhs_mean, status."""
    rho, f = _f64(rho), _f64(f)
    p = np.empty_like(f)
    info = np.zeros(3)
    st = _load().vdpo_solve_cg_g(*_dims(f), *_geom(L, geom), _ptr(rho), _ptr(f), _ptr(p), float(tol), int(maxit),
                                 _ptr(info))
    return p, {"iters": int(info[0]), "rel_res": float(info[1]), "rhs_mean": float(info[2]),
               "status": STATUS.get(st, st)}


def inverse_laplacian(g, L: float, geom=None) -> np.ndarray:
    """Constant-coefficient 7-point Laplacian inverse (zero mode removed), by plain DFTs (a plain
    cosine transform along x in the duct)."""
    g = _f64(g)
    out = np.empty_like(g)
    _load().vdpo_inverse_laplacian_g(*_dims(g), *_geom(L, geom), _ptr(g), _ptr(out))
    return out


def solve_fixed_point(rho, f, L: float, tol: float = 1e-12, maxit: int = 1000, omega: float = 1.0, geom=None):
    """The paper's iteration of Eq. (Pois); returns (p, info) like solve_cg."""
    rho, f = _f64(rho), _f64(f)
    p = np.empty_like(f)
    info = np.zeros(3)
    st = _load().vdpo_solve_fixed_point_g(*_dims(f), *_geom(L, geom), _ptr(rho), _ptr(f), _ptr(p), float(tol),
                                          int(maxit), float(omega), _ptr(info))
    return p, {"iters": int(info[0]), "rel_res": float(info[1]), "rhs_mean": float(info[2]),
               "status": STATUS.get(st, st)}


def divergence(u, L: float) -> np.ndarray:
    """Cell-centre divergence of a face field u = (ux, uy, uz) stored on the low faces."""
    ux, uy, uz = (_f64(x) for x in u)
    out = np.empty_like(ux)
    _load().vdpo_divergence(*_dims(ux), float(L), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(out))
    return out


def face_velocity(rho, m):
    """(ux, uy, uz) = face momenta m divided by the App. B face density."""
    rho = _f64(rho)
    mx, my, mz = (_f64(x) for x in m)
    u = tuple(np.empty_like(rho) for _ in range(3))
    st = _load().vdpo_face_velocity(*_dims(rho), _ptr(rho), _ptr(mx), _ptr(my), _ptr(mz), *(_ptr(x) for x in u))
    if st != 0:
        raise ValueError(f"face_velocity: {STATUS.get(st, st)}")
    return u


def projection_rhs(rho, m, rhs_div, c: float, L: float) -> np.ndarray:
    """RHS^Pois = (div(m / rho_face) - rhs_div) / c of App. A (mean not removed); rhs_div may be None."""
    rho = _f64(rho)
    mx, my, mz = (_f64(x) for x in m)
    rd = None if rhs_div is None else _f64(rhs_div)
    f = np.empty_like(rho)
    st = _load().vdpo_projection_rhs(*_dims(rho), float(L), _ptr(rho), _ptr(mx), _ptr(my), _ptr(mz),
                                     None if rd is None else _ptr(rd), float(c), _ptr(f))
    if st != 0:
        raise ValueError(f"projection_rhs: {STATUS.get(st, st)}")
    return f


def projection_correct(p, m, c: float, L: float):
    """Eq. (mom): the face momenta m minus c times the face pressure gradient (new arrays)."""
    p = _f64(p)
    mx, my, mz = (_f64(x) for x in m)
    out = tuple(np.empty_like(p) for _ in range(3))
    st = _load().vdpo_projection_correct(*_dims(p), float(L), _ptr(p), float(c), _ptr(mx), _ptr(my), _ptr(mz),
                                         *(_ptr(x) for x in out))
    if st != 0:
        raise ValueError(f"projection_correct: {STATUS.get(st, st)}")
    return out


def project(rho, m, rhs_div, c: float, L: float, tol: float = 1e-13):
    """The App. A projection: right side, solve, correction.  Returns (m_new, p, info)."""
    f = projection_rhs(rho, m, rhs_div, c, L)
    p, info = solve_cg(rho, f, L, tol=tol)
    return projection_correct(p, m, c, L), p, info


from .spectral_cg import fft_inverse_laplacian, solve_pcg_spectral  # noqa: E402,F401
