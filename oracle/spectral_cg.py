"""Reference pressure for large periodic grids -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` (and, through the package, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py``) may use this module; it shares no code with the GPU library.

The solution it returns is the plain definition of the discrete problem of Sec. 3.4 and App. A
(arXiv:1601.05448): the zero-mean p with A p = f - <f>, A the oracle's pinned face-flux operator
(``oracle.apply``, C).  At 256^3 and 512^3 the Jacobi-preconditioned conjugate gradients of the
oracle need thousands of iterations (about five minutes at 256^3 on 8 cores, hours at 512^3), so
this solver reaches the same p with conjugate gradients preconditioned by the constant-
coefficient inverse (-L_h)^-1 -- the inverse the paper's own solver applies in Sec. 3.4 --
evaluated with a library FFT (scipy.fft) instead of the oracle's plain O(n^2) DFT:

  * ``fft_inverse_laplacian(g, L)``: L_h^-1 g with the zero mode removed, L_h the 7-point
    Laplacian with coefficient 1/h_d^2 on every face; eigenvalue of Fourier mode k
    lambda(k) = -sum_d 4 sin^2(pi k_d / n_d) / h_d^2.  Pinned against the oracle's plain-DFT
    inverse and a Fourier mode's closed form.
  * ``solve_pcg_spectral(rho, f, L, tol)``: preconditioned CG on (-A) p = -(f - <f>) from p = 0;
    the recursive residual says when to look, the true residual f0 - A p (recomputed with the
    pinned operator) says when to stop; on a miss the search restarts from the true residual.
    Pinned against ``oracle.solve_cg`` and a dense solve on small grids.  The preconditioner is
    symmetric positive definite on mean-free vectors, so CG stays valid; it changes how fast the
    iteration gets there, not where it goes.

Arrays are float64 of shape (nz, ny, nx), x fastest.
"""
from __future__ import annotations

import math

import numpy as np

try:
    import scipy.fft as _sfft

    def _rfftn(a):
        return _sfft.rfftn(a, workers=-1)

    def _irfftn(a, shape):
        return _sfft.irfftn(a, s=shape, workers=-1)
except Exception:  # pragma: no cover - numpy's FFT when scipy is absent
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, shape):
        return np.fft.irfftn(a, s=shape)


def _lengths(L):
    if np.isscalar(L):
        return float(L), float(L), float(L)
    Lx, Ly, Lz = L
    return float(Lx), float(Ly), float(Lz)


def laplacian_eigenvalues(shape, L) -> np.ndarray:
    """lambda(k) on the rfftn half grid (kz, ky, kx <= nx/2) of the periodic box."""
    nz, ny, nx = shape
    Lx, Ly, Lz = _lengths(L)
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    sx = np.sin(math.pi * np.arange(nx // 2 + 1) / nx) ** 2 / (hx * hx)
    sy = np.sin(math.pi * np.arange(ny) / ny) ** 2 / (hy * hy)
    sz = np.sin(math.pi * np.arange(nz) / nz) ** 2 / (hz * hz)
    return -4.0 * (sz[:, None, None] + sy[None, :, None] + sx[None, None, :])


class _Inverse:
    """(-L_h)^-1 with the zero mode set to zero, eigenvalues computed once per grid."""

    def __init__(self, shape, L):
        self.shape = tuple(shape)
        lam = laplacian_eigenvalues(shape, L)
        lam[0, 0, 0] = 1.0
        self.inv = -1.0 / lam          # 1 / (-lambda) > 0
        self.inv[0, 0, 0] = 0.0

    def neg(self, r: np.ndarray) -> np.ndarray:
        """(-L_h)^-1 r."""
        return _irfftn(_rfftn(r) * self.inv, self.shape)


def fft_inverse_laplacian(g, L) -> np.ndarray:
    """L_h^-1 g (zero mode removed) by a library real FFT."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    return -_Inverse(g.shape, L).neg(g)


def solve_pcg_spectral(rho, f, L, tol: float = 1e-13, maxit: int = 2000, max_restarts: int = 4):
    """Zero-mean p with A p = f - <f> (A: the oracle's face-flux operator), by CG on -A
    preconditioned with (-L_h)^-1.  Returns (p, info) with the keys of ``oracle.solve_cg``.

    In FP64 the true residual of this operator cannot fall below about eps ||A|| ||p|| / ||f||
    (1e-12 at 512^3 with hot spots: the recursive residual goes on falling, the true one does not).
    A restart that does not at least halve the true residual ends the solve: status "ok" if the
    true residual met tol, else "stagnated" (info["rel_res"] says where it stopped)."""
    import oracle

    rho = np.ascontiguousarray(rho, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    Lx, Ly, Lz = _lengths(L)
    geom = (Lx, Ly, Lz, 0)
    b = oracle.face_coefficients(rho, Lx, geom)
    mf = oracle.mean(f)
    f0 = f - mf
    fn = math.sqrt(oracle.dot(f0, f0))
    p = np.zeros_like(f0)
    info = {"iters": 0, "rel_res": 0.0, "rhs_mean": mf, "status": "ok", "restarts": 0}
    if fn == 0.0:
        return p, info
    P = _Inverse(f0.shape, (Lx, Ly, Lz))
    r = -f0                      # r = b - (-A) p with b = -f0 and p = 0
    it, restart, last_true = 0, True, 1.0
    while True:
        if restart:
            z = P.neg(r)
            d = z.copy()
            rz = oracle.dot(r, z)
            restart = False
        if it >= maxit:
            info["status"] = "enotconv"
            break
        q = oracle.apply(b, d)
        np.negative(q, out=q)    # q = (-A) d
        dq = oracle.dot(d, q)
        if not dq > 0.0:
            info["status"] = "ebreakdown"
            break
        alpha = rz / dq
        p += alpha * d
        r -= alpha * q
        it += 1
        if math.sqrt(oracle.dot(r, r)) <= tol * fn:
            tr = f0 - oracle.apply(b, p)               # true residual of A p = f0
            trn = math.sqrt(oracle.dot(tr, tr)) / fn
            if trn <= tol:
                break
            if info["restarts"] >= max_restarts or trn > 0.5 * last_true:
                info["status"] = "stagnated"
                break
            last_true = trn
            np.negative(tr, out=r)                     # r = -(f0 - A p)
            restart = True
            info["restarts"] += 1
            continue
        z = P.neg(r)
        rz_new = oracle.dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        d *= beta
        d += z
    p -= oracle.mean(p)
    info["iters"] = it
    tr = f0 - oracle.apply(b, p)
    info["rel_res"] = math.sqrt(oracle.dot(tr, tr)) / fn
    return p, info
