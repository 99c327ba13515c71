"""Geometric multigrid preconditioner for the variable-coefficient Poisson operator -- TEST
INFRASTRUCTURE ONLY (part of the CPU oracle; only tests/, the smoke check and the CPU leg of the
benchmark may use it).  Plain FP64 numpy, written from the textbook definition of a symmetric
V-cycle; it shares no code with the GPU library.

The paper solves its pressure equation with a constant-coefficient FFT inverse (Sec. 3.4); a
V-cycle is the standard mesh-independent alternative that needs no FFT-friendly grid size.  It
approximates (-A)^-1 for the discrete operator A of div((1/rho) grad .) (the face coefficients of
the oracle, App. B face density), on the cell-centred periodic grid:

  levels    level 0 is the grid itself; a level is halved in every direction while all three
            sizes are even and it has more than 64 cells.  The coarsest level must have at most
            512 cells (else the grid is not supported).
  coarse    face coefficient of a coarse low face = 1/2 x the sum of the four fine low-face
  operator  coefficients it covers (the 2h rediscretisation of the face flux: for constant rho it
            is 8 times the operator on the 2h grid, the volume ratio of the summed equations).
  P         cell-centred linear interpolation: along each axis a fine cell takes 3/4 of its
            parent and 1/4 of the parent's neighbour on its side (tensor product in 3-D).
  R         the transpose of P (so each coarse value sums its fine neighbourhood with weights
            (1/4, 3/4, 3/4, 1/4) per axis; the weights total 8).
  smoother  one weighted Jacobi sweep x += w D^-1 (r - (-A) x), w = 0.8, before the coarse
            correction (from x = 0) and one after it; D = diag(-A).
  coarsest  the exact pseudo-inverse of -A on the coarsest grid (constants are its null space).

With the same smoother before and after, R = P^T and a symmetric coarse solve, the V-cycle is a
fixed symmetric linear operator; on mean-free vectors it is positive definite (checked densely by
the pins), so it can precondition conjugate gradients.

Pins (tests/test_oracle_multigrid.py): R = P^T and P reproduces constants; the coarse operator of
a constant density equals 8 x the operator on the 2h grid; a grid with no coarser level is solved
exactly (the V-cycle is the pseudo-inverse); the V-cycle is symmetric positive definite on
mean-free vectors (dense, small grids) with the spectrum of M(-A) in (0, 1]; on a constant
density a smooth Fourier mode stays a Fourier mode and the two-grid cycle's error on it falls at
second order in h; preconditioned CG reaches the plain oracle solution and its iteration count
does not grow with the grid.
"""
from __future__ import annotations

import numpy as np

from . import face_coefficients

OMEGA = 0.8           # Jacobi weight
MIN_COARSEN = 64      # a level with at most this many cells is not coarsened further
MAX_COARSEST = 512    # the coarsest level's pseudo-inverse is dense


def _dims(a):
    nz, ny, nx = a.shape
    return nx, ny, nz


def apply(b, p):
    """A p for face coefficients b = (bx, by, bz) stored on the low faces (numpy axis of x is 2)."""
    out = np.zeros_like(p)
    for d in range(3):
        ax = 2 - d
        hi = np.roll(b[d], -1, axis=ax)
        out += hi * (np.roll(p, -1, axis=ax) - p) - b[d] * (p - np.roll(p, 1, axis=ax))
    return out


def diagonal(b):
    """D = diag(-A): the sum of the six face coefficients around each cell."""
    return sum(b[d] + np.roll(b[d], -1, axis=2 - d) for d in range(3))


def level_shapes(nx: int, ny: int, nz: int):
    """(nz, ny, nx) of every level, or None when the coarsest level would exceed MAX_COARSEST."""
    shapes = [(nz, ny, nx)]
    while True:
        z, y, x = shapes[-1]
        if x % 2 or y % 2 or z % 2 or x * y * z <= MIN_COARSEN:
            break
        shapes.append((z // 2, y // 2, x // 2))
    z, y, x = shapes[-1]
    return shapes if x * y * z <= MAX_COARSEST else None


def supported(nx: int, ny: int, nz: int) -> bool:
    return level_shapes(nx, ny, nz) is not None


def coarsen(b):
    """Coarse face coefficients: 1/2 x the sum of the four fine low faces under each coarse low
    face (the fine cells with an even index along the face normal)."""
    nz, ny, nx = b[0].shape
    out = []
    for d in range(3):
        ax = 2 - d
        sel = [slice(None)] * 3
        sel[ax] = slice(0, None, 2)
        faces = b[d][tuple(sel)]                  # fine low faces on coarse low faces
        fz, fy, fx = faces.shape
        # sum the 2 x 2 fine faces in the two tangential directions
        shape = [fz, fy, fx]
        blocks = []
        for a in range(3):
            if a == ax:
                blocks.append((shape[a], 1))
            else:
                blocks.append((shape[a] // 2, 2))
        r = faces.reshape(blocks[0][0], blocks[0][1], blocks[1][0], blocks[1][1], blocks[2][0], blocks[2][1])
        out.append(0.5 * r.sum(axis=(1, 3, 5)))
    return out


def _neighbours(x, ax, wall):
    """The coarse neighbours below and above along axis ax, periodic; with wall (the duct's x
    ends) a cell at an end is its own neighbour there (the interpolant is constant up to the
    wall, as zero flux through it implies)."""
    below, above = np.roll(x, 1, axis=ax), np.roll(x, -1, axis=ax)
    if wall:
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = 0
        last[ax] = -1
        below[tuple(first)] = x[tuple(first)]
        above[tuple(last)] = x[tuple(last)]
    return below, above


def prolong(xc, bc_x: int = 0):
    """Cell-centred linear interpolation to the grid twice as fine in every direction (bc_x = 1:
    no interpolation across the duct's x ends)."""
    x = xc
    for ax in range(3):
        below, above = _neighbours(x, ax, bc_x == 1 and ax == 2)
        lo = 0.75 * x + 0.25 * below    # fine child on the low side
        hi = 0.75 * x + 0.25 * above    # fine child on the high side
        shape = list(x.shape)
        shape[ax] *= 2
        y = np.empty(shape)
        s_lo = [slice(None)] * 3
        s_hi = [slice(None)] * 3
        s_lo[ax] = slice(0, None, 2)
        s_hi[ax] = slice(1, None, 2)
        y[tuple(s_lo)] = lo
        y[tuple(s_hi)] = hi
        x = y
    return x


def restrict(r, bc_x: int = 0):
    """The transpose of prolong (axis by axis, in the reverse order)."""
    x = r
    for ax in (2, 1, 0):
        s_lo = [slice(None)] * 3
        s_hi = [slice(None)] * 3
        s_lo[ax] = slice(0, None, 2)
        s_hi[ax] = slice(1, None, 2)
        lo, hi = x[tuple(s_lo)], x[tuple(s_hi)]
        # coarse C collects 3/4 of both children, 1/4 of the low child of C+1 and of the high
        # child of C-1 (the fine cells whose interpolation used C as the neighbour)
        from_above = np.roll(lo, -1, axis=ax)
        from_below = np.roll(hi, 1, axis=ax)
        if bc_x == 1 and ax == 2:  # at the duct's ends the own child took that 1/4 instead
            first = [slice(None)] * 3
            last = [slice(None)] * 3
            first[ax] = 0
            last[ax] = -1
            from_below[tuple(first)] = lo[tuple(first)]
            from_above[tuple(last)] = hi[tuple(last)]
        x = 0.75 * lo + 0.75 * hi + 0.25 * from_above + 0.25 * from_below
    return x


def dense_negative_operator(b):
    """-A as a dense matrix (column q = -A e_q)."""
    shape = b[0].shape
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        M[:, q] = -apply(b, e.reshape(shape)).ravel()
    return M


class Hierarchy:
    """The levels of a V-cycle for face coefficients b (level 0)."""

    def __init__(self, b, max_levels: int = 0, bc_x: int = 0):
        """max_levels > 0 keeps only that many levels (the last one still solved exactly; for the
        two-grid pins).  bc_x = 1: the duct (b has no x faces at the ends; the transfers do not
        reach across them)."""
        self.bc_x = int(bc_x)
        nz, ny, nx = b[0].shape
        if max_levels > 0:
            shapes = [(nz, ny, nx)]
            while len(shapes) < max_levels and all(v % 2 == 0 for v in shapes[-1]):
                z, y, x = shapes[-1]
                shapes.append((z // 2, y // 2, x // 2))
        else:
            shapes = level_shapes(nx, ny, nz)
        if shapes is None:
            raise ValueError("grid not supported by the V-cycle (coarsest level too large)")
        self.b = [tuple(np.asarray(x, dtype=np.float64) for x in b)]
        for _ in shapes[1:]:
            self.b.append(tuple(coarsen(self.b[-1])))
        self.D = [diagonal(x) for x in self.b]
        # the exact null space of -A is the constants (eigenvalue 0); rounding leaves it at about
        # 1e-16 of the largest eigenvalue, which a pseudo-inverse must not invert
        self.coarse_pinv = np.linalg.pinv(dense_negative_operator(self.b[-1]), rcond=1e-10, hermitian=True)

    @classmethod
    def from_density(cls, rho, L: float, max_levels: int = 0, geom=None):
        bc_x = 0 if geom is None else int(geom[3])
        return cls(face_coefficients(rho, L, geom), max_levels, bc_x)

    @property
    def nlevels(self):
        return len(self.b)

    def vcycle(self, r, level: int = 0):
        """Approximation of (-A_level)^-1 r by one symmetric V-cycle."""
        b, D = self.b[level], self.D[level]
        if level == self.nlevels - 1:
            return (self.coarse_pinv @ r.ravel()).reshape(r.shape)
        x = OMEGA * r / D                               # pre-smoothing sweep from x = 0
        res = r + apply(b, x)                           # r - (-A) x
        xc = self.vcycle(restrict(res, self.bc_x), level + 1)      # coarse-grid correction
        x = x + prolong(xc, self.bc_x)
        x = x + OMEGA * (r + apply(b, x)) / D           # post-smoothing sweep
        return x


def solve_pcg(rho, f, L: float, tol: float = 1e-12, maxit: int = 1000, geom=None):
    """CG on -A p = -(f - <f>) preconditioned by the V-cycle; returns (p, info) with the zero-mean
    p and info keys iters, rel_res (true residual), rhs_mean, status."""
    H = Hierarchy.from_density(rho, L, geom=geom)
    b = H.b[0]
    f = np.asarray(f, dtype=np.float64)
    mu = float(f.mean())
    g = -(f - mu)                                      # -A p = g
    gn = float(np.linalg.norm(g))
    p = np.zeros_like(g)
    if gn == 0.0:
        return p, {"iters": 0, "rel_res": 0.0, "rhs_mean": mu, "status": "ok"}
    r = g.copy()
    z = H.vcycle(r)
    z -= z.mean()
    d = z.copy()
    rz = float(np.vdot(r, z))
    status = "enotconv"
    it = 0
    for it in range(1, maxit + 1):
        q = -apply(b, d)
        alpha = rz / float(np.vdot(d, q))
        p += alpha * d
        r -= alpha * q
        if float(np.linalg.norm(r)) <= tol * gn:
            status = "ok"
            break
        z = H.vcycle(r)
        z -= z.mean()
        rz_new = float(np.vdot(r, z))
        d = z + (rz_new / rz) * d
        rz = rz_new
    p -= p.mean()
    rel = float(np.linalg.norm(g + apply(b, p)) / gn)
    return p, {"iters": it, "rel_res": rel, "rhs_mean": mu, "status": status}
