"""Seeded synthetic inputs for the variable-density Poisson solve (shared by the GPU path, the CPU
oracle, the tests and the benchmark).

This module only MAKES inputs -- density fields rho and right-hand sides f on the cell centres of
a periodic box -- from a seed.  It contains none of the solver's arithmetic (no face
coefficients, no Poisson operator, no Krylov or fixed-point step).

The paper (arXiv:1601.05448) has no public data set; its variable density comes from an ideal
gas heated by particles, rho = P0 / (R T) (Sec. 2), with radiatively heated particles warming the
gas around them (Eq. (PEE)).  The recipes below mimic that structure:

* ``density_modes``: rho = 1 + a g with g a sum of a few random Fourier modes, rescaled to span
  exactly [-1, 1] on the grid (density ratio (1 + a) / (1 - a); a = 0.5 gives 3).
* ``density_hotspots``: T = 1 + 0.3 F + s H, rho = T0 / T with T0 = 1, where F is a random
  Fourier field (max-abs normalised) and H a sum of Gaussian hot spots (std-dev 1.5 cells,
  amplitude U[0.5, 2], truncated at 4 std-devs) centred at uniform-random particle positions;
  s = 1, or found by bisection so that max(rho)/min(rho) hits a target ratio.
* ``rhs_divergence``: f = discrete divergence on the staggered grid of a seeded random velocity
  field (each face-normal component a sum over all integer wave vectors 1 <= |k| <= kmax of
  a cos(k.x) + b sin(k.x), a, b ~ N(0,1), sampled on its own faces and scaled to zero mean and
  unit variance); f has zero mean by telescoping, like the divergence that feeds the paper's
  pressure equation (App. A).

* ``face_momenta`` / ``divergence_target``: inputs of the projection steps either side of the
  solve (App. A): random face momenta (rho u)~ on the low faces of each cell, and a smooth
  cell-centre field standing for RHS^div.

Arrays are float64 with shape (nz, ny, nx) -- C order, x fastest -- and the box is [0, L)^3 with
cell (i, j, k) centred at ((i+1/2) hx, (j+1/2) hy, (k+1/2) hz), h_d = L / n_d.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

try:  # threaded FFTs when scipy is present; numpy's otherwise
    import scipy.fft as _fft

    def _ifftn(a):
        return _fft.ifftn(a, workers=-1)
except Exception:  # pragma: no cover
    _ifftn = np.fft.ifftn

TWO_PI = 2.0 * math.pi


def integer_wavevectors(kmin: float, kmax: float) -> np.ndarray:
    """All integer 3-vectors k with kmin <= |k| <= kmax, shape (m, 3) as (kx, ky, kz)."""
    r = int(math.floor(kmax))
    g = np.arange(-r, r + 1)
    kx, ky, kz = np.meshgrid(g, g, g, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1)
    n2 = (k * k).sum(axis=1)
    keep = (n2 >= kmin * kmin - 1e-9) & (n2 <= kmax * kmax + 1e-9)
    return k[keep]


def modes_field(shape, kvecs: np.ndarray, coefs: np.ndarray, offset=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Re sum_m coefs[m] exp(i 2 pi k_m . (idx + offset) / n) sampled on the grid.

    ``offset`` is the sample point inside a cell in cell units per axis (x, y, z): 0.5 = centre,
    0 = the low face.  Evaluated by one inverse FFT of a sparse spectrum.
    """
    nz, ny, nx = shape
    spec = np.zeros(shape, dtype=np.complex128)
    ox, oy, oz = offset
    for (kx, ky, kz), c in zip(kvecs, coefs):
        phase = np.exp(1j * TWO_PI * (kx * ox / nx + ky * oy / ny + kz * oz / nz))
        spec[int(kz) % nz, int(ky) % ny, int(kx) % nx] += c * phase
    out = _ifftn(spec).real * float(nx * ny * nz)
    return np.ascontiguousarray(out)


def _minmax_unit(g: np.ndarray) -> np.ndarray:
    lo, hi = float(g.min()), float(g.max())
    if hi - lo <= 0.0:
        return np.zeros_like(g)
    return (2.0 * g - (hi + lo)) / (hi - lo)


def random_modes(rng: np.random.Generator, nmodes: int, kmax: float):
    """nmodes wave vectors drawn uniformly from {1 <= |k| <= kmax}, amplitudes U[0.5,1], phases U[0,2pi)."""
    pool = integer_wavevectors(1.0, kmax)
    pick = rng.integers(0, len(pool), size=nmodes)
    amp = rng.uniform(0.5, 1.0, size=nmodes)
    phi = rng.uniform(0.0, TWO_PI, size=nmodes)
    return pool[pick], amp * np.exp(1j * phi)


def density_modes(shape, rng: np.random.Generator, nmodes: int = 8, kmax: float = 4.0,
                  amplitude: float = 0.5) -> np.ndarray:
    """rho = 1 + amplitude * g, g = random Fourier modes rescaled to span exactly [-1, 1]."""
    k, c = random_modes(rng, nmodes, kmax)
    g = _minmax_unit(modes_field(shape, k, c))
    return 1.0 + amplitude * g


def hotspot_field(shape, L: float, rng: np.random.Generator, nspots: int, width_cells: float = 1.5,
                  amp_lo: float = 0.5, amp_hi: float = 2.0, cutoff: float = 4.0,
                  chunk: int = 4096) -> np.ndarray:
    """H = sum_p A_p exp(-|x - x_p|^2 / (2 sigma^2)), periodic distance, truncated at cutoff*sigma."""
    nz, ny, nx = shape
    n = (nx, ny, nz)
    h = (L / nx, L / ny, L / nz)
    sig = tuple(width_cells * hd for hd in h)
    pos = rng.uniform(0.0, L, size=(nspots, 3))
    amp = rng.uniform(amp_lo, amp_hi, size=nspots)
    H = np.zeros(nx * ny * nz, dtype=np.float64)
    reach = int(math.ceil(cutoff * width_cells + 0.5))
    offs = np.arange(-reach, reach + 1)
    for s0 in range(0, nspots, chunk):
        p = pos[s0:s0 + chunk]
        a = amp[s0:s0 + chunk]
        m = p.shape[0]
        idx_axes, d2_axes = [], []
        for ax in range(3):
            i0 = np.floor(p[:, ax] / h[ax]).astype(np.int64)
            ii = i0[:, None] + offs[None, :]                      # (m, w) unwrapped cell index
            delta = (ii + 0.5) * h[ax] - p[:, ax:ax + 1]           # centre minus spot position
            idx_axes.append(np.mod(ii, n[ax]))
            d2_axes.append((delta / sig[ax]) ** 2)
        r2 = (d2_axes[2][:, :, None, None] + d2_axes[1][:, None, :, None] + d2_axes[0][:, None, None, :])
        w = a[:, None, None, None] * np.exp(-0.5 * r2)
        w[r2 > cutoff * cutoff] = 0.0
        flat = (idx_axes[0][:, None, None, :] + nx * (idx_axes[1][:, None, :, None]
                + ny * idx_axes[2][:, :, None, None]))
        H += np.bincount(flat.ravel(), weights=w.ravel(), minlength=H.size)
        del r2, w, flat
    return H.reshape(shape)


def _ratio(T: np.ndarray) -> float:
    return float(T.max() / T.min())


def _extreme_candidates(base: np.ndarray, H: np.ndarray, S: float):
    """The cells that can hold the maximum or the minimum of base + s H for some s in [0, S]
    (H >= 0), as flat arrays (base, H).  Both extremes are nondecreasing in s: a cell can be the
    maximum only if base + S H reaches max(base), and the minimum only if base stays at or below
    min(base + S H).  The extremes over these cells equal those over the whole grid, value for
    value, so a bisection over them takes the same steps, just faster."""
    b, h = base.ravel(), H.ravel()
    if float(h.min()) < 0.0:
        return b, h
    top = b + S * h
    keep = (top >= float(b.max())) | (b <= float(top.min()))
    return b[keep], h[keep]


def hotspot_scale(base: np.ndarray, H: np.ndarray, goal: float, cand=None) -> float:
    """s >= 0 with max(base + s H) / min(base + s H) = goal (H >= 0): the first power of two whose
    ratio reaches the goal brackets s, then 60 bisection steps.  cand: (base, H) restricted to
    the cells that can hold the extremes for every s up to the bracket (``_extreme_candidates``
    with a bound at least as large), or None to find them here."""
    lo, hi = 0.0, 1.0
    if cand is None:
        while _ratio(base + hi * H) < goal and hi < 1e6:
            hi *= 2.0
        bc, Hc = _extreme_candidates(base, H, hi)
    else:
        bc, Hc = cand
        while _ratio(bc + hi * Hc) < goal and hi < 1e6:
            hi *= 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _ratio(bc + mid * Hc) < goal:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def density_hotspots(shape, L: float, rng: np.random.Generator, nspots: int, kmax_F: float = 8.0,
                     nmodes_F: int = 16, F_amp: float = 0.3, target_ratio: float | None = None,
                     max_ratio: float | None = None):
    """rho = 1 / T with T = 1 + F_amp F + s H (T0 = 1).  Returns (rho, info).

    ``target_ratio``: choose s >= 0 by bisection so that max(T)/min(T) equals it (when the s = 0
    field already exceeds the target, F is scaled down instead).  ``max_ratio``: keep s = 1 unless
    the ratio exceeds max_ratio, then bisect down to it.
    """
    k, c = random_modes(rng, nmodes_F, kmax_F)
    F = modes_field(shape, k, c)
    F = F / float(np.abs(F).max())
    H = hotspot_field(shape, L, rng, nspots) if nspots > 0 else np.zeros(shape)
    base = 1.0 + F_amp * F
    s, fa = 1.0, F_amp
    goal = None
    if target_ratio is not None:
        goal = float(target_ratio)
    elif max_ratio is not None and _ratio(base + H) > max_ratio:
        goal = float(max_ratio)
    if goal is not None:
        if _ratio(base) >= goal:
            # even without hot spots the ratio is too large: shrink the Fourier part
            s = 0.0
            lo, hi = 0.0, F_amp
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if _ratio(1.0 + mid * F) < goal:
                    lo = mid
                else:
                    hi = mid
            fa = 0.5 * (lo + hi)
            base = 1.0 + fa * F
        else:
            s = hotspot_scale(base, H, goal)
    T = base + s * H
    rho = 1.0 / T
    info = {"hotspot_scale": s, "F_amp": fa, "nspots": nspots, "ratio": float(rho.max() / rho.min())}
    return np.ascontiguousarray(rho), info


def rhs_divergence(shape, L: float, rng: np.random.Generator, kmax: float = 4.0) -> np.ndarray:
    """f = discrete divergence of a random face-sampled velocity field (zero mean)."""
    nz, ny, nx = shape
    h = (L / nx, L / ny, L / nz)
    kv = integer_wavevectors(1.0, kmax)
    f = np.zeros(shape, dtype=np.float64)
    for d in range(3):  # d = 0: x, 1: y, 2: z
        a = rng.standard_normal(len(kv))
        b = rng.standard_normal(len(kv))
        # u_d lives on the low d-face of each cell: offset 0 along d, cell centre elsewhere
        off = [0.5, 0.5, 0.5]
        off[d] = 0.0
        u = modes_field(shape, kv, a - 1j * b, offset=tuple(off))
        u -= u.mean()
        sd = float(u.std())
        if sd > 0:
            u /= sd
        axis = 2 - d  # numpy axis of direction d
        f += (np.roll(u, -1, axis=axis) - u) / h[d]
    return np.ascontiguousarray(f)


def face_momenta(shape, L: float, rng: np.random.Generator, kmax: float = 4.0):
    """(mx, my, mz): seeded random face momenta, each component sampled on its own low faces
    (a sum over all integer wave vectors 1 <= |k| <= kmax of a cos(k.x) + b sin(k.x), a, b ~ N(0,1),
    scaled to unit standard deviation, plus a uniform mean flow in [-1, 1])."""
    kv = integer_wavevectors(1.0, kmax)
    out = []
    for d in range(3):
        a = rng.standard_normal(len(kv))
        b = rng.standard_normal(len(kv))
        off = [0.5, 0.5, 0.5]
        off[d] = 0.0
        m = modes_field(shape, kv, a - 1j * b, offset=tuple(off))
        sd = float(m.std())
        if sd > 0:
            m /= sd
        m += rng.uniform(-1.0, 1.0)
        out.append(np.ascontiguousarray(m))
    return tuple(out)


def divergence_target(shape, rng: np.random.Generator, mean: float = 0.1, amplitude: float = 0.05,
                      kmax: float = 4.0) -> np.ndarray:
    """A seeded cell-centre field standing for RHS^div of App. A (thermal expansion from the
    heated particles): mean + amplitude * g, g a few random modes spanning [-1, 1]."""
    kv, coefs = random_modes(rng, 8, kmax)
    g = _minmax_unit(modes_field(shape, kv, coefs))
    return np.ascontiguousarray(mean + amplitude * g)


def duct_problem(shape, lengths, seed: int, amplitude: float = 0.6, tol: float = 1e-10):
    """A seeded problem on the inflow-outflow duct of lengths (Lx, Ly, Lz): rho = 1 + amplitude g
    (8 random modes, density ratio (1 + a) / (1 - a)) and f = the discrete divergence recipe above
    with the spacing of y (any mean-free right side will do for the pressure solve)."""
    rng = np.random.default_rng(seed)
    rho = density_modes(shape, rng, amplitude=amplitude)
    f = rhs_divergence(shape, float(lengths[1]), rng)
    f -= f.mean()
    prob = Problem("duct", tuple(shape), float(lengths[1]), rho, f, tol, "fp64",
                   {"ratio": float(rho.max() / rho.min()), "seed": seed, "lengths": tuple(lengths)})
    return prob


@dataclass
class Problem:
    """One seeded solve: shape (nz, ny, nx), box length L, rho, f, tolerance and precision mode."""
    name: str
    shape: tuple
    L: float
    rho: np.ndarray
    f: np.ndarray
    tol: float
    precision: str = "fp64"
    info: dict = field(default_factory=dict)

    @property
    def n(self):
        nz, ny, nx = self.shape
        return nx, ny, nz


def smooth_problem(shape, seed: int, L: float = TWO_PI, amplitude: float = 0.5, tol: float = 1e-10,
                   name: str = "smooth") -> Problem:
    """Recipe of the 32^3 case at any shape: rho = 1 + amplitude*g (8 modes |k|<=4), f = div of a
    random |k|<=4 velocity field."""
    rng = np.random.default_rng(seed)
    rho = density_modes(shape, rng, amplitude=amplitude)
    f = rhs_divergence(shape, L, rng)
    return Problem(name, tuple(shape), L, rho, f, tol, "fp64",
                   {"ratio": float(rho.max() / rho.min()), "seed": seed})


def hotspot_problem(n: int, seed: int, nspots: int, L: float = TWO_PI, tol: float = 1e-10,
                    target_ratio=None, max_ratio=None, precision: str = "fp64",
                    name: str = "hotspots") -> Problem:
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    rho, info = density_hotspots(shape, L, rng, nspots, target_ratio=target_ratio, max_ratio=max_ratio)
    f = rhs_divergence(shape, L, rng)
    info["seed"] = seed
    return Problem(name, shape, L, rho, f, tol, precision, info)


# ---- the five workloads ---------------------------------------------------------------------

def config0() -> Problem:
    """32^3 box L = 2 pi, rho = 1 + 0.5 g (ratio 3), FP64 to relative residual 1e-10."""
    p = smooth_problem((32, 32, 32), seed=1, tol=1e-10, name="c0_32^3_fp64")
    return p


def config1() -> Problem:
    """256^3, rho = T0/T with 20k hot spots, hot-spot amplitude scaled so the density ratio is 4;
    FP64 to relative residual 1e-10."""
    return hotspot_problem(256, seed=2, nspots=20000, tol=1e-10, target_ratio=4.0, name="c1_256^3_fp64")


def config2() -> Problem:
    """512^3, 200k hot spots, ratio capped at 10, mixed precision refined to 1e-8."""
    return hotspot_problem(512, seed=3, nspots=200000, tol=1e-8, max_ratio=10.0, precision="mixed",
                           name="c2_512^3_mixed")


BATCH_SIZES = (64, 96, 128, 192)


def config3_instance(i: int) -> Problem:
    """Instance i of the 64-grid batch: n ~ U{64,96,128,192}, ratio R ~ U[2,10], mixed to 1e-8."""
    rng = np.random.default_rng(1000 + i)
    n = int(BATCH_SIZES[rng.integers(0, len(BATCH_SIZES))])
    R = float(rng.uniform(2.0, 10.0))
    nspots = int(round(20000 * n ** 3 / 256 ** 3))
    return hotspot_problem(n, seed=int(rng.integers(0, 2**31)), nspots=nspots, tol=1e-8, target_ratio=R,
                           precision="mixed", name=f"c3_inst{i}_{n}^3")


SERVE_SIZES = (32, 48, 64, 96, 128, 192, 256)


@dataclass
class Request:
    j: int
    arrival_s: float
    n: int
    ratio: float
    tol: float
    seed: int


def config4_requests(count: int = 5000, rate: float = 200.0, seed: int = 99999):
    """Poisson arrival stream: exponential gaps (mean 1/rate), n ~ U(SERVE_SIZES), R ~ U[2,10],
    tol log-uniform in [1e-10, 1e-6]; request j's fields come from seed 100000 + j."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for j in range(count):
        n = int(SERVE_SIZES[rng.integers(0, len(SERVE_SIZES))])
        R = float(rng.uniform(2.0, 10.0))
        tol = float(10.0 ** rng.uniform(-10.0, -6.0))
        out.append(Request(j, float(t[j]), n, R, tol, 100000 + j))
    return out


SERVE_BANK = 4          # seeded field sets per served grid size


def serve_bank(n: int, k: int):
    """Field set k of the served grid size n (seed 300000 + 10 n + k): the hot-spot recipe's
    pieces before the density ratio is chosen -- base = 1 + 0.3 F (F: 16 random modes |k| <= 8,
    max-abs normalised) and H (hot spots scaled by volume, 20000 n^3 / 256^3) -- and f (the
    divergence recipe).  Returns (base, H, f)."""
    rng = np.random.default_rng(300000 + 10 * n + k)
    shape = (n, n, n)
    kv, c = random_modes(rng, 16, 8.0)
    F = modes_field(shape, kv, c)
    F = F / float(np.abs(F).max())
    H = hotspot_field(shape, TWO_PI, rng, int(round(20000 * n ** 3 / 256 ** 3)))
    f = rhs_divergence(shape, TWO_PI, rng)
    return 1.0 + 0.3 * F, H, f


def request_draw(req: Request, bank_size: int = SERVE_BANK):
    """Request j's seeded choices (seed 100000 + j): its field set, and the periodic shifts (in
    cells, per axis z, y, x) applied to its density and to its right side."""
    rng = np.random.default_rng(req.seed)
    k = int(rng.integers(0, bank_size))
    shift_rho = tuple(int(x) for x in rng.integers(0, req.n, size=3))
    shift_f = tuple(int(x) for x in rng.integers(0, req.n, size=3))
    return k, shift_rho, shift_f


def request_fields(req: Request, bank, draw):
    """rho and f of a served request (numpy): rho = 1 / (base + s H) of its field set, s =
    hotspot_scale(base, H, req.ratio), and f, each shifted periodically by its draw."""
    base, H, f = bank
    _, shift_rho, shift_f = draw
    s = hotspot_scale(base, H, req.ratio)
    rho = np.roll(1.0 / (base + s * H), shift_rho, axis=(0, 1, 2))
    return np.ascontiguousarray(rho), np.ascontiguousarray(np.roll(f, shift_f, axis=(0, 1, 2)))


def request_problem(req: Request) -> Problem:
    nspots = int(round(20000 * req.n ** 3 / 256 ** 3))
    return hotspot_problem(req.n, seed=req.seed, nspots=nspots, tol=req.tol, target_ratio=req.ratio,
                           precision="mixed", name=f"req{req.j}_{req.n}^3")
