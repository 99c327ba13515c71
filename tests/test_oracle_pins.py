"""Pins for the CPU oracle (no GPU): each test checks the oracle against something other than
itself -- a closed form, an invariant, a textbook/library routine, or an independent solver.

The solved problem is div((1/rho) grad p) = f on the periodic staggered grid (Sec. 3.4 of
arXiv:1601.05448), with f replaced by f - <f> (the compatibility constant chi' of App. A) and
the zero-mean p returned.
"""
import math

import numpy as np
import pytest

import oracle
import vdp_inputs as V

TWO_PI = 2.0 * math.pi


def centres(shape, L):
    nz, ny, nx = shape
    x = (np.arange(nx) + 0.5) * (L / nx)
    y = (np.arange(ny) + 0.5) * (L / ny)
    z = (np.arange(nz) + 0.5) * (L / nz)
    return np.meshgrid(z, y, x, indexing="ij")[::-1]  # X, Y, Z arrays of shape (nz, ny, nx)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---- 1. constant density: the discrete Fourier modes are exact eigenvectors -------------------

FOURIER_CASES = [
    ((8, 8, 8), TWO_PI, (1, 0, 0)),
    ((16, 12, 10), TWO_PI, (2, 3, 1)),
    ((12, 16, 8), 3.0, (1, -2, 3)),
    ((32, 32, 32), TWO_PI, (4, 1, -2)),
]


def _mode(shape, L, k):
    """cos of the discrete mode k sampled on cell centres, and its exact eigenvalue of the
    constant-coefficient second-difference Laplacian: -sum_d 4 sin^2(pi k_d / n_d) / h_d^2."""
    nz, ny, nx = shape
    X, Y, Z = centres(shape, L)
    kx, ky, kz = k
    theta = TWO_PI * (kx * X / L + ky * Y / L + kz * Z / L)
    lam = -4.0 * sum(math.sin(math.pi * kd / nd) ** 2 / (L / nd) ** 2 for kd, nd in zip(k, (nx, ny, nz)))
    return np.cos(theta + 0.3), lam


@pytest.mark.parametrize("shape,L,k", FOURIER_CASES)
def test_constant_density_fourier_eigenvector(shape, L, k):
    rho0 = 1.7
    rho = np.full(shape, rho0)
    u, lam = _mode(shape, L, k)
    Au = oracle.apply_rho(rho, L, u)
    # A = (1/rho0) * Laplacian_h  =>  A u = (lam / rho0) u, exactly up to rounding
    assert rel(Au, (lam / rho0) * u) < 1e-12


@pytest.mark.parametrize("shape,L,k", FOURIER_CASES)
def test_constant_density_fourier_solution(shape, L, k):
    rho0 = 0.6
    rho = np.full(shape, rho0)
    f, lam = _mode(shape, L, k)
    p, info = oracle.solve_cg(rho, f, L, tol=1e-13)
    assert info["status"] == "ok"
    exact = rho0 * f / lam
    exact -= exact.mean()
    assert rel(p, exact) < 1e-11


# ---- 2. density varying along one axis: flux integration closed form ---------------------------

def closed_form_1d(rho_line, f_line, h):
    """Periodic 1-D problem (b_{i+1}(p_{i+1}-p_i) - b_i(p_i-p_{i-1})) = f_i with
    b_i = 2/(rho_{i-1}+rho_i)/h^2.  The face flux q_i = b_i (p_i - p_{i-1}) obeys
    q_{i+1} - q_i = f_i, so q_i = q_0 + sum_{m<i} f_m; periodicity of p fixes q_0 through
    sum_i q_i / b_i = 0.  Then p_i = p_{i-1} + q_i / b_i, shifted to zero mean."""
    n = len(rho_line)
    b = [2.0 / (rho_line[i - 1] + rho_line[i]) / h ** 2 for i in range(n)]
    f0 = [fi - sum(f_line) / n for fi in f_line]
    partial = [0.0] * n
    for i in range(1, n):
        partial[i] = partial[i - 1] + f0[i - 1]
    q0 = -sum(partial[i] / b[i] for i in range(n)) / sum(1.0 / b[i] for i in range(n))
    q = [q0 + partial[i] for i in range(n)]
    p = [0.0] * n
    for i in range(1, n):
        p[i] = p[i - 1] + q[i] / b[i]
    m = sum(p) / n
    return np.array([pi - m for pi in p])


@pytest.mark.parametrize("axis", [0, 1, 2])  # direction x, y, z
def test_one_dimensional_closed_form(axis):
    shape = (10, 12, 14)  # (nz, ny, nx): different n per direction
    L = 2.5
    nz, ny, nx = shape
    ndir = (nx, ny, nz)[axis]
    rng = np.random.default_rng(11 + axis)
    rho_line = rng.uniform(0.3, 3.0, ndir)       # density ratio ~10, jagged
    f_line = rng.standard_normal(ndir) + 0.7      # nonzero mean on purpose
    bshape = [1, 1, 1]
    bshape[2 - axis] = ndir
    rho = np.broadcast_to(rho_line.reshape(bshape), shape).copy()
    f = np.broadcast_to(f_line.reshape(bshape), shape).copy()
    p, info = oracle.solve_cg(rho, f, L, tol=1e-13)
    assert info["status"] == "ok"
    assert abs(info["rhs_mean"] - f_line.mean()) < 1e-14
    exact_line = closed_form_1d(list(rho_line), list(f_line), L / ndir)
    exact = np.broadcast_to(exact_line.reshape(bshape), shape)
    assert rel(p, exact) < 1e-11


# ---- 3. operator invariants ---------------------------------------------------------------

def test_operator_symmetry_nullspace_energy():
    shape = (9, 10, 12)
    L = 1.3
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.2, 2.0, shape)
    u = rng.standard_normal(shape)
    v = rng.standard_normal(shape)
    b = oracle.face_coefficients(rho, L)
    Au, Av = oracle.apply(b, u), oracle.apply(b, v)
    # symmetric
    s1, s2 = float((u * Av).sum()), float((Au * v).sum())
    assert abs(s1 - s2) <= 1e-12 * abs(s1)
    # constants are in the null space, exactly
    assert np.all(oracle.apply(b, np.full(shape, 3.25)) == 0.0)
    # columns sum to zero (the left side integrates to zero over the periodic box, App. A)
    assert abs(float(Av.sum())) <= 1e-12 * float(np.abs(Av).sum())
    # negative semi-definite, with -<v, A v> = sum over faces of b * (jump of v)^2
    energy = 0.0
    for d, bd in enumerate(b):
        jump = v - np.roll(v, 1, axis=2 - d)   # v[c] - v[c - e_d] across the low face of c
        energy += float((bd * jump * jump).sum())
    assert abs(-float((v * Av).sum()) - energy) <= 1e-12 * energy


# ---- 4. dense direct solve on tiny grids (library LU) --------------------------------------

@pytest.mark.parametrize("shape", [(4, 4, 4), (8, 8, 8), (4, 6, 8)])
def test_dense_direct(shape):
    nz, ny, nx = shape
    N = nx * ny * nz
    L = 2.0
    rng = np.random.default_rng(N)
    rho = rng.uniform(0.25, 2.5, shape)
    f = rng.standard_normal(shape)
    h = (L / nx, L / ny, L / nz)
    # assemble from a list of faces: every face couples its two cells with weight 1/rho_face/h^2
    M = np.zeros((N, N))
    flat = lambda i, j, k: (i % nx) + nx * ((j % ny) + ny * (k % nz))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for d, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    a, c = flat(i, j, k), flat(i + di, j + dj, k + dk)
                    w = 1.0 / (0.5 * (rho[k, j, i] + rho[(k + dk) % nz, (j + dj) % ny, (i + di) % nx])) / h[d] ** 2
                    M[a, a] -= w
                    M[c, c] -= w
                    M[a, c] += w
                    M[c, a] += w
    f0 = f.ravel() - f.mean()
    # A p = f0 with sum(p) = 0  <=>  (A - 11^T) p = f0  (A 1 = 0, 1^T f0 = 0)
    p_ref = np.linalg.solve(M - np.ones((N, N)), f0)
    p, info = oracle.solve_cg(rho, f, L, tol=1e-13)
    assert info["status"] == "ok"
    assert rel(p.ravel(), p_ref) < 1e-11


# ---- 5. second-order convergence to a smooth continuous solution -----------------------------

def manufactured(n):
    """rho = 1 + 0.5 sin x cos y sin z, p* = sin x cos 2y + cos z sin y on [0, 2pi)^3;
    f = div(grad p*/rho) = lap(p*)/rho - grad(rho).grad(p*)/rho^2, differentiated by hand."""
    shape = (n, n, n)
    X, Y, Z = centres(shape, TWO_PI)
    sx, cx, sy, cy, sz, cz = np.sin(X), np.cos(X), np.sin(Y), np.cos(Y), np.sin(Z), np.cos(Z)
    rho = 1.0 + 0.5 * sx * cy * sz
    rx, ry, rz = 0.5 * cx * cy * sz, -0.5 * sx * sy * sz, 0.5 * sx * cy * cz
    p = sx * np.cos(2 * Y) + cz * sy
    px = cx * np.cos(2 * Y)
    py = -2.0 * sx * np.sin(2 * Y) + cz * cy
    pz = -sz * sy
    lap = -5.0 * sx * np.cos(2 * Y) - 2.0 * cz * sy
    f = lap / rho - (rx * px + ry * py + rz * pz) / rho ** 2
    return rho, f, p - p.mean()


def test_second_order_convergence():
    errs = []
    for n in (16, 32, 64):
        rho, f, pex = manufactured(n)
        p, info = oracle.solve_cg(rho, f, TWO_PI, tol=1e-12)
        assert info["status"] == "ok"
        errs.append(float(np.sqrt(np.mean((p - pex) ** 2))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


# ---- 6. the paper's own iteration (Eq. (Pois)) reaches the same discrete solution ------------

def test_paper_fixed_point_matches_cg():
    prob = V.config0()
    p_cg, i_cg = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    p_fp, i_fp = oracle.solve_fixed_point(prob.rho, prob.f, prob.L, tol=1e-12, maxit=200)
    assert i_cg["status"] == "ok" and i_fp["status"] == "ok"
    assert rel(p_fp, p_cg) < 1e-11


def test_inverse_laplacian_is_exact_on_a_mode():
    shape, L, k = (12, 10, 8), 2.0, (2, -1, 3)
    u, lam = _mode(shape, L, k)
    u = u - u.mean()
    assert rel(oracle.inverse_laplacian(u, L), u / lam) < 1e-12


# ---- 7. compatibility, gauge and degenerate inputs ------------------------------------------

def test_rhs_mean_is_removed_and_reported():
    prob = V.smooth_problem((12, 12, 12), seed=3)
    p1, i1 = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    p2, i2 = oracle.solve_cg(prob.rho, prob.f + 5.0, prob.L, tol=1e-13)
    assert abs(i2["rhs_mean"] - i1["rhs_mean"] - 5.0) < 1e-12
    assert rel(p2, p1) < 1e-11
    assert abs(float(p2.mean())) < 1e-14 * float(np.abs(p2).max())


def test_zero_and_constant_rhs_give_zero_pressure():
    rho = np.random.default_rng(0).uniform(0.5, 2.0, (6, 6, 6))
    for f in (np.zeros((6, 6, 6)), np.full((6, 6, 6), 2.5)):
        p, info = oracle.solve_cg(rho, f, 1.0, tol=1e-12)
        assert info["status"] == "ok" and info["iters"] == 0
        assert np.all(p == 0.0)


def test_bad_density_is_rejected():
    f = np.ones((4, 4, 4))
    for bad in (0.0, -1.0, np.nan, np.inf):
        rho = np.ones((4, 4, 4))
        rho[1, 2, 3] = bad
        p, info = oracle.solve_cg(rho, f, 1.0)
        assert info["status"] == "edensity"


# ---- 8. the input recipes --------------------------------------------------------------------

def test_config0_inputs():
    a, b = V.config0(), V.config0()
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.f, b.f)      # seeded
    assert abs(a.rho.max() / a.rho.min() - 3.0) < 1e-12                   # ratio 3 exactly
    assert abs(float(a.f.mean())) < 1e-13 * float(np.abs(a.f).max())       # divergence: mean-free


def test_hotspot_ratio_targeting():
    prob = V.hotspot_problem(32, seed=4, nspots=40, target_ratio=6.0)
    assert abs(prob.rho.max() / prob.rho.min() - 6.0) < 1e-9
    assert prob.rho.min() > 0


# ---- 9. the projection steps either side of the solve (App. A, Eq. (mom)) ----------------------
#
# Face momenta live on the low face of each cell.  The pins use constructions that do not go
# through the oracle's own formulas: a discrete gradient built here with np.roll, fields whose
# every difference vanishes by construction, summation by parts, and the density-weighted
# least-change characterisation of the projection solved by dense null-space linear algebra.

def _low_face_gradient(phi, L):
    nz, ny, nx = phi.shape
    h = (L / nx, L / ny, L / nz)
    return tuple((phi - np.roll(phi, 1, axis=2 - d)) / h[d] for d in range(3))


def _face_density(rho, d):
    return 0.5 * (np.roll(rho, 1, axis=2 - d) + rho)


def test_divergence_is_minus_the_adjoint_of_the_face_gradient():
    rng = np.random.default_rng(21)
    shape, L = (5, 7, 6), 1.7
    phi = rng.standard_normal(shape)
    u = tuple(rng.standard_normal(shape) for _ in range(3))
    lhs = float(np.sum(phi * oracle.divergence(u, L)))
    rhs = -sum(float(np.sum(a * b)) for a, b in zip(u, _low_face_gradient(phi, L)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_divergence_of_gradient_over_face_density_is_the_operator():
    # div(grad(phi) / rho_face) composed from the projection parts equals the pinned operator A
    rng = np.random.default_rng(22)
    shape, L = (8, 6, 10), 2.5
    rho = V.density_modes(shape, rng, amplitude=0.7)
    phi = rng.standard_normal(shape)
    comp = oracle.divergence(oracle.face_velocity(rho, _low_face_gradient(phi, L)), L)
    ref = oracle.apply_rho(rho, L, phi)
    assert np.abs(comp - ref).max() <= 1e-12 * np.abs(ref).max()


def test_projection_removes_a_pure_gradient():
    rng = np.random.default_rng(23)
    shape, L, c = (12, 10, 16), 2.0, 0.3
    rho = V.density_modes(shape, rng, amplitude=0.8)             # ratio 9
    phi = rng.standard_normal(shape)
    m = tuple(c * g for g in _low_face_gradient(phi, L))
    m_new, p, info = oracle.project(rho, m, None, c, L)
    assert info["status"] == "ok"
    scale = max(float(np.abs(x).max()) for x in m)
    assert max(float(np.abs(x).max()) for x in m_new) <= 1e-9 * scale
    assert np.abs(p - (phi - phi.mean())).max() <= 1e-9 * np.abs(phi).max()


def test_projection_keeps_a_weighted_solenoidal_field():
    # u_x depends on (y, z) only, u_y on (x, z), u_z on (x, y): each direction's face difference
    # vanishes, so u is discretely solenoidal and the momenta rho_face u pass unchanged
    rng = np.random.default_rng(24)
    shape, L, c = (10, 12, 8), 3.0, 0.05
    nz, ny, nx = shape
    rho = V.density_modes(shape, rng, amplitude=0.6)
    ux = np.broadcast_to(rng.standard_normal((nz, ny, 1)), shape)
    uy = np.broadcast_to(rng.standard_normal((nz, 1, nx)), shape)
    uz = np.broadcast_to(rng.standard_normal((1, ny, nx)), shape)
    m = tuple(np.ascontiguousarray(_face_density(rho, d) * u) for d, u in enumerate((ux, uy, uz)))
    f = oracle.projection_rhs(rho, m, None, c, L)
    h = L / max(shape)
    assert np.abs(f).max() <= 1e-13 * 3.0 * np.abs(ux).max() / (h * c) * 10
    m_new, p, info = oracle.project(rho, m, None, c, L)
    for a, b in zip(m_new, m):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("shape", [(8, 6, 10), (16, 16, 16)])
def test_projection_meets_the_divergence_constraint(shape):
    # App. A: div u_new = RHS^div - chi with chi = -c <RHS^Pois>; the divergence of the momenta
    # sums to zero on the periodic box, so chi = <RHS^div> and div u_new = RHS^div - <RHS^div>
    rng = np.random.default_rng(25)
    L, c = 2.0 * math.pi, 0.5 * 2e-3
    rho = V.density_modes(shape, rng, amplitude=0.6)
    m = V.face_momenta(shape, L, rng)
    rd = V.divergence_target(shape, rng)
    f = oracle.projection_rhs(rho, m, rd, c, L)
    chi = -c * float(f.mean())
    assert abs(chi - float(rd.mean())) <= 1e-12 * float(np.abs(rd).max()) * 1e3
    d0 = c * (f - f.mean())                       # divergence the correction has to remove
    m_new, p, info = oracle.project(rho, m, rd, c, L)
    assert info["status"] == "ok"
    div = oracle.divergence(oracle.face_velocity(rho, m_new), L)
    err = np.abs(div - (rd - rd.mean())).max()
    assert err <= 1e-11 * float(np.linalg.norm(d0))


def test_projection_is_idempotent_and_scales_with_c():
    rng = np.random.default_rng(26)
    shape, L = (8, 8, 12), 1.0
    rho = V.density_modes(shape, rng, amplitude=0.5)
    m = V.face_momenta(shape, L, rng)
    m1, p1, _ = oracle.project(rho, m, None, 0.25, L)
    m2, p2, _ = oracle.project(rho, m1, None, 0.25, L)
    m3, p3, _ = oracle.project(rho, m, None, 0.5, L)
    s = max(float(np.abs(x).max()) for x in m)
    for a, b in zip(m2, m1):
        assert np.abs(a - b).max() <= 1e-10 * s
    for a, b in zip(m3, m1):                      # the corrected momenta do not depend on c ...
        assert np.abs(a - b).max() <= 1e-10 * s
    assert np.abs(0.5 * p3 - 0.25 * p1).max() <= 1e-10 * np.abs(0.25 * p1).max()  # ... c p does


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4)])
def test_projection_is_the_density_weighted_least_change(shape):
    # Among all face velocities u with div u = RHS^div - <RHS^div>, the corrected one minimises
    # sum rho_face (u - u~)^2: found here by dense linear algebra on the null space of the
    # divergence matrix (whose columns are divergences of unit face fields)
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(27)
    L, c = 1.3, 0.7
    n = int(np.prod(shape))
    rho = V.density_modes(shape, rng, amplitude=0.7)
    m = tuple(rng.standard_normal(shape) for _ in range(3))
    rd = rng.standard_normal(shape)
    cols = []
    for d in range(3):
        for q in range(n):
            e = [np.zeros(shape) for _ in range(3)]
            e[d].flat[q] = 1.0
            cols.append(oracle.divergence(tuple(e), L).ravel())
    D = np.stack(cols, axis=1)                                          # n x 3n
    w = np.concatenate([_face_density(rho, d).ravel() for d in range(3)])
    u0 = np.concatenate([(m[d] / _face_density(rho, d)).ravel() for d in range(3)])
    r = (rd - rd.mean()).ravel()
    up = np.linalg.lstsq(D, r, rcond=None)[0]                           # a particular solution
    N = scipy_linalg.null_space(D)
    sw = np.sqrt(w)
    y = np.linalg.lstsq(sw[:, None] * N, sw * (u0 - up), rcond=None)[0]
    u_best = up + N @ y
    m_new, p, info = oracle.project(rho, m, rd, c, L)
    u_new = np.concatenate([(m_new[d] / _face_density(rho, d)).ravel() for d in range(3)])
    assert np.abs(u_new - u_best).max() <= 1e-9 * np.abs(u0).max()


@pytest.mark.parametrize("geom", [None, (3.0, 1.0, 0.75, 1)])
def test_paper_iteration_is_exact_in_one_step_for_constant_density(geom):
    # Eq. (Pois): with rho constant the dropped term rho grad(1/rho) . grad(dp) is zero, so one
    # step p = L^-1 (rho f) solves div((1/rho) grad p) = f exactly (periodic box and duct)
    rng = np.random.default_rng(46)
    shape = (6, 8, 24)
    rho = np.full(shape, 2.5)
    f = rng.standard_normal(shape)
    p, info = oracle.solve_fixed_point(rho, f, 1.3, tol=1e-12, geom=geom)
    assert info["status"] == "ok" and info["iters"] == 1 and info["rel_res"] <= 1e-13
    assert oracle.relative_residual(rho, 1.3, f, p, geom=geom) <= 1e-13


# ---- 10. the large-grid reference solver (oracle.solve_pcg_spectral) ----------------------------
#
# CG on the pinned operator, preconditioned by the constant-coefficient inverse through a library
# FFT.  Its answer is pinned to the dense solve and to the oracle's Jacobi CG; its FFT inverse to
# the oracle's plain DFT and to a Fourier mode's closed form.  A wrong preconditioner could only
# slow it down (the true residual of the pinned operator decides the stop), which the last pin
# shows with a deliberately wrong eigenvalue.

@pytest.mark.parametrize("shape,L", [((8, 12, 16), 2.0), ((16, 16, 16), TWO_PI), ((6, 10, 24), (3.0, 1.5, 0.75))])
def test_fft_inverse_equals_the_plain_dft_inverse(shape, L):
    g = np.random.default_rng(sum(shape)).standard_normal(shape)
    if np.isscalar(L):
        ref = oracle.inverse_laplacian(g, L)
    else:
        ref = oracle.inverse_laplacian(g, None, geom=(L[0], L[1], L[2], 0))
    assert rel(oracle.fft_inverse_laplacian(g, L), ref) < 1e-12


def test_fft_inverse_on_a_mode():
    shape, L, k = (12, 10, 16), 2.0, (3, -2, 1)
    u, lam = _mode(shape, L, k)
    u = u - u.mean()
    assert rel(oracle.fft_inverse_laplacian(u, L), u / lam) < 1e-12


@pytest.mark.parametrize("shape", [(4, 4, 4), (8, 8, 8), (4, 6, 8)])
def test_spectral_pcg_equals_dense_solve(shape):
    nz, ny, nx = shape
    L = 2.0
    rng = np.random.default_rng(nx * ny * nz)      # the dense pin's density and right side
    rho = rng.uniform(0.25, 2.5, shape)
    f = rng.standard_normal(shape)
    p_cg, _ = oracle.solve_cg(rho, f, L, tol=1e-13)
    p, info = oracle.solve_pcg_spectral(rho, f, L, tol=1e-13)
    assert info["status"] == "ok" and info["rel_res"] <= 1e-13
    assert rel(p, p_cg) < 1e-11


@pytest.mark.parametrize("make", [lambda: V.config0(),
                                  lambda: V.hotspot_problem(48, seed=66, nspots=130, target_ratio=8.0)])
def test_spectral_pcg_equals_jacobi_cg(make):
    prob = make()
    p_cg, i_cg = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    p, info = oracle.solve_pcg_spectral(prob.rho, prob.f, prob.L, tol=1e-13)
    assert info["status"] == "ok" and abs(info["rhs_mean"] - i_cg["rhs_mean"]) < 1e-15
    assert rel(p, p_cg) < 1e-11
    assert abs(float(p.mean())) < 1e-14 * float(np.abs(p).max())
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, p) <= 1e-13
    assert 5 * info["iters"] < i_cg["iters"]        # the preconditioner does its job


def test_spectral_pcg_answer_does_not_depend_on_the_preconditioner(monkeypatch):
    """A planted mistake in the eigenvalues (sin instead of sin^2) leaves the answer alone and only
    costs iterations: the stop is decided by the pinned operator's true residual."""
    from oracle import spectral_cg as S
    prob = V.hotspot_problem(32, seed=67, nspots=40, target_ratio=5.0)
    p_ok, i_ok = oracle.solve_pcg_spectral(prob.rho, prob.f, prob.L, tol=1e-13)
    good = S.laplacian_eigenvalues

    def wrong(shape, L):
        lam = good(shape, L)
        return -np.sqrt(-lam) * 3.0
    monkeypatch.setattr(S, "laplacian_eigenvalues", wrong)
    p_bad, i_bad = oracle.solve_pcg_spectral(prob.rho, prob.f, prob.L, tol=1e-13)
    assert i_bad["status"] == "ok" and rel(p_bad, p_ok) < 1e-11
    assert i_bad["iters"] > i_ok["iters"]
