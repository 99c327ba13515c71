"""Pins for the oracle's inflow-outflow duct (no GPU): periodic in y and z, no pressure flux through
the two x ends (Sec. 3.2 configuration 2 of arXiv:1601.05448; the pressure condition is a
reading), with per-direction box lengths.  Each test checks the oracle against a closed form, an
invariant, dense linear algebra or an independent solver.
"""
import math

import numpy as np
import pytest

import oracle
import vdp_inputs as V

TWO_PI = 2.0 * math.pi


def _cosine_fourier_mode(shape, geom, k):
    """cos(pi kx (i + 1/2) / nx) exp(i 2 pi (ky y + kz z)) real part, and its closed-form
    eigenvalue of the 7-point operator with unit coefficient (zero flux at the x ends)."""
    nz, ny, nx = shape
    Lx, Ly, Lz, _ = geom
    kx, ky, kz = k
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    l = np.arange(nz) + 0.5
    ax = np.cos(math.pi * kx * i / nx)
    ph = 2 * math.pi * (ky * j[None, :] / ny + kz * l[:, None] / nz)     # (nz, ny)
    u = np.cos(ph)[:, :, None] * ax[None, None, :]
    h = (Lx / nx, Ly / ny, Lz / nz)
    lam = -(4 / h[0] ** 2 * math.sin(math.pi * kx / (2 * nx)) ** 2 +
            4 / h[1] ** 2 * math.sin(math.pi * ky / ny) ** 2 +
            4 / h[2] ** 2 * math.sin(math.pi * kz / nz) ** 2)
    return u, lam


DUCTS = [((6, 8, 24), (3.0, 1.0, 0.75, 1), (1, 0, 0)),
         ((8, 8, 32), (4.0, 1.0, 1.0, 1), (3, 2, 1)),
         ((4, 6, 16), (2.0, 0.5, 0.5, 1), (15, 1, 3)),
         ((6, 8, 16), (2.0, 1.0, 1.0, 1), (0, 2, 1))]


@pytest.mark.parametrize("shape,geom,k", DUCTS)
def test_cosine_fourier_modes_are_eigenvectors(shape, geom, k):
    u, lam = _cosine_fourier_mode(shape, geom, k)
    Au = oracle.apply_rho(np.ones(shape), 0.0, u, geom=geom)
    assert np.abs(Au - lam * u).max() <= 1e-10 * abs(lam) * np.abs(u).max()
    p, info = oracle.solve_cg(np.ones(shape), lam * u, 0.0, tol=1e-13, geom=geom)
    assert np.abs(p - u).max() <= 1e-9 * np.abs(u).max()
    z = oracle.inverse_laplacian(lam * u, 0.0, geom=geom)          # the cosine-transform inverse
    assert np.abs(z - u).max() <= 1e-10 * np.abs(u).max()


def test_no_coupling_across_the_x_ends_and_an_exact_null_space():
    rng = np.random.default_rng(41)
    shape, geom = (4, 5, 8), (2.0, 1.0, 1.5, 1)
    rho = V.density_modes(shape, rng, amplitude=0.7, kmax=3.0)
    bx, by, bz = oracle.face_coefficients(rho, 0.0, geom=geom)
    assert np.all(bx[:, :, 0] == 0.0) and np.all(bx[:, :, 1:] > 0.0)
    p = rng.standard_normal(shape)
    q = p.copy()
    q[:, :, 0] += 1.0                                # change only cells at the inflow end
    d = oracle.apply_rho(rho, 0.0, q, geom=geom) - oracle.apply_rho(rho, 0.0, p, geom=geom)
    assert np.all(d[:, :, -1] == 0.0)                # the outflow end does not see it
    assert np.abs(oracle.apply_rho(rho, 0.0, np.ones(shape), geom=geom)).max() <= 1e-12 * bx.max()
    n = rho.size                                     # symmetric, one-dimensional null space
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        A[:, c] = oracle.apply_rho(rho, 0.0, e.reshape(shape), geom=geom).ravel()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(-A)
    assert abs(ev[0]) <= 1e-10 * ev[-1] and ev[1] > 1e-6 * ev[-1]


def test_one_dimensional_closed_form_along_x():
    # rho and f vary along x only: the zero-flux ends give the face fluxes by summation,
    # G_{i} = sum_{j < i} f_j (with G_0 = 0 at the inflow face), and p_i - p_{i-1} = G_i / b_i
    rng = np.random.default_rng(42)
    nx, ny, nz = 32, 2, 3
    geom = (5.0, 1.0, 1.0, 1)
    h = geom[0] / nx
    rho_line = rng.uniform(1.0, 10.0, nx)
    f_line = rng.standard_normal(nx)
    f_line -= f_line.mean()
    rho = np.broadcast_to(rho_line, (nz, ny, nx)).copy()
    f = np.broadcast_to(f_line, (nz, ny, nx)).copy()
    b = np.zeros(nx)
    b[1:] = 2.0 / (rho_line[:-1] + rho_line[1:]) / h ** 2
    G = np.concatenate([[0.0], np.cumsum(f_line)[:-1]])
    p_line = np.concatenate([[0.0], np.cumsum(G[1:] / b[1:])])
    p_line -= p_line.mean()
    p, info = oracle.solve_cg(rho, f, 0.0, tol=1e-14, geom=geom)
    assert info["status"] == "ok"
    assert np.abs(p - p_line[None, None, :]).max() <= 1e-9 * np.abs(p_line).max()


def test_dense_direct_solve_on_a_tiny_duct():
    rng = np.random.default_rng(43)
    shape, geom = (3, 4, 8), (2.0, 1.0, 0.8, 1)
    rho = V.density_modes(shape, rng, amplitude=0.8, kmax=2.0)
    f = rng.standard_normal(shape)
    n = rho.size
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        A[:, c] = oracle.apply_rho(rho, 0.0, e.reshape(shape), geom=geom).ravel()
    ref = np.linalg.lstsq(A, (f - f.mean()).ravel(), rcond=None)[0]
    ref -= ref.mean()
    p, info = oracle.solve_cg(rho, f, 0.0, tol=1e-14, geom=geom)
    assert np.abs(p.ravel() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_paper_iteration_reaches_the_cg_solution_in_a_duct():
    rng = np.random.default_rng(44)
    shape, geom = (12, 12, 48), (4 * TWO_PI / 4, TWO_PI / 4, TWO_PI / 4, 1)
    rho = V.density_modes(shape, rng, amplitude=0.6)
    f = V.rhs_divergence(shape, geom[1], rng)
    p1, i1 = oracle.solve_cg(rho, f, 0.0, tol=1e-13, geom=geom)
    p2, i2 = oracle.solve_fixed_point(rho, f, 0.0, tol=1e-12, geom=geom)
    assert i1["status"] == "ok" and i2["status"] == "ok"
    assert np.abs(p1 - p2).max() <= 1e-9 * np.abs(p1).max()


def test_second_order_convergence_in_a_duct():
    # p = cos(pi x / Lx) cos(2 pi y / Ly) has zero normal derivative at x = 0, Lx; with
    # rho = 2 + sin(2 pi z / Lz) the continuous f = div((1/rho) grad p) is written out below
    Lx, Ly, Lz = 2.0, 1.0, 1.0
    errs = []
    for n in (8, 16, 32):
        shape = (n, n, 2 * n)
        nz, ny, nx = shape
        x = (np.arange(nx) + 0.5) * Lx / nx
        y = (np.arange(ny) + 0.5) * Ly / ny
        z = (np.arange(nz) + 0.5) * Lz / nz
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        a, b, c = math.pi / Lx, 2 * math.pi / Ly, 2 * math.pi / Lz
        rho = 2.0 + np.sin(c * Z)
        p_ex = np.cos(a * X) * np.cos(b * Y)
        f = -(a * a + b * b) * p_ex / rho            # grad(1/rho) is along z, grad p has no z part
        p, info = oracle.solve_cg(rho, f, 0.0, tol=1e-13, geom=(Lx, Ly, Lz, 1))
        errs.append(np.abs(p - (p_ex - p_ex.mean())).max())
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0, errs


def _fft_tridiagonal_inverse(g, geom):
    """The paper's constant-coefficient solve in the duct (Sec. 3.4): Fourier transforms in the
    periodic directions y, z, then one tridiagonal solve along x per (ky, kz) with zero flux
    through both ends; the zero mode is removed.  numpy FFTs and a dense tridiagonal solve."""
    nz, ny, nx = g.shape
    Lx, Ly, Lz, _ = geom
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    G = np.fft.fft(np.fft.fft(g, axis=1), axis=0)          # (kz, ky, x)
    T = np.zeros((nx, nx))
    for i in range(nx):                                     # second difference along x, no end flux
        if i > 0:
            T[i, i - 1] = 1.0
            T[i, i] -= 1.0
        if i < nx - 1:
            T[i, i + 1] = 1.0
            T[i, i] -= 1.0
    T /= hx * hx
    P = np.empty_like(G)
    for kz in range(nz):
        for ky in range(ny):
            lam = (4 / hy ** 2 * math.sin(math.pi * ky / ny) ** 2 + 4 / hz ** 2 * math.sin(math.pi * kz / nz) ** 2)
            M = T - lam * np.eye(nx)
            if kz == 0 and ky == 0:                         # singular: the constant is free
                sol = np.linalg.lstsq(M, G[kz, ky], rcond=None)[0]
                P[kz, ky] = sol - sol.mean()
            else:
                P[kz, ky] = np.linalg.solve(M, G[kz, ky])
    return np.real(np.fft.ifft(np.fft.ifft(P, axis=0), axis=1))


@pytest.mark.parametrize("shape,geom", [((6, 8, 20), (3.0, 1.0, 0.75, 1)), ((4, 5, 12), (2.0, 0.5, 1.5, 1))])
def test_cosine_inverse_equals_the_papers_fft_tridiagonal_solve(shape, geom):
    rng = np.random.default_rng(45)
    g = rng.standard_normal(shape)
    ref = _fft_tridiagonal_inverse(g, geom)
    got = oracle.inverse_laplacian(g, 0.0, geom=geom)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
