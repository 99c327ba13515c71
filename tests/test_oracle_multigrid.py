"""Pins for the oracle's multigrid V-cycle (no GPU): each test checks it against something other
than itself -- the adjoint relation of its transfer operators, the operator on a coarser grid,
an independent solver, dense linear algebra, a Fourier mode, and the mesh-independence a V-cycle
must show.  The V-cycle preconditions CG for div((1/rho) grad p) = f (Sec. 3.4 of
arXiv:1601.05448) on the periodic staggered grid.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import multigrid as MG
import vdp_inputs as V

TWO_PI = 2.0 * math.pi


def test_restriction_is_the_transpose_of_prolongation():
    rng = np.random.default_rng(31)
    xc = rng.standard_normal((3, 4, 5))
    rf = rng.standard_normal((6, 8, 10))
    lhs = float(np.sum(MG.prolong(xc) * rf))
    rhs = float(np.sum(xc * MG.restrict(rf)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.allclose(MG.prolong(np.ones((3, 4, 5))), 1.0, rtol=0, atol=1e-15)  # constants kept
    assert np.allclose(MG.restrict(np.ones((6, 8, 10))), 8.0, rtol=0, atol=1e-14)


def test_prolongation_is_linear_interpolation_between_cell_centres():
    # a field linear along x between coarse centres is reproduced at the fine centres (away from
    # the periodic wrap): coarse centres at 2h(i + 1/2), fine at h(j + 1/2)
    nxc = 8
    xc_pos = 2.0 * (np.arange(nxc) + 0.5)
    xc = np.broadcast_to(xc_pos, (2, 2, nxc)).copy()
    xf = MG.prolong(xc)[0, 0]
    fine_pos = np.arange(2 * nxc) + 0.5
    inner = slice(1, 2 * nxc - 1)
    assert np.allclose(xf[inner], fine_pos[inner], rtol=0, atol=1e-13)


def test_coarse_operator_of_constant_density_is_the_2h_operator_times_8():
    L, shape = 2.0, (8, 12, 16)
    rho = np.full(shape, 3.0)
    b = oracle.face_coefficients(rho, L)
    bc = MG.coarsen(b)
    ref = oracle.face_coefficients(np.full((4, 6, 8), 3.0), L)
    for a, r in zip(bc, ref):
        assert np.allclose(a, 8.0 * r, rtol=1e-14, atol=0)


def test_level_rule_and_supported_sizes():
    assert MG.level_shapes(256, 256, 256)[-1] == (4, 4, 4) and len(MG.level_shapes(256, 256, 256)) == 7
    assert MG.level_shapes(48, 48, 48)[-1] == (3, 3, 3)
    assert MG.level_shapes(80, 80, 80)[-1] == (5, 5, 5)
    assert MG.level_shapes(32, 32, 8)[-1] == (1, 4, 4)
    assert MG.supported(8, 8, 8) and MG.level_shapes(8, 8, 8) == [(8, 8, 8), (4, 4, 4)]
    assert not MG.supported(48, 36, 40)      # stops at 12 x 9 x 10 = 1080 cells
    assert not MG.supported(17, 9, 16)


def test_vcycle_is_the_pseudo_inverse_when_there_is_no_coarser_level():
    rng = np.random.default_rng(32)
    shape, L = (4, 4, 4), 1.5
    rho = V.density_modes(shape, rng, amplitude=0.6)
    H = MG.Hierarchy.from_density(rho, L)
    assert H.nlevels == 1
    r = rng.standard_normal(shape)
    r -= r.mean()
    z = H.vcycle(r)
    p, info = oracle.solve_cg(rho, -r, L, tol=1e-14)        # A p = -r  <=>  (-A) p = r
    assert np.abs(z - p).max() <= 1e-10 * np.abs(p).max()


@pytest.mark.parametrize("shape,ratio", [((8, 8, 8), 10.0), ((8, 8, 16), 4.0), ((6, 6, 6), 30.0)])
def test_vcycle_is_symmetric_positive_definite_on_mean_free_vectors(shape, ratio):
    rng = np.random.default_rng(33)
    a = (ratio - 1.0) / (ratio + 1.0)
    rho = V.density_modes(shape, rng, amplitude=a, kmax=3.0)
    H = MG.Hierarchy.from_density(rho, 2.0)
    assert H.nlevels >= 2
    n = rho.size
    Pm = np.eye(n) - 1.0 / n
    M = np.zeros((n, n))
    for q in range(n):
        M[:, q] = H.vcycle(Pm[:, q].reshape(shape)).ravel()
    M = Pm @ M @ Pm
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-6 * ev[-1]   # one zero (constants), the rest > 0
    # as a preconditioner of -A the spectrum of M(-A) lies in (0, 1]: the cycle never over-corrects
    A = MG.dense_negative_operator(H.b[0])
    lam = np.sort(np.linalg.eigvals(M @ A).real)[1:]
    assert lam.min() > 0.05 and lam.max() <= 1.0 + 1e-9


def _mode_response(H, n, L):
    xs = (np.arange(n) + 0.5) * (L / n)
    e = np.broadcast_to(np.cos(xs), (n, n, n)).copy()
    en = e - H.vcycle(-MG.apply(H.b[0], e))      # error after one cycle, from error e
    keep = float(np.vdot(en, e) / np.vdot(e, e))  # the part of e left
    perp = float(np.linalg.norm(en - keep * e) / np.linalg.norm(e))
    return keep, perp


def test_cycle_keeps_a_fourier_mode_and_two_grid_error_is_second_order():
    # constant density: cos(x) is an eigenvector of A; the cycle must map it (almost) onto itself,
    # and the exact two-grid cycle must remove it, up to an O(h^2) remainder
    L = TWO_PI
    keep16, perp16 = _mode_response(MG.Hierarchy.from_density(np.ones((16,) * 3), L), 16, L)
    assert 0.0 < keep16 < 0.5 and perp16 <= 0.03
    k12, p12 = _mode_response(MG.Hierarchy.from_density(np.ones((12,) * 3), L, max_levels=2), 12, L)
    k24, p24 = _mode_response(MG.Hierarchy.from_density(np.ones((24,) * 3), L, max_levels=2), 24, L)
    assert p12 <= 0.02 and p24 <= 0.005
    assert 0.0 < k24 <= 0.3 * k12 and k12 < 0.2


def test_pcg_reaches_the_oracle_solution_with_mesh_independent_iterations():
    its = []
    for n in (16, 32, 64):
        prob = V.hotspot_problem(n, seed=2, nspots=max(1, round(20000 * n ** 3 / 256 ** 3)), target_ratio=4.0)
        p, info = MG.solve_pcg(prob.rho, prob.f, prob.L, tol=1e-12)
        assert info["status"] == "ok" and info["rel_res"] <= 1e-11
        ref, _ = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
        assert np.linalg.norm(p - ref) <= 1e-9 * np.linalg.norm(ref)
        its.append(info["iters"])
    assert max(its) - min(its) <= 3, its
    assert max(its) <= 25, its


def test_pcg_at_a_high_density_ratio():
    prob = V.hotspot_problem(32, seed=5, nspots=40, target_ratio=50.0)
    p, info = MG.solve_pcg(prob.rho, prob.f, prob.L, tol=1e-10)
    assert info["status"] == "ok"
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, p) <= 1.01e-10


def test_coarse_faces_are_half_the_piecewise_constant_galerkin_faces():
    # P0 = piecewise-constant injection; P0^T (-A) P0 couples two neighbouring coarse cells through
    # exactly the fine faces that lie between them, so its off-diagonal entries give, for any
    # density, which fine faces make up each coarse face (the coarse operator is half of it)
    rng = np.random.default_rng(34)
    shape, L = (8, 8, 8), 1.0
    rho = V.density_modes(shape, rng, amplitude=0.8, kmax=3.0)
    b = oracle.face_coefficients(rho, L)
    A = MG.dense_negative_operator(b)
    cz, cy, cx = 4, 4, 4
    nc = cz * cy * cx
    P0 = np.zeros((rho.size, nc))
    for k in range(8):
        for j in range(8):
            for i in range(8):
                P0[i + 8 * (j + 8 * k), (i // 2) + cx * ((j // 2) + cy * (k // 2))] = 1.0
    G = P0.T @ A @ P0
    bc = MG.coarsen(b)
    for d, (ex, ey, ez) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        for k in range(cz):
            for j in range(cy):
                for i in range(cx):
                    C = i + cx * (j + cy * k)
                    Cm = (i - ex) % cx + cx * ((j - ey) % cy + cy * ((k - ez) % cz))
                    assert abs(-G[C, Cm] - 2.0 * bc[d][k, j, i]) <= 1e-12 * abs(G[C, Cm])


# ---- the inflow-outflow duct: no faces at the x ends, transfers that do not reach across them ---

DUCT = (4.0, 1.0, 1.0, 1)


def test_duct_transfers_are_adjoint_and_keep_constants():
    rng = np.random.default_rng(35)
    xc = rng.standard_normal((3, 4, 5))
    rf = rng.standard_normal((6, 8, 10))
    lhs = float(np.sum(MG.prolong(xc, 1) * rf))
    rhs = float(np.sum(xc * MG.restrict(rf, 1)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.allclose(MG.prolong(np.ones((3, 4, 5)), 1), 1.0, rtol=0, atol=1e-15)
    # nothing crosses the ends: a coarse value at the last x cell does not reach the first fine one
    e = np.zeros((3, 4, 5))
    e[:, :, -1] = 1.0
    assert np.all(MG.prolong(e, 1)[:, :, 0] == 0.0)
    assert np.all(MG.prolong(e, 0)[:, :, 0] > 0.0)   # (it does in the periodic box)


def test_duct_vcycle_is_symmetric_positive_definite():
    rng = np.random.default_rng(36)
    shape = (8, 8, 16)
    rho = V.density_modes(shape, rng, amplitude=(30 - 1) / (30 + 1), kmax=3.0)
    H = MG.Hierarchy.from_density(rho, 0.0, geom=(2.0, 1.0, 1.0, 1))
    n = rho.size
    Pm = np.eye(n) - 1.0 / n
    M = np.zeros((n, n))
    for q in range(n):
        M[:, q] = H.vcycle(Pm[:, q].reshape(shape)).ravel()
    M = Pm @ M @ Pm
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    lam = np.sort(np.linalg.eigvals(M @ MG.dense_negative_operator(H.b[0])).real)[1:]
    assert lam.min() > 0.05 and lam.max() <= 1.0 + 1e-9


def test_duct_pcg_reaches_the_oracle_solution_with_mesh_independent_iterations():
    its = []
    for n in (16, 32):
        prob = V.duct_problem((n, n, 4 * n), DUCT[:3], seed=n)
        p, info = MG.solve_pcg(prob.rho, prob.f, 0.0, tol=1e-11, geom=DUCT)
        ref, _ = oracle.solve_cg(prob.rho, prob.f, 0.0, tol=1e-13, geom=DUCT)
        assert info["status"] == "ok"
        assert np.linalg.norm(p - ref) <= 1e-9 * np.linalg.norm(ref)
        its.append(info["iters"])
    assert max(its) - min(its) <= 2 and max(its) <= 25, its
