"""GPU parity of the projection steps around the solve (App. A: the Poisson right side; Eq. (mom):
the momentum correction), through the C ABI, against the FP64 CPU oracle on the same seeded
inputs.

Tolerances: the right side and the correction are single FP64 passes, compared element by
element within a few units in the last place of the largest term that enters each cell (the two
sides round 1/rho_face, 1/h and 1/c in different orders); the whole projection is checked by the
App. A divergence constraint on the corrected velocity (to the solve's tolerance) and by the
pressure against the oracle's solve (relative L2 <= 1e-9 in FP64).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1601_05448_gb300 as vdp  # noqa: E402
import vdp_inputs as V  # noqa: E402

DEV = "cuda:0"
EPS = np.finfo(np.float64).eps
TWO_PI = 2.0 * math.pi


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _face_density(rho, d):
    return 0.5 * (np.roll(rho, 1, axis=2 - d) + rho)


def _rhs_scale(rho, m, rd, c, L):
    """Per cell: the sum of the magnitudes of every term of the right side (a rounding bound)."""
    nz, ny, nx = rho.shape
    h = (L / nx, L / ny, L / nz)
    s = np.zeros_like(rho) if rd is None else np.abs(rd)
    for d in range(3):
        u = np.abs(m[d] / _face_density(rho, d)) / h[d]
        s = s + u + np.roll(u, -1, axis=2 - d)
    return s / c


def _inputs(shape, seed, L, amplitude=0.6, with_div=True):
    rng = np.random.default_rng(seed)
    rho = V.density_modes(shape, rng, amplitude=amplitude)
    m = V.face_momenta(shape, L, rng)
    rd = V.divergence_target(shape, rng) if with_div else None
    return rho, m, rd


# (nz, ny, nx): cubic, ragged against the 32 x 8 column tiles, odd and thin, 1-D in x
SHAPES = [(32, 32, 32), (20, 18, 40), (17, 9, 16), (3, 5, 64), (1, 1, 8), (64, 48, 48)]


@pytest.mark.parametrize("with_div", [True, False])
@pytest.mark.parametrize("shape", SHAPES)
def test_projection_rhs_matches_oracle(shape, with_div):
    L, c = TWO_PI, 0.5 * 2e-3
    rho, m, rd = _inputs(shape, sum(shape) + 3, L, with_div=with_div)
    ref = oracle.projection_rhs(rho, m, rd, c, L)
    nz, ny, nx = shape
    f = torch.empty(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L) as s:
        s.set_density(_dev(rho))
        s.projection_rhs(tuple(_dev(x) for x in m), None if rd is None else _dev(rd), c, f)
    err = np.abs(f.cpu().numpy() - ref)
    bound = 16 * EPS * _rhs_scale(rho, m, rd, c, L)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("shape", SHAPES)
def test_projection_correct_matches_oracle(shape):
    L, c = 3.0, 0.25
    rng = np.random.default_rng(sum(shape) + 5)
    p = rng.standard_normal(shape)
    m = V.face_momenta(shape, L, rng)
    ref = oracle.projection_correct(p, m, c, L)
    nz, ny, nx = shape
    md = tuple(_dev(x) for x in m)
    with vdp.Solver(nx, ny, nz, L) as s:          # needs no density
        s.projection_correct(_dev(p), c, md)
    h = (L / nx, L / ny, L / nz)
    for d in range(3):
        got = md[d].cpu().numpy()
        scale = np.abs(m[d]) + c * (np.abs(p) + np.abs(np.roll(p, 1, axis=2 - d))) / h[d]
        assert np.all(np.abs(got - ref[d]) <= 8 * EPS * scale)


def _check_projection(rho, m, rd, c, L, m_new, p, tol, p_tol=1e-9):
    # App. A: div u_new = RHS^div - <RHS^div> to the solve's tolerance
    f = oracle.projection_rhs(rho, m, rd, c, L)
    d0 = c * (f - f.mean())
    div = oracle.divergence(oracle.face_velocity(rho, m_new), L)
    target = np.zeros_like(rho) if rd is None else rd - rd.mean()
    err = float(np.linalg.norm(div - target))
    assert err <= 1.01 * tol * float(np.linalg.norm(d0)), err / float(np.linalg.norm(d0))
    # the correction is exactly Eq. (mom) with the returned pressure
    ref_m = oracle.projection_correct(p, m, c, L)
    for a, b in zip(m_new, ref_m):
        assert np.abs(a - b).max() <= 64 * EPS * np.abs(b).max()
    # and the pressure is the oracle's
    p_ref, info = oracle.solve_cg(rho, f, L, tol=1e-13)
    assert float(np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref)) <= p_tol


@pytest.mark.parametrize("shape", [(32, 32, 32), (20, 18, 40), (17, 9, 16)])
def test_project_fp64_cg(shape):
    L, c, tol = TWO_PI, 1e-3, 1e-11
    rho, m, rd = _inputs(shape, sum(shape) + 7, L)
    nz, ny, nx = shape
    md = tuple(_dev(x) for x in m)
    p = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L) as s:
        s.set_density(_dev(rho))
        st = s.project(md, _dev(rd), c, tol, p)
    assert st.ok and st.rel_res <= tol
    assert abs(-c * st.rhs_mean - float(rd.mean())) <= 1e-9 * abs(float(rd.mean()))  # chi of App. A
    _check_projection(rho, m, rd, c, L, tuple(x.cpu().numpy() for x in md), p.cpu().numpy(), tol)


@pytest.mark.parametrize("precision,method,precond,tol,p_tol", [
    ("fp64", vdp.VDP_METHOD_FIXED_POINT, vdp.VDP_PRECOND_SPECTRAL, 1e-10, 1e-9),
    ("fp64", vdp.VDP_METHOD_CG, vdp.VDP_PRECOND_SPECTRAL, 1e-10, 1e-9),
    ("mixed", vdp.VDP_METHOD_FIXED_POINT, vdp.VDP_PRECOND_SPECTRAL, 1e-9, 1e-8),
])
def test_project_with_solver_options(precision, method, precond, tol, p_tol):
    shape, L, c = (64, 48, 64), TWO_PI, 0.5e-3
    rho, m, rd = _inputs(shape, 41, L, amplitude=0.6)
    nz, ny, nx = shape
    md = tuple(_dev(x) for x in m)
    p = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L, precision=precision, method=method, precond=precond) as s:
        s.set_density(_dev(rho))
        st = s.project(md, _dev(rd), c, tol, p)
    assert st.ok and st.rel_res <= tol, st
    _check_projection(rho, m, rd, c, L, tuple(x.cpu().numpy() for x in md), p.cpu().numpy(), tol, p_tol)


def test_project_full_size_256():
    """The 256^3 hot-spot density (ratio 4) with random face momenta and a divergence target."""
    prob = V.config1()
    L, c, tol = prob.L, 0.5e-3, 1e-10
    rng = np.random.default_rng(77)
    m = V.face_momenta(prob.shape, L, rng)
    rd = V.divergence_target(prob.shape, rng)
    nz, ny, nx = prob.shape
    md = tuple(_dev(x) for x in m)
    f = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
    p = torch.zeros(prob.shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L, method=vdp.VDP_METHOD_FIXED_POINT,
                    precond=vdp.VDP_PRECOND_SPECTRAL) as s:
        s.set_density(_dev(prob.rho))
        s.projection_rhs(md, _dev(rd), c, f)
        ref = oracle.projection_rhs(prob.rho, m, rd, c, L)
        err = np.abs(f.cpu().numpy() - ref)
        assert np.all(err <= 16 * EPS * _rhs_scale(prob.rho, m, rd, c, L))
        st = s.project(md, _dev(rd), c, tol, p)
    assert st.ok and st.rel_res <= tol
    m_new = tuple(x.cpu().numpy() for x in md)
    pn = p.cpu().numpy()
    d0 = c * (ref - ref.mean())
    div = oracle.divergence(oracle.face_velocity(prob.rho, m_new), L)
    assert float(np.linalg.norm(div - (rd - rd.mean()))) <= 1.01 * tol * float(np.linalg.norm(d0))
    ref_m = oracle.projection_correct(pn, m, c, L)
    for a, b in zip(m_new, ref_m):
        assert np.abs(a - b).max() <= 64 * EPS * np.abs(b).max()


def test_project_leaves_momenta_alone_when_the_solve_fails():
    shape, L, c = (16, 16, 16), 1.0, 0.1
    rho, m, rd = _inputs(shape, 5, L, amplitude=0.8)
    md = tuple(_dev(x) for x in m)
    p = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(16, 16, 16, L, max_iter=1) as s:
        s.set_density(_dev(rho))
        st = s.project(md, _dev(rd), c, 1e-12, p, check=False)
    assert st.status == vdp.VDP_ENOTCONV
    for a, b in zip(md, m):
        assert np.array_equal(a.cpu().numpy(), b)


def test_projection_argument_errors():
    shape, L = (8, 8, 8), 1.0
    rho, m, rd = _inputs(shape, 9, L)
    md = tuple(_dev(x) for x in m)
    f = torch.empty(shape, dtype=torch.float64, device=DEV)
    p = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(8, 8, 8, L) as s:
        # no density yet
        assert vdp.vdp_projection_rhs(s.ctx, *md, None, 0.1, f) == vdp.VDP_EINVAL
        assert vdp.vdp_project(s.ctx, *md, None, 0.1, 1e-8, p) == vdp.VDP_EINVAL
        s.set_density(_dev(rho))
        for c in (0.0, -1.0, float("nan"), float("inf")):
            assert vdp.vdp_projection_rhs(s.ctx, *md, None, c, f) == vdp.VDP_EINVAL
            assert vdp.vdp_projection_correct(s.ctx, p, c, *md) == vdp.VDP_EINVAL
            assert vdp.vdp_project(s.ctx, *md, None, c, 1e-8, p) == vdp.VDP_EINVAL
        # host arrays and aliasing
        assert vdp.vdp_projection_rhs(s.ctx, m[0], *md[1:], None, 0.1, f) == vdp.VDP_EINVAL
        assert vdp.vdp_projection_rhs(s.ctx, *md, None, 0.1, md[0]) == vdp.VDP_EINVAL
        assert vdp.vdp_projection_correct(s.ctx, md[0], 0.1, *md) == vdp.VDP_EINVAL
        assert vdp.vdp_projection_correct(s.ctx, p, 0.1, md[0], md[0], md[2]) == vdp.VDP_EINVAL
        assert vdp.vdp_project(s.ctx, *md, None, 0.1, 0.0, p) == vdp.VDP_EINVAL
        # the context still works afterwards
        s.projection_rhs(md, None, 0.1, f)
        assert torch.isfinite(f).all()


def test_project_timed_equals_project():
    shape, L, c = (32, 32, 32), TWO_PI, 1e-3
    rho, m, rd = _inputs(shape, 12, L)
    outs = []
    for timed in (False, True):
        md = tuple(_dev(x) for x in m)
        p = torch.zeros(shape, dtype=torch.float64, device=DEV)
        with vdp.Solver(32, 32, 32, L) as s:
            s.set_density(_dev(rho))
            if timed:
                st, ms = s.project_timed(md, _dev(rd), c, 1e-10, p)
                assert ms["rhs_ms"] > 0 and ms["correct_ms"] > 0 and ms["solve_ms"] > 0
            else:
                st = s.project(md, _dev(rd), c, 1e-10, p)
        outs.append((st.iters, p.cpu().numpy(), [x.cpu().numpy() for x in md]))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])
    for a, b in zip(outs[0][2], outs[1][2]):
        assert np.array_equal(a, b)
