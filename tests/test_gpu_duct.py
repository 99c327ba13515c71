"""GPU parity on the inflow-outflow duct (Sec. 3.2 configuration 2: periodic y, z; no pressure flux
through the x ends -- the reading the oracle takes) with per-direction box lengths, through the C
ABI, against the CPU oracle's duct solvers on the same seeded inputs.  Tolerances as in the
periodic box: FP64 relative L2 <= 1e-9 at tol 1e-10, mixed <= 1e-8 at tol 1e-9; the spectral
inverse (FP32 FFTs of the even extension) <= 2e-6 against the oracle's plain cosine transform.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import multigrid as MG  # noqa: E402
import paper_1601_05448_gb300 as vdp  # noqa: E402
import vdp_inputs as V  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _solve(prob, precision="fp64", tol=1e-10, check=True, **opts):
    nz, ny, nx = prob.shape
    Lx, Ly, Lz = prob.info["lengths"]
    with vdp.Solver(nx, ny, nz, Ly, precision=precision, lengths=(Lx, Ly, Lz), bc_x=vdp.VDP_BC_DUCT,
                    **opts) as s:
        s.set_density(_dev(prob.rho))
        p = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
        st = s.solve(_dev(prob.f), p, tol, check=check)
    return p.cpu().numpy(), st


def _geom(prob):
    Lx, Ly, Lz = prob.info["lengths"]
    return (Lx, Ly, Lz, 1)


_REF = {}


def _ref(prob, key):
    if key not in _REF:
        p, info = oracle.solve_cg(prob.rho, prob.f, 0.0, tol=1e-13, geom=_geom(prob))
        assert info["status"] == "ok"
        _REF[key] = p
    return _REF[key]


# (nz, ny, nx), (Lx, Ly, Lz): long ducts, a non-power-of-two cross-section, ragged tiles
DUCTS = [((16, 16, 64), (4.0, 1.0, 1.0)), ((12, 20, 48), (3.0, 1.25, 0.75)), ((8, 9, 40), (5.0, 1.0, 1.0))]


@pytest.mark.parametrize("shape,lengths", DUCTS)
def test_operator_matches_the_oracle(shape, lengths):
    prob = V.duct_problem(shape, lengths, seed=sum(shape))
    nz, ny, nx = shape
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, 1.0, lengths=lengths, bc_x=vdp.VDP_BC_DUCT) as s:
        s.set_density(_dev(prob.rho))
        s.apply(_dev(x), out)
    ref = oracle.apply_rho(prob.rho, 0.0, x, geom=_geom(prob))
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("mixed", 1e-9, 1e-8)])
@pytest.mark.parametrize("shape,lengths", DUCTS)
def test_jacobi_cg_matches_the_oracle(shape, lengths, precision, tol, bound):
    prob = V.duct_problem(shape, lengths, seed=sum(shape))
    p, st = _solve(prob, precision, tol)
    ref = _ref(prob, shape)
    assert st.ok and st.rel_res <= tol
    assert rel(p, ref) <= bound, rel(p, ref)
    assert oracle.relative_residual(prob.rho, 0.0, prob.f, p, geom=_geom(prob)) <= 1.01 * tol


# duct spectral sizes: 2 nx must be an FFT length
SPECTRAL_DUCTS = [((32, 32, 128), (4.0, 1.0, 1.0)), ((32, 48, 64), (2.0, 1.5, 1.0))]


@pytest.mark.parametrize("shape,lengths", SPECTRAL_DUCTS)
def test_inverse_laplacian_is_the_cosine_transform_inverse(shape, lengths):
    nz, ny, nx = shape
    rng = np.random.default_rng(5)
    g = rng.standard_normal(shape)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, 1.0, lengths=lengths, bc_x=vdp.VDP_BC_DUCT) as s:
        s.inverse_laplacian(_dev(g), out)
    ref = oracle.inverse_laplacian(g, 0.0, geom=(*lengths, 1))
    assert rel(out.cpu().numpy(), ref) <= 2e-6, rel(out.cpu().numpy(), ref)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("mixed", 1e-9, 1e-8)])
@pytest.mark.parametrize("shape,lengths", SPECTRAL_DUCTS)
def test_spectral_cg_and_fixed_point_match_the_oracle(shape, lengths, precision, tol, bound):
    prob = V.duct_problem(shape, lengths, seed=sum(shape) + 2)
    ref = _ref(prob, ("spec",) + shape)
    p, st = _solve(prob, precision, tol, precond=vdp.VDP_PRECOND_SPECTRAL)
    assert st.ok and rel(p, ref) <= bound, (st, rel(p, ref))
    pf, stf = _solve(prob, precision, tol, method=vdp.VDP_METHOD_FIXED_POINT)
    assert stf.ok and rel(pf, ref) <= bound, (stf, rel(pf, ref))
    assert oracle.relative_residual(prob.rho, 0.0, prob.f, pf, geom=_geom(prob)) <= 1.01 * tol
    if precision == "fp64":   # the same iteration as the oracle's (its inverse is a plain DCT)
        _, info = oracle.solve_fixed_point(prob.rho, prob.f, 0.0, tol=tol, geom=_geom(prob))
        assert abs(stf.iters - info["iters"]) <= 1, (stf.iters, info["iters"])


def test_duct_limits():
    with pytest.raises(vdp.VdpError):       # 2 x 40 = 80 is not an FFT length
        vdp.Solver(40, 32, 32, 1.0, lengths=(4.0, 1.0, 1.0), bc_x=vdp.VDP_BC_DUCT, precond=vdp.VDP_PRECOND_SPECTRAL)
    with pytest.raises(vdp.VdpError):
        vdp.Solver(64, 32, 32, 1.0, lengths=(4.0, -1.0, 1.0), bc_x=vdp.VDP_BC_DUCT)
    with pytest.raises(vdp.VdpError):
        vdp.Solver(64, 32, 32, 1.0, lengths=(4.0, 1.0, 1.0), bc_x=7)
    prob = V.duct_problem((16, 16, 64), (4.0, 1.0, 1.0), seed=3)
    m = tuple(_dev(np.zeros((16, 16, 64))) for _ in range(3))
    f = torch.empty((16, 16, 64), dtype=torch.float64, device=DEV)
    with vdp.Solver(64, 16, 16, 1.0, lengths=(4.0, 1.0, 1.0), bc_x=vdp.VDP_BC_DUCT) as s:
        s.set_density(_dev(prob.rho))
        assert vdp.vdp_projection_rhs(s.ctx, *m, None, 0.1, f) == vdp.VDP_EINVAL


def test_periodic_box_with_unequal_lengths():
    # vdp_create_bc also serves a periodic box that is not a cube
    prob = V.duct_problem((16, 24, 32), (2.0, 1.0, 0.5), seed=9)
    nz, ny, nx = prob.shape
    with vdp.Solver(nx, ny, nz, 1.0, lengths=(2.0, 1.0, 0.5), bc_x=vdp.VDP_BC_PERIODIC) as s:
        s.set_density(_dev(prob.rho))
        p = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
        st = s.solve(_dev(prob.f), p, 1e-10)
    ref, _ = oracle.solve_cg(prob.rho, prob.f, 0.0, tol=1e-13, geom=(2.0, 1.0, 0.5, 0))
    assert st.ok and rel(p.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("shape,lengths", [((16, 16, 64), (4.0, 1.0, 1.0)), ((12, 20, 48), (3.0, 1.25, 0.75))])
def test_vcycle_in_the_duct_matches_the_oracle_cycle(shape, lengths):
    prob = V.duct_problem(shape, lengths, seed=sum(shape) + 4)
    nz, ny, nx = shape
    g = np.random.default_rng(6).standard_normal(shape)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, 1.0, lengths=lengths, bc_x=vdp.VDP_BC_DUCT) as s:
        s.set_density(_dev(prob.rho))
        s.mg_apply(_dev(g), out)
    ref = MG.Hierarchy.from_density(prob.rho, 0.0, geom=(*lengths, 1)).vcycle(g)
    assert rel(out.cpu().numpy(), ref) <= 2e-5, rel(out.cpu().numpy(), ref)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("mixed", 1e-9, 1e-8)])
def test_cg_mg_in_the_duct_matches_the_oracle(precision, tol, bound):
    prob = V.duct_problem((32, 32, 128), (4.0, 1.0, 1.0), seed=12)
    ref = _ref(prob, "mg")
    p, st = _solve(prob, precision, tol, precond=vdp.VDP_PRECOND_MG)
    assert st.ok and rel(p, ref) <= bound, (st, rel(p, ref))
    if precision == "fp64":
        _, info = MG.solve_pcg(prob.rho, prob.f, 0.0, tol=tol, geom=_geom(prob))
        assert abs(st.iters - info["iters"]) <= 2, (st.iters, info["iters"])
