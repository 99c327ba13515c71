"""GPU parity of the multigrid preconditioner (VDP_PRECOND_MG) through the C ABI against the CPU
oracle's V-cycle (oracle/multigrid.py) and its solvers, on the same seeded inputs.

Tolerances: one V-cycle in FP32 against the FP64 oracle cycle, relative L2 <= 2e-5; solves as
everywhere else (FP64 relative L2 <= 1e-9 at tol 1e-10, mixed <= 1e-8 at tol 1e-9), and the CG
iteration count within two of the oracle's V-cycle-preconditioned CG (the FP32 cycle is not
bitwise the FP64 one).
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


# (nz, ny, nx): cubic, non-cubic with a 30-cell coarsest level, FFT-unfriendly 40 and 80
APPLY_SHAPES = [(32, 32, 32), (16, 24, 40), (40, 40, 40), (64, 48, 64), (8, 16, 16)]


@pytest.mark.parametrize("shape", APPLY_SHAPES)
def test_vcycle_matches_the_oracle_cycle(shape):
    rng = np.random.default_rng(sum(shape))
    rho = V.density_modes(shape, rng, amplitude=0.7)
    g = rng.standard_normal(shape)
    L = 2.0
    H = MG.Hierarchy.from_density(rho, L)
    ref = H.vcycle(g)
    nz, ny, nx = shape
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L) as s:
        s.set_density(_dev(rho))
        s.mg_apply(_dev(g), out)
    got = out.cpu().numpy()
    assert H.nlevels == vdp.vdp_mg_levels(nx, ny, nz)
    assert rel(got, ref) <= 2e-5, rel(got, ref)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("mixed", 1e-9, 1e-8)])
@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 40), (40, 40, 40)])
def test_cg_mg_matches_the_oracle(shape, precision, tol, bound):
    prob = V.smooth_problem(shape, seed=sum(shape) + 1)
    nz, ny, nx = shape
    with vdp.Solver(nx, ny, nz, prob.L, precision=precision, precond=vdp.VDP_PRECOND_MG) as s:
        s.set_density(_dev(prob.rho))
        p = torch.empty(shape, dtype=torch.float64, device=DEV)
        st = s.solve(_dev(prob.f), p, tol)
    ref, _ = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    pn = p.cpu().numpy()
    assert st.ok and st.rel_res <= tol
    assert rel(pn, ref) <= bound, rel(pn, ref)
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, pn) <= 1.01 * tol
    if precision == "fp64":
        _, info = MG.solve_pcg(prob.rho, prob.f, prob.L, tol=tol)
        assert abs(st.iters - info["iters"]) <= 2, (st.iters, info["iters"])


def test_cg_mg_iterations_do_not_grow_with_the_grid():
    its = {}
    for n in (32, 64, 128):
        prob = V.hotspot_problem(n, seed=2, nspots=max(1, round(20000 * n ** 3 / 256 ** 3)), target_ratio=4.0)
        with vdp.Solver(n, n, n, prob.L, precision="mixed", precond=vdp.VDP_PRECOND_MG) as s:
            s.set_density(_dev(prob.rho))
            p = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
            st = s.solve(_dev(prob.f), p, 1e-8)
        assert st.ok
        assert oracle.relative_residual(prob.rho, prob.L, prob.f, p.cpu().numpy()) <= 1.01e-8
        its[n] = st.iters
    assert max(its.values()) - min(its.values()) <= 4, its


def test_cg_mg_at_a_high_density_ratio():
    prob = V.hotspot_problem(64, seed=7, nspots=300, target_ratio=50.0)
    rho, f = _dev(prob.rho), _dev(prob.f)
    p = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(64, 64, 64, prob.L, precond=vdp.VDP_PRECOND_MG) as s:
        s.set_density(rho)
        st = s.solve(f, p, 1e-10)
    assert st.ok and st.iters <= 60, st
    ref, _ = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    assert rel(p.cpu().numpy(), ref) <= 1e-9
    with vdp.Solver(64, 64, 64, prob.L) as s2:               # Jacobi-preconditioned CG
        s2.set_density(rho)
        st2 = s2.solve(f, p, 1e-10)
    assert st2.iters >= 5 * st.iters, (st.iters, st2.iters)


def test_mg_timed_solve_equals_solve_and_counts_cycles():
    prob = V.smooth_problem((32, 48, 64), seed=66)
    nz, ny, nx = prob.shape
    rho, f = _dev(prob.rho), _dev(prob.f)
    with vdp.Solver(nx, ny, nz, prob.L, precision="mixed", precond=vdp.VDP_PRECOND_MG) as s:
        s.set_density(rho)
        p1, p2 = torch.empty_like(f), torch.empty_like(f)
        st1 = s.solve(f, p1, 1e-9)
        st2, kinds = s.solve_timed(f, p2, 1e-9)
        assert torch.equal(p1, p2) and st1.iters == st2.iters
        assert kinds["mg"]["launches"] == st2.iters          # one V-cycle per Krylov iteration
        assert kinds["stencil"]["launches"] == st2.iters and kinds["mg"]["ms"] > 0
        # a new density rebuilds the levels
        s.set_density(_dev(prob.rho[::-1].copy()))
        st3 = s.solve(f, p1, 1e-9)
        assert st3.ok
        ref, _ = oracle.solve_cg(prob.rho[::-1].copy(), prob.f, prob.L, tol=1e-13)
        assert rel(p1.cpu().numpy(), ref) <= 1e-8


def test_mg_limits():
    with pytest.raises(vdp.VdpError) as e:      # 36 -> 18 -> 9: the coarsest level is too large
        vdp.Solver(48, 36, 40, 1.0, precond=vdp.VDP_PRECOND_MG)
    assert e.value.status == vdp.VDP_EINVAL
    with pytest.raises(vdp.VdpError):           # no coarser level at all
        vdp.Solver(8, 8, 1, 1.0, precond=vdp.VDP_PRECOND_MG)
    prob = V.smooth_problem((32, 32, 32), seed=3)
    with vdp.Solver(32, 32, 32, prob.L, precond=vdp.VDP_PRECOND_MG) as s:
        g = _dev(prob.f)
        out = torch.empty_like(g)
        assert vdp.vdp_mg_apply(s.ctx, g, out) == vdp.VDP_EINVAL   # no density yet
        s.set_density(_dev(prob.rho))
        p = torch.empty_like(g)
        with vdp.Batch("mixed", persistent=True) as b:     # the persistent kernel has no V-cycle
            s.set_options(precision="mixed")
            with pytest.raises(vdp.VdpError):
                b.add(s, g, p, 1e-8)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_mg_members_in_a_batch_equal_alone(precision):
    """Batch of ordinary launches with V-cycle members of different sizes (FFT-unfriendly 40^3
    among them), a spectral member and a Jacobi member: every result equals its solve alone,
    bit for bit."""
    mg = {"precond": vdp.VDP_PRECOND_MG}
    probs = [(V.smooth_problem((40, 40, 40), seed=71), 1e-9, mg),
             (V.hotspot_problem(64, seed=72, nspots=300, target_ratio=6.0), 1e-8, mg),
             (V.smooth_problem((16, 24, 32), seed=73), 1e-10, mg),
             (V.smooth_problem((32, 32, 32), seed=74), 1e-9, {"precond": vdp.VDP_PRECOND_SPECTRAL}),
             (V.smooth_problem((12, 20, 24), seed=75), 1e-9, {})]
    members = []
    for prob, tol, opts in probs:
        nz, ny, nx = prob.shape
        s = vdp.Solver(nx, ny, nz, prob.L, precision=precision, **opts)
        s.set_density(_dev(prob.rho))
        f = _dev(prob.f)
        p_alone = torch.empty_like(f)
        st_alone = s.solve(f, p_alone, tol)
        members.append((prob, tol, s, f, p_alone, st_alone))
    with vdp.Batch(precision, persistent=False) as b:
        outs = []
        for prob, tol, s, f, *_ in members:
            p = torch.full_like(f, -1.0)
            b.add(s, f, p, tol)
            outs.append(p)
        b.run_to_completion(max_pairs=8)
        for (prob, tol, s, f, p_alone, st_alone), p in zip(members, outs):
            st = s.stats()
            assert st.ok and st.iters == st_alone.iters and st.rel_res <= tol
            assert torch.equal(p, p_alone), prob.name
    ref, _ = oracle.solve_cg(probs[0][0].rho, probs[0][0].f, probs[0][0].L, tol=1e-13)
    assert rel(outs[0].cpu().numpy(), ref) <= 1e-7
    for _, _, s, *_ in members:
        s.close()
