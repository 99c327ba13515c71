"""Batch engine: many solves of different sizes, densities and tolerances advanced in the same
launches must give, for every member, exactly the result of solving it alone -- bit for bit,
since each member keeps its own unit layout and fixed-order reductions -- whether the batch runs
as one persistent cooperative kernel or as ordinary launches, and whether members join while
others are running (continuous batching)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1601_05448_gb300 as vdp  # noqa: E402
import vdp_inputs as V  # noqa: E402

DEV = "cuda:0"


def problems():
    return [(V.smooth_problem((16, 16, 24), seed=51), 1e-9),
            (V.smooth_problem((32, 32, 32), seed=52), 1e-10),
            (V.hotspot_problem(40, seed=53, nspots=80, target_ratio=6.0), 1e-8),
            (V.smooth_problem((24, 40, 48), seed=54), 1e-9),
            (V.hotspot_problem(64, seed=55, nspots=312, target_ratio=8.0), 1e-8),
            (V.smooth_problem((8, 12, 96), seed=56), 1e-10)]


def setup(prob, precision):
    nz, ny, nx = prob.shape
    s = vdp.Solver(nx, ny, nz, prob.L, precision=precision)
    s.set_density(torch.from_numpy(prob.rho).to(DEV))
    f = torch.from_numpy(prob.f).to(DEV)
    return s, f


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("precision", ["mixed", "fp64", "mixed_bf16"])
def test_batch_equals_alone(precision, persistent):
    members = []
    for prob, tol in problems():
        s, f = setup(prob, precision)
        p_alone = torch.empty_like(f)
        st_alone = s.solve(f, p_alone, tol)
        members.append((prob, tol, s, f, p_alone, st_alone))
    with vdp.Batch(precision, persistent=persistent) as b:
        outs = []
        for prob, tol, s, f, *_ in members:
            p = torch.full_like(f, 3.0)
            b.add(s, f, p, tol)
            outs.append(p)
        b.run_to_completion(max_pairs=16)
        for (prob, tol, s, f, p_alone, st_alone), p in zip(members, outs):
            assert b.done(s)
            st = s.stats()
            assert st.ok and st.iters == st_alone.iters and st.rel_res <= tol
            assert torch.equal(p, p_alone), prob.name
    for prob, tol, s, *_ in members:
        s.close()


def test_batch_parity_with_oracle():
    prob, tol = problems()[4]
    s, f = setup(prob, "mixed")
    p = torch.empty_like(f)
    with vdp.Batch("mixed") as b:
        b.add(s, f, p, 1e-9)
        b.run_to_completion(max_pairs=32)
    ref, _ = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    err = float(np.linalg.norm(p.cpu().numpy() - ref) / np.linalg.norm(ref))
    assert s.stats().ok and err <= 1e-8
    s.close()


def test_continuous_admission_and_retirement():
    items = problems()
    solvers = [setup(prob, "mixed") for prob, _ in items]
    alone = []
    for (prob, tol), (s, f) in zip(items, solvers):
        p = torch.empty_like(f)
        s.solve(f, p, tol)
        alone.append(p)
    outs = [torch.zeros_like(f) for _, f in solvers]
    with vdp.Batch("mixed", persistent=True) as b:
        # two members first, then the rest join while those are running
        for i in (0, 1):
            b.add(solvers[i][0], solvers[i][1], outs[i], items[i][1])
        b.run(max_pairs=8)
        for i in range(2, len(items)):
            b.add(solvers[i][0], solvers[i][1], outs[i], items[i][1])
            b.run(max_pairs=4)
        finished = set()
        for _ in range(100000):
            active = b.run(max_pairs=8)
            for i, (s, _) in enumerate(solvers):
                if i not in finished and b.done(s):
                    finished.add(i)
                    b.remove(s)  # retire as soon as it is done
            if active == 0:
                break
        assert len(b) == len(items) - len(finished)
    for i, (p, q) in enumerate(zip(outs, alone)):
        assert torch.equal(p, q), items[i][0].name
    for s, _ in solvers:
        s.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_spectral_members_equal_alone(precision):
    """Batch of ordinary launches with spectrally preconditioned and fixed-point members
    (FFT-supported sizes), mixed with a Jacobi member: every result equals its solve alone, bit
    for bit."""
    fp = {"method": vdp.VDP_METHOD_FIXED_POINT}
    probs = [(V.hotspot_problem(32, seed=57, nspots=40, target_ratio=5.0), 1e-9, {"precond": vdp.VDP_PRECOND_SPECTRAL}),
             (V.smooth_problem((48, 32, 64), seed=58), 1e-10, {"precond": vdp.VDP_PRECOND_SPECTRAL}),
             (V.smooth_problem((16, 16, 24), seed=51), 1e-9, {}),
             (V.hotspot_problem(64, seed=59, nspots=312, target_ratio=8.0), 1e-8, {"precond": vdp.VDP_PRECOND_SPECTRAL}),
             (V.hotspot_problem(48, seed=60, nspots=130, target_ratio=6.0), 1e-9, fp),
             (V.smooth_problem((32, 64, 32), seed=61), 1e-10, fp)]
    members = []
    for prob, tol, opts in probs:
        nz, ny, nx = prob.shape
        s = vdp.Solver(nx, ny, nz, prob.L, precision=precision, **opts)
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        f = torch.from_numpy(prob.f).to(DEV)
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
    # every member against the oracle: 1e-9 for FP64 at 1e-10, 1e-8 otherwise
    for (prob, tol, *_), p in zip(members, outs):
        ref, _ = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
        err = np.linalg.norm(p.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= (1e-9 if precision == "fp64" and tol <= 1e-10 else 1e-8), (prob.name, err)
    for _, _, s, *_ in members:
        s.close()


def test_grid_barrier_wait_expires_and_batch_recovers():
    """Failure detection on the GPU without a fault: a run that waits for a block that never
    arrives gives up after the (shortened) wait limit with VDP_ETIMEOUT; the members stay
    usable and finish with exactly the results they have alone."""
    import time
    items = problems()[:2]
    members = []
    for prob, tol in items:
        s, f = setup(prob, "mixed")
        p_alone = torch.empty_like(f)
        s.solve(f, p_alone, tol)
        members.append((prob, tol, s, f, p_alone))
    with vdp.Batch("mixed", persistent=True) as b:
        b.set_wait_limit(0.05)
        outs = []
        for prob, tol, s, f, _ in members:
            p = torch.empty_like(f)
            b.add(s, f, p, tol)
            outs.append(p)
        b.run(2)  # a normal run first
        b.inject_lost_arrival()
        t0 = time.perf_counter()
        with pytest.raises(vdp.VdpError) as e:
            b.run(2)
        assert e.value.status == vdp.VDP_ETIMEOUT and time.perf_counter() - t0 < 5.0
        b.run_to_completion(max_pairs=16)
        for (prob, tol, s, f, p_alone), p in zip(members, outs):
            assert b.done(s) and s.stats().ok
            assert torch.equal(p, p_alone), prob.name
    with vdp.Batch("mixed", persistent=False) as b2:  # no grid barrier to starve
        with pytest.raises(vdp.VdpError):
            b2.inject_lost_arrival()
    for _, _, s, *_ in members:
        s.close()
