"""Serving loop (continuous batching with HBM-budget admission) and the layout autotuner.

Every served result must equal the same request solved alone (bitwise: the batch engine keeps
each member's arithmetic), requests that arrive while others run must join them, and the memory
held by resident contexts must stay within the budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1601_05448_gb300 as vdp  # noqa: E402
import vdp_inputs as V  # noqa: E402
from paper_1601_05448_gb300 import serve, tune  # noqa: E402

DEV = "cuda:0"


def request_stream(count=12, seed=7):
    rng = np.random.default_rng(seed)
    shapes = [(16, 16, 16), (24, 32, 32), (40, 40, 40), (48, 48, 48), (32, 32, 64)]
    t = np.cumsum(rng.exponential(0.004, size=count))
    reqs = []
    for j in range(count):
        shape = shapes[rng.integers(0, len(shapes))]
        prob = V.smooth_problem(shape, seed=300 + j, amplitude=float(rng.uniform(0.3, 0.8)))
        tol = float(10.0 ** rng.uniform(-10, -7))
        reqs.append(serve.ServeRequest(j, float(t[j]), prob.shape, prob.L, prob.rho, prob.f, tol))
    return reqs


def solve_alone(req, precision, precond="jacobi"):
    nz, ny, nx = req.shape
    fft = precond != "jacobi" and vdp.spectral_supported(nx, ny, nz)
    mg = precond != "jacobi" and not fft and vdp.vdp_mg_levels(nx, ny, nz) > 0
    opts = {"precond": vdp.VDP_PRECOND_SPECTRAL if fft else (vdp.VDP_PRECOND_MG if mg else 0), "inner_tol": 1e-4}
    if fft and precond == "fixed_point":
        opts["method"] = vdp.VDP_METHOD_FIXED_POINT
    with vdp.Solver(nx, ny, nz, req.L, precision=precision, **opts) as s:
        s.set_density(torch.from_numpy(req.rho).to(DEV))
        p = torch.empty(req.shape, dtype=torch.float64, device=DEV)
        st = s.solve(torch.from_numpy(req.f).to(DEV), p, req.tol)
    return p, st


@pytest.mark.parametrize("mode,persistent,precond", [("batch", True, "jacobi"), ("batch", False, "jacobi"),
                                                    ("batch", False, "spectral"), ("batch", False, "fixed_point"),
                                                    ("streams", False, "fixed_point"), ("streams", False, "jacobi")])
def test_served_results_equal_alone(mode, persistent, precond):
    reqs = request_stream()
    seen_overlap = []

    with serve.Server("mixed", max_active=4 if mode == "streams" else 8, pairs_per_run=4, persistent=persistent,
                      precond=precond, mode=mode) as srv:
        if mode == "streams":  # contexts made before the stream, as the benchmark does
            assert srv.warm(sorted({r.shape for r in reqs}), reqs[0].L) > 0
        stats = srv.run(reqs, on_done=lambda r: seen_overlap.append(r.t_admit))
    s = stats.summary()
    assert s["completed"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    # continuous batching: some request was admitted before an earlier one finished
    assert any(b.t_admit < a.t_done for a in reqs for b in reqs if b.arrival_s > a.arrival_s)
    for r in reqs:
        assert r.status == vdp.VDP_OK
        p, st = solve_alone(r, "mixed", precond)
        assert st.iters == r.iters
        assert torch.equal(p, r.p), r.rid


def test_hbm_budget_admission():
    reqs = request_stream(count=8, seed=11)
    budget = 2 * serve.BYTES_PER_CELL * 48 ** 3  # room for about two of the larger contexts
    with serve.Server("mixed", hbm_budget=budget, max_active=8, pairs_per_run=4, precond="jacobi") as srv:
        stats = srv.run(reqs)
    assert stats.completed == len(reqs) and stats.peak_bytes <= budget
    # every served pressure against the oracle, at the accuracy its tolerance states (mixed
    # precision: 1e-8 for requests asking 1e-8 or less, the request's tolerance above that)
    for r in reqs:
        ref, _ = oracle.solve_cg(r.rho, r.f, r.L, tol=1e-13)
        err = np.linalg.norm(r.p.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= max(r.tol, 1e-8), (r.rid, r.tol, err)


def test_autotuner_picks_a_valid_layout(tmp_path, monkeypatch):
    monkeypatch.setenv("VDP_TUNE_CACHE", str(tmp_path / "tune.json"))
    prob = V.smooth_problem((32, 32, 64), seed=12)
    nz, ny, nx = prob.shape
    rho = torch.from_numpy(prob.rho).to(DEV)
    f = torch.from_numpy(prob.f).to(DEV)
    best = tune.tune(nx, ny, nz, prob.L, rho, f, "mixed", iters=20)
    assert tune.cached_options(nx, ny, nz, "mixed") == best
    with vdp.Solver(nx, ny, nz, prob.L, precision="mixed", **best) as s:
        s.set_density(rho)
        p = torch.empty_like(f)
        st = s.solve(f, p, 1e-9)
    ref, _ = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
    assert st.ok and np.linalg.norm(p.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-8


def test_rejection_and_cancellation():
    """Host-side failure handling: a request larger than the whole HBM budget is rejected with
    VDP_ENOMEM at once instead of waiting forever; a request cancelled while queued or running
    leaves with status CANCELLED; everything else completes and matches its solve alone."""
    reqs = request_stream(count=8, seed=13)
    big = V.smooth_problem((64, 64, 64), seed=14)
    reqs.append(serve.ServeRequest(100, 0.0, big.shape, big.L, big.rho, big.f, 1e-8))
    budget = 2 * serve.BYTES_PER_CELL * 48 ** 3
    victim = max(r.rid for r in reqs if r.rid != 100)
    with serve.Server("mixed", hbm_budget=budget, max_active=4, pairs_per_run=2, precond="jacobi") as srv:
        stats = srv.run(reqs, on_done=lambda r: srv.cancel(victim))
    by_id = {r.rid: r for r in reqs}
    assert by_id[100].status == vdp.VDP_ENOMEM and stats.rejected == 1
    assert stats.cancelled <= 1
    if stats.cancelled:
        assert by_id[victim].status == serve.CANCELLED
    for r in reqs:
        if r.rid in (100,) or r.status == serve.CANCELLED:
            continue
        assert r.status == vdp.VDP_OK
        p, st = solve_alone(r, "mixed")
        assert torch.equal(p, r.p) and st.iters == r.iters
    assert stats.completed + stats.rejected + stats.cancelled == len(reqs)
