"""The served stream's request inputs (host logic, no GPU): each request gets its seeded field
set, its exact density ratio and seeded periodic shifts; the benchmark's batched torch version of
the density-ratio bisection returns the host recipe's scales bit for bit."""
import numpy as np
import pytest

import vdp_inputs as V

torch = pytest.importorskip("torch")


def test_request_fields_hit_the_ratio_and_are_seeded():
    reqs = [r for r in V.config4_requests(60) if r.n <= 64][:6]
    assert reqs
    for r in reqs:
        draw = V.request_draw(r)
        assert draw == V.request_draw(r)                       # seeded
        bank = V.serve_bank(r.n, draw[0])
        rho, f = V.request_fields(r, bank, draw)
        assert rho.shape == (r.n, r.n, r.n) and rho.min() > 0
        assert abs(rho.max() / rho.min() - r.ratio) <= 1e-12 * r.ratio
        assert np.array_equal(np.sort(f.ravel()), np.sort(bank[2].ravel()))   # a shift of f
        assert abs(float(f.mean())) <= 1e-13 * float(np.abs(f).max())


def test_batched_bisection_equals_the_host_recipe():
    import bench
    base, H, _ = V.serve_bank(32, 1)
    goals = [2.0, 3.7, 6.25, 9.99, 5.0]
    host = [V.hotspot_scale(base, H, g) for g in goals]
    dev = bench.gpu_hotspot_scales(torch, torch.from_numpy(base), torch.from_numpy(H), goals, chunk=2)
    assert dev == host
