"""GPU parity: the sm_103a library (through its C ABI) against the FP64 CPU oracle on the same
seeded inputs.

Tolerances: relative L2 pressure error <= 1e-9 for the FP64 path and <= 1e-8 for the mixed
FP32/BF16-inside-FP64-refinement paths; the library's own FP64 residual must meet the requested
tolerance, and the oracle's operator must agree that it does.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1601_05448_gb300 as vdp  # noqa: E402
import vdp_inputs as V  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_solve(prob, precision="fp64", tol=None, check=True, **opts):
    nz, ny, nx = prob.shape
    rho = torch.from_numpy(prob.rho).to(DEV)
    f = torch.from_numpy(prob.f).to(DEV)
    p = torch.empty_like(f)
    with vdp.Solver(nx, ny, nz, prob.L, precision=precision, **opts) as s:
        s.set_density(rho)
        st = s.solve(f, p, prob.tol if tol is None else tol, check=check)
    return p.cpu().numpy(), st


_ORACLE = {}


def oracle_solution(prob, key):
    if key not in _ORACLE:
        p, info = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=1e-13)
        assert info["status"] == "ok"
        _ORACLE[key] = p
    return _ORACLE[key]


# (nz, ny, nx): cubic, ragged against the default unit shape, odd y/z, thin, 1-D in x
SHAPES = [(8, 8, 8), (12, 20, 24), (32, 32, 32), (17, 9, 16), (40, 36, 48), (3, 5, 64), (1, 1, 8), (24, 30, 8)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_matches_oracle(shape):
    prob = V.smooth_problem(shape, seed=sum(shape))
    p, st = gpu_solve(prob, "fp64", tol=1e-10)
    ref = oracle_solution(prob, ("smooth", shape))
    assert st.ok and st.rel_res <= 1e-10
    assert rel(p, ref) <= 1e-9, (st, rel(p, ref))
    assert abs(float(p.mean())) <= 1e-13 * float(np.abs(p).max())
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, p) <= 1.01e-10


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (40, 36, 48), (17, 9, 16)])
def test_mixed_matches_oracle(shape, precision):
    prob = V.smooth_problem(shape, seed=sum(shape))
    p, st = gpu_solve(prob, precision, tol=1e-9)
    ref = oracle_solution(prob, ("smooth", shape))
    assert st.ok and st.rel_res <= 1e-9, st
    assert rel(p, ref) <= 1e-8, (st, rel(p, ref))
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, p) <= 1.01e-9


def test_config0_fp64():
    prob = V.config0()
    p, st = gpu_solve(prob, "fp64")
    ref = oracle_solution(prob, "c0")
    err = rel(p, ref)
    print(f"config0 fp64: iters={st.iters} outer={st.outer_iters} rel_res={st.rel_res:.3e} err={err:.3e}")
    assert st.ok and err <= 1e-9


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
def test_config0_mixed(precision):
    prob = V.config0()
    p, st = gpu_solve(prob, precision, tol=1e-8)
    ref = oracle_solution(prob, "c0")
    err = rel(p, ref)
    print(f"config0 {precision} tol 1e-8: iters={st.iters} outer={st.outer_iters} rel_res={st.rel_res:.3e} err={err:.3e}")
    assert st.ok and st.rel_res <= 1e-8
    assert err <= 1e-8, err


def test_hotspot_96_all_precisions():
    prob = V.hotspot_problem(96, seed=21, nspots=int(round(20000 * 96 ** 3 / 256 ** 3)), target_ratio=8.0)
    ref = oracle_solution(prob, "hot96")
    for precision, tol, bound in (("fp64", 1e-10, 1e-9), ("mixed", 1e-9, 1e-8), ("mixed_bf16", 1e-9, 1e-8)):
        p, st = gpu_solve(prob, precision, tol=tol)
        err = rel(p, ref)
        print(f"hot96 {precision}: iters={st.iters} outer={st.outer_iters} rel_res={st.rel_res:.3e} err={err:.3e}")
        assert st.ok and st.rel_res <= tol and err <= bound


def test_operator_matches_oracle():
    prob = V.smooth_problem((20, 12, 16), seed=3)
    nz, ny, nx = prob.shape
    u = np.random.default_rng(1).standard_normal(prob.shape)
    out = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, prob.L) as s:
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        s.apply(torch.from_numpy(u).to(DEV), out)
    ref = oracle.apply_rho(prob.rho, prob.L, u)
    assert rel(out.cpu().numpy(), ref) <= 1e-14


def test_deterministic_and_host_pointers():
    prob = V.smooth_problem((16, 16, 32), seed=9)
    p1, s1 = gpu_solve(prob, "mixed", tol=1e-9)
    p2, s2 = gpu_solve(prob, "mixed", tol=1e-9)
    assert np.array_equal(p1, p2) and s1.iters == s2.iters
    nz, ny, nx = prob.shape
    ph = np.empty_like(prob.f)
    with vdp.Solver(nx, ny, nz, prob.L, precision="mixed") as s:
        s.set_density(prob.rho)            # host pointers: staged by the library
        s.solve(prob.f, ph, 1e-9)
    assert np.array_equal(ph, p1)


def test_compatibility_gauge_and_degenerate_rhs():
    prob = V.smooth_problem((16, 12, 24), seed=4)
    nz, ny, nx = prob.shape
    with vdp.Solver(nx, ny, nz, prob.L) as s:
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        p0 = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
        st0 = s.solve(torch.from_numpy(prob.f).to(DEV), p0, 1e-11)
        p1 = torch.empty_like(p0)
        st1 = s.solve(torch.from_numpy(prob.f + 3.5).to(DEV), p1, 1e-11)  # nonzero mean
        assert abs(st1.rhs_mean - st0.rhs_mean - 3.5) < 1e-12
        assert rel(p1.cpu().numpy(), p0.cpu().numpy()) < 1e-9
        for const in (0.0, 2.0):
            pz = torch.full(prob.shape, 7.0, dtype=torch.float64, device=DEV)
            stz = s.solve(torch.full(prob.shape, const, dtype=torch.float64, device=DEV), pz, 1e-10)
            assert stz.ok and stz.iters == 0 and bool((pz == 0).all())


def test_initial_guess_and_errors():
    prob = V.smooth_problem((8, 8, 16), seed=5)
    nz, ny, nx = prob.shape
    ref = oracle_solution(prob, "guess")
    with vdp.Solver(nx, ny, nz, prob.L, use_guess=1) as s:
        f = torch.from_numpy(prob.f).to(DEV)
        p = torch.from_numpy(ref.copy()).to(DEV)
        with pytest.raises(vdp.VdpError) as e:   # solve before set_density
            s.solve(f, p, 1e-10)
        assert e.value.status == vdp.VDP_EINVAL
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        st = s.solve(f, p, 1e-10)                # the exact answer as a guess: no iteration
        assert st.ok and st.iters == 0 and st.outer_iters == 1
        bad = prob.rho.copy()
        bad[3, 2, 1] = -1.0
        with pytest.raises(vdp.VdpError) as e:
            s.set_density(torch.from_numpy(bad).to(DEV))
        assert e.value.status == vdp.VDP_EDENSITY
        bad[3, 2, 1] = float("nan")
        with pytest.raises(vdp.VdpError):
            s.set_density(torch.from_numpy(bad).to(DEV))
        st = s.solve(f, p, 1e-10)                # previous density kept
        assert st.ok
        with pytest.raises(vdp.VdpError) as e:   # misaligned device pointer
            s.solve(f, torch.empty(prob.f.size + 1, dtype=torch.float64, device=DEV)[1:], 1e-10)
        assert e.value.status == vdp.VDP_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("opts", [{}, {"method": vdp.VDP_METHOD_FIXED_POINT}, {"stencil": 1}],
                         ids=["cg", "fixed_point", "cg_tma_stencil"])
def test_output_buffer_is_not_read(precision, opts):
    """Without use_guess the solve never reads p (the first correction writes it): a p filled with
    NaN gives bitwise the answer of a zeroed p, and a solve that ends before any correction (a
    tolerance the zero start already meets) returns p = 0 -- also with the TMA-staged stencil,
    whose residual sweep stages p in shared memory (the zero start is staged as zeros)."""
    prob = V.smooth_problem((32, 48, 64), seed=70)
    nz, ny, nx = prob.shape
    with vdp.Solver(nx, ny, nz, prob.L, precision=precision, **opts) as s:
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        f = torch.from_numpy(prob.f).to(DEV)
        p0 = torch.zeros(prob.shape, dtype=torch.float64, device=DEV)
        st0 = s.solve(f, p0, 1e-9)
        pn = torch.full(prob.shape, float("nan"), dtype=torch.float64, device=DEV)
        stn = s.solve(f, pn, 1e-9)
        assert st0.ok and torch.equal(p0, pn) and stn.iters == st0.iters
        pz = torch.full(prob.shape, float("nan"), dtype=torch.float64, device=DEV)
        stz = s.solve(f, pz, 2.0)
        assert stz.ok and stz.iters == 0 and bool((pz == 0).all())


def test_iteration_cap_reports_notconv():
    prob = V.smooth_problem((32, 32, 32), seed=6)
    nz, ny, nx = prob.shape
    with vdp.Solver(nx, ny, nz, prob.L, max_iter=5) as s:
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        p = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
        st = s.solve(torch.from_numpy(prob.f).to(DEV), p, 1e-10, check=False)
    assert st.status == vdp.VDP_ENOTCONV and st.iters == 5
    pc = p.cpu().numpy()
    assert np.isfinite(pc).all() and abs(float(pc.mean())) < 1e-12 * float(np.abs(pc).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("degree", [2, 4, 8])
def test_chebyshev_preconditioner_matches_oracle(precision, degree):
    prob = V.hotspot_problem(48, seed=61, nspots=int(round(20000 * 48 ** 3 / 256 ** 3)), target_ratio=6.0)
    tol = 1e-10 if precision == "fp64" else 1e-9
    p_j, st_j = gpu_solve(prob, precision, tol=tol)
    p_c, st_c = gpu_solve(prob, precision, tol=tol, precond=vdp.VDP_PRECOND_CHEB, cheb_degree=degree)
    ref = oracle_solution(prob, "hot48")
    print(f"cheb {precision} k={degree}: iters {st_j.iters} -> {st_c.iters}, sweeps {st_j.sweeps} -> {st_c.sweeps}")
    assert st_c.ok and st_c.rel_res <= tol
    assert rel(p_c, ref) <= (1e-9 if precision == "fp64" else 1e-8)
    assert st_c.iters < st_j.iters  # a polynomial preconditioner cuts the Krylov iterations


def test_chebyshev_degree_one_is_jacobi():
    prob = V.smooth_problem((24, 24, 32), seed=62)
    p_j, st_j = gpu_solve(prob, "fp64", tol=1e-10)
    p_c, st_c = gpu_solve(prob, "fp64", tol=1e-10, precond=vdp.VDP_PRECOND_CHEB, cheb_degree=1)
    assert st_c.iters == st_j.iters and rel(p_c, p_j) < 1e-12


@pytest.mark.parametrize("precision,cheb", [("fp64", 0), ("mixed", 0), ("mixed", 3), ("mixed_bf16", 0)])
def test_timed_solve_is_the_solve(precision, cheb):
    prob = V.smooth_problem((24, 32, 40), seed=63)
    nz, ny, nx = prob.shape
    opts = dict(precond=vdp.VDP_PRECOND_CHEB, cheb_degree=cheb) if cheb else {}
    rho = torch.from_numpy(prob.rho).to(DEV)
    f = torch.from_numpy(prob.f).to(DEV)
    with vdp.Solver(nx, ny, nz, prob.L, precision=precision, **opts) as s:
        s.set_density(rho)
        p1, p2 = torch.empty_like(f), torch.empty_like(f)
        st1 = s.solve(f, p1, 1e-9)
        st2, kinds = s.solve_timed(f, p2, 1e-9)
    assert torch.equal(p1, p2)
    assert (st1.iters, st1.outer_iters, st1.sweeps) == (st2.iters, st2.outer_iters, st2.sweeps)
    # one stencil and one update launch per Krylov iteration, one residual launch per refinement step
    assert kinds["stencil"]["launches"] == st2.iters == kinds["update"]["launches"]
    assert kinds["res64"]["launches"] == st2.outer_iters
    assert (kinds["cheb"]["launches"] > 0) == bool(cheb)
    assert sum(k["launches"] for k in kinds.values()) == st2.sweeps
    for k in kinds.values():
        assert (k["ms"] > 0) == (k["launches"] > 0) and k["ms_min"] <= k["ms_mean"] + 1e-12


# ---- the spectral preconditioner (the paper's constant-coefficient inverse, Sec. 3.4) -----------

# (nz, ny, nx): every supported line length along some axis, including 192 and 256 along x (the
# X passes' half-length complex FFTs of 96 and 128), y and z (the 256^3 and 192^3 workloads)
@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 64, 32), (64, 48, 96), (32, 32, 512), (96, 32, 48),
                                   (256, 32, 32), (32, 256, 64), (192, 48, 32), (32, 192, 32), (32, 32, 256),
                                   (32, 48, 192)])
def test_inverse_laplacian_matches_oracle(shape):
    nz, ny, nx = shape
    L = 2.0 * np.pi
    g = np.random.default_rng(sum(shape)).standard_normal(shape)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L) as s:
        s.inverse_laplacian(torch.from_numpy(g).to(DEV), out)
    ref = oracle.inverse_laplacian(g, L)
    err = rel(out.cpu().numpy(), ref)
    print(f"inverse Laplacian {shape}: rel err {err:.2e}")
    assert err <= 2e-6
    assert abs(float(out.mean())) <= 1e-6 * float(out.abs().max())


def test_inverse_laplacian_fourier_mode_closed_form():
    """A single discrete Fourier mode: L_h^-1 u = u / lambda(k) exactly (up to FP32 rounding)."""
    nz, ny, nx = 32, 48, 64
    L = 3.0
    k = (3, -5, 7)
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) * (L / n) for n in (nz, ny, nx)], indexing="ij")
    u = np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) / L + 0.4)
    lam = -4.0 * sum(np.sin(np.pi * kd / nd) ** 2 / (L / nd) ** 2 for kd, nd in zip(k, (nx, ny, nz)))
    out = torch.empty(u.shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, L) as s:
        s.inverse_laplacian(torch.from_numpy(u).to(DEV), out)
    assert rel(out.cpu().numpy(), u / lam) <= 2e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_spectral_preconditioner_matches_oracle(precision):
    prob = V.hotspot_problem(48, seed=61, nspots=int(round(20000 * 48 ** 3 / 256 ** 3)), target_ratio=6.0)
    tol = 1e-10 if precision == "fp64" else 1e-9
    p_j, st_j = gpu_solve(prob, precision, tol=tol)
    p_s, st_s = gpu_solve(prob, precision, tol=tol, precond=vdp.VDP_PRECOND_SPECTRAL)
    ref = oracle_solution(prob, "hot48")
    err = rel(p_s, ref)
    print(f"spectral {precision}: iters {st_j.iters} -> {st_s.iters} (outer {st_s.outer_iters}), err {err:.2e}")
    assert st_s.ok and st_s.rel_res <= tol
    assert err <= (1e-9 if precision == "fp64" else 1e-8)
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, p_s) <= 1.01 * tol
    assert 4 * st_s.iters < st_j.iters  # the density ratio (6) bounds the condition number


@pytest.mark.parametrize("shape", [(32, 64, 96), (64, 32, 32), (96, 48, 64)])
def test_spectral_preconditioner_shapes(shape):
    prob = V.smooth_problem(shape, seed=sum(shape) + 7)
    p, st = gpu_solve(prob, "fp64", tol=1e-10, precond=vdp.VDP_PRECOND_SPECTRAL)
    ref = oracle_solution(prob, ("smooth", shape))
    assert st.ok and rel(p, ref) <= 1e-9, (st, rel(p, ref))
    pm, stm = gpu_solve(prob, "mixed", tol=1e-9, precond=vdp.VDP_PRECOND_SPECTRAL)
    assert stm.ok and rel(pm, ref) <= 1e-8


def test_spectral_timed_and_limits():
    prob = V.smooth_problem((32, 48, 64), seed=65)
    nz, ny, nx = prob.shape
    rho = torch.from_numpy(prob.rho).to(DEV)
    f = torch.from_numpy(prob.f).to(DEV)
    with vdp.Solver(nx, ny, nz, prob.L, precision="mixed", precond=vdp.VDP_PRECOND_SPECTRAL) as s:
        s.set_density(rho)
        p1, p2 = torch.empty_like(f), torch.empty_like(f)
        st1 = s.solve(f, p1, 1e-9)
        st2, kinds = s.solve_timed(f, p2, 1e-9)
        assert torch.equal(p1, p2) and st1.iters == st2.iters
        # one preconditioner application per Krylov iteration
        napp = kinds["spec_z"]["launches"]
        assert napp == st2.iters
        assert kinds["spec_x"]["launches"] == 2 * napp == kinds["spec_y"]["launches"]
        assert kinds["stencil"]["launches"] == st2.iters
        with vdp.Batch("mixed", persistent=True) as b:  # the persistent kernel has no FFT passes
            with pytest.raises(vdp.VdpError):
                b.add(s, f, p1, 1e-9)
    with pytest.raises(vdp.VdpError) as e:  # 40 is not a supported FFT length
        vdp.Solver(40, 32, 32, 1.0, precond=vdp.VDP_PRECOND_SPECTRAL)
    assert e.value.status == vdp.VDP_EINVAL


# ---- the paper's own fixed-point iteration (Sec. 3.4, Eq. (Pois)) on the GPU ------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("damping", [1.0, 0.8])
def test_fixed_point_matches_oracle_iteration(precision, damping):
    """Same algorithm as the oracle's second solver: the same iteration count (the FP32 spectral
    inverse may move the crossing of the tolerance by one iteration) and the oracle's answer."""
    prob = V.config0()
    _, info = oracle.solve_fixed_point(prob.rho, prob.f, prob.L, tol=1e-10, maxit=500, omega=damping)
    assert info["status"] == "ok"
    p, st = gpu_solve(prob, precision, tol=1e-10, method=vdp.VDP_METHOD_FIXED_POINT, damping=damping)
    ref = oracle_solution(prob, "c0")
    err = rel(p, ref)
    print(f"fixed point {precision} damping {damping}: gpu {st.iters} iters, oracle {info['iters']}, err {err:.2e}")
    assert st.ok and st.rel_res <= 1e-10
    if precision == "fp64":  # the FP64 residual recursion follows the oracle's iteration exactly
        assert abs(st.iters - info["iters"]) <= 1
    else:  # FP32 inner steps to 1e-4, checked by FP64 residuals: a few steps past the oracle's
        assert info["iters"] - 1 <= st.iters <= info["iters"] + 4
    assert err <= 1e-9
    assert oracle.relative_residual(prob.rho, prob.L, prob.f, p) <= 1.01e-10


def test_fixed_point_on_hot_spots_and_its_limits():
    prob = V.hotspot_problem(64, seed=66, nspots=312, target_ratio=3.0)
    _, info = oracle.solve_fixed_point(prob.rho, prob.f, prob.L, tol=1e-9, maxit=2000)
    p, st = gpu_solve(prob, "fp64", tol=1e-9, method=vdp.VDP_METHOD_FIXED_POINT, check=False)
    print(f"fixed point hot spots ratio 3: gpu {st.iters} ({vdp.vdp_strerror(st.status)}), oracle {info['iters']} "
          f"({info['status']})")
    if info["status"] == "ok":
        assert st.ok and abs(st.iters - info["iters"]) <= 1
        assert rel(p, oracle_solution(prob, "hot64r3")) <= 1e-8
    else:
        assert st.status == vdp.VDP_ENOTCONV and np.isfinite(p).all()
    nz, ny, nx = prob.shape
    with vdp.Solver(nx, ny, nz, prob.L) as s:  # the density weight is taken at vdp_set_density
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        s.set_options(method=vdp.VDP_METHOD_FIXED_POINT)
        f = torch.from_numpy(prob.f).to(DEV)
        with pytest.raises(vdp.VdpError) as e:
            s.solve(f, torch.empty_like(f), 1e-9)
        assert e.value.status == vdp.VDP_EINVAL
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        st2 = s.solve(f, torch.empty_like(f), 1e-9, check=False)
        assert st2.iters == st.iters
    with pytest.raises(vdp.VdpError):
        vdp.Solver(40, 32, 32, 1.0, method=vdp.VDP_METHOD_FIXED_POINT)
    with pytest.raises(vdp.VdpError):
        vdp.Solver(32, 32, 32, 1.0, method=vdp.VDP_METHOD_FIXED_POINT, damping=2.5)


@pytest.mark.parametrize("opts", [{}, {"precond": vdp.VDP_PRECOND_SPECTRAL}, {"method": vdp.VDP_METHOD_FIXED_POINT}])
def test_device_loop_equals_polling_schedule(opts):
    """The device-side solve loop (one graph launch per solve) and the host-polled schedule run
    the same kernels in the same order: bitwise the same pressure and iteration counts."""
    prob = V.smooth_problem((32, 48, 64), seed=67)
    p_dev, st_dev = gpu_solve(prob, "mixed", tol=1e-9, **opts)
    p_host, st_host = gpu_solve(prob, "mixed", tol=1e-9, steps_per_sync=16, **opts)
    print(f"device loop {st_dev.launches} launches, polling {st_host.launches}")
    assert np.array_equal(p_dev, p_host)
    assert (st_dev.iters, st_dev.outer_iters, st_dev.sweeps) == (st_host.iters, st_host.outer_iters, st_host.sweeps)


@pytest.mark.parametrize("slab", [1, 7, 16])
def test_spectral_slabs_change_nothing(slab):
    """The spectral passes run slab by slab (X+ / Y+ and Y- / X- alternating over groups of z
    planes) give bitwise the answer of one whole-grid application: the inverse alone, the paper's
    iteration and spectral CG, including an uneven last slab."""
    prob = V.hotspot_problem(48, seed=68, nspots=130, target_ratio=5.0)
    nz, ny, nx = prob.shape
    g = torch.from_numpy(np.random.default_rng(5).standard_normal(prob.shape)).to(DEV)
    outs = []
    for sl in (0, slab):
        with vdp.Solver(nx, ny, nz, prob.L, spec_slab=sl) as s:
            o = torch.empty_like(g)
            s.inverse_laplacian(g, o)
            outs.append(o)
    assert torch.equal(outs[0], outs[1])
    for opts in ({"method": vdp.VDP_METHOD_FIXED_POINT}, {"precond": vdp.VDP_PRECOND_SPECTRAL}):
        p0, st0 = gpu_solve(prob, "mixed", tol=1e-9, **opts)
        p1, st1 = gpu_solve(prob, "mixed", tol=1e-9, spec_slab=slab, **opts)
        assert np.array_equal(p0, p1) and st0.iters == st1.iters
    with vdp.Solver(nx, ny, nz, prob.L, spec_slab=slab, method=vdp.VDP_METHOD_FIXED_POINT) as s:
        assert s.spectral_slabs() == (nz + slab - 1) // slab
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        f = torch.from_numpy(prob.f).to(DEV)
        p2 = torch.empty_like(f)
        st2, kinds = s.solve_timed(f, p2, 1e-9)
        assert kinds["spec_z"]["launches"] == st2.iters
        assert kinds["spec_x"]["launches"] == 2 * s.spectral_slabs() * st2.iters
