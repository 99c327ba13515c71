"""vdp_solve_noalloc: the solve for callers that cannot allocate device memory (hosts whose GPU
memory is reserved by a pool or budget manager that forbids side allocations, latency-critical
loops that cannot take cudaMalloc's device-wide synchronisation).  Its intermediates live in a
fixed device array owned by the library, so it is checked against the ordinary vdp_solve entry
point, through the C ABI, on two calls in a row (the second call must not be disturbed by what
the first one left in the shared array).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1601_05448_gb300 as vdp  # noqa: E402
import vdp_inputs as V  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def reference(prob, tol, precision):
    nz, ny, nx = prob.shape
    p = torch.empty(prob.shape, dtype=torch.float64, device=DEV)
    with vdp.Solver(nx, ny, nz, prob.L, precision=precision) as s:
        s.set_density(torch.from_numpy(prob.rho).to(DEV))
        st = s.solve(torch.from_numpy(prob.f).to(DEV), p, tol)
    return p.cpu().numpy(), st


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_noalloc_matches_vdp_solve_twice(precision):
    probs = [V.smooth_problem((32, 32, 32), seed=31), V.hotspot_problem(40, seed=32, nspots=80, target_ratio=6.0)]
    for prob in probs:  # two calls in a row, different sizes and densities
        nz, ny, nx = prob.shape
        ref, st_ref = reference(prob, 1e-10, precision)
        p = torch.full(prob.shape, 123.0, dtype=torch.float64, device=DEV)
        st, stats = vdp.vdp_solve_noalloc(nx, ny, nz, prob.L, torch.from_numpy(prob.rho).to(DEV),
                                          torch.from_numpy(prob.f).to(DEV), p, 1e-10,
                                          vdp.PRECISIONS[precision])
        torch.cuda.synchronize()
        assert st == vdp.VDP_OK and stats.status == vdp.VDP_OK
        assert stats.rel_res <= 1e-10 and stats.iters == st_ref.iters
        assert rel(p.cpu().numpy(), ref) <= 1e-9


def test_noalloc_rejects_oversize_and_host_pointers():
    n = (vdp.VDP_NOALLOC_MAX_CELLS // (64 * 32)) + 1  # one plane too many for 64 x 32 planes
    a = torch.ones((n, 32, 64), dtype=torch.float64, device=DEV)
    st, _ = vdp.vdp_solve_noalloc(64, 32, n, 1.0, a, a, torch.empty_like(a), 1e-8)
    assert st == vdp.VDP_EINVAL
    h = np.ones((8, 8, 8))
    st, _ = vdp.vdp_solve_noalloc(8, 8, 8, 1.0, h, h, np.empty_like(h), 1e-8)
    assert st == vdp.VDP_EINVAL
    # arrays of the wrong size: the binding refuses them before the call
    b = torch.ones((8, 8, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        vdp.vdp_solve_noalloc(8, 8, 8, 1.0, b, b[:-1], torch.empty_like(b), 1e-8)
    # through the C ABI directly, an output whose allocation ends before nx*ny*nz doubles is
    # rejected and left untouched: a 12 MB buffer from cudaMalloc itself (a tensor of torch's
    # caching allocator may sit inside a larger driver allocation), its last 64 doubles passed
    rt = _cudart()
    ptr = ctypes.c_void_p()
    nbytes = 12 << 20
    assert rt.cudaMalloc(ctypes.byref(ptr), ctypes.c_size_t(nbytes)) == 0
    try:
        assert rt.cudaMemset(ptr, ctypes.c_int(0), ctypes.c_size_t(nbytes)) == 0
        tail = ptr.value + nbytes - 64 * 8
        s = vdp.vdp_stats()
        st = vdp.load().vdp_solve_noalloc(8, 8, 8, 1.0, b.data_ptr(), b.data_ptr(), tail, 1e-8, 0, None,
                                          vdp.ctypes.byref(s))
        assert st == vdp.VDP_EINVAL
        host = np.ones(nbytes // 8)
        assert rt.cudaMemcpy(host.ctypes.data_as(ctypes.c_void_p), ptr, ctypes.c_size_t(nbytes), 2) == 0
        assert not host.any()
    finally:
        rt.cudaFree(ptr)


def _cudart():
    """The CUDA runtime the library is linked with (already loaded with it)."""
    vdp.load()
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            lib = ctypes.CDLL(name)
        except OSError:
            continue
        lib.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
        lib.cudaMemset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t]
        lib.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        lib.cudaFree.argtypes = [ctypes.c_void_p]
        return lib
    pytest.skip("CUDA runtime library not found")
