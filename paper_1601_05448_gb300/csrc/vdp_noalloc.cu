// vdp_noalloc.cu -- vdp_solve_noalloc: a complete small solve that allocates no device memory.
//
// Who needs this.  Some callers cannot call cudaMalloc: hosts whose device memory is owned by a
// pool or budget manager that reserves the GPU up front and forbids side allocations (there a
// cudaMalloc fails, or takes memory the manager has promised to someone else), and latency-
// sensitive loops that cannot take the implicit device-wide synchronisation of cudaMalloc and
// cudaFree.  vdp_solve_noalloc serves them: the caller passes rho, rhs and p; every intermediate
// the solve needs (face coefficients, Jacobi scaling, Krylov vectors, partial sums, solver state)
// lives in one file-scope __device__ array of fixed size that the CUDA runtime creates when the
// library is loaded, on every GPU that loads it, and keeps until the process exits.
//
// The solve runs the same kernels, unit layout and state machine as vdp_solve with default
// options, so the two return the same pressure.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "vdp.h"
#include "vdp_internal.cuh"
#include "vdp_launch.h"

using namespace vdp;

namespace {

constexpr long long kMaxCells = VDP_NOALLOC_MAX_CELLS;
constexpr int kMaxUnits = kMaxCells / 8 + 16;  // stencil units (<= ny*nz) plus flat units (<= 16)
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array for kMaxCells cells (offsets in bytes).
constexpr size_t kF64 = align_up(sizeof(double) * kMaxCells);     // one FP64 field
constexpr size_t kBf16 = align_up(sizeof(uint16_t) * kMaxCells);  // the BF16 diagonal correction
constexpr size_t kOffFields = 0;  // bx by bz sinv sx sy sz x r d0 d1 q dg
constexpr size_t kNumF64 = 13;
constexpr size_t kOffSd = kOffFields + kNumF64 * kF64;
constexpr size_t kOffPart = kOffSd + kBf16;
constexpr size_t kOffUnits = kOffPart + align_up(sizeof(double) * kSlots * kMaxUnits);
constexpr size_t kOffDesc = kOffUnits + align_up(sizeof(UnitRef) * kMaxUnits);
constexpr size_t kOffState = kOffDesc + align_up(sizeof(InstDesc));
constexpr size_t kOffTicket = kOffState + align_up(sizeof(InstState));
constexpr size_t kOffFlag = kOffTicket + kAlign;
constexpr size_t kScratchBytes = kOffFlag + kAlign;

// The scratch array.  In host code its name is only a host-side stand-in, not a device address
// (a kernel given it would fault, or silently use the wrong memory); the device address comes
// from cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;

// Driver calls reached through the runtime's entry-point lookup (the library does not link
// libcuda directly, so it still loads on machines without a driver).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
using MemGetAddressRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
MemGetAddressRangeFn g_addr_range = nullptr;
bool g_driver_looked_up = false;

template <class F>
bool driver_fn(const char* name, F* out) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  *out = reinterpret_cast<F>(fn);
  return true;
}

bool driver_ready() {  // called with g_mu held
  if (!g_driver_looked_up) {
    g_driver_looked_up = true;
    if (!driver_fn("cuCtxGetCurrent", &g_ctx_current) || !driver_fn("cuCtxGetId", &g_ctx_id) ||
        !driver_fn("cuMemGetAddressRange", &g_addr_range)) {
      g_ctx_current = nullptr;
      g_ctx_id = nullptr;
      g_addr_range = nullptr;
    }
  }
  return g_ctx_current && g_ctx_id && g_addr_range;
}

// The symbol address is looked up once per device and context: a context that was torn down
// and created again (cudaDeviceReset) gets a new id, and with it a fresh lookup, since the
// module -- and so the array -- may then sit at another address.
struct Slot {
  unsigned long long ctx_id = 0;
  unsigned char* base = nullptr;
};
Slot g_slot[kMaxDevices];

// Device address of the scratch array in the current device's current context.
int scratch_base(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VDP_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!driver_ready()) return VDP_ECUDA;
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS) return VDP_ECUDA;
  void* p = nullptr;
  if (!ctx) {  // no context current yet: the runtime creates the primary one on this lookup
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VDP_ECUDA;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return VDP_ECUDA;
  }
  unsigned long long id = 0;
  if (g_ctx_id(ctx, &id) != CUDA_SUCCESS) return VDP_ECUDA;
  Slot& sl = g_slot[dev];
  if (!sl.base || sl.ctx_id != id) {
    if (!p && (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)) return VDP_ECUDA;
    sl.base = static_cast<unsigned char*>(p);
    sl.ctx_id = id;
  }
  *out = sl.base;
  return VDP_OK;
}

// True when p is device (or managed) memory of the current device and the allocation it lies
// in holds at least `bytes` bytes from p on.
bool on_this_device(const void* p, size_t bytes) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (!(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) return false;
  if (a.type == cudaMemoryTypeDevice && a.device != dev) return false;
  CUdeviceptr base = 0;
  size_t size = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!driver_ready()) return false;
    if (g_addr_range(&base, &size, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return false;
  }
  const uintptr_t lo = (uintptr_t)p, end = (uintptr_t)base + size;
  return lo >= (uintptr_t)base && lo <= end && end - lo >= bytes;
}

#define NA_CK(call)                             \
  do {                                          \
    if ((call) != cudaSuccess) return VDP_ECUDA; \
  } while (0)

}  // namespace

static_assert(sizeof(InstState) <= kAlign, "scratch slots");
static_assert(kScratchBytes == VDP_NOALLOC_SCRATCH_BYTES, "keep the header's size in sync");

extern "C" int vdp_solve_noalloc(int nx, int ny, int nz, double L, const double* rho,
                                 const double* rhs, double* p, double tol, int precision,
                                 void* stream, vdp_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (nx < 8 || nx % 8 != 0 || ny < 1 || nz < 1 || !(L > 0.0) || !(tol > 0.0)) return VDP_EINVAL;
  if (precision < VDP_FP64 || precision > VDP_MIXED_BF16) return VDP_EINVAL;
  const long long n = (long long)nx * ny * nz;
  if (n > kMaxCells) return VDP_EINVAL;  // larger than the fixed scratch array
  const size_t bytes = sizeof(double) * (size_t)n;
  if (!rho || !rhs || !p || !on_this_device(rho, bytes) || !on_this_device(rhs, bytes) ||
      !on_this_device(p, bytes))
    return VDP_EINVAL;
  if (((uintptr_t)rhs & 15) || ((uintptr_t)p & 15)) return VDP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int st = scratch_base(&base);
  if (st != VDP_OK) return st;

  double* f64[kNumF64];
  for (size_t i = 0; i < kNumF64; ++i)
    f64[i] = reinterpret_cast<double*>(base + kOffFields + i * kF64);
  double *bx = f64[0], *by = f64[1], *bz = f64[2], *sinv = f64[3];
  void *sx = f64[4], *sy = f64[5], *sz = f64[6];
  void* sd = base + kOffSd;
  double* part = reinterpret_cast<double*>(base + kOffPart);
  UnitRef* units = reinterpret_cast<UnitRef*>(base + kOffUnits);
  InstDesc* desc = reinterpret_cast<InstDesc*>(base + kOffDesc);
  InstState* state = reinterpret_cast<InstState*>(base + kOffState);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(base + kOffTicket);
  int* flag = reinterpret_cast<int*>(base + kOffFlag);

  // density check, then the coefficients (the flag must start at zero on every call)
  int bad = 0;
  NA_CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
  NA_CK(launch_check_density(rho, n, flag, s));
  NA_CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (bad) return VDP_EDENSITY;
  double* dg = f64[12];
  NA_CK(launch_build_coefficients(rho, nx, ny, nz, L / nx, L / ny, L / nz, 0, bx, by, bz, sinv, dg, s));
  NA_CK(launch_scaled(precision, bx, by, bz, sinv, nx, ny, nz, sx, sy, sz, sd, s));

  // the default unit layout of vdp_solve
  Layout lay;
  if (!plan_layout(nx, ny, nz, precision, 0, 0, 0, 0, 0, &lay)) return VDP_EINVAL;
  const int nunits = lay.nunits, nunits_f = lay.nunits_f;

  UnitRef hu[kMaxUnits];
  for (int i = 0; i < nunits; ++i) hu[i] = UnitRef{0, i};
  for (int i = 0; i < nunits_f; ++i) hu[nunits + i] = UnitRef{0, i};
  InstDesc d{};
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.ty = lay.ty;
  d.uy = lay.uy;
  d.nunits = nunits;
  d.nunits_f = nunits_f;
  d.stages = lay.stages;
  d.zc = lay.zc;
  d.mode = lay.mode;
  d.ncell = n;
  d.bx = bx;
  d.by = by;
  d.bz = bz;
  d.sinv = sinv;
  d.dg = dg;
  d.sx = sx;
  d.sy = sy;
  d.sz = sz;
  d.sd = sd;
  d.x = f64[7];
  d.r = f64[8];
  d.d0 = f64[9];
  d.d1 = f64[10];
  d.q = f64[11];
  d.part = part;
  d.ticket = ticket;
  d.st = state;
  // pageable host sources: these copies complete before the calls return
  NA_CK(cudaMemcpyAsync(units, hu, sizeof(UnitRef) * (nunits + nunits_f), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
  NA_CK(prepare_step(precision, lay.mode, lay.smem));
  // the per-solve state and the ticket are reset on the device by the init kernel
  const int max_iter = 20000;
  NA_CK(launch_init(desc, rhs, p, tol, 1e-4, max_iter, max_iter, 0, precision, s));

  const int m = 16;  // (stencil, flat) launch pairs per convergence check
  const long long max_rounds = (2LL * max_iter + 4096 + m - 1) / m;
  InstState h{};
  bool done = false;
  long long rounds = 0;
  while (!done && rounds < max_rounds) {
    for (int i = 0; i < m; ++i) {
      NA_CK(launch_res64(precision, desc, units, nunits, lay.threads, s));
      NA_CK(launch_stencil(precision, lay.mode, 0, desc, units, nunits, lay.threads, lay.smem, s));
      NA_CK(launch_flat(precision, desc, units + nunits, nunits_f, s));
    }
    ++rounds;
    NA_CK(cudaMemcpyAsync(&h, state, sizeof(h), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    done = h.phase >= PH_DONE;
  }
  const int status = done ? h.status : VDP_ETIMEOUT;
  if (stats) {
    stats->status = status;
    stats->iters = h.iters;
    stats->outer_iters = h.outer;
    stats->rel_res = h.rel_res;
    stats->rhs_mean = h.mu_f;
    stats->ms = 0.0;
    stats->sweeps = h.sweeps;
    stats->launches = (int)(1 + rounds * 3 * m);
  }
  return status;
}
