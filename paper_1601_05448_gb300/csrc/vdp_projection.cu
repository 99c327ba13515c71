// vdp_projection.cu -- the steps either side of the pressure solve in one projection substep
// (App. A): the right side of the variable-coefficient Poisson equation
//
//     RHS^Pois = ( div( (rho u)~ / rho_new ) - RHS^div ) / c,        c = C_pre[k] dt,
//
// and the momentum correction of Eq. (mom),  (rho u)_new = (rho u)~ - c grad p.
//
// Face momenta live on the low face of each cell (mx[i] on the face shared by cells i - e_x and
// i), the layout of the face coefficients b_d = 1 / (rho_face h_d^2) that vdp_set_density builds
// from rho_new with the App. B face average.  The velocity flux through a face divided by h_d is
// therefore h_d b_d m_d, and the discrete divergence pairs with the operator A exactly: the
// corrected velocity satisfies div u_new = RHS^div - <RHS^div> to the tolerance of the solve.
//
// Both kernels march along z with one thread per (x, y) column segment: the z-neighbour value of
// the previous plane is carried in a register, the x- and y-neighbour loads hit L1 / L2 (the rows
// of the neighbouring lanes and warps), so each array is read from HBM about once.  On GB300 the
// FP64 pipe (2 FMA / clk / SM) rather than HBM bounds them: about 10 FP64 operations per cell in
// the right side and 6 in the correction, against 64 and 56 bytes of traffic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "vdp.h"
#include "vdp_ctx.h"
#include "vdp_march.cuh"

using namespace vdp;

namespace {

constexpr int kTx = kMarchTx, kTy = kMarchTy;
constexpr int kMinBlocks = 6;  // 6 x 256 threads per SM: at most 40 registers

// f = ( hx ((bx mx)|_{x+} - bx mx) + hy (...) + hz (...) - rhs_div ) / c
template <bool DIV>
__global__ void __launch_bounds__(kTx* kTy, kMinBlocks)
    k_projection_rhs(const double* __restrict__ mx, const double* __restrict__ my,
                     const double* __restrict__ mz, const double* __restrict__ bx,
                     const double* __restrict__ by, const double* __restrict__ bz,
                     const double* __restrict__ rd, int nx, int ny, int nz, MarchPlan m,
                     double hx, double hy, double hz, double inv_c, double* __restrict__ f) {
  const long long plane = (long long)nx * ny;
  for (int it = blockIdx.x; it < m.items; it += gridDim.x) {
    int x, y, z0, z1;
    if (!march_item(m, it, threadIdx.x, threadIdx.y, nx, ny, nz, x, y, z0, z1)) continue;
    const long long dxp = x == nx - 1 ? -(long long)(nx - 1) : 1;
    const long long dyp = y == ny - 1 ? -(long long)(ny - 1) * nx : (long long)nx;
    long long c = x + (long long)nx * y + plane * z0;
    double fz_lo = bz[c] * mz[c];  // z-flux (without h_z) through the low face of the cell
    for (int z = z0; z < z1; ++z) {
      const long long czp = z == nz - 1 ? c - plane * (nz - 1) : c + plane;
      const double fz_hi = bz[czp] * mz[czp];
      const double dx = fma(bx[c + dxp], mx[c + dxp], -(bx[c] * mx[c]));
      const double dy = fma(by[c + dyp], my[c + dyp], -(by[c] * my[c]));
      const double dz = fz_hi - fz_lo;
      const double v = fma(hx, dx, fma(hy, dy, DIV ? fma(hz, dz, -rd[c]) : hz * dz));
      f[c] = v * inv_c;
      fz_lo = fz_hi;
      c += plane;
    }
  }
}

// m_d -= (c / h_d) (p - p[-e_d]), in place
__global__ void __launch_bounds__(kTx* kTy, kMinBlocks)
    k_projection_correct(const double* __restrict__ p, int nx, int ny, int nz, MarchPlan m,
                         double cx, double cy, double cz, double* __restrict__ mx,
                         double* __restrict__ my, double* __restrict__ mz) {
  const long long plane = (long long)nx * ny;
  for (int it = blockIdx.x; it < m.items; it += gridDim.x) {
    int x, y, z0, z1;
    if (!march_item(m, it, threadIdx.x, threadIdx.y, nx, ny, nz, x, y, z0, z1)) continue;
    const long long dxm = x == 0 ? (long long)(nx - 1) : -1;
    const long long dym = y == 0 ? (long long)(ny - 1) * nx : -(long long)nx;
    long long c = x + (long long)nx * y + plane * z0;
    double p_lo = p[z0 == 0 ? c + plane * (nz - 1) : c - plane];  // p one plane below
    int z = z0;
    // two planes per step: all loads of both planes are issued before the first store
    for (; z + 1 < z1; z += 2) {
      const long long c1 = c + plane;
      const double p0 = p[c], p1 = p[c1];
      const double px0 = p[c + dxm], px1 = p[c1 + dxm], py0 = p[c + dym], py1 = p[c1 + dym];
      const double mx0 = mx[c], mx1 = mx[c1], my0 = my[c], my1 = my[c1], mz0 = mz[c],
                   mz1 = mz[c1];
      mx[c] = fma(-cx, p0 - px0, mx0);
      my[c] = fma(-cy, p0 - py0, my0);
      mz[c] = fma(-cz, p0 - p_lo, mz0);
      mx[c1] = fma(-cx, p1 - px1, mx1);
      my[c1] = fma(-cy, p1 - py1, my1);
      mz[c1] = fma(-cz, p1 - p0, mz1);
      p_lo = p1;
      c = c1 + plane;
    }
    if (z < z1) {
      const double pc = p[c];
      mx[c] = fma(-cx, pc - p[c + dxm], mx[c]);
      my[c] = fma(-cy, pc - p[c + dym], my[c]);
      mz[c] = fma(-cz, pc - p_lo, mz[c]);
    }
  }
}

bool dev_aligned(const void* a) { return a && is_device_ptr(a) && ((uintptr_t)a & 7) == 0; }

bool bad_c(double c) { return !(c > 0.0) || !std::isfinite(c); }

cudaError_t launch_rhs(const vdp_ctx* ctx, const double* mx, const double* my, const double* mz,
                       const double* rd, double c, double* f, cudaStream_t s) {
  const double hx = ctx->Lx / ctx->nx, hy = ctx->Ly / ctx->ny, hz = ctx->Lz / ctx->nz;
  if (rd) {
    static const int R = resident_blocks(k_projection_rhs<true>);
    const MarchPlan m = march_plan(ctx->nx, ctx->ny, ctx->nz, R);
    k_projection_rhs<true><<<m.blocks, dim3(kTx, kTy), 0, s>>>(
        mx, my, mz, ctx->bx, ctx->by, ctx->bz, rd, ctx->nx, ctx->ny, ctx->nz, m, hx, hy, hz,
        1.0 / c, f);
  } else {
    static const int R = resident_blocks(k_projection_rhs<false>);
    const MarchPlan m = march_plan(ctx->nx, ctx->ny, ctx->nz, R);
    k_projection_rhs<false><<<m.blocks, dim3(kTx, kTy), 0, s>>>(
        mx, my, mz, ctx->bx, ctx->by, ctx->bz, nullptr, ctx->nx, ctx->ny, ctx->nz, m, hx, hy, hz,
        1.0 / c, f);
  }
  return cudaGetLastError();
}

cudaError_t launch_correct(const vdp_ctx* ctx, const double* p, double c, double* mx, double* my,
                           double* mz, cudaStream_t s) {
  static const int R = resident_blocks(k_projection_correct);
  const MarchPlan m = march_plan(ctx->nx, ctx->ny, ctx->nz, R);
  const double hx = ctx->Lx / ctx->nx, hy = ctx->Ly / ctx->ny, hz = ctx->Lz / ctx->nz;
  k_projection_correct<<<m.blocks, dim3(kTx, kTy), 0, s>>>(p, ctx->nx, ctx->ny, ctx->nz, m, c / hx,
                                                           c / hy, c / hz, mx, my, mz);
  return cudaGetLastError();
}

bool distinct(const void* const* a, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (a[i] && a[i] == a[j]) return false;
  return true;
}

// Run `body` (kernel launches on the stream it is given) once on the context's stream, captured
// into a graph between two event records, so that the events bracket the kernels alone (on an
// idle stream a plain event record would fire before the host had submitted the kernel).
template <class Body>
cudaError_t time_on_graph(vdp_ctx* ctx, Body body, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = cudaEventRecordWithFlags(e0, ctx->cap, cudaEventRecordExternal);
      if (e2 == cudaSuccess) e2 = body(ctx->cap);
      if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(e1, ctx->cap, cudaEventRecordExternal);
      e = cudaStreamEndCapture(ctx->cap, &g);
      if (e2 != cudaSuccess) e = e2;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(x, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (x) cudaGraphExecDestroy(x);
  if (g) cudaGraphDestroy(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" int vdp_projection_rhs(vdp_ctx* ctx, const double* mx, const double* my,
                                  const double* mz, const double* rhs_div, double c, double* f) {
  if (!ctx || !ctx->has_density || bad_c(c) || ctx->bc_x != VDP_BC_PERIODIC) return VDP_EINVAL;
  if (!dev_aligned(mx) || !dev_aligned(my) || !dev_aligned(mz) || !dev_aligned(f) ||
      (rhs_div && !dev_aligned(rhs_div)))
    return VDP_EINVAL;
  if (f == mx || f == my || f == mz || f == rhs_div) return VDP_EINVAL;  // inputs are read-only
  VDP_CK(launch_rhs(ctx, mx, my, mz, rhs_div, c, f, ctx->stream));
  VDP_CK(cudaStreamSynchronize(ctx->stream));
  return VDP_OK;
}

extern "C" int vdp_projection_correct(vdp_ctx* ctx, const double* p, double c, double* mx,
                                      double* my, double* mz) {
  if (!ctx || bad_c(c) || ctx->bc_x != VDP_BC_PERIODIC) return VDP_EINVAL;
  if (!dev_aligned(p) || !dev_aligned(mx) || !dev_aligned(my) || !dev_aligned(mz))
    return VDP_EINVAL;
  const void* all[] = {p, mx, my, mz};
  if (!distinct(all, 4)) return VDP_EINVAL;
  VDP_CK(launch_correct(ctx, p, c, mx, my, mz, ctx->stream));
  VDP_CK(cudaStreamSynchronize(ctx->stream));
  return VDP_OK;
}

static int project(vdp_ctx* ctx, double* mx, double* my, double* mz, const double* rhs_div,
                   double c, double tol, double* p, float* ms) {
  if (!ctx || !ctx->has_density || bad_c(c) || !(tol > 0.0) || !std::isfinite(tol) ||
      ctx->bc_x != VDP_BC_PERIODIC)
    return VDP_EINVAL;
  if (!dev_aligned(mx) || !dev_aligned(my) || !dev_aligned(mz) || !dev_aligned(p) ||
      ((uintptr_t)p & 15) || (rhs_div && !dev_aligned(rhs_div)))
    return VDP_EINVAL;
  const void* all[] = {mx, my, mz, p, rhs_div};
  if (!distinct(all, 5)) return VDP_EINVAL;
  if (!ctx->proj_f) VDP_CK(cudaMalloc((void**)&ctx->proj_f, sizeof(double) * (size_t)ctx->n));
  double* f = ctx->proj_f;
  auto rhs = [&](cudaStream_t s) { return launch_rhs(ctx, mx, my, mz, rhs_div, c, f, s); };
  auto corr = [&](cudaStream_t s) { return launch_correct(ctx, p, c, mx, my, mz, s); };
  if (ms)
    VDP_CK(time_on_graph(ctx, rhs, &ms[0]));
  else
    VDP_CK(rhs(ctx->stream));
  const int s = vdp_solve(ctx, f, p, tol);
  if (ms) ms[1] = (float)ctx->stats.ms;
  if (s != VDP_OK) return s;  // the momenta stay as they were
  if (ms)
    VDP_CK(time_on_graph(ctx, corr, &ms[2]));
  else
    VDP_CK(corr(ctx->stream));
  VDP_CK(cudaStreamSynchronize(ctx->stream));
  return VDP_OK;
}

extern "C" int vdp_project(vdp_ctx* ctx, double* mx, double* my, double* mz,
                           const double* rhs_div, double c, double tol, double* p) {
  return project(ctx, mx, my, mz, rhs_div, c, tol, p, nullptr);
}

extern "C" int vdp_project_timed(vdp_ctx* ctx, double* mx, double* my, double* mz,
                                 const double* rhs_div, double c, double tol, double* p,
                                 float* ms) {
  if (!ms) return VDP_EINVAL;
  ms[0] = ms[1] = ms[2] = 0.f;
  return project(ctx, mx, my, mz, rhs_div, c, tol, p, ms);
}
