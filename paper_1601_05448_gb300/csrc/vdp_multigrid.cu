// vdp_multigrid.cu -- geometric multigrid V-cycle that preconditions CG for the variable-
// coefficient operator A of div((1/rho) grad .) (Sec. 3.4) on any grid whose coarsening reaches
// at most 512 cells (all sizes even down to it), where the FFT passes of the spectral
// preconditioner need lengths built from 2 and 3.
//
// The cycle (cell-centred, periodic, FP32, unscaled variables):
//   levels      halve every direction while all sizes are even and the level has > 64 cells;
//   coarse A    face coefficient = 1/2 x the sum of the four fine low faces under the coarse low
//               face (the 2h rediscretisation of the face flux, 8 x the 2h operator for constant
//               rho: the restricted equations are sums over 8 children);
//   P, R        cell-centred linear interpolation (3/4 parent, 1/4 its neighbour on the fine
//               cell's side, per axis) and its transpose;
//   smoothing   one weighted Jacobi sweep (weight 0.8) before the coarse correction, from zero,
//               and one after it;
//   coarsest    the dense pseudo-inverse of -A (built on the host in double precision).
// Same smoother before and after, R = P^T and a symmetric coarse solve make the cycle a fixed
// symmetric positive (semi-)definite operator M ~ (-A)^-1, as CG needs.  Used on the solve's
// scaled residual rt = D^-1/2 r: z = W M W rt with W = D^1/2 (the weight omega), like the
// spectral preconditioner.
//
// Per level and cycle four launches: pre-smoothing + residual (down), restriction, prolongation
// + pre-smoothed iterate, post-smoothing (up); one launch solves the coarsest level.  The level
// sweeps are z-marching column kernels (one-wave work-item plan); the z-neighbours are carried in
// registers.  All launches return at once unless the solve is in its preconditioner phase.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "vdp_device.cuh"
#include "vdp_march.cuh"
#include "vdp_multigrid.h"

namespace vdp {

namespace {

constexpr int kMgThreads = kMarchTx * kMarchTy;  // 1-D blocks of 256 (tile 32 x 8)
constexpr int kCoarseThreads = 512;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return narrow(v); }
__device__ __forceinline__ void from_f(float v, float* out) { *out = v; }
__device__ __forceinline__ void from_f(float v, double* out) { *out = widen(v); }

__device__ __forceinline__ bool mg_active(const InstState* st) {
  return st == nullptr || __ldcg(&st->phase) == PH_SPEC;
}

struct Nbr {
  long long dxm, dxp, dym, dyp;
};

__device__ __forceinline__ Nbr neighbours(int x, int y, int nx, int ny) {
  Nbr d;
  d.dxm = x == 0 ? (long long)(nx - 1) : -1;
  d.dxp = x == nx - 1 ? -(long long)(nx - 1) : 1;
  d.dym = y == 0 ? (long long)(ny - 1) * nx : -(long long)nx;
  d.dyp = y == ny - 1 ? -(long long)(ny - 1) * nx : (long long)nx;
  return d;
}

#define MG_MARCH_BEGIN(lv)                                                                      \
  const int nx = (lv).nx, ny = (lv).ny, nz = (lv).nz;                                          \
  const long long plane = (long long)nx * ny;                                                  \
  for (int it = blockIdx.x; it < m.items; it += gridDim.x) {                                   \
    int x, y, z0, z1;                                                                          \
    if (!march_item(m, it, threadIdx.x & 31, threadIdx.x >> 5, nx, ny, nz, x, y, z0, z1))      \
      continue;                                                                                \
    const Nbr d = neighbours(x, y, nx, ny);                                                    \
    long long c = x + (long long)nx * y + plane * z0;

// Every smoothed level works in scaled variables (y = W x, W = D^1/2 = omega): the scaled operator
// At = W^-1 (-A) W^-1 = I - offdiag(bt) has a unit diagonal, so a Jacobi sweep is y += w (rt - At y)
// and no diagonal is read.  lv.bx, by, bz hold bt in FP32; level 0 takes W from the solve, the
// coarser levels keep their own (om, oinv = 1 / om).  Restriction and prolongation act on the
// unscaled quantities.

// Down: y1 = w rt (from zero), scaled residual rt - At y1 = (1 - w) rt + w sum bt rt_nb, stored
// unscaled (times omega) in t for the restriction.
template <class T>
__global__ void __launch_bounds__(kMgThreads, 4)
    k_mg_down0(MgLevel lv, MarchPlan m, const T* __restrict__ rt, const float* __restrict__ om,
               const InstState* st) {
  if (!mg_active(st)) return;
  const float w = kMgOmega;
  MG_MARCH_BEGIN(lv)
  float r_m = to_f(__ldg(rt + (z0 == 0 ? c + plane * (nz - 1) : c - plane)));
  float r_c = to_f(__ldg(rt + c));
  float bz_c = __ldg(lv.bz + c);
  for (int z = z0; z < z1; ++z) {
    const long long czp = z == nz - 1 ? c - plane * (nz - 1) : c + plane;
    const float r_p = to_f(__ldg(rt + czp));
    const float bz_p = __ldg(lv.bz + czp);
    float s = __ldg(lv.bx + c) * to_f(__ldg(rt + c + d.dxm));
    s = fmaf(__ldg(lv.bx + c + d.dxp), to_f(__ldg(rt + c + d.dxp)), s);
    s = fmaf(__ldg(lv.by + c), to_f(__ldg(rt + c + d.dym)), s);
    s = fmaf(__ldg(lv.by + c + d.dyp), to_f(__ldg(rt + c + d.dyp)), s);
    s = fmaf(bz_c, r_m, s);
    s = fmaf(bz_p, r_p, s);
    lv.t[c] = __ldg(om + c) * fmaf(1.f - w, r_c, w * s);
    r_m = r_c;
    r_c = r_p;
    bz_c = bz_p;
    c += plane;
  }
  }
}

// Up: y3 = y2 + w (rt - At y2) = (1 - w) y2 + w (rt + sum bt y2_nb), y2 = t.  Level 0 (COARSE
// false) stores y3 as the solve's scaled z and, with a state, <rt, z>, and completes the sweep; a
// coarser level stores its unscaled result x = oinv y3 for the next finer prolongation.
template <class T, class TOUT, bool COARSE>
__global__ void __launch_bounds__(kMgThreads, 4)
    k_mg_up(MgLevel lv, MarchPlan m, const T* __restrict__ rt, TOUT* __restrict__ out,
            InstState* st, const InstDesc* I) {
  if (!mg_active(st)) return;
  const float w = kMgOmega;
  const float* __restrict__ t = lv.t;
  float acc = 0.f;
  MG_MARCH_BEGIN(lv)
  float v_m = __ldg(t + (z0 == 0 ? c + plane * (nz - 1) : c - plane));
  float v_c = __ldg(t + c);
  float bz_c = __ldg(lv.bz + c);
  for (int z = z0; z < z1; ++z) {
    const long long czp = z == nz - 1 ? c - plane * (nz - 1) : c + plane;
    const float v_p = __ldg(t + czp);
    const float bz_p = __ldg(lv.bz + czp);
    float s = to_f(__ldg(rt + c));
    const float r_c = s;
    s = fmaf(__ldg(lv.bx + c), __ldg(t + c + d.dxm), s);
    s = fmaf(__ldg(lv.bx + c + d.dxp), __ldg(t + c + d.dxp), s);
    s = fmaf(__ldg(lv.by + c), __ldg(t + c + d.dym), s);
    s = fmaf(__ldg(lv.by + c + d.dyp), __ldg(t + c + d.dyp), s);
    s = fmaf(bz_c, v_m, s);
    s = fmaf(bz_p, v_p, s);
    const float y3 = fmaf(1.f - w, v_c, w * s);
    if constexpr (COARSE) {
      lv.x[c] = __ldg(lv.oinv + c) * y3;
    } else {
      from_f(y3, out + c);
      acc = fmaf(r_c, y3, acc);
    }
    v_m = v_c;
    v_c = v_p;
    bz_c = bz_p;
    c += plane;
  }
  }
  if constexpr (!COARSE) {
    if (st) {
      const float part[1] = {acc};
      store_partials<1, float>(part, I->part, gridDim.x, blockIdx.x);
      finish_sweep(*I, st, PH_SPEC, gridDim.x);
    }
  }
}

// Prolongation, marching the fine column (x, y) along z: the bilinear xy interpolation of coarse
// plane K at the column, L(K), is computed once and carried; fine plane k = 2K takes
// 3/4 L(K) + 1/4 L(K-1), k = 2K + 1 takes 3/4 L(K) + 1/4 L(K+1).  With the pre-smoothed iterate:
// t = w rt + omega P xc   (scaled: y1 + W P xc; xc is the coarse level's unscaled result)
template <class T>
__global__ void __launch_bounds__(kMgThreads, 4)
    k_mg_prolong(MgLevel lv, MgLevel cv, MarchPlan m, const T* __restrict__ rt,
                 const float* __restrict__ om, int wall_x, const InstState* st) {
  if (!mg_active(st)) return;
  const int cx = cv.nx, cy = cv.ny, cz = cv.nz;
  const long long cplane = (long long)cx * cy;
  const float* __restrict__ xc = cv.x;
  MG_MARCH_BEGIN(lv)
  (void)d;
  const int I0 = x >> 1, J0 = y >> 1;
  // neighbour of the parent on the fine cell's side; at the duct's x ends the parent itself
  const int I1 = (x & 1) ? (I0 + 1 == cx ? (wall_x ? I0 : 0) : I0 + 1)
                         : (I0 == 0 ? (wall_x ? I0 : cx - 1) : I0 - 1);
  const int J1 = (y & 1) ? (J0 + 1 == cy ? 0 : J0 + 1) : (J0 == 0 ? cy - 1 : J0 - 1);
  const long long q00 = I0 + (long long)cx * J0, q10 = I1 + (long long)cx * J0;
  const long long q01 = I0 + (long long)cx * J1, q11 = I1 + (long long)cx * J1;
  auto L = [&](int K) {
    const float* pl = xc + cplane * K;
    const float a = fmaf(0.75f, __ldg(pl + q00), 0.25f * __ldg(pl + q10));
    const float b = fmaf(0.75f, __ldg(pl + q01), 0.25f * __ldg(pl + q11));
    return fmaf(0.75f, a, 0.25f * b);
  };
  int K = z0 >> 1;
  float Lm = L(K == 0 ? cz - 1 : K - 1), Lc = L(K), Lp = L(K + 1 == cz ? 0 : K + 1);
  for (int z = z0; z < z1; ++z) {
    const float pxc = (z & 1) ? fmaf(0.75f, Lc, 0.25f * Lp) : fmaf(0.75f, Lc, 0.25f * Lm);
    lv.t[c] = fmaf(kMgOmega, to_f(__ldg(rt + c)), __ldg(om + c) * pxc);
    if ((z & 1) && z + 1 < z1) {  // the next fine plane belongs to coarse plane K + 1
      ++K;
      Lm = Lc;
      Lc = Lp;
      Lp = L(K + 1 == cz ? 0 : K + 1);
    }
    c += plane;
  }
  }
}

// Restriction r_coarse = P^T t, marching the coarse column (I, J) along K: a warp covers 32
// consecutive I of one coarse row, each lane loads its two fine cells (2I, 2I + 1) of a fine row
// as one float2 and takes 2I - 1 and 2I + 2 from its neighbour lanes (edge lanes load them), so a
// fine row costs one 8-byte load per coarse cell.  The xy sums of fine planes 2K - 1 and 2K are
// carried from the previous K.
// The coarse right side is stored scaled (times oinv) unless the coarse level is the coarsest
// (solved unscaled by the pseudo-inverse; oinv null).
__global__ void __launch_bounds__(kMgThreads, 4)
    k_mg_restrict(MgLevel fv, MgLevel cv, MarchPlan m, const float* __restrict__ oinv,
                  int wall_x, const InstState* st) {
  if (!mg_active(st)) return;
  const int nx = fv.nx, ny = fv.ny, nz = fv.nz;
  const int cx = cv.nx, cy = cv.ny, cz = cv.nz;
  const long long fplane = (long long)nx * ny, cplane = (long long)cx * cy;
  const float* __restrict__ t = fv.t;
  const int lane = threadIdx.x & 31;
  for (int it = blockIdx.x; it < m.items; it += gridDim.x) {
    int I, J, K0, K1;
    const bool on = march_item(m, it, lane, threadIdx.x >> 5, cx, cy, cz, I, J, K0, K1);
    // the whole warp takes part in the shuffles; a warp never straddles two coarse rows
    const int Jc = J < cy ? J : cy - 1;
    const int Ic = on ? I : 0;
    int yj[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) yj[b] = (2 * Jc - 1 + b + ny) % ny;
    const bool lload = lane == 0 || !on || Ic == 0;                 // 2I - 1 not in lane - 1
    const bool rload = lane == 31 || Ic == cx - 1;                  // 2I + 2 not in lane + 1
    const int xl = 2 * Ic == 0 ? nx - 1 : 2 * Ic - 1;
    const int xr = 2 * Ic + 2 == nx ? 0 : 2 * Ic + 2;
    // xy sum of fine plane k (weights 1/4, 3/4, 3/4, 1/4 per axis)
    auto plane_sum = [&](int k) {
      const float* pk = t + fplane * k;
      float sum = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float* row = pk + (long long)nx * yj[b];
        float2 v = make_float2(0.f, 0.f);
        if (on) v = __ldg(reinterpret_cast<const float2*>(row + 2 * Ic));
        float left = __shfl_up_sync(0xffffffffu, v.y, 1);
        float right = __shfl_down_sync(0xffffffffu, v.x, 1);
        if (on && lload) left = __ldg(row + xl);
        if (on && rload) right = __ldg(row + xr);
        // the duct's x ends: the end child took the quarter the far side would have given
        if (wall_x && Ic == 0) left = v.x;
        if (wall_x && Ic == cx - 1) right = v.y;
        const float rs = fmaf(0.25f, left + right, 0.75f * (v.x + v.y));
        const float wb = (b == 0 || b == 3) ? 0.25f : 0.75f;
        sum = fmaf(wb, rs, sum);
      }
      return sum;
    };
    int kk = 2 * K0 - 1;
    float s_a = plane_sum(kk < 0 ? kk + nz : kk);   // fine plane 2K - 1
    float s_b = plane_sum(2 * K0);                  // fine plane 2K
    for (int K = K0; K < K1; ++K) {
      const float s_c = plane_sum(2 * K + 1);
      const float s_d = plane_sum(2 * K + 2 == nz ? 0 : 2 * K + 2);
      if (on) {
        const long long C = I + (long long)cx * J + cplane * K;
        const float v = fmaf(0.25f, s_a + s_d, 0.75f * (s_b + s_c));
        cv.r[C] = oinv ? __ldg(oinv + C) * v : v;
      }
      s_a = s_c;
      s_b = s_d;
    }
  }
}

// Coarsest level: x = pinv r (one block; pinv is symmetric, so thread i reads column i).
__global__ void __launch_bounds__(kCoarseThreads)
    k_mg_coarse(MgLevel lv, const float* __restrict__ pinv, int n, const InstState* st) {
  if (!mg_active(st)) return;
  __shared__ float r[kMgMaxCoarsest];
  for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = lv.r[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < n; ++j) s = fmaf(__ldg(pinv + (long long)j * n + i), r[j], s);
    lv.x[i] = s;
  }
}

// ---- set-up -------------------------------------------------------------------------------------

// level 0 from the FP64 face coefficients: the scaled coefficients bt = b sinv sinv_nb in FP32
__global__ void k_mg_level0(const double* __restrict__ bx, const double* __restrict__ by,
                            const double* __restrict__ bz, const double* __restrict__ sinv,
                            MgLevel lv) {
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < lv.n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / plane);
    const long long xm = c - x + (x == 0 ? nx - 1 : x - 1);
    const long long ym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    const long long zm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    const double s = sinv[c];
    lv.bx[c] = (float)(bx[c] * s * sinv[xm]);
    lv.by[c] = (float)(by[c] * s * sinv[ym]);
    lv.bz[c] = (float)(bz[c] * s * sinv[zm]);
  }
}

// coarse faces: 1/2 x the sum of the four fine low faces under each coarse low face
template <class TB>
__global__ void k_mg_coarsen(const TB* __restrict__ fbx, const TB* __restrict__ fby,
                             const TB* __restrict__ fbz, int fnx, int fny, MgLevel cv) {
  for (long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x; C < cv.n;
       C += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(C % cv.nx), J = (int)((C / cv.nx) % cv.ny);
    const int K = (int)(C / ((long long)cv.nx * cv.ny));
    auto f = [&](int i, int j, int k) { return (long long)i + (long long)fnx * (j + (long long)fny * k); };
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const double sx = (double)fbx[f(i0, j0, k0)] + (double)fbx[f(i0, j0 + 1, k0)] +
                      (double)fbx[f(i0, j0, k0 + 1)] + (double)fbx[f(i0, j0 + 1, k0 + 1)];
    const double sy = (double)fby[f(i0, j0, k0)] + (double)fby[f(i0 + 1, j0, k0)] +
                      (double)fby[f(i0, j0, k0 + 1)] + (double)fby[f(i0 + 1, j0, k0 + 1)];
    const double sz = (double)fbz[f(i0, j0, k0)] + (double)fbz[f(i0 + 1, j0, k0)] +
                      (double)fbz[f(i0, j0 + 1, k0)] + (double)fbz[f(i0 + 1, j0 + 1, k0)];
    cv.bx[C] = (float)(0.5 * sx);
    cv.by[C] = (float)(0.5 * sy);
    cv.bz[C] = (float)(0.5 * sz);
  }
}

// W = D^1/2 and 1 / W of an (unscaled) coarse level
__global__ void k_mg_weights(MgLevel lv) {
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < lv.n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / plane);
    const long long xp = c - x + (x == nx - 1 ? 0 : x + 1);
    const long long yp = c + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx;
    const long long zp = c + (long long)((z == nz - 1 ? 0 : z + 1) - z) * plane;
    const double D = (double)lv.bx[c] + lv.bx[xp] + lv.by[c] + lv.by[yp] + lv.bz[c] + lv.bz[zp];
    const double w = sqrt(D);
    lv.om[c] = (float)w;
    lv.oinv[c] = (float)(1.0 / w);
  }
}

// scale a coarse level's faces in place: bt = b oinv oinv_nb (after the next level was coarsened
// from the unscaled faces)
__global__ void k_mg_scale_faces(MgLevel lv) {
  const int nx = lv.nx, ny = lv.ny, nz = lv.nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < lv.n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / plane);
    const long long xm = c - x + (x == 0 ? nx - 1 : x - 1);
    const long long ym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    const long long zm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    const float s = lv.oinv[c];
    lv.bx[c] = lv.bx[c] * s * lv.oinv[xm];
    lv.by[c] = lv.by[c] * s * lv.oinv[ym];
    lv.bz[c] = lv.bz[c] * s * lv.oinv[zm];
  }
}

// out = in rounded to FP32 (the FP64 solve's scaled residual, read by the level-0 sweeps)
__global__ void k_mg_narrow(const double* __restrict__ in, long long n, float* __restrict__ out,
                            const InstState* st) {
  if (!mg_active(st)) return;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    out[c] = narrow(in[c]);
}

// out = in * sinv (between the unscaled and the scaled variables of level 0)
__global__ void k_mg_scale(const double* __restrict__ in, const double* __restrict__ sinv,
                           long long n, double* __restrict__ out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    out[c] = in[c] * sinv[c];
}

int flat_grid(long long n) {
  long long b = (n + kMgThreads - 1) / kMgThreads;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

// Pseudo-inverse of the singular SPD matrix -A (n x n, null space: constants) in double:
// (-A)^+ = (-A + a J/n)^-1 - J / (a n), J the all-ones matrix, a > 0 (here the mean diagonal).
bool pseudo_inverse(std::vector<double>& A, int n, std::vector<double>& out) {
  double a = 0.0;
  for (int i = 0; i < n; ++i) a += A[(size_t)i * n + i];
  a = a > 0.0 ? a / n : 1.0;
  std::vector<double> M(A);
  for (size_t q = 0; q < M.size(); ++q) M[q] += a / n;
  // Cholesky M = L L^T (lower triangle in place)
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    M[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
      M[(size_t)i * n + j] = s / d;
    }
  }
  out.assign((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int col = 0; col < n; ++col) {  // solve L L^T x = e_col
    for (int i = 0; i < n; ++i) {
      double s = i == col ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= M[(size_t)i * n + k] * y[k];
      y[i] = s / M[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= M[(size_t)k * n + i] * out[(size_t)k * n + col];
      out[(size_t)i * n + col] = s / M[(size_t)i * n + i];
    }
  }
  for (size_t q = 0; q < out.size(); ++q) out[q] -= 1.0 / (a * n);
  return true;
}

template <class K>
int cached_resident(K kernel, int* cache) {
  if (*cache <= 0) *cache = resident_blocks(kernel);
  return *cache;
}

}  // namespace

int mg_level_dims(int nx, int ny, int nz, int (*dims)[3]) {
  int n = 0;
  int x = nx, y = ny, z = nz;
  for (;;) {
    dims[n][0] = x;
    dims[n][1] = y;
    dims[n][2] = z;
    ++n;
    if (x % 2 || y % 2 || z % 2 || (long long)x * y * z <= kMgMinCoarsen || n == kMgMaxLevels) break;
    x /= 2;
    y /= 2;
    z /= 2;
  }
  // at least one coarser level (a grid of at most 64 cells is not a multigrid problem)
  return n >= 2 && (long long)x * y * z <= kMgMaxCoarsest ? n : 0;
}

size_t mg_bytes(int nx, int ny, int nz) {
  int d[kMgMaxLevels][3];
  const int L = mg_level_dims(nx, ny, nz, d);
  if (!L) return 0;
  size_t cells = 0;
  for (int l = 0; l < L; ++l) cells += (size_t)(l == 0 ? 5 : 8) * d[l][0] * d[l][1] * d[l][2];
  const size_t nc = (size_t)d[L - 1][0] * d[L - 1][1] * d[L - 1][2];
  return sizeof(float) * (cells + nc * nc) + 64 * (size_t)(8 * L + 1);
}

cudaError_t mg_alloc(MgHier* h, int nx, int ny, int nz, int wall_x) {
  int d[kMgMaxLevels][3];
  const int L = mg_level_dims(nx, ny, nz, d);
  if (!L) return cudaErrorInvalidValue;
  const size_t bytes = mg_bytes(nx, ny, nz);
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) return e;
  char* p = static_cast<char*>(mem);
  auto take = [&](size_t count) {
    float* q = reinterpret_cast<float*>(p);
    p += ((sizeof(float) * count + 63) / 64) * 64;  // 64-byte aligned arrays
    return q;
  };
  MgHier hh;
  hh.nlev = L;
  hh.wall_x = wall_x;
  for (int l = 0; l < L; ++l) {
    MgLevel& v = hh.lev[l];
    v.nx = d[l][0];
    v.ny = d[l][1];
    v.nz = d[l][2];
    v.n = (long long)v.nx * v.ny * v.nz;
    v.bx = take(v.n);
    v.by = take(v.n);
    v.bz = take(v.n);
    v.om = l ? take(v.n) : nullptr;  // level 0 uses the solve's W
    v.oinv = l ? take(v.n) : nullptr;
    v.t = take(v.n);
    v.r = take(v.n);  // level 0: the FP32 copy of an FP64 right side
    v.x = l ? take(v.n) : nullptr;
  }
  hh.ncoarse = (int)hh.lev[L - 1].n;
  hh.pinv = take((size_t)hh.ncoarse * hh.ncoarse);
  hh.mem = mem;
  hh.bytes = bytes;
  *h = hh;
  return cudaSuccess;
}

void mg_free(MgHier* h) {
  if (h->mem) cudaFree(h->mem);
  *h = MgHier();
}

cudaError_t mg_setup(MgHier* h, const double* bx, const double* by, const double* bz,
                     const double* sinv, cudaStream_t s) {
  if (!h->mem) return cudaErrorInvalidValue;
  const MgLevel& l0 = h->lev[0];
  k_mg_level0<<<flat_grid(l0.n), kMgThreads, 0, s>>>(bx, by, bz, sinv, l0);
  for (int l = 1; l < h->nlev; ++l) {
    const MgLevel& f = h->lev[l - 1];
    const MgLevel& c = h->lev[l];
    if (l == 1)  // from the FP64 coefficients
      k_mg_coarsen<double><<<flat_grid(c.n), kMgThreads, 0, s>>>(bx, by, bz, f.nx, f.ny, c);
    else
      k_mg_coarsen<float><<<flat_grid(c.n), kMgThreads, 0, s>>>(f.bx, f.by, f.bz, f.nx, f.ny, c);
    if (l >= 2)  // level l - 1 has been coarsened from: scale it now (the coarsest stays unscaled)
      k_mg_scale_faces<<<flat_grid(f.n), kMgThreads, 0, s>>>(f);
    if (l < h->nlev - 1) k_mg_weights<<<flat_grid(c.n), kMgThreads, 0, s>>>(c);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the coarsest operator on the host
  const MgLevel& cl = h->lev[h->nlev - 1];
  const int n = (int)cl.n;
  std::vector<float> b(3 * (size_t)n);
  if ((e = cudaMemcpyAsync(b.data(), cl.bx, sizeof(float) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b.data() + n, cl.by, sizeof(float) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b.data() + 2 * n, cl.bz, sizeof(float) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return e;
  std::vector<double> A((size_t)n * n, 0.0);
  for (int k = 0; k < cl.nz; ++k)
    for (int j = 0; j < cl.ny; ++j)
      for (int i = 0; i < cl.nx; ++i) {
        const int c = i + cl.nx * (j + cl.ny * k);
        const int nb[3] = {(i == 0 ? cl.nx - 1 : i - 1) + cl.nx * (j + cl.ny * k),
                           i + cl.nx * ((j == 0 ? cl.ny - 1 : j - 1) + cl.ny * k),
                           i + cl.nx * (j + cl.ny * (k == 0 ? cl.nz - 1 : k - 1))};
        for (int d = 0; d < 3; ++d) {  // the low face of c in direction d joins c and nb[d]
          const double w = b[(size_t)d * n + c];
          const int m = nb[d];
          A[(size_t)c * n + c] += w;
          A[(size_t)m * n + m] += w;
          A[(size_t)c * n + m] -= w;
          A[(size_t)m * n + c] -= w;
        }
      }
  std::vector<double> P;
  if (!pseudo_inverse(A, n, P)) return cudaErrorInvalidValue;
  std::vector<float> Pf(P.begin(), P.end());
  if ((e = cudaMemcpyAsync(h->pinv, Pf.data(), sizeof(float) * Pf.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(s);
}

int mg_launches(const MgHier& h, int prec) { return 4 * (h.nlev - 1) + 1 + (prec == PREC_FP64); }

// One V-cycle; T is the type of the solve's rt and z.  An FP64 rt is rounded to FP32 once (into
// level 0's r), so the level-0 sweeps read FP32 only.
// One V-cycle; T is the type of the solve's rt and z.  An FP64 rt is rounded to FP32 once (into
// level 0's r), so the level-0 sweeps read FP32 only.
template <class T>
static cudaError_t vcycle(const MgHier& h, const MgArgs& a, cudaStream_t s) {
  static int r_down = 0, r_up0 = 0, r_up = 0, r_pro = 0, r_res = 0;
  const int L = h.nlev;
  if (L < 2 || !a.omega) return cudaErrorInvalidValue;
  const float* in;
  if constexpr (sizeof(T) == 8) {
    k_mg_narrow<<<flat_grid(h.lev[0].n), kMgThreads, 0, s>>>(static_cast<const double*>(a.in),
                                                             h.lev[0].n, h.lev[0].r, a.st);
    in = h.lev[0].r;
  } else {
    in = static_cast<const float*>(a.in);
  }
  T* out = static_cast<T*>(a.out);
  auto rhs = [&](int l) { return l == 0 ? in : static_cast<const float*>(h.lev[l].r); };
  auto wgt = [&](int l) { return l == 0 ? a.omega : static_cast<const float*>(h.lev[l].om); };
  for (int l = 0; l < L - 1; ++l) {
    const MgLevel& v = h.lev[l];
    const MgLevel& cv = h.lev[l + 1];
    const MarchPlan m = march_plan(v.nx, v.ny, v.nz, cached_resident(k_mg_down0<float>, &r_down));
    k_mg_down0<float><<<m.blocks, kMgThreads, 0, s>>>(v, m, rhs(l), wgt(l), a.st);
    const MarchPlan mr = march_plan(cv.nx, cv.ny, cv.nz, cached_resident(k_mg_restrict, &r_res));
    k_mg_restrict<<<mr.blocks, kMgThreads, 0, s>>>(v, cv, mr, l + 1 < L - 1 ? cv.oinv : nullptr,
                                                   h.wall_x, a.st);
  }
  k_mg_coarse<<<1, kCoarseThreads, 0, s>>>(h.lev[L - 1], h.pinv, h.ncoarse, a.st);
  for (int l = L - 2; l >= 0; --l) {
    const MgLevel& v = h.lev[l];
    const MarchPlan mp = march_plan(v.nx, v.ny, v.nz, cached_resident(k_mg_prolong<float>, &r_pro));
    k_mg_prolong<float><<<mp.blocks, kMgThreads, 0, s>>>(v, h.lev[l + 1], mp, rhs(l), wgt(l),
                                                         h.wall_x, a.st);
    if (l == 0) {
      const MarchPlan m = march_plan(v.nx, v.ny, v.nz, cached_resident(k_mg_up<float, T, false>, &r_up0));
      k_mg_up<float, T, false><<<m.blocks, kMgThreads, 0, s>>>(v, m, in, out, a.st, a.I);
    } else {
      const MarchPlan m = march_plan(v.nx, v.ny, v.nz, cached_resident(k_mg_up<float, float, true>, &r_up));
      k_mg_up<float, float, true><<<m.blocks, kMgThreads, 0, s>>>(v, m, rhs(l), nullptr, a.st, a.I);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_mg_scale(const double* in, const double* sinv, long long n, double* out,
                            cudaStream_t s) {
  k_mg_scale<<<flat_grid(n), kMgThreads, 0, s>>>(in, sinv, n, out);
  return cudaGetLastError();
}

cudaError_t launch_mg_vcycle(const MgHier& h, int prec, const MgArgs& a, cudaStream_t s) {
  if (!h.mem) return cudaErrorInvalidValue;
  return prec == PREC_FP64 ? vcycle<double>(h, a, s) : vcycle<float>(h, a, s);
}

}  // namespace vdp
