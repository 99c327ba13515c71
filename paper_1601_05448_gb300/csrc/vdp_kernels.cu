// vdp_kernels.cu -- sm_103a kernels of libvdp.
//
// Problem (Sec. 3.4 of Pouransari, Mortazavi & Mani, arXiv:1601.05448): div((1/rho) grad p) = f
// on a uniform triply periodic staggered grid (Sec. 3.1, Sec. 3.2 case 1), discretised in
// conservative face-flux form with 1/rho on a face taken from the arithmetic mean of the two
// adjacent cell densities (the averaging App. B applies to rho off the cell centres), and
// f replaced by f - <f> (the compatibility constant chi' of App. A).
//
// Solver.  With A the FP64 operator and D its (negated) diagonal, the inner Krylov solver works
// on the Jacobi-scaled system  At = D^-1/2 (-A) D^-1/2  (unit diagonal, off-diagonal -bt with
// bt = b sinv_l sinv_r on each face).  Conjugate gradients on At is Jacobi-preconditioned CG in
// scaled variables, with one coefficient stream fewer and fewer FP64 operations per cell.  An
// outer FP64 loop evaluates the true residual r = (f - <f>) - A p, hands rt = D^-1/2 r to the
// inner solver (FP64, or FP32 with FP32/BF16 coefficients), and applies p -= D^-1/2 x.
//
// Kernels: the coefficient builders (set-up), and one step kernel that performs one sweep of
// the phase each instance is in (see vdp_internal.cuh).  A sweep is split into work units of
// full x rows x ty rows x tz planes; stencil sweeps march in z through a three-plane ring in
// shared memory that holds the rows of the unit plus one halo row on each side, so every
// value that feeds the 7-point stencil is loaded from global memory once per unit.
#include "vdp_internal.cuh"
#include "vdp_launch.h"

namespace vdp {

// ---- small helpers ----------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float ldc(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ double ldc(const double* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ldc(const __nv_bfloat16* p, long long i) {
  return __bfloat162float(p[i]);
}

template <class T> __device__ __forceinline__ T from_double_rn(double v);
template <> __device__ __forceinline__ double from_double_rn<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double_rn<float>(double v) {
  return __double2float_rn(v);
}

// global row index of ring row ry (0 = halo row above the unit, ty_eff + 1 = halo row below)
__device__ __forceinline__ int ring_gy(int ry, int y0, int ny) {
  int gy = y0 + ry - 1;
  if (gy < 0) gy += ny;
  if (gy >= ny) gy -= ny;
  return gy;
}

struct Unit {
  int y0, ty, z0, tz;
};

__device__ __forceinline__ Unit unit_geometry(const InstDesc& I, int unit) {
  Unit u;
  int uyi = unit % I.uy, uzi = unit / I.uy;
  u.y0 = uyi * I.ty;
  u.ty = min(I.ty, I.ny - u.y0);
  u.z0 = uzi * I.tz;
  u.tz = min(I.tz, I.nz - u.z0);
  return u;
}

// ---- reductions: per-unit partial slots, last unit reduces them in a fixed order --------------

__device__ __forceinline__ void store_partials(double (&v)[kSlots], double* part, int nunits,
                                               int unit) {
  __shared__ double red[kThreads / 32][kSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSlots; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kSlots; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      double s = lane < kThreads / 32 ? red[lane][k] : 0.0;
      s = warp_sum(s);
      if (lane == 0) part[k * nunits + unit] = s;
    }
  }
}

// Returns true in every thread of the unit that arrives last for its instance.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket, int nunits) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // partials of this unit visible before its ticket
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == (unsigned)nunits - 1u);
    if (last) __threadfence();
  }
  __syncthreads();
  return last != 0;
}

// Fixed-order sum of one slot over all units (warp 0; identical result in every lane).
__device__ __forceinline__ double sum_slot(const double* part, int nunits) {
  double s = 0.0;
  for (int i = threadIdx.x & 31; i < nunits; i += 32) s += __ldcg(part + i);
  return warp_sum(s);
}

// ---- phase transitions (run by thread 0 of the last unit) -------------------------------------

__device__ void transition(const InstDesc& I, InstState* st, int phase, const double (&S)[kSlots]) {
  st->sweeps += 1;
  switch (phase) {
    case PH_MEANF:
      st->mu_f = S[0] / (double)I.ncell;
      st->f2 = S[1];
      st->first_res = 1;
      st->phase = PH_RES64;
      break;
    case PH_RES64: {
      double rr64 = S[0], rrt = S[1];
      st->sum_p = S[2];
      if (st->first_res) {
        st->fn2 = S[3];
        st->first_res = 0;
      }
      st->outer += 1;
      double fn2 = st->fn2;
      if (fn2 <= 1e-28 * st->f2) {  // f is constant up to rounding: p = 0
        st->zero_sol = 1;
        st->rel_res = 0.0;
        st->phase = PH_FINAL;
        break;
      }
      double rel = sqrt(rr64 / fn2);
      st->rel_res = rel;
      if (!isfinite(rel)) {
        st->status = 5;  // VDP_EBREAKDOWN
        st->phase = PH_FINAL;
      } else if (rel <= st->tol) {
        st->phase = PH_FINAL;
      } else if (st->iters >= st->max_iter) {
        st->status = 4;  // VDP_ENOTCONV
        st->phase = PH_FINAL;
      } else if (rrt == 0.0) {  // residual below the inner type's range: cannot refine further
        st->status = 4;
        st->phase = PH_FINAL;
      } else {
        // How far the FP64 residual fell during the last inner solve compared with the scaled
        // inner residual; the next inner target is tightened by it (at least 1).
        if (st->outer > 1 && st->inner_ratio > 0.0) {
          double obs = sqrt(rr64 / st->rr64_prev) / st->inner_ratio;
          st->eta = fmax(1.0, fmin(obs, 1e6));
        }
        double tau = 0.5 * st->tol * sqrt(fn2 / rr64) / st->eta;
        if (st->precision != PREC_FP64) tau = fmax(tau, st->inner_tol);
        tau = fmin(tau, 0.5);
        st->tau2 = tau * tau;
        st->rr64_prev = rr64;
        st->rr64 = rr64;
        st->rr = rrt;
        st->rr0 = rrt;
        st->beta = 0.0;
        st->inner_iters = 0;
        st->phase = PH_STENCIL;
      }
      st->rr64 = rr64;
      break;
    }
    case PH_STENCIL: {
      double dq = S[0];
      if (dq > 0.0 && isfinite(dq)) {
        st->alpha = st->rr / dq;
        st->phase = PH_UPDATE;
      } else if (st->inner_iters > 0) {
        // loss of curvature at the end of an inner solve: hand the iterate to the refinement
        st->inner_ratio = sqrt(st->rr / st->rr0);
        st->phase = PH_CORRECT;
      } else {
        st->status = 5;
        st->phase = PH_FINAL;
      }
      break;
    }
    case PH_UPDATE: {
      double rn = S[0];
      st->inner_iters += 1;
      st->iters += 1;
      if (!isfinite(rn)) {
        st->status = 5;
        st->phase = PH_FINAL;
      } else if (rn <= st->tau2 * st->rr0 || st->iters >= st->max_iter ||
                 st->inner_iters >= st->inner_max) {
        st->inner_ratio = sqrt(rn / st->rr0);
        st->phase = PH_CORRECT;
      } else {
        st->beta = rn / st->rr;
        st->rr = rn;
        st->parity ^= 1;
        st->phase = PH_STENCIL;
      }
      break;
    }
    case PH_CORRECT:
      st->phase = PH_RES64;
      break;
    case PH_FINAL:
      st->phase = PH_DONE;
      break;
    default:
      break;
  }
}

// ---- sweeps -----------------------------------------------------------------------------------

// <f>, and p := 0 unless p is the caller's initial guess.
template <class T>
__device__ void sweep_meanf(const InstDesc& I, const InstState* st, const Unit& u,
                            double (&acc)[kSlots]) {
  const long long plane = (long long)I.nx * I.ny;
  const bool zero_p = !st->use_guess;
  const int len = u.ty * I.nx;  // multiple of 8: nx is
  double s = 0.0, s2 = 0.0;
  for (int k = 0; k < u.tz; ++k) {
    long long base = (long long)(u.z0 + k) * plane + (long long)u.y0 * I.nx;
    const double2* f2 = reinterpret_cast<const double2*>(I.rhs + base);
    double2* p2 = reinterpret_cast<double2*>(I.p + base);
    for (int v = threadIdx.x; v < len / 2; v += kThreads) {
      double2 fv = __ldg(f2 + v);
      s += fv.x;
      s += fv.y;
      s2 = fma(fv.x, fv.x, s2);
      s2 = fma(fv.y, fv.y, s2);
      if (zero_p) p2[v] = make_double2(0.0, 0.0);
    }
  }
  acc[0] = s;
  acc[1] = s2;
}

// p -= D^-1/2 x (x in the inner type)
template <class T>
__device__ void sweep_correct(const InstDesc& I, const Unit& u) {
  const long long plane = (long long)I.nx * I.ny;
  const int len = u.ty * I.nx;
  const T* x = static_cast<const T*>(I.x);
  for (int k = 0; k < u.tz; ++k) {
    long long base = (long long)(u.z0 + k) * plane + (long long)u.y0 * I.nx;
    for (int v = threadIdx.x; v < len; v += kThreads) {
      long long c = base + v;
      I.p[c] = fma(-__ldg(I.sinv + c), (double)x[c], I.p[c]);
    }
  }
}

// p -= <p>   (or p = 0 when the right-hand side was constant)
__device__ void sweep_final(const InstDesc& I, const InstState* st, const Unit& u) {
  const long long plane = (long long)I.nx * I.ny;
  const int len = u.ty * I.nx;
  const double mp = st->sum_p / (double)I.ncell;
  const bool zero = st->zero_sol != 0;
  for (int k = 0; k < u.tz; ++k) {
    long long base = (long long)(u.z0 + k) * plane + (long long)u.y0 * I.nx;
    double2* p2 = reinterpret_cast<double2*>(I.p + base);
    for (int v = threadIdx.x; v < len / 2; v += kThreads) {
      double2 pv = p2[v];
      p2[v] = zero ? make_double2(0.0, 0.0) : make_double2(pv.x - mp, pv.y - mp);
    }
  }
}

// x += alpha d (x = alpha d on the first inner iteration); rt -= alpha q; <rt, rt>
template <class T>
__device__ void sweep_update(const InstDesc& I, const InstState* st, const Unit& u,
                             double (&acc)[kSlots]) {
  const long long plane = (long long)I.nx * I.ny;
  const int len = u.ty * I.nx;
  const T alpha = (T)st->alpha;
  const bool first = st->inner_iters == 0;
  const T* d = static_cast<const T*>(st->parity ? I.d0 : I.d1);  // written by the last stencil
  const T* q = static_cast<const T*>(I.q);
  T* x = static_cast<T*>(I.x);
  T* r = static_cast<T*>(I.r);
  T s = 0;
  for (int k = 0; k < u.tz; ++k) {
    long long base = (long long)(u.z0 + k) * plane + (long long)u.y0 * I.nx;
    for (int v = threadIdx.x; v < len; v += kThreads) {
      long long c = base + v;
      T dv = d[c], qv = q[c];
      T xv = first ? (T)0 : x[c];
      x[c] = fma(alpha, dv, xv);
      T rv = fma(-alpha, qv, r[c]);
      r[c] = rv;
      s = fma(rv, rv, s);
    }
  }
  acc[0] = (double)s;
}

// d = rt + beta d_old on ring slot `slot` for plane zg (all ring rows of the unit)
template <class T>
__device__ __forceinline__ void fill_direction(const InstDesc& I, const Unit& u, T* ring,
                                               int stride, int slot, int zg, const T* rt,
                                               const T* dold, T beta, bool use_old) {
  const int nx = I.nx;
  const int cells = (u.ty + 2) * nx;
  const long long pz = (long long)zg * nx * I.ny;
  T* dst = ring + slot * stride;
  for (int m = threadIdx.x; m < cells; m += kThreads) {
    int ry = m / nx, x = m - ry * nx;
    long long c = pz + (long long)ring_gy(ry, u.y0, I.ny) * nx + x;
    T v = rt[c];
    if (use_old) v = fma(beta, dold[c], v);
    dst[m] = v;
  }
}

// d = rt + beta d_old (formed on the fly), q = At d, <d, q>; writes d and q for the unit
template <class T, class BT>
__device__ void sweep_stencil(const InstDesc& I, const InstState* st, const Unit& u,
                              double (&acc)[kSlots], T* ring) {
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int stride = (I.ty + 2) * nx;
  const long long plane = (long long)nx * ny;
  const T beta = (T)st->beta;
  const bool use_old = st->inner_iters > 0;
  const T* rt = static_cast<const T*>(I.r);
  const T* dold = static_cast<const T*>(st->parity ? I.d1 : I.d0);
  T* dnew = static_cast<T*>(st->parity ? I.d0 : I.d1);
  T* q = static_cast<T*>(I.q);
  const BT* sx = static_cast<const BT*>(I.sx);
  const BT* sy = static_cast<const BT*>(I.sy);
  const BT* sz = static_cast<const BT*>(I.sz);

  int zm = u.z0 - 1;
  if (zm < 0) zm += nz;
  fill_direction<T>(I, u, ring, stride, 0, zm, rt, dold, beta, use_old);
  fill_direction<T>(I, u, ring, stride, 1, u.z0, rt, dold, beta, use_old);
  T s = 0;
  const int own = u.ty * nx;
  for (int k = 0; k < u.tz; ++k) {
    const int z = u.z0 + k;
    const int zp = z + 1 == nz ? 0 : z + 1;
    const int sm = k % 3, sc = (k + 1) % 3, sp = (k + 2) % 3;
    fill_direction<T>(I, u, ring, stride, sp, zp, rt, dold, beta, use_old);
    __syncthreads();
    const T* Rm = ring + sm * stride;
    const T* Rc = ring + sc * stride;
    const T* Rp = ring + sp * stride;
    for (int m = threadIdx.x; m < own; m += kThreads) {
      const int ry = m / nx + 1, x = m - (ry - 1) * nx;
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      const int gy = u.y0 + ry - 1;
      const int gyp = gy + 1 == ny ? 0 : gy + 1;
      const long long row = (long long)z * plane + (long long)gy * nx;
      const long long c = row + x;
      const int o = ry * nx;
      T dc = Rc[o + x];
      T qv = dc;
      qv = fma(-(T)ldc(sx, c), Rc[o + xm], qv);
      qv = fma(-(T)ldc(sx, row + xp), Rc[o + xp], qv);
      qv = fma(-(T)ldc(sy, c), Rc[o - nx + x], qv);
      qv = fma(-(T)ldc(sy, (long long)z * plane + (long long)gyp * nx + x), Rc[o + nx + x], qv);
      qv = fma(-(T)ldc(sz, c), Rm[o + x], qv);
      qv = fma(-(T)ldc(sz, (long long)zp * plane + (long long)gy * nx + x), Rp[o + x], qv);
      dnew[c] = dc;
      q[c] = qv;
      s = fma(dc, qv, s);
    }
    __syncthreads();
  }
  acc[0] = (double)s;
}

// copy plane zg of p (all ring rows) into ring slot
__device__ __forceinline__ void fill_p(const InstDesc& I, const Unit& u, double* ring, int stride,
                                       int slot, int zg) {
  const int nx = I.nx;
  const int cells = (u.ty + 2) * nx;
  const long long pz = (long long)zg * nx * I.ny;
  double* dst = ring + slot * stride;
  for (int m = threadIdx.x; m < cells; m += kThreads) {
    int ry = m / nx, x = m - ry * nx;
    dst[m] = I.p[pz + (long long)ring_gy(ry, u.y0, I.ny) * nx + x];
  }
}

// FP64 residual r = (f - <f>) - A p; rt = D^-1/2 r in the inner type; sums of r^2, rt^2, p and,
// on the first call, (f - <f>)^2
template <class T>
__device__ void sweep_res64(const InstDesc& I, const InstState* st, const Unit& u,
                            double (&acc)[kSlots], double* ring) {
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int stride = (I.ty + 2) * nx;
  const long long plane = (long long)nx * ny;
  const double mu = st->mu_f;
  const bool first = st->first_res != 0;
  T* rt = static_cast<T*>(I.r);
  int zm = u.z0 - 1;
  if (zm < 0) zm += nz;
  fill_p(I, u, ring, stride, 0, zm);
  fill_p(I, u, ring, stride, 1, u.z0);
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const int own = u.ty * nx;
  for (int k = 0; k < u.tz; ++k) {
    const int z = u.z0 + k;
    const int zp = z + 1 == nz ? 0 : z + 1;
    const int sm = k % 3, sc = (k + 1) % 3, sp = (k + 2) % 3;
    fill_p(I, u, ring, stride, sp, zp);
    __syncthreads();
    const double* Rm = ring + sm * stride;
    const double* Rc = ring + sc * stride;
    const double* Rp = ring + sp * stride;
    for (int m = threadIdx.x; m < own; m += kThreads) {
      const int ry = m / nx + 1, x = m - (ry - 1) * nx;
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      const int gy = u.y0 + ry - 1;
      const int gyp = gy + 1 == ny ? 0 : gy + 1;
      const long long row = (long long)z * plane + (long long)gy * nx;
      const long long c = row + x;
      const int o = ry * nx;
      const double pc = Rc[o + x];
      double ap = __ldg(I.bx + row + xp) * (Rc[o + xp] - pc) - __ldg(I.bx + c) * (pc - Rc[o + xm]);
      ap += __ldg(I.by + (long long)z * plane + (long long)gyp * nx + x) * (Rc[o + nx + x] - pc) -
            __ldg(I.by + c) * (pc - Rc[o - nx + x]);
      ap += __ldg(I.bz + (long long)zp * plane + (long long)gy * nx + x) * (Rp[o + x] - pc) -
            __ldg(I.bz + c) * (pc - Rm[o + x]);
      const double f0 = __ldg(I.rhs + c) - mu;
      const double r = f0 - ap;
      const T tv = from_double_rn<T>(__ldg(I.sinv + c) * r);
      rt[c] = tv;
      a0 = fma(r, r, a0);
      a1 = fma((double)tv, (double)tv, a1);
      a2 += pc;
      if (first) a3 = fma(f0, f0, a3);
    }
    __syncthreads();
  }
  acc[0] = a0;
  acc[1] = a1;
  acc[2] = a2;
  acc[3] = a3;
}

// ---- the step kernel --------------------------------------------------------------------------

template <class T, class BT>
__global__ void __launch_bounds__(kThreads) k_step(const InstDesc* __restrict__ insts,
                                                   const UnitRef* __restrict__ units) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const UnitRef ur = units[blockIdx.x];
  const InstDesc& I = insts[ur.inst];
  InstState* st = I.st;
  const int phase = st->phase;
  if (phase >= PH_DONE) return;
  const Unit u = unit_geometry(I, ur.unit);
  double acc[kSlots] = {0.0, 0.0, 0.0, 0.0};
  switch (phase) {
    case PH_MEANF: sweep_meanf<T>(I, st, u, acc); break;
    case PH_RES64: sweep_res64<T>(I, st, u, acc, reinterpret_cast<double*>(smem_raw)); break;
    case PH_STENCIL: sweep_stencil<T, BT>(I, st, u, acc, reinterpret_cast<T*>(smem_raw)); break;
    case PH_UPDATE: sweep_update<T>(I, st, u, acc); break;
    case PH_CORRECT: sweep_correct<T>(I, u); break;
    case PH_FINAL: sweep_final(I, st, u); break;
    default: break;
  }
  store_partials(acc, I.part, I.nunits, ur.unit);
  if (arrive_last(I.ticket, I.nunits)) {
    if (threadIdx.x < 32) {
      double S[kSlots];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) S[k] = sum_slot(I.part + k * I.nunits, I.nunits);
      if (threadIdx.x == 0) {
        transition(I, st, phase, S);
        *I.ticket = 0u;
        __threadfence();
      }
    }
  }
}

// Per-solve initialisation of one instance's state.
__global__ void k_init(InstDesc* desc, const double* rhs, double* p, double tol, double inner_tol,
                       int max_iter, int inner_max, int use_guess, int precision) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  desc->rhs = rhs;
  desc->p = p;
  InstState* st = desc->st;
  InstState s;
  memset(&s, 0, sizeof(s));
  s.phase = PH_MEANF;
  s.status = 0;
  s.max_iter = max_iter;
  s.inner_max = inner_max;
  s.use_guess = use_guess;
  s.precision = precision;
  s.tol = tol;
  s.inner_tol = inner_tol;
  s.eta = 1.0;
  *st = s;
  *desc->ticket = 0u;
}

// ---- coefficient set-up -----------------------------------------------------------------------

__global__ void k_check_density(const double* __restrict__ rho, long long n, int* bad) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double v = rho[c];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, 1);
  }
}

// b_d[c] = 2 / (rho[c - e_d] + rho[c]) / h_d^2 on the low d-face of every cell
__global__ void k_faces(const double* __restrict__ rho, int nx, int ny, int nz, double ihx2,
                        double ihy2, double ihz2, double* bx, double* by, double* bz) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int x = (int)(c % nx);
    int y = (int)((c / nx) % ny);
    int z = (int)(c / plane);
    long long cxm = c - x + (x == 0 ? nx - 1 : x - 1);
    long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    double rc = rho[c];
    bx[c] = 2.0 / (rho[cxm] + rc) * ihx2;
    by[c] = 2.0 / (rho[cym] + rc) * ihy2;
    bz[c] = 2.0 / (rho[czm] + rc) * ihz2;
  }
}

// sinv = D^-1/2 with D = sum of the six face coefficients of the cell
__global__ void k_diag(const double* __restrict__ bx, const double* __restrict__ by,
                       const double* __restrict__ bz, int nx, int ny, int nz, double* sinv) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int x = (int)(c % nx);
    int y = (int)((c / nx) % ny);
    int z = (int)(c / plane);
    long long cxp = c - x + (x == nx - 1 ? 0 : x + 1);
    long long cyp = c + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx;
    long long czp = c + (long long)((z == nz - 1 ? 0 : z + 1) - z) * plane;
    double D = bx[c] + bx[cxp] + by[c] + by[cyp] + bz[c] + bz[czp];
    sinv[c] = 1.0 / sqrt(D);
  }
}

template <class BT> __device__ __forceinline__ BT to_coef(double v);
template <> __device__ __forceinline__ double to_coef<double>(double v) { return v; }
// rounded toward zero: the stored off-diagonals never exceed the exact ones, so the inner
// operator stays diagonally dominant (positive definite) after rounding
template <> __device__ __forceinline__ float to_coef<float>(double v) { return __double2float_rz(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_coef<__nv_bfloat16>(double v) {
  return __float2bfloat16_rz(__double2float_rz(v));
}

// bt_d[c] = b_d[c] sinv[c - e_d] sinv[c]
template <class BT>
__global__ void k_scaled(const double* __restrict__ bx, const double* __restrict__ by,
                         const double* __restrict__ bz, const double* __restrict__ sinv, int nx,
                         int ny, int nz, BT* sx, BT* sy, BT* sz) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int x = (int)(c % nx);
    int y = (int)((c / nx) % ny);
    int z = (int)(c / plane);
    long long cxm = c - x + (x == 0 ? nx - 1 : x - 1);
    long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    double s = sinv[c];
    sx[c] = to_coef<BT>(bx[c] * sinv[cxm] * s);
    sy[c] = to_coef<BT>(by[c] * sinv[cym] * s);
    sz[c] = to_coef<BT>(bz[c] * sinv[czm] * s);
  }
}

// out = A p (FP64)
__global__ void k_apply(const double* __restrict__ bx, const double* __restrict__ by,
                        const double* __restrict__ bz, const double* __restrict__ p, int nx, int ny,
                        int nz, double* __restrict__ out) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int x = (int)(c % nx);
    int y = (int)((c / nx) % ny);
    int z = (int)(c / plane);
    long long cxm = c - x + (x == 0 ? nx - 1 : x - 1), cxp = c - x + (x == nx - 1 ? 0 : x + 1);
    long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    long long cyp = c + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx;
    long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    long long czp = c + (long long)((z == nz - 1 ? 0 : z + 1) - z) * plane;
    double pc = p[c];
    out[c] = bx[cxp] * (p[cxp] - pc) - bx[c] * (pc - p[cxm]) + by[cyp] * (p[cyp] - pc) -
             by[c] * (pc - p[cym]) + bz[czp] * (p[czp] - pc) - bz[c] * (pc - p[czm]);
  }
}

// ---- host launchers ---------------------------------------------------------------------------

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_check_density(const double* rho, long long n, int* bad, cudaStream_t s) {
  k_check_density<<<grid_for(n), 256, 0, s>>>(rho, n, bad);
  return cudaGetLastError();
}

cudaError_t launch_build_coefficients(const double* rho, int nx, int ny, int nz, double L,
                                      double* bx, double* by, double* bz, double* sinv,
                                      cudaStream_t s) {
  long long n = (long long)nx * ny * nz;
  double hx = L / nx, hy = L / ny, hz = L / nz;
  k_faces<<<grid_for(n), 256, 0, s>>>(rho, nx, ny, nz, 1.0 / (hx * hx), 1.0 / (hy * hy),
                                      1.0 / (hz * hz), bx, by, bz);
  k_diag<<<grid_for(n), 256, 0, s>>>(bx, by, bz, nx, ny, nz, sinv);
  return cudaGetLastError();
}

cudaError_t launch_scaled(int prec, const double* bx, const double* by, const double* bz,
                          const double* sinv, int nx, int ny, int nz, void* sx, void* sy, void* sz,
                          cudaStream_t s) {
  long long n = (long long)nx * ny * nz;
  if (prec == PREC_FP64)
    k_scaled<double><<<grid_for(n), 256, 0, s>>>(bx, by, bz, sinv, nx, ny, nz, (double*)sx,
                                                 (double*)sy, (double*)sz);
  else if (prec == PREC_MIXED)
    k_scaled<float><<<grid_for(n), 256, 0, s>>>(bx, by, bz, sinv, nx, ny, nz, (float*)sx,
                                                (float*)sy, (float*)sz);
  else
    k_scaled<__nv_bfloat16><<<grid_for(n), 256, 0, s>>>(bx, by, bz, sinv, nx, ny, nz,
                                                        (__nv_bfloat16*)sx, (__nv_bfloat16*)sy,
                                                        (__nv_bfloat16*)sz);
  return cudaGetLastError();
}

cudaError_t launch_apply(const double* bx, const double* by, const double* bz, const double* p,
                         int nx, int ny, int nz, double* out, cudaStream_t s) {
  long long n = (long long)nx * ny * nz;
  k_apply<<<grid_for(n), 256, 0, s>>>(bx, by, bz, p, nx, ny, nz, out);
  return cudaGetLastError();
}

cudaError_t launch_init(InstDesc* desc, const double* rhs, double* p, double tol, double inner_tol,
                        int max_iter, int inner_max, int use_guess, int precision,
                        cudaStream_t s) {
  k_init<<<1, 32, 0, s>>>(desc, rhs, p, tol, inner_tol, max_iter, inner_max, use_guess,
                          precision);
  return cudaGetLastError();
}

static void* step_fn(int prec) {
  if (prec == PREC_FP64) return (void*)k_step<double, double>;
  if (prec == PREC_MIXED) return (void*)k_step<float, float>;
  return (void*)k_step<float, __nv_bfloat16>;
}

cudaError_t prepare_step(int prec, size_t smem_bytes) {
  return cudaFuncSetAttribute(step_fn(prec), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes);
}

cudaError_t launch_step(int prec, const InstDesc* desc, const UnitRef* units, int nunits,
                        size_t smem_bytes, cudaStream_t s) {
  if (prec == PREC_FP64)
    k_step<double, double><<<nunits, kThreads, smem_bytes, s>>>(desc, units);
  else if (prec == PREC_MIXED)
    k_step<float, float><<<nunits, kThreads, smem_bytes, s>>>(desc, units);
  else
    k_step<float, __nv_bfloat16><<<nunits, kThreads, smem_bytes, s>>>(desc, units);
  return cudaGetLastError();
}

}  // namespace vdp
