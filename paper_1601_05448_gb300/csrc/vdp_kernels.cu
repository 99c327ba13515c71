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
// The preconditioned residual z (Chebyshev polynomial or the spectral passes of
// vdp_spectral.cu) replaces rt as the stencil sweep's source; the paper's fixed-point iteration
// runs as the same sweeps with beta = 0 and alpha = 1.
//
// Kernels: the coefficient builders (set-up) and three sweep kernels, each advancing every
// instance whose phase is of its kind (see vdp_internal.cuh): k_res64_direct (FP64 residual),
// k_stencil_direct (search direction, stencil product and <d, q>; Chebyshev sweeps in its
// CHEBOK variant) and k_flat (element-wise phases).  The direct sweeps march each work unit
// through a z chunk with three planes in registers: a thread owns 16 bytes of one row, takes
// its x neighbours from the adjacent lanes by warp shuffle and the rows above and below from
// L1/L2, and waits on no other warp.  k_stencil_tma is the TMA-staged variant (cp.async.bulk
// row blocks into a shared-memory ring, mbarrier completion with bounded waits, one block
// barrier per plane), kept as an option; k_persistent runs all of them for a batch.
#include "vdp_device.cuh"
#include "vdp_internal.cuh"
#include "vdp_launch.h"

namespace vdp {

// ---- small helpers ----------------------------------------------------------------------------

template <class T> __device__ __forceinline__ T from_double_rn(double v);
template <> __device__ __forceinline__ double from_double_rn<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double_rn<float>(double v) {
  return __double2float_rn(v);
}

// global row index of ring row ry (0 = halo row above the tile, ty + 1 = halo row below)
__device__ __forceinline__ int ring_gy(int ry, int y0, int ny) {
  int gy = y0 + ry - 1;
  if (gy < 0) gy += ny;
  if (gy >= ny) gy -= ny;
  return gy;
}

// Vector width per thread: 16-byte accesses of the inner type.
template <class T> struct VecW;
template <> struct VecW<float> { static constexpr int V = 4; };
template <> struct VecW<double> { static constexpr int V = 2; };

template <class T, int V> struct VecIO;
template <> struct VecIO<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&o)[4]) {
    float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <> struct VecIO<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&o)[2]) {
    double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&o)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  }
};

// the same, through the read-only (non-coherent) load path: only for data no thread of the
// running kernel writes
template <class T, int V> struct LdgIO;
template <> struct LdgIO<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&o)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
};
template <> struct LdgIO<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&o)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = t.x; o[1] = t.y;
  }
};
// V coefficients of storage type BT into arithmetic type T
template <class BT, class T, int V> struct CoefIO;
template <> struct CoefIO<float, float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&o)[4]) {
    VecIO<float, 4>::ld(p, o);
  }
  static __device__ __forceinline__ void ldg(const float* p, float (&o)[4]) {
    LdgIO<float, 4>::ld(p, o);
  }
};
template <> struct CoefIO<double, double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&o)[2]) {
    VecIO<double, 2>::ld(p, o);
  }
  static __device__ __forceinline__ void ldg(const double* p, double (&o)[2]) {
    LdgIO<double, 2>::ld(p, o);
  }
};
template <> struct CoefIO<__nv_bfloat16, float, 4> {
  static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float (&o)[4]) {
    uint2 u = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
  }
  static __device__ __forceinline__ void ldg(const __nv_bfloat16* p, float (&o)[4]) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    o[0] = __uint_as_float(u.x << 16); o[1] = __uint_as_float(u.x & 0xffff0000u);
    o[2] = __uint_as_float(u.y << 16); o[3] = __uint_as_float(u.y & 0xffff0000u);
  }
};

__device__ __forceinline__ float ldg1(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldg1(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg1(const __nv_bfloat16* p) {
  const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
  return __uint_as_float((unsigned)u << 16);
}

__device__ __forceinline__ float ld1(const float* p) { return *p; }
__device__ __forceinline__ double ld1(const double* p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// ---- TMA bulk copies and mbarriers (inline PTX) -----------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared accesses before later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier, giving up after ~2 s (returns false); no hang.
__device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
}

// ---- unit geometry -------------------------------------------------------------------------------

struct Seg {
  int y0, ty;   // row tile: first row, rows
  int z0, nzs;  // first plane, planes
};

// Calls fn(seg) for the z run of work unit `unit`: row tile unit % uy, z chunk unit / uy.  Units
// that run at the same time share z chunks, so the halo rows one unit reads are the rows its
// neighbours stream at about the same moment (L2 hits rather than DRAM re-reads).
template <class F>
__device__ __forceinline__ void for_each_segment(const InstDesc& I, int unit, F&& fn) {
  const int tile = unit % I.uy, chunk = unit / I.uy;
  Seg s;
  s.y0 = tile * I.ty;
  s.ty = min(I.ty, I.ny - s.y0);
  s.z0 = (int)((long long)chunk * I.nz / I.zc);
  s.nzs = (int)((long long)(chunk + 1) * I.nz / I.zc) - s.z0;
  if (s.nzs > 0) fn(s);
}

// ---- flat (element-wise) sweeps ------------------------------------------------------------------
// Run by k_flat, a kernel without dynamic shared memory (full occupancy).  Flat unit u of
// nunits_f covers the contiguous cells [flat_begin(u), flat_begin(u + 1)), multiples of 8, so
// every access is a 16-byte vector; each thread keeps four vectors in flight and several
// independent partial sums.

__device__ __forceinline__ long long flat_begin(const InstDesc& I, int u) {
  return ((long long)u * (I.ncell / 8) / I.nunits_f) * 8;
}

// Vectors per thread kept in flight by the FP64 flat sweeps below: all loads of a round are issued
// before the first use (one vector per thread per round left these sweeps latency bound).
constexpr int kFlatU = 4;

__device__ __forceinline__ double widen_t(float v) { return widen(v); }
__device__ __forceinline__ double widen_t(double v) { return v; }

// <f>, ||f||^2; p := 0 unless p is the caller's initial guess.
__device__ void sweep_meanf(const InstDesc& I, long long c0, long long c1, double& sum) {
  // <f> in FP64, one addition per cell.  p is not cleared here: from p = 0 the first residual
  // does not read it, the first correction writes it without reading it, and the gauge writes
  // zeros if no correction ever came.
  double s[2] = {0.0, 0.0};
  const long long step = 2LL * blockDim.x;
  for (long long cb = c0 + 2 * threadIdx.x; cb < c1; cb += kFlatU * step) {
    double2 fv[kFlatU];
#pragma unroll
    for (int u = 0; u < kFlatU; ++u) {
      const long long c = cb + u * step;
      fv[u] = c < c1 ? __ldg(reinterpret_cast<const double2*>(I.rhs + c)) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < kFlatU; ++u) {
      s[0] += fv[u].x;
      s[1] += fv[u].y;
    }
  }
  sum = s[0] + s[1];
}

// p -= D^-1/2 x (x in the inner type); sums the new p (the final gauge needs its mean).  fresh:
// p is still the zero start (never written), so p = -D^-1/2 x without reading it.
template <class T>
__device__ void sweep_correct(const InstDesc& I, long long c0, long long c1, bool fresh,
                              double& psum) {
  const T* x = static_cast<const T*>(I.x);
  double s = 0.0;
  const long long step = 2LL * blockDim.x;
  constexpr int U = kFlatU / 2;  // four operands per vector: half the vectors in flight
  for (long long cb = c0 + 2 * threadIdx.x; cb < c1; cb += U * step) {
    double2 sv[U], pv[U];
    T xa[U], xb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long c = cb + u * step;
      if (c < c1) {
        sv[u] = __ldg(reinterpret_cast<const double2*>(I.sinv + c));
        pv[u] = fresh ? make_double2(0.0, 0.0) : *reinterpret_cast<const double2*>(I.p + c);
        xa[u] = x[c];
        xb[u] = x[c + 1];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long c = cb + u * step;
      if (c < c1) {
        double2 p = pv[u];
        p.x = fma(-sv[u].x, widen_t(xa[u]), p.x);
        p.y = fma(-sv[u].y, widen_t(xb[u]), p.y);
        *reinterpret_cast<double2*>(I.p + c) = p;
        s += p.x + p.y;
      }
    }
  }
  psum = s;
}

// p -= <p>   (or p = 0 when the right-hand side was constant)
__device__ void sweep_final(const InstDesc& I, const InstState* st, long long c0, long long c1) {
  const double mp = st->sum_p / (double)I.ncell;
  const bool zero = st->zero_sol != 0 || st->p_set == 0;  // no iterate: the answer is p = 0
  const long long step = 2LL * blockDim.x;
  for (long long cb = c0 + 2 * threadIdx.x; cb < c1; cb += kFlatU * step) {
    double2 pv[kFlatU];
#pragma unroll
    for (int u = 0; u < kFlatU; ++u) {
      const long long c = cb + u * step;
      if (c < c1) pv[u] = *reinterpret_cast<const double2*>(I.p + c);
    }
#pragma unroll
    for (int u = 0; u < kFlatU; ++u) {
      const long long c = cb + u * step;
      if (c < c1)
        *reinterpret_cast<double2*>(I.p + c) =
            zero ? make_double2(0.0, 0.0) : make_double2(pv[u].x - mp, pv[u].y - mp);
    }
  }
}

// x += alpha d (x = alpha d on the first inner iteration); rt -= alpha q; <rt, rt>
template <class T>
__device__ void sweep_update(const InstDesc& I, const InstState* st, long long c0, long long c1,
                             T& part) {
  constexpr int V = VecW<T>::V;
  constexpr int U = 2;  // vectors per thread per round
  const T alpha = (T)st->alpha;
  const bool first = st->inner_iters == 0;
  // written by the last stencil sweep (the fixed-point iteration's direction is z itself)
  const T* d = static_cast<const T*>(I.pc == PC_FIXED ? I.za : (st->parity ? I.d0 : I.d1));
  const T* q = static_cast<const T*>(I.q);
  T* x = static_cast<T*>(I.x);
  T* rt = static_cast<T*>(I.r);
  T s[U];
#pragma unroll
  for (int u = 0; u < U; ++u) s[u] = 0;
  const long long step = (long long)V * blockDim.x;
  for (long long cb = c0 + (long long)V * threadIdx.x; cb < c1; cb += U * step) {
    T dv[U][V], qv[U][V], xv[U][V], rv[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long c = cb + u * step;
      if (c < c1) {
        VecIO<T, V>::ld(d + c, dv[u]);
        VecIO<T, V>::ld(q + c, qv[u]);
        VecIO<T, V>::ld(rt + c, rv[u]);
        if (!first) VecIO<T, V>::ld(x + c, xv[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long c = cb + u * step;
      if (c >= c1) continue;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        xv[u][k] = fma(alpha, dv[u][k], first ? (T)0 : xv[u][k]);
        rv[u][k] = fma(-alpha, qv[u][k], rv[u][k]);
        s[u] = fma(rv[u][k], rv[u][k], s[u]);
      }
      VecIO<T, V>::st(x + c, xv[u]);
      VecIO<T, V>::st(rt + c, rv[u]);
    }
  }
  T tot = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) tot += s[u];
  part = tot;
}

// ---- the stencil sweep: TMA-fed z march -----------------------------------------------------------

// BF16 coefficients carry a per-cell diagonal correction (see k_diag_correction).
template <class BT> struct CoefTraits { static constexpr bool kDiag = false; };
template <> struct CoefTraits<__nv_bfloat16> { static constexpr bool kDiag = true; };

template <class T, class BT>
struct StageLayout {
  int nx, ty;
  __device__ __forceinline__ size_t r_off() const { return 0; }
  __device__ __forceinline__ size_t o_off() const { return (size_t)(ty + 2) * nx * sizeof(T); }
  __device__ __forceinline__ size_t bx_off() const { return (size_t)2 * (ty + 2) * nx * sizeof(T); }
  __device__ __forceinline__ size_t by_off() const { return bx_off() + (size_t)ty * nx * sizeof(BT); }
  __device__ __forceinline__ size_t bz_off() const {
    return by_off() + (size_t)(ty + 1) * nx * sizeof(BT);
  }
  __device__ __forceinline__ size_t bd_off() const { return bz_off() + (size_t)ty * nx * sizeof(BT); }
};

// Issue part `part` (0..3) of the bulk copies of plane `j` (j = -1 .. nzs) of segment `sg` into
// stage buffer `buf`; lane 0 of warps 0..3 issue one part each, so the four arrive on the stage's
// mbarrier (count 4) with their own byte counts.  Part 0: rt rows (tile + one halo row above and
// below); 1: d_old rows (when the direction recurrence needs it); 2: x and y coefficients;
// 3: z coefficients (+ BF16 diagonal correction).  Plane -1 needs only rt / d_old (it supplies d
// below the segment); plane nzs needs rt / d_old and the z coefficients (its low z face is the
// high face of the last plane).
template <class T, class BT>
__device__ __forceinline__ void issue_part(int part, const InstDesc& I, const Seg& sg, int j,
                                           unsigned char* buf, uint64_t* bar, const T* rt,
                                           const T* dold, bool use_old, const BT* sx,
                                           const BT* sy, const BT* sz, const BT* sd) {
  const StageLayout<T, BT> L{I.nx, I.ty};
  int zg = sg.z0 + j;
  if (zg < 0) zg += I.nz;
  if (zg >= I.nz) zg -= I.nz;
  const int nx = I.nx;
  const long long plane = (long long)zg * I.ny;
  const uint32_t rowT = nx * sizeof(T), rowB = nx * sizeof(BT);
  if (part <= 1) {
    const T* src = part == 0 ? rt : dold;
    if (part == 1 && !use_old) {
      mbar_arrive_expect_tx(bar, 0);
      return;
    }
    const int top = ring_gy(0, sg.y0, I.ny), bot = ring_gy(sg.ty + 1, sg.y0, I.ny);
    unsigned char* R = buf + (part == 0 ? L.r_off() : L.o_off());
    mbar_arrive_expect_tx(bar, (uint32_t)(sg.ty + 2) * rowT);
    bulk_g2s(R, src + (plane + top) * nx, rowT, bar);
    bulk_g2s(R + rowT, src + (plane + sg.y0) * nx, sg.ty * rowT, bar);
    bulk_g2s(R + (sg.ty + 1) * rowT, src + (plane + bot) * nx, rowT, bar);
  } else if (part == 2) {
    if (!(j >= 0 && j < sg.nzs)) {
      mbar_arrive_expect_tx(bar, 0);
      return;
    }
    mbar_arrive_expect_tx(bar, (uint32_t)(2 * sg.ty + 1) * rowB);
    bulk_g2s(buf + L.bx_off(), sx + (plane + sg.y0) * nx, sg.ty * rowB, bar);
    unsigned char* BY = buf + L.by_off();
    if (sg.y0 + sg.ty < I.ny) {
      bulk_g2s(BY, sy + (plane + sg.y0) * nx, (sg.ty + 1) * rowB, bar);
    } else {  // the row below the tile wraps to row 0
      bulk_g2s(BY, sy + (plane + sg.y0) * nx, sg.ty * rowB, bar);
      bulk_g2s(BY + sg.ty * rowB, sy + plane * nx, rowB, bar);
    }
  } else {
    const bool need_z = j >= 0, need_d = CoefTraits<BT>::kDiag && j >= 0 && j < sg.nzs;
    mbar_arrive_expect_tx(bar, (uint32_t)((need_z ? sg.ty : 0) + (need_d ? sg.ty : 0)) * rowB);
    if (need_z) bulk_g2s(buf + L.bz_off(), sz + (plane + sg.y0) * nx, sg.ty * rowB, bar);
    if (need_d) bulk_g2s(buf + L.bd_off(), sd + (plane + sg.y0) * nx, sg.ty * rowB, bar);
  }
}

// d = rt + beta d_old in place over all ring rows of a stage
template <class T>
__device__ __forceinline__ void form_direction(T* R, const T* O, int cells, T beta) {
  constexpr int V = VecW<T>::V;
  for (int v = threadIdx.x; v < cells / V; v += blockDim.x) {
    T a[V], b[V];
    VecIO<T, V>::ld(R + v * V, a);
    VecIO<T, V>::ld(O + v * V, b);
#pragma unroll
    for (int k = 0; k < V; ++k) a[k] = fma(beta, b[k], a[k]);
    VecIO<T, V>::st(R + v * V, a);
  }
}

// One z march per segment.  Iteration k (plane k of the segment) forms d two planes ahead
// (plane k + 2, stage k + 3) while it applies the stencil to plane k from the stages of planes
// k - 1, k, k + 1, so one block barrier per plane separates the two; the barrier also frees the
// stage of plane k - 1, which thread 0 then refills with plane k - 1 + S.  S >= 4 stages.
template <class T, class BT>
__device__ void sweep_stencil(const InstDesc& I, InstState* st, int unit, T& part,
                              unsigned char* smem) {
  constexpr int V = VecW<T>::V;
  constexpr bool kDiag = CoefTraits<BT>::kDiag;
  __shared__ __align__(8) uint64_t bars[kMaxStages];
  __shared__ int timed_out;
  const int S = I.stages;
  const int nx = I.nx;
  const StageLayout<T, BT> L{nx, I.ty};
  const size_t sbytes = stage_bytes(nx, I.ty, sizeof(T), sizeof(BT), kDiag);
  const T beta = (T)st->beta;
  const bool use_old = st->inner_iters > 0;
  const T* rt = static_cast<const T*>(I.r);
  const T* dold = static_cast<const T*>(st->parity ? I.d1 : I.d0);
  T* dnew = static_cast<T*>(st->parity ? I.d0 : I.d1);
  T* q = static_cast<T*>(I.q);
  const BT* sx = static_cast<const BT*>(I.sx);
  const BT* sy = static_cast<const BT*>(I.sy);
  const BT* sz = static_cast<const BT*>(I.sz);
  const BT* sd = static_cast<const BT*>(I.sd);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 4);  // four issuing lanes arrive per fill
    fence_mbar_init();
    timed_out = 0;
  }
  __syncthreads();
  uint32_t parity = 0;  // bit s: phase parity of the next completion of stage s
  T sum[V];
#pragma unroll
  for (int k = 0; k < V; ++k) sum[k] = 0;

  auto stage_ptr = [&](int jj) { return smem + (size_t)(jj % S) * sbytes; };
  auto wait_stage = [&](int jj) {
    const int s = jj % S;
    if (!timed_out && !mbar_wait(&bars[s], (parity >> s) & 1u)) timed_out = 1;
    parity ^= 1u << s;
  };
  auto ready = [&](int jj, int ring_cells) {  // wait for stage jj and form d in it
    wait_stage(jj);
    if (use_old) {
      unsigned char* b = stage_ptr(jj);
      form_direction<T>(reinterpret_cast<T*>(b + L.r_off()),
                        reinterpret_cast<const T*>(b + L.o_off()), ring_cells, beta);
    }
  };

  for_each_segment(I, unit, [&](const Seg& sg) {
    const int np = sg.nzs + 2;  // planes -1 .. nzs, stage index jj = j + 1
    const int ring_cells = (sg.ty + 2) * nx;
    const int part = threadIdx.x >> 5;  // issuing lanes: lane 0 of warps 0..3
    const bool issuer = (threadIdx.x & 31) == 0 && part < 4;
    if (issuer) {
      fence_proxy_async_smem();  // stage buffers were last touched by ordinary loads/stores
      for (int jj = 0; jj < min(S, np); ++jj)
        issue_part<T, BT>(part, I, sg, jj - 1, stage_ptr(jj), &bars[jj % S], rt, dold, use_old, sx,
                          sy, sz, sd);
    }
    ready(0, ring_cells);  // plane -1
    ready(1, ring_cells);  // plane 0
    ready(2, ring_cells);  // plane 1 (exists: np >= 3)
    __syncthreads();
    const int vrow = nx / V;
    const int own = sg.ty * vrow;  // vectors in the tile's own rows
    for (int k = 0; k < sg.nzs; ++k) {
      const int z = sg.z0 + k;
      if (k + 3 < np) ready(k + 3, ring_cells);  // plane k + 2
      const unsigned char* bm = stage_ptr(k);
      const unsigned char* bc = stage_ptr(k + 1);
      const unsigned char* bp = stage_ptr(k + 2);
      const T* Dm = reinterpret_cast<const T*>(bm + L.r_off());
      const T* Dc = reinterpret_cast<const T*>(bc + L.r_off());
      const T* Dp = reinterpret_cast<const T*>(bp + L.r_off());
      const BT* Bx = reinterpret_cast<const BT*>(bc + L.bx_off());
      const BT* By = reinterpret_cast<const BT*>(bc + L.by_off());
      const BT* Bz = reinterpret_cast<const BT*>(bc + L.bz_off());
      const BT* Bd = reinterpret_cast<const BT*>(bc + L.bd_off());
      const BT* Bzp = reinterpret_cast<const BT*>(bp + L.bz_off());
      for (int v = threadIdx.x; v < own; v += blockDim.x) {
        const int row = v / vrow;               // 0 .. ty-1
        const int x0 = (v - row * vrow) * V;
        const int o = (row + 1) * nx;           // ring row of this tile row
        const int ob = row * nx;                // coefficient row
        T dc[V], du[V], dd[V], dzm[V], dzp[V];
        T bx[V], by[V], byd[V], bz[V], bzp[V], bd[V];
        VecIO<T, V>::ld(Dc + o + x0, dc);
        VecIO<T, V>::ld(Dc + o - nx + x0, du);
        VecIO<T, V>::ld(Dc + o + nx + x0, dd);
        VecIO<T, V>::ld(Dm + o + x0, dzm);
        VecIO<T, V>::ld(Dp + o + x0, dzp);
        CoefIO<BT, T, V>::ld(Bx + ob + x0, bx);
        CoefIO<BT, T, V>::ld(By + ob + x0, by);
        CoefIO<BT, T, V>::ld(By + ob + nx + x0, byd);
        CoefIO<BT, T, V>::ld(Bz + ob + x0, bz);
        CoefIO<BT, T, V>::ld(Bzp + ob + x0, bzp);
        if (kDiag) CoefIO<BT, T, V>::ld(Bd + ob + x0, bd);
        const int xl = x0 == 0 ? nx - 1 : x0 - 1;
        const int xr = x0 + V == nx ? 0 : x0 + V;
        const T dl = Dc[o + xl], dr = Dc[o + xr];
        const T bxr = (T)ld1(Bx + ob + xr);
        T qv[V];
#pragma unroll
        for (int k2 = 0; k2 < V; ++k2) {
          const T left = k2 == 0 ? dl : dc[k2 - 1];
          const T right = k2 == V - 1 ? dr : dc[k2 + 1];
          const T bright = k2 == V - 1 ? bxr : bx[k2 + 1];
          T a = dc[k2];
          if (kDiag) a = fma(bd[k2], dc[k2], a);
          a = fma(-bx[k2], left, a);
          a = fma(-bright, right, a);
          a = fma(-by[k2], du[k2], a);
          a = fma(-byd[k2], dd[k2], a);
          a = fma(-bz[k2], dzm[k2], a);
          a = fma(-bzp[k2], dzp[k2], a);
          qv[k2] = a;
          sum[k2] = fma(dc[k2], a, sum[k2]);
        }
        const long long g = ((long long)z * I.ny + sg.y0 + row) * nx + x0;
        VecIO<T, V>::st(dnew + g, dc);
        VecIO<T, V>::st(q + g, qv);
      }
      fence_proxy_async_smem();  // this thread's shared accesses before the refill's TMA writes
      __syncthreads();           // stage k (plane k - 1) is free; plane k + 2 is formed
      if (issuer && k + S < np) {
        issue_part<T, BT>(part, I, sg, k + S - 1, stage_ptr(k + S), &bars[(k + S) % S], rt, dold,
                          use_old, sx, sy, sz, sd);
      }
    }
  });
  if (timed_out && threadIdx.x == 0) atomicExch(&st->fault, 1);
  T tot = 0;
#pragma unroll
  for (int k = 0; k < V; ++k) tot += sum[k];
  part = tot;
}

// ---- the stencil sweep, direct form: register z march, no shared memory, no block barrier --------
// Each thread owns V consecutive cells of one row of the unit's row tile (tile = blockDim * V / nx
// rows) and marches them through the unit's z chunk, keeping d of planes z-1, z, z+1 in registers.
// Per plane it loads, as 16-byte vectors, rt and d_old of its own row at z+1 and of the rows above
// and below at z (forming d there: the neighbouring threads' rows, so these loads hit L1/L2), and
// the coefficients of its cells; x neighbours come from the adjacent lanes by warp shuffle (row
// ends, which wrap, are loaded).  Nothing waits on another warp, so many warps per SM keep many
// independent loads in flight.  Measured on the 256^3 FP32 sweep this runs at about 90 % of the
// HBM copy bandwidth, against about 50 % for the TMA-staged variant above, whose per-plane block
// barrier serialises the copy latency with the arithmetic.
//
// CHEB = true: one sweep j of the Chebyshev polynomial preconditioner instead (same march, the
// marched field is the Chebyshev iterate z_j, z_1 = rt / theta formed on the fly):
//   d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) (rt - At z_j),  z_{j+1} = z_j + d_j,
// with rho_0 = 1 / sigma, rho_j = 1 / (2 sigma - rho_{j-1}), sigma = theta / delta, d_0 = z_1;
// the last sweep also sums <rt, z>.
template <class T> struct IsF64 { static constexpr bool value = false; };
template <> struct IsF64<double> { static constexpr bool value = true; };

// VAR selects the variant at compile time (a predicated-off FMA still costs FP64-pipe slots):
//   0  first iteration of an inner CG solve (no search-direction history), or a Chebyshev sweep
//   1  CG with history (d = z + beta d_old)
//   2  the paper's fixed-point iteration (no history, no <d, q>, d not stored)
template <class T, class BT, bool CHEB, int VAR>
__device__ void sweep_stencil_direct(const InstDesc& I, const InstState* st, int unit, T& part) {
  constexpr int V = VecW<T>::V;
  constexpr bool kDiag = CoefTraits<BT>::kDiag;
  // FP64 sweeps are bound by the FP64 pipe, not by HBM: there the stencil is applied to the
  // preconditioned residual z itself, and q = At d follows from q = At z + beta q_old, with
  // d = z + beta d_old formed for the thread's own cells only (9 FP64 operations per cell
  // instead of also forming d for the rows above and below and the row ends).  FP32 sweeps are
  // HBM bound and keep forming d, which reads one vector (q_old) less.
  constexpr bool QREC = !CHEB && IsF64<T>::value;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int tpr = nx / V;  // threads per row
  const int tile = unit % I.uy, chunk = unit / I.uy;
  const int row = threadIdx.x / tpr;
  const int x0 = (threadIdx.x - row * tpr) * V;
  const int yr = tile * I.ty + row;
  const bool active = row < I.ty && yr < ny;
  const int y = active ? yr : ny - 1;  // idle threads follow a valid row (shuffles need them)
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int z0 = (int)((long long)chunk * nz / I.zc), z1 = (int)((long long)(chunk + 1) * nz / I.zc);
  const int lane = threadIdx.x & 31;
  const bool row_start = x0 == 0, row_end = x0 + V == nx;
  const int xl = row_start ? nx - 1 : x0 - 1, xr = row_end ? 0 : x0 + V;
  // STENCIL: marched field d = src + beta d_old, src = rt (Jacobi) or the final Chebyshev z
  // CHEB:    marched field z_j = src * scale, src = rt / z buffer, scale = 1 / theta or 1
  const int cj = CHEB ? st->cheb_j : 0;
  const bool last = CHEB && cj == I.cheb_k - 1;
  T beta = (T)st->beta, scale = 1, c1 = 0, c2 = 0;
  // the paper's fixed-point iteration has no search-direction history (beta = 0) and needs
  // neither d nor q: the sweep applies the update itself on the thread's own cells,
  // x += z and rt -= At z, and sums <rt, rt> (one pass instead of a stencil and an update sweep)
  constexpr bool fixed = VAR == 2;
  const bool first_inner = st->inner_iters == 0;
  T* xv = static_cast<T*>(I.x);
  T* rw = static_cast<T*>(I.r);
  constexpr bool use_old = VAR == 1 && !CHEB;
  constexpr bool form = use_old && !QREC;  // form d = src + beta d_old for every marched value
  const T* rt = static_cast<const T*>(I.r);
  const T* src = I.pc != PC_JACOBI ? static_cast<const T*>(I.za) : rt;
  // the fixed-point iteration's z comes from the FP32 spectral passes and is stored as FP32
  // (exactly representable: widening it loses nothing)
  const float* srcf = static_cast<const float*>(I.za);
  const T* dold = static_cast<const T*>(st->parity ? I.d1 : I.d0);
  T* dnew = static_cast<T*>(st->parity ? I.d0 : I.d1);
  T* q = static_cast<T*>(I.q);
  T* zout = nullptr;
  T* dch = static_cast<T*>(I.dch);
  if (CHEB) {
    // sweep j reads z_j from buffer (k - j) % 2 and writes z_{j+1} to (k - 1 - j) % 2, so the
    // last sweep (j = k - 1) leaves z in za
    const int k = I.cheb_k;
    src = cj == 1 ? rt : static_cast<const T*>(((k - cj) & 1) ? I.zb : I.za);
    zout = static_cast<T*>(((k - 1 - cj) & 1) ? I.zb : I.za);
    scale = cj == 1 ? (T)(1.0 / I.cheb_theta) : (T)1;
    const double sigma = I.cheb_theta / I.cheb_delta;
    double rp = 1.0 / sigma, r = rp;
    for (int i = 1; i <= cj; ++i) {
      rp = r;
      r = 1.0 / (2.0 * sigma - rp);
    }
    c1 = (T)(r * rp);                  // rho_j rho_{j-1}
    c2 = (T)(2.0 * r / I.cheb_delta);  // 2 rho_j / delta
    beta = 0;
  }
  const BT* sx = static_cast<const BT*>(I.sx);
  const BT* sy = static_cast<const BT*>(I.sy);
  const BT* sz = static_cast<const BT*>(I.sz);
  const BT* sd = static_cast<const BT*>(I.sd);
  const long long plane = (long long)nx * ny;
  const long long dym = (long long)(ym - y) * nx, dyp = (long long)(yp - y) * nx;
  const int dxl = xl - x0, dxr = xr - x0;
  const long long cell0 = (long long)y * nx + x0;  // offset of the thread's cells in a plane
  auto zoff = [&](int z) -> long long {             // plane z (may be -1 or nz) + own cells
    return (long long)(z < 0 ? z + nz : (z >= nz ? z - nz : z)) * plane + cell0;
  };
  // all loads of a plane are issued together (non-coherent read-only path), then used
  auto dvec = [&](long long o, T (&d)[V]) {  // marched field, V cells at offset o
    if constexpr (fixed && IsF64<T>::value) {
#pragma unroll
      for (int k = 0; k < V; k += 2) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(srcf + o + k));
        d[k] = widen(t.x);
        d[k + 1] = widen(t.y);
      }
    } else {
      LdgIO<T, V>::ld(src + o, d);
    }
    if (CHEB) {
#pragma unroll
      for (int k = 0; k < V; ++k) d[k] *= scale;
    } else if (form) {
      T b[V];
      LdgIO<T, V>::ld(dold + o, b);
#pragma unroll
      for (int k = 0; k < V; ++k) d[k] = fma(beta, b[k], d[k]);
    }
  };
  auto d1 = [&](long long o) -> T {
    if constexpr (fixed && IsF64<T>::value) return widen(__ldg(srcf + o));
    if (CHEB) return __ldg(src + o) * scale;
    return form ? fma(beta, __ldg(dold + o), __ldg(src + o)) : __ldg(src + o);
  };

  T dm[V], dc[V], dp[V];
  if (z0 < z1) {
    dvec(zoff(z0 - 1), dm);
    dvec(zoff(z0), dc);
  }
  T sum[V];
#pragma unroll
  for (int k = 0; k < V; ++k) sum[k] = 0;
  float sumf = 0.f;  // FP64 fixed-point sweep: <rt, rt> in FP32
  for (int z = z0; z < z1; ++z) {
    const long long oc = zoff(z), op = zoff(z + 1);
    T du[V], dd[V], bx[V], by[V], byd[V], bz[V], bzp[V], bd[V];
    dvec(op, dp);
    dvec(oc + dym, du);
    dvec(oc + dyp, dd);
    CoefIO<BT, T, V>::ldg(sx + oc, bx);
    CoefIO<BT, T, V>::ldg(sy + oc, by);
    CoefIO<BT, T, V>::ldg(sy + oc + dyp, byd);
    CoefIO<BT, T, V>::ldg(sz + oc, bz);
    CoefIO<BT, T, V>::ldg(sz + op, bzp);
    if (kDiag) CoefIO<BT, T, V>::ldg(sd + oc, bd);
    T qo[V], dol[V];  // QREC: q_old and d_old of the own cells
    if (QREC && use_old) {
      VecIO<T, V>::ld(q + oc, qo);  // q is rewritten below by this thread only
      LdgIO<T, V>::ld(dold + oc, dol);
    }
    T ro[V], xo[V];  // fixed point: rt and x of the own cells (rewritten by this thread only)
    if (fixed) {
      VecIO<T, V>::ld(rw + oc, ro);
      if (first_inner) {
#pragma unroll
        for (int k = 0; k < V; ++k) xo[k] = 0;
      } else {
        VecIO<T, V>::ld(xv + oc, xo);
      }
    }
    const T bxr = (T)ldg1(sx + oc + dxr);
    // x neighbours of the first and last cell: adjacent lanes, or a load at row ends / warp ends
    T left = __shfl_up_sync(0xffffffffu, dc[V - 1], 1);
    T right = __shfl_down_sync(0xffffffffu, dc[0], 1);
    if (lane == 0 || row_start) left = d1(oc + dxl);
    if (lane == 31 || row_end) right = d1(oc + dxr);
    T qv[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const T l = k == 0 ? left : dc[k - 1];
      const T r = k == V - 1 ? right : dc[k + 1];
      const T br = k == V - 1 ? bxr : bx[k + 1];
      T a = dc[k];
      if (kDiag) a = fma(bd[k], dc[k], a);
      a = fma(-bx[k], l, a);
      a = fma(-br, r, a);
      a = fma(-by[k], du[k], a);
      a = fma(-byd[k], dd[k], a);
      a = fma(-bz[k], dm[k], a);
      a = fma(-bzp[k], dp[k], a);
      qv[k] = a;
      if (!CHEB && !QREC && !fixed) sum[k] = fma(dc[k], a, sum[k]);
    }
    if (fixed) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        ro[k] -= qv[k];
        xo[k] += dc[k];
        if constexpr (IsF64<T>::value) {  // <rt, rt> only steers the inner stop: FP32 suffices,
          const float rf = narrow(ro[k]);   // and keeps the FP64 pipe to the update itself
          sumf = fmaf(rf, rf, sumf);
        } else {
          sum[k] = fma(ro[k], ro[k], sum[k]);
        }
      }
    }
    T dn[V];
    if (QREC && !fixed) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        dn[k] = use_old ? fma(beta, dol[k], dc[k]) : dc[k];
        qv[k] = use_old ? fma(beta, qo[k], qv[k]) : qv[k];
        if (!fixed) sum[k] = fma(dn[k], qv[k], sum[k]);
      }
    }
    if (CHEB) {
      T r[V], dprev[V], zn[V], dn[V];
      LdgIO<T, V>::ld(rt + oc, r);
      if (cj == 1) {
#pragma unroll
        for (int k = 0; k < V; ++k) dprev[k] = dc[k];  // d_0 = z_1
      } else {
        LdgIO<T, V>::ld(dch + oc, dprev);
      }
#pragma unroll
      for (int k = 0; k < V; ++k) {
        dn[k] = fma(c1, dprev[k], c2 * (r[k] - qv[k]));
        zn[k] = dc[k] + dn[k];
        if (last) sum[k] = fma(r[k], zn[k], sum[k]);
      }
      if (active) {
        VecIO<T, V>::st(zout + oc, zn);
        if (!last) VecIO<T, V>::st(dch + oc, dn);
      }
    } else if (active && fixed) {
      VecIO<T, V>::st(rw + oc, ro);
      VecIO<T, V>::st(xv + oc, xo);
    } else if (active) {
      if (QREC)
        VecIO<T, V>::st(dnew + oc, dn);
      else
        VecIO<T, V>::st(dnew + oc, dc);
      VecIO<T, V>::st(q + oc, qv);
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      dm[k] = dc[k];
      dc[k] = dp[k];
    }
  }
  if (!active) {
#pragma unroll
    for (int k = 0; k < V; ++k) sum[k] = 0;
    sumf = 0.f;
  }
  T tot = 0;
#pragma unroll
  for (int k = 0; k < V; ++k) tot += sum[k];
  if (fixed && IsF64<T>::value) tot = (T)sumf;
  part = tot;
}

// FP64 residual sweep in the same direct form (same unit and thread geometry as the stencil
// sweep: a thread owns VR = 16 / sizeof(T) cells of one row): p of planes z-1, z, z+1 in
// registers, rows above and below loaded per plane.  r = (f - <f>) - A p with the FP64 face
// coefficients; rt = D^-1/2 r stored in the inner type; sums of r^2, rt^2, p and, on the first
// call, (f - <f>)^2.  The sweep is bound by the FP64 pipe, so the residual is formed in the
// diagonal form r = (f - <f>) + D p_c - sum of b_face p_neighbour (D stored per cell): one FMA
// per term, 8 FP64 operations per cell against 13 for the face-difference form; in the mixed
// precisions the scaling rt = D^-1/2 r is an FP32 product; the norms are summed in FP32.
template <class T, bool FIRST, bool F0 = false>
__device__ __forceinline__ void res64_march(const InstDesc& I, const InstState* st, int unit,
                                            double (&acc)[kSlots]) {
  constexpr int VR = VecW<T>::V;  // cells per thread (4 for FP32 inner, 2 for FP64)
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int tpr = nx / VR;
  const int tile = unit % I.uy, chunk = unit / I.uy;
  const int row = threadIdx.x / tpr;
  const int x0 = (threadIdx.x - row * tpr) * VR;
  const int yr = tile * I.ty + row;
  const bool active = row < I.ty && yr < ny;
  const int y = active ? yr : ny - 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int z0 = (int)((long long)chunk * nz / I.zc), z1 = (int)((long long)(chunk + 1) * nz / I.zc);
  const int lane = threadIdx.x & 31;
  const bool row_start = x0 == 0, row_end = x0 + VR == nx;
  const int xl = row_start ? nx - 1 : x0 - 1, xr = row_end ? 0 : x0 + VR;
  const double mu = st->mu_f;
  const double* p = I.p;
  T* rt = static_cast<T*>(I.r);
  auto at = [&](int z, int yy) -> long long {
    const int zz = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    return ((long long)zz * ny + yy) * nx;
  };
  auto ldv = [&](const double* a, long long o, double (&v)[VR]) {
#pragma unroll
    for (int k = 0; k < VR; k += 2) {
      const double2 t = *reinterpret_cast<const double2*>(a + o + k);
      v[k] = t.x;
      v[k + 1] = t.y;
    }
  };
  double pm[VR], pc[VR], pp[VR];
  if (z0 < z1) {
    ldv(p, at(z0 - 1, y) + x0, pm);
    ldv(p, at(z0, y) + x0, pc);
  }
  double a2 = 0, a3 = 0;
  float a0 = 0.f, a1 = 0.f;  // norms steer the refinement only: summed in FP32 (cells narrowed
                             // by integer repacking), the FP64 pipe kept for the residual itself
  for (int z = z0; z < z1; ++z) {
    const long long oc = at(z, y), op = at(z + 1, y), oyp = at(z, yp), oym = at(z, ym);
    ldv(p, op + x0, pp);
    const double bxr = I.bx[oc + xr];
    double left = __shfl_up_sync(0xffffffffu, pc[VR - 1], 1);
    double right = __shfl_down_sync(0xffffffffu, pc[0], 1);
    if (lane == 0 || row_start) left = p[oc + xl];
    if (lane == 31 || row_end) right = p[oc + xr];
    // two cells at a time keeps the live registers down
#pragma unroll
    for (int h = 0; h < VR; h += 2) {
      const long long o = oc + x0 + h;
      const double2 pu = *reinterpret_cast<const double2*>(p + oym + x0 + h);
      const double2 pd = *reinterpret_cast<const double2*>(p + oyp + x0 + h);
      const double2 bx = *reinterpret_cast<const double2*>(I.bx + o);
      const double2 by = *reinterpret_cast<const double2*>(I.by + o);
      const double2 byd = *reinterpret_cast<const double2*>(I.by + oyp + x0 + h);
      const double2 bz = *reinterpret_cast<const double2*>(I.bz + o);
      const double2 bzp = *reinterpret_cast<const double2*>(I.bz + op + x0 + h);
      const double2 dg = *reinterpret_cast<const double2*>(I.dg + o);
      // F0: f - <f> as the first residual stored it (one FP64 operation fewer per cell)
      const double2 f = *reinterpret_cast<const double2*>((F0 ? I.f0 : I.rhs) + o);
      const double2 si = *reinterpret_cast<const double2*>(I.sinv + o);
      const double l0 = h == 0 ? left : pc[h - 1];
      const double r1 = h + 2 == VR ? right : pc[h + 2];
      const double br1 = h + 2 == VR ? bxr : I.bx[o + 2];
      const double c0 = pc[h], c1 = pc[h + 1];
      // r = (f - <f>) - A p with (A p)_c = sum of b_face p_neighbour - D_c p_c: the diagonal
      // term first, then one FMA per face (8 FP64 operations per cell; rounding error of order
      // eps D |p|, below 1e-12 of ||f - <f>|| on the grids here)
      double res0 = fma(dg.x, c0, F0 ? f.x : f.x - mu), res1 = fma(dg.y, c1, F0 ? f.y : f.y - mu);
      res0 = fma(-bx.x, l0, res0);
      res0 = fma(-bx.y, c1, res0);
      res1 = fma(-bx.y, c0, res1);
      res1 = fma(-br1, r1, res1);
      res0 = fma(-by.x, pu.x, res0);
      res1 = fma(-by.y, pu.y, res1);
      res0 = fma(-byd.x, pd.x, res0);
      res1 = fma(-byd.y, pd.y, res1);
      res0 = fma(-bz.x, pm[h], res0);
      res1 = fma(-bz.y, pm[h + 1], res1);
      res0 = fma(-bzp.x, pp[h], res0);
      res1 = fma(-bzp.y, pp[h + 1], res1);
      T t0, t1;
      float r0f = narrow(res0), r1f = narrow(res1), t0f, t1f;
      if constexpr (IsF64<T>::value) {
        t0 = si.x * res0;
        t1 = si.y * res1;
        t0f = narrow(t0);
        t1f = narrow(t1);
      } else {  // the inner residual in FP32: D^-1/2 r from the FP32 factors (the inner solve's
                // own rounding), no FP64 multiply
        t0 = t0f = narrow(si.x) * r0f;
        t1 = t1f = narrow(si.y) * r1f;
      }
      if (active) {
        rt[o] = t0;
        rt[o + 1] = t1;
        a0 = fmaf(r0f, r0f, fmaf(r1f, r1f, a0));
        a1 = fmaf(t0f, t0f, fmaf(t1f, t1f, a1));
        if (FIRST) {
          const double f0 = f.x - mu, f1 = f.y - mu;
          a2 += c0 + c1;
          a3 = fma(f0, f0, fma(f1, f1, a3));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      pm[k] = pc[k];
      pc[k] = pp[k];
    }
  }
  acc[0] = (double)a0;
  acc[1] = (double)a1;
  acc[2] = a2;
  acc[3] = a3;
}

// The first residual of a solve started from p = 0 is r = f - <f>: no stencil, no p reads.
template <class T>
__device__ void res64_zero_p(const InstDesc& I, const InstState* st, int unit,
                             double (&acc)[kSlots]) {
  constexpr int VR = VecW<T>::V;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int tpr = nx / VR;
  const int tile = unit % I.uy, chunk = unit / I.uy;
  const int row = threadIdx.x / tpr;
  const int x0 = (threadIdx.x - row * tpr) * VR;
  const int yr = tile * I.ty + row;
  const int z0 = (int)((long long)chunk * nz / I.zc), z1 = (int)((long long)(chunk + 1) * nz / I.zc);
  const double mu = st->mu_f;
  T* rt = static_cast<T*>(I.r);
  double a0 = 0;
  T a1 = 0;
  if (row < I.ty && yr < ny) {
    for (int z = z0; z < z1; ++z) {
      const long long o = ((long long)z * ny + yr) * nx + x0;
#pragma unroll
      for (int h = 0; h < VR; h += 2) {
        const double2 f = *reinterpret_cast<const double2*>(I.rhs + o + h);
        const double2 si = *reinterpret_cast<const double2*>(I.sinv + o + h);
        const double f0 = f.x - mu, f1 = f.y - mu;
        if (I.f0) *reinterpret_cast<double2*>(I.f0 + o + h) = make_double2(f0, f1);
        if constexpr (IsF64<T>::value) {
          const T t0 = si.x * f0, t1 = si.y * f1;
          rt[o + h] = t0;
          rt[o + h + 1] = t1;
          a0 = fma(f0, f0, fma(f1, f1, a0));
          a1 = fma(t0, t0, fma(t1, t1, a1));
        } else {  // as the full residual of the mixed precisions: the FP32 product of the narrowed
                  // factors; ||f - <f>||^2, the denominator of every relative residual of the
                  // solve, stays an FP64 sum (any magnitude of f)
          const float t0 = narrow(si.x) * narrow(f0), t1 = narrow(si.y) * narrow(f1);
          rt[o + h] = t0;
          rt[o + h + 1] = t1;
          a0 = fma(f0, f0, fma(f1, f1, a0));
          a1 = fmaf(t0, t0, fmaf(t1, t1, a1));
        }
      }
    }
  }
  acc[0] = a0;          // ||r||^2
  acc[1] = (double)a1;  // ||rt||^2
  acc[2] = 0.0;         // sum of p
  acc[3] = a0;          // ||f - <f>||^2 (this is the first residual)
}

template <class T>
__device__ void sweep_res64_direct(const InstDesc& I, const InstState* st, int unit,
                                   double (&acc)[kSlots]) {
  if (st->first_res != 0 && !st->use_guess)
    res64_zero_p<T>(I, st, unit, acc);
  else if (st->first_res != 0)
    res64_march<T, true>(I, st, unit, acc);
  else if (I.f0 && !st->use_guess)  // f - <f> stored by the first residual
    res64_march<T, false, true>(I, st, unit, acc);
  else
    res64_march<T, false>(I, st, unit, acc);
}

// ---- the FP64 residual sweep (a few times per solve): z march through a three-plane ring ---------

// zero: the solve starts from p = 0 and p has not been written yet (it is not read)
__device__ __forceinline__ void fill_p(const InstDesc& I, const Seg& sg, double* ring, int stride,
                                       int slot, int zg, bool zero) {
  const int nx = I.nx;
  const int cells = (sg.ty + 2) * nx;
  const long long pz = (long long)zg * nx * I.ny;
  double* dst = ring + slot * stride;
  for (int m = threadIdx.x; m < cells; m += blockDim.x) {
    const int ry = m / nx, x = m - ry * nx;
    dst[m] = zero ? 0.0 : I.p[pz + (long long)ring_gy(ry, sg.y0, I.ny) * nx + x];
  }
}

// r = (f - <f>) - A p; rt = D^-1/2 r in the inner type; sums of r^2, rt^2, p and, on the first
// call, (f - <f>)^2
template <class T>
__device__ void sweep_res64(const InstDesc& I, const InstState* st, int unit,
                            double (&acc)[kSlots], double* ring) {
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int stride = (I.ty + 2) * nx;
  const long long plane = (long long)nx * ny;
  const double mu = st->mu_f;
  const bool first = st->first_res != 0;
  const bool zero = st->p_set == 0;  // from p = 0, before the first correction
  T* rt = static_cast<T*>(I.r);
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for_each_segment(I, unit, [&](const Seg& sg) {
    int zm = sg.z0 - 1;
    if (zm < 0) zm += nz;
    __syncthreads();  // ring reuse across segments
    fill_p(I, sg, ring, stride, 0, zm, zero);
    fill_p(I, sg, ring, stride, 1, sg.z0, zero);
    const int own = sg.ty * nx;
    for (int k = 0; k < sg.nzs; ++k) {
      const int z = sg.z0 + k;
      const int zp = z + 1 == nz ? 0 : z + 1;
      const int sm = k % 3, sc = (k + 1) % 3, sp = (k + 2) % 3;
      fill_p(I, sg, ring, stride, sp, zp, zero);
      __syncthreads();
      const double* Rm = ring + sm * stride;
      const double* Rc = ring + sc * stride;
      const double* Rp = ring + sp * stride;
      for (int m = threadIdx.x; m < own; m += blockDim.x) {
        const int ry = m / nx + 1, x = m - (ry - 1) * nx;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const int gy = sg.y0 + ry - 1;
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
  });
  acc[0] = a0;
  acc[1] = a1;
  acc[2] = a2;
  acc[3] = a3;
}

// ---- the step kernels ----------------------------------------------------------------------------
// One sweep per launch for every instance of the batch whose phase is of the kernel's kind: the
// stencil kind (RES64, STENCIL: shared-memory z march, stencil units) or the flat kind (MEANF,
// UPDATE, CORRECT, FINAL: streaming, flat units).  The host alternates the two kinds; a launch
// whose instances are all in the other kind's phase exits at once.

// One stencil-kind unit of instance I: WHICH = 0 handles the RES64 and STENCIL phases, 1 only
// STENCIL, 2 only RES64; a no-op for other phases.
// KIND (direct form): 0 = CG sweeps only (the Chebyshev sweep compiled out, so the kernel keeps
// the register budget of the plain stencil sweep), 1 = CG and Chebyshev sweeps, 2 = the
// fixed-point iteration's sweep only.  The persistent batch kernel uses 1.
template <class T, class BT, int MODE, int WHICH = 0, int KIND = 1>
__device__ __forceinline__ void stencil_kind_unit(const InstDesc& I, int unit,
                                                  unsigned char* smem_raw) {
  InstState* st = I.st;
  const int phase = __ldcg(&st->phase);  // one load decides whether this unit has work
  if (phase != PH_RES64 && phase != PH_STENCIL && phase != PH_CHEB) return;
  if ((WHICH == 1 && phase == PH_RES64) || (WHICH == 2 && phase != PH_RES64)) return;
  if ((MODE != 0 || KIND != 1) && phase == PH_CHEB) return;  // direct form, KIND 1 only
  const InstState sn = snapshot(st);
  if (WHICH != 1 && phase == PH_RES64) {
    double acc[kSlots] = {0.0, 0.0, 0.0, 0.0};
    if (MODE == 0)
      sweep_res64_direct<T>(I, &sn, unit, acc);
    else
      sweep_res64<T>(I, &sn, unit, acc, reinterpret_cast<double*>(smem_raw));
    store_partials<kSlots, double>(acc, I.part, I.nunits, unit);
  } else if (WHICH != 2) {
    T part[1] = {0};
    if constexpr (MODE != 0) {
      sweep_stencil<T, BT>(I, st, unit, part[0], smem_raw);
    } else if constexpr (KIND == 2) {
      sweep_stencil_direct<T, BT, false, 2>(I, &sn, unit, part[0]);
    } else {
      if (KIND == 1 && phase == PH_CHEB)
        sweep_stencil_direct<T, BT, KIND == 1, 0>(I, &sn, unit, part[0]);
      else if (I.pc == PC_FIXED)  // the persistent kernel runs every kind of instance
        sweep_stencil_direct<T, BT, false, 2>(I, &sn, unit, part[0]);
      else if (sn.inner_iters > 0)
        sweep_stencil_direct<T, BT, false, 1>(I, &sn, unit, part[0]);
      else
        sweep_stencil_direct<T, BT, false, 0>(I, &sn, unit, part[0]);
    }
    store_partials<1, T>(part, I.part, I.nunits, unit);
  }
  finish_sweep(I, st, phase, I.nunits);
}

// One flat-kind unit (MEANF, UPDATE, CORRECT or FINAL phase) of instance I.
template <class T>
__device__ __forceinline__ void flat_kind_unit(const InstDesc& I, int unit) {
  InstState* st = I.st;
  const int phase = __ldcg(&st->phase);
  if (phase != PH_MEANF && phase != PH_UPDATE && phase != PH_CORRECT && phase != PH_FINAL) return;
  const InstState sn = snapshot(st);
  const long long c0 = flat_begin(I, unit), c1 = flat_begin(I, unit + 1);
  switch (phase) {
    case PH_MEANF: {
      double sum[1] = {0.0};
      sweep_meanf(I, c0, c1, sum[0]);
      store_partials<1, double>(sum, I.part, I.nunits_f, unit);
      break;
    }
    case PH_UPDATE: {
      T part[1] = {0};
      sweep_update<T>(I, &sn, c0, c1, part[0]);
      store_partials<1, T>(part, I.part, I.nunits_f, unit);
      break;
    }
    case PH_CORRECT: {
      double ps[1] = {0.0};
      sweep_correct<T>(I, c0, c1, sn.p_set == 0, ps[0]);
      store_partials<1, double>(ps, I.part, I.nunits_f, unit);
      break;
    }
    default: sweep_final(I, &sn, c0, c1); break;
  }
  finish_sweep(I, st, phase, I.nunits_f);
}

// Direct register march, STENCIL phase only: at most 256 threads, three units per SM (24 warps
// keep enough loads in flight).
#ifndef VDP_DIRECT_MIN_BLOCKS
#define VDP_DIRECT_MIN_BLOCKS 2
#endif
// Units per SM the register budget is sized for: three (80 registers, no spills) for every kind;
// measured at 256^3 against two units with the unconstrained allocation: FP64 CG sweep 315 ->
// 307 us, FP64 fused fixed-point sweep 299 -> 284 us.
template <class T, int KIND> struct DirectOcc { static constexpr int kMinBlocks = VDP_DIRECT_MIN_BLOCKS + 1; };

template <class T, class BT, int KIND>
__global__ void __launch_bounds__(kDirectThreads, DirectOcc<T, KIND>::kMinBlocks) k_stencil_direct(
    const InstDesc* __restrict__ insts, const UnitRef* __restrict__ units) {
  const UnitRef ur = units[blockIdx.x];
  stencil_kind_unit<T, BT, 0, 1, KIND>(insts[ur.inst], ur.unit, nullptr);
}

// Direct register march, RES64 phase only (a few launches per solve do work; the kernel has its
// own register allocation so that the FP64 residual does not limit the stencil's occupancy).
// Units per SM: three for the FP64 inner type (80 registers, no spills), two for FP32 (whose
// variant would spill at three).
template <class T> struct Res64Occ { static constexpr int kMinBlocks = IsF64<T>::value ? 3 : 2; };

template <class T>
__global__ void __launch_bounds__(kDirectThreads, Res64Occ<T>::kMinBlocks) k_res64_direct(
    const InstDesc* __restrict__ insts, const UnitRef* __restrict__ units) {
  const UnitRef ur = units[blockIdx.x];
  stencil_kind_unit<T, T, 0, 2>(insts[ur.inst], ur.unit, nullptr);
}

// TMA-staged pipeline
template <class T, class BT>
__global__ void __launch_bounds__(kMaxThreads) k_stencil_tma(const InstDesc* __restrict__ insts,
                                                             const UnitRef* __restrict__ units) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const UnitRef ur = units[blockIdx.x];
  stencil_kind_unit<T, BT, 1>(insts[ur.inst], ur.unit, smem_raw);
}

template <class T>
__global__ void __launch_bounds__(kFlatThreads, 4) k_flat(const InstDesc* __restrict__ insts,
                                                          const UnitRef* __restrict__ units) {
  const UnitRef ur = units[blockIdx.x];
  flat_kind_unit<T>(insts[ur.inst], ur.unit);
}

// Grid-wide barrier of the persistent kernel (all CTAs co-resident: cooperative launch).  Bounded:
// after the batch's wait limit (2 s by default) it gives up, sets the fault word and returns
// false, so a lost arrival ends the launch with an error status instead of a hang.
__device__ bool grid_sync(BatchCtl* ctl) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &ctl->gen;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&ctl->count, 1u) + 1u;
    const unsigned long long limit = ctl->limit_ns;
    ok = 1;
    if (arrived == gridDim.x + ctl->extra) {
      ctl->count = 0u;
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*vgen == gen) {
        if (global_ns() - t0 > limit) {
          atomicExch(&ctl->fault, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// The batch engine's persistent kernel: `pairs` rounds of (stencil-kind sweep of every
// instance, grid barrier, flat-kind sweep of every instance, grid barrier), units distributed
// over the resident CTAs; stops early once every instance is done.
template <class T, class BT>
__global__ void __launch_bounds__(kDirectThreads, VDP_DIRECT_MIN_BLOCKS)
    k_persistent(const InstDesc* __restrict__ insts, const UnitRef* __restrict__ sunits, int ns,
                 const UnitRef* __restrict__ funits, int nf, int pairs, BatchCtl* ctl) {
  for (int it = 0; it < pairs; ++it) {
    // uniform: `remaining` only changes in flat sweeps, and every CTA reads it after a barrier
    if (*(volatile int*)&ctl->remaining <= 0) break;
    for (int u = blockIdx.x; u < ns; u += gridDim.x) {
      const UnitRef ur = sunits[u];
      stencil_kind_unit<T, BT, 0>(insts[ur.inst], ur.unit, nullptr);
    }
    if (!grid_sync(ctl)) return;
    for (int u = blockIdx.x; u < nf; u += gridDim.x) {
      const UnitRef ur = funits[u];
      flat_kind_unit<T>(insts[ur.inst], ur.unit);
    }
    if (!grid_sync(ctl)) return;
  }
}

// Copies the state of n instances into a contiguous array (one D2H copy for the host).
__global__ void k_gather_states(const InstDesc* __restrict__ insts, int n, InstState* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = *insts[i].st;  // a separate launch: the solver kernels have finished
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
  s.p_set = use_guess ? 1 : 0;
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
    const double v = rho[c];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, 1);
  }
}

// b_d[c] = 2 / (rho[c - e_d] + rho[c]) / h_d^2 on the low d-face of every cell
// duct: the face at the x ends (slot x = 0, shared by x = 0 and x = Lx) carries no flux
__global__ void k_faces(const double* __restrict__ rho, int nx, int ny, int nz, double ihx2,
                        double ihy2, double ihz2, int duct, double* bx, double* by, double* bz) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx);
    const int y = (int)((c / nx) % ny);
    const int z = (int)(c / plane);
    const long long cxm = c - x + (x == 0 ? nx - 1 : x - 1);
    const long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    const long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    const double rc = rho[c];
    bx[c] = (duct && x == 0) ? 0.0 : 2.0 / (rho[cxm] + rc) * ihx2;
    by[c] = 2.0 / (rho[cym] + rc) * ihy2;
    bz[c] = 2.0 / (rho[czm] + rc) * ihz2;
  }
}

// sinv = D^-1/2 with D = sum of the six face coefficients of the cell
__global__ void k_diag(const double* __restrict__ bx, const double* __restrict__ by,
                       const double* __restrict__ bz, int nx, int ny, int nz, double* sinv,
                       double* dg) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx);
    const int y = (int)((c / nx) % ny);
    const int z = (int)(c / plane);
    const long long cxp = c - x + (x == nx - 1 ? 0 : x + 1);
    const long long cyp = c + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx;
    const long long czp = c + (long long)((z == nz - 1 ? 0 : z + 1) - z) * plane;
    const double D = bx[c] + bx[cxp] + by[c] + by[cyp] + bz[c] + bz[czp];
    sinv[c] = 1.0 / sqrt(D);
    dg[c] = D;
  }
}

// Rounded to nearest: the rounding errors of the stored off-diagonals have no common sign, so
// they do not add up to a spurious diagonal shift that would swamp the operator's smallest
// eigenvalues (a directed rounding would, at BF16 precision).
template <class BT> __device__ __forceinline__ BT to_coef(double v);
template <> __device__ __forceinline__ double to_coef<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_coef<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_coef<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
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
    const int x = (int)(c % nx);
    const int y = (int)((c / nx) % ny);
    const int z = (int)(c / plane);
    const long long cxm = c - x + (x == 0 ? nx - 1 : x - 1);
    const long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    const long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    const double s = sinv[c];
    sx[c] = to_coef<BT>(bx[c] * sinv[cxm] * s);
    sy[c] = to_coef<BT>(by[c] * sinv[cym] * s);
    sz[c] = to_coef<BT>(bz[c] * sinv[czm] * s);
  }
}

// BF16 coefficients: the rounded off-diagonals no longer sum (with the weights sqrt(D)) to the
// unit diagonal, and at BF16 precision that inconsistency is large enough to create spurious
// near-zero or negative eigenvalues.  The correction dg = sum_faces bt' s_nb / s_c - 1 (s =
// sqrt(D), bt' the stored BF16 values) restores sqrt(D) as an exact null vector of the stored
// inner operator  (1 + dg) I - offdiag(bt'), which is then congruent to a graph Laplacian with
// non-negative weights, i.e. symmetric positive semi-definite.
__global__ void k_diag_correction(const __nv_bfloat16* __restrict__ sx,
                                  const __nv_bfloat16* __restrict__ sy,
                                  const __nv_bfloat16* __restrict__ sz,
                                  const double* __restrict__ sinv, int nx, int ny, int nz,
                                  __nv_bfloat16* dg) {
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx);
    const int y = (int)((c / nx) % ny);
    const int z = (int)(c / plane);
    const long long cxm = c - x + (x == 0 ? nx - 1 : x - 1), cxp = c - x + (x == nx - 1 ? 0 : x + 1);
    const long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    const long long cyp = c + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx;
    const long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    const long long czp = c + (long long)((z == nz - 1 ? 0 : z + 1) - z) * plane;
    // s_nb / s_c = sinv_c / sinv_nb
    const double sc = sinv[c];
    double g = (double)__bfloat162float(sx[c]) * sc / sinv[cxm] +
               (double)__bfloat162float(sx[cxp]) * sc / sinv[cxp] +
               (double)__bfloat162float(sy[c]) * sc / sinv[cym] +
               (double)__bfloat162float(sy[cyp]) * sc / sinv[cyp] +
               (double)__bfloat162float(sz[c]) * sc / sinv[czm] +
               (double)__bfloat162float(sz[czp]) * sc / sinv[czp];
    dg[c] = __double2bfloat16(g - 1.0);
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
    const int x = (int)(c % nx);
    const int y = (int)((c / nx) % ny);
    const int z = (int)(c / plane);
    const long long cxm = c - x + (x == 0 ? nx - 1 : x - 1), cxp = c - x + (x == nx - 1 ? 0 : x + 1);
    const long long cym = c + (long long)((y == 0 ? ny - 1 : y - 1) - y) * nx;
    const long long cyp = c + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx;
    const long long czm = c + (long long)((z == 0 ? nz - 1 : z - 1) - z) * plane;
    const long long czp = c + (long long)((z == nz - 1 ? 0 : z + 1) - z) * plane;
    const double pc = p[c];
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

cudaError_t launch_build_coefficients(const double* rho, int nx, int ny, int nz, double hx,
                                      double hy, double hz, int duct, double* bx, double* by,
                                      double* bz, double* sinv, double* dg, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  k_faces<<<grid_for(n), 256, 0, s>>>(rho, nx, ny, nz, 1.0 / (hx * hx), 1.0 / (hy * hy),
                                      1.0 / (hz * hz), duct, bx, by, bz);
  k_diag<<<grid_for(n), 256, 0, s>>>(bx, by, bz, nx, ny, nz, sinv, dg);
  return cudaGetLastError();
}

cudaError_t launch_scaled(int prec, const double* bx, const double* by, const double* bz,
                          const double* sinv, int nx, int ny, int nz, void* sx, void* sy, void* sz,
                          void* sd, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  if (prec == PREC_FP64)
    k_scaled<double><<<grid_for(n), 256, 0, s>>>(bx, by, bz, sinv, nx, ny, nz, (double*)sx,
                                                 (double*)sy, (double*)sz);
  else if (prec == PREC_MIXED)
    k_scaled<float><<<grid_for(n), 256, 0, s>>>(bx, by, bz, sinv, nx, ny, nz, (float*)sx,
                                                (float*)sy, (float*)sz);
  else {
    k_scaled<__nv_bfloat16><<<grid_for(n), 256, 0, s>>>(bx, by, bz, sinv, nx, ny, nz,
                                                        (__nv_bfloat16*)sx, (__nv_bfloat16*)sy,
                                                        (__nv_bfloat16*)sz);
    k_diag_correction<<<grid_for(n), 256, 0, s>>>((const __nv_bfloat16*)sx,
                                                  (const __nv_bfloat16*)sy,
                                                  (const __nv_bfloat16*)sz, sinv, nx, ny, nz,
                                                  (__nv_bfloat16*)sd);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(const double* bx, const double* by, const double* bz, const double* p,
                         int nx, int ny, int nz, double* out, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
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

template <int KIND>
static void* direct_fn(int prec) {
  if (prec == PREC_FP64) return (void*)k_stencil_direct<double, double, KIND>;
  if (prec == PREC_MIXED) return (void*)k_stencil_direct<float, float, KIND>;
  return (void*)k_stencil_direct<float, __nv_bfloat16, KIND>;
}

static void* stencil_fn(int prec, int mode, int kind) {
  if (mode == 0) return kind == 2 ? direct_fn<2>(prec) : kind == 1 ? direct_fn<1>(prec) : direct_fn<0>(prec);
  if (prec == PREC_FP64) return (void*)k_stencil_tma<double, double>;
  if (prec == PREC_MIXED) return (void*)k_stencil_tma<float, float>;
  return (void*)k_stencil_tma<float, __nv_bfloat16>;
}

cudaError_t prepare_step(int prec, int mode, size_t smem_bytes) {
  if (mode == 0) return cudaSuccess;  // the direct sweeps use no dynamic shared memory
  return cudaFuncSetAttribute(stencil_fn(prec, mode, 0),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_res64(int prec, const InstDesc* desc, const UnitRef* units, int nunits,
                         int threads, cudaStream_t s) {
  if (prec == PREC_FP64)
    k_res64_direct<double><<<nunits, threads, 0, s>>>(desc, units);
  else
    k_res64_direct<float><<<nunits, threads, 0, s>>>(desc, units);
  return cudaGetLastError();
}

cudaError_t launch_stencil(int prec, int mode, int kind, const InstDesc* desc,
                           const UnitRef* units, int nunits, int threads, size_t smem_bytes,
                           cudaStream_t s) {
  void* fn = stencil_fn(prec, mode, kind);
  void* args[] = {(void*)&desc, (void*)&units};
  return cudaLaunchKernel(fn, dim3(nunits), dim3(threads), args, smem_bytes, s);
}

static void* persistent_fn(int prec) {
  if (prec == PREC_FP64) return (void*)k_persistent<double, double>;
  if (prec == PREC_MIXED) return (void*)k_persistent<float, float>;
  return (void*)k_persistent<float, __nv_bfloat16>;
}

cudaError_t persistent_grid(int prec, int* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_fn(prec),
                                                                kDirectThreads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_persistent(int prec, const InstDesc* desc, const UnitRef* sunits, int ns,
                              const UnitRef* funits, int nf, int pairs, BatchCtl* ctl, int grid,
                              cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kDirectThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident: the grid barrier is safe
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&desc, (void*)&sunits, (void*)&ns, (void*)&funits, (void*)&nf,
                  (void*)&pairs, (void*)&ctl};
  return cudaLaunchKernelExC(&cfg, persistent_fn(prec), args);
}

// The body of a solve's device-side loop ends with this kernel: it keeps the loop going while
// the solve is unfinished and the round count is below its bound.
__global__ void k_continue(const InstState* st, cudaGraphConditionalHandle handle, unsigned* rounds,
                           unsigned max_rounds) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const unsigned r = *rounds + 1u;
    *rounds = r;
    const bool more = __ldcg(&st->phase) < PH_DONE && r < max_rounds;
    cudaGraphSetConditional(handle, more ? 1u : 0u);
  }
}

cudaError_t launch_continue(const InstState* st, cudaGraphConditionalHandle handle,
                            unsigned* rounds, unsigned max_rounds, cudaStream_t s) {
  k_continue<<<1, 32, 0, s>>>(st, handle, rounds, max_rounds);
  return cudaGetLastError();
}

cudaError_t launch_gather(const InstDesc* desc, int n, InstState* out, cudaStream_t s) {
  k_gather_states<<<(n + 127) / 128, 128, 0, s>>>(desc, n, out);
  return cudaGetLastError();
}

cudaError_t launch_flat(int prec, const InstDesc* desc, const UnitRef* units, int nunits,
                        cudaStream_t s) {
  if (prec == PREC_FP64)
    k_flat<double><<<nunits, kFlatThreads, 0, s>>>(desc, units);
  else
    k_flat<float><<<nunits, kFlatThreads, 0, s>>>(desc, units);
  return cudaGetLastError();
}

}  // namespace vdp
