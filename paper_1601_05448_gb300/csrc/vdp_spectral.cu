// vdp_spectral.cu -- the constant-coefficient spectral inverse (Sec. 3.4) on sm_103a, used as a
// preconditioner of the inner conjugate-gradient solve and exposed as vdp_inverse_laplacian.
//
// The paper solves the variable-density equation by repeated constant-coefficient Poisson
// solves done with FFTs.  Here the same operator, the inverse of the 7-point Laplacian L_h on
// the periodic grid (eigenvalues -sum_d 4 sin^2(pi k_d / n_d) / h_d^2, zero mode removed), is
// applied to the Jacobi-scaled inner residual as
//     z = W (-L_h)^-1 W rt,   W = D^1/2 (D: diagonal of the variable-coefficient operator),
// which is the constant-coefficient inverse in unscaled variables.  Between the smallest and the
// largest face value of 1/rho the variable operator is bounded by multiples of -L_h, so the
// preconditioned condition number is at most the density ratio, whatever the grid size.
//
// Five passes over a half spectrum S[kz][ky][kx] (kx = 0 .. nx/2, complex FP32, row pitch nxp):
//   X+  each row of nx reals is read as nx/2 complex pairs, weighted by W, transformed by a
//       complex FFT of length nx/2 and unpacked into the nx/2 + 1 bins of the real transform;
//   Y+  complex FFTs along y of tiles of 8 consecutive kx columns;
//   Z   FFT along z, division by the eigenvalue (and by nx ny nz), inverse FFT along z: the
//       whole z line is in the block, so the solve costs one pass;
//   Y-  inverse FFTs along y;
//   X-  the real inverse transform of each row, weighted by W, stored as z; in the solve this
//       pass also sums <rt, z> and, as the last unit to finish, moves the solve to its next
//       phase (the same fixed-order reduction as every other sweep).
// Every line FFT is a four-step factorisation n = M1 x M2 (both products of 2 and 3, at most
// 32): M2-point DFTs in registers, twiddles W_n^(j1 k2), an exchange through shared memory,
// M1-point DFTs in registers.  Global accesses are coalesced: rows are contiguous in the X
// passes and the Y/Z tiles read 8 consecutive complex values (64 bytes) per line element.
// One application moves about 49 bytes per cell for the FP32 inner solve; at 512^3 the X and Y
// passes run at 0.85-0.91 of the copy bandwidth and Z, which does two transforms per element,
// is bound by its instruction issue.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "vdp.h"
#include "vdp_device.cuh"
#include "vdp_internal.cuh"
#include "vdp_spectral.h"

namespace vdp {

// ---- complex arithmetic and small DFTs in registers ---------------------------------------------

// exp(-2 pi i k / 96): the roots of unity of every register DFT size used here (all divide 96).
__constant__ float2 c_w96[96];

// Complex sums, differences and real scalings as one paired FP32 instruction (add / sub / mul
// .rn.f32x2: both lanes rounded as the scalar operation would round them); the FFT butterflies
// are mostly these, and the Z pass is bound by its instruction issue.
#define VDP_F32X2(op)                                                                        \
  "{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n " op        \
  ".rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm(VDP_F32X2("add") : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm(VDP_F32X2("sub") : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 cscale(float2 a, float s) {
  float2 r;
  asm(VDP_F32X2("mul") : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(s), "f"(s));
  return r;
}
#undef VDP_F32X2
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// v * W_M^k with W = exp(-2 pi i / M) (INV: the conjugate root).  k and M are constants after
// unrolling, so the trivial roots cost nothing and the others are constant-bank operands.
template <bool INV>
__device__ __forceinline__ float2 rot(float2 v, int k, int M) {
  k %= M;
  if (k == 0) return v;
  if (2 * k == M) return make_float2(-v.x, -v.y);
  if (4 * k == M) return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  if (4 * k == 3 * M) return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  const float2 w = c_w96[(96 / M) * k];
  return cmul(v, INV ? cconj(w) : w);
}

// y[k] = sum_j x[O + S j] W_M^(j k), k < M: recursive decimation in time (radix 2, then 3).
template <int M, int O, int S, bool INV, int N>
__device__ __forceinline__ void dft(const float2 (&x)[N], float2 (&y)[M]) {
  static_assert(O + S * (M - 1) < N, "dft reads outside its input");
  if constexpr (M == 1) {
    y[0] = x[O];
  } else if constexpr (M % 2 == 0) {
    constexpr int H = M / 2;
    float2 e[H], o[H];
    dft<H, O, 2 * S, INV>(x, e);
    dft<H, O + S, 2 * S, INV>(x, o);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 t = rot<INV>(o[k], k, M);
      y[k] = cadd(e[k], t);
      y[k + H] = csub(e[k], t);
    }
  } else {
    static_assert(M % 3 == 0, "register DFT sizes are products of 2 and 3");
    constexpr int T = M / 3;
    constexpr float kS3 = 0.86602540378443864676f;  // sin(pi / 3)
    float2 a[T], b[T], c[T];
    dft<T, O, 3 * S, INV>(x, a);
    dft<T, O + S, 3 * S, INV>(x, b);
    dft<T, O + 2 * S, 3 * S, INV>(x, c);
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const float2 tb = rot<INV>(b[k], k, M), tc = rot<INV>(c[k], 2 * k, M);
      const float2 s = cadd(tb, tc), d = csub(tb, tc);
      const float2 m = make_float2(a[k].x - 0.5f * s.x, a[k].y - 0.5f * s.y);
      // forward: W_3 = -1/2 - i sin(pi/3); (tb - tc) times -i sin(pi/3) (+i for the inverse)
      const float2 j = INV ? make_float2(-kS3 * d.y, kS3 * d.x) : make_float2(kS3 * d.y, -kS3 * d.x);
      y[k] = cadd(a[k], s);
      y[k + T] = cadd(m, j);
      y[k + 2 * T] = csub(m, j);
    }
  }
}

// ---- table layout ---------------------------------------------------------------------------------

struct Tables {
  const float2* wm;  // W_m^k, m = nx / 2
  const float2* wr;  // W_nx^k, k = 0 .. m
  const float2* wy;  // W_ny^k
  const float2* wz;  // W_nz^k
  const float* lx;   // 4 sin^2(pi k / nx) / hx^2, k = 0 .. m
  const float* ly;
  const float* lz;
};

__device__ __forceinline__ Tables tables(const SpecArgs& a) {
  const int m = a.nx / 2;
  Tables t;
  t.wm = a.tw;
  t.wr = a.tw + m;
  t.wy = a.tw + 2 * m + 1;
  t.wz = a.tw + 2 * m + 1 + a.ny;
  t.lx = a.lam;
  t.ly = a.lam + m + 1;
  t.lz = a.lam + m + 1 + a.ny;
  return t;
}

// In the solve every pass first checks that the instance is in the spectral phase (one L2
// load); the stand-alone inverse passes st = nullptr and always runs.
__device__ __forceinline__ bool spec_active(const SpecArgs& a) {
  return a.st == nullptr || __ldcg(&a.st->phase) == PH_SPEC;
}

template <class T> struct Pair;
template <> struct Pair<float> {
  static __device__ __forceinline__ float2 ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
  static __device__ __forceinline__ void st(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
  static __device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
  }
};
template <> struct Pair<double> {
  static __device__ __forceinline__ float2 ld(const double* p) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    return make_float2(narrow(v.x), narrow(v.y));
  }
  static __device__ __forceinline__ void st(double* p, float2 v) {
    *reinterpret_cast<double2*>(p) = make_double2(widen(v.x), widen(v.y));
  }
  static __device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
  }
};

// Shared-memory row strides (in complex values) congruent to 8 modulo 16: the four rows (or
// line groups) a warp touches then fall on alternating halves of the 32 banks.
__host__ __device__ constexpr int pad_stride(int len) { return ((len + 7) / 16) * 16 + 8; }

// Shared memory of one row in the X passes: the four-step exchange, reused for the whole
// transformed row (X+ unpack).
template <int M1, int M2>
constexpr int x_row_stride() {
  return pad_stride(M2 * (M1 + 1)) > pad_stride(M1 * M2 + 1) ? pad_stride(M2 * (M1 + 1))
                                                              : pad_stride(M1 * M2 + 1);
}

// Rows per block of the X passes: at most 256 threads and about 40 KB of shared memory, and a
// multiple of 32 threads (the block reduction works on whole warps).
template <int M1, int M2>
constexpr int rows_per_block() {
  for (int ry = 256 / M1; ry > 1; --ry)
    if ((M1 * ry) % 32 == 0 && 8 * ry * x_row_stride<M1, M2>() <= 40960) return ry;
  return 32;  // not reached for the supported sizes
}

// Rows per block of X- (register bound: half the rows of X+, so that more blocks share an SM).
template <int M1, int M2>
constexpr int inv_rows_per_block() {
  for (int ry = 256 / M1; ry > 1; --ry)
    if ((M1 * ry) % 32 == 0 &&
        8 * ry * (pad_stride(M2 * (M1 + 1)) + pad_stride(M1 * M2 + 1)) <= 40960)
      return ry;
  return 32;  // not reached for the supported sizes
}

// The four-step exchange of one line through shared memory: step A's thread j1 writes its
// M2 outputs to [k2][j1], step B's thread k2 reads them back; rows of M1 + 1 values keep the
// step B reads (stride M1 + 1) free of bank conflicts.
template <int M1>
__device__ __forceinline__ int ex(int k2, int j1) { return k2 * (M1 + 1) + j1; }

// ---- X+ : real rows -> half spectrum -----------------------------------------------------------

// The X+ transform of RY rows (one per group of M1 threads: t = lane in the row, r = row in the
// group), row `row` of the grid in thread group r; `ra` is the row's shared buffer of SX values
// (the exchange, then the transformed row).  store(k, X) receives bin k of the row's half
// spectrum for k < nxp (zero beyond nx/2).  Every thread of the block calls it (barriers).
template <class T, int M1, int M2, bool MIRROR, class Store>
__device__ __forceinline__ void x_fwd_rows(const SpecArgs& a, const Tables& tb, float2* ra,
                                           long long row, bool live, int t, Store&& store) {
  constexpr int m = M1 * M2;
  float2* rb = ra;
  // step A: M2-point DFTs over j2 of z[t + M1 j2] = (x[2j], x[2j+1]) * W
  if (live) {
    const T* in = static_cast<const T*>(a.in) + row * a.nxd;
    const float* om = a.omega_in ? a.omega_in + row * a.nxd : nullptr;
    float2 v[M2], y[M2];
#pragma unroll
    for (int j2 = 0; j2 < M2; ++j2) {
      const int j = t + M1 * j2;
      // pair j of the transformed row; mirrored rows read their second half backwards:
      // cells (2j, 2j + 1) of the extension are cells (q + 1, q) of the row, q = 2 nxd - 2 - 2j
      const bool back = MIRROR && 2 * j >= a.nxd;
      const int q = back ? 2 * a.nxd - 2 - 2 * j : 2 * j;
      float2 z = Pair<T>::ld(in + q);
      if (om) {
        const float2 w = *reinterpret_cast<const float2*>(om + q);
        z = make_float2(z.x * w.x, z.y * w.y);
      }
      v[j2] = back ? make_float2(z.y, z.x) : z;
    }
    dft<M2, 0, 1, false>(v, y);
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2)
      ra[ex<M1>(k2, t)] = k2 == 0 || t == 0 ? y[k2] : cmul(y[k2], tb.wm[t * k2]);
  }
  __syncthreads();
  // step B: M1-point DFTs over j1 -> Z[k2 + M2 k1]; the exchange is read completely before the
  // transformed row overwrites it
  constexpr int R = (M2 + M1 - 1) / M1;
  float2 u[R][M1];
  if (live) {
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k2 = t + M1 * rr;
      if (k2 < M2) {
#pragma unroll
        for (int j1 = 0; j1 < M1; ++j1) u[rr][j1] = ra[ex<M1>(k2, j1)];
      }
    }
  }
  __syncthreads();
  if (live) {
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k2 = t + M1 * rr;
      if (k2 < M2) {
        float2 o[M1];
        dft<M1, 0, 1, false>(u[rr], o);
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) rb[k2 + M2 * k1] = o[k1];
      }
    }
  }
  __syncthreads();
  // unpack: X[k] = E[k] + W_nx^k O[k], E = (Z[k] + conj Z[m-k]) / 2, O = (Z[k] - conj Z[m-k]) / 2i
  if (live) {
    for (int k = t; k < a.nxp; k += M1) {
      float2 X = make_float2(0.f, 0.f);
      if (k <= m) {
        const float2 p = rb[k == m ? 0 : k], q = cconj(rb[k == 0 ? 0 : m - k]);
        const float2 e = cscale(cadd(p, q), 0.5f);
        const float2 d = csub(p, q);
        const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
        X = cadd(e, cmul(tb.wr[k], o));
      }
      store(k, X);
    }
  }
}

// The X tables W_m^k (k < m) and W_nx^k (k <= m) copied to the block's shared memory (every
// lookup of a row transform is then a shared-memory load); returns the tables with them.
template <int M1, int M2>
__device__ __forceinline__ Tables x_tables_shared(const SpecArgs& a, float2* st) {
  constexpr int m = M1 * M2;
  Tables tb = tables(a);
  for (int k = threadIdx.x; k < 2 * m + 1; k += blockDim.x) st[k] = k < m ? tb.wm[k] : tb.wr[k - m];
  __syncthreads();
  tb.wm = st;
  tb.wr = st + m;
  return tb;
}

// X+ of FP32 rows: one group of RY rows per block, tables read through L1.  The 512^3 mixed solve
// takes 33.6 ms with it against 34.4 ms with the persistent form below for FP32 rows too (whose
// loop needs 80 registers: one block per SM less for the loads in flight).
template <class T, int M1, int M2, bool MIRROR>
__global__ void __launch_bounds__(M1 * rows_per_block<M1, M2>(), 1024 / (M1 * rows_per_block<M1, M2>()))
    k_spec_x_fwd(SpecArgs a) {
  constexpr int RY = rows_per_block<M1, M2>();
  constexpr int SX = x_row_stride<M1, M2>();
  __shared__ float2 sx[RY * SX];  // per row: the exchange, then the transformed row
  if (!spec_active(a)) return;
  const Tables tb = tables(a);
  const int t = threadIdx.x % M1, r = threadIdx.x / M1;
  const long long row = (long long)a.z0 * a.ny + (long long)blockIdx.x * RY + r;
  const bool live = row < (long long)a.z1 * a.ny;
  float2* out = a.spec + row * a.nxp;
  x_fwd_rows<T, M1, M2, MIRROR>(a, tb, sx + r * SX, row, live, t,
                                 [&](int k, float2 X) { out[k] = X; });
}

// X+ of FP64 rows on a persistent grid: groups of RY rows (group = block, block + grid, ...) of
// the planes [z0, z1), tables in shared memory; at least 768 resident threads per SM (80
// registers a thread).  The 512^3 FP64 solve: 47.3 ms against 49.2 ms with the form above.
template <class T, int M1, int M2, bool MIRROR>
__global__ void __launch_bounds__(M1 * rows_per_block<M1, M2>(), 768 / (M1 * rows_per_block<M1, M2>()))
    k_spec_x_fwd_persistent(SpecArgs a) {
  constexpr int RY = rows_per_block<M1, M2>();
  constexpr int SX = x_row_stride<M1, M2>();
  __shared__ float2 sx[RY * SX];  // per row: the exchange, then the transformed row
  __shared__ float2 stab[2 * M1 * M2 + 1];
  if (!spec_active(a)) return;
  const Tables tb = x_tables_shared<M1, M2>(a, stab);
  const int t = threadIdx.x % M1, r = threadIdx.x / M1;
  const long long rows = (long long)(a.z1 - a.z0) * a.ny;
  for (long long g = blockIdx.x; g * RY < rows; g += gridDim.x) {
    const long long row = (long long)a.z0 * a.ny + g * RY + r;
    const bool live = g * RY + r < rows;
    float2* out = a.spec + row * a.nxp;
    x_fwd_rows<T, M1, M2, MIRROR>(a, tb, sx + r * SX, row, live, t,
                                   [&](int k, float2 X) { out[k] = X; });
    __syncthreads();  // the row buffers are reused by the next group
  }
}

// ---- X- : half spectrum -> real rows, z = W x ----------------------------------------------------

// The X- transform of one row per group of M1 threads: `src` is the row of the half spectrum
// (global or shared memory), `rb` the group's shared exchange buffer; z = W x is stored to row
// `row` of a.out.  Every thread of the block calls it (barrier).
template <class T, int M1, int M2, bool MIRROR>
__device__ __forceinline__ void x_inv_rows(const SpecArgs& a, const Tables& tb, float2* rb,
                                           const float2* src, long long row, bool live, int t) {
  constexpr int m = M1 * M2;
  // the output weights of this thread's cells are loaded first, so that their latency overlaps
  // the transforms (cells 2l, 2l + 1 with l = k2 + M2 k1, k2 = t, t + M1, ...)
  constexpr int R = (M2 + M1 - 1) / M1;
  float2 wv[R][M1];
  const float* om = a.omega_out ? a.omega_out + row * a.nxd : nullptr;
#pragma unroll
  for (int rr = 0; rr < R; ++rr)
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) {
      const int k2 = t + M1 * rr;
      const int l = k2 + M2 * k1;
      wv[rr][k1] = make_float2(1.f, 1.f);
      if (live && om && k2 < M2 && (!MIRROR || 2 * l < a.nxd))
        wv[rr][k1] = *reinterpret_cast<const float2*>(om + 2 * l);
    }
  // Z'[k] = (X[k] + conj X[m-k]) + i conj(W_nx^k) (X[k] - conj X[m-k]); inverse M2-point DFTs.
  // Both X[k] and X[m-k] are read straight from the spectrum: for a fixed j2 the lanes of a row
  // read consecutive values, ascending and descending.
  if (live) {
    float2 xa[M2], xb[M2];
#pragma unroll
    for (int j2 = 0; j2 < M2; ++j2) {
      const int k = t + M1 * j2;
      xa[j2] = src[k];
      xb[j2] = src[m - k];
    }
    float2 v[M2], y[M2];
#pragma unroll
    for (int j2 = 0; j2 < M2; ++j2) {
      const int k = t + M1 * j2;
      const float2 p = xa[j2], q = cconj(xb[j2]);
      const float2 e = cadd(p, q);
      const float2 o = cmulc(csub(p, q), tb.wr[k]);
      v[j2] = make_float2(e.x - o.y, e.y + o.x);
    }
    dft<M2, 0, 1, true>(v, y);
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2)
      rb[ex<M1>(k2, t)] = k2 == 0 || t == 0 ? y[k2] : cmulc(y[k2], tb.wm[t * k2]);
  }
  __syncthreads();
  if (live) {
    T* out = static_cast<T*>(a.out) + row * a.nxd;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k2 = t + M1 * rr;
      if (k2 >= M2) break;
      float2 u[M1], o[M1];
#pragma unroll
      for (int j1 = 0; j1 < M1; ++j1) u[j1] = rb[ex<M1>(k2, j1)];
      dft<M1, 0, 1, true>(u, o);
#pragma unroll
      for (int k1 = 0; k1 < M1; ++k1) {
        const int l = k2 + M2 * k1;  // cells 2l, 2l + 1 of the row
        if (MIRROR && 2 * l >= a.nxd) continue;  // the second half is the reflection
        const float2 z = make_float2(o[k1].x * wv[rr][k1].x, o[k1].y * wv[rr][k1].y);
        Pair<T>::st(out + 2 * l, z);
      }
    }
  }
}

// X- on a persistent grid: groups of RY rows (group = block, block + grid, ...), tables in
// shared memory.  The 512^3 mixed solve: 33.6 ms against 34.1 ms with one row group per block
// and the tables read through L1; and a launch in another phase of the solve exits after 3 us
// instead of 29 us.
template <class T, int M1, int M2, bool MIRROR>
__global__ void __launch_bounds__(M1 * inv_rows_per_block<M1, M2>())
    k_spec_x_inv_persistent(SpecArgs a) {
  constexpr int RY = inv_rows_per_block<M1, M2>();
  constexpr int SB = pad_stride(M2 * (M1 + 1));
  __shared__ float2 sb[RY * SB];
  __shared__ float2 stab[2 * M1 * M2 + 1];
  if (!spec_active(a)) return;
  const Tables tb = x_tables_shared<M1, M2>(a, stab);
  const int t = threadIdx.x % M1, r = threadIdx.x / M1;
  const long long rows = (long long)(a.z1 - a.z0) * a.ny;
  for (long long g = blockIdx.x; g * RY < rows; g += gridDim.x) {
    const long long row = (long long)a.z0 * a.ny + g * RY + r;
    const bool live = g * RY + r < rows;
    x_inv_rows<T, M1, M2, MIRROR>(a, tb, sb + r * SB, a.spec + row * a.nxp, row, live, t);
    __syncthreads();  // the exchange buffers are reused by the next group
  }
  if (a.st) {  // the solve: the last block of the application's X- launches completes the
               // preconditioner sweep, with <rt, z> from the partial sums the Z pass stored
    const InstDesc& I = *a.I;
    finish_sweep(I, I.st, PH_SPEC, a.xunits, a.zunits);
  }
}

// Whether X+ of FP32 rows also runs on a persistent grid (measured at 512^3, see the X+ forms:
// it does not; X+ of FP64 rows and X- always do).
constexpr bool kXFwdF32Persistent = false;

// ---- Y and Z: tiles of TX consecutive kx columns, whole lines -----------------------------------

constexpr int kTX = 8;  // columns per tile (64 bytes of each line element)

// shared-memory index of line element e (of a tile column c) when lines are grouped by g
// elements: groups of g * kTX values padded to a stride = 8 (mod 16)
template <int G>
__device__ __forceinline__ int tx(int group, int e, int c) {
  return group * pad_stride(G * kTX) + e * kTX + c;
}

// 16-byte asynchronous copy global -> shared (cached in L2 only), and its group wait: the copies
// hold no registers while in flight, so a block can fetch its next tile while it finishes this
// one.  wait_group is a hardware wait for this thread's own copies (no spin loop).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Tiles of the Y and Z passes: nz (or ny) line elements of kTX columns.  Element e = t + M1 j2 of
// column c is copied to slot (j2, t, c) of the tile buffer, the layout step A reads; step A
// writes the exchange to slots (k2, t, c) of the same buffer.
template <int M1, int M2>
constexpr int line_buffer() { return M2 * pad_stride(M1 * kTX); }  // complex values of one tile
// Y: at least 512 resident threads per SM (at most 128 registers a thread); lines of 512: four
// blocks of 128 threads.  Z: at least 640 (96 registers, a few bytes spilled): at 512^3 Z
// 352 -> 327 us with five blocks per SM, while Y at five (or six) blocks ran 191 -> 209 us.
template <int M1> struct LineOcc { static constexpr int kMinBlocks = (512 + M1 * kTX - 1) / (M1 * kTX); };
template <int M1> struct ZOcc { static constexpr int kMinBlocks = (640 + M1 * kTX - 1) / (M1 * kTX); };

// Copies of the tile of n = M1 x M2 line elements at g (element stride es) into the buffer sm:
// 4 pieces of 16 bytes per element, spread over the block's threads; one commit group.
template <int M1, int M2>
__device__ __forceinline__ void fetch_tile(float2* sm, const float2* g, long long es) {
  constexpr int S = pad_stride(M1 * kTX);
  for (int q = threadIdx.x; q < 4 * M1 * M2; q += M1 * kTX) {
    const int e = q >> 2, part = q & 3;
    cp_async16(sm + (e / M1) * S + (e % M1) * kTX + 2 * part, g + e * es + 2 * part);
  }
  cp_async_commit();
}

template <int M1, int M2>
constexpr size_t y_smem() {  // tile buffer, twiddles W_ny^k
  return sizeof(float2) * (size_t)(line_buffer<M1, M2>() + M1 * M2);
}

// Y pass (forward or inverse), in place.  Tiles are (column tile, kz); a persistent grid walks
// them (tile = block, block + grid, ...).  The twiddles W_ny^k are copied to shared memory once
// per block; a tile's copies go out as soon as the previous tile's exchange is read, so they
// overlap its step B and stores.  Step A: M2-point DFTs over j2 (thread (t, c)), twiddles, the
// exchange; step B: M1-point DFTs over j1 by owner k2, element k2 + M2 k1 stored.
template <int M1, int M2, bool INV>
__global__ void __launch_bounds__(M1 * kTX, LineOcc<M1>::kMinBlocks) k_spec_y(SpecArgs a) {
  constexpr int R = (M2 + M1 - 1) / M1;
  constexpr int n = M1 * M2;
  constexpr int S = pad_stride(M1 * kTX);
  extern __shared__ __align__(16) float2 ybuf[];
  float2* sm = ybuf;                          // the tile
  float2* wy = ybuf + line_buffer<M1, M2>();  // W_ny^k, k < ny
  if (!spec_active(a)) return;
  const Tables tb = tables(a);
  const int c = threadIdx.x % kTX, t = threadIdx.x / kTX;
  const int tiles = a.nxp / kTX;
  const int ntile = tiles * (a.z1 - a.z0);
  const long long es = a.nxp;  // element stride along y
  auto base = [&](int tile) {
    return a.spec + (long long)(a.z0 + tile / tiles) * a.ny * a.nxp + (tile % tiles) * kTX;
  };
  int tile = blockIdx.x;
  if (tile < ntile) fetch_tile<M1, M2>(sm, base(tile), es);
  for (int k = threadIdx.x; k < n; k += M1 * kTX) wy[k] = tb.wy[k];
  for (; tile < ntile; tile += gridDim.x) {
    cp_async_wait_all();  // this thread's copies of the tile have landed
    __syncthreads();      // ... and every other thread's (and the twiddles are in place)
    {
      float2 v[M2], y[M2];
#pragma unroll
      for (int j2 = 0; j2 < M2; ++j2) v[j2] = sm[j2 * S + t * kTX + c];
      dft<M2, 0, 1, INV>(v, y);
      __syncthreads();  // every input slot is read before the exchange overwrites it
#pragma unroll
      for (int k2 = 0; k2 < M2; ++k2) {
        const float2 w = wy[t * k2];
        sm[tx<M1>(k2, t, c)] = k2 == 0 || t == 0 ? y[k2] : (INV ? cmulc(y[k2], w) : cmul(y[k2], w));
      }
    }
    __syncthreads();
    float2 u[R][M1];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k2 = t + M1 * rr;
      if (k2 < M2) {
#pragma unroll
        for (int j1 = 0; j1 < M1; ++j1) u[rr][j1] = sm[tx<M1>(k2, j1, c)];
      }
    }
    __syncthreads();  // the tile is read: the next tile's copies may go out
    if (tile + (int)gridDim.x < ntile) fetch_tile<M1, M2>(sm, base(tile + gridDim.x), es);
    float2* g = base(tile) + c;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k2 = t + M1 * rr;
      if (k2 < M2) {
        float2 o[M1];
        dft<M1, 0, 1, INV>(u[rr], o);
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) g[(k2 + M2 * k1) * es] = o[k1];
      }
    }
  }
}

// Z pass: forward FFT along z, scale by sign / (N lambda), inverse FFT along z.  Tiles are
// (column tile, ky); a persistent grid walks them (tile = block, block + grid, ...).  The twiddles
// W_nz^k and the z eigenvalues are copied to shared memory once per block (every lookup of a
// thread is then a shared-memory load: the table loads from L1 were the pass's main stall), and
// the copies of a tile's nz x 8 values go out as soon as the previous tile's values are read, so
// they overlap its inverse transform and stores.  Element e = t + M1 j2 of column c arrives at
// slot (j2, t, c); forward: A (M2-point over j2, thread (t, c)) writes slot (k2, t, c), B
// (M1-point over j1 = t) leaves owner k2 with X[k2 + M2 k1]; the owner scales and runs A' (M1-
// point over k1) and writes back to the slots it read, (k2, l2), so B -> scaling -> A' needs no
// barrier and keeps no line in registers across one; B' (M2-point over k2) reads slots (k2, t).
// In the solve it also stores this block's part of <y, (-L_h)^-1 y> = sum_k |Y(k)|^2 s(k)
// (Parseval; y = W rt, the half spectrum counting kx = 1 .. nx/2 - 1 twice), which is <rt, z>:
// FP32 per tile, summed over the block's tiles in FP64, always in the same order.
template <int M1, int M2>
constexpr size_t z_smem() {  // tile buffer, twiddles W_nz^k, eigenvalues lz
  return sizeof(float2) * (size_t)(line_buffer<M1, M2>() + M1 * M2) + sizeof(float) * (size_t)(M1 * M2);
}

template <int M1, int M2>
__global__ void __launch_bounds__(M1 * kTX, ZOcc<M1>::kMinBlocks) k_spec_z(SpecArgs a) {
  constexpr int R = (M2 + M1 - 1) / M1;
  constexpr int n = M1 * M2;
  constexpr int S = pad_stride(M1 * kTX);
  extern __shared__ __align__(16) float2 zbuf[];
  float2* sm = zbuf;                         // the tile
  float2* wz = zbuf + line_buffer<M1, M2>();  // W_nz^k, k < nz
  float* lz = reinterpret_cast<float*>(wz + n);
  if (!spec_active(a)) return;
  const Tables tb = tables(a);
  const int c = threadIdx.x % kTX, t = threadIdx.x / kTX;
  const int tiles = a.nxp / kTX;
  const int ntile = tiles * a.ny;
  const long long es = (long long)a.ny * a.nxp;  // element stride along z
  const int m = a.nx / 2;
  auto fetch = [&](int tile) {
    fetch_tile<M1, M2>(sm, a.spec + (long long)(tile / tiles) * a.nxp + (tile % tiles) * kTX, es);
  };
  int tile = blockIdx.x;
  if (tile < ntile) fetch(tile);
  for (int k = threadIdx.x; k < n; k += M1 * kTX) {
    wz[k] = tb.wz[k];
    lz[k] = tb.lz[k];
  }
  double energy_sum = 0.0;
  for (; tile < ntile; tile += gridDim.x) {
    cp_async_wait_all();  // this thread's copies of the tile have landed
    __syncthreads();      // ... and every other thread's (and the tables are in place)
    const int ky = tile / tiles, kx = (tile % tiles) * kTX + c;
    {
      float2 v[M2], y[M2];
#pragma unroll
      for (int j2 = 0; j2 < M2; ++j2) v[j2] = sm[j2 * S + t * kTX + c];
      dft<M2, 0, 1, false>(v, y);
      __syncthreads();  // every input slot is read before the exchange overwrites it
#pragma unroll
      for (int k2 = 0; k2 < M2; ++k2)
        sm[tx<M1>(k2, t, c)] = k2 == 0 || t == 0 ? y[k2] : cmul(y[k2], wz[t * k2]);
    }
    __syncthreads();
    const bool pad = kx > m;  // padding columns of the row pitch: set to 0
    const float lxy = pad ? 0.f : tb.lx[kx] + tb.ly[ky];
    const float wkx = (kx == 0 || kx == m) ? 1.f : 2.f;  // conjugate partners of the half spectrum
    float energy = 0.f;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k2 = t + M1 * rr;
      if (k2 < M2) {
        float2 u[M1], o[M1];
#pragma unroll
        for (int j1 = 0; j1 < M1; ++j1) u[j1] = sm[tx<M1>(k2, j1, c)];
        dft<M1, 0, 1, false>(u, o);
#pragma unroll
        for (int k1 = 0; k1 < M1; ++k1) {
          const float lam = lxy + lz[k2 + M2 * k1];
          // zero mode removed; the quotient is the hardware's approximate one (2 ulp)
          const float s = (lam > 0.f && !pad) ? __fdividef(a.scale, lam) : 0.f;
          energy = fmaf(wkx * s, fmaf(o[k1].x, o[k1].x, o[k1].y * o[k1].y), energy);
          o[k1] = cscale(o[k1], s);
        }
        dft<M1, 0, 1, true>(o, u);
#pragma unroll
        for (int l2 = 0; l2 < M1; ++l2)
          sm[tx<M1>(k2, l2, c)] = l2 == 0 || k2 == 0 ? u[l2] : cmulc(u[l2], wz[k2 * l2]);
      }
    }
    energy_sum += (double)energy;
    __syncthreads();
    float2 w[M2];
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) w[k2] = sm[tx<M1>(k2, t, c)];
    __syncthreads();  // the tile is read: the next tile's copies may go out
    if (tile + (int)gridDim.x < ntile) fetch(tile + gridDim.x);
    float2 o[M2];
    dft<M2, 0, 1, true>(w, o);
    float2* g = a.spec + (long long)ky * a.nxp + kx;
#pragma unroll
    for (int l1 = 0; l1 < M2; ++l1) g[(t + M1 * l1) * es] = o[l1];
  }
  if (a.st) {
    const double part[1] = {energy_sum * (double)a.ewt};
    store_partials<1, double>(part, a.I->part, gridDim.x, blockIdx.x);
  }
}

// ---- host side ----------------------------------------------------------------------------------

namespace {

// n = M1 x M2 for the supported line lengths (0 = unsupported)
void factor(int n, int* m1, int* m2) {
  switch (n) {
    case 16: *m1 = 4; *m2 = 4; return;
    case 24: *m1 = 4; *m2 = 6; return;
    case 32: *m1 = 4; *m2 = 8; return;
    case 48: *m1 = 6; *m2 = 8; return;  // x rows; y and z lines use 4 x 12 (warp-sized blocks)
    case 64: *m1 = 8; *m2 = 8; return;
    case 96: *m1 = 8; *m2 = 12; return;
    case 128: *m1 = 8; *m2 = 16; return;
    case 192: *m1 = 12; *m2 = 16; return;
    case 256: *m1 = 16; *m2 = 16; return;
    case 512: *m1 = 16; *m2 = 32; return;
    default: *m1 = 0; *m2 = 0; return;
  }
}

using SpecKernel = void (*)(SpecArgs);

template <class T>
SpecKernel x_kernel(int m, bool inverse, bool mirror, int* threads) {
  int m1, m2;
  factor(m, &m1, &m2);
#define VDP_X(M1, M2)                                                                       \
  if (m1 == M1 && m2 == M2) {                                                               \
    *threads = M1 * (inverse ? inv_rows_per_block<M1, M2>() : rows_per_block<M1, M2>());     \
    if (inverse)                                                                            \
      return mirror ? k_spec_x_inv_persistent<T, M1, M2, true>                              \
                    : k_spec_x_inv_persistent<T, M1, M2, false>;                            \
    if constexpr (sizeof(T) == 8 || kXFwdF32Persistent)                                     \
      return mirror ? k_spec_x_fwd_persistent<T, M1, M2, true>                              \
                    : k_spec_x_fwd_persistent<T, M1, M2, false>;                            \
    else                                                                                    \
      return mirror ? k_spec_x_fwd<T, M1, M2, true> : k_spec_x_fwd<T, M1, M2, false>;     \
  }
  VDP_X(4, 4) VDP_X(4, 6) VDP_X(4, 8) VDP_X(6, 8) VDP_X(8, 8) VDP_X(8, 12) VDP_X(8, 16)
  VDP_X(16, 16)
#undef VDP_X
  return nullptr;
}

int x_rows_per_block(int m, bool inverse) {
  int m1, m2;
  factor(m, &m1, &m2);
#define VDP_R(M1, M2) \
  if (m1 == M1 && m2 == M2) return inverse ? inv_rows_per_block<M1, M2>() : rows_per_block<M1, M2>();
  VDP_R(4, 4) VDP_R(4, 6) VDP_R(4, 8) VDP_R(6, 8) VDP_R(8, 8) VDP_R(8, 12) VDP_R(8, 16)
  VDP_R(16, 16)
#undef VDP_R
  return 0;
}

SpecKernel yz_kernel(int n, int which, int* threads, size_t* smem = nullptr) {
  // which: 0 = Y+, 1 = Y-, 2 = Z; smem: the pass's dynamic shared memory
  int m1, m2;
  factor(n, &m1, &m2);
  if (n == 48) {  // blocks of M1 * 8 threads: a whole number of warps for the block reduction
    m1 = 4;
    m2 = 12;
  }
#define VDP_YZ(M1, M2)                                                                  \
  if (m1 == M1 && m2 == M2) {                                                           \
    *threads = M1 * kTX;                                                                \
    if (smem) *smem = which == 2 ? z_smem<M1, M2>() : y_smem<M1, M2>();               \
    return which == 0 ? k_spec_y<M1, M2, false> : which == 1 ? k_spec_y<M1, M2, true>   \
                                                             : k_spec_z<M1, M2>;        \
  }
  VDP_YZ(4, 8) VDP_YZ(4, 12) VDP_YZ(8, 8) VDP_YZ(8, 12) VDP_YZ(8, 16) VDP_YZ(12, 16)
  VDP_YZ(16, 16) VDP_YZ(16, 32)
#undef VDP_YZ
  return nullptr;
}

// Resident blocks per SM of the Y+ / Y- / Z passes for each supported line length, per device
// (filled when the spectral passes are first prepared on the device): a persistent grid is that
// times the SMs.
constexpr int kLineLengths[] = {32, 48, 64, 96, 128, 192, 256, 512};
constexpr int kLineCount = sizeof(kLineLengths) / sizeof(kLineLengths[0]);
constexpr int kMaxDevices = 64;
int g_per_sm[kMaxDevices][3][kLineCount];

int current_device() {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices ? dev : -1;
}

int line_index(int n) {
  for (int i = 0; i < kLineCount; ++i)
    if (kLineLengths[i] == n) return i;
  return -1;
}

// Resident blocks per SM of the X kernels, per device (filled with the line tables).
std::vector<std::pair<SpecKernel, int>> g_x_per_sm[kMaxDevices];
constexpr int kXHalfLengths[] = {16, 24, 32, 48, 64, 96, 128, 256};  // nx / 2

bool x_f64(int prec, bool inv, const SpecArgs& a) { return prec == PREC_FP64 && !(inv && a.out_f32); }

SpecKernel x_pass_kernel(int prec, bool inv, const SpecArgs& a, int* threads) {
  const int m = a.nx / 2;
  return x_f64(prec, inv, a) ? x_kernel<double>(m, inv, a.mirror != 0, threads)
                             : x_kernel<float>(m, inv, a.mirror != 0, threads);
}

// Grid of an X pass over `rows` rows: a persistent grid for the persistent forms (0 if not
// prepared), else one block per group of rows.
long long x_grid(int prec, bool inv, const SpecArgs& a, long long rows) {
  int threads = 0;
  const SpecKernel k = x_pass_kernel(prec, inv, a, &threads);
  const int dev = current_device(), ry = x_rows_per_block(a.nx / 2, inv);
  if (!k || dev < 0 || ry <= 0) return 0;
  const bool persistent = inv || x_f64(prec, inv, a) || kXFwdF32Persistent;
  if (!persistent) return (rows + ry - 1) / ry;
  int per_sm = 0;
  for (const auto& e : g_x_per_sm[dev])
    if (e.first == k) per_sm = e.second;
  if (per_sm < 1) return 0;
  const long long groups = (rows + ry - 1) / ry, grid = (long long)per_sm * kSMs;
  return groups < grid ? groups : grid;
}

// Persistent grid of a Y (which 0, 1) or Z (2) pass over `tiles` tiles: 0 if not prepared.
long long line_grid(int which, int n, long long tiles) {
  const int dev = current_device(), i = line_index(n);
  const int per_sm = dev >= 0 && i >= 0 ? g_per_sm[dev][which][i] : 0;
  if (per_sm < 1) return 0;
  const long long grid = (long long)per_sm * kSMs;
  return tiles < grid ? tiles : grid;
}

bool x_supported(int nx) {
  if (nx % 2) return false;
  int threads = 0;
  return x_kernel<float>(nx / 2, false, false, &threads) != nullptr;
}

bool yz_supported(int n) {
  int threads = 0;
  return n != 16 && n != 24 && yz_kernel(n, 0, &threads) != nullptr;
}

}  // namespace

bool spectral_supported(int nx, int ny, int nz) {
  return x_supported(nx) && yz_supported(ny) && yz_supported(nz);
}

int spectral_pitch(int nx) { return ((nx / 2 + 1 + kTX - 1) / kTX) * kTX; }

size_t spectral_table_floats(int nx, int ny, int nz) {
  const int m = nx / 2;
  return 2 * (size_t)(2 * m + 1 + ny + nz) + (size_t)(m + 1 + ny + nz);
}

void spectral_tables(int nx, int ny, int nz, double hx, double hy, double hz,
                     std::vector<float>& out) {
  const int m = nx / 2;
  out.assign(spectral_table_floats(nx, ny, nz), 0.f);
  size_t i = 0;
  auto roots = [&](int n, int count) {
    for (int k = 0; k < count; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)n;
      out[i++] = (float)std::cos(ang);
      out[i++] = (float)std::sin(ang);
    }
  };
  roots(m, m);
  roots(nx, m + 1);
  roots(ny, ny);
  roots(nz, nz);
  auto eig = [&](int n, int count, double h) {
    for (int k = 0; k < count; ++k) {
      const double s = std::sin(M_PI * (double)k / (double)n);
      out[i++] = (float)(4.0 * s * s / (h * h));
    }
  };
  eig(nx, m + 1, hx);
  eig(ny, ny, hy);
  eig(nz, nz, hz);
}

cudaError_t spectral_upload_roots() {
  float2 w[96];
  for (int k = 0; k < 96; ++k) {
    const double ang = -2.0 * M_PI * (double)k / 96.0;
    w[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  cudaError_t e = cudaMemcpyToSymbol(c_w96, w, sizeof(w));
  const int dev = current_device();
  if (e == cudaSuccess && dev < 0) e = cudaErrorInvalidDevice;
  // the Y and Z passes' tile buffer and tables: dynamic shared memory (37 and 41 KB for lines
  // of 512), then the resident blocks per SM that size their persistent grids
  for (int which = 0; which < 3 && e == cudaSuccess; ++which)
    for (int i = 0; i < kLineCount && e == cudaSuccess; ++i) {
      int threads = 0;
      size_t smem = 0;
      const SpecKernel k = yz_kernel(kLineLengths[i], which, &threads, &smem);
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int per_sm = 0;
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
      if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
      if (e == cudaSuccess) g_per_sm[dev][which][i] = per_sm;
    }
  // the X kernels (static shared memory): resident blocks per SM, for the persistent grids
  g_x_per_sm[dev < 0 ? 0 : dev].clear();
  for (const int m : kXHalfLengths)
    for (int v = 0; v < 8 && e == cudaSuccess; ++v) {
      const bool f64 = v & 1, inv = v & 2, mirror = v & 4;
      int threads = 0, per_sm = 0;
      const SpecKernel k = f64 ? x_kernel<double>(m, inv, mirror, &threads)
                               : x_kernel<float>(m, inv, mirror, &threads);
      if (!k) continue;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0);
      if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
      if (e == cudaSuccess) g_x_per_sm[dev].push_back({k, per_sm});
    }
  return e;
}

cudaError_t launch_spectral_pass(int prec, int pass, const SpecArgs& a, cudaStream_t s) {
  int threads = 0;
  size_t smem = 0;
  SpecKernel k = nullptr;
  unsigned grid = 0;
  if (a.z0 < 0 || a.z1 > a.nz || a.z0 >= a.z1) return cudaErrorInvalidValue;
  switch (pass) {
    case SPEC_X_FWD:
    case SPEC_X_INV: {
      const bool inv = pass == SPEC_X_INV;
      k = x_pass_kernel(prec, inv, a, &threads);
      grid = (unsigned)x_grid(prec, inv, a, (long long)a.ny * (a.z1 - a.z0));
      break;
    }
    case SPEC_Y_FWD:
    case SPEC_Y_INV: {
      const int which = pass == SPEC_Y_FWD ? 0 : 1;
      k = yz_kernel(a.ny, which, &threads, &smem);
      grid = (unsigned)line_grid(which, a.ny, (long long)(a.nxp / kTX) * (a.z1 - a.z0));
      break;
    }
    case SPEC_Z:
      k = yz_kernel(a.nz, 2, &threads, &smem);
      grid = (unsigned)spectral_units(a.nx, a.ny, a.nz);
      break;
    default:
      break;
  }
  if (!k || !grid) return cudaErrorInvalidValue;
  k<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

// Slabs only on request: measured on the 512^3 mixed solve (half spectrum 553 MB), slabs of
// 128, 64 and 32 planes made one application 12 %, 20 % and 34 % slower than the whole grid --
// the passes gain less from the L2 hand-over than they lose to the extra launches and tails.
int spectral_slab_planes(int nx, int ny, int nz, int req) {
  (void)nx;
  (void)ny;
  return req > 0 && req < nz ? req : nz;
}

void spectral_schedule(int nz, int slab, std::vector<SpecLaunch>& out) {
  out.clear();
  if (slab < 1) slab = nz;
  for (int z0 = 0; z0 < nz; z0 += slab) {
    const int z1 = z0 + slab < nz ? z0 + slab : nz;
    out.push_back(SpecLaunch{SPEC_X_FWD, z0, z1});
    out.push_back(SpecLaunch{SPEC_Y_FWD, z0, z1});
  }
  out.push_back(SpecLaunch{SPEC_Z, 0, nz});
  for (int z0 = 0; z0 < nz; z0 += slab) {
    const int z1 = z0 + slab < nz ? z0 + slab : nz;
    out.push_back(SpecLaunch{SPEC_Y_INV, z0, z1});
    out.push_back(SpecLaunch{SPEC_X_INV, z0, z1});
  }
}

int spectral_xinv_units(int prec, const SpecArgs& a, int slab) {
  if (slab < 1) slab = a.nz;
  long long u = 0;
  for (int z0 = 0; z0 < a.nz; z0 += slab) {
    const int z1 = z0 + slab < a.nz ? z0 + slab : a.nz;
    u += x_grid(prec, true, a, (long long)a.ny * (z1 - z0));
  }
  return (int)u;
}

SpecArgs spectral_launch_args(int prec, const SpecArgs& a, const SpecLaunch& l, int slab) {
  SpecArgs b = a;
  b.z0 = l.z0;
  b.z1 = l.z1;
  b.xunits = spectral_xinv_units(prec, a, slab);
  return b;
}

cudaError_t launch_spectral_apply(int prec, const SpecArgs& a, int slab, cudaStream_t s) {
  std::vector<SpecLaunch> sched;
  spectral_schedule(a.nz, slab, sched);
  for (const SpecLaunch& l : sched) {
    const cudaError_t e = launch_spectral_pass(prec, l.pass, spectral_launch_args(prec, a, l, slab), s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int spectral_units(int nx, int ny, int nz) {  // CTAs of the Z pass (they store <rt, z> parts)
  return (int)line_grid(2, nz, (long long)(spectral_pitch(nx) / kTX) * ny);
}

__global__ void k_omega(const double* __restrict__ sinv, long long n, float* __restrict__ omega) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    omega[c] = (float)(1.0 / sinv[c]);
}

cudaError_t launch_omega(const double* sinv, long long n, float* omega, cudaStream_t s) {
  k_omega<<<152 * 8, 256, 0, s>>>(sinv, n, omega);
  return cudaGetLastError();
}

__global__ void k_rho_weight(const double* __restrict__ rho, const double* __restrict__ sinv,
                             long long n, float* __restrict__ out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    out[c] = (float)(rho[c] / sinv[c]);
}

cudaError_t launch_rho_weight(const double* rho, const double* sinv, long long n, float* out,
                              cudaStream_t s) {
  k_rho_weight<<<152 * 8, 256, 0, s>>>(rho, sinv, n, out);
  return cudaGetLastError();
}

}  // namespace vdp
