// vdp_internal.cuh -- device-side data structures shared by the solver kernels and the host
// driver of libvdp.  Not part of the public ABI (include/vdp.h is).
//
// The solve is a small state machine per problem instance, advanced one "sweep" at a time by
// the step kernel.  A sweep is a pass over the instance's grid.  The grid is cut into row tiles
// (full x rows, ty rows); the (row tile, z plane) pairs, ordered tile-major with z fastest, are
// split into `nunits` equal contiguous ranges, one per work unit (CTA).  A unit therefore walks
// one or two long runs of consecutive z planes ("segments") of at most two row tiles, which is
// what the z-marching stencil sweeps need.  Each unit writes its partial sums into its own slot
// and the last unit to finish (atomic ticket) reduces the slots in a fixed order and moves the
// instance to its next phase.  Results are therefore bitwise reproducible for a fixed
// (ty, nunits), whether an instance runs alone or inside a batch.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace vdp {

// Phases of one solve (see the step kernel for what each sweep does).
enum Phase : int {
  PH_MEANF = 0,    // <f>, ||f||; p := 0 unless the caller gave a guess
  PH_RES64 = 1,    // FP64 residual r = (f - <f>) - A p, inner rhs rt = D^-1/2 r, norms, sum(p)
  PH_STENCIL = 2,  // d = rt + beta d_old; q = At d; <d, q>
  PH_UPDATE = 3,   // x += alpha d; rt -= alpha q; <rt, rt>
  PH_CORRECT = 4,  // p -= D^-1/2 x   (refinement step of the outer FP64 loop)
  PH_FINAL = 5,    // p -= <p>  (gauge)
  PH_CHEB = 6,     // one Chebyshev sweep of the polynomial preconditioner z = P(At) rt
  PH_SPEC = 7,     // preconditioner z = M^-1 rt: five FFT passes (spectral) or a V-cycle (multigrid)
  PH_DONE = 8
};

// Preconditioner applied to the Jacobi-scaled inner system (InstDesc::pc).
// PC_FIXED: not a preconditioner but the paper's fixed-point iteration, which applies the
// spectral passes (with a density-weighted input) between FP64 residuals instead of running CG.
enum PrecondKind : int { PC_JACOBI = 0, PC_CHEB = 1, PC_SPECTRAL = 2, PC_FIXED = 3, PC_MG = 4 };

enum Prec : int { PREC_FP64 = 0, PREC_MIXED = 1, PREC_MIXED_BF16 = 2 };

constexpr int kSlots = 4;          // partial-sum slots per unit
constexpr int kMaxThreads = 512;   // threads per stencil work unit (CTA), at most
constexpr int kFlatThreads = 256;  // threads per flat work unit
constexpr int kDirectThreads = 256;  // threads per direct-stencil work unit, at most
constexpr int kMaxStages = 8;      // shared-memory pipeline stages of the stencil sweep

// Mutable per-instance solver state (device memory).
struct InstState {
  int phase;
  int status;          // vdp_status
  int iters;           // total inner iterations
  int inner_iters;     // iterations of the current inner solve
  int outer;           // FP64 residual evaluations
  int parity;          // which direction buffer holds the current search direction
  int first_res;       // next RES64 also measures ||f - <f>||
  int zero_sol;        // f - <f> == 0: the answer is p = 0
  int sweeps;          // sweeps executed (all phases)
  int max_iter;
  int inner_max;
  int use_guess;
  int precision;
  int fault;           // a unit's bounded wait expired (reported as VDP_ETIMEOUT)
  int cheb_j;          // Chebyshev sweep index (1 .. cheb_k - 1)
  int p_set;           // p holds an iterate: the caller's guess, or a correction was applied
                       // (from p = 0 the first correction writes p without reading it)
  double rz;           // <rt, z> (preconditioned inner product; = <rt, rt> for Jacobi)
  double tol;          // requested relative residual
  double inner_tol;    // mixed: minimum relative reduction per inner solve
  double mu_f;         // <f>
  double fn2;          // ||f - <f>||^2
  double f2;           // n <f>^2 (the constant-f test compares ||f - <f>||^2 with it)
  double rr64;         // ||r||^2 at the last RES64
  double rr64_prev;    // ... at the RES64 before
  double rr;           // <rt, rt> (current inner)
  double rr0;          // <rt, rt> at the start of the inner solve
  double alpha, beta;
  double tau2;         // inner stop: rr <= tau2 * rr0
  double eta;          // observed ratio between FP64 and scaled inner residual reductions
  double inner_ratio;  // sqrt(rr / rr0) at the end of the last inner solve
  double sum_p;        // sum of p at the last RES64
  double rel_res;      // FP64 relative residual at the last RES64
};

// Constant per-instance description (device memory).  Stencil sweeps split the grid into
// nunits = uy * zc units (row tile x z chunk); flat sweeps split the cells into `nunits_f`
// contiguous ranges.
struct InstDesc {
  int nx, ny, nz;
  int ty;              // rows per row tile
  int uy;              // row tiles
  int nunits;          // stencil work units (CTAs) per sweep
  int stages;          // shared-memory pipeline stages of the stencil sweep
  int nunits_f;        // flat work units per sweep
  int zc;              // z chunks: stencil unit u = (row tile u % uy, z chunk u / uy)
  int mode;            // stencil sweep: 0 = direct register march, 1 = TMA-staged pipeline
  long long ncell;
  const double* rhs;   // caller's f (set per solve)
  double* p;           // caller's p (set per solve)
  const double* bx;    // FP64 face coefficients 2/(rho_l+rho_r)/h^2 on the low faces
  const double* by;
  const double* bz;
  const double* sinv;  // D^-1/2, D = sum of the six face coefficients of a cell
  const double* dg;    // D itself (the FP64 residual's diagonal term)
  double* f0;          // f - <f> (null: the residual subtracts <f> itself); written by the first
                       // residual of a solve from p = 0, read by the later ones
  const void* sx;      // scaled coefficients bt = b sinv_l sinv_r in the inner storage type
  const void* sy;
  const void* sz;
  const void* sd;      // BF16 only: diagonal correction of the stored inner operator
  void* x;             // inner solution (correction), inner type
  void* r;             // inner residual
  void* d0;            // search direction, double buffered
  void* d1;
  void* q;             // At d
  void* za;            // Chebyshev: z iterates (double buffered; the final z is in za) and
  void* zb;            //   the Chebyshev correction d_j (null without the polynomial)
  void* dch;
  int cheb_k;          // polynomial preconditioner: number of terms (1 = Jacobi only)
  int pc;              // PrecondKind (PC_CHEB only with cheb_k > 1)
  double cheb_theta;   // Chebyshev interval [a, b]: theta = (b + a) / 2, delta = (b - a) / 2
  double cheb_delta;
  double* part;        // kSlots x nunits partial sums
  unsigned int* ticket;
  InstState* st;
  int* remaining;      // batch: count of unfinished instances (decremented at DONE), or null
};

// Control words of a batch's persistent kernel (device memory).
struct BatchCtl {
  unsigned int count;  // grid barrier arrivals
  unsigned int gen;    // grid barrier generation
  int remaining;       // unfinished instances
  int fault;           // a grid barrier wait expired
  unsigned int extra;  // arrivals expected beyond the grid (failure injection for tests; 0)
  unsigned int pad;
  unsigned long long limit_ns;  // bound on one grid barrier wait
};

struct UnitRef {
  int inst;            // index into the batch's InstDesc table
  int unit;            // unit index within the instance
};

// Bytes of one stencil pipeline stage: d/rt and d_old rows with one halo row on each side,
// then the three coefficient arrays (x: ty rows, y: ty + 1 rows, z: ty rows) and, for BF16
// coefficients, the diagonal correction (ty rows); each piece is a whole number of rows, so
// 16-byte aligned whenever a row is.
__host__ __device__ inline size_t stage_bytes(int nx, int ty, int tsize, int bsize, bool diag) {
  size_t b = (size_t)2 * (ty + 2) * nx * tsize + (size_t)(3 * ty + 1 + (diag ? ty : 0)) * nx * bsize;
  return (b + 127) & ~(size_t)127;
}

// Bytes of the three-plane ring of the FP64 residual sweep.
__host__ __device__ inline size_t ring_bytes(int nx, int ty) {
  return (size_t)3 * (ty + 2) * nx * sizeof(double);
}

// ---- work decomposition (host) ------------------------------------------------------------------

constexpr int kSMs = 152;                 // GB300
constexpr size_t kSmemPerSM = 227 * 1024; // shared memory per SM available to CTAs
constexpr size_t kSmemBudget = 225 * 1024;

struct Layout {
  int mode;            // stencil sweep variant (0 direct, 1 TMA pipeline)
  int ty;              // rows per row tile
  int uy;              // row tiles
  int stages;          // stencil pipeline stages
  int threads;         // stencil threads per unit
  int zc;              // z chunks
  int nunits;          // stencil units = uy * zc
  int nunits_f;        // flat units
  size_t smem;         // dynamic shared memory of the stencil kernel
};

// Inner type size, coefficient size and BF16 diagonal correction per precision.
inline void prec_sizes(int prec, int* ts, int* bs, bool* diag) {
  *ts = prec == PREC_FP64 ? 8 : 4;
  *bs = prec == PREC_FP64 ? 8 : (prec == PREC_MIXED ? 4 : 2);
  *diag = prec == PREC_MIXED_BF16;
}

// Unit layout for an nx x ny x nz grid in precision `prec`; zero arguments pick the defaults.
// mode 0 (direct, default): units of up to 256 threads (whole rows, whole warps), one thread per
// 16-byte vector of a row tile of threads * V / nx rows (V = 4 FP32, 2 FP64), about 12 units per
// SM worth of z chunks.
// mode 1 (TMA pipeline): FP64 512-thread units with about 2048 cells per plane, FP32/BF16 256
// threads with about 1024; the row tile shrinks until four pipeline stages fit; stages default to
// what fits (at most 6), or to 4 when that lets two units share an SM; about four waves.
// Both: stencil units = row tiles x z chunks (chunk-major); flat units of about 4096+ cells (at
// most 8 per SM).  In mode 1 the dynamic shared memory also covers the FP64 residual sweep's ring.
// Returns false when the configuration cannot run (rows too long, bad counts).
inline bool plan_layout(int nx, int ny, int nz, int prec, int mode, int tile_y, int units,
                        int stages, int threads, Layout* L) {
  int ts, bs;
  bool diag;
  prec_sizes(prec, &ts, &bs, &diag);
  const int V = 16 / ts;
  int nt, ty, S = 0, per_sm;
  size_t smem;
  if (mode == 0) {
    // largest block of whole rows that is a whole number of warps: a multiple of
    // lcm(nx / V, 32) threads, at most kDirectThreads
    const int tpr = nx / V;
    int g = tpr, b = 32;
    while (b) {
      const int t = g % b;
      g = b;
      b = t;
    }
    const int unit = tpr / g * 32;
    nt = threads > 0 ? threads : (kDirectThreads / unit) * unit;
    if (nt < 32 || nt > kDirectThreads || nt % 32 || (nt * V) % nx) return false;
    ty = nt * V / nx;  // the tile is exactly one vector per thread
    if (ty < 1) return false;
    if (tile_y > 0 && tile_y != ty) return false;
    smem = 0;  // no shared memory: both stencil-kind sweeps march in registers
    per_sm = 6;
  } else if (mode == 1) {
    nt = threads > 0 ? threads : (prec == PREC_FP64 ? 512 : 256);
    if (nt < 128 || nt > kMaxThreads || nt % 32) return false;  // four warps issue the copies
    const int cells = prec == PREC_FP64 ? 2048 : 1024;
    ty = tile_y > 0 ? tile_y : (cells / nx > 1 ? cells / nx : 1);
    if (ty > ny) ty = ny;
    while (ty > 1 && 4 * stage_bytes(nx, ty, ts, bs, diag) > kSmemBudget) --ty;
    const size_t sb = stage_bytes(nx, ty, ts, bs, diag);
    const int fit = (int)(kSmemBudget / sb);
    if (fit < 4) return false;
    S = stages;
    if (S <= 0) {
      S = fit < 6 ? fit : 6;
      if (4 * sb + 1024 <= kSmemPerSM / 2 && 2 * nt <= 2048) S = 4;  // two units per SM
    }
    if (S < 4 || S > kMaxStages || S > fit) return false;
    smem = (size_t)S * sb > ring_bytes(nx, ty) ? (size_t)S * sb : ring_bytes(nx, ty);
    per_sm = (2 * (smem + 1024) <= kSmemPerSM && 2 * nt <= 2048) ? 2 : 1;
    per_sm *= 2;  // about four waves of units
  } else {
    return false;
  }
  if (ty > ny) ty = ny;
  const int uy = (ny + ty - 1) / ty;
  const long long want = units > 0 ? units : 2LL * kSMs * per_sm;
  long long zc = (want + uy - 1) / uy;
  if (zc > nz) zc = nz;
  if (zc < 1) zc = 1;
  const long long ncell = (long long)nx * ny * nz;
  long long nf = ncell / 4096;
  if (nf > kSMs * 8) nf = kSMs * 8;
  if (nf < 1) nf = 1;
  L->mode = mode;
  L->ty = ty;
  L->uy = uy;
  L->stages = S;
  L->threads = nt;
  L->zc = (int)zc;
  L->nunits = (int)(zc * uy);
  L->nunits_f = (int)nf;
  L->smem = smem;
  return true;
}

}  // namespace vdp
