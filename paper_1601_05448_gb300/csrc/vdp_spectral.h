// vdp_spectral.h -- host interface of the spectral passes in vdp_spectral.cu (internal to libvdp).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "vdp_internal.cuh"

namespace vdp {

// The five passes of one application of the constant-coefficient inverse, in launch order.
enum SpecPass : int { SPEC_X_FWD = 0, SPEC_Y_FWD = 1, SPEC_Z = 2, SPEC_Y_INV = 3, SPEC_X_INV = 4,
                      SPEC_PASSES = 5 };

// Arguments of every spectral pass (by value).
struct SpecArgs {
  const void* in;        // X+: nxd*ny*nz values of the inner type (FP64 or FP32)
  void* out;             // X-: output, same layout; the inner type, or FP32 with out_f32
  int out_f32;           // X-: store FP32 (the fixed-point iteration's z)
  const float* omega_in;   // per-cell weight applied before X+ (or null: 1)
  const float* omega_out;  // per-cell weight applied after X- (or null: 1)
  float2* spec;          // half spectrum [nz][ny][nxp]
  const float2* tw;      // tables built by spectral_tables (twiddles first, then eigenvalues)
  const float* lam;
  int nx, ny, nz, nxp;   // transform lengths (nx: the x transform) and the spectrum's row pitch
  int nxd;               // cells per row of in / out: nx, or nx / 2 with mirror
  int mirror;            // duct: the x transform acts on the even extension of each row
                         // (cells 0 .. nxd - 1, then nxd - 1 .. 0), whose periodic Laplacian
                         // is the zero-flux one on the first half; X- keeps the first half
  float ewt;             // weight of the <rt, z> energy (1, or 1/2 for the doubled rows)
  float scale;           // sign / (nx ny nz): +1 applies (-L_h)^-1, -1 applies L_h^-1
  InstState* st;         // the solve's state: passes run only in PH_SPEC (null: always run)
  const InstDesc* I;     // the solve's description, with st: Z stores the partial sums of
                         // <rt, z>, X- completes the sweep
  int zunits;            // CTAs of the Z pass (partial slots), with st
  int z0, z1;            // X and Y passes: the planes [z0, z1) of this launch (a slab)
  int xunits;            // CTAs of all X- launches of one application (the sweep's arrivals)
};
// Passed by value to every pass: kept at 128 bytes.  One more int (136 bytes) made the X and Z
// passes of the 512^3 mixed solve 5-20 % slower (the solve 35.9 against 34.1 ms, same kernels).
static_assert(sizeof(SpecArgs) <= 128, "SpecArgs grew past 128 bytes");

// One launch of an application: the pass and its plane range.
struct SpecLaunch {
  int pass;
  int z0, z1;
};

bool spectral_supported(int nx, int ny, int nz);
int spectral_pitch(int nx);                       // nxp
size_t spectral_table_floats(int nx, int ny, int nz);
// twiddles (float2 pairs) W_m (m = nx/2), W_nx (m + 1), W_ny, W_nz, then the eigenvalue factors
// 4 sin^2(pi k / n_d) / h_d^2 for kx = 0..m, ky, kz; computed in double, stored as float
void spectral_tables(int nx, int ny, int nz, double hx, double hy, double hz,
                     std::vector<float>& out);
cudaError_t spectral_upload_roots();               // the register-DFT roots, once per device
cudaError_t launch_spectral_pass(int prec, int pass, const SpecArgs& a, cudaStream_t s);
int spectral_units(int nx, int ny, int nz);        // CTAs of the Z pass (partial slots)
// Planes per slab of one application: req (vdp_opts.spec_slab) when positive and below nz, else
// nz (a single slab).  With slabs the X+ / Y+ passes (and Y- / X-) run slab by slab,
// interleaved, so that a slab's spectrum can still be in L2 when the next pass reads it.
int spectral_slab_planes(int nx, int ny, int nz, int req);
// The launch sequence of one application: X+, Y+ per slab; Z; Y-, X- per slab.
void spectral_schedule(int nz, int slab, std::vector<SpecLaunch>& out);
// CTAs of all X- launches of one application (prec: PREC_*, as passed to the launches)
int spectral_xinv_units(int prec, const SpecArgs& a, int slab);
// Args of launch l (the plane range and the X- unit count filled in).
SpecArgs spectral_launch_args(int prec, const SpecArgs& a, const SpecLaunch& l, int slab);
// All launches of one application, in order.
cudaError_t launch_spectral_apply(int prec, const SpecArgs& a, int slab, cudaStream_t s);
cudaError_t launch_omega(const double* sinv, long long n, float* omega, cudaStream_t s);
// out = rho / sinv (the fixed-point iteration's input weight)
cudaError_t launch_rho_weight(const double* rho, const double* sinv, long long n, float* out,
                              cudaStream_t s);

}  // namespace vdp
