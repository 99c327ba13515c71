// vdp_ctx.h -- the solver context behind the opaque vdp_ctx handle of include/vdp.h, and the
// host helpers shared by the single-solve driver (vdp_api.cu) and the batch engine
// (vdp_batch.cu).  Internal to libvdp.
#pragma once

#include <cuda_runtime.h>

#include "vdp.h"
#include "vdp_internal.cuh"
#include "vdp_multigrid.h"

namespace vdp {

constexpr double kChebRange = 20.0;  // Chebyshev interval [2 / kChebRange, 2]

int cuda_fail(cudaError_t e, const char* where);  // records the message, maps to a vdp_status
bool is_device_ptr(const void* p);

}  // namespace vdp

#define VDP_CK(call)                                         \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return vdp::cuda_fail(_e, #call); \
  } while (0)

struct vdp_ctx {
  int nx = 0, ny = 0, nz = 0;
  double Lx = 0, Ly = 0, Lz = 0;   // box lengths
  int bc_x = VDP_BC_PERIODIC;      // VDP_BC_DUCT: no pressure flux through the x ends
  long long n = 0;
  int device = 0;
  vdp_opts opts{};
  cudaStream_t stream = nullptr;   // work stream (opts.stream)
  cudaStream_t cap = nullptr;      // private stream used only to capture graphs
  // FP64 operator data
  double *bx = nullptr, *by = nullptr, *bz = nullptr, *sinv = nullptr;
  double* dg = nullptr;  // D: the sum of the six face coefficients of each cell (FP64 residual)
  double* f0 = nullptr;  // f - <f>, written by the first residual of a solve from p = 0
  // inner-precision data (sized for FP64, reinterpreted for FP32 / BF16)
  void *sx = nullptr, *sy = nullptr, *sz = nullptr, *sd = nullptr;
  void *x = nullptr, *r = nullptr, *d0 = nullptr, *d1 = nullptr, *q = nullptr;
  void *za = nullptr, *zb = nullptr, *dch = nullptr;  // preconditioned z; Chebyshev iterates
  // spectral preconditioner / constant-coefficient inverse
  float2* spec = nullptr;          // half spectrum
  float* omega = nullptr;          // D^1/2 per cell (FP32)
  float* sptab = nullptr;          // twiddle and eigenvalue tables
  bool omega_valid = false;        // omega matches the current density
  float* rho_w = nullptr;          // fixed-point iteration: rho D^1/2 per cell (FP32)
  bool rho_w_valid = false;        // rho_w was computed from the current density
  vdp::MgHier* mg = nullptr;       // multigrid levels (VDP_PRECOND_MG, vdp_mg_apply)
  bool mg_valid = false;           // the levels were built from the current density
  int scaled_prec = -1;            // precision the scaled coefficients were built for
  bool has_density = false;
  // bookkeeping
  double* part = nullptr;
  unsigned int* ticket = nullptr;
  vdp::InstState* st = nullptr;
  vdp::InstDesc* desc = nullptr;
  vdp::UnitRef* units = nullptr;
  int* flag = nullptr;
  double *stage_a = nullptr, *stage_b = nullptr;  // staging for host pointers
  double* proj_f = nullptr;        // vdp_project: the assembled Poisson right side
  vdp::InstState* hstate = nullptr;     // pinned, 2 entries
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs[2] = {nullptr, nullptr};
  // layout
  vdp::Layout lay{};
  vdp::InstDesc hdesc{};           // host copy of the device description (after layout)
  bool hdesc_valid = false;
  int layout_prec = -1;
  bool layout_dirty = true;
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  int g_prec = -1, g_steps = 0;
  // device-side loop: one graph per solve whose WHILE node repeats the rounds until done
  cudaGraphExec_t wexec = nullptr;
  int w_prec = -1;
  bool w_failed = false;           // the driver cannot build it: use the polling schedule
  unsigned* d_rounds = nullptr;
  vdp_stats stats{};
};


namespace vdp {

// Make the context ready to run in precision `prec`: scaled coefficients built and the unit
// layout (and its device description) configured.
int configure_layout(vdp_ctx* c, int prec);
int ensure_scaled(vdp_ctx* c, int prec);
// length of the x transform of the spectral passes: nx, or 2 nx in the duct (even extension)
inline int spectral_nx(const vdp_ctx* c) { return c->bc_x == VDP_BC_DUCT ? 2 * c->nx : c->nx; }
// allocate the spectral buffers and tables (no-op when present); VDP_EINVAL for unsupported grids
int ensure_spectral(vdp_ctx* c);
// the arguments of the five spectral passes of a solve on this context (gated on its state)
struct SpecArgs;
void solve_spec_args(const vdp_ctx* c, int prec, SpecArgs* a);
int spec_slab(const vdp_ctx* c);  // planes per slab of the spectral passes
// allocate the multigrid levels and the z and omega buffers (no-op when present); VDP_EINVAL
// for grids the V-cycle does not support
int ensure_mg(vdp_ctx* c);
// kernel launches of one application of the solve's preconditioner (spectral passes, V-cycle)
int precond_launches(const vdp_ctx* c);
// before a solve that uses the spectral passes or the V-cycle: the weights (and the multigrid
// levels) for the current density (VDP_EINVAL when the fixed-point method's density weight is
// missing)
int prepare_spectral_solve(vdp_ctx* c);

}  // namespace vdp
