// vdp_multigrid.h -- host interface of the geometric multigrid preconditioner in
// vdp_multigrid.cu (internal to libvdp).
#pragma once

#include <cuda_runtime.h>

#include "vdp_internal.cuh"

namespace vdp {

constexpr int kMgMaxLevels = 16;
constexpr int kMgMinCoarsen = 64;    // a level with at most this many cells is not coarsened
constexpr int kMgMaxCoarsest = 512;  // the coarsest level is solved by a dense pseudo-inverse
constexpr float kMgOmega = 0.8f;     // weight of the Jacobi smoothing sweeps

// One level of the V-cycle, FP32.  The smoothed levels work in scaled variables (unit diagonal:
// bx, by, bz hold the scaled coefficients bt); level 0 is the solve's grid (its right side is the
// solve's scaled residual, its output the solve's z); the coarsest level is unscaled (solved by
// the pseudo-inverse).
struct MgLevel {
  int nx, ny, nz;
  long long n;
  float *bx, *by, *bz;  // face coefficients on the low faces
  float* om;            // W = D^1/2, D = sum of the six unscaled faces (levels >= 1 except the
  float* oinv;          //   coarsest) and 1 / W
  float* r;             // right side (restricted residual of the finer level; level 0: the
                        // FP32 copy of an FP64 rt)
  float* t;             // residual after pre-smoothing, then the prolonged iterate
  float* x;             // the level's result
};

struct MgHier {
  int nlev = 0;
  int wall_x = 0;         // the duct: transfers do not reach across the x ends
  MgLevel lev[kMgMaxLevels] = {};
  float* pinv = nullptr;  // ncoarse x ncoarse pseudo-inverse of -A on the coarsest level
  int ncoarse = 0;
  void* mem = nullptr;    // one allocation holds every array
  size_t bytes = 0;
};

// Number of levels for a grid (level 0 = the grid), or 0 when the coarsest level would exceed
// kMgMaxCoarsest cells or the grid has no coarser level; dims receives (nx, ny, nz) of each level.
int mg_level_dims(int nx, int ny, int nz, int (*dims)[3]);
inline bool mg_supported(int nx, int ny, int nz) {
  int d[kMgMaxLevels][3];
  return mg_level_dims(nx, ny, nz, d) > 0;
}
size_t mg_bytes(int nx, int ny, int nz);
cudaError_t mg_alloc(MgHier* h, int nx, int ny, int nz, int wall_x);
void mg_free(MgHier* h);
// Build every level's coefficients from the FP64 face coefficients of the grid (level 0 scaled
// by sinv = D^-1/2 on both sides) and the coarsest level's pseudo-inverse (host, double
// precision); synchronises stream s.
cudaError_t mg_setup(MgHier* h, const double* bx, const double* by, const double* bz,
                     const double* sinv, cudaStream_t s);
// out = in * sinv (n doubles)
cudaError_t launch_mg_scale(const double* in, const double* sinv, long long n, double* out,
                            cudaStream_t s);

// Arguments of one V-cycle application.
struct MgArgs {
  const void* in;      // scaled right side rt in the solve's precision (FP64 or FP32)
  void* out;           // scaled result z = W M W rt, same type
  const float* omega;  // W = D^1/2 per cell (FP32)
  InstState* st;       // the solve's state: the launches work only in PH_SPEC (null: always)
  const InstDesc* I;   // with st: the last launch stores <in, out> and completes the sweep
};
// prec: PREC_FP64 (double in/out) or an inner precision (float in/out).
cudaError_t launch_mg_vcycle(const MgHier& h, int prec, const MgArgs& a, cudaStream_t s);
int mg_launches(const MgHier& h, int prec);  // kernel launches of one V-cycle

}  // namespace vdp
