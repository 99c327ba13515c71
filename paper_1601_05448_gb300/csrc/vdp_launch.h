// vdp_launch.h -- host-side launchers of the kernels in vdp_kernels.cu (internal to libvdp).
#pragma once

#include <cuda_runtime.h>

#include "vdp_internal.cuh"

namespace vdp {

cudaError_t launch_check_density(const double* rho, long long n, int* bad, cudaStream_t s);
// face coefficients on the low faces (spacings h_d; duct: no flux through the x ends) and D^-1/2
cudaError_t launch_build_coefficients(const double* rho, int nx, int ny, int nz, double hx,
                                      double hy, double hz, int duct, double* bx, double* by,
                                      double* bz, double* sinv, double* dg, cudaStream_t s);
cudaError_t launch_scaled(int prec, const double* bx, const double* by, const double* bz,
                          const double* sinv, int nx, int ny, int nz, void* sx, void* sy, void* sz,
                          void* sd, cudaStream_t s);
cudaError_t launch_apply(const double* bx, const double* by, const double* bz, const double* p,
                         int nx, int ny, int nz, double* out, cudaStream_t s);
cudaError_t launch_init(InstDesc* desc, const double* rhs, double* p, double tol, double inner_tol,
                        int max_iter, int inner_max, int use_guess, int precision,
                        cudaStream_t s);
cudaError_t prepare_step(int prec, int mode, size_t smem_bytes);
// mode 0 only: the FP64 residual sweep (its own kernel, launched before each stencil launch)
cudaError_t launch_res64(int prec, const InstDesc* desc, const UnitRef* units, int nunits,
                         int threads, cudaStream_t s);
// kind (direct sweep variants): 0 = CG, 1 = CG and Chebyshev preconditioner sweeps (PH_CHEB),
// 2 = the fixed-point iteration; stencil_kind(pc) picks it for an instance's preconditioner
inline int stencil_kind(int pc) { return pc == PC_FIXED ? 2 : (pc == PC_CHEB ? 1 : 0); }
cudaError_t launch_stencil(int prec, int mode, int kind, const InstDesc* desc,
                           const UnitRef* units, int nunits, int threads, size_t smem_bytes,
                           cudaStream_t s);
cudaError_t launch_flat(int prec, const InstDesc* desc, const UnitRef* units, int nunits,
                        cudaStream_t s);

cudaError_t persistent_grid(int prec, int* grid);
cudaError_t launch_persistent(int prec, const InstDesc* desc, const UnitRef* sunits, int ns,
                              const UnitRef* funits, int nf, int pairs, BatchCtl* ctl, int grid,
                              cudaStream_t s);
cudaError_t launch_gather(const InstDesc* desc, int n, InstState* out, cudaStream_t s);
// device-side solve loop: sets the WHILE condition `handle` to continue while the instance is
// unfinished and fewer than max_rounds loop iterations have run (*rounds counts them)
cudaError_t launch_continue(const InstState* st, cudaGraphConditionalHandle handle,
                            unsigned* rounds, unsigned max_rounds, cudaStream_t s);

}  // namespace vdp
