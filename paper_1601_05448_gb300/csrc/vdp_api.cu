// vdp_api.cu -- the C ABI of libvdp (include/vdp.h): contexts, device buffers, the solve driver.
//
// A solve is one instance of the per-instance state machine (vdp_internal.cuh, transitions in
// vdp_device.cuh), advanced by the sweep kernels of vdp_kernels.cu and vdp_spectral.cu.  The
// driver launches one graph per solve whose WHILE node repeats rounds -- residual, (five
// spectral passes,) stencil and flat kernels, each returning at once unless the phase is its
// own -- until a condition kernel sees the solve done.  With steps_per_sync > 0 (or a driver
// without conditional nodes) it instead replays graphs of that many rounds, copies the state to
// pinned host memory after each, and keeps two in flight so the host check overlaps device work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vdp.h"
#include "vdp_internal.cuh"
#include "vdp_launch.h"
#include "vdp_ctx.h"
#include "vdp_spectral.h"

using namespace vdp;

namespace {
std::mutex g_err_mu;
std::string g_last_cuda_error;
}  // namespace

namespace vdp {

int cuda_fail(cudaError_t e, const char* where) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_last_cuda_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? VDP_ENOMEM : VDP_ECUDA;
}


bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace vdp

extern "C" {

void vdp_default_options(vdp_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = VDP_FP64;
  o->max_iter = 20000;
  o->inner_tol = 1e-4;
  o->precond = VDP_PRECOND_JACOBI;
  o->cheb_degree = 4;
  o->use_guess = 0;
  o->stream = nullptr;
  o->tile_y = 0;
  o->stencil = 0;
  o->units = 0;
  o->stages = 0;
  o->threads = 0;
  o->steps_per_sync = 0;
  o->method = VDP_METHOD_CG;
  o->damping = 1.0;
  o->spec_slab = 0;
}

const char* vdp_strerror(int s) {
  switch (s) {
    case VDP_OK: return "VDP_OK";
    case VDP_EINVAL: return "VDP_EINVAL: invalid argument or call order";
    case VDP_ENOMEM: return "VDP_ENOMEM: out of device memory or budget";
    case VDP_EDENSITY: return "VDP_EDENSITY: density not positive and finite";
    case VDP_ENOTCONV: return "VDP_ENOTCONV: iteration limit reached";
    case VDP_EBREAKDOWN: return "VDP_EBREAKDOWN: Krylov breakdown";
    case VDP_ETIMEOUT: return "VDP_ETIMEOUT: bounded device wait expired";
    case VDP_ECUDA: return "VDP_ECUDA: CUDA runtime error";
    default: return "VDP_?: unknown status";
  }
}

const char* vdp_last_cuda_error(void) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_last_cuda_error.c_str();
}

int vdp_version(void) { return 2; }

}  // extern "C"

namespace vdp {

void free_ctx(vdp_ctx* c) {
  if (!c) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->wexec) cudaGraphExecDestroy(c->wexec);
  if (c->mg) {
    mg_free(c->mg);
    delete c->mg;
  }
  void* bufs[] = {c->bx, c->by, c->bz, c->sinv, c->dg, c->f0, c->sx, c->sy, c->sz, c->sd, c->x, c->r, c->d0, c->d1,
                  c->za, c->zb, c->dch, c->spec, c->omega, c->sptab, c->rho_w, c->d_rounds,
                  c->q, c->part, c->ticket, c->st, c->desc, c->units, c->flag, c->stage_a,
                  c->stage_b, c->proj_f};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->hstate) cudaFreeHost(c->hstate);
  cudaEvent_t evs[] = {c->ev0, c->ev1, c->evs[0], c->evs[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (prev >= 0) cudaSetDevice(prev);
  delete c;
}

int choose_layout(const vdp_ctx* c, int prec, Layout* out) {
  return plan_layout(c->nx, c->ny, c->nz, prec, c->opts.stencil, c->opts.tile_y, c->opts.units,
                     c->opts.stages, c->opts.threads, out)
             ? VDP_OK
             : VDP_EINVAL;
}

int configure_layout(vdp_ctx* c, int prec) {
  Layout lay;
  int s = choose_layout(c, prec, &lay);
  if (s != VDP_OK) return s;
  c->lay = lay;
  c->hdesc_valid = false;
  std::vector<UnitRef> u(lay.nunits + lay.nunits_f);
  for (int i = 0; i < lay.nunits; ++i) u[i] = UnitRef{0, i};
  for (int i = 0; i < lay.nunits_f; ++i) u[lay.nunits + i] = UnitRef{0, i};
  VDP_CK(cudaMemcpyAsync(c->units, u.data(), sizeof(UnitRef) * u.size(), cudaMemcpyHostToDevice,
                         c->stream));
  InstDesc d{};
  d.nx = c->nx;
  d.ny = c->ny;
  d.nz = c->nz;
  d.ty = lay.ty;
  d.uy = lay.uy;
  d.nunits = lay.nunits;
  d.nunits_f = lay.nunits_f;
  d.stages = lay.stages;
  d.zc = lay.zc;
  d.mode = lay.mode;
  d.ncell = c->n;
  d.bx = c->bx;
  d.by = c->by;
  d.bz = c->bz;
  d.sinv = c->sinv;
  d.dg = c->dg;
  d.f0 = c->f0;
  d.sx = c->sx;
  d.sy = c->sy;
  d.sz = c->sz;
  d.sd = c->sd;
  d.x = c->x;
  d.r = c->r;
  d.d0 = c->d0;
  d.d1 = c->d1;
  d.q = c->q;
  d.za = c->za;
  d.zb = c->zb;
  d.dch = c->dch;
  // polynomial preconditioner: Chebyshev on [b / kChebRange, b], b = 2 >= the largest
  // eigenvalue of the unit-diagonal operator
  d.cheb_k = c->opts.precond == VDP_PRECOND_CHEB ? c->opts.cheb_degree : 1;
  d.pc = c->opts.method == VDP_METHOD_FIXED_POINT ? PC_FIXED
         : c->opts.precond == VDP_PRECOND_SPECTRAL ? PC_SPECTRAL
         : c->opts.precond == VDP_PRECOND_MG       ? PC_MG
                                                   : (d.cheb_k > 1 ? PC_CHEB : PC_JACOBI);
  {
    const double b = 2.0, a = b / kChebRange;
    d.cheb_theta = 0.5 * (b + a);
    d.cheb_delta = 0.5 * (b - a);
  }
  d.part = c->part;
  d.ticket = c->ticket;
  d.st = c->st;
  c->hdesc = d;
  c->hdesc_valid = true;
  VDP_CK(cudaMemcpyAsync(c->desc, &d, sizeof(d), cudaMemcpyHostToDevice, c->stream));
  VDP_CK(cudaStreamSynchronize(c->stream));
  VDP_CK(prepare_step(prec, lay.mode, lay.smem));
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  if (c->wexec) {
    cudaGraphExecDestroy(c->wexec);
    c->wexec = nullptr;
  }
  c->layout_prec = prec;
  c->layout_dirty = false;
  return VDP_OK;
}

int steps_per_sync(const vdp_ctx* c) {
  if (c->opts.steps_per_sync > 0) return c->opts.steps_per_sync;
  return 16;
}

// One round of the solve's launch schedule: residual kernel (direct form), the five spectral
// passes (spectral preconditioner or fixed-point iteration), stencil kernel, flat kernel; each
// returns at once unless the instance's phase is its own.
cudaError_t launch_round(vdp_ctx* c, int prec, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (c->lay.mode == 0)  // the residual sweep has its own kernel in the direct mode
    e = launch_res64(prec, c->desc, c->units, c->lay.nunits, c->lay.threads, s);
  if (e == cudaSuccess && c->hdesc.pc == PC_MG) {  // z = W M W rt by one V-cycle
    const MgArgs a{c->r, c->za, c->omega, c->st, c->desc};
    e = launch_mg_vcycle(*c->mg, prec, a, s);
  } else if (e == cudaSuccess && c->hdesc.pc >= PC_SPECTRAL) {  // z = M^-1 rt first
    SpecArgs a;
    solve_spec_args(c, prec, &a);
    e = launch_spectral_apply(prec, a, spec_slab(c), s);
  }
  if (e == cudaSuccess)
    e = launch_stencil(prec, c->lay.mode, stencil_kind(c->hdesc.pc), c->desc, c->units,
                       c->lay.nunits, c->lay.threads, c->lay.smem, s);
  if (e == cudaSuccess) e = launch_flat(prec, c->desc, c->units + c->lay.nunits, c->lay.nunits_f, s);
  return e;
}

int ensure_graph(vdp_ctx* c, int prec) {
  int m = steps_per_sync(c);
  if (c->gexec && c->g_prec == prec && c->g_steps == m) return VDP_OK;
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  VDP_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < m; ++i) {
    cudaError_t e = launch_round(c, prec, c->cap);
    if (e != cudaSuccess) {
      cudaGraph_t junk;
      cudaStreamEndCapture(c->cap, &junk);
      if (junk) cudaGraphDestroy(junk);
      return cuda_fail(e, "sweep launch (capture)");
    }
  }
  VDP_CK(cudaStreamEndCapture(c->cap, &g));
  cudaError_t e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  c->g_prec = prec;
  c->g_steps = m;
  return VDP_OK;
}

// The device-side loop: a graph whose WHILE node repeats kWhileRounds rounds and a condition
// kernel until the instance is done (or a round bound is reached), so a whole solve is one
// graph launch -- no host polling between rounds and at most kWhileRounds - 1 idle rounds at
// the end.  Returns false (and remembers it) if the driver cannot build such a graph; the
// solve then uses the polling schedule.
constexpr int kWhileRounds = 2;

bool ensure_while_graph(vdp_ctx* c, int prec) {
  if (c->w_failed) return false;
  if (c->wexec && c->w_prec == prec) return true;
  if (c->wexec) {
    cudaGraphExecDestroy(c->wexec);
    c->wexec = nullptr;
  }
  if (!c->d_rounds && cudaMalloc((void**)&c->d_rounds, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    c->d_rounds = nullptr;
    c->w_failed = true;
    return false;
  }
  const int k = c->opts.precond == VDP_PRECOND_CHEB ? std::max(1, c->opts.cheb_degree) : 1;
  const long long bound = (2LL * (k + 1) * c->opts.max_iter + 4096) / kWhileRounds + 1;
  const unsigned max_loops = (unsigned)std::min<long long>(bound, 0x7fffffffLL);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle h = 0;
  ok = ok && cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  ok = ok && cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      cudaError_t e = cudaSuccess;
      for (int i = 0; i < kWhileRounds && e == cudaSuccess; ++i) e = launch_round(c, prec, c->cap);
      if (e == cudaSuccess) e = launch_continue(c->st, h, c->d_rounds, max_loops, c->cap);
      cudaGraph_t out = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(c->cap, &out);
      ok = e == cudaSuccess && e2 == cudaSuccess;
    }
  }
  ok = ok && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();  // clear the error: this schedule is optional
    if (exec) cudaGraphExecDestroy(exec);
    c->w_failed = true;
    return false;
  }
  c->wexec = exec;
  c->w_prec = prec;
  return true;
}

int ensure_scaled(vdp_ctx* c, int prec) {
  if (c->scaled_prec == prec) return VDP_OK;
  VDP_CK(launch_scaled(prec, c->bx, c->by, c->bz, c->sinv, c->nx, c->ny, c->nz, c->sx, c->sy,
                       c->sz, c->sd, c->stream));
  c->scaled_prec = prec;
  return VDP_OK;
}

int ensure_spectral(vdp_ctx* c) {
  if (!spectral_supported(spectral_nx(c), c->ny, c->nz)) return VDP_EINVAL;
  if (c->spec && c->sptab && c->za) return VDP_OK;
  static std::mutex mu;
  static std::vector<int> uploaded;  // devices whose register-DFT roots are in place
  {
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(uploaded.begin(), uploaded.end(), c->device) == uploaded.end()) {
      VDP_CK(spectral_upload_roots());
      uploaded.push_back(c->device);
    }
  }
  std::vector<float> tab;
  spectral_tables(spectral_nx(c), c->ny, c->nz, c->Lx / c->nx, c->Ly / c->ny, c->Lz / c->nz, tab);
  const size_t spec_bytes =
      sizeof(float2) * (size_t)spectral_pitch(spectral_nx(c)) * c->ny * c->nz;
  cudaError_t e = cudaSuccess;
  if (!c->za) e = cudaMalloc(&c->za, sizeof(double) * (size_t)c->n);
  if (e == cudaSuccess && !c->spec) e = cudaMalloc((void**)&c->spec, spec_bytes);
  if (e == cudaSuccess && !c->omega) e = cudaMalloc((void**)&c->omega, sizeof(float) * (size_t)c->n);
  if (e == cudaSuccess && !c->sptab) e = cudaMalloc((void**)&c->sptab, sizeof(float) * tab.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(c->sptab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    for (void** b : {(void**)&c->spec, (void**)&c->omega, (void**)&c->sptab}) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    return cuda_fail(e, "spectral buffers");
  }
  c->omega_valid = false;
  return VDP_OK;
}

void solve_spec_args(const vdp_ctx* c, int prec, SpecArgs* a) {
  const int nxt = spectral_nx(c);  // x transform length (twice the cells in the duct)
  const int m = nxt / 2;
  const bool fixed = c->opts.method == VDP_METHOD_FIXED_POINT;
  a->in = c->r;
  // CG: z = W (-L_h)^-1 W rt, W = D^1/2.  Fixed point: with rt = D^-1/2 r the input weight
  // rho D^1/2 gives rho r, and z = damping D^1/2 (-L_h)^-1 (rho r) is the scaled form of the
  // paper's update p += damping L_h^-1 (rho r) (applied as p -= D^-1/2 x, x the sum of the z)
  a->out = c->za;
  a->out_f32 = fixed ? 1 : 0;  // the fixed-point sweep reads z as FP32
  a->omega_in = fixed ? c->rho_w : c->omega;
  a->omega_out = c->omega;
  a->spec = c->spec;
  a->tw = reinterpret_cast<const float2*>(c->sptab);
  a->lam = c->sptab + 2 * (2 * m + 1 + c->ny + c->nz);
  a->nx = nxt;
  a->ny = c->ny;
  a->nz = c->nz;
  a->nxp = spectral_pitch(nxt);
  a->nxd = c->nx;
  a->mirror = c->bc_x == VDP_BC_DUCT;
  a->ewt = a->mirror ? 0.5f : 1.f;
  a->scale = (float)((fixed ? c->opts.damping : 1.0) / ((double)nxt * c->ny * c->nz));
  a->st = c->st;
  a->I = c->desc;
  a->zunits = spectral_units(nxt, c->ny, c->nz);
  a->z0 = 0;
  a->z1 = c->nz;
  a->xunits = spectral_xinv_units(prec, *a, c->nz);
}

int spec_slab(const vdp_ctx* c) {
  return spectral_slab_planes(spectral_nx(c), c->ny, c->nz, c->opts.spec_slab);
}

int ensure_mg(vdp_ctx* c) {
  if (!mg_supported(c->nx, c->ny, c->nz)) return VDP_EINVAL;
  cudaError_t e = cudaSuccess;
  if (!c->za) e = cudaMalloc(&c->za, sizeof(double) * (size_t)c->n);
  if (e == cudaSuccess && !c->omega) {
    e = cudaMalloc((void**)&c->omega, sizeof(float) * (size_t)c->n);
    c->omega_valid = false;
  }
  if (e == cudaSuccess && !c->mg) {
    MgHier* h = new MgHier();
    e = mg_alloc(h, c->nx, c->ny, c->nz, c->bc_x == VDP_BC_DUCT);
    if (e == cudaSuccess) {
      c->mg = h;
      c->mg_valid = false;
    } else {
      delete h;
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "multigrid buffers");
  return VDP_OK;
}

int precond_launches(const vdp_ctx* c) {
  if (c->hdesc.pc == PC_MG) return c->mg ? mg_launches(*c->mg, c->opts.precision) : 0;
  return c->hdesc.pc >= PC_SPECTRAL ? SPEC_PASSES : 0;
}

int prepare_spectral_solve(vdp_ctx* c) {
  if (c->hdesc.pc < PC_SPECTRAL) return VDP_OK;
  if (c->hdesc.pc == PC_MG) {
    if (!c->mg) return VDP_EINVAL;
    if (!c->omega_valid) {
      VDP_CK(launch_omega(c->sinv, c->n, c->omega, c->stream));
      c->omega_valid = true;
    }
    if (!c->mg_valid) {
      VDP_CK(mg_setup(c->mg, c->bx, c->by, c->bz, c->sinv, c->stream));
      c->mg_valid = true;
    }
    return VDP_OK;
  }
  if (c->hdesc.pc == PC_FIXED && !c->rho_w_valid) return VDP_EINVAL;
  if (!c->omega_valid) {
    VDP_CK(launch_omega(c->sinv, c->n, c->omega, c->stream));
    c->omega_valid = true;
  }
  return VDP_OK;
}

}  // namespace vdp

extern "C" {

int vdp_create(int nx, int ny, int nz, double L, vdp_ctx** out) {
  return vdp_create_bc(nx, ny, nz, L, L, L, VDP_BC_PERIODIC, out);
}

int vdp_create_bc(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                  vdp_ctx** out) {
  if (!out) return VDP_EINVAL;
  *out = nullptr;
  auto ok = [](double v) { return v > 0.0 && std::isfinite(v); };
  if (nx < 8 || nx % 8 != 0 || ny < 1 || nz < 1 || !ok(Lx) || !ok(Ly) || !ok(Lz) ||
      (bc_x != VDP_BC_PERIODIC && bc_x != VDP_BC_DUCT))
    return VDP_EINVAL;
  if ((long long)nx * ny * nz > (1LL << 34)) return VDP_EINVAL;
  vdp_ctx* c = new (std::nothrow) vdp_ctx();
  if (!c) return VDP_ENOMEM;
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->Lx = Lx;
  c->Ly = Ly;
  c->Lz = Lz;
  c->bc_x = bc_x;
  c->n = (long long)nx * ny * nz;
  vdp_default_options(&c->opts);
  cudaGetDevice(&c->device);
  size_t bytes = sizeof(double) * (size_t)c->n;
  size_t maxunits = (size_t)std::max(ny * (size_t)nz, (size_t)kSMs * 16);
  cudaError_t e = cudaSuccess;
  double** f64[] = {&c->bx, &c->by, &c->bz, &c->sinv, &c->dg, &c->f0};
  for (double** b : f64)
    if (e == cudaSuccess) e = cudaMalloc((void**)b, bytes);
  // (the Chebyshev buffers za, zb, dch are allocated by vdp_set_options when that
  // preconditioner is first selected)
  void** vv[] = {&c->sx, &c->sy, &c->sz, &c->x, &c->r, &c->d0, &c->d1, &c->q};
  if (e == cudaSuccess) e = cudaMalloc(&c->sd, sizeof(uint16_t) * (size_t)c->n);
  for (void** b : vv)
    if (e == cudaSuccess) e = cudaMalloc(b, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->part, sizeof(double) * kSlots * maxunits);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ticket, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->st, sizeof(InstState));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->desc, sizeof(InstDesc));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->units, sizeof(UnitRef) * (maxunits + kSMs * 8));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->hstate, 2 * sizeof(InstState));
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->evs[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->evs[1], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemset(c->ticket, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    int s = cuda_fail(e, "vdp_create");
    free_ctx(c);
    return s;
  }
  std::memset(c->hstate, 0, 2 * sizeof(InstState));
  Layout lay;
  if (choose_layout(c, c->opts.precision, &lay) != VDP_OK) {  // rows too long for any stage
    free_ctx(c);
    return VDP_EINVAL;
  }
  *out = c;
  return VDP_OK;
}

void vdp_destroy(vdp_ctx* c) { free_ctx(c); }

int vdp_set_options(vdp_ctx* c, const vdp_opts* o) {
  if (!c || !o) return VDP_EINVAL;
  if (o->precision < VDP_FP64 || o->precision > VDP_MIXED_BF16) return VDP_EINVAL;
  if (o->max_iter < 1 || !(o->inner_tol > 0.0 && o->inner_tol < 1.0)) return VDP_EINVAL;
  if (o->precond != VDP_PRECOND_JACOBI && o->precond != VDP_PRECOND_CHEB &&
      o->precond != VDP_PRECOND_SPECTRAL && o->precond != VDP_PRECOND_MG)
    return VDP_EINVAL;
  if (o->precond == VDP_PRECOND_MG && o->method == VDP_METHOD_CG &&
      (o->stencil != 0 || !mg_supported(c->nx, c->ny, c->nz)))
    return VDP_EINVAL;
  if (o->precond == VDP_PRECOND_SPECTRAL &&
      (o->stencil != 0 || !spectral_supported(spectral_nx(c), c->ny, c->nz)))
    return VDP_EINVAL;
  if (o->method != VDP_METHOD_CG && o->method != VDP_METHOD_FIXED_POINT) return VDP_EINVAL;
  if (o->method == VDP_METHOD_FIXED_POINT &&
      (o->stencil != 0 || !spectral_supported(spectral_nx(c), c->ny, c->nz) || !(o->damping > 0.0) ||
       o->damping > 2.0))
    return VDP_EINVAL;
  if (o->precond == VDP_PRECOND_CHEB && (o->cheb_degree < 1 || o->cheb_degree > 16 || o->stencil != 0))
    return VDP_EINVAL;
  if (o->tile_y < 0 || o->units < 0 || o->stages < 0 || o->threads < 0 || o->steps_per_sync < 0 ||
      o->stencil < 0 || o->stencil > 1 || o->spec_slab < 0)
    return VDP_EINVAL;
  if (o->units > 152 * 16 || o->stages > kMaxStages || (o->stages > 0 && o->stages < 4))
    return VDP_EINVAL;
  vdp_opts old = c->opts;
  c->opts = *o;
  Layout lay;
  if (choose_layout(c, o->precision, &lay) != VDP_OK) {
    c->opts = old;
    return VDP_EINVAL;
  }
  if (o->precond == VDP_PRECOND_CHEB && o->cheb_degree > 1 && !(c->za && c->zb && c->dch)) {
    const size_t bytes = sizeof(double) * (size_t)c->n;
    cudaError_t e = cudaSuccess;
    for (void** b : {&c->za, &c->zb, &c->dch})
      if (e == cudaSuccess && !*b) e = cudaMalloc(b, bytes);
    if (e != cudaSuccess) {  // keep what other options use; za is shared with the spectral path
      for (void** b : {&c->zb, &c->dch}) {
        if (*b) cudaFree(*b);
        *b = nullptr;
      }
      c->opts = old;
      return cuda_fail(e, "vdp_set_options (Chebyshev buffers)");
    }
  }
  if (o->precond == VDP_PRECOND_SPECTRAL || o->method == VDP_METHOD_FIXED_POINT) {
    const int sres = ensure_spectral(c);
    if (sres != VDP_OK) {
      c->opts = old;
      return sres;
    }
  }
  if (o->precond == VDP_PRECOND_MG && o->method == VDP_METHOD_CG) {
    const int mres = ensure_mg(c);
    if (mres != VDP_OK) {
      c->opts = old;
      return mres;
    }
  }
  if (o->method == VDP_METHOD_FIXED_POINT && !c->rho_w) {
    cudaError_t e = cudaMalloc((void**)&c->rho_w, sizeof(float) * (size_t)c->n);
    if (e != cudaSuccess) {
      c->rho_w = nullptr;
      c->opts = old;
      return cuda_fail(e, "vdp_set_options (density weight)");
    }
    c->rho_w_valid = false;
  }
  c->stream = (cudaStream_t)o->stream;
  c->layout_dirty = true;
  return VDP_OK;
}

int vdp_get_options(const vdp_ctx* c, vdp_opts* o) {
  if (!c || !o) return VDP_EINVAL;
  *o = c->opts;
  return VDP_OK;
}

int vdp_set_density(vdp_ctx* c, const double* rho) {
  if (!c || !rho) return VDP_EINVAL;
  const double* src = rho;
  size_t bytes = sizeof(double) * (size_t)c->n;
  if (!is_device_ptr(rho)) {
    if (!c->stage_a) VDP_CK(cudaMalloc((void**)&c->stage_a, bytes));
    VDP_CK(cudaMemcpyAsync(c->stage_a, rho, bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->stage_a;
  }
  VDP_CK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  VDP_CK(launch_check_density(src, c->n, c->flag, c->stream));
  int bad = 0;
  VDP_CK(cudaMemcpyAsync(&bad, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VDP_CK(cudaStreamSynchronize(c->stream));
  if (bad) return VDP_EDENSITY;
  VDP_CK(launch_build_coefficients(src, c->nx, c->ny, c->nz, c->Lx / c->nx, c->Ly / c->ny,
                                   c->Lz / c->nz, c->bc_x == VDP_BC_DUCT, c->bx, c->by, c->bz,
                                   c->sinv, c->dg, c->stream));
  c->scaled_prec = -1;
  c->omega_valid = false;
  c->rho_w_valid = false;
  c->mg_valid = false;
  if (c->rho_w) {  // the fixed-point iteration's weight needs rho itself
    VDP_CK(launch_rho_weight(src, c->sinv, c->n, c->rho_w, c->stream));
    c->rho_w_valid = true;
  }
  int s = ensure_scaled(c, c->opts.precision);
  if (s != VDP_OK) return s;
  VDP_CK(cudaStreamSynchronize(c->stream));
  c->has_density = true;
  return VDP_OK;
}

int vdp_solve(vdp_ctx* c, const double* rhs, double* p, double tol) {
  if (!c || !rhs || !p || !(tol > 0.0) || !std::isfinite(tol)) return VDP_EINVAL;
  if (!c->has_density) return VDP_EINVAL;
  const int prec = c->opts.precision;
  size_t bytes = sizeof(double) * (size_t)c->n;
  const bool host_rhs = !is_device_ptr(rhs), host_p = !is_device_ptr(p);
  if ((!host_rhs && ((uintptr_t)rhs & 15)) || (!host_p && ((uintptr_t)p & 15))) return VDP_EINVAL;
  int s;
  if ((s = ensure_scaled(c, prec)) != VDP_OK) return s;
  if ((c->layout_dirty || c->layout_prec != prec) && (s = configure_layout(c, prec)) != VDP_OK)
    return s;
  const bool dev_loop = c->opts.steps_per_sync == 0 && ensure_while_graph(c, prec);
  if (!dev_loop && (s = ensure_graph(c, prec)) != VDP_OK) return s;
  if ((s = prepare_spectral_solve(c)) != VDP_OK) return s;
  const double* drhs = rhs;
  double* dp = p;
  if (host_rhs) {
    if (!c->stage_a) VDP_CK(cudaMalloc((void**)&c->stage_a, bytes));
    VDP_CK(cudaMemcpyAsync(c->stage_a, rhs, bytes, cudaMemcpyHostToDevice, c->stream));
    drhs = c->stage_a;
  }
  if (host_p) {
    if (!c->stage_b) VDP_CK(cudaMalloc((void**)&c->stage_b, bytes));
    if (c->opts.use_guess)
      VDP_CK(cudaMemcpyAsync(c->stage_b, p, bytes, cudaMemcpyHostToDevice, c->stream));
    dp = c->stage_b;
  }
  VDP_CK(cudaEventRecord(c->ev0, c->stream));
  VDP_CK(launch_init(c->desc, drhs, dp, tol, c->opts.inner_tol, c->opts.max_iter,
                     c->opts.max_iter, c->opts.use_guess ? 1 : 0, prec, c->stream));
  const int per_round = (c->lay.mode == 0 ? 3 : 2) + precond_launches(c);
  if (dev_loop) {  // the whole solve is one graph launch; the device decides when to stop
    VDP_CK(cudaMemsetAsync(c->d_rounds, 0, sizeof(unsigned), c->stream));
    VDP_CK(cudaGraphLaunch(c->wexec, c->stream));
    VDP_CK(cudaMemcpyAsync(&c->hstate[0], c->st, sizeof(InstState), cudaMemcpyDeviceToHost,
                           c->stream));
    VDP_CK(cudaEventRecord(c->ev1, c->stream));
    if (host_p) VDP_CK(cudaMemcpyAsync(p, dp, bytes, cudaMemcpyDeviceToHost, c->stream));
    unsigned loops = 0;  // on the solver's stream: solves on other streams are not waited for
    VDP_CK(cudaMemcpyAsync(&loops, c->d_rounds, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    VDP_CK(cudaStreamSynchronize(c->stream));
    const InstState& hs = c->hstate[0];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->stats.status = hs.phase >= PH_DONE ? hs.status : VDP_ETIMEOUT;
    c->stats.iters = hs.iters;
    c->stats.outer_iters = hs.outer;
    c->stats.rel_res = hs.rel_res;
    c->stats.rhs_mean = hs.mu_f;
    c->stats.ms = ms;
    c->stats.sweeps = hs.sweeps;
    c->stats.launches = (int)(1 + (long long)loops * (per_round * kWhileRounds + 1));
    return c->stats.status;
  }
  // Polling schedule: graphs of m rounds, two in flight, the host checks the state after each.
  // Upper bound on launch pairs: one per inner iteration plus the outer phases; the state
  // machine itself stops at max_iter, this only guards the host loop.
  const long long max_pairs = 2LL * c->opts.max_iter + 4096;
  const int m = c->g_steps;
  const long long max_graphs = (max_pairs + m - 1) / m;
  long long issued = 0, checked = 0;
  bool done = false;
  auto issue = [&]() -> int {
    VDP_CK(cudaGraphLaunch(c->gexec, c->stream));
    VDP_CK(cudaMemcpyAsync(&c->hstate[issued & 1], c->st, sizeof(InstState),
                           cudaMemcpyDeviceToHost, c->stream));
    VDP_CK(cudaEventRecord(c->evs[issued & 1], c->stream));
    ++issued;
    return VDP_OK;
  };
  if ((s = issue()) != VDP_OK) return s;
  while (!done) {
    if (issued < max_graphs && (s = issue()) != VDP_OK) return s;
    VDP_CK(cudaEventSynchronize(c->evs[checked & 1]));
    if (c->hstate[checked & 1].phase >= PH_DONE) done = true;
    ++checked;
    if (!done && checked == issued) break;
  }
  VDP_CK(cudaEventRecord(c->ev1, c->stream));
  if (host_p) VDP_CK(cudaMemcpyAsync(p, dp, bytes, cudaMemcpyDeviceToHost, c->stream));
  VDP_CK(cudaStreamSynchronize(c->stream));
  const InstState& hs = c->hstate[(checked - 1) & 1];
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->stats.status = done ? hs.status : VDP_ETIMEOUT;
  c->stats.iters = hs.iters;
  c->stats.outer_iters = hs.outer;
  c->stats.rel_res = hs.rel_res;
  c->stats.rhs_mean = hs.mu_f;
  c->stats.ms = ms;
  c->stats.sweeps = hs.sweeps;
  c->stats.launches = (int)(1 + issued * per_round * m);
  return c->stats.status;
}

int vdp_get_stats(const vdp_ctx* c, vdp_stats* s) {
  if (!c || !s) return VDP_EINVAL;
  *s = c->stats;
  return VDP_OK;
}

int vdp_spectral_slabs(const vdp_ctx* c) {
  if (!c || !(c->opts.precond == VDP_PRECOND_SPECTRAL || c->opts.method == VDP_METHOD_FIXED_POINT))
    return 0;
  const int slab = spec_slab(c);
  return slab > 0 ? (c->nz + slab - 1) / slab : 0;
}

int vdp_inverse_laplacian(vdp_ctx* c, const double* g, double* out) {
  if (!c || !g || !out || g == out) return VDP_EINVAL;
  if (!is_device_ptr(g) || !is_device_ptr(out) || ((uintptr_t)g & 15) || ((uintptr_t)out & 15))
    return VDP_EINVAL;
  int s;
  if ((s = ensure_spectral(c)) != VDP_OK) return s;
  SpecArgs a;
  solve_spec_args(c, PREC_FP64, &a);
  a.in = g;
  a.out = out;
  a.out_f32 = 0;
  a.omega_in = nullptr;
  a.omega_out = nullptr;
  a.scale = (float)(-1.0 / ((double)a.nx * c->ny * c->nz));  // L_h^-1, not (-L_h)^-1
  a.st = nullptr;
  a.I = nullptr;
  VDP_CK(launch_spectral_apply(PREC_FP64, a, spec_slab(c), c->stream));
  VDP_CK(cudaStreamSynchronize(c->stream));
  return VDP_OK;
}

int vdp_mg_levels(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1) return 0;
  int d[kMgMaxLevels][3];
  return mg_level_dims(nx, ny, nz, d);
}

int vdp_mg_apply(vdp_ctx* c, const double* g, double* out) {
  if (!c || !g || !out || g == out || !c->has_density) return VDP_EINVAL;
  if (!is_device_ptr(g) || !is_device_ptr(out) || ((uintptr_t)g & 15) || ((uintptr_t)out & 15))
    return VDP_EINVAL;
  int s;
  if ((s = ensure_mg(c)) != VDP_OK) return s;
  if (!c->omega_valid) {
    VDP_CK(launch_omega(c->sinv, c->n, c->omega, c->stream));
    c->omega_valid = true;
  }
  if (!c->mg_valid) {
    VDP_CK(mg_setup(c->mg, c->bx, c->by, c->bz, c->sinv, c->stream));
    c->mg_valid = true;
  }
  // the cycle works in the solve's scaled variables: M g = D^-1/2 (W M W) (D^-1/2 g)
  double* rt = static_cast<double*>(c->d0);  // FP64-sized work vectors of the context
  double* z = static_cast<double*>(c->d1);
  VDP_CK(launch_mg_scale(g, c->sinv, c->n, rt, c->stream));
  const MgArgs a{rt, z, c->omega, nullptr, nullptr};
  VDP_CK(launch_mg_vcycle(*c->mg, PREC_FP64, a, c->stream));
  VDP_CK(launch_mg_scale(z, c->sinv, c->n, out, c->stream));
  VDP_CK(cudaStreamSynchronize(c->stream));
  return VDP_OK;
}

int vdp_apply(vdp_ctx* c, const double* p, double* out) {
  if (!c || !p || !out || p == out) return VDP_EINVAL;
  if (!c->has_density) return VDP_EINVAL;
  size_t bytes = sizeof(double) * (size_t)c->n;
  const bool hp = !is_device_ptr(p), ho = !is_device_ptr(out);
  const double* dp = p;
  double* dout = out;
  if (hp) {
    if (!c->stage_a) VDP_CK(cudaMalloc((void**)&c->stage_a, bytes));
    VDP_CK(cudaMemcpyAsync(c->stage_a, p, bytes, cudaMemcpyHostToDevice, c->stream));
    dp = c->stage_a;
  }
  if (ho) {
    if (!c->stage_b) VDP_CK(cudaMalloc((void**)&c->stage_b, bytes));
    dout = c->stage_b;
  }
  VDP_CK(launch_apply(c->bx, c->by, c->bz, dp, c->nx, c->ny, c->nz, dout, c->stream));
  if (ho) VDP_CK(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, c->stream));
  VDP_CK(cudaStreamSynchronize(c->stream));
  return VDP_OK;
}

}  // extern "C"
