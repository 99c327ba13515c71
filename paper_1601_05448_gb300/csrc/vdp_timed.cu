// vdp_timed.cu -- vdp_solve_timed: a solve whose kernel launches are timed one by one.
//
// The graph-driven solve (vdp_api.cu) launches fixed (residual, stencil, flat) triples and lets
// the per-instance state machine decide which launch works and which returns at once.  Here the
// host reads the state before every launch and issues only the kernel that advances the current
// phase; the kernels and the units they cover are the same, so the arithmetic (and the result) is
// the same, launch by launch.  Each kernel kind is captured once into a three-node graph
// (event record, kernel, event record) so that the two timestamps bracket the kernel alone: with
// separate stream calls the first event would fire on an idle stream before the host had even
// submitted the kernel, and the submission latency would be counted as kernel time.
#include <cuda_runtime.h>

#include <vector>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "vdp.h"
#include "vdp_ctx.h"
#include "vdp_internal.cuh"
#include "vdp_launch.h"
#include "vdp_spectral.h"

using namespace vdp;

namespace {

int sweep_kind(int phase) {
  switch (phase) {
    case PH_RES64: return VDP_SWEEP_RES64;
    case PH_STENCIL: return VDP_SWEEP_STENCIL;
    case PH_CHEB: return VDP_SWEEP_CHEB;
    case PH_UPDATE: return VDP_SWEEP_UPDATE;
    default: return VDP_SWEEP_OTHER;  // PH_MEANF, PH_CORRECT, PH_FINAL
  }
}

// Launch the one kernel that advances `phase` (the same kernels and unit lists that the
// graph-driven solve launches) on stream `s`.
cudaError_t launch_for_phase(vdp_ctx* c, int prec, int phase, cudaStream_t s) {
  const Layout& l = c->lay;
  switch (phase) {
    case PH_RES64:
      if (l.mode == 0) return launch_res64(prec, c->desc, c->units, l.nunits, l.threads, s);
      return launch_stencil(prec, l.mode, 0, c->desc, c->units, l.nunits, l.threads, l.smem, s);
    case PH_STENCIL:
    case PH_CHEB:
      return launch_stencil(prec, l.mode, stencil_kind(c->hdesc.pc), c->desc, c->units, l.nunits,
                            l.threads, l.smem, s);
    default:
      return launch_flat(prec, c->desc, c->units + l.nunits, l.nunits_f, s);
  }
}

// The three launch shapes: residual kernel, stencil kernel, flat kernel.
int launch_shape(int phase) {
  switch (phase) {
    case PH_RES64: return 0;
    case PH_STENCIL:
    case PH_CHEB: return 1;
    default: return 2;
  }
}

// graph 3: one whole multigrid V-cycle; the spectral launches of one application (X+ and Y+
// slab by slab, Z, Y- and X- slab by slab) have a graph each in TimedGraphs::spec
constexpr int kTimedGraphs = 4;
constexpr int kMgGraph = 3;
constexpr int kMgPass = 1000;  // capture_timed: the V-cycle instead of a spectral pass
constexpr int kSpecKind[SPEC_PASSES] = {VDP_SWEEP_SPEC_X, VDP_SWEEP_SPEC_Y, VDP_SWEEP_SPEC_Z,
                                        VDP_SWEEP_SPEC_Y, VDP_SWEEP_SPEC_X};

struct TimedGraphs {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraphExec_t g[kTimedGraphs] = {};
  std::vector<cudaGraphExec_t> spec;
  std::vector<SpecLaunch> sched;
  ~TimedGraphs() {
    for (auto& x : g)
      if (x) cudaGraphExecDestroy(x);
    for (auto& x : spec)
      if (x) cudaGraphExecDestroy(x);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// spec_launch >= 0: that launch of the spectral schedule instead of the phase's kernel
cudaError_t capture_timed(vdp_ctx* c, int prec, int phase, int spec_launch, TimedGraphs& t,
                          cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e2 = cudaEventRecordWithFlags(t.e0, c->cap, cudaEventRecordExternal);
  if (e2 == cudaSuccess) {
    if (spec_launch == kMgPass) {
      const MgArgs a{c->r, c->za, c->omega, c->st, c->desc};
      e2 = launch_mg_vcycle(*c->mg, prec, a, c->cap);
    } else if (spec_launch >= 0) {
      SpecArgs a;
      solve_spec_args(c, prec, &a);
      const SpecLaunch& l = t.sched[spec_launch];
      e2 = launch_spectral_pass(prec, l.pass, spectral_launch_args(prec, a, l, spec_slab(c)), c->cap);
    } else {
      e2 = launch_for_phase(c, prec, phase, c->cap);
    }
  }
  if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(t.e1, c->cap, cudaEventRecordExternal);
  e = cudaStreamEndCapture(c->cap, &g);
  if (e2 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e2 != cudaSuccess ? e2 : e;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

}  // namespace

extern "C" int vdp_solve_timed(vdp_ctx* c, const double* rhs, double* p, double tol,
                               vdp_sweep_times* times) {
  if (!c || !rhs || !p || !times || !(tol > 0.0) || !std::isfinite(tol)) return VDP_EINVAL;
  if (!c->has_density) return VDP_EINVAL;
  if (!is_device_ptr(rhs) || !is_device_ptr(p) || ((uintptr_t)rhs & 15) || ((uintptr_t)p & 15))
    return VDP_EINVAL;
  std::memset(times, 0, sizeof(*times));
  const int prec = c->opts.precision;
  int s;
  if ((s = ensure_scaled(c, prec)) != VDP_OK) return s;
  if ((c->layout_dirty || c->layout_prec != prec) && (s = configure_layout(c, prec)) != VDP_OK)
    return s;
  TimedGraphs t;
  VDP_CK(cudaEventCreate(&t.e0));
  VDP_CK(cudaEventCreate(&t.e1));
  const int shape_phase[3] = {PH_RES64, PH_STENCIL, PH_UPDATE};
  for (int i = 0; i < 3; ++i) VDP_CK(capture_timed(c, prec, shape_phase[i], -1, t, &t.g[i]));
  const bool mg = c->hdesc.pc == PC_MG;
  const bool spectral = c->hdesc.pc >= PC_SPECTRAL && !mg;
  if (spectral || mg) {
    if ((s = prepare_spectral_solve(c)) != VDP_OK) return s;
  }
  if (spectral) {
    spectral_schedule(c->nz, spec_slab(c), t.sched);
    t.spec.assign(t.sched.size(), nullptr);
    for (size_t i = 0; i < t.sched.size(); ++i)
      VDP_CK(capture_timed(c, prec, PH_SPEC, (int)i, t, &t.spec[i]));
  }
  if (mg) VDP_CK(capture_timed(c, prec, PH_SPEC, kMgPass, t, &t.g[kMgGraph]));
  auto fail = [&](cudaError_t e, const char* where) { return cuda_fail(e, where); };
  cudaError_t e;
  if ((e = cudaEventRecord(c->ev0, c->stream)) != cudaSuccess) return fail(e, "cudaEventRecord");
  e = launch_init(c->desc, rhs, p, tol, c->opts.inner_tol, c->opts.max_iter, c->opts.max_iter,
                  c->opts.use_guess ? 1 : 0, prec, c->stream);
  if (e != cudaSuccess) return fail(e, "launch_init");
  // Every launch advances the state machine by one phase; this only bounds the host loop.
  const int k = c->opts.precond == VDP_PRECOND_CHEB ? std::max(1, c->opts.cheb_degree) : 1;
  const long long max_launches = (long long)(k + 1) * c->opts.max_iter + 4096;
  InstState& hs = c->hstate[0];
  bool done = false;
  for (long long i = 0; i < max_launches; ++i) {
    if ((e = cudaMemcpyAsync(&hs, c->st, sizeof(InstState), cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return fail(e, "state read");
    if (hs.phase >= PH_DONE) {
      done = true;
      break;
    }
    const bool spec = spectral && hs.phase == PH_SPEC;
    const bool vcyc = mg && hs.phase == PH_SPEC;
    const int nl = spec ? (int)t.sched.size() : 1;
    for (int l = 0; l < nl; ++l) {
      const int kind = spec ? kSpecKind[t.sched[l].pass] : (vcyc ? VDP_SWEEP_MG : sweep_kind(hs.phase));
      cudaGraphExec_t ge = spec ? t.spec[l] : t.g[vcyc ? kMgGraph : launch_shape(hs.phase)];
      if ((e = cudaGraphLaunch(ge, c->stream)) != cudaSuccess) return fail(e, "sweep launch");
      if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return fail(e, "cudaStreamSynchronize");
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, t.e0, t.e1)) != cudaSuccess)
        return fail(e, "cudaEventElapsedTime");
      times->ms[kind] += ms;
      if (times->launches[kind] == 0 || ms < times->ms_min[kind]) times->ms_min[kind] = ms;
      times->launches[kind] += 1;
    }
  }
  cudaEventRecord(c->ev1, c->stream);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  int launches = 1;
  for (int j = 0; j < VDP_SWEEP_KINDS; ++j) launches += times->launches[j];
  c->stats.status = done ? hs.status : VDP_ETIMEOUT;
  c->stats.iters = hs.iters;
  c->stats.outer_iters = hs.outer;
  c->stats.rel_res = hs.rel_res;
  c->stats.rhs_mean = hs.mu_f;
  c->stats.ms = ms;
  c->stats.sweeps = hs.sweeps;
  c->stats.launches = launches;
  return c->stats.status;
}
