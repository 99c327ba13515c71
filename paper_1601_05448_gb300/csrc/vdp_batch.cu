// vdp_batch.cu -- the batch engine: many independent solves (different grid sizes, density
// fields and tolerances, one precision) advanced together.
//
// Every member keeps its own context (coefficients, Krylov vectors, state, unit layout), so
// its arithmetic -- and its result, bit for bit -- is the same as when it is solved alone with
// vdp_solve.  A run launches either one persistent cooperative kernel that loops over
// (stencil-kind sweep of every member, grid barrier, flat-kind sweep, grid barrier) rounds, or
// the equivalent sequence of ordinary launches; either is captured once into a CUDA graph per
// membership and replayed.  Members can be added and retired between runs (continuous batching):
// the device tables are rebuilt and the graph re-captured only when membership changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vdp.h"
#include "vdp_ctx.h"
#include "vdp_internal.cuh"
#include "vdp_launch.h"
#include "vdp_spectral.h"

using namespace vdp;

namespace {

struct Member {
  vdp_ctx* ctx;
  const double* rhs;
  double* p;
  double tol;
  bool done;
};

}  // namespace

struct vdp_batch {
  int prec = 0;
  int persistent = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  int device = 0;
  std::vector<Member> members;
  std::vector<int> active;      // indices of members in the device tables
  InstDesc* d_desc = nullptr;
  int cap_desc = 0;
  UnitRef* d_units = nullptr;
  long long cap_units = 0;
  int ns = 0, nf = 0;
  InstState* d_states = nullptr;
  InstState* h_states = nullptr;  // pinned
  int cap_states = 0;
  BatchCtl* d_ctl = nullptr;
  BatchCtl* h_ctl = nullptr;      // pinned
  bool dirty = true;
  cudaGraphExec_t gexec = nullptr;
  int g_pairs = 0;
  int grid = 0;
  double wait_limit_s = 2.0;  // bound on each grid barrier wait of the persistent kernel
  bool inject = false;        // next persistent run: one arrival more than the grid (tests)
  bool ctl_stale = false;     // the control words must be reset before the next run
  // graph branches for the members' spectral passes (captured from these streams)
  static constexpr int kBranches = 4;
  cudaStream_t aux[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
};

namespace {

void drop_graph(vdp_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
}

template <class X>
int grow(X** ptr, long long* cap, long long need) {
  if (need <= *cap) return VDP_OK;
  long long nc = std::max(need, *cap * 2);
  X* np = nullptr;
  VDP_CK(cudaMalloc((void**)&np, sizeof(X) * nc));
  if (*ptr) cudaFree(*ptr);
  *ptr = np;
  *cap = nc;
  return VDP_OK;
}

int rebuild(vdp_batch* b) {
  b->active.clear();
  for (size_t i = 0; i < b->members.size(); ++i)
    if (!b->members[i].done) b->active.push_back((int)i);
  const int n = (int)b->active.size();
  long long cd = b->cap_desc;
  int s;
  if ((s = grow(&b->d_desc, &cd, std::max(n, 1))) != VDP_OK) return s;
  b->cap_desc = (int)cd;
  if (n > b->cap_states) {
    if (b->d_states) cudaFree(b->d_states);
    if (b->h_states) cudaFreeHost(b->h_states);
    b->d_states = nullptr;
    b->h_states = nullptr;
    b->cap_states = 0;
    VDP_CK(cudaMalloc((void**)&b->d_states, sizeof(InstState) * n));
    VDP_CK(cudaMallocHost((void**)&b->h_states, sizeof(InstState) * n));
    b->cap_states = n;
  }
  std::vector<InstDesc> desc(n);
  std::vector<UnitRef> su, fu;
  for (int k = 0; k < n; ++k) {
    const Member& m = b->members[b->active[k]];
    InstDesc d = m.ctx->hdesc;
    d.rhs = m.rhs;
    d.p = m.p;
    d.remaining = &b->d_ctl->remaining;
    desc[k] = d;
    for (int u = 0; u < d.nunits; ++u) su.push_back(UnitRef{k, u});
    for (int u = 0; u < d.nunits_f; ++u) fu.push_back(UnitRef{k, u});
  }
  b->ns = (int)su.size();
  b->nf = (int)fu.size();
  if ((s = grow(&b->d_units, &b->cap_units, std::max<long long>(1, b->ns + b->nf))) != VDP_OK)
    return s;
  if (n > 0) {
    VDP_CK(cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice,
                           b->stream));
    VDP_CK(cudaMemcpyAsync(b->d_units, su.data(), sizeof(UnitRef) * b->ns, cudaMemcpyHostToDevice,
                           b->stream));
    VDP_CK(cudaMemcpyAsync(b->d_units + b->ns, fu.data(), sizeof(UnitRef) * b->nf,
                           cudaMemcpyHostToDevice, b->stream));
  }
  BatchCtl ctl{};
  ctl.remaining = n;
  ctl.limit_ns = (unsigned long long)(b->wait_limit_s * 1e9);
  *b->h_ctl = ctl;
  b->ctl_stale = false;
  VDP_CK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, b->stream));
  VDP_CK(cudaStreamSynchronize(b->stream));
  drop_graph(b);
  b->dirty = false;
  return VDP_OK;
}

int capture(vdp_batch* b, int pairs) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  VDP_CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (b->persistent) {
    e = launch_persistent(b->prec, b->d_desc, b->d_units, b->ns, b->d_units + b->ns, b->nf, pairs,
                          b->d_ctl, b->grid, b->cap);
  } else {
    // one stencil kernel for all members: the fixed-point variant if every member uses that
    // method, the variant with Chebyshev sweeps if any member needs it (it also runs the
    // fixed-point sweep), the CG variant otherwise
    int nfixed = 0, ncheb = 0;
    for (int k : b->active) {
      nfixed += b->members[k].ctx->hdesc.pc == PC_FIXED;
      ncheb += b->members[k].ctx->hdesc.pc == PC_CHEB;
    }
    const int kind = nfixed == (int)b->active.size() ? 2 : (ncheb || nfixed) ? 1 : 0;
    for (int i = 0; i < pairs && e == cudaSuccess; ++i) {
      e = launch_res64(b->prec, b->d_desc, b->d_units, b->ns, kDirectThreads, b->cap);
      // members with the spectral passes or the V-cycle: their kernels (each gated on its own
      // member's phase), between the residual and the stencil sweeps as in a solve alone.  The
      // members' chains are independent, so they go to up to four graph branches that the GPU
      // runs concurrently (small grids alone would leave most SMs idle).
      int nspec = 0;
      for (int k : b->active) nspec += b->members[k].ctx->hdesc.pc >= PC_SPECTRAL;
      const int nb = std::min(nspec, (int)vdp_batch::kBranches);
      if (nb > 0 && e == cudaSuccess) e = cudaEventRecord(b->fork, b->cap);
      for (int j = 0; j < nb && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(b->aux[j], b->fork, 0);
      int slot = 0;
      for (size_t k = 0; k < b->active.size() && e == cudaSuccess; ++k) {
        const vdp_ctx* c = b->members[b->active[k]].ctx;
        if (c->hdesc.pc < PC_SPECTRAL) continue;
        cudaStream_t br = b->aux[slot++ % nb];
        if (c->hdesc.pc == PC_MG) {
          const MgArgs a{c->r, c->za, c->omega, c->st, c->desc};
          e = launch_mg_vcycle(*c->mg, b->prec, a, br);
          continue;
        }
        SpecArgs a;
        solve_spec_args(c, b->prec, &a);
        e = launch_spectral_apply(b->prec, a, spec_slab(c), br);
      }
      for (int j = 0; j < nb && e == cudaSuccess; ++j) {
        e = cudaEventRecord(b->join[j], b->aux[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[j], 0);
      }
      if (e == cudaSuccess)
        e = launch_stencil(b->prec, 0, kind, b->d_desc, b->d_units, b->ns, kDirectThreads, 0,
                           b->cap);
      if (e == cudaSuccess) e = launch_flat(b->prec, b->d_desc, b->d_units + b->ns, b->nf, b->cap);
    }
  }
  cudaGraph_t junk = nullptr;
  if (e != cudaSuccess) {
    cudaStreamEndCapture(b->cap, &junk);
    if (junk) cudaGraphDestroy(junk);
    return cuda_fail(e, "batch launch (capture)");
  }
  VDP_CK(cudaStreamEndCapture(b->cap, &g));
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
  b->g_pairs = pairs;
  return VDP_OK;
}

Member* find(vdp_batch* b, vdp_ctx* c, size_t* idx) {
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i].ctx == c) {
      if (idx) *idx = i;
      return &b->members[i];
    }
  return nullptr;
}

}  // namespace

extern "C" {

int vdp_batch_create(int precision, int persistent, void* stream, vdp_batch** out) {
  if (!out) return VDP_EINVAL;
  *out = nullptr;
  if (precision < VDP_FP64 || precision > VDP_MIXED_BF16) return VDP_EINVAL;
  vdp_batch* b = new (std::nothrow) vdp_batch();
  if (!b) return VDP_ENOMEM;
  b->prec = precision;
  b->persistent = persistent ? 1 : 0;
  b->stream = (cudaStream_t)stream;
  cudaGetDevice(&b->device);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int j = 0; j < vdp_batch::kBranches && e == cudaSuccess; ++j) {
    e = cudaStreamCreateWithFlags(&b->aux[j], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = persistent_grid(precision, &b->grid);
  if (e == cudaSuccess && b->grid < 1) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) {
    int s = cuda_fail(e, "vdp_batch_create");
    vdp_batch_destroy(b);
    return s;
  }
  *out = b;
  return VDP_OK;
}

void vdp_batch_destroy(vdp_batch* b) {
  if (!b) return;
  drop_graph(b);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_units) cudaFree(b->d_units);
  if (b->d_states) cudaFree(b->d_states);
  if (b->h_states) cudaFreeHost(b->h_states);
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int j = 0; j < vdp_batch::kBranches; ++j) {
    if (b->aux[j]) cudaStreamDestroy(b->aux[j]);
    if (b->join[j]) cudaEventDestroy(b->join[j]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

int vdp_batch_add(vdp_batch* b, vdp_ctx* c, const double* rhs, double* p, double tol) {
  if (!b || !c || !rhs || !p || !(tol > 0.0)) return VDP_EINVAL;
  if (!c->has_density || c->opts.precision != b->prec || c->opts.stencil != 0) return VDP_EINVAL;
  // the spectral passes and the V-cycle are separate kernels: members with them need the batch
  // of ordinary launches, not the persistent kernel
  if ((c->opts.precond == VDP_PRECOND_SPECTRAL || c->opts.precond == VDP_PRECOND_MG ||
       c->opts.method == VDP_METHOD_FIXED_POINT) &&
      b->persistent)
    return VDP_EINVAL;
  if (!is_device_ptr(rhs) || !is_device_ptr(p) || ((uintptr_t)rhs & 15) || ((uintptr_t)p & 15))
    return VDP_EINVAL;
  if (find(b, c, nullptr)) return VDP_EINVAL;  // already a member
  int s;
  if ((s = ensure_scaled(c, b->prec)) != VDP_OK) return s;
  if ((c->layout_dirty || c->layout_prec != b->prec || !c->hdesc_valid) &&
      (s = configure_layout(c, b->prec)) != VDP_OK)
    return s;
  if ((s = prepare_spectral_solve(c)) != VDP_OK) return s;
  VDP_CK(cudaStreamSynchronize(c->stream));
  VDP_CK(launch_init(c->desc, rhs, p, tol, c->opts.inner_tol, c->opts.max_iter, c->opts.max_iter,
                     c->opts.use_guess ? 1 : 0, b->prec, b->stream));
  b->members.push_back(Member{c, rhs, p, tol, false});
  b->dirty = true;
  return VDP_OK;
}

int vdp_batch_run(vdp_batch* b, int max_pairs, int* active_out) {
  if (!b || max_pairs < 1) return VDP_EINVAL;
  int s;
  if (b->dirty && (s = rebuild(b)) != VDP_OK) return s;
  const int n = (int)b->active.size();
  if (n == 0) {
    if (active_out) *active_out = 0;
    return VDP_OK;
  }
  if (!b->gexec || b->g_pairs != max_pairs) {
    if ((s = capture(b, max_pairs)) != VDP_OK) return s;
  }
  if (b->ctl_stale || b->inject) {  // fresh barrier words (after an expired wait, or to inject)
    BatchCtl ctl{};
    ctl.remaining = n;
    ctl.limit_ns = (unsigned long long)(b->wait_limit_s * 1e9);
    ctl.extra = b->inject ? 1u : 0u;
    *b->h_ctl = ctl;
    VDP_CK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, b->stream));
    b->ctl_stale = b->inject;  // an injected run leaves words to reset
    b->inject = false;
  }
  VDP_CK(cudaGraphLaunch(b->gexec, b->stream));
  VDP_CK(launch_gather(b->d_desc, n, b->d_states, b->stream));
  VDP_CK(cudaMemcpyAsync(b->h_states, b->d_states, sizeof(InstState) * n, cudaMemcpyDeviceToHost,
                         b->stream));
  VDP_CK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream));
  VDP_CK(cudaStreamSynchronize(b->stream));
  int remaining = 0;
  for (int k = 0; k < n; ++k) {
    Member& m = b->members[b->active[k]];
    const InstState& h = b->h_states[k];
    if (h.phase >= PH_DONE) {
      m.done = true;
      b->dirty = true;  // retire it from the device tables at the next run
      vdp_stats& st = m.ctx->stats;
      st.status = h.status;
      st.iters = h.iters;
      st.outer_iters = h.outer;
      st.rel_res = h.rel_res;
      st.rhs_mean = h.mu_f;
      st.ms = 0.0;
      st.sweeps = h.sweeps;
      st.launches = 0;
    } else {
      ++remaining;
    }
  }
  if (active_out) *active_out = remaining;
  if (b->h_ctl->fault) {
    b->ctl_stale = true;  // the members stay usable: their last completed sweeps are consistent
    return VDP_ETIMEOUT;
  }
  return VDP_OK;
}

int vdp_batch_set_wait_limit(vdp_batch* b, double seconds) {
  if (!b || !(seconds > 0.0) || !(seconds <= 60.0)) return VDP_EINVAL;
  b->wait_limit_s = seconds;
  b->ctl_stale = true;
  return VDP_OK;
}

int vdp_batch_inject_lost_arrival(vdp_batch* b) {
  if (!b || !b->persistent) return VDP_EINVAL;
  b->inject = true;
  return VDP_OK;
}

int vdp_batch_done(vdp_batch* b, vdp_ctx* c) {
  if (!b || !c) return -VDP_EINVAL;
  Member* m = find(b, c, nullptr);
  if (!m) return -VDP_EINVAL;
  return m->done ? 1 : 0;
}

int vdp_batch_remove(vdp_batch* b, vdp_ctx* c) {
  if (!b || !c) return VDP_EINVAL;
  size_t i = 0;
  if (!find(b, c, &i)) return VDP_EINVAL;
  if (!b->members[i].done) b->dirty = true;
  b->members.erase(b->members.begin() + (long)i);
  return VDP_OK;
}

int vdp_batch_size(const vdp_batch* b) { return b ? (int)b->members.size() : 0; }

}  // extern "C"
