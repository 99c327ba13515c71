// vdp_device.cuh -- device code shared by the solver's translation units (vdp_kernels.cu and
// vdp_spectral.cu): deterministic partial sums, the last-unit ticket, the phase transitions of
// the per-instance state machine, and the state snapshot.  Internal to libvdp.
#pragma once

#include "vdp_internal.cuh"

namespace vdp {

// Conversions between binary64 and binary32 by repacking the IEEE 754 fields with integer
// operations: on this GPU the conversion instructions run on the FP64 pipe (2 results per clock
// per SM), which FP64 kernels otherwise spend a large share of their time in.
//   to binary32: exponent rebiased (1023 -> 127), the 23 leading fraction bits kept (rounding
//                toward zero), magnitudes below the binary32 normal range flushed to zero and
//                above it (infinities, NaNs) sent to infinity -- adequate for a preconditioner
//                input, which the FP32 transforms round anyway;
//   to binary64: exact for every binary32 normal number and zero (subnormals flush to zero).
__device__ __forceinline__ float narrow(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned bits = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : (sign | ((unsigned)e << 23) | frac));
  return __uint_as_float(bits);
}
__device__ __forceinline__ double widen(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, frac = b & 0x7fffffu;
  const unsigned hi = e == 0 ? sign : (sign | ((e + 1023u - 127u) << 20) | (frac >> 3));
  const unsigned lo = e == 0 ? 0u : (frac << 29);
  return __hiloint2double((int)hi, (int)lo);
}


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- reductions: per-unit partial slots, last unit reduces them in a fixed order --------------

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of NS per-thread partials of type A (float partials stay FP32 within a warp;
// the warp totals are combined in FP64) into slot k of this unit: part[k * nunits + unit].
// Fixed shuffle tree and fixed warp order: deterministic.
template <int NS, class A>
__device__ __forceinline__ void store_partials(const A (&v)[NS], double* part, int nunits,
                                               int unit) {
  __shared__ double red[kMaxThreads / 32][kSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  A w[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) w[k] = warp_sum(v[k]);
  __syncthreads();  // red[] may still be read by a previous use
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) red[warp][k] = (double)w[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double s = lane < nwarps ? red[lane][k] : 0.0;
      s = warp_sum(s);
      if (lane == 0) part[k * nunits + unit] = s;
    }
  }
}

// Returns true in every thread of the unit that arrives last for its instance.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket, int nunits) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // partials of this unit visible before its ticket
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == (unsigned)nunits - 1u);
    if (last) __threadfence();
  }
  __syncthreads();
  return last != 0;
}

// Fixed-order sum of one slot over all units (warp 0; identical result in every lane).
// Fixed-order sum of one slot over all units by the last unit: 64 lanes (warps 0 and 1) each
// add the slots lane, lane + 64, ... in index order with eight loads in flight, then a fixed
// shuffle tree per warp, warp 0's total plus warp 1's.  The order does not depend on the block
// size, so an instance sums identically whatever launch it runs in.  Every thread returns it.
static __device__ __noinline__ double block_sum_slot(const double* part, int nunits) {
  __shared__ double wsum[2];
  constexpr int U = 8, LANES = 64;
  const int t = threadIdx.x;
  double s = 0.0;
  if (t < LANES) {
    for (int i0 = t; i0 < nunits; i0 += U * LANES) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * LANES;
        v[u] = i < nunits ? __ldcg(part + i) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) s += v[u];
    }
    s = warp_sum(s);
  }
  __syncthreads();  // wsum may be in use by a previous call
  if (t == 0 || t == 32) wsum[t >> 5] = s;
  __syncthreads();
  return wsum[0] + wsum[1];
}

// ---- phase transitions (run by thread 0 of the last unit) -------------------------------------

static __device__ void transition(const InstDesc& I, volatile InstState* st, int phase,
                           const double (&S)[kSlots]) {
  st->sweeps += 1;
  if (st->fault && phase != PH_FINAL) {  // a bounded wait expired: stop with what p holds
    st->status = 6;                      // VDP_ETIMEOUT
    st->phase = PH_FINAL;
    return;
  }
  switch (phase) {
    case PH_MEANF:
      st->mu_f = S[0] / (double)I.ncell;
      st->f2 = (double)I.ncell * st->mu_f * st->mu_f;
      st->first_res = 1;
      st->phase = PH_RES64;
      break;
    case PH_RES64: {
      const double rr64 = S[0], rrt = S[1];
      if (st->first_res) st->sum_p = S[2];  // later: summed by the correction sweep
      if (st->first_res) {
        st->fn2 = S[3];
        st->first_res = 0;
      }
      st->outer += 1;
      const double fn2 = st->fn2;
      if (fn2 <= 1e-28 * st->f2) {  // f is constant up to the rounding of its mean: p = 0
        st->zero_sol = 1;
        st->rel_res = 0.0;
        st->phase = PH_FINAL;
        break;
      }
      const double rel = sqrt(rr64 / fn2);
      st->rel_res = rel;
      if (!isfinite(rel)) {
        st->status = 5;  // VDP_EBREAKDOWN
        st->phase = PH_FINAL;
      } else if (rel <= st->tol) {
        st->phase = PH_FINAL;
      } else if (st->iters >= st->max_iter) {
        st->status = 4;  // VDP_ENOTCONV
        st->phase = PH_FINAL;
      } else if (rrt == 0.0) {  // residual below the inner type's range: cannot refine further
        st->status = 4;
        st->phase = PH_FINAL;
      } else if (I.pc == PC_FIXED && rel > 1e4) {  // the paper's iteration is diverging (the
        st->status = 4;                              // density varies too much for it)
        st->phase = PH_FINAL;
      } else {
        // How far the FP64 residual fell during the last inner solve compared with the scaled
        // inner residual; the next inner target is tightened by it (at least 1).
        if (st->outer > 1 && st->inner_ratio > 0.0) {
          const double obs = sqrt(rr64 / st->rr64_prev) / st->inner_ratio;
          st->eta = fmax(1.0, fmin(obs, 1e6));
        }
        double tau = 0.5 * st->tol * sqrt(fn2 / rr64) / st->eta;
        if (st->precision != PREC_FP64) tau = fmax(tau, st->inner_tol);
        tau = fmin(tau, 0.5);
        st->tau2 = tau * tau;
        st->rr64_prev = rr64;
        st->rr = rrt;
        st->rr0 = rrt;
        st->rz = rrt;
        st->beta = 0.0;
        st->inner_iters = 0;
        st->cheb_j = 1;
        st->phase = I.pc == PC_CHEB ? PH_CHEB : (I.pc >= PC_SPECTRAL ? PH_SPEC : PH_STENCIL);
      }
      st->rr64 = rr64;
      break;
    }
    case PH_STENCIL: {
      const double dq = S[0];
      if (I.pc == PC_FIXED) {
        // the paper's iteration: the stencil sweep has also applied the update x += z,
        // rt -= At z and summed <rt, rt> (S[0]); continue as after an update sweep
        phase = PH_UPDATE;
        goto after_update;
      } else if (dq > 0.0 && isfinite(dq)) {
        st->alpha = (I.pc != PC_JACOBI ? st->rz : st->rr) / dq;
        st->phase = PH_UPDATE;
      } else if (st->inner_iters > 0) {
        // loss of curvature at the end of an inner solve: hand the iterate to the refinement
        st->inner_ratio = sqrt(st->rr / st->rr0);
        st->phase = PH_CORRECT;
      } else {
        st->status = 5;
        st->phase = PH_FINAL;
      }
      break;
    }
    case PH_UPDATE:
    after_update: {
      const double rn = S[0];
      st->inner_iters += 1;
      st->iters += 1;
      if (!isfinite(rn)) {
        st->status = 5;
        st->phase = PH_FINAL;
      } else if (rn <= st->tau2 * st->rr0 || st->iters >= st->max_iter ||
                 st->inner_iters >= st->inner_max ||
                 (I.pc == PC_FIXED && rn > 1e8 * st->rr0)) {  // a diverging iteration stops
        st->inner_ratio = sqrt(rn / st->rr0);
        st->phase = PH_CORRECT;
      } else if (I.pc != PC_JACOBI) {  // preconditioned: z = M^-1 rt first, then beta from <rt, z>
        st->rr = rn;
        st->cheb_j = 1;
        st->phase = I.pc == PC_CHEB ? PH_CHEB : PH_SPEC;
      } else {
        st->beta = rn / st->rr;
        st->rr = rn;
        st->rz = rn;
        st->parity ^= 1;
        st->phase = PH_STENCIL;
      }
      break;
    }
    case PH_CHEB:
    case PH_SPEC: {
      if (I.pc == PC_FIXED) {  // z = the scaled update of the paper's iteration
        st->beta = 0.0;
        st->phase = PH_STENCIL;
        break;
      }
      if (phase == PH_CHEB && st->cheb_j < I.cheb_k - 1) {
        st->cheb_j += 1;
        break;
      }
      const double rz = S[0];
      if (!(rz > 0.0) || !isfinite(rz)) {  // the preconditioner must stay positive definite
        if (st->inner_iters > 0) {
          st->inner_ratio = sqrt(st->rr / st->rr0);
          st->phase = PH_CORRECT;
        } else {
          st->status = 5;
          st->phase = PH_FINAL;
        }
        break;
      }
      if (st->inner_iters == 0) {
        st->beta = 0.0;
      } else {
        st->beta = rz / st->rz;
        st->parity ^= 1;
      }
      st->rz = rz;
      st->phase = PH_STENCIL;
      break;
    }
    case PH_CORRECT:
      st->sum_p = S[0];  // sum of the corrected p (for the gauge at the end)
      st->p_set = 1;
      st->phase = PH_RES64;
      break;
    case PH_FINAL:
      st->phase = PH_DONE;
      if (I.remaining) atomicSub(I.remaining, 1);
      break;
    default:
      break;
  }
}

// partial-sum slots each phase produces
__device__ __forceinline__ int phase_slots(int phase) {
  switch (phase) {
    case PH_MEANF: return 1;
    case PH_RES64: return 4;
    case PH_STENCIL:
    case PH_UPDATE:
    case PH_CORRECT:
    case PH_CHEB:
    case PH_SPEC: return 1;
    default: return 0;
  }
}

// nunits units arrive; their partial slots were written by nparts units (default: the same),
// which lets a sweep of several kernels reduce what an earlier kernel of the sweep stored.
__device__ __forceinline__ void finish_sweep(const InstDesc& I, InstState* st, int phase,
                                             int nunits, int nparts = 0) {
  if (nparts <= 0) nparts = nunits;
  if (arrive_last(I.ticket, nunits)) {  // uniform in the block
    double S[kSlots] = {0.0, 0.0, 0.0, 0.0};
    const int ns = phase_slots(phase);
    for (int k = 0; k < ns; ++k) S[k] = block_sum_slot(I.part + k * nparts, nparts);
    if (threadIdx.x == 0) {
      transition(I, st, phase, S);
      *I.ticket = 0u;
      __threadfence();
    }
  }
}

// Snapshot of the state fields the sweeps read.  Loaded with ld.global.cg (L2, not L1): in the
// persistent kernel the previous phase's transition may have been written by another SM moments
// ago, so an L1 copy must not be used; the loads are independent, so they overlap.
__device__ __forceinline__ InstState snapshot(const InstState* st) {
  InstState s;
  s.phase = __ldcg(&st->phase);
  s.inner_iters = __ldcg(&st->inner_iters);
  s.parity = __ldcg(&st->parity);
  s.first_res = __ldcg(&st->first_res);
  s.zero_sol = __ldcg(&st->zero_sol);
  s.use_guess = __ldcg(&st->use_guess);
  s.mu_f = __ldcg(&st->mu_f);
  s.alpha = __ldcg(&st->alpha);
  s.beta = __ldcg(&st->beta);
  s.sum_p = __ldcg(&st->sum_p);
  s.cheb_j = __ldcg(&st->cheb_j);
  s.p_set = __ldcg(&st->p_set);
  return s;
}

}  // namespace vdp
