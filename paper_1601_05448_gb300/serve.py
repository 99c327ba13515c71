"""Continuous-batching server for Poisson solves.

Requests (a grid, a density, a right-hand side, a tolerance) arrive over time.  The server
keeps a pool of solver contexts resident on the device (face coefficients, Jacobi scaling and
Krylov vectors stay in HBM; a context is reused by later requests of the same grid size) and one
batch engine.  Between batch runs it

  * moves arrived requests to the waiting queue,
  * admits waiting requests (first come, first served) while a context slot and the HBM budget
    allow -- a new context costs 98 bytes per cell, plus about 16 with the spectral
    preconditioner -- uploading their inputs and adding them to the running batch, so new work
    overlaps with requests already on the GPU,
  * retires finished members, records their latency (arrival to result ready) and returns their
    contexts to the pool (idle contexts are freed, oldest first, when the budget needs room).

Every member is solved exactly as it would be alone (the batch engine guarantees bitwise
identical results), so serving changes latency and throughput, never answers.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import PRECISIONS, VDP_ENOMEM, VDP_METHOD_FIXED_POINT, VDP_PRECOND_JACOBI, VDP_PRECOND_MG, \
    VDP_PRECOND_SPECTRAL, Batch, Solver, VdpError, spectral_extra_bytes, spectral_supported, vdp_mg_levels

BYTES_PER_CELL = 96 + 2  # device memory of one context per cell (FP64-sized buffers + BF16 diag)
# the multigrid levels (about 25 B per fine cell), z (8 B) and the weights (4 B)
MG_EXTRA_BYTES_PER_CELL = 25 + 8 + 4
CANCELLED = -2           # ServeRequest.status of a request cancelled before it finished


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float          # offset from the start of the run
    shape: tuple              # (nz, ny, nx)
    L: float
    rho: object               # host numpy array or torch tensor (float64)
    f: object
    tol: float
    # filled in by the server
    t_admit: float = float("nan")
    t_done: float = float("nan")
    status: int = -1
    iters: int = 0
    p: object = None          # device tensor with the result

    @property
    def latency_s(self) -> float:
        return self.t_done - self.arrival_s

    @property
    def queue_s(self) -> float:
        return self.t_admit - self.arrival_s


@dataclass
class ServeStats:
    completed: int = 0
    rejected: int = 0         # larger than the whole HBM budget (status VDP_ENOMEM)
    cancelled: int = 0
    elapsed_s: float = 0.0
    latencies_s: list = field(default_factory=list)
    queue_s: list = field(default_factory=list)
    peak_bytes: int = 0
    contexts_created: int = 0
    runs: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_s) if self.latencies_s else np.array([np.nan])
        q = np.array(self.queue_s) if self.queue_s else np.array([np.nan])
        return {"completed": self.completed, "rejected": self.rejected, "cancelled": self.cancelled,
                "elapsed_s": self.elapsed_s,
                "solves_per_s": self.completed / self.elapsed_s if self.elapsed_s > 0 else None,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_queue_s": float(np.mean(q)), "peak_context_bytes": self.peak_bytes,
                "contexts_created": self.contexts_created, "batch_runs": self.runs}


class Server:
    """``Server(precision="mixed", hbm_budget=64 GB, max_active=64).run(requests)``.

    precond="fixed_point" solves every request whose grid the FFT passes support by the paper's
    fixed-point iteration, "spectral" by CG with the spectral preconditioner (the others by CG
    with the multigrid V-cycle where the grid coarsens, else Jacobi-preconditioned CG); both need
    the batch of ordinary launches (persistent=False).
    precond="jacobi" uses Jacobi-preconditioned CG everywhere.  inner_tol: the mixed path's
    reduction per inner solve."""

    def __init__(self, precision: str = "mixed", hbm_budget: int = 64 << 30, max_active: int = 64,
                 pairs_per_run: int = 8, persistent: bool = False, tuned: bool = False, device: str = "cuda:0",
                 precond: str = "fixed_point", inner_tol: float = 1e-5):
        import torch
        self.torch = torch
        self.precision = precision
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.pairs = int(pairs_per_run)
        self.tuned = tuned
        if precond not in ("fixed_point", "spectral", "jacobi") or (precond != "jacobi" and persistent):
            raise ValueError("precond must be 'jacobi', or 'fixed_point' / 'spectral' with persistent=False")
        self.precond = precond
        self.inner_tol = float(inner_tol)
        self.device = torch.device(device)
        self.batch = Batch(precision, persistent=persistent)
        self.idle = collections.OrderedDict()   # ctx id -> (Solver, shape) available for reuse
        self._cancel = set()                     # request ids to cancel (any thread)
        self._cancel_lock = threading.Lock()
        self.bytes_in_use = 0                    # contexts alive (idle or busy)
        self.stats = ServeStats()

    # ---- context pool -----------------------------------------------------------------------

    def _spectral(self, shape) -> bool:
        nz, ny, nx = shape
        return self.precond != "jacobi" and spectral_supported(nx, ny, nz)

    def _multigrid(self, shape) -> bool:
        nz, ny, nx = shape
        return self.precond != "jacobi" and not self._spectral(shape) and vdp_mg_levels(nx, ny, nz) > 0

    def _ctx_bytes(self, shape) -> int:
        nz, ny, nx = shape
        extra = spectral_extra_bytes(nx, ny, nz) if self._spectral(shape) else 0
        if self._multigrid(shape):
            extra = MG_EXTRA_BYTES_PER_CELL * nx * ny * nz
        return BYTES_PER_CELL * nx * ny * nz + extra

    def _acquire(self, shape, L):
        for k, (s, shp) in list(self.idle.items()):
            if shp == shape and abs(s.L - L) == 0.0:
                del self.idle[k]
                return s
        need = self._ctx_bytes(shape)
        while self.bytes_in_use + need > self.budget and self.idle:
            _, (s, shp) = self.idle.popitem(last=False)   # free the oldest idle context
            s.close()
            self.bytes_in_use -= self._ctx_bytes(shp)
        if self.bytes_in_use + need > self.budget:
            return None
        nz, ny, nx = shape
        opts = {}
        if self.tuned:
            from .tune import cached_options
            opts = cached_options(nx, ny, nz, self.precision, batchable=True) or {}
        opts["precond"] = (VDP_PRECOND_SPECTRAL if self._spectral(shape) else
                           VDP_PRECOND_MG if self._multigrid(shape) else VDP_PRECOND_JACOBI)
        if self._spectral(shape) and self.precond == "fixed_point":
            opts["method"] = VDP_METHOD_FIXED_POINT
        opts["inner_tol"] = self.inner_tol
        try:
            s = Solver(nx, ny, nz, L, precision=self.precision, **opts)
        except VdpError:
            return None
        self.bytes_in_use += need
        self.stats.contexts_created += 1
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.bytes_in_use)
        return s

    def _release(self, s, shape):
        self.idle[id(s)] = (s, shape)

    def cancel(self, rid: int) -> None:
        """Cancel request `rid` (safe from another thread or an on_done callback): a waiting
        request is dropped, a running one leaves the batch at the next step; its status
        becomes CANCELLED."""
        with self._cancel_lock:
            self._cancel.add(rid)

    def _take_cancels(self):
        with self._cancel_lock:
            c, self._cancel = self._cancel, set()
        return c

    # ---- the loop ---------------------------------------------------------------------------

    def run(self, requests, time_scale: float = 1.0, on_done=None) -> ServeStats:
        """Serve `requests` (sorted by arrival), arrivals replayed in real time scaled by
        `time_scale`; returns the statistics.  Results are left in req.p (device tensors)."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting = collections.deque()
        active = {}   # ctx id -> (req, solver)
        t0 = time.perf_counter()
        now = lambda: (time.perf_counter() - t0) / time_scale
        cancelled = set()
        while pending or waiting or active:
            t = now()
            while pending and pending[0].arrival_s <= t:
                waiting.append(pending.popleft())
            cancelled |= self._take_cancels()
            if cancelled:  # drop cancelled requests, waiting or running
                for req in [r for r in waiting if r.rid in cancelled]:
                    waiting.remove(req)
                    req.status, req.t_done = CANCELLED, now()
                    self.stats.cancelled += 1
                for k, (req, s) in list(active.items()):
                    if req.rid in cancelled:
                        self.batch.remove(s)
                        del active[k]
                        req.status, req.t_done, req._f = CANCELLED, now(), None
                        self._release(s, req.shape)
                        self.stats.cancelled += 1
            # a request larger than the whole budget can never be admitted: reject it
            for req in [r for r in waiting if self._ctx_bytes(r.shape) > self.budget]:
                waiting.remove(req)
                req.status, req.t_done = VDP_ENOMEM, now()
                self.stats.rejected += 1
            # admission: FCFS while a slot and memory allow
            while waiting and len(active) < self.max_active:
                req = waiting[0]
                s = self._acquire(req.shape, req.L)
                if s is None:
                    break
                waiting.popleft()
                rho = torch.as_tensor(req.rho, dtype=torch.float64).to(self.device).contiguous()
                f = torch.as_tensor(req.f, dtype=torch.float64).to(self.device).contiguous()
                s.set_density(rho)
                req.p = torch.empty_like(f)
                req._f = f
                self.batch.add(s, f, req.p, req.tol)
                req.t_admit = now()
                active[id(s)] = (req, s)
            if active:
                self.batch.run(self.pairs)
                self.stats.runs += 1
                for k, (req, s) in list(active.items()):
                    if self.batch.done(s):
                        st = s.stats()
                        req.t_done = now()
                        req.status, req.iters = st.status, st.iters
                        self.batch.remove(s)
                        del active[k]
                        req._f = None
                        self._release(s, req.shape)
                        self.stats.completed += 1
                        self.stats.latencies_s.append(req.latency_s)
                        self.stats.queue_s.append(req.queue_s)
                        if on_done:
                            on_done(req)
            elif pending and not waiting:
                time.sleep(max(0.0, min(0.01, (pending[0].arrival_s - now()) * time_scale)))
            elif waiting and not active:
                # nothing runs and the head was not admitted: it cannot get a context even with
                # every idle one freed (the device or the budget has no room for it): reject it
                req = waiting.popleft()
                req.status, req.t_done = VDP_ENOMEM, now()
                self.stats.rejected += 1
        self.stats.elapsed_s = now()
        return self.stats

    def close(self) -> None:
        for _, (s, _) in list(self.idle.items()):
            s.close()
        self.idle.clear()
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
