"""Continuous-batching server for Poisson solves.

Requests (a grid, a density, a right-hand side, a tolerance) arrive over time.  The server
keeps a pool of solver contexts resident on the device (face coefficients, Jacobi scaling,
spectral tables and iteration vectors stay in HBM; a context is reused by later requests of the
same grid size) and admits requests first come, first served while a slot and the HBM budget
allow -- a new context costs 114 bytes per cell, plus about 16 and the half spectrum with the
FFT passes -- freeing idle contexts, oldest first, when the budget needs room.  Requests that
arrive while others are on the GPU start as soon as a slot frees up; their work overlaps on the
device.  Two engines run the admitted work:

  * mode="streams" (default): `max_active` worker slots, each a host thread with its own CUDA
    stream and its own contexts.  An admitted request's density is set and its solve launched
    on the slot's stream -- one graph launch whose device-side loop runs the whole solve -- so
    up to `max_active` solves of any sizes run on the GPU at once, and a finished slot takes the
    next request at once (no batch graph to rebuild when membership changes).
  * mode="batch": every admitted request joins one batch (vdp_batch_*: a persistent kernel or
    ordinary launches under a CUDA graph); finished members retire between batch runs.

Every request is solved exactly as it would be alone (same kernels, layout and arithmetic on its
own context), so serving changes latency and throughput, never answers.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import PRECISIONS, VDP_ENOMEM, VDP_METHOD_FIXED_POINT, VDP_PRECOND_JACOBI, VDP_PRECOND_MG, \
    VDP_PRECOND_SPECTRAL, Batch, Solver, VdpError, spectral_extra_bytes, spectral_supported, vdp_mg_levels

BYTES_PER_CELL = 112 + 2  # device memory of one context per cell (FP64-sized buffers + BF16 diag)
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
    # optional torch.cuda.Event recorded after the device tensors rho and f were written: the
    # slot's stream waits for it (a client need not synchronise before submitting)
    ready: object = None
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
    max_loop_gap_s: float = 0.0     # longest pause of the dispatcher loop (streams engine)
    max_loop_gap_at_s: float = 0.0  # when it ended (stream time)

    def summary(self) -> dict:
        lat = np.array(self.latencies_s) if self.latencies_s else np.array([np.nan])
        q = np.array(self.queue_s) if self.queue_s else np.array([np.nan])
        return {"completed": self.completed, "rejected": self.rejected, "cancelled": self.cancelled,
                "elapsed_s": self.elapsed_s,
                "solves_per_s": self.completed / self.elapsed_s if self.elapsed_s > 0 else None,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_queue_s": float(np.mean(q)), "peak_context_bytes": self.peak_bytes,
                "contexts_created": self.contexts_created, "batch_runs": self.runs,
                "max_loop_gap_s": self.max_loop_gap_s, "max_loop_gap_at_s": self.max_loop_gap_at_s}


class _Slot:
    """One worker slot of the streams engine: a host thread with its own CUDA stream."""

    def __init__(self, server, index: int):
        torch = server.torch
        self.index = index
        self.stream = torch.cuda.Stream(device=server.device)
        self.inbox = queue.Queue()
        self.busy = False
        self.thread = threading.Thread(target=self._work, args=(server,), daemon=True,
                                       name=f"vdp-serve-{index}")
        self.thread.start()

    def _work(self, server):
        torch = server.torch
        torch.cuda.set_device(server.device)
        while True:
            item = self.inbox.get()
            if item is None:
                return
            req, solver = item
            try:
                with torch.cuda.stream(self.stream):
                    if req.ready is not None:  # the client's writes of rho and f come first
                        self.stream.wait_event(req.ready)
                    rho = torch.as_tensor(req.rho, dtype=torch.float64).to(server.device, non_blocking=False)
                    f = torch.as_tensor(req.f, dtype=torch.float64).to(server.device, non_blocking=False)
                    rho, f = rho.contiguous(), f.contiguous()
                    p = torch.empty_like(f)
                # (the library works on this stream, after the copies above; its own calls wait
                # for the results)
                solver.set_density(rho)
                st = solver.solve(f, p, req.tol, check=False)
                req.p = p
                del rho, f, p
                server._done.put((self, req, solver, st.status, st.iters, None))
            except Exception as e:  # reported to the dispatcher, which records the failure
                server._done.put((self, req, solver, -1, 0, e))


class Server:
    """``Server(precision="mixed", hbm_budget=64 GB, max_active=8).run(requests)``.

    mode="streams" (default): `max_active` worker slots with their own streams (see the module
    docstring); mode="batch": one batch of all admitted requests (vdp_batch_*, `persistent` and
    `pairs_per_run` apply there only).
    precond="fixed_point" solves every request whose grid the FFT passes support by the paper's
    fixed-point iteration, "spectral" by CG with the spectral preconditioner (the others by CG
    with the multigrid V-cycle where the grid coarsens, else Jacobi-preconditioned CG); in batch
    mode both need the batch of ordinary launches (persistent=False).
    precond="jacobi" uses Jacobi-preconditioned CG everywhere.  inner_tol: the mixed path's
    reduction per inner solve."""

    def __init__(self, precision: str = "mixed", hbm_budget: int = 64 << 30, max_active: int = 8,
                 pairs_per_run: int = 8, persistent: bool = False, tuned: bool = False, device: str = "cuda:0",
                 precond: str = "fixed_point", inner_tol: float = 1e-4, mode: str = "streams"):
        import torch
        self.torch = torch
        self.precision = precision
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.pairs = int(pairs_per_run)
        self.tuned = tuned
        if mode not in ("streams", "batch"):
            raise ValueError("mode must be 'streams' or 'batch'")
        if precond not in ("fixed_point", "spectral", "jacobi") or (precond != "jacobi" and persistent):
            raise ValueError("precond must be 'jacobi', or 'fixed_point' / 'spectral' with persistent=False")
        if mode == "streams" and persistent:
            raise ValueError("persistent=True is a batch-mode option")
        self.mode = mode
        self.precond = precond
        self.inner_tol = float(inner_tol)
        self.device = torch.device(device)
        self.batch = Batch(precision, persistent=persistent) if mode == "batch" else None
        # idle contexts available for reuse, oldest first: key -> (Solver, shape, slot index)
        self.idle = collections.OrderedDict()
        self._cancel = set()                     # request ids to cancel (any thread)
        self._cancel_lock = threading.Lock()
        self.bytes_in_use = 0                    # contexts alive (idle or busy)
        self.stats = ServeStats()
        self._slots = []
        self._done = queue.Queue()
        if mode == "streams":
            self._slots = [_Slot(self, i) for i in range(self.max_active)]

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

    def _acquire(self, shape, L, slot=None):
        """A context for `shape` (bound to `slot`'s stream in streams mode): an idle one, or a
        new one if the budget allows after freeing idle contexts oldest first; else None."""
        want = None if slot is None else slot.index
        for k, (s, shp, si) in list(self.idle.items()):
            if shp == shape and si == want and abs(s.L - L) == 0.0:
                del self.idle[k]
                return s
        need = self._ctx_bytes(shape)
        while self.bytes_in_use + need > self.budget and self.idle:
            _, (s, shp, _) = self.idle.popitem(last=False)   # free the oldest idle context
            s.close()
            self.bytes_in_use -= self._ctx_bytes(shp)
        if self.bytes_in_use + need > self.budget:
            return None
        nz, ny, nx = shape
        opts = {}
        if self.tuned:
            from .tune import cached_options
            opts = cached_options(nx, ny, nz, self.precision, batchable=self.mode == "batch") or {}
        opts["precond"] = (VDP_PRECOND_SPECTRAL if self._spectral(shape) else
                           VDP_PRECOND_MG if self._multigrid(shape) else VDP_PRECOND_JACOBI)
        if self._spectral(shape) and self.precond == "fixed_point":
            opts["method"] = VDP_METHOD_FIXED_POINT
        opts["inner_tol"] = self.inner_tol
        if slot is not None:
            opts["stream"] = slot.stream
        try:
            s = Solver(nx, ny, nz, L, precision=self.precision, **opts)
        except VdpError:
            return None
        self.bytes_in_use += need
        self.stats.contexts_created += 1
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.bytes_in_use)
        return s

    def _release(self, s, shape, slot=None):
        self.idle[id(s)] = (s, shape, None if slot is None else slot.index)

    def warm(self, shapes, L: float) -> int:
        """Create the contexts the stream will need before it starts: for every slot (streams
        mode; one set in batch mode) and every grid shape, a context within the budget, and run
        one short solve on it (a density ratio of 2 to relative residual 1e-2) through the slot's
        own thread, so context creation, graph capture and each thread's first allocations on
        its stream -- work that would otherwise stall admissions early in the stream -- are
        done.  Returns the contexts created."""
        torch = self.torch
        made = 0
        slots = self._slots if self.mode == "streams" else [None]
        for shape in shapes:
            shape = tuple(shape)
            nz, ny, nx = shape
            x = torch.arange(nx, dtype=torch.float64, device=self.device) * (6.283185307179586 / nx)
            rho = (1.5 + 0.5 * torch.cos(x)).expand(nz, ny, nx).contiguous()
            f = torch.sin(x).expand(nz, ny, nx).contiguous()
            for slot in slots:
                if self._ctx_bytes(shape) + self.bytes_in_use > self.budget:
                    continue
                s = self._acquire(shape, L, slot)
                if s is None:
                    continue
                made += 1
                if slot is None:
                    s.set_density(rho)
                    s.solve(f, torch.empty_like(f), 1e-2)
                    self._release(s, shape, slot)
                    continue
                req = ServeRequest(-1, 0.0, shape, L, rho, f, 1e-2)
                slot.busy = True
                slot.inbox.put((req, s))
                done_slot, _, s_back, status, _, exc = self._done.get()
                done_slot.busy = False
                self._release(s_back, shape, done_slot)
                if exc is not None:
                    raise exc
        torch.cuda.synchronize(self.device)
        return made

    def cancel(self, rid: int) -> None:
        """Cancel request `rid` (safe from another thread or an on_done callback): a waiting
        request is dropped; a running one leaves at its next step (batch mode) or has its result
        discarded when its solve ends (streams mode); its status becomes CANCELLED."""
        with self._cancel_lock:
            self._cancel.add(rid)

    def _take_cancels(self):
        with self._cancel_lock:
            c, self._cancel = self._cancel, set()
        return c

    # ---- the loop ---------------------------------------------------------------------------

    def run(self, requests, time_scale: float = 1.0, on_done=None, source=None) -> ServeStats:
        """Serve `requests` (sorted by arrival), arrivals replayed in real time scaled by
        `time_scale`; returns the statistics.  Results are left in req.p (device tensors).
        source: optional callable(req) that fills req.rho / req.f when the request arrives (a
        client producing its inputs at that moment)."""
        t0 = time.perf_counter()
        self._now = lambda: (time.perf_counter() - t0) / time_scale
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        if self.mode == "streams":
            self._run_streams(pending, on_done, source, time_scale)
        else:
            self._run_batch(pending, on_done, source, time_scale)
        self.stats.elapsed_s = self._now()
        return self.stats

    def _arrivals(self, pending, waiting, source):
        t = self._now()
        while pending and pending[0].arrival_s <= t:
            req = pending.popleft()
            if source is not None:
                source(req)
            waiting.append(req)

    def _reject_oversize(self, waiting):
        # a request larger than the whole budget can never be admitted: reject it
        for req in [r for r in waiting if self._ctx_bytes(r.shape) > self.budget]:
            waiting.remove(req)
            req.status, req.t_done = VDP_ENOMEM, self._now()
            self.stats.rejected += 1

    def _drop_cancelled_waiting(self, waiting, cancelled):
        for req in [r for r in waiting if r.rid in cancelled]:
            waiting.remove(req)
            req.status, req.t_done = CANCELLED, self._now()
            self.stats.cancelled += 1

    def _finish(self, req, status, iters, on_done):
        req.t_done = self._now()
        req.status, req.iters = status, iters
        self.stats.completed += 1
        self.stats.latencies_s.append(req.latency_s)
        self.stats.queue_s.append(req.queue_s)
        if on_done:
            on_done(req)

    def _run_streams(self, pending, on_done, source, time_scale):
        waiting = collections.deque()
        running = {}      # rid -> (req, slot)
        cancelled = set()
        error = None
        last = time.perf_counter()
        while pending or waiting or running:
            now_w = time.perf_counter()
            if now_w - last > self.stats.max_loop_gap_s:
                self.stats.max_loop_gap_s = now_w - last
                self.stats.max_loop_gap_at_s = self._now()
            last = now_w
            self._arrivals(pending, waiting, source)
            cancelled |= self._take_cancels()
            self._drop_cancelled_waiting(waiting, cancelled)
            self._reject_oversize(waiting)
            # admission: FCFS while a slot is free and the budget allows the context
            while waiting:
                free = [sl for sl in self._slots if not sl.busy]
                if not free:
                    break
                req = waiting[0]
                # prefer a free slot that already holds an idle context of this size
                holders = {si for (_, shp, si) in self.idle.values() if shp == req.shape}
                slot = next((sl for sl in free if sl.index in holders), free[0])
                s = self._acquire(req.shape, req.L, slot)
                if s is None:
                    if not running:  # nothing runs and no room even with every idle context freed
                        waiting.popleft()
                        req.status, req.t_done = VDP_ENOMEM, self._now()
                        self.stats.rejected += 1
                        continue
                    break
                waiting.popleft()
                req.t_admit = self._now()
                slot.busy = True
                running[req.rid] = (req, slot)
                slot.inbox.put((req, s))
                self.stats.runs += 1
            # completions (block briefly when nothing else can happen)
            timeout = 0.0005 if (pending or waiting) else 0.05
            if pending and not waiting and running:
                timeout = max(0.0, min(timeout, (pending[0].arrival_s - self._now()) * time_scale))
            try:
                item = self._done.get(timeout=timeout) if running else None
            except queue.Empty:
                item = None
            if item is None and not running and pending and not waiting:
                time.sleep(max(0.0, min(0.01, (pending[0].arrival_s - self._now()) * time_scale)))
            while item is not None:
                slot, req, s, status, iters, exc = item
                slot.busy = False
                running.pop(req.rid, None)
                self._release(s, req.shape, slot)
                if exc is not None and error is None:
                    error = exc
                if req.rid in cancelled:
                    req.status, req.t_done, req.p = CANCELLED, self._now(), None
                    self.stats.cancelled += 1
                else:
                    self._finish(req, status, iters, on_done)
                try:
                    item = self._done.get_nowait()
                except queue.Empty:
                    item = None
        if error is not None:
            raise error

    def _run_batch(self, pending, on_done, source, time_scale):
        torch = self.torch
        waiting = collections.deque()
        active = {}   # ctx id -> (req, solver)
        cancelled = set()
        while pending or waiting or active:
            self._arrivals(pending, waiting, source)
            cancelled |= self._take_cancels()
            if cancelled:  # drop cancelled requests, waiting or running
                self._drop_cancelled_waiting(waiting, cancelled)
                for k, (req, s) in list(active.items()):
                    if req.rid in cancelled:
                        self.batch.remove(s)
                        del active[k]
                        req.status, req.t_done, req._f = CANCELLED, self._now(), None
                        self._release(s, req.shape)
                        self.stats.cancelled += 1
            self._reject_oversize(waiting)
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
                req.t_admit = self._now()
                active[id(s)] = (req, s)
            if active:
                self.batch.run(self.pairs)
                self.stats.runs += 1
                for k, (req, s) in list(active.items()):
                    if self.batch.done(s):
                        st = s.stats()
                        self.batch.remove(s)
                        del active[k]
                        req._f = None
                        self._release(s, req.shape)
                        self._finish(req, st.status, st.iters, on_done)
            elif pending and not waiting:
                time.sleep(max(0.0, min(0.01, (pending[0].arrival_s - self._now()) * time_scale)))
            elif waiting and not active:
                # nothing runs and the head was not admitted: it cannot get a context even with
                # every idle one freed (the device or the budget has no room for it): reject it
                req = waiting.popleft()
                req.status, req.t_done = VDP_ENOMEM, self._now()
                self.stats.rejected += 1

    def close(self) -> None:
        for sl in self._slots:
            sl.inbox.put(None)
        for sl in self._slots:
            sl.thread.join(timeout=30)
        self._slots = []
        for _, (s, _, _) in list(self.idle.items()):
            s.close()
        self.idle.clear()
        if self.batch is not None:
            self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
