"""Continuous-batching request loop over preloaded reduced systems.

Requests (system id, a vector of complex shifts) arrive over time.  A
dispatcher admits them into micro-batches as stream slots and device memory
free up, and hands each micro-batch to a worker that runs one batched
multi-system solve (ssv_solve_many) on its own CUDA stream; the solve call
releases the GIL, so micro-batches dispatched while others are still on the
GPU overlap on the device.  Admission is bounded by a device-memory budget:
a micro-batch starts only when the bytes already in flight plus its own
footprint (ssv_footprint of every request + its output) fit.

Every result is the same as the request solved alone: each shift is computed
by the same per-shift arithmetic whatever else shares the launch.

Latency of a request = completion time (its micro-batch finished on the GPU)
- arrival time, on the host clock.
"""
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ssv


@dataclass
class Request:
    rid: int
    system: int
    shifts: np.ndarray          # complex128, host
    t_arrival: float = 0.0      # seconds on the server clock
    t_done: float = -1.0
    result: torch.Tensor = None  # (p, s*m) complex128 on the device
    status: torch.Tensor = None
    footprint: int = 0


@dataclass
class ServeStats:
    completed: int = 0
    shifts: int = 0
    batches: int = 0
    max_inflight_batches: int = 0
    max_inflight_bytes: int = 0
    latencies: list = field(default_factory=list)

    def summary(self, wall):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {
            "requests": self.completed, "shifts": self.shifts, "batches": self.batches,
            "wall_s": wall, "shift_solves_per_s": self.shifts / wall if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_inflight_batches": self.max_inflight_batches,
            "max_inflight_bytes": self.max_inflight_bytes,
        }


class Server:
    """Continuous batching over `handles` (list of ssv.Handle) with `slots` streams."""

    def __init__(self, handles, slots=4, mem_budget=8 << 30, max_batch_shifts=4096, mode="g",
                 precision="fp64"):
        self.handles = list(handles)
        self.slots = slots
        self.mem_budget = int(mem_budget)
        self.max_batch_shifts = max_batch_shifts
        self.mode = mode
        self.precision = precision
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_slots = queue.Queue()
        for i in range(slots):
            self.free_slots.put(i)
        self.lock = threading.Lock()
        self.inflight_bytes = 0
        self.inflight_batches = 0
        self.stats = ServeStats()
        self.t0 = 0.0
        self.device = torch.device("cuda", torch.cuda.current_device())

    def footprint(self, req):
        h = self.handles[req.system]
        s = len(req.shifts)
        rows = h.out_rows(self.mode)
        return ssv.footprint(h.n, h.m, h.p, s, precision=self.precision, mode=self.mode) + \
            16 * rows * h.m * s + 20 * s

    def now(self):
        return time.perf_counter() - self.t0

    # -- worker side ----------------------------------------------------------------
    def _run_batch(self, slot, batch, nbytes):
        stream = self.streams[slot]
        try:
            with torch.cuda.stream(stream):
                hs = [self.handles[r.system] for r in batch]
                xs = [torch.from_numpy(r.shifts).pin_memory().to(self.device, non_blocking=True)
                      for r in batch]
                outs, sts = ssv.solve_many(hs, xs, mode=self.mode, precision=self.precision,
                                           stream=stream)
            stream.synchronize()
            t = self.now()
            for r, o, st in zip(batch, outs, sts):
                r.result, r.status, r.t_done = o, st, t
            with self.lock:
                self.stats.batches += 1
                for r in batch:
                    self.stats.completed += 1
                    self.stats.shifts += len(r.shifts)
                    self.stats.latencies.append(r.t_done - r.t_arrival)
        finally:
            with self.lock:
                self.inflight_bytes -= nbytes
                self.inflight_batches -= 1
            self.free_slots.put(slot)

    # -- dispatcher ---------------------------------------------------------------------
    def run(self, requests, realtime=True, idle_sleep=2e-4):
        """Serve `requests` (sorted by t_arrival).  With realtime=True a request is
        visible only once the server clock passes its arrival time."""
        for r in requests:
            r.footprint = self.footprint(r)
            if r.footprint > self.mem_budget:
                raise ValueError("request %d needs %d bytes > budget %d" % (r.rid, r.footprint,
                                                                            self.mem_budget))
        pending = []
        nxt = 0
        workers = []
        self.t0 = time.perf_counter()
        if not realtime:
            for r in requests:
                r.t_arrival = 0.0
        while nxt < len(requests) or pending:
            t = self.now()
            while nxt < len(requests) and (not realtime or requests[nxt].t_arrival <= t):
                pending.append(requests[nxt])
                nxt += 1
            if not pending:
                time.sleep(min(idle_sleep, max(0.0, requests[nxt].t_arrival - t)))
                continue
            try:
                slot = self.free_slots.get(timeout=idle_sleep)
            except queue.Empty:
                continue
            # admit the oldest pending requests that fit the memory budget
            batch, nbytes, nsh = [], 0, 0
            with self.lock:
                room = self.mem_budget - self.inflight_bytes
            rest = []
            for r in pending:
                if nbytes + r.footprint <= room and nsh + len(r.shifts) <= self.max_batch_shifts:
                    batch.append(r)
                    nbytes += r.footprint
                    nsh += len(r.shifts)
                else:
                    rest.append(r)
            if not batch:
                self.free_slots.put(slot)
                time.sleep(idle_sleep)
                continue
            pending = rest
            with self.lock:
                self.inflight_bytes += nbytes
                self.inflight_batches += 1
                self.stats.max_inflight_batches = max(self.stats.max_inflight_batches,
                                                      self.inflight_batches)
                self.stats.max_inflight_bytes = max(self.stats.max_inflight_bytes,
                                                    self.inflight_bytes)
            w = threading.Thread(target=self._run_batch, args=(slot, batch, nbytes), daemon=True)
            w.start()
            workers.append(w)
        for w in workers:
            w.join()
        torch.cuda.synchronize()
        return self.stats.summary(self.now())


def make_requests(reqs):
    """From workloads.serving_requests tuples (t, system, shifts) to Request objects."""
    return [Request(rid=i, system=int(s), shifts=np.asarray(sh, dtype=np.complex128), t_arrival=float(t))
            for i, (t, s, sh) in enumerate(reqs)]
