"""Continuous-batching plan server for many vehicles on one GPU.

Plan requests from many vehicles arrive at any time.  Each names its
vehicle, its candidate count N, horizon H and control interval dt.  The server
keeps every vehicle's prepared terrain and its last best controls (the warm
start) resident on the device.  It admits queued requests into ragged batches
as candidate slots and device memory free up, and runs each batch as one
atp_plan_batch launch, preceded by one atp_sample per request (candidates
drawn on the device around the warm start).  Batches on separate streams
overlap on the GPU, so requests that arrive while others run start without
waiting for them to finish.

`Server.serve` runs a request trace in real time and records, per request,
arrival, launch and completion (result on the host) times.  `Server.sequential`
runs the same trace through the plain single-plan path, one request at a time,
as the baseline.  Both use the same candidates and warm starts, so their
per-request results must agree bit for bit.
"""
from __future__ import annotations

import bisect
import contextlib
import gc
import math
import time
from dataclasses import dataclass

import numpy as np

from . import atp

ALIGN = 256


def _align(n: int) -> int:
    return (n + ALIGN - 1) // ALIGN * ALIGN


@dataclass
class Request:
    rid: int
    vehicle: int
    N: int
    H: int
    dt: float
    t_arrive: float           # seconds after the start of the trace


def poisson_trace(n_vehicles: int = 32, rate_hz: float = 20.0, duration_s: float = 60.0,
                  seed: int = 0, sizes=(1024, 4096, 16384, 32768), h_range=(40, 150),
                  dts=tuple(0.005 * k for k in range(4, 11))):
    """Each vehicle sends plan requests as a Poisson process of rate_hz; every
    request draws N from `sizes`, H uniformly in h_range and dt from `dts`."""
    rng = np.random.default_rng(seed)
    reqs = []
    for v in range(n_vehicles):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            reqs.append((t, v, int(rng.choice(sizes)), int(rng.integers(h_range[0], h_range[1] + 1)),
                         float(rng.choice(dts))))
            t += rng.exponential(1.0 / rate_hz)
    reqs.sort()
    return [Request(i, v, N, H, dt, t) for i, (t, v, N, H, dt) in enumerate(reqs)]


class DeviceArena:
    """Best-fit allocator over one preallocated device buffer; the server
    admits a request only when its buffers fit."""

    def __init__(self, nbytes: int, device="cuda"):
        import torch
        self.nbytes = _align(nbytes)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.free = [(0, self.nbytes)]          # sorted, coalesced (offset, size)
        self.used = 0

    def alloc(self, nbytes: int):
        n = _align(max(nbytes, 1))
        best = None
        for i, (off, size) in enumerate(self.free):
            if size >= n and (best is None or size < self.free[best][1]):
                best = i
        if best is None:
            return None
        off, size = self.free[best]
        if size == n:
            del self.free[best]
        else:
            self.free[best] = (off + n, size - n)
        self.used += n
        return off

    def release(self, off: int, nbytes: int):
        n = _align(max(nbytes, 1))
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # coalesce with neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]
        self.used -= n

    def view(self, off: int, shape, dtype):
        import torch
        n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        return self.buf[off:off + n].view(dtype).view(*shape)


def request_layout(N: int, H: int):
    """Byte offsets of one request's buffers inside its arena block: its
    candidates' controls.  The plan writes its best controls straight into
    the vehicle's warm-start buffer and its result into the stream's result
    row; the per-candidate outputs stay in the library's scratch."""
    parts = [("ctrl", (H, N, 2), "f4")]
    off, lay = 0, []
    for name, shape, dt in parts:
        n = int(np.prod(shape)) * np.dtype(dt).itemsize
        lay.append((name, off, shape, dt))
        off = _align(off + n)
    return lay, off


@dataclass
class Vehicle:
    veh: dict
    cost: dict
    x0: list
    terrain: object               # atp.Terrain (texels resident on the device)
    prev: object                  # CUDA float32 [H_max, 2], last best controls
    prev_H: int = 0
    key: tuple = (0, 0)
    busy: bool = False
    marsh: object = None          # the C-ABI structs of veh, cost, terrain and x0 (Server sets it)


@dataclass
class Record:
    rid: int
    vehicle: int
    N: int
    H: int
    t_arrive: float
    t_launch: float = math.nan
    t_done: float = math.nan
    batch: int = 0
    best_idx: int = -1
    best_cost: float = math.nan


@contextlib.contextmanager
def collector_paused():
    """Pause Python's automatic garbage collector for a real-time loop and
    restore its previous state after.  A full collection in a process with
    torch loaded walks a few hundred thousand objects and takes about 0.1 s,
    longer than dozens of plans; reference counting still frees everything
    that is not part of a cycle while the collector is paused."""
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


@dataclass
class _Batch:
    reqs: list
    blocks: list
    event: object
    out_host: object
    slot: int
    t_launch: float


def admit(queue, vehicles, max_batch: int, slot_candidates: int, alloc):
    """One admission pass over the arrived requests, in arrival order: a
    request joins the batch if its vehicle has no plan in flight and no
    earlier request still waiting, the batch has room (max_batch requests,
    slot_candidates candidates) and alloc(request) finds it device memory
    (an offset, or None).  Returns (batch, offsets, requests kept waiting);
    admitted vehicles are marked busy."""
    batch, blocks, keep, cands = [], [], [], 0
    waiting = set()                       # vehicles with an earlier request kept back
    for r in queue:
        v = vehicles[r.vehicle]
        if (v.busy or r.vehicle in waiting or len(batch) >= max_batch or
                cands + r.N > slot_candidates):
            keep.append(r)
            waiting.add(r.vehicle)
            continue
        off = alloc(r)
        if off is None:                   # no memory: wait for completions
            keep.append(r)
            waiting.add(r.vehicle)
            continue
        v.busy = True
        batch.append(r)
        blocks.append(off)
        cands += r.N
    return batch, blocks, keep


def check_trace(trace, vehicles):
    """Every request names a vehicle of the fleet and a horizon that fits its
    warm-start buffer, into which the plan writes its best controls: refused
    up front otherwise (ValueError), before anything is launched."""
    for r in trace:
        if not 0 <= r.vehicle < len(vehicles):
            raise ValueError(f"request {r.rid}: no vehicle {r.vehicle}")
        rows = int(vehicles[r.vehicle].prev.shape[0])
        if not 1 <= r.H <= rows:
            raise ValueError(f"request {r.rid}: H = {r.H} outside 1..{rows}")


class Server:
    """Continuous batching over `streams` CUDA streams (one atp context each).
    The vehicles' parameters (vehicle, cost, start state) are marshalled for
    the C-ABI once, here: change a vehicle's parameters by building a new
    Server.  Each plan writes its best controls into its vehicle's warm-start
    buffer and its result into a per-stream result row; it keeps no per-step
    margins."""

    def __init__(self, vehicles, streams: int = 2, slot_candidates: int = 1 << 17,
                 arena_bytes: int = 1 << 30, max_batch: int = 64, sigma=(0.2, 0.3),
                 h_max: int = 150, device: int = 0):
        import torch
        self.torch = torch
        self.vehicles = vehicles
        self.sigma = sigma
        self.slot_candidates = slot_candidates
        self.max_batch = min(max_batch, 64)
        self.ctxs = [atp.Context(device) for _ in range(streams)]
        for c in self.ctxs:
            c.reserve(slot_candidates, h_max)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.arena = DeviceArena(arena_bytes, device=f"cuda:{device}")
        self.inflight = [None] * streams
        self.pinned = torch.empty((self.max_batch * streams, 6), dtype=torch.int32).pin_memory()
        # each stream's result rows (atp_plan_out), read back by one copy per batch
        self.outs = [torch.zeros((self.max_batch, 6), dtype=torch.int32, device=f"cuda:{device}")
                     for _ in range(streams)]
        # What the loop hands the C-ABI, prepared once: each vehicle's
        # marshalled parameters, the raw addresses of the arena, the result
        # rows and the warm starts, the stream handles, one request array and
        # one completion event per stream.  Building these per request cost
        # more host time than the plan's launch (measured: 57 us per request).
        for v in vehicles:
            vc, cc, xc = atp.vehicle(v.veh), atp.cost(v.cost), atp.state(v.x0)
            v.marsh = (vc, cc, xc, atp.C.pointer(vc), atp.C.pointer(cc), atp.C.pointer(v.terrain.c),
                       atp.C.pointer(xc), v.prev.data_ptr())
        self.arena_ptr = self.arena.buf.data_ptr()
        self.out_ptrs = [o.data_ptr() for o in self.outs]
        self.stream_ptrs = [atp.C.c_void_p(st.cuda_stream) for st in self.streams]
        self.req_arrays = [(atp.PlanRequest * self.max_batch)() for _ in range(streams)]
        self.events = [torch.cuda.Event() for _ in range(streams)]
        self.pinned_np = self.pinned.numpy()
        self.h_max = h_max
        # (seconds, trace time): the longest interval between two passes of
        # the serving loop (served) or the longest launch-to-result time
        # (sequential) in the last run; a host stall shows up here
        self.max_loop_gap = (0.0, 0.0)

    # -- per request -----------------------------------------------------
    def _enqueue(self, s, reqs, blocks):
        """Sample every request's candidates and run the batch on stream s.
        Each plan writes its best controls into its vehicle's warm-start
        buffer (after its own sampler has read them, on the same stream) and
        its result into row i of the stream's result rows."""
        ctx, sp, arr = self.ctxs[s], self.stream_ptrs[s], self.req_arrays[s]
        out0 = self.out_ptrs[s]
        for i, (r, off) in enumerate(zip(reqs, blocks)):
            v = self.vehicles[r.vehicle]
            m = v.marsh
            ctrl = self.arena_ptr + off
            ctx.sample_raw(r.N, r.H, self.sigma[0], self.sigma[1], v.key, r.rid,
                           m[7] if v.prev_H > 0 else 0, v.prev_H, 1, ctrl, sp)
            arr[i] = atp.PlanRequest(m[3], m[4], m[5], m[6], None, ctrl, r.N, r.H, r.dt, 0,
                                     out0 + 24 * i, m[7], None, None, None, None, None)
        ctx.plan_batch_raw(arr, len(reqs), sp)
        for r in reqs:
            self.vehicles[r.vehicle].prev_H = r.H

    # -- continuous batching ----------------------------------------------
    def serve(self, trace, idle_sleep: float = 2e-5):
        """Run the trace in real time; returns one Record per request."""
        check_trace(trace, self.vehicles)
        with collector_paused():
            return self._serve(trace, idle_sleep)

    def _serve(self, trace, idle_sleep):
        torch = self.torch
        recs = {r.rid: Record(r.rid, r.vehicle, r.N, r.H, r.t_arrive) for r in trace}
        pending = list(trace)                  # not yet arrived
        queue = []                             # arrived, not admitted
        pi = 0
        done = 0
        t0 = time.perf_counter()
        t_prev, self.max_loop_gap = 0.0, (0.0, 0.0)
        while done < len(trace):
            now = time.perf_counter() - t0
            if now - t_prev > self.max_loop_gap[0]:      # the host loop's longest pause
                self.max_loop_gap = (now - t_prev, t_prev)
            t_prev = now
            while pi < len(pending) and pending[pi].t_arrive <= now:
                queue.append(pending[pi])
                pi += 1
            # completions
            for s, b in enumerate(self.inflight):
                if b is not None and b.event.query():
                    t_done = time.perf_counter() - t0
                    base = b.slot * self.max_batch
                    res = self.pinned_np[base:base + len(b.reqs)]
                    for i, r in enumerate(b.reqs):
                        rec = recs[r.rid]
                        rec.t_done = t_done
                        rec.best_idx = int(np.uint32(res[i, 0]))
                        rec.best_cost = float(res[i, 2:3].view(np.float32)[0])
                        self.vehicles[r.vehicle].busy = False
                        self.arena.release(b.blocks[i], request_layout(r.N, r.H)[1])
                    done += len(b.reqs)
                    self.inflight[s] = None
            # admission into a free stream slot
            for s in range(len(self.streams)):
                if self.inflight[s] is not None or not queue:
                    continue
                batch, blocks, queue = admit(queue, self.vehicles, self.max_batch, self.slot_candidates,
                                             lambda r: self.arena.alloc(request_layout(r.N, r.H)[1]))
                if not batch:
                    continue
                stream = self.streams[s]
                t_launch = time.perf_counter() - t0
                self._enqueue(s, batch, blocks)
                with torch.cuda.stream(stream):
                    base = s * self.max_batch
                    host = self.pinned[base:base + len(batch)]
                    host.copy_(self.outs[s][:len(batch)], non_blocking=True)
                    ev = self.events[s]
                    ev.record(stream)
                for r in batch:
                    recs[r.rid].t_launch = t_launch
                    recs[r.rid].batch = len(batch)
                self.inflight[s] = _Batch(batch, blocks, ev, host, s, t_launch)
            if all(b is None for b in self.inflight) and not queue and pi < len(pending):
                wait = pending[pi].t_arrive - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
            else:
                time.sleep(idle_sleep)
        return [recs[r.rid] for r in trace]

    # -- baseline ----------------------------------------------------------
    def sequential(self, trace):
        """The plain single-plan path: one request at a time, in arrival order."""
        check_trace(trace, self.vehicles)
        with collector_paused():
            return self._sequential(trace)

    def _sequential(self, trace):
        torch = self.torch
        ctx, stream = self.ctxs[0], self.streams[0]
        out_host = self.pinned[0:1]
        recs = []
        t0 = time.perf_counter()
        self.max_loop_gap = (0.0, 0.0)
        for r in trace:
            while time.perf_counter() - t0 < r.t_arrive:
                time.sleep(2e-5)
            rec = Record(r.rid, r.vehicle, r.N, r.H, r.t_arrive)
            off = self.arena.alloc(request_layout(r.N, r.H)[1])
            v = self.vehicles[r.vehicle]
            m = v.marsh
            ctrl = self.arena_ptr + off
            sp = self.stream_ptrs[0]
            rec.t_launch = time.perf_counter() - t0
            ctx.sample_raw(r.N, r.H, self.sigma[0], self.sigma[1], v.key, r.rid,
                           m[7] if v.prev_H > 0 else 0, v.prev_H, 1, ctrl, sp)
            ctx.plan_raw(m[3], m[4], m[5], m[6], ctrl, r.N, r.H, r.dt, 0, self.out_ptrs[0], m[7], sp)
            v.prev_H = r.H
            with torch.cuda.stream(stream):
                out_host[0].copy_(self.outs[0][0], non_blocking=True)
            stream.synchronize()
            rec.t_done = time.perf_counter() - t0
            if rec.t_done - rec.t_launch > self.max_loop_gap[0]:
                self.max_loop_gap = (rec.t_done - rec.t_launch, rec.t_launch)
            rec.best_idx = int(out_host[0, 0])
            rec.best_cost = float(out_host[0, 2:3].view(torch.float32)[0])
            rec.batch = 1
            self.arena.release(off, request_layout(r.N, r.H)[1])
            recs.append(rec)
        return recs


def latency_summary(recs, duration=None):
    lat = np.array([r.t_done - r.t_arrive for r in recs]) * 1000.0
    work = sum(r.N * r.H for r in recs)
    span = max(r.t_done for r in recs) - min(r.t_arrive for r in recs)
    return {"requests": len(recs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "mean_batch": float(np.mean([r.batch for r in recs])),
            "rollout_steps_per_s": work / span if span > 0 else math.nan}


def resident_vehicles(fleet, device: int = 0, h_max: int = 150):
    """Device-resident state of a fleet: each vehicle's prepared terrain and
    a zeroed warm-start buffer.  `fleet` items carry terrain (heights, cell,
    x0, y0), vehicle, cost, x0 and key, as gen.fleet() makes them."""
    import torch
    ctx = atp.Context(device)
    out = []
    for f in fleet:
        t = f.terrain
        ter = ctx.terrain_prepare(torch.as_tensor(t.heights).to(f"cuda:{device}"), t.cell, t.x0, t.y0)
        prev = torch.zeros((h_max, 2), dtype=torch.float32, device=f"cuda:{device}")
        out.append(Vehicle(veh=f.vehicle, cost=f.cost, x0=[float(q) for q in f.x0], terrain=ter,
                           prev=prev, prev_H=0, key=tuple(int(k) for k in f.key)))
    torch.cuda.synchronize()
    ctx.close()
    return out


def reset_warm_start(vehicles):
    """Forget every vehicle's previous plan (before replaying a trace).  The
    clears run on the current stream and the server's streams do not wait for
    it, so this waits for the device before returning."""
    import torch
    for v in vehicles:
        v.prev.zero_()
        v.prev_H = 0
        v.busy = False
    torch.cuda.synchronize()
