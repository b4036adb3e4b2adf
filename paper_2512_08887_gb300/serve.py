"""Continuous-batching FBST server: requests of different arrays admitted by device memory, batched
as they arrive, overlapped on several CUDA streams, with every plan resident on the device.

A request is one block of N snapshots of one of the server's arrays (a plan). The loop:

* arrivals join a pending queue (arrival order);
* whenever a stream slot is free, the scheduler forms a batch from the pending queue in arrival
  order: requests whose array is already in an in-flight batch wait (a plan's workspace serves one
  batch at a time), at most `max_per_array` requests of one array go into a batch (the plan's
  block capacity), and admission stops at the first request whose device buffers (input + output)
  would exceed the memory budget, so large requests are not starved;
* the executor copies the batch's inputs to the device, runs all its arrays in one grouped launch
  sequence (fbst_batch_enqueue; a batch of one request runs fbst_execute on the array's resident
  one-block buffers), copies the outputs back and records an event, all on one stream;
  batches on different streams overlap on the GPU;
* completions free the requests' memory and their arrays, and admit waiting work.

The scheduling policy (`Scheduler`) is plain Python and is tested on the CPU with a simulated
executor; `GPUExecutor` is the device side. `serve_plain` is the comparison: one request at a
time, three kernels per block (fbst_execute), in arrival order.
"""
from __future__ import annotations

import collections
import dataclasses
import time


@dataclasses.dataclass
class Request:
    rid: int
    array: int                # index of the array (plan) in the server's plan list
    y: object                 # host input block [1][M][N] complex64 (pinned torch tensor on a GPU)
    t_arrival: float          # seconds on the server clock
    t_admit: float | None = None
    t_launch: float | None = None
    t_done: float | None = None
    out: object = None        # host output block [1][B][N], filled on completion if kept
    batch_id: int = -1


class Scheduler:
    """Admission by device memory and formation of batches (no GPU work)."""

    def __init__(self, req_bytes, mem_budget: int, max_per_array: int, req_work=None, max_batch_work=None):
        self.req_bytes = list(req_bytes)     # device bytes one request of array i holds while active
        self.mem_budget = int(mem_budget)
        self.max_per_array = int(max_per_array)
        # Optional cap on the work of one batch (e.g. beam-samples): later requests wait for the
        # next stream slot, so a backlog becomes several pipelined batches instead of one long one.
        self.req_work = list(req_work) if req_work is not None else None
        self.max_batch_work = max_batch_work
        self.pending: collections.deque = collections.deque()
        self.mem_used = 0
        self.busy: set = set()
        self.peak_mem = 0
        self.batches = 0

    def arrive(self, req: Request) -> None:
        self.pending.append(req)

    def form_batch(self, now: float) -> list:
        batch, per_array, waiting, work = [], {}, collections.deque(), 0
        while self.pending:
            r = self.pending.popleft()
            a = r.array
            if a in self.busy or per_array.get(a, 0) >= self.max_per_array:
                waiting.append(r)
                continue
            if self.mem_used + self.req_bytes[a] > self.mem_budget:
                waiting.append(r)
                break                                   # first-come first-served on memory
            if batch and self.max_batch_work is not None and work + self.req_work[a] > self.max_batch_work:
                waiting.append(r)
                break
            if self.req_work is not None:
                work += self.req_work[a]
            per_array[a] = per_array.get(a, 0) + 1
            self.mem_used += self.req_bytes[a]
            r.t_admit = now
            r.batch_id = self.batches
            batch.append(r)
        waiting.extend(self.pending)
        self.pending = waiting
        if batch:
            self.busy.update(per_array)
            self.batches += 1
            self.peak_mem = max(self.peak_mem, self.mem_used)
        return batch

    def complete(self, batch: list) -> None:
        for r in batch:
            self.mem_used -= self.req_bytes[r.array]
        self.busy.difference_update({r.array for r in batch})


def run_loop(requests: list, scheduler: Scheduler, executor, clock=time.perf_counter) -> dict:
    """Serve `requests` (sorted by t_arrival) until all complete; returns summary statistics."""
    t0 = clock()
    n, i, done = len(requests), 0, 0
    while done < n:
        now = clock() - t0
        while i < n and requests[i].t_arrival <= now:
            scheduler.arrive(requests[i])
            i += 1
        for batch in executor.poll():
            t = clock() - t0
            for r in batch:
                r.t_done = t
            scheduler.complete(batch)
            done += len(batch)
        if executor.can_submit() and scheduler.pending:
            batch = scheduler.form_batch(now)
            if batch:
                executor.submit(batch, now)
    return summarize(requests, executor_units=getattr(executor, "units", None), batches=scheduler.batches,
                     peak_mem=scheduler.peak_mem)


def summarize(requests: list, executor_units=None, batches=None, peak_mem=None) -> dict:
    import numpy as np
    lat = np.array([r.t_done - r.t_arrival for r in requests])
    span = max(r.t_done for r in requests) - min(r.t_arrival for r in requests)
    out = {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
           "span_s": float(span)}
    if executor_units is not None:
        units = sum(executor_units[r.array] for r in requests)
        out["beam_samples_per_s"] = float(units / span)
    if batches is not None:
        out["batches"] = batches
        out["mean_batch"] = len(requests) / max(1, batches)
    if peak_mem is not None:
        out["peak_device_bytes"] = int(peak_mem)
    return out


class GPUExecutor:
    """Device side: one grouped launch sequence per batch on one of `n_streams` CUDA streams."""

    def __init__(self, plans, n_streams: int = 3, keep_outputs: bool = False):
        import torch
        from ._native import Batch
        self.torch = torch
        self.plans = list(plans)
        self.batch = Batch(self.plans)
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.free = list(range(n_streams))
        self.inflight = []
        self.keep = keep_outputs
        self.dims = [(p.M, p.N, p.B) for p in self.plans]
        self.units = [p.B * p.N for p in self.plans]
        self.out_pool = collections.defaultdict(list)   # pinned host output buffers per array
        # One-block device buffers per array for single-request batches. The scheduler never has
        # two batches of the same array in flight, so they are never used twice at once.
        self.single = {}

    def can_submit(self) -> bool:
        return bool(self.free)

    def _out_buffer(self, a: int):
        if self.out_pool[a]:
            return self.out_pool[a].pop()
        M, N, B = self.dims[a]
        return self.torch.empty((1, B, N), dtype=self.torch.complex64).pin_memory()

    def _submit_single(self, r, st):
        """One request: fbst_execute on the array's resident one-block buffers (no grouping)."""
        torch = self.torch
        a = r.array
        if a not in self.single:
            M, N, B = self.dims[a]
            self.single[a] = (torch.empty((1, M, N), dtype=torch.complex64, device="cuda"),
                              torch.empty((1, B, N), dtype=torch.complex64, device="cuda"))
        yd, od = self.single[a]
        yd.copy_(r.y, non_blocking=True)
        self.plans[a].execute(yd, od, 1, st)
        h = self._out_buffer(a)
        h.copy_(od, non_blocking=True)
        return [], [(r, h)]

    def submit(self, batch: list, now: float) -> None:
        torch = self.torch
        si = self.free.pop(0)
        st = self.streams[si]
        if len(batch) == 1:
            with torch.cuda.stream(st):
                keep, hosts = self._submit_single(batch[0], st)
                ev = torch.cuda.Event()
                ev.record(st)
            batch[0].t_launch = now
            self.inflight.append((si, ev, batch, keep, hosts))
            return
        groups = collections.defaultdict(list)
        for r in batch:
            groups[r.array].append(r)
        n = len(self.plans)
        ys, outs, nb, keep, hosts = [0] * n, [0] * n, [0] * n, [], []
        with torch.cuda.stream(st):
            for a, rs in groups.items():
                M, N, B = self.dims[a]
                yd = torch.empty((len(rs), M, N), dtype=torch.complex64, device="cuda")
                od = torch.empty((len(rs), B, N), dtype=torch.complex64, device="cuda")
                for j, r in enumerate(rs):
                    yd[j].copy_(r.y[0], non_blocking=True)
                ys[a], outs[a], nb[a] = yd, od, len(rs)
                keep += [yd, od]
            self.batch.enqueue(ys, outs, nb, st)
            for a, rs in groups.items():
                for j, r in enumerate(rs):
                    h = self._out_buffer(a)
                    h.copy_(outs[a][j:j + 1], non_blocking=True)
                    hosts.append((r, h))
            ev = torch.cuda.Event()
            ev.record(st)
        for r in batch:
            r.t_launch = now
        self.inflight.append((si, ev, batch, keep, hosts))

    def poll(self) -> list:
        done, still = [], []
        for item in self.inflight:
            si, ev, batch, keep, hosts = item
            if ev.query():
                for r, h in hosts:
                    if self.keep:
                        r.out = h.clone()
                    self.out_pool[r.array].append(h)
                self.free.append(si)
                done.append(batch)
            else:
                still.append(item)
        self.inflight = still
        return done

    def close(self) -> None:
        self.torch.cuda.synchronize()
        self.batch.close()


def serve_plain(requests: list, plans, keep_outputs: bool = False, clock=time.perf_counter) -> dict:
    """Comparison server: one request at a time in arrival order, fbst_execute per block."""
    import torch
    dev_in = [torch.empty((1, p.M, p.N), dtype=torch.complex64, device="cuda") for p in plans]
    dev_out = [torch.empty((1, p.B, p.N), dtype=torch.complex64, device="cuda") for p in plans]
    host_out = [torch.empty((1, p.B, p.N), dtype=torch.complex64).pin_memory() for p in plans]
    t0 = clock()
    for r in requests:
        while clock() - t0 < r.t_arrival:
            pass
        a = r.array
        r.t_admit = r.t_launch = clock() - t0
        dev_in[a].copy_(r.y, non_blocking=True)
        plans[a].execute(dev_in[a], dev_out[a], 1)
        host_out[a].copy_(dev_out[a], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        r.t_done = clock() - t0
        if keep_outputs:
            r.out = host_out[a].clone()
    return summarize(requests, executor_units=[p.B * p.N for p in plans])


def poisson_requests(rate: float, count: int, arrays: list, seed: int) -> list:
    """`count` requests with exponential inter-arrival times at `rate` per second; request k uses
    array arrays_choice[k] drawn uniformly; `arrays` holds, per array, a list of host input blocks
    that the requests cycle through."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    which = rng.integers(0, len(arrays), count)
    reqs, used = [], collections.Counter()
    for k in range(count):
        a = int(which[k])
        pool = arrays[a]
        reqs.append(Request(k, a, pool[used[a] % len(pool)], float(t[k])))
        used[a] += 1
    return reqs
