"""Continuous-batching FBST server: requests of different arrays admitted by device memory, batched
as they arrive, overlapped on several CUDA streams, with every plan resident on the device.

A request is one block of N snapshots of one of the server's arrays (a plan). The loop:

* arrivals join a pending queue (arrival order);
* whenever a stream slot is free, the scheduler forms a batch from the pending queue in arrival
  order: requests whose array is already in an in-flight batch wait (a plan's workspace serves one
  batch at a time), at most `max_per_array` requests of one array go into a batch (the plan's
  block capacity), and admission stops at the first request whose device buffers (input + output)
  would exceed the memory budget or the batch's memory (one stream's arena), so large requests
  are not starved;
* the executor copies the batch's inputs into its stream's resident device arena, runs all its
  arrays in one grouped launch sequence (fbst_batch_enqueue; a batch of one request runs
  fbst_execute), copies the outputs into the stream's resident pinned host arena and records an
  event, all on one stream; batches on different streams overlap on the GPU. The arenas are sized
  from the device's free memory when the executor starts, and nothing is allocated in the loop;
* completions free the requests' memory and their arrays, and admit waiting work;
* a batch whose submission fails (a malformed request, an error of the library) is reported: its
  requests complete with `error` set and the loop goes on serving the others.

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
    error: str | None = None  # set when the request's batch could not be run


class Scheduler:
    """Admission by device memory and formation of batches (no GPU work)."""

    def __init__(self, req_bytes, mem_budget: int, max_per_array: int, req_work=None, max_batch_work=None,
                 max_batch_bytes=None):
        self.req_bytes = list(req_bytes)     # device bytes one request of array i holds while active
        self.mem_budget = int(mem_budget)
        self.max_per_array = int(max_per_array)
        # Optional cap on one batch's device bytes (the executor's per-stream arena).
        self.max_batch_bytes = max_batch_bytes
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
        batch, per_array, waiting, work, nbytes = [], {}, collections.deque(), 0, 0
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
            if batch and self.max_batch_bytes is not None and nbytes + self.req_bytes[a] > self.max_batch_bytes:
                waiting.append(r)
                break
            nbytes += self.req_bytes[a]
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
                try:
                    executor.submit(batch, now)
                except Exception as e:                  # report the batch, keep serving the rest
                    t = clock() - t0
                    for r in batch:
                        r.error = f"{type(e).__name__}: {e}"
                        r.t_done = t
                    scheduler.complete(batch)
                    done += len(batch)
    return summarize(requests, executor_units=getattr(executor, "units", None), batches=scheduler.batches,
                     peak_mem=scheduler.peak_mem)


def summarize(requests: list, executor_units=None, batches=None, peak_mem=None) -> dict:
    """Latency percentiles and throughput over the requests that were served (failed ones are
    counted apart)."""
    import numpy as np
    ok = [r for r in requests if r.error is None]
    lat = np.array([r.t_done - r.t_arrival for r in ok]) if ok else np.zeros(1)
    span = max(r.t_done for r in requests) - min(r.t_arrival for r in requests)
    out = {"requests": len(requests), "failed": len(requests) - len(ok),
           "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
           "span_s": float(span)}
    if executor_units is not None:
        units = sum(executor_units[r.array] for r in ok)
        out["beam_samples_per_s"] = float(units / span) if span > 0 else 0.0
    if batches is not None:
        out["batches"] = batches
        out["mean_batch"] = len(requests) / max(1, batches)
    if peak_mem is not None:
        out["peak_device_bytes"] = int(peak_mem)
    return out


class GPUExecutor:
    """Device side: one grouped launch sequence per batch on one of `n_streams` CUDA streams.

    Each stream owns a resident device arena and a resident pinned host arena of `arena_bytes`
    (default: a share of the device's free memory, at most 256 MiB); a batch's inputs, outputs and
    host copies of the outputs are carved from its stream's arenas, so the loop allocates nothing.
    `device_budget` is the memory the scheduler should admit against (all arenas)."""

    ALIGN = 256

    def __init__(self, plans, n_streams: int = 3, keep_outputs: bool = False, arena_bytes: int | None = None,
                 free_fraction: float = 0.25):
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
        if arena_bytes is None:
            free_bytes, _ = torch.cuda.mem_get_info()
            arena_bytes = min(256 << 20, int(free_bytes * free_fraction) // n_streams)
        self.arena_bytes = int(arena_bytes) // self.ALIGN * self.ALIGN
        self.dev_arena = [torch.empty(self.arena_bytes, dtype=torch.uint8, device="cuda") for _ in range(n_streams)]
        self.host_arena = [torch.empty(self.arena_bytes, dtype=torch.uint8).pin_memory() for _ in range(n_streams)]
        self.device_budget = self.arena_bytes * n_streams

    def request_bytes(self, a: int) -> int:
        """Device bytes of one request of array a in an arena (input and output block, aligned)."""
        M, N, B = self.dims[a]
        return self._aligned(8 * M * N) + self._aligned(8 * B * N)

    def _aligned(self, n: int) -> int:
        return (n + self.ALIGN - 1) // self.ALIGN * self.ALIGN

    def can_submit(self) -> bool:
        return bool(self.free)

    def _carve(self, arena, off: int, shape):
        n = 8 * shape[0] * shape[1] * shape[2]
        if off + n > self.arena_bytes:
            raise MemoryError(f"batch needs more than the {self.arena_bytes >> 20} MiB arena of a stream")
        return arena[off:off + n].view(self.torch.complex64).view(shape), off + self._aligned(n)

    def submit(self, batch: list, now: float) -> None:
        torch = self.torch
        si = self.free.pop(0)
        try:
            self._submit(si, batch)
        except Exception:
            self.free.insert(0, si)
            raise
        for r in batch:
            r.t_launch = now

    def _submit(self, si: int, batch: list) -> None:
        torch = self.torch
        st = self.streams[si]
        dev, host = self.dev_arena[si], self.host_arena[si]
        groups = collections.defaultdict(list)
        for r in batch:
            groups[r.array].append(r)
        n = len(self.plans)
        ys, outs, nb, hosts = [0] * n, [0] * n, [0] * n, []
        off = hoff = 0
        views = {}
        for a, rs in groups.items():
            M, N, B = self.dims[a]
            yd, off = self._carve(dev, off, (len(rs), M, N))
            od, off = self._carve(dev, off, (len(rs), B, N))
            oh, hoff = self._carve(host, hoff, (len(rs), B, N))
            for r in rs:
                if tuple(r.y.shape[-2:]) != (M, N):
                    raise ValueError(f"request {r.rid}: input {tuple(r.y.shape)} does not fit array {a} ({M}x{N})")
            views[a] = (yd, od, oh)
        with torch.cuda.stream(st):
            for a, rs in groups.items():
                yd, od, oh = views[a]
                for j, r in enumerate(rs):
                    yd[j].copy_(r.y.reshape(yd.shape[1:]), non_blocking=True)
                ys[a], outs[a], nb[a] = yd, od, len(rs)
            if len(batch) == 1:
                a = batch[0].array
                self.plans[a].execute(ys[a], outs[a], 1, st)
            else:
                self.batch.enqueue(ys, outs, nb, st)
            for a, rs in groups.items():
                yd, od, oh = views[a]
                oh.copy_(od, non_blocking=True)
                hosts += [(r, oh[j:j + 1]) for j, r in enumerate(rs)]
            ev = torch.cuda.Event()
            ev.record(st)
        self.inflight.append((si, ev, batch, hosts))

    def poll(self) -> list:
        done, still = [], []
        for item in self.inflight:
            si, ev, batch, hosts = item
            if ev.query():
                if self.keep:
                    for r, h in hosts:
                        r.out = h.clone()
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
