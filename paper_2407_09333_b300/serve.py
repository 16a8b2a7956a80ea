"""Continuous-batching hash server on one GPU.

Requests (one algorithm each, 1..4096 messages) arrive over time.  The
server keeps every admitted request's bytes in a device arena whose size is
the memory budget; a request is admitted (first come, first served) as soon
as its bytes fit, and waits otherwise.  Up to `slots` batches are on the GPU
at once, each slot with its own CUDA stream, its own ragged-path plan
(private bucketing scratch) and a CUDA graph captured once over the slot's
fixed metadata and digest buffers.  Whenever a slot is free, every admitted
request that is not yet on the GPU is packed into one batch:

  1. the batch's metadata (message offsets into the arena, lengths,
     algorithm codes) and the request copy records go to the device in one
     host-to-device copy per section;
  2. one gather kernel moves the requests' bytes into their arena places;
  3. the slot's graph hashes the batch (longest-first chunks, persistent);
  4. the digest slots come back to pinned host memory; an event marks the end.

A request is finished as soon as the kernel raises its done flag (host
memory the device writes after the request's last message): its latency
(completion minus arrival) is recorded and its arena space is released,
which lets waiting requests in, while longer requests of the same batch are
still running.  A slot is free again when its batch's event has completed;
requests that arrive meanwhile join the next batch on another slot and run
concurrently with the earlier ones.

The arena bookkeeping (`Arena`) and the admission/batching policy
(`Scheduler`) are plain Python and testable without a GPU; `Server` adds the
device work.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

ALIGN = 256


class Arena:
    """First-fit allocator over [0, capacity) in ALIGN-byte units."""

    def __init__(self, capacity: int, align: int = ALIGN):
        self.capacity = int(capacity) // align * align
        self.align = align
        self.free = [(0, self.capacity)]  # sorted, coalesced (start, size)
        self.used = 0
        self.peak = 0

    def round(self, size: int) -> int:
        return max(self.align, (int(size) + self.align - 1) // self.align * self.align)

    def alloc(self, size: int):
        """(start, rounded size), or None when no free range is large enough."""
        size = self.round(size)
        for i, (st, sz) in enumerate(self.free):
            if sz >= size:
                if sz == size:
                    del self.free[i]
                else:
                    self.free[i] = (st + size, sz - size)
                self.used += size
                self.peak = max(self.peak, self.used)
                return st, size
        return None

    def release(self, start: int, size: int):
        lo, hi = 0, len(self.free)
        while lo < hi:
            mid = (lo + hi) // 2
            if self.free[mid][0] < start:
                lo = mid + 1
            else:
                hi = mid
        self.free.insert(lo, (start, size))
        # coalesce with the neighbours
        if lo + 1 < len(self.free) and self.free[lo][0] + self.free[lo][1] == self.free[lo + 1][0]:
            self.free[lo] = (self.free[lo][0], self.free[lo][1] + self.free[lo + 1][1])
            del self.free[lo + 1]
        if lo > 0 and self.free[lo - 1][0] + self.free[lo - 1][1] == self.free[lo][0]:
            self.free[lo - 1] = (self.free[lo - 1][0], self.free[lo - 1][1] + self.free[lo][1])
            del self.free[lo]
        self.used -= size


@dataclasses.dataclass
class Req:
    rid: int
    arrival: float               # seconds since the start of the run
    alg: int
    lengths: np.ndarray          # uint32 per message
    segments: list               # [(pool offset, bytes)] whose concatenation is the payload
    nbytes: int = 0
    local_offsets: np.ndarray | None = None
    arena: tuple | None = None   # (start, rounded size) once admitted
    admitted: float = -1.0
    done: float = -1.0
    digests: np.ndarray | None = None

    def __post_init__(self):
        self.lengths = np.asarray(self.lengths, dtype=np.uint32)
        self.nbytes = int(self.lengths.astype(np.uint64).sum())
        offs = np.zeros(self.lengths.shape[0], dtype=np.uint64)
        if self.lengths.shape[0]:
            offs[1:] = np.cumsum(self.lengths.astype(np.uint64))[:-1]
        self.local_offsets = offs


class Scheduler:
    """Admission and batching policy, independent of the device.

    `arrive` queues a request; `admit` moves queued requests (in arrival
    order) into the arena while they fit -- a request larger than the whole
    budget is rejected; `next_batch` hands every admitted, not yet launched
    request to a free slot, up to max_msgs messages and max_reqs requests;
    `finish` releases a batch's arena space.
    """

    def __init__(self, budget: int, max_msgs: int, max_reqs: int):
        self.arena = Arena(budget)
        self.max_msgs = max_msgs
        self.max_reqs = max_reqs
        self.waiting = collections.deque()
        self.ready = collections.deque()
        self.rejected = []

    def arrive(self, req: Req):
        self.waiting.append(req)

    def admit(self, now: float) -> int:
        n = 0
        while self.waiting:
            req = self.waiting[0]
            if self.arena.round(req.nbytes) > self.arena.capacity or \
                    req.lengths.shape[0] > self.max_msgs:
                self.waiting.popleft()
                self.rejected.append(req)
                continue
            got = self.arena.alloc(req.nbytes)
            if got is None:
                break  # first come, first served: wait for space
            self.waiting.popleft()
            req.arena = got
            req.admitted = now
            self.ready.append(req)
            n += 1
        return n

    def next_batch(self) -> list:
        batch, msgs = [], 0
        while self.ready and len(batch) < self.max_reqs:
            m = int(self.ready[0].lengths.shape[0])
            if batch and msgs + m > self.max_msgs:
                break
            batch.append(self.ready.popleft())
            msgs += m
        return batch

    def finish(self, batch: list):
        for req in batch:
            self.arena.release(*req.arena)
            req.arena = None


class _Slot:
    def __init__(self, server, max_msgs: int, max_reqs: int):
        torch, api = server.torch, server.api
        dev = server.device
        self.stream = torch.cuda.Stream(device=dev)
        self.plan = api.Plan(max_msgs, shape=server.shape, warps_per_sm=server.warps_per_sm)
        self.d_algs = torch.zeros(max_msgs, dtype=torch.uint8, device=dev)
        self.d_offsets = torch.zeros(max_msgs, dtype=torch.int64, device=dev)
        self.d_lengths = torch.zeros(max_msgs, dtype=torch.int32, device=dev)
        self.d_digests = torch.zeros((max_msgs, 32), dtype=torch.uint8, device=dev)
        self.d_copies = torch.zeros((max_reqs * 4, 3), dtype=torch.int64, device=dev)
        self.h_algs = torch.zeros(max_msgs, dtype=torch.uint8).pin_memory()
        self.h_offsets = torch.zeros(max_msgs, dtype=torch.int64).pin_memory()
        self.h_lengths = torch.zeros(max_msgs, dtype=torch.int32).pin_memory()
        self.h_copies = torch.zeros((max_reqs * 4, 3), dtype=torch.int64).pin_memory()
        self.h_digests = torch.zeros((max_msgs, 32), dtype=torch.uint8).pin_memory()
        # per-request completion: message -> request, messages left, done flags
        self.d_msg_req = torch.zeros(max_msgs, dtype=torch.int32, device=dev)
        self.d_remaining = torch.zeros(max_reqs, dtype=torch.int32, device=dev)
        self.h_msg_req = torch.zeros(max_msgs, dtype=torch.int32).pin_memory()
        self.h_remaining = torch.zeros(max_reqs, dtype=torch.int32).pin_memory()
        self.h_done = torch.zeros(max_reqs, dtype=torch.int32).pin_memory()
        self.done_np = self.h_done.numpy()
        self.plan.set_completion(self.d_msg_req, self.d_remaining, self.h_done)
        self.plan.capture(self.d_algs, server.arena_dev, self.d_offsets, self.d_lengths,
                          self.d_digests, grid=server.grid)
        self.event = torch.cuda.Event()
        self.batch = None
        self.open = None   # indices of the batch's requests not yet finished
        self.nmsgs = 0


class Server:
    """The device side: arena tensor, payload pool, slots."""

    def __init__(self, pool, budget: int = 8 << 30, slots: int = 16, max_msgs: int = 1 << 17,
                 max_reqs: int = 512, grid: int = 0, shape: int = 18, warps_per_sm: int = 4,
                 min_batch_bytes: int = 0, max_wait_ms: float = 0.0, device="cuda"):
        import torch
        from . import api
        self.torch, self.api, self.device = torch, api, device
        self.pool = pool                                     # device uint8 tensor
        self.pool_addr = pool.data_ptr()
        self.sched = Scheduler(budget, max_msgs, max_reqs)
        self.arena_dev = torch.empty(self.sched.arena.capacity, dtype=torch.uint8, device=device)
        self.arena_addr = self.arena_dev.data_ptr()
        # One-warp blocks: a warp that runs out of chunks leaves at once and
        # frees its SM resources for other batches, while warps holding long
        # serial chains keep running.
        self.grid = grid
        self.shape = shape
        self.warps_per_sm = warps_per_sm
        # Batch formation: a free slot takes the admitted requests at once
        # when nothing else is running, when they hold min_batch_bytes, or
        # when the oldest of them has waited max_wait_ms; otherwise it waits
        # for more (every batch lasts at least its longest serial chain, so
        # larger batches carry more bytes per slot-time).
        self.min_batch_bytes = min_batch_bytes
        self.max_wait_s = max_wait_ms * 1e-3
        self.slots = [_Slot(self, max_msgs, max_reqs) for _ in range(slots)]
        self.batches = 0
        self.batched_reqs = 0

    def _launch(self, slot: _Slot, batch: list):
        torch, api = self.torch, self.api
        n = 0
        c = 0
        slot.done_np[:len(batch)] = 0
        for j, req in enumerate(batch):
            m = int(req.lengths.shape[0])
            base = req.arena[0]
            slot.h_offsets.numpy()[n:n + m] = (req.local_offsets + np.uint64(base)).view(np.int64)
            slot.h_lengths.numpy()[n:n + m] = req.lengths.view(np.int32)
            slot.h_algs.numpy()[n:n + m] = req.alg
            slot.h_msg_req.numpy()[n:n + m] = j
            slot.h_remaining.numpy()[j] = m
            dst = self.arena_addr + base
            for off, ln in req.segments:
                slot.h_copies.numpy()[c] = (self.pool_addr + off, dst, ln)
                dst += ln
                c += 1
            n += m
        with torch.cuda.stream(slot.stream):
            slot.d_offsets[:n].copy_(slot.h_offsets[:n], non_blocking=True)
            slot.d_lengths[:n].copy_(slot.h_lengths[:n], non_blocking=True)
            slot.d_algs[:n].copy_(slot.h_algs[:n], non_blocking=True)
            slot.d_copies[:c].copy_(slot.h_copies[:c], non_blocking=True)
            slot.d_msg_req[:n].copy_(slot.h_msg_req[:n], non_blocking=True)
            slot.d_remaining[:len(batch)].copy_(slot.h_remaining[:len(batch)], non_blocking=True)
            api.gather(slot.d_copies, c, stream=slot.stream)
            slot.plan.replay(n, stream=slot.stream)
            slot.h_digests[:n].copy_(slot.d_digests[:n], non_blocking=True)
            slot.event.record(slot.stream)
        slot.batch = batch
        slot.open = list(range(len(batch)))
        slot.nmsgs = n
        self.batches += 1
        self.batched_reqs += len(batch)

    def _batch_due(self, now: float) -> bool:
        if self.min_batch_bytes <= 0 and self.max_wait_s <= 0:
            return True
        if all(slot.batch is None for slot in self.slots):
            return True
        ready = self.sched.ready
        if now - ready[0].admitted >= self.max_wait_s > 0:
            return True
        return sum(r.nbytes for r in ready) >= self.min_batch_bytes > 0

    def _poll_requests(self, slot: _Slot, now: float) -> int:
        """Finish the requests whose done flag the kernel has raised: their
        arena space is free again even though the batch is still running."""
        count = 0
        still = []
        for j in slot.open:
            if slot.done_np[j]:
                req = slot.batch[j]
                req.done = now
                self.sched.arena.release(*req.arena)
                req.arena = None
                count += 1
            else:
                still.append(j)
        slot.open = still
        return count

    def _complete(self, slot: _Slot, now: float, keep_digests: bool) -> int:
        count = self._poll_requests(slot, now)
        for j in slot.open:   # flags read before the event completed
            req = slot.batch[j]
            if req.done < 0:
                req.done = now
            self.sched.arena.release(*req.arena)
            req.arena = None
            count += 1
        if keep_digests:
            n = 0
            digests = slot.h_digests.numpy()
            for req in slot.batch:
                m = int(req.lengths.shape[0])
                req.digests = digests[n:n + m].copy()
                n += m
        slot.batch = None
        slot.open = None
        return count

    def run(self, requests: list, keep_digests: bool = False, time_limit_s: float = 600.0):
        """Serve `requests` (sorted by arrival) in real time; returns them,
        finished (done >= 0) or rejected."""
        torch = self.torch
        torch.cuda.synchronize()
        sched = self.sched
        nreq = len(requests)
        finished = 0
        i = 0
        t0 = time.perf_counter()
        while finished + len(sched.rejected) < nreq:
            now = time.perf_counter() - t0
            if now > time_limit_s:
                raise RuntimeError("serving run exceeded %.0f s" % time_limit_s)
            while i < nreq and requests[i].arrival <= now:
                sched.arrive(requests[i])
                i += 1
            for slot in self.slots:
                if slot.batch is None:
                    continue
                if slot.event.query():
                    finished += self._complete(slot, time.perf_counter() - t0, keep_digests)
                elif slot.open:
                    finished += self._poll_requests(slot, time.perf_counter() - t0)
            sched.admit(time.perf_counter() - t0)
            if sched.ready and self._batch_due(time.perf_counter() - t0):
                for slot in self.slots:
                    if slot.batch is None and sched.ready:
                        self._launch(slot, sched.next_batch())
        # every request is finished; let the last batches end (their digests
        # come back with the batch)
        for slot in self.slots:
            if slot.batch is not None:
                slot.event.synchronize()
                self._complete(slot, time.perf_counter() - t0, keep_digests)
        torch.cuda.synchronize()
        return requests

    def close(self):
        for slot in self.slots:
            slot.plan.close()


# ---------------------------------------------------------------------------
# synthetic load

def make_requests(count: int, rate_per_s: float, seed: int, pool_bytes: int,
                  max_msgs: int = 4096, min_len: int = 16, max_len: int = 1 << 20) -> list:
    """Poisson request stream; each request's payload is a (wrapped) range of
    the random-byte pool, chosen by its seed, starting 16-byte aligned."""
    from . import workloads
    out = []
    for k, r in enumerate(workloads.serve_requests(count, rate_per_s, seed, max_msgs, min_len, max_len)):
        req = Req(k, r.arrival_s, r.alg, r.lengths, [])
        rng = np.random.Generator(np.random.PCG64(r.seed))
        left = req.nbytes
        off = int(rng.integers(0, max(pool_bytes - 16, 1))) // 16 * 16
        while left > 0:
            take = min(left, pool_bytes - off)
            req.segments.append((off, take))
            left -= take
            off = 0
        out.append(req)
    return out


def latency_stats(requests: list) -> dict:
    done = [r for r in requests if r.done >= 0]
    if not done:
        return {"completed": 0}
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    nbytes = sum(r.nbytes for r in done)
    t_end = max(r.done for r in done)
    t_start = min(r.arrival for r in done)
    return {"completed": len(done), "rejected": len(requests) - len(done),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "gbs": nbytes / max(t_end - t_start, 1e-9) / 1e9,
            "bytes": nbytes, "span_s": t_end - t_start}
