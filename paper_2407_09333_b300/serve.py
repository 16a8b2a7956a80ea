"""Continuous-batching hash server on one GPU, streaming long messages.

Requests (one algorithm each, 1..4096 messages of up to 1 MiB) arrive over
time.  A message is a serial chain of compressions (the Merkle-Damgard
iteration of RFC 1321 Sec. 3.4, FIPS 180-4 Sec. 6, GB/T 32905 Sec. 5.3):
a 1 MiB SM3 message takes tens of milliseconds however many SMs are free.  A
server that held each admitted request's bytes in device memory until its
last message finished would tie its memory budget to those chains; this one
streams every message through the device in segments (`segment_bytes`, per
algorithm) instead, keeping only each message's 32-byte chaining value between them
("state kept on device").

Device side (one budget, fixed at start):
  * a ring of message entries (source address, length, progress, request,
    algorithm, state, 32-byte slot) and per-request counters;
  * `rounds` streaming rounds (hash_round_* in the C-ABI), each with its own
    CUDA stream, staging area and captured graph.  A round claims the oldest
    ready messages, copies their next segments into its staging area, hashes
    them with the ragged path and advances them; a message whose last
    segment is hashed leaves its digest in its slot, and the last message of
    a request raises the request's done flag in host memory.
Rounds run concurrently on their streams, so the copies and the hashing of
different rounds overlap, and a message's next segment goes to whichever
round is free next.

With `in_place=True` a round skips the copy and hashes each segment where
the client's bytes are; the staging budget then only caps the bytes the
rounds have claimed at a time (the server owns no copy of the payload).

Host ingress: when the clients' pool is pinned host memory, the rounds'
copy step brings each segment over the bus into the staging area as the
segment's turn comes (the device never holds a whole request), so the
device budget bounds the segments in flight and the bus bounds throughput.

Host side (this module, plain Python): admission in arrival order while the
ring and the request table have room (`RingBook`), one batch of metadata
copies per loop for the newly admitted requests, round launches, and the
done flags.  Digests stay on the device; `keep_digests` copies each request's
digests out when it completes (for tests).

Admission by predicted time (`Admission`, optional): the fitted cost model
(costmodel: Eq. 2's linear form plus the serial-chain bound) gives each
request a predicted completion time when it is admitted; the server can hold
requests on the host while the predicted in-flight work exceeds a cap, and
shed a request at arrival when its predicted latency exceeds a target.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import time

import numpy as np

RING_ENTRY_BYTES = 8 + 8 + 4 + 4 + 1 + 4 + 32      # src, prior, len, req, alg, state, slot
ROUND_ENTRY_BYTES = 1 + 8 + 4 + 8 + 4 + 24 + 4     # batch arrays, copy record, permutation


class RingBook:
    """Bookkeeping of the message ring and the request table.

    Messages take consecutive ring positions (counters modulo `capacity`);
    requests take consecutive request slots (modulo `req_capacity`).  A
    request is admitted when both have room; positions are reused once every
    earlier request has finished (the head only moves past finished
    requests, in admission order).
    """

    def __init__(self, capacity: int, req_capacity: int):
        if capacity & (capacity - 1) or req_capacity & (req_capacity - 1):
            raise ValueError("capacities must be powers of two")
        self.capacity = capacity
        self.req_capacity = req_capacity
        self.head = self.tail = 0          # message counters
        self.req_head = self.req_tail = 0  # request counters
        self.open = collections.deque()    # [req counter, first, m, finished]
        self.by_req = {}

    def fits(self, m: int) -> bool:
        return (self.tail + m - self.head <= self.capacity and
                self.req_tail + 1 - self.req_head <= self.req_capacity)

    def admit(self, m: int) -> tuple[int, int]:
        """(request counter, first message counter) of a request of m messages."""
        if not self.fits(m):
            raise ValueError("no room")
        rc, first = self.req_tail, self.tail
        self.req_tail += 1
        self.tail += m
        ent = [rc, first, m, False]
        self.open.append(ent)
        self.by_req[rc] = ent
        return rc, first

    def finish(self, rc: int):
        self.by_req.pop(rc)[3] = True
        while self.open and self.open[0][3]:
            _, _, m, _ = self.open.popleft()
            self.head += m
            self.req_head += 1

    def spans(self, first: int, count: int, capacity: int | None = None) -> list:
        """[(ring position, offset into the run, length)] of counters
        [first, first + count), split where the ring wraps."""
        cap = capacity or self.capacity
        out, done = [], 0
        while done < count:
            pos = (first + done) % cap
            take = min(count - done, cap - pos)
            out.append((pos, done, take))
            done += take
        return out


@dataclasses.dataclass
class Req:
    rid: int
    arrival: float               # seconds since the start of the run
    alg: int
    lengths: np.ndarray          # uint32 per message
    src: np.ndarray              # uint64 pool offset of each message
    nbytes: int = 0
    counter: int = -1            # request counter once admitted
    first: int = -1              # first message counter once admitted
    admitted: float = -1.0
    done: float = -1.0
    digests: np.ndarray | None = None
    rejected: bool = False       # shed at arrival by the admission policy
    work_s: float = 0.0          # predicted GPU-seconds (Admission)
    chain_s: float = 0.0         # predicted longest serial chain (Admission)
    predicted_done: float = -1.0 # predicted completion time, set at admission
    chain_bound: bool = False    # the prediction was set by the longest chain

    def __post_init__(self):
        self.lengths = np.asarray(self.lengths, dtype=np.uint32)
        self.src = np.asarray(self.src, dtype=np.uint64)
        self.nbytes = int(self.lengths.astype(np.uint64).sum())


class Admission:
    """Admission of requests by predicted completion time.

    The GPU is modelled as one work-conserving server: an admitted request
    adds its predicted GPU-seconds (`model.work_seconds`: the fitted
    throughput and per-message terms) to a backlog that drains at `drain`
    GPU-seconds per second while requests are in flight -- 1 if serving ran
    at the fitted launches' rate; the served path's own rate is lower
    (rounds, segments, the tails of serial chains), and `drain` is that ratio
    measured on a burst of requests (`calibrate_drain`).  A request admitted
    at time t is predicted to finish at

        t + max(backlog(t) + work / drain, chain) + t0

    -- after the work admitted before it and its own, and not before its
    longest message's serial chain (`model.chain_time`); t0 is the fixed
    cost of a request (admission copies, the rounds' cadence).

    Policies (both optional):
      cap_s  hold: while the backlog exceeds cap_s GPU-seconds and something
             is in flight, waiting requests stay on the host (in arrival
             order), so the device holds only the work that keeps it busy
             and the predicted order of completion is the admission order;
      slo_s  shed: at arrival, a request whose predicted completion --
             counted from its arrival, after the backlog and the work of the
             requests still waiting ahead of it -- would exceed slo_s is
             rejected at once instead of queued.

    The chain term follows the load: a chain shares its SM sub-partition with
    more busy warps when the device is fuller, so every request that finishes
    with a chain-bound prediction updates a running factor (`chain_scale`,
    exponentially weighted, weight `adapt`) by its measured chain time over
    the model's; later predictions use the model's chain times times that
    factor.  adapt = 0 keeps the model's chain times.

    Time is whatever clock the caller passes (seconds), so the policy runs
    under a fake clock in tests.
    """

    def __init__(self, model, cap_s: float | None = None, slo_s: float | None = None,
                 t0: float | None = None, drain: float = 1.0, adapt: float = 0.05):
        if drain <= 0:
            raise ValueError("drain must be positive")
        self.model = model
        self.cap_s = cap_s
        self.slo_s = slo_s
        self.drain = drain
        self.adapt = adapt
        self.chain_scale = 1.0
        self.t0 = float(getattr(model, "latency_t0", 0.0)) if t0 is None else t0
        self._backlog = 0.0
        self._t = 0.0
        self.inflight = 0
        self.waiting_s = 0.0       # predicted work of requests waiting to be admitted

    def estimate(self, req):
        """(work seconds at the served rate, chain seconds) of a request,
        also stored on it."""
        work, req.chain_s = self.model.request_costs(req.lengths, req.alg)
        req.work_s = work / self.drain
        return req.work_s, req.chain_s

    def backlog(self, now: float) -> float:
        """Predicted seconds of admitted work not yet done at `now`."""
        if now > self._t:
            if self.inflight:
                self._backlog = max(0.0, self._backlog - (now - self._t))
            self._t = now
        return self._backlog

    def predicted_latency(self, req, now: float) -> float:
        """Latency from arrival if the request joined the queue at `now`."""
        ahead = self.backlog(now) + self.waiting_s
        return (now - req.arrival) + max(ahead + req.work_s, self.chain_scale * req.chain_s) + self.t0

    def arrive(self, req, now: float) -> bool:
        """False when the request is shed; otherwise it waits for admission."""
        self.estimate(req)
        if self.slo_s is not None and self.predicted_latency(req, now) > self.slo_s:
            req.rejected = True
            return False
        self.waiting_s += req.work_s
        return True

    def hold(self, now: float) -> bool:
        """Whether waiting requests should stay on the host for now."""
        return (self.cap_s is not None and self.inflight > 0
                and self.backlog(now) > self.cap_s)

    def admit(self, req, now: float):
        b = self.backlog(now)
        chain = self.chain_scale * req.chain_s
        req.predicted_done = now + max(b + req.work_s, chain) + self.t0
        req.chain_bound = chain > b + req.work_s
        self._backlog = b + req.work_s
        self.waiting_s = max(0.0, self.waiting_s - req.work_s)
        self.inflight += 1

    def finish(self, req, now: float):
        self.backlog(now)
        self.inflight -= 1
        if self.inflight == 0:
            self._backlog = 0.0    # nothing in flight: the device is idle
        if self.adapt > 0 and getattr(req, "chain_bound", False) and req.chain_s > 0:
            seen = (now - req.admitted - self.t0) / req.chain_s
            seen = min(max(seen, 0.25), 8.0)
            self.chain_scale += self.adapt * (seen - self.chain_scale)


def calibrate_drain(model, requests: list) -> float:
    """The served path's rate relative to the model's, from requests served
    in one burst (all arriving at once, so the device never idles): bytes of
    the requests finishing between the 10th and 90th percentile of finishing
    times, over that interval, against the bytes per second the model's
    throughput terms predict for the same requests."""
    done = [r for r in requests if r.done >= 0]
    if len(done) < 10:
        raise ValueError("too few finished requests")
    fin = np.array([r.done for r in done])
    t10, t90 = np.percentile(fin, [10, 90])
    mid = [r for r in done if t10 < r.done <= t90]
    if t90 <= t10 or not mid:
        raise ValueError("finishing times too close together")
    served = sum(r.nbytes for r in mid) / (t90 - t10)
    work = sum(model.work_seconds(r.lengths, r.alg) for r in done)
    modelled = sum(r.nbytes for r in done) / work
    return served / modelled


def prediction_stats(requests: list) -> dict:
    """Predicted against measured completion of the served requests: the
    median ratio of measured to predicted latency (from arrival) and the
    share of requests within 25% of their prediction."""
    done = [r for r in requests if r.done >= 0 and r.predicted_done >= 0]
    if not done:
        return {"requests": 0}
    pred = np.array([r.predicted_done - r.arrival for r in done])
    meas = np.array([r.done - r.arrival for r in done])
    ratio = meas / np.maximum(pred, 1e-9)
    return {"requests": len(done), "median_measured_over_predicted": float(np.median(ratio)),
            "p10_ratio": float(np.percentile(ratio, 10)), "p90_ratio": float(np.percentile(ratio, 90)),
            "within_25pct": float(np.mean(np.abs(ratio - 1.0) <= 0.25)),
            "p99_predicted_ms": float(np.percentile(pred, 99) * 1e3)}


def device_bytes(capacity: int, req_capacity: int, rounds: int, max_msgs: int) -> int:
    """Device memory of everything but the staging areas."""
    groups = 3 * 32 * 64                        # (cost bucket, algorithm) groups
    ws = 4 * (2 * groups + 32) + 4 * (max_msgs + 31 * groups)
    return capacity * RING_ENTRY_BYTES + req_capacity * 4 + rounds * (
        max_msgs * ROUND_ENTRY_BYTES + ws + 256)


class _RoundSlot:
    def __init__(self, server, staging, nbytes):
        torch, api = server.torch, server.api
        self.stream = torch.cuda.Stream(device=server.device)
        self.round = api.Round(server.ring, server.max_msgs, staging, nbytes,
                               server.segment_bytes, server.shape, server.warps_per_sm)
        self.event = torch.cuda.Event()
        self.busy = False
        self.again = False   # its last launch claimed work: launch it again


class Server:
    """Streaming server: ring, rounds and the host loop."""

    # Segments per algorithm (MD5, SHA-1, SM3): about the same chain time each
    # (an SM3 block costs about three MD5 blocks and two SHA-1 blocks).
    DEFAULT_SEGMENTS = (96 << 10, 64 << 10, 32 << 10)

    def __init__(self, pool, budget: int = 8 << 30, rounds: int = 2,
                 segment_bytes=DEFAULT_SEGMENTS, max_msgs: int = 1 << 17,
                 capacity: int = 1 << 21, req_capacity: int = 1 << 14,
                 shape: int = 11, warps_per_sm: int = 8, in_place: bool = True,
                 device="cuda"):
        import torch
        from . import api
        self.torch, self.api, self.device = torch, api, device
        # the clients' bytes: a device tensor, or pinned host memory (host
        # ingress: each round's copy step reads its segments over the bus, so
        # only segments, never whole requests, occupy device memory)
        self.pool = pool
        self.host_ingress = not pool.is_cuda
        if self.host_ingress:
            if not pool.is_pinned():
                raise ValueError("a host pool must be pinned memory")
            if in_place:
                raise ValueError("a host pool is served through the staging copy (in_place=False)")
        # with unified addressing, pinned host memory has the same address on
        # the device as on the host
        self.pool_addr = pool.data_ptr()
        self.max_msgs = max_msgs
        self.shape = shape
        self.warps_per_sm = warps_per_sm
        if isinstance(segment_bytes, int):
            segment_bytes = (segment_bytes,) * 3
        self.segment_bytes = tuple(int(x) for x in segment_bytes)
        fixed = device_bytes(capacity, req_capacity, rounds, max_msgs)
        staging_total = (budget - fixed) // rounds // 256 * 256 * rounds
        if staging_total < rounds * max(self.segment_bytes):
            raise ValueError("budget too small for the ring and the rounds")
        self.budget = budget
        self.staging_per_round = staging_total // rounds
        self.book = RingBook(capacity, req_capacity)
        dev = device
        self.ring = {
            "src": torch.zeros(capacity, dtype=torch.int64, device=dev),
            "prior": torch.zeros(capacity, dtype=torch.int64, device=dev),
            "len": torch.zeros(capacity, dtype=torch.int32, device=dev),
            "req": torch.zeros(capacity, dtype=torch.int32, device=dev),
            "alg": torch.zeros(capacity, dtype=torch.uint8, device=dev),
            "state": torch.zeros(capacity, dtype=torch.int32, device=dev),
            "slots": torch.zeros((capacity, 32), dtype=torch.uint8, device=dev),
            "req_remaining": torch.zeros(req_capacity, dtype=torch.int32, device=dev),
            "req_done": torch.zeros(req_capacity, dtype=torch.int32).pin_memory(),
        }
        self.done_np = self.ring["req_done"].numpy()
        # in place: segments are hashed where the client's bytes are, and the
        # same byte budget only caps what the rounds claim at a time
        self.in_place = in_place
        self.staging = None if in_place else torch.empty(staging_total, dtype=torch.uint8, device=dev)
        self.slots = [_RoundSlot(self, None if in_place else self.staging[i * self.staging_per_round:],
                                 self.staging_per_round) for i in range(rounds)]
        # host staging of admissions (pinned; reused once the last admission's
        # copies have finished)
        self.h_src = torch.zeros(capacity, dtype=torch.int64).pin_memory()
        self.h_len = torch.zeros(capacity, dtype=torch.int32).pin_memory()
        self.h_req = torch.zeros(capacity, dtype=torch.int32).pin_memory()
        self.h_alg = torch.zeros(capacity, dtype=torch.uint8).pin_memory()
        self.h_rem = torch.zeros(req_capacity, dtype=torch.int32).pin_memory()
        # constant sources for progress (0) and state (READY): admission only
        # copies, so it never waits for an SM while the rounds fill the GPU
        self.h_zero = torch.zeros(capacity, dtype=torch.int64).pin_memory()
        self.h_ready = torch.full((capacity,), api.RING_READY, dtype=torch.int32).pin_memory()
        self.fin_np = np.zeros(req_capacity, dtype=bool)     # finished, by request slot
        self.admit_stream = torch.cuda.Stream(device=dev)
        self.admit_event = torch.cuda.Event()
        self.admit_event.record(self.admit_stream)
        self.rounds_launched = 0
        self.segments = 0
        self.loop_iters = 0
        self.admit_s = 0.0

    # -- admission -------------------------------------------------------
    def _write_admissions(self, reqs: list):
        """Ring entries and request counters of newly admitted requests (one
        contiguous run of message and request counters)."""
        torch, book, ring = self.torch, self.book, self.ring
        self.admit_event.synchronize()          # host staging is free again
        first = reqs[0].first
        total = sum(int(r.lengths.shape[0]) for r in reqs)
        src = np.concatenate([r.src for r in reqs]).view(np.int64) + self.pool_addr
        ln = np.concatenate([r.lengths for r in reqs]).view(np.int32)
        rq = np.concatenate([np.full(r.lengths.shape[0], r.counter % book.req_capacity, np.int32)
                             for r in reqs])
        al = np.concatenate([np.full(r.lengths.shape[0], r.alg, np.uint8) for r in reqs])
        rem = np.array([r.lengths.shape[0] for r in reqs], dtype=np.int32)
        for r in reqs:
            q = r.counter % book.req_capacity
            self.done_np[q] = 0
            self.fin_np[q] = False
        hs, hl, hr, ha = (self.h_src.numpy(), self.h_len.numpy(), self.h_req.numpy(),
                          self.h_alg.numpy())
        hs[:total], hl[:total], hr[:total], ha[:total] = src, ln, rq, al
        self.h_rem.numpy()[:rem.shape[0]] = rem
        with torch.cuda.stream(self.admit_stream):
            spans = book.spans(first, total)
            for pos, off, cnt in spans:
                ring["src"][pos:pos + cnt].copy_(self.h_src[off:off + cnt], non_blocking=True)
                ring["len"][pos:pos + cnt].copy_(self.h_len[off:off + cnt], non_blocking=True)
                ring["req"][pos:pos + cnt].copy_(self.h_req[off:off + cnt], non_blocking=True)
                ring["alg"][pos:pos + cnt].copy_(self.h_alg[off:off + cnt], non_blocking=True)
                ring["prior"][pos:pos + cnt].copy_(self.h_zero[:cnt], non_blocking=True)
            for pos, off, cnt in book.spans(reqs[0].counter, len(reqs), book.req_capacity):
                ring["req_remaining"][pos:pos + cnt].copy_(self.h_rem[off:off + cnt],
                                                           non_blocking=True)
            for pos, off, cnt in spans:                  # ready last
                ring["state"][pos:pos + cnt].copy_(self.h_ready[:cnt], non_blocking=True)
            self.admit_event.record(self.admit_stream)

    # -- the loop ----------------------------------------------------------
    def run(self, requests: list, keep_digests: bool = False, time_limit_s: float = 600.0,
            admission: Admission | None = None):
        """Serve `requests` (sorted by arrival) in real time; returns them,
        finished (done >= 0) or rejected (done < 0).  With `admission`, each
        admitted request gets a predicted completion time and the policy may
        hold requests on the host or shed them at arrival."""
        # the loop allocates no reference cycles; a collector pause would
        # stall round launches, so the cyclic collector waits until the end
        gc_was_on = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, keep_digests, time_limit_s, admission)
        finally:
            if gc_was_on:
                gc.enable()

    def _run(self, requests: list, keep_digests: bool, time_limit_s: float,
             adm: Admission | None = None):
        torch, book = self.torch, self.book
        torch.cuda.synchronize()
        nreq = len(requests)
        pending = collections.deque()
        inflight = {}                 # request slot -> Req
        finished = rejected = 0
        wake_all = False
        i = 0
        t0 = time.perf_counter()
        while finished + rejected < nreq:
            now = time.perf_counter() - t0
            if now > time_limit_s:
                raise RuntimeError("serving run exceeded %.0f s" % time_limit_s)
            while i < nreq and requests[i].arrival <= now:
                r = requests[i]
                i += 1
                if adm is not None and r.lengths.shape[0] and not adm.arrive(r, now):
                    rejected += 1               # shed: predicted too late
                    continue
                pending.append(r)
            # admission, first come first served
            new = []
            while pending:
                r = pending[0]
                m = int(r.lengths.shape[0])
                if m > book.capacity:
                    pending.popleft()
                    rejected += 1
                    if adm is not None:
                        adm.waiting_s = max(0.0, adm.waiting_s - r.work_s)
                    continue
                if m == 0:                      # nothing to hash: done on arrival
                    pending.popleft()
                    r.admitted = r.done = now
                    r.digests = np.zeros((0, 32), np.uint8) if keep_digests else None
                    finished += 1
                    continue
                if adm is not None and adm.hold(now):
                    break
                if not book.fits(m):
                    break
                pending.popleft()
                r.counter, r.first = book.admit(m)
                r.admitted = now
                if adm is not None:
                    adm.admit(r, now)
                inflight[r.counter % book.req_capacity] = r
                new.append(r)
            self.loop_iters += 1
            if new:
                ta = time.perf_counter()
                self._write_admissions(new)
                self.admit_s += time.perf_counter() - ta
                wake_all = True
            # rounds: a round that comes back with work is launched again (its
            # unfinished messages are ready again); all idle rounds are woken
            # by an admission or by a round that filled its batch (more ready
            # work is likely waiting)
            for s in self.slots:
                if s.busy and s.event.query():
                    s.busy = False
                    seg, nb = s.round.report()
                    self.segments += seg
                    s.again = seg > 0
                    if seg >= self.max_msgs or nb + max(self.segment_bytes) > self.staging_per_round:
                        wake_all = True
            if inflight:
                for s in self.slots:
                    if not s.busy and (s.again or wake_all):
                        s.stream.wait_event(self.admit_event)
                        s.round.launch(book.head, book.tail, stream=s.stream)
                        s.event.record(s.stream)
                        s.busy = True
                        s.again = False
                        self.rounds_launched += 1
            wake_all = False
            # completions: done flags of the open requests, by request slot
            lo, hi, R = book.req_head, book.req_tail, book.req_capacity
            if hi > lo:
                a, b = lo % R, (hi - 1) % R + 1
                parts = [np.arange(a, b)] if a < b else [np.arange(a, R), np.arange(0, b)]
                hit = []
                for idx in parts:
                    sel = idx[(self.done_np[idx] != 0) & ~self.fin_np[idx]]
                    if sel.size:
                        hit.append(sel)
                if hit:
                    t = time.perf_counter() - t0
                    for q in np.concatenate(hit).tolist():
                        r = inflight.pop(q)
                        r.done = t
                        self.fin_np[q] = True
                        if adm is not None:
                            adm.finish(r, t)
                        if keep_digests:
                            r.digests = self._digests(r)
                        book.finish(r.counter)
                        finished += 1
        for s in self.slots:
            if s.busy:
                s.event.synchronize()
                s.busy = False
        torch.cuda.synchronize()
        return requests

    def _digests(self, r: Req) -> np.ndarray:
        m = int(r.lengths.shape[0])
        parts = [self.ring["slots"][pos:pos + cnt].cpu().numpy()
                 for pos, _, cnt in self.book.spans(r.first, m)]
        return np.concatenate(parts) if parts else np.zeros((0, 32), np.uint8)

    def close(self):
        for s in self.slots:
            s.round.close()


# ---------------------------------------------------------------------------
# synthetic load

def make_requests(count: int, rate_per_s: float, seed: int, pool_bytes: int,
                  max_msgs: int = 4096, min_len: int = 16, max_len: int = 1 << 20,
                  align: int = 16) -> list:
    """Poisson request stream; each message's bytes are a range of the
    random-byte pool starting at an offset that is a multiple of `align`
    (1 = any byte), chosen from the request's seed."""
    from . import workloads
    if align < 1:
        raise ValueError("align must be >= 1")
    out = []
    for k, r in enumerate(workloads.serve_requests(count, rate_per_s, seed, max_msgs, min_len, max_len)):
        rng = np.random.Generator(np.random.PCG64(r.seed))
        lens = r.lengths.astype(np.uint64)
        hi = (np.uint64(pool_bytes) - lens) // np.uint64(align)
        src = (rng.random(lens.shape[0]) * (hi.astype(np.float64) + 1)).astype(np.uint64) * np.uint64(align)
        src = np.minimum(src, np.uint64(pool_bytes) - lens)
        out.append(Req(k, r.arrival_s, r.alg, r.lengths, src))
    return out


def latency_stats(requests: list) -> dict:
    done = [r for r in requests if r.done >= 0]
    if not done:
        return {"completed": 0}
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    nbytes = sum(r.nbytes for r in done)
    t_end = max(r.done for r in done)
    t_start = min(r.arrival for r in done)
    # steady state: bytes of the requests finishing between the 10th and the
    # 90th percentile of finishing times, over that interval (leaves out the
    # ramp-up and the drain after the last arrival)
    fin = np.array([r.done for r in done])
    nb = np.array([r.nbytes for r in done], dtype=np.float64)
    t10, t90 = np.percentile(fin, [10, 90])
    mid = (fin > t10) & (fin <= t90)
    steady = float(nb[mid].sum() / (t90 - t10) / 1e9) if t90 > t10 else 0.0
    return {"completed": len(done), "rejected": len(requests) - len(done),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "gbs": nbytes / max(t_end - t_start, 1e-9) / 1e9, "steady_gbs": steady,
            "bytes": nbytes, "span_s": t_end - t_start}
