"""Served counting: a request loop with continuous batching.

Requests (a byte string each, in pinned host memory) arrive over time.  The
loop keeps up to `max_rounds` rounds on the GPU at once, each on its own CUDA
stream.  Whenever a stream is free it admits every request that has arrived
(up to a byte budget per round), copies them host -> device into the round's
resident text buffer, and counts them all with one wc_count_batched call: each
request is a document, answered with its own table (32-bit counts, sorted by
count desc then word asc) and its top-k (the table's first k rows).  Requests
that arrive while rounds are running are admitted as soon as a stream and
device memory free up, so their work overlaps on the device.  The context's
device-memory budget bounds what is admitted; a round the budget cannot hold
waits for running rounds to finish.

`serve_fifo` is the plain path for comparison: one request at a time, in
arrival order, one wc_count launch per request.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import wc


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    data: object            # pinned uint8 torch tensor (host)


@dataclasses.dataclass
class Answer:
    rid: int
    arrival: float
    done: float
    words: np.ndarray       # uint8
    offs: np.ndarray        # uint64 [n+1]
    counts: np.ndarray      # uint32 [n]
    topk: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def as_list(self, limit: int | None = None):
        n = self.counts.size if limit is None else min(limit, self.counts.size)
        return [(self.words[self.offs[i]:self.offs[i + 1]].tobytes(), int(self.counts[i])) for i in range(n)]


class _Round:
    def __init__(self, reqs, stream, dev_text, dev_offs, batch, h_offs):
        self.reqs = reqs
        self.stream = stream
        self.dev_text = dev_text
        self.dev_offs = dev_offs
        self.batch = batch
        self.h_offs = h_offs
        import torch
        self.event = torch.cuda.Event()
        self.event.record(stream)


def _wait_until(t_target: float, t0: float):
    while True:
        dt = t_target - (time.perf_counter() - t0)
        if dt <= 0:
            return
        time.sleep(min(dt, 0.0005) if dt > 0.0002 else 0)


def serve_batched(counter: wc.Counter, requests: list[Request], topk: int = 100, max_rounds: int = 4,
                  round_bytes: int = 512 << 20, keep_tables: bool = True, device: int = 0):
    """Runs the request stream through the continuous-batching loop and returns
    one Answer per request (in request order) plus run statistics."""
    import torch
    dev = torch.device("cuda", device)
    streams = [torch.cuda.Stream(device=dev) for _ in range(max_rounds)]
    free_streams = deque(streams)
    pending: deque[Request] = deque()
    running: deque[_Round] = deque()
    answers: dict[int, Answer] = {}
    order = sorted(requests, key=lambda r: r.arrival)
    nxt = 0
    t0 = time.perf_counter()
    rounds = 0

    def finish(rd: _Round):
        rd.event.synchronize()
        b = rd.batch
        if b.status() != wc.WC_OK:
            raise wc.WcError(b.status(), wc.wc_last_error(counter.ctx))
        ds, dn, w, o, c = b.export(rd.stream)
        now = time.perf_counter() - t0
        for j, rq in enumerate(rd.reqs):
            s0, n = int(ds[j]), int(dn[j])
            m = n if keep_tables else min(n, topk)
            ww = w[o[s0]:o[s0 + m]].copy()
            oo = (o[s0:s0 + m + 1] - o[s0]).astype(np.uint64)
            answers[rq.rid] = Answer(rq.rid, rq.arrival, now, ww, oo, c[s0:s0 + m].copy(), topk)
        del rd.batch
        free_streams.append(rd.stream)

    while len(answers) < len(order):
        now = time.perf_counter() - t0
        while nxt < len(order) and order[nxt].arrival <= now:
            pending.append(order[nxt])
            nxt += 1
        # completed rounds first: they free streams and memory
        while running and running[0].event.query():
            finish(running.popleft())
        if pending and free_streams:
            take, nbytes = [], 0
            while pending and (not take or nbytes + pending[0].data.numel() <= round_bytes):
                r = pending.popleft()
                take.append(r)
                nbytes += r.data.numel()
            stream = free_streams.popleft()
            h_offs = np.zeros(len(take) + 1, dtype=np.uint64)
            h_offs[1:] = np.cumsum([r.data.numel() for r in take])
            try:
                with torch.cuda.stream(stream):
                    text = torch.empty(max(16, nbytes), dtype=torch.uint8, device=dev)
                    for j, r in enumerate(take):
                        if r.data.numel():
                            text[int(h_offs[j]):int(h_offs[j + 1])].copy_(r.data, non_blocking=True)
                    offs = torch.from_numpy(h_offs.view(np.int64)).to(dev, non_blocking=False)
                    batch = counter.count_batched(text, offs, h_offs, stream=stream)
            except wc.WcError as e:
                if e.status != wc.WC_ERR_BUDGET or not running:
                    raise
                for r in reversed(take):  # memory is busy: wait for a round to finish
                    pending.appendleft(r)
                free_streams.appendleft(stream)
                finish(running.popleft())
                continue
            running.append(_Round(take, stream, text, offs, batch, h_offs))
            rounds += 1
            continue
        if running and (not pending or not free_streams):
            if nxt < len(order) and not pending:
                # idle until the next arrival or a completion, whichever comes first
                if running[0].event.query():
                    continue
                time.sleep(0.00005)
                continue
            finish(running.popleft())
            continue
        if nxt < len(order):
            _wait_until(order[nxt].arrival, t0)
    wall = time.perf_counter() - t0
    out = [answers[r.rid] for r in requests]
    return out, {"rounds": rounds, "wall_s": wall}


def serve_fifo(counter: wc.Counter, requests: list[Request], topk: int = 100, keep_tables: bool = True,
               device: int = 0):
    """The plain path: one request at a time in arrival order, one wc_count
    launch per request (host -> device copy, count, top-k, table -> host)."""
    import torch
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(device=dev)
    answers = {}
    order = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in order:
        _wait_until(r.arrival, t0)
        with torch.cuda.stream(stream):
            text = torch.empty(max(16, r.data.numel()), dtype=torch.uint8, device=dev)[:r.data.numel()]
            if r.data.numel():
                text.copy_(r.data, non_blocking=True)
            t = counter.count_checked(text, stream=stream)
            w, o, c = t.export(stream)
        now = time.perf_counter() - t0
        m = c.size if keep_tables else min(c.size, topk)
        answers[r.rid] = Answer(r.rid, r.arrival, now, w[:o[m]].copy(), o[:m + 1].copy(),
                                c[:m].astype(np.uint32), topk)
        t.free()
    wall = time.perf_counter() - t0
    return [answers[r.rid] for r in requests], {"wall_s": wall}
