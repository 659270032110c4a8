"""Served counting: a request loop with continuous batching.

Requests (a byte string each, in pinned host memory) arrive over time.  The
loop keeps up to `max_inflight` units of work on the GPU at once, each on its
own CUDA stream:
  - small requests (up to `big_bytes`) that have arrived are admitted
    together as one round: copied host -> device into the round's resident
    text buffer and counted by one wc_count_batched call, each request a
    document with its own table;
  - a large request is a unit of its own, counted by wc_count (all SMs,
    shared-memory head, capacities learned from earlier requests).
Requests that arrive while work is running are admitted as soon as a stream
and device memory free up, so their work overlaps on the device.  Each
request's table (32-bit counts, count desc then word asc) is built and kept
on the device; the answer returned to the host is its top-k (the table's
first k rows, gathered on the device: wc_topk for a single count,
wc_batch_topk for a round), and the whole table too when keep_tables is set.
The context's device-memory budget bounds admission: each unit's request text
is allocated from the context's budgeted pool (wc_buffer_alloc) like the
library's own tables and scratch, so a unit whose text or tables the budget
cannot hold waits for running work to finish and free its memory (memory freed in stream order is charged until its stream has passed the
free, so with nothing running the loop first waits for the device; a round
still refused then is cut to fewer requests, and a single request larger than
the whole budget is an error).  A round whose device tables
overflow is recounted request by request with growing capacities, so answers
are always exact.

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
    words: np.ndarray       # uint8: the top-k rows, or the whole table when kept
    offs: np.ndarray        # uint64 [n+1]
    counts: np.ndarray      # uint32 [n]
    topk: int
    full: bool = False      # words/offs/counts hold the whole table

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def as_list(self, limit: int | None = None):
        """The first rows of the answer (all rows held when limit is None)."""
        n = self.counts.size if limit is None else min(limit, self.counts.size)
        return [(self.words[self.offs[i]:self.offs[i + 1]].tobytes(), int(self.counts[i])) for i in range(n)]


class _Work:
    """One unit on the GPU: a round of small requests or one large request."""

    def __init__(self, reqs, stream, buf, keep=None, batch=None, table=None, h_offs=None):
        import torch
        self.reqs = reqs
        self.stream = stream
        self.buf = buf            # the unit's request text (budgeted device buffer)
        self.keep = keep          # device tensors that must outlive the work
        self.batch = batch
        self.table = table
        self.h_offs = h_offs
        self.event = torch.cuda.Event()
        self.event.record(stream)


def _wait_until(t_target: float, t0: float):
    while True:
        dt = t_target - (time.perf_counter() - t0)
        if dt <= 0:
            return
        time.sleep(min(dt, 0.0005) if dt > 0.0002 else 0)


def _to_device(counter, reqs, stream):
    """The requests' text copied into one budgeted device buffer (raises
    WcError with WC_ERR_BUDGET, allocating nothing, when it does not fit)."""
    import torch
    h_offs = np.zeros(len(reqs) + 1, dtype=np.uint64)
    h_offs[1:] = np.cumsum([r.data.numel() for r in reqs])
    n = int(h_offs[-1])
    buf = counter.buffer(max(16, n), stream)
    with torch.cuda.stream(stream):
        for j, r in enumerate(reqs):
            if r.data.numel():
                buf.tensor[int(h_offs[j]):int(h_offs[j + 1])].copy_(r.data, non_blocking=True)
    return buf, h_offs


def serve_batched(counter: wc.Counter, requests: list[Request], topk: int = 100, max_inflight: int = 6,
                  round_bytes: int = 256 << 20, big_bytes: int = 4 << 20, keep_tables: bool = False,
                  device: int = 0):
    """Runs the request stream through the continuous-batching loop and returns
    one Answer per request (in request order) plus run statistics."""
    import torch
    dev = torch.device("cuda", device)
    free_streams = deque(torch.cuda.Stream(device=dev) for _ in range(max_inflight))
    small: deque[Request] = deque()
    big: deque[Request] = deque()
    running: deque[_Work] = deque()
    answers: dict[int, Answer] = {}
    order = sorted(requests, key=lambda r: r.arrival)
    nxt = 0
    t0 = time.perf_counter()
    stats = {"rounds": 0, "large": 0, "recounted": 0, "capacity_errors": [], "budget_waits": 0,
             "max_running": 0}

    def answer(rq, w, o, c, s0, n, full):
        now = time.perf_counter() - t0
        answers[rq.rid] = Answer(rq.rid, rq.arrival, now, w[o[s0]:o[s0 + n]],
                                 (o[s0:s0 + n + 1] - o[s0]).astype(np.uint64), c[s0:s0 + n].astype(np.uint32), topk,
                                 full)

    def answer_table(rq, t, stream):  # one request's device table -> its answer
        if keep_tables:
            w, o, c = with_budget(lambda: t.export(stream))
            answer(rq, w, o, c, 0, c.size, True)
        else:
            top = with_budget(lambda: counter.topk(t, topk, stream))
            w, o, c = with_budget(lambda: top.export(stream))
            top.free()
            answer(rq, w, o, c, 0, c.size, False)

    def recount(rq, stream):  # exact fallback with growing capacities
        while True:
            try:
                buf, _ = _to_device(counter, [rq], stream)
                break
            except wc.WcError as e:
                if e.status != wc.WC_ERR_BUDGET or not make_room():
                    raise
        with torch.cuda.stream(stream):
            t = counter.count_checked(buf.tensor[:rq.data.numel()], stream=stream)
            answer_table(rq, t, stream)
            t.free()
        buf.free(stream)
        stats["recounted"] += 1

    def with_budget(fn):
        """Runs fn(); when the budget refuses one of its allocations (a
        finished unit's top-k table or export scratch), the other running
        units are finished first to free their memory, then fn runs again."""
        while True:
            try:
                return fn()
            except wc.WcError as e:
                if e.status != wc.WC_ERR_BUDGET or not make_room():
                    raise

    def make_room():
        """Frees budget for a refused allocation: finishes the oldest running
        unit; with nothing running, waits for the device, since memory freed
        in stream order is charged until its stream has passed the free.
        False when neither frees anything."""
        if running:
            finish(running.popleft())
            return True
        used = counter.mem_usage()[0]
        if used:
            torch.cuda.synchronize(dev)
            return counter.mem_usage()[0] < used
        return False

    def finish(wk: _Work):
        wk.event.synchronize()
        if wk.buf is not None:  # the counts have read the text: its budget is free again
            wk.buf.free(wk.stream)
            wk.buf = None
        if wk.table is not None:
            st = wk.table.status()
            if st == wc.WC_ERR_CAPACITY:
                if len(stats["capacity_errors"]) < 8:
                    stats["capacity_errors"].append(wc.wc_last_error(counter.ctx))
                recount(wk.reqs[0], wk.stream)
            else:
                answer_table(wk.reqs[0], wk.table, wk.stream)
            wk.table.free()
        else:
            st = wk.batch.status()
            if st == wc.WC_ERR_CAPACITY:
                if len(stats["capacity_errors"]) < 8:
                    stats["capacity_errors"].append(wc.wc_last_error(counter.ctx))
                for rq in wk.reqs:
                    recount(rq, wk.stream)
            elif st != wc.WC_OK:
                raise wc.WcError(st, wc.wc_last_error(counter.ctx))
            elif keep_tables:
                ds, dn, w, o, c = with_budget(lambda: wk.batch.export(wk.stream))
                for j, rq in enumerate(wk.reqs):
                    answer(rq, w, o, c, int(ds[j]), int(dn[j]), True)
            else:  # every request's top-k gathered on the device, one small copy
                top, first, n = with_budget(lambda: wk.batch.topk(topk))
                w, o, c = with_budget(lambda: top.export(wk.stream))
                for j, rq in enumerate(wk.reqs):
                    answer(rq, w, o, c, int(first[j]), int(n[j]), False)
            del wk.batch
        free_streams.append(wk.stream)

    round_limit = [round_bytes]  # cut while a round is refused with nothing running

    def launch(stream):
        """Starts the next unit on `stream`; False if the budget refused it."""
        if big and (not small or big[0].arrival <= small[0].arrival):
            rq = big.popleft()
            buf = None
            try:
                buf, _ = _to_device(counter, [rq], stream)
                tab = counter.count(buf.tensor[:rq.data.numel()], stream=stream)
            except wc.WcError as e:
                if buf is not None:
                    buf.free(stream)
                big.appendleft(rq)
                if e.status != wc.WC_ERR_BUDGET:
                    raise
                return False
            running.append(_Work([rq], stream, buf, table=tab))
            stats["large"] += 1
            return True
        take, nbytes = [], 0
        while small and (not take or nbytes + small[0].data.numel() <= round_limit[0]):
            r = small.popleft()
            take.append(r)
            nbytes += r.data.numel()
        buf = None
        try:
            buf, h_offs = _to_device(counter, take, stream)
            with torch.cuda.stream(stream):
                offs = torch.from_numpy(h_offs.view(np.int64)).to(dev, non_blocking=True)
            batch = counter.count_batched(buf.tensor[:max(16, nbytes)], offs, h_offs, stream=stream)
        except wc.WcError as e:
            if buf is not None:
                buf.free(stream)
            for r in reversed(take):
                small.appendleft(r)
            if e.status != wc.WC_ERR_BUDGET:
                raise
            return False
        running.append(_Work(take, stream, buf, keep=offs, batch=batch, h_offs=h_offs))
        stats["rounds"] += 1
        return True

    while len(answers) < len(order):
        now = time.perf_counter() - t0
        while nxt < len(order) and order[nxt].arrival <= now:
            r = order[nxt]
            (big if r.data.numel() > big_bytes else small).append(r)
            nxt += 1
        progressed = False
        while running and running[0].event.query():
            finish(running.popleft())
            progressed = True
        if (small or big) and free_streams:
            stream = free_streams.popleft()
            if launch(stream):
                stats["max_running"] = max(stats["max_running"], len(running))
                continue
            stats["budget_waits"] += 1
            free_streams.appendleft(stream)  # budget: wait for running work
            if make_room():
                pass
            elif small and round_limit[0] > 1:
                round_limit[0] //= 2  # nothing else holds memory: admit a smaller round
            else:
                raise wc.WcError(wc.WC_ERR_BUDGET, "a request larger than the whole device-memory budget")
            continue
        if progressed:
            continue
        if running:
            if nxt < len(order) and not (small or big):
                time.sleep(0.00005)  # idle until the next arrival or a completion
                continue
            finish(running.popleft())
            continue
        if nxt < len(order):
            _wait_until(order[nxt].arrival, t0)
    stats["wall_s"] = time.perf_counter() - t0
    return [answers[r.rid] for r in requests], stats


def serve_fifo(counter: wc.Counter, requests: list[Request], topk: int = 100, keep_tables: bool = False,
               device: int = 0):
    """The plain path: one request at a time in arrival order, one wc_count
    launch per request (host -> device copy, count, top-k on the device,
    top-k (or the whole table) -> host)."""
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
            if keep_tables:
                w, o, c = t.export(stream)
            else:
                top = counter.topk(t, topk, stream)
                w, o, c = top.export(stream)
                top.free()
        now = time.perf_counter() - t0
        answers[r.rid] = Answer(r.rid, r.arrival, now, w, o, c.astype(np.uint32), topk, keep_tables)
        t.free()
    wall = time.perf_counter() - t0
    return [answers[r.rid] for r in requests], {"wall_s": wall}
