"""Continuous-batching request loop over sb_run (the served form).

Requests (a stereo pair in pinned host memory plus its parameters) arrive at
any time through ``Server.submit``.  A scheduler thread admits waiting
requests in arrival order while their device-memory estimate fits the budget,
batches everything admitted into one ``sb_run(SB_RUN_BATCHED)`` call on the
first free stream (three by default, so new batches are copied in and
launched while earlier ones compute; a batch of one request replays its
shape's CUDA graph, which the stream's context keeps),
and resolves each request's future when its batch's completion event has
fired (in the stream's waiter thread, which then wakes the scheduler).  Inputs, intermediate maps and results of admitted requests stay
resident on the device until the batch completes; results are copied back to
pinned host memory in the same stream.

Pinned result buffers come from a per-shape free list that the scheduler
fills; a client that is done with a result hands its buffers back with
``Server.recycle`` so that steady-state serving pins no new host memory (a
fresh pinned allocation costs milliseconds and holds the interpreter lock).

The scheduler never polls: it sleeps on a condition variable that new
requests and batch completions signal (one waiter thread per stream blocks
on its batch's completion event, finishes the batch and frees the stream).  ``Server.cancel`` drops a request that is
still waiting for admission.

The pipeline is deterministic per pair, so a request's result does not depend
on what it was batched with.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import queue as _queue
import threading
import time
from typing import Dict, List, Tuple

import torch

from . import Context, Pair, SB_RUN_BATCHED, SB_RUN_GRAPH, sb_params, sb_run


def request_bytes(h: int, w: int) -> int:
    """Device bytes one admitted request holds: RGB in (2x3), RGB out (3),
    disparity out (2) and the library workspace (about 18 bytes per pixel)."""
    n = h * w
    return n * (6 + 3 + 2 + 18) + (1 << 20)


class Request:
    __slots__ = ("left", "right", "params", "future", "arrival", "bytes", "out_rgb", "out_disp", "h", "w")

    def __init__(self, left, right, params: sb_params):
        self.left, self.right, self.params = left, right, params
        self.h, self.w = int(left.shape[0]), int(left.shape[1])
        self.future: cf.Future = cf.Future()
        self.arrival = time.perf_counter()
        self.bytes = request_bytes(self.h, self.w)
        self.out_rgb = self.out_disp = None


class Server:
    def __init__(self, device: int = 0, mem_budget_bytes: int = 40 << 30, max_batch: int = 64, n_streams: int = 3):
        self.device = device
        self.budget = int(mem_budget_bytes)
        self.max_batch = max_batch
        torch.cuda.set_device(device)
        self.streams = [torch.cuda.Stream(device) for _ in range(n_streams)]
        self.ctxs = [Context(device, 0, s) for s in self.streams]
        self.busy = [None] * n_streams   # (event, requests, device tensors) per stream
        self.queue: collections.deque = collections.deque()
        self.used = 0
        self.cv = threading.Condition()
        self.running = True
        self.completed: List[Tuple[float, float]] = []   # (arrival, done) per finished request
        self.batches = 0
        self.cancelled = 0
        self._free: Dict[Tuple[int, int], list] = collections.defaultdict(list)
        self._free_lock = threading.Lock()
        self._events = [_queue.Queue() for _ in range(n_streams)]
        self.waiters = [threading.Thread(target=self._wait_loop, args=(i,), daemon=True) for i in range(n_streams)]
        for t in self.waiters:
            t.start()
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ------------------------------------------------------------ client side
    def submit(self, left_host, right_host, params: sb_params) -> cf.Future:
        """Queue one pair (pinned host uint8 [h, w, 3] tensors); the future
        resolves to (out_rgb, out_disp) host tensors."""
        req = Request(left_host, right_host, params)
        if req.bytes > self.budget:
            req.future.set_exception(MemoryError("request needs %d bytes, budget is %d" % (req.bytes, self.budget)))
            return req.future
        with self.cv:
            self.queue.append(req)
            self.cv.notify()
        return req.future

    def cancel(self, future: cf.Future) -> bool:
        """Drop the request of ``future`` if it is still waiting for admission
        (the future is then cancelled); False once it is admitted or done."""
        with self.cv:
            for r in self.queue:
                if r.future is future:
                    self.queue.remove(r)
                    self.cancelled += 1
                    r.future.cancel()
                    return True
        return False

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify()
        self.thread.join()
        for q in self._events:
            q.put(None)
        for t in self.waiters:
            t.join()
        for c in self.ctxs:
            c.close()

    def latencies(self) -> List[float]:
        return [d - a for a, d in self.completed]

    def recycle(self, result):
        """Return a result's (out_rgb, out_disp) host buffers for reuse; the
        caller must not touch them afterwards."""
        rgb, disp = result
        with self._free_lock:
            self._free[(int(rgb.shape[0]), int(rgb.shape[1]))].append((rgb, disp))

    def _take_outputs(self, h: int, w: int):
        with self._free_lock:
            lst = self._free.get((h, w))
            if lst:
                return lst.pop()
        return (torch.empty((h, w, 3), dtype=torch.uint8, pin_memory=True),
                torch.empty((h, w), dtype=torch.int16, pin_memory=True))

    # ---------------------------------------------------------- scheduler side
    def _finish(self, i: int):
        # in stream i's waiter thread, once the batch's event has fired
        ev, reqs, _keep = self.busy[i]
        now = time.perf_counter()
        err = None
        try:
            self.ctxs[i].synchronize()
        except Exception as e:  # a failed batch fails its requests, the server keeps going
            err = e
        with self.cv:
            for r in reqs:
                self.used -= r.bytes
                self.completed.append((r.arrival, now))
            self.busy[i] = None   # the stream is free (its device tensors go with the entry)
            self.cv.notify()
        for r in reqs:
            if err is None:
                r.future.set_result((r.out_rgb, r.out_disp))
            else:
                r.future.set_exception(err)
            r.left = r.right = r.out_rgb = r.out_disp = None

    def _launch(self, i: int, reqs: List[Request]):
        s = self.streams[i]
        keep = []
        pairs = []
        with torch.cuda.stream(s):
            for r in reqs:
                r.out_rgb, r.out_disp = self._take_outputs(r.h, r.w)
                dl = r.left.to(self.device, non_blocking=True)
                dr = r.right.to(self.device, non_blocking=True)
                do = torch.empty((r.h, r.w, 3), dtype=torch.uint8, device=self.device)
                dd = torch.empty((r.h, r.w), dtype=torch.int16, device=self.device)
                keep += [dl, dr, do, dd]
                pairs.append(Pair(dl, dr, r.params, do, dd))
            # a lone request replays its shape's CUDA graph (one launch instead of
            # one per kernel: the host side of a pair is most of its latency);
            # a batch of several runs batched, since its composition rarely recurs
            sb_run(self.ctxs[i], pairs, SB_RUN_BATCHED | (SB_RUN_GRAPH if len(pairs) == 1 else 0))
            for r, q in zip(reqs, pairs):
                r.out_rgb.copy_(q.out_rgb, non_blocking=True)
                r.out_disp.copy_(q.out_disp, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.busy[i] = (ev, reqs, keep)
        self.batches += 1
        self._events[i].put(ev)

    def _wait_loop(self, i: int):
        # blocks (without the interpreter lock) until stream i's batch is done,
        # then finishes it here: one thread hand-off fewer than waking the
        # scheduler to do it
        while True:
            ev = self._events[i].get()
            if ev is None:
                return
            try:
                ev.synchronize()
            except Exception:   # a failed batch: _finish reports the error on its requests
                pass
            self._finish(i)

    def _admissible(self) -> bool:
        return bool(self.queue) and self.used + self.queue[0].bytes <= self.budget

    def _loop(self):
        while True:
            with self.cv:
                while True:
                    free = any(b is None for b in self.busy)
                    if free and self._admissible():
                        break
                    if not self.running and not self.queue and all(b is None for b in self.busy):
                        return
                    self.cv.wait()
            free = [i for i, b in enumerate(self.busy) if b is None]
            if free:
                with self.cv:
                    batch = []
                    while self.queue and len(batch) < self.max_batch and self.used + self.queue[0].bytes <= self.budget:
                        r = self.queue.popleft()
                        self.used += r.bytes
                        batch.append(r)
                if batch:
                    self._launch(free[0], batch)


def percentile(vals, q):
    v = sorted(vals)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[k]
