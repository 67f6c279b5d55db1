"""Serving loop: continuous admission of detect-and-clean requests.

Requests arrive on a schedule (e.g. a Poisson stream).  A request is
admitted as soon as a library slot and enough of the HBM budget are free
-- whatever is still running -- and runs on a stream of its own
(lacos_submit_async), so its kernels overlap on the device with the
requests already in flight.  Completions are polled; each request's
latency is completion minus arrival.  The budget covers every byte a
request holds on the device while in flight: its output buffers (uint8 mask,
float32 cleaned frame) and the library's scratch.  Input frames are device
tensors the caller provides (already received).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

from . import lacos


@dataclass
class Request:
    frame: object          # device tensor (float32 or uint16), ny x nx
    params: lacos.Params
    arrival: float         # seconds after the start of the run


@dataclass
class Record:
    index: int
    arrival: float
    admitted: float
    done: float
    npix: int
    result: lacos.FrameResult
    mask: object = None
    clean: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Stats:
    n: int
    mpix_per_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    max_in_flight: int
    makespan_s: float
    records: list = field(default_factory=list)


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


class Server:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 120 << 30, max_slots: int = 64,
                 keep_outputs: bool = False):
        import torch
        self.device = torch.device("cuda", device)
        self.budget = int(hbm_budget_bytes)
        self.ctx = lacos.Context(device, hbm_budget_bytes=self.budget, max_slots=max_slots)
        self.keep = keep_outputs
        self._free = collections.defaultdict(list)  # (ny, nx) -> [(mask, clean)]
        self.in_use = 0

    def _request_bytes(self, ny, nx, params):
        """Device bytes of one request in flight: its outputs (uint8 mask and
        float32 cleaned frame, 5 B/px) and the library scratch its parameters
        need (one more bit-plane with satgrow > 0)."""
        import ctypes
        return ny * nx * 5 + self.ctx.lib.lacos_request_bytes(ny, nx, ctypes.byref(params))

    def _buffers(self, ny, nx):
        import torch
        if self._free[(ny, nx)]:
            return self._free[(ny, nx)].pop()
        return (torch.empty((ny, nx), dtype=torch.uint8, device=self.device),
                torch.empty((ny, nx), dtype=torch.float32, device=self.device))

    def run(self, requests: list, poll_sleep: float = 2e-5) -> Stats:
        """Serve the requests (sorted by arrival) and return latency/throughput stats.

        The cyclic garbage collector is held off while the loop runs (a full
        collection of a large heap would stall admission and polling for
        milliseconds); it is restored, and run once, afterwards."""
        import gc
        enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, poll_sleep)
        finally:
            if enabled:
                gc.enable()
                gc.collect()

    def _run(self, requests, poll_sleep):
        import torch
        torch.cuda.synchronize(self.device)
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        queue = collections.deque()
        inflight = {}
        records = []
        nxt = 0
        max_inflight = 0
        t0 = time.perf_counter()
        while nxt < len(order) or queue or inflight:
            now = time.perf_counter() - t0
            while nxt < len(order) and requests[order[nxt]].arrival <= now:
                queue.append(order[nxt])
                nxt += 1
            # Admit in arrival order while a slot and budget are free.
            while queue:
                i = queue[0]
                rq = requests[i]
                ny, nx = rq.frame.shape
                need = self._request_bytes(ny, nx, rq.params)
                if self.in_use + need > self.budget and inflight:
                    break
                mask, clean = self._buffers(ny, nx)
                try:
                    t = self.ctx.submit_async(rq.frame, rq.params, mask, clean)
                except lacos.LacosError as e:
                    self._free[(ny, nx)].append((mask, clean))
                    if e.code == lacos.EAGAIN and inflight:
                        break
                    raise
                queue.popleft()
                self.in_use += need
                inflight[t] = (i, time.perf_counter() - t0, mask, clean, need)
                max_inflight = max(max_inflight, len(inflight))
            # Retire completed requests.
            progressed = False
            for t in list(inflight):
                r = self.ctx.poll(t)
                if r is None:
                    continue
                i, adm, mask, clean, need = inflight.pop(t)
                done = time.perf_counter() - t0
                rq = requests[i]
                ny, nx = rq.frame.shape
                rec = Record(i, rq.arrival, adm, done, ny * nx, r)
                if self.keep:
                    rec.mask, rec.clean = mask, clean
                else:
                    self._free[(ny, nx)].append((mask, clean))
                self.in_use -= need
                records.append(rec)
                progressed = True
            if not progressed and poll_sleep:
                time.sleep(poll_sleep)
        makespan = max(r.done for r in records) - min(r.arrival for r in records)
        lat = [r.latency * 1e3 for r in records]
        return Stats(n=len(records), mpix_per_s=sum(r.npix for r in records) / 1e6 / makespan,
                     p50_ms=_percentile(lat, 50), p99_ms=_percentile(lat, 99),
                     mean_ms=sum(lat) / len(lat), max_in_flight=max_inflight,
                     makespan_s=makespan, records=records)

    def close(self):
        self._free.clear()
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def poisson_requests(frames, params, rate_hz: float, n: int, seed=(3, 1 << 21)):
    """n requests cycling through `frames` (with matching `params`), Poisson arrivals."""
    import math
    from . import synth
    arr = synth.poisson_arrivals(rate_hz, n, seed) if math.isfinite(rate_hz) else [0.0] * n
    arr = [a - arr[0] for a in arr]
    return [Request(frames[i % len(frames)], params[i % len(params)], float(arr[i])) for i in range(n)]
