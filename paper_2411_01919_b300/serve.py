"""Request loop for many depth cameras on one GPU: continuous batching.

Requests (one depth frame of one camera stream) arrive over time.  The loop
keeps `n_lanes` execution lanes, each a libpm context with its own CUDA
stream and room for `max_batch` frames.  Whenever a lane is idle it takes the
oldest admitted requests (at most one per stream per batch), copies their
depth from pinned host memory into the stream's device buffer for that lane,
and enqueues the whole path for the batch without waiting
(pm_process_batch_async).  With one lane a stream's frames complete in
arrival order; with several, a later frame of a stream can complete first
when its lane's batch finishes sooner.  Frames carry no state between them,
so each result is still exact; a consumer that needs them in order sorts
them by `Request.k`.  Requests that arrive while
batches are on the GPU are admitted as memory frees up and go into the next
batch of whichever lane frees first; with two lanes one batch runs while the
next is being filled and launched, so their work overlaps on the device.

Admission is by memory: a request holds, while it is queued or on the GPU,
the scratch bytes its frame size needs (pm_scratch_bytes for one frame) plus
its input bytes; the sum over admitted requests stays within the budget
(default 4 GiB) minus what the lanes and the per-stream buffers hold for good.
A request not admitted within `max_wait_s` of its arrival is refused.  A
request that cannot be served at all (a frame larger than the lanes, an
unsupported depth type, intrinsics that are not finite with fx, fy > 0, a
stream that changes its frame size) is refused at admission with the reason
in `error`, and the loop goes on serving the others; a batch whose launch
still fails marks only its own requests.

Each frame's result is bit-identical to processing it alone with
pm_process_frame (the batched kernels never mix frames), which the test suite
checks on a mixed stream load.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from ._ffi import PmError
from .pipeline import _DT, Params, Pipeline, Planes, scratch_bytes


@dataclass
class Request:
    stream: int
    k: int                      # frame number within the stream
    t_arrival: float            # seconds since the start of the run
    depth: torch.Tensor         # pinned host [h, w] (uint16 / float16 / float32)
    K: tuple
    frame_idx: int
    iters: int = -1
    bytes: int = 0
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    planes: Optional[Planes] = None
    refused: bool = False
    failed: bool = False        # admitted, but the launch of its batch failed
    error: Optional[str] = None  # why the request was refused as invalid, or its batch failed


@dataclass
class _Lane:
    pipe: Pipeline
    stream: torch.cuda.Stream
    index: int
    batch: List[Request] = field(default_factory=list)
    event: Optional[torch.cuda.Event] = None
    seq: int = 0                # launch order of the lane's batch

    @property
    def busy(self):
        return bool(self.batch)


class Server:
    def __init__(self, params: Params, budget_bytes: int = 4 << 30, max_batch: int = 16,
                 n_lanes: int = 2, max_w: int = 1280, max_h: int = 720,
                 max_wait_s: float = 1.0, use_graph='full'):
        """use_graph: True (every batch replays a CUDA graph captured once per
        batch shape), False (direct launches), or 'full' (graphs for full
        batches, whose shape repeats under load; direct launches for the
        partial batches of light load, whose shapes vary)."""
        self.p = params
        self.max_batch = max_batch
        self.max_wait_s = max_wait_s
        self.use_graph = use_graph
        self.max_w, self.max_h = max_w, max_h
        self.lanes = [_Lane(Pipeline(params, max_w, max_h, max_batch), torch.cuda.Stream(), i)
                      for i in range(n_lanes)]
        self.static_bytes = n_lanes * scratch_bytes(max_w, max_h, max_batch, params.hypotheses,
                                                    params.max_planes)
        if self.static_bytes > budget_bytes:
            raise ValueError('lanes alone need %d bytes, above the budget of %d'
                             % (self.static_bytes, budget_bytes))
        self.budget = budget_bytes
        self.in_use = 0                       # admitted requests
        self.stream_bytes = 0                 # per-stream device buffers
        self.dev: Dict[int, List[torch.Tensor]] = {}
        self.stats = collections.Counter()

    # -- memory -----------------------------------------------------------
    def request_bytes(self, r: Request) -> int:
        h, w = r.depth.shape
        return (scratch_bytes(w, h, 1, self.p.hypotheses, self.p.max_planes)
                + r.depth.numel() * r.depth.element_size())

    def invalid(self, r: Request) -> Optional[str]:
        """Why a request cannot be served (None if it can): checked at
        admission so that one malformed request is refused alone."""
        d = r.depth
        if not isinstance(d, torch.Tensor) or d.dim() != 2 or d.dtype not in _DT:
            return 'depth must be a 2-D uint16 / float16 / float32 tensor'
        h, w = d.shape
        if not (1 <= w <= self.max_w and 1 <= h <= self.max_h):
            return 'frame %dx%d outside 1x1 .. %dx%d' % (w, h, self.max_w, self.max_h)
        if d.stride(1) != 1:
            return 'depth rows must be contiguous'
        try:
            fx, fy, cx, cy = (float(x) for x in r.K)
        except (TypeError, ValueError):
            return 'intrinsics must be four numbers'
        if not (fx > 0 and fy > 0 and all(math.isfinite(x) for x in (fx, fy, cx, cy))):
            return 'intrinsics must be finite with fx, fy > 0'
        if r.iters > 100000:
            return 'iters out of range'
        bufs = self.dev.get(r.stream)
        if bufs is not None and (bufs[0].shape != d.shape or bufs[0].dtype != d.dtype):
            return 'stream %d changed its frame size or dtype' % r.stream
        return None

    def _room(self) -> int:
        return self.budget - self.static_bytes - self.stream_bytes - self.in_use

    def _stream_buffers(self, r: Request) -> List[torch.Tensor]:
        bufs = self.dev.get(r.stream)
        if bufs is not None and (bufs[0].shape != r.depth.shape or bufs[0].dtype != r.depth.dtype):
            raise ValueError('stream %d changed its frame size or dtype' % r.stream)
        if bufs is None:
            bufs = [torch.empty(r.depth.shape, dtype=r.depth.dtype, device='cuda')
                    for _ in self.lanes]
            self.dev[r.stream] = bufs
            self.stream_bytes += sum(b.numel() * b.element_size() for b in bufs)
        return bufs

    # -- the loop -----------------------------------------------------------
    def _launch(self, lane: _Lane, batch: List[Request]):
        frames = []
        try:
            with torch.cuda.stream(lane.stream):
                for r in batch:
                    buf = self._stream_buffers(r)[lane.index]
                    buf.copy_(r.depth, non_blocking=True)
                    frames.append(dict(depth=buf, K=r.K, frame_idx=r.frame_idx, iters=r.iters))
                graph = (len(batch) == self.max_batch if self.use_graph == 'full'
                         else bool(self.use_graph))
                lane.pipe.submit_batch(frames, use_graph=graph, stream=lane.stream)
                lane.event = torch.cuda.Event()
                lane.event.record(lane.stream)
        except (PmError, ValueError) as e:
            # nothing was enqueued for the batch: its requests fail, the lane stays free
            for r in batch:
                r.refused = True
                r.failed = True
                r.error = 'batch failed: %s' % e
                self.in_use -= r.bytes
            self.stats['failed_batches'] += 1
            return
        lane.batch = batch
        lane.seq = self.stats['batches']
        self.stats['batches'] += 1
        self.stats['graph_batches'] += int(graph)
        self.stats['batched_frames'] += len(batch)

    def _finish(self, lane: _Lane, now: float, done: List[Request]):
        res = lane.pipe.collect_batch()
        for r, planes in zip(lane.batch, res):
            r.planes = planes
            r.t_done = now
            self.in_use -= r.bytes
            done.append(r)
        lane.batch = []
        lane.event = None

    def _admit(self, waiting: collections.deque, admitted: collections.deque, now: float):
        while waiting:
            r = waiting[0]
            why = self.invalid(r)
            if why is not None:
                waiting.popleft()
                r.refused = True
                r.error = why
                self.stats['invalid'] += 1
                continue
            if now - r.t_arrival > self.max_wait_s:
                waiting.popleft()
                r.refused = True
                self.stats['refused'] += 1
                continue
            need = self.request_bytes(r)
            if r.stream not in self.dev:
                # a stream's first request also reserves its device buffers
                extra = len(self.lanes) * r.depth.numel() * r.depth.element_size()
                if need + extra > self._room():
                    break
                self._stream_buffers(r)
            elif need > self._room():
                break
            waiting.popleft()
            r.bytes = need
            r.t_admit = now
            self.in_use += need
            self.stats['peak_in_use'] = max(self.stats['peak_in_use'], self.in_use)
            admitted.append(r)

    def _take_batch(self, admitted: collections.deque) -> List[Request]:
        batch, seen, rest = [], set(), collections.deque()
        while admitted and len(batch) < self.max_batch:
            r = admitted.popleft()
            if r.stream in seen:
                rest.append(r)
            else:
                seen.add(r.stream)
                batch.append(r)
        while rest:
            admitted.appendleft(rest.pop())
        return batch

    def run(self, requests: Sequence[Request], realtime: bool = True) -> List[Request]:
        """Serve `requests` (sorted by arrival).  realtime: requests become
        visible at their arrival time on the wall clock; otherwise all are
        visible at once (throughput mode).  Returns every request, with
        t_done/planes filled in or refused set."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        waiting, admitted = collections.deque(), collections.deque()
        done: List[Request] = []
        i = 0
        t0 = time.perf_counter()
        while i < len(reqs) or waiting or admitted or any(l.busy for l in self.lanes):
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].t_arrival <= now):
                if not realtime:
                    reqs[i].t_arrival = now
                waiting.append(reqs[i])
                i += 1
            progressed = False
            for lane in self.lanes:
                if lane.busy and lane.event.query():
                    self._finish(lane, time.perf_counter() - t0, done)
                    progressed = True
            self._admit(waiting, admitted, now)
            for lane in self.lanes:
                if not lane.busy and admitted:
                    batch = self._take_batch(admitted)
                    if batch:
                        self._launch(lane, batch)
                        progressed = True
            if not progressed:
                busy = [l for l in self.lanes if l.busy]
                if len(busy) == len(self.lanes):
                    # every lane is busy and nothing can start before one
                    # finishes: wait for the oldest batch (a blocking event
                    # wait; arrivals meanwhile are admitted right after it)
                    min(busy, key=lambda l: l.seq).event.synchronize()
                    continue
                if realtime and i < len(reqs) and not admitted and not waiting:
                    nxt = reqs[i].t_arrival - (time.perf_counter() - t0)
                    if nxt > 0 and not busy:
                        time.sleep(min(nxt, 0.002))
                        continue
                time.sleep(20e-6)
        self.elapsed = time.perf_counter() - t0
        return reqs

    def close(self):
        for lane in self.lanes:
            lane.pipe.close()


def summarize(reqs: Sequence[Request], elapsed: float) -> dict:
    ok = [r for r in reqs if r.t_done is not None]
    lat = sorted(1e3 * (r.t_done - r.t_arrival) for r in ok)

    def pct(q):
        if not lat:
            return None
        return lat[min(len(lat) - 1, int(round(q / 100.0 * (len(lat) - 1))))]

    return {'frames': len(ok), 'refused': sum(r.refused for r in reqs),
            'invalid': sum(r.error is not None and not r.failed for r in reqs),
            'failed': sum(r.failed for r in reqs),
            'frames_per_s': len(ok) / elapsed if elapsed > 0 else None,
            'p50_ms': pct(50), 'p99_ms': pct(99), 'max_ms': lat[-1] if lat else None,
            'elapsed_s': elapsed}


def poisson_arrivals(n_streams: int, duration_s: float, mean_gap_s: float, seed: int):
    """(stream, k, t) for Poisson arrivals of every stream over duration_s."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_streams):
        t = rng.uniform(0, mean_gap_s)
        k = 0
        while t < duration_s:
            out.append((s, k, t))
            t += rng.exponential(mean_gap_s)
            k += 1
    out.sort(key=lambda x: x[2])
    return out
