"""Served tracking: a request loop over many camera streams with continuous
batching and admission by an HBM budget.

A request is "the next frame of stream s has arrived on the host" (frame(s)
and keypoints in pinned host memory).  The loop:

* admits a stream when its device footprint (pyramids, input slots, point
  buffers) fits the HBM budget; a stream that does not fit waits until an
  admitted stream ends and frees its memory;
* whenever a batch slot is free and requests are pending, takes every
  pending request whose stream is admitted and has nothing in flight, and
  issues one batched run for all of them (H2D of their frames and points, the
  vt_batch graph, D2H of points and status) on that slot's CUDA stream; two
  slots alternate, so a batch is assembled and launched while the previous
  one still runs and their work overlaps on the device;
* completes a request when its slot's event has fired, recording the latency
  from the request's arrival time to the moment all its results (temporal
  and, for a stereo stream, left->right points and status) are on the host.

A request's features are the previous frame's keypoints it tracks through
the whole step (forward-backward temporal tracking, plus the left->right
check of the new frame's keypoints on a stereo stream), as in the batched
benchmark; the stereo pairs are counted separately.

The plain baseline serves the same trace one request at a time with the
single-pair calls.
"""

from __future__ import annotations

import functools
import gc
import time
from dataclasses import dataclass, field

import numpy as np

from . import vt
from .engine import BatchedTracker


def _without_gc(fn):
    """Run a request loop with Python's cyclic garbage collector paused (one
    collection before), so that no collection pause lands inside a
    request's latency; reference counting still frees memory."""

    @functools.wraps(fn)
    def run(*args, **kwargs):
        gc.collect()
        was = gc.isenabled()
        gc.disable()
        try:
            return fn(*args, **kwargs)
        finally:
            if was:
                gc.enable()

    return run


@dataclass
class Request:
    sid: int
    frame: int  # index into the stream's frame store
    prev_frame: int  # index of the stream's previous frame (-1 for the first)
    t_arrive: float  # seconds from the trace start
    t_done: float = -1.0
    n_features: int = 0
    n_stereo: int = 0


@dataclass
class ServeStats:
    served: int
    features: int
    wall_s: float
    stereo_pairs: int = 0
    latencies_ms: list = field(default_factory=list)
    batches: int = 0
    mean_batch: float = 0.0
    admitted_max: int = 0
    admission_waits: int = 0
    rejected: int = 0
    peak_bytes: int = 0

    def summary(self):
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {
            "requests": self.served,
            "features_per_s": self.features / self.wall_s if self.wall_s > 0 else 0.0,
            "stereo_pairs_per_s": self.stereo_pairs / self.wall_s if self.wall_s > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "p999_ms": float(np.percentile(lat, 99.9)),
            "max_ms": float(lat.max()),
            "batches": self.batches,
            "mean_batch_requests": self.mean_batch,
            "admitted_max": self.admitted_max,
            "admission_waits": self.admission_waits,
            "rejected": self.rejected,
            "peak_bytes": self.peak_bytes,
            "wall_s": self.wall_s,
        }


def make_trace(specs, n_requests, seed, rate_hz=(20.0, 30.0), jitter=0.1, frames_per_stream=4,
               session=None):
    """Seeded arrival trace.  Stream s has period 1/U(rate_hz); the gap before
    each frame is period * (1 + Exp(jitter)).  Frames cycle 0, 1, ..., F-1,
    F-2, ..., 1, 0, 1, ... so consecutive requests are adjacent frames.
    `session` (requests per stream) ends streams so that waiting streams can
    be admitted; by default each stream lives for the whole trace."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = len(specs)
    per = int(np.ceil(n_requests / S)) if session is None else session
    F = frames_per_stream
    P = max(1, 2 * (F - 1))
    out = []
    for s in range(S):
        period = 1.0 / rng.uniform(*rate_hz)
        t = rng.uniform(0.0, period) + (0.0 if session is None else s * 0.0)
        for k in range(per):
            t += period * (1.0 + rng.exponential(jitter)) if k > 0 else 0.0
            kk = k % P
            f = kk if kk < F else P - kk
            pk = (k - 1) % P
            pf = -1 if k == 0 else (pk if pk < F else P - pk)
            out.append(Request(s, f, pf, t))
    out.sort(key=lambda r: r.t_arrive)
    return out[:n_requests]


class Server:
    """Continuous-batching request loop (see module docstring)."""

    def __init__(self, specs, frames, params: vt.KltParams, budget_bytes: int, grad_type=vt.VT_GRAD_S16,
                 slots: int = 2):
        import torch

        self.torch = torch
        self.specs = specs
        self.params = params
        self.budget = budget_bytes
        self.tr = BatchedTracker(specs, params, grad_type)
        self.S = len(specs)
        # pinned host copies of every stream's frames and keypoints
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        self.h_left = [[pin(x) for x in fr.left] for fr in frames]
        self.h_right = [[pin(x) if x is not None else None for x in fr.right] for fr in frames]
        self.h_kps = [[pin(k) for k in fr.kps] for fr in frames]
        # host results per stream: temporal points and status, then (stereo)
        # left->right points and status
        self.h_out = [tuple(t for _ in range(2 if s.stereo else 1)
                            for t in (torch.empty((s.n_max, 2), dtype=torch.float32).pin_memory(),
                                      torch.empty(s.n_max, dtype=torch.uint8).pin_memory()))
                      for s in self.tr.streams]
        self.footprint = [self._footprint(i) for i in range(self.S)]
        self._prm_c = self.params.c()
        self._prm = vt.C.byref(self._prm_c)
        self._addresses()
        self.slots = [dict(stream=torch.cuda.Stream(), event=torch.cuda.Event(), batch=vt.Batch(
            self.tr.batch_capacity[0], self.tr.batch_capacity[1]), reqs=None) for _ in range(slots)]

    def _footprint(self, i):
        s = self.tr.streams[i]
        b = sum(p.info()[3] for p in s.pyr) + (s.pyr_r.info()[3] if s.pyr_r is not None else 0)
        b += s.w * s.h * (2 if s.stereo else 1)  # input slots
        b += s.n_max * (8 + 8 + 1 + 4) * (2 if s.stereo else 1)  # points in/out, status, err
        return b

    def _addresses(self):
        """Device and pinned-host addresses of every stream's slots, frames,
        keypoints and results (fixed for the server's lifetime)."""
        self._dev = []
        for i, s in enumerate(self.tr.streams):
            d = dict(left=s.in_left.data_ptr(), bytes=s.w * s.h, kp_t=s.kp_t.data_ptr(),
                     out_t=(s.out_t[0].data_ptr(), s.out_t[1].data_ptr()))
            if s.stereo:
                d.update(right=s.in_right.data_ptr(), kp_s=s.kp_s.data_ptr(),
                         out_s=(s.out_s[0].data_ptr(), s.out_s[1].data_ptr()))
            d["h_left"] = [x.data_ptr() for x in self.h_left[i]]
            d["h_right"] = [x.data_ptr() if x is not None else 0 for x in self.h_right[i]]
            d["h_kps"] = [k.data_ptr() for k in self.h_kps[i]]
            d["n_kps"] = [int(k.shape[0]) for k in self.h_kps[i]]
            d["h_out"] = [t.data_ptr() for t in self.h_out[i]]
            self._dev.append(d)
        self._tables = {}

    def _request_copies(self, r):
        """(uploads, downloads, n_t, n_s) of one request: its frame(s) and
        keypoints into the stream's slots, its results back to the host."""
        d = self._dev[r.sid]
        up = [(d["left"], d["h_left"][r.frame], d["bytes"])]
        down = []
        nt = ns = 0
        if r.prev_frame >= 0:
            nt = d["n_kps"][r.prev_frame]
            up.append((d["kp_t"], d["h_kps"][r.prev_frame], 8 * nt))
            down += [(d["h_out"][0], d["out_t"][0], 8 * nt), (d["h_out"][1], d["out_t"][1], nt)]
        if "right" in d:
            ns = d["n_kps"][r.frame]
            up += [(d["right"], d["h_right"][r.frame], d["bytes"]), (d["kp_s"], d["h_kps"][r.frame], 8 * ns)]
            down += [(d["h_out"][2], d["out_s"][0], 8 * ns), (d["h_out"][3], d["out_s"][1], ns)]
        return up, down, nt, ns

    def _stream_tables(self, sid, nt, ns):
        """The stream's frame and task descriptors for its next step (cached:
        they depend only on the stream, which of its pyramids is current and
        the point counts)."""
        key = (sid, self.tr.streams[sid].built % 2, nt, ns)
        t = self._tables.get(key)
        if t is None:
            fa, nf, ta, ntk, _ = self.tr.step_tables([sid], [nt], [ns])
            t = ([fa[k] for k in range(nf)], [ta[k] for k in range(ntk)])
            self._tables[key] = t
        return t

    def _issue(self, slot, reqs):
        tr = self.tr
        cs = slot["stream"]
        up, down, frames, tasks = [], [], [], []
        for r in reqs:
            u, d, nt, ns = self._request_copies(r)
            up += u
            down += d
            r.n_features = nt
            r.n_stereo = ns
            f, t = self._stream_tables(r.sid, nt, ns)
            frames += f
            tasks += t
        vt.vt_copy_async(up, cs)
        fa = (vt.vt_frame_job * max(1, len(frames)))(*frames)
        ta = (vt.vt_track_task * max(1, len(tasks)))(*tasks)
        code = vt._lib.vt_batch_set(slot["batch"], fa, len(frames), tr.grad_type, ta, len(tasks), self._prm)
        if code != vt.VT_OK:
            raise vt.VTError("vt_batch_set", code)
        vt.vt_batch_run_graph(slot["batch"], cs)
        tr.advance([r.sid for r in reqs])
        vt.vt_copy_async(down, cs)
        slot["event"].record(cs)
        slot["reqs"] = reqs

    @_without_gc
    def serve(self, trace, realtime=True, max_batch=64, stall_s=60.0):
        """Run the trace; returns ServeStats.  With realtime=False every
        request is available at time 0 (throughput mode)."""
        torch = self.torch
        trace = list(trace)
        last_progress = time.perf_counter()
        pending = []  # arrived, not issued
        nxt = 0
        admitted = set()
        used = 0
        remaining = {}
        for r in trace:
            remaining[r.sid] = remaining.get(r.sid, 0) + 1
        waiting = []  # streams waiting for admission, in order of first arrival
        in_flight = set()
        stats = ServeStats(0, 0, 0.0)
        batch_sizes = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        done = 0
        total = len(trace)
        while done < total:
            t = now()
            while nxt < total and (not realtime or trace[nxt].t_arrive <= t):
                r = trace[nxt]
                if not realtime:
                    r.t_arrive = 0.0
                pending.append(r)
                if r.sid not in admitted and r.sid not in waiting:
                    waiting.append(r.sid)
                nxt += 1
            # admission in arrival order while the budget allows; a stream
            # larger than the whole budget can never run and is rejected
            while waiting and self.footprint[waiting[0]] > self.budget:
                s = waiting.pop(0)
                dropped = [r for r in pending if r.sid == s]
                pending = [r for r in pending if r.sid != s]
                stats.rejected += len(dropped) + sum(1 for r in trace[nxt:] if r.sid == s)
                done += len(dropped) + sum(1 for r in trace[nxt:] if r.sid == s)
                trace = trace[:nxt] + [r for r in trace[nxt:] if r.sid != s]
                total = len(trace)
            while waiting and used + self.footprint[waiting[0]] <= self.budget:
                s = waiting.pop(0)
                admitted.add(s)
                used += self.footprint[s]
            stats.peak_bytes = max(stats.peak_bytes, used)
            if time.perf_counter() - last_progress > stall_s:
                raise RuntimeError("served loop made no progress")
            if waiting:
                stats.admission_waits += 1
            stats.admitted_max = max(stats.admitted_max, len(admitted))
            # completions
            for slot in self.slots:
                if slot["reqs"] is not None and slot["event"].query():
                    td = now()
                    for r in slot["reqs"]:
                        r.t_done = td
                        stats.latencies_ms.append((td - r.t_arrive) * 1e3)
                        stats.features += r.n_features
                        stats.stereo_pairs += r.n_stereo
                        in_flight.discard(r.sid)
                        remaining[r.sid] -= 1
                        if remaining[r.sid] == 0:  # stream ended: free its budget
                            admitted.discard(r.sid)
                            used -= self.footprint[r.sid]
                    done += len(slot["reqs"])
                    stats.served += len(slot["reqs"])
                    slot["reqs"] = None
                    last_progress = time.perf_counter()
            # issue on a free slot
            free = [sl for sl in self.slots if sl["reqs"] is None]
            if free and pending:
                take, keep, seen = [], [], set()
                for r in pending:
                    if (r.sid in admitted and r.sid not in in_flight and r.sid not in seen
                            and len(take) < max_batch):
                        take.append(r)
                        seen.add(r.sid)
                    else:
                        keep.append(r)
                if take:
                    pending = keep
                    for r in take:
                        in_flight.add(r.sid)
                    self._issue(free[0], take)
                    stats.batches += 1
                    batch_sizes.append(len(take))
        torch.cuda.synchronize()
        stats.wall_s = now()
        stats.mean_batch = float(np.mean(batch_sizes)) if batch_sizes else 0.0
        return stats

    @_without_gc
    def serve_plain(self, trace, realtime=True):
        """Baseline: every request alone, in arrival order, single-pair calls."""
        torch = self.torch
        tr = self.tr
        stats = ServeStats(0, 0, 0.0)
        cs = self.slots[0]["stream"]
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        for r in trace:
            if realtime:
                while now() < r.t_arrive:
                    pass
            else:
                r.t_arrive = 0.0
            up, down, nt, ns = self._request_copies(r)
            vt.vt_copy_async(up, cs)
            tr.plain_step([r.sid], [nt], [ns], stream=cs)
            tr.advance([r.sid])
            vt.vt_copy_async(down, cs)
            cs.synchronize()
            td = now()
            stats.latencies_ms.append((td - r.t_arrive) * 1e3)
            stats.features += nt
            stats.stereo_pairs += ns
            stats.served += 1
        stats.wall_s = now()
        stats.batches = stats.served
        stats.mean_batch = 1.0
        return stats

    def free(self):
        for sl in self.slots:
            sl["batch"].free()
        self.tr.free()
