"""Host runtime of the batched tracking path: per-stream device state and the
per-step job tables of vt_batch.

A camera stream keeps two left pyramids (previous / current, swapped by
index, never copied), one right pyramid when it is stereo, fixed device input
slots for the incoming frames and output buffers for its tracking tasks.
With an input ring (``ring=``) a stream instead has one pyramid per ring
slot whose level 0 is that slot (vt_pyramid_create_on): a frame that lands
in a slot is level 0 as it is, the step names the slots of the previous and
the current frame, and no build copies a frame.
One step of a stream with new frame(s):

  mono:   build cur-left; track prev-left -> cur-left (forward, backward, FB)
  stereo: build cur-left and right; track prev-left -> cur-left and
          cur-left -> right (the cross-camera check), both with FB; with a
          gate, the left->right pairs then go through the stereo
          triangulation gate (disparity, depth range, reprojection)

All streams of a step go into one vt_batch run (persistent launches, CUDA
graph).  The plain path issues the same work as single-pair calls, one
stream after another.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

from . import vt


@dataclass
class StreamState:
    sid: int
    w: int
    h: int
    levels: int
    stereo: bool
    n_max: int
    pyr: list = field(default_factory=list)  # two left pyramids
    pyr_r: object = None
    in_left: object = None  # device input slot [h, w] uint8
    in_right: object = None
    kp_t: object = None  # device float2 [n_max]: points tracked prev -> cur
    kp_s: object = None  # device float2 [n_max]: points tracked left -> right
    out_t: tuple = ()  # (pts, status, err, reason)
    out_s: tuple = ()
    ring_left: list = field(default_factory=list)  # input ring slots (level 0 of pyr[k]), if any
    ring_right: list = field(default_factory=list)  # right slots (level 0 of pyr_rs[k])
    pyr_rs: list = field(default_factory=list)  # right pyramids of a ring stream
    rig: object = None  # vt.StereoRig of a gated stereo stream
    gate_out: tuple = ()  # (status uint8 [n_max], xyz float [n_max, 3], reason uint8 [n_max])
    built: int = 0  # number of frames built so far (cur index = built % 2 after a build)


class BatchedTracker:
    """Many independent camera streams tracked one step at a time."""

    def __init__(self, specs, params: vt.KltParams, grad_type: int = vt.VT_GRAD_S16, device="cuda",
                 gate: vt.GateParams | None = None, rigs=None, ring=None):
        """gate / rigs: stereo triangulation gate parameters and one
        vt.StereoRig per spec (None for mono streams); without them stereo
        pairs are only flow-checked.  ring: per spec a pair (left slots,
        right slots or None) of 2-D uint8 device tensors [h, w] (rows
        16-byte aligned, 32 readable bytes after the last row, see
        vt_pyramid_create_on); steps then name ring slots (``ring_idx``)."""
        import torch

        self.torch = torch
        self.params = params
        self.grad_type = grad_type
        self.gate = gate
        self.streams = []
        # every stream's outputs are slices of four contiguous buffers, so one
        # copy each brings a whole step's results to the host
        total = sum(sp.n_kp * (2 if sp.stereo else 1) for sp in specs)
        self.out_pts = torch.zeros((max(1, total), 2), dtype=torch.float32, device=device)
        self.out_st = torch.zeros(max(1, total), dtype=torch.uint8, device=device)
        self.out_err = torch.zeros(max(1, total), dtype=torch.float32, device=device)
        self.out_rs = torch.zeros(max(1, total), dtype=torch.uint8, device=device)  # VT_LOST_* per point
        off = 0
        for j, sp in enumerate(specs):
            s = StreamState(sp.sid, sp.w, sp.h, sp.levels, sp.stereo, sp.n_kp)
            if ring is not None:
                s.ring_left = list(ring[j][0])
                s.ring_right = list(ring[j][1]) if sp.stereo else []
                s.pyr = [vt.vt_pyramid_create_on(b, sp.levels) for b in s.ring_left]
                s.pyr_rs = [vt.vt_pyramid_create_on(b, sp.levels) for b in s.ring_right]
            else:
                s.pyr = [vt.vt_pyramid_create(sp.w, sp.h, sp.levels) for _ in range(2)]
                s.pyr_r = vt.vt_pyramid_create(sp.w, sp.h, sp.levels) if sp.stereo else None
                s.in_left = torch.zeros((sp.h, sp.w), dtype=torch.uint8, device=device)
                s.in_right = torch.zeros((sp.h, sp.w), dtype=torch.uint8, device=device) if sp.stereo else None
            s.kp_t = torch.zeros((sp.n_kp, 2), dtype=torch.float32, device=device)
            s.kp_s = torch.zeros((sp.n_kp, 2), dtype=torch.float32, device=device) if sp.stereo else None
            def mk(o, n=sp.n_kp):
                return self.out_pts[o:o + n], self.out_st[o:o + n], self.out_err[o:o + n], self.out_rs[o:o + n]

            s.out_t = mk(off)
            off += sp.n_kp
            if sp.stereo:
                s.out_s = mk(off)
                off += sp.n_kp
            if gate is not None and sp.stereo:
                s.rig = rigs[j]
                s.gate_out = (torch.zeros(sp.n_kp, dtype=torch.uint8, device=device),
                              torch.zeros((sp.n_kp, 3), dtype=torch.float32, device=device),
                              torch.zeros(sp.n_kp, dtype=torch.uint8, device=device))
            self.streams.append(s)
        nf = sum(2 if s.stereo else 1 for s in self.streams)
        self.batch_capacity = (max(1, nf), max(1, nf))
        self.batch = vt.Batch(*self.batch_capacity)
        self._flops = None
        # order of the tasks in a run's work queue: "stream" (as the streams
        # are listed) or "cost" (most pyramid levels first, then most
        # points): the persistent tracking launch hands out points in task
        # order, so costly points first leave cheaper ones for the tail
        self.task_order = "stream"

    # ------------------------------------------------------------ descriptors
    def _step_pyramids(self, k, i, left, right, ring_idx):
        """(previous, current, right pyramid, left image, right image) of
        stream i's next step (k: its position in the step's stream list)."""
        s = self.streams[i]
        if s.ring_left:
            if ring_idx is None:
                raise ValueError("a ring stream's step names its ring slots (ring_idx)")
            kp, kc = ring_idx[k]
            return (s.pyr[kp], s.pyr[kc], s.pyr_rs[kc] if s.stereo else None, s.ring_left[kc],
                    s.ring_right[kc] if s.stereo else None)
        prev, cur = s.pyr[s.built % 2], s.pyr[(s.built + 1) % 2]
        return (prev, cur, s.pyr_r, left[k] if left is not None else s.in_left,
                (right[k] if right is not None else s.in_right) if s.stereo else None)

    def step_tables(self, sids, n_t, n_s, left=None, right=None, flops=None, kpt=None, kps=None, gate=True,
                    ring_idx=None):
        """ctypes arrays (frames, tasks) and gate tasks of one step for streams `sids`.

        n_t / n_s: point counts of the temporal / stereo task per stream;
        left / right: per-stream device images to build from (default: the
        stream's input slots); kpt / kps: per-stream device point arrays
        (default: the stream's point buffers); flops: optional per-stream
        (t, s) int32 arrays; gate: False leaves the stereo gate out of this
        step even when the tracker has one; ring_idx: per stream the ring
        slots (previous, current) of a ring tracker (left / right unused)."""
        frames, tasks, gates, keyed = [], [], [], []
        pyrs = [self._step_pyramids(k, i, left, right, ring_idx) for k, i in enumerate(sids)]
        for k, i in enumerate(sids):
            s = self.streams[i]
            _, cur, pyr_r, li, ri = pyrs[k]
            frames.append(vt.frame_job(li, cur))
            if s.stereo:
                frames.append(vt.frame_job(ri, pyr_r))
        for k, i in enumerate(sids):
            s = self.streams[i]
            prev, cur, pyr_r, _, _ = pyrs[k]
            if n_t[k] > 0:
                fl = flops[k][0] if flops is not None else None
                pts = (kpt[k] if kpt is not None else s.kp_t)[:n_t[k]]
                keyed.append(((-s.levels, -n_t[k]), vt.track_task(prev, cur, pts, s.out_t[0], s.out_t[1], s.out_t[2],
                                                                   fb=True, flops=fl, levels=s.levels,
                                                                   reason=s.out_t[3])))
            if s.stereo and n_s[k] > 0:
                fl = flops[k][1] if flops is not None else None
                pts = (kps[k] if kps is not None else s.kp_s)[:n_s[k]]
                keyed.append(((-s.levels, -n_s[k]), vt.track_task(cur, pyr_r, pts, s.out_s[0], s.out_s[1],
                                                                   s.out_s[2], fb=True, flops=fl, levels=s.levels,
                                                                   reason=s.out_s[3])))
                if s.rig is not None and gate:
                    g = s.gate_out
                    gates.append(vt.gate_task(pts, s.out_s[0], s.rig, g[0], status_in=s.out_s[1], xyz=g[1],
                                              reason=g[2]))
        if self.task_order == "cost":
            keyed.sort(key=lambda kt: kt[0])  # stable: equal costs keep stream order
        tasks = [t for _, t in keyed]
        fa = (vt.vt_frame_job * max(1, len(frames)))(*frames)
        ta = (vt.vt_track_task * max(1, len(tasks)))(*tasks)
        return fa, len(frames), ta, len(tasks), gates

    def stage(self, tables):
        fa, nf, ta, nt, gates = tables
        prm = self.params.c()
        code = vt._lib.vt_batch_set(self.batch, fa, nf, self.grad_type, ta, nt, C.byref(prm))
        if code != vt.VT_OK:
            raise vt.VTError("vt_batch_set", code)
        if gates:
            vt.vt_batch_set_gates(self.batch, gates, self.gate)

    def advance(self, sids):
        """After a step has been issued: the current pyramid becomes previous."""
        for i in sids:
            self.streams[i].built += 1

    def run(self, stream=None, graph=True, events=None):
        if events is not None:
            vt.vt_batch_run_timed(self.batch, stream, *events)
        elif graph:
            vt.vt_batch_run_graph(self.batch, stream)
        else:
            vt.vt_batch_run(self.batch, stream)

    # ------------------------------------------------------------- plain path
    def plain_step(self, sids, n_t, n_s, left=None, right=None, stream=None, kpt=None, kps=None, gate=True,
                   ring_idx=None):
        """The same step as single-pair calls, stream after stream."""
        import copy

        for k, i in enumerate(sids):
            s = self.streams[i]
            prm = copy.copy(self.params)
            prm.levels = s.levels
            prev, cur, pyr_r, li, ri = self._step_pyramids(k, i, left, right, ring_idx)
            self._build(li, s.levels, stream, cur)
            if s.stereo:
                self._build(ri, s.levels, stream, pyr_r)
            if n_t[k] > 0:
                pts = (kpt[k] if kpt is not None else s.kp_t)[:n_t[k]]
                vt.vt_klt_track_fb(prev, cur, pts, prm, s.out_t[0], s.out_t[1], s.out_t[2], reason=s.out_t[3],
                                   stream=stream)
            if s.stereo and n_s[k] > 0:
                pts = (kps[k] if kps is not None else s.kp_s)[:n_s[k]]
                vt.vt_klt_track_fb(cur, pyr_r, pts, prm, s.out_s[0], s.out_s[1], s.out_s[2], reason=s.out_s[3],
                                   stream=stream)
                if s.rig is not None and gate:
                    g = s.gate_out
                    vt.vt_stereo_gate(pts, s.out_s[0], s.rig, self.gate, g[0], status_in=s.out_s[1], xyz_out=g[1],
                                      reason_out=g[2], stream=stream)

    def _build(self, img, levels, stream, out):
        if self.grad_type == vt.VT_GRAD_NONE:  # the tracker computes gradients itself
            vt.vt_pyramid_build(img, levels, stream, out=out)
        else:
            vt.vt_pyramid_build_grad(img, levels, self.grad_type, stream, out=out)

    def plain_launches(self, sids, n_t, n_s, gate=True):
        """Kernel launches of plain_step (the level-0 copy is a memcpy, not a kernel)."""
        n = 0
        for k, i in enumerate(sids):
            s = self.streams[i]
            per_pyr = (s.levels - 1) + (0 if self.grad_type == vt.VT_GRAD_NONE else 1)
            n += per_pyr * (2 if s.stereo else 1)
            n += int(n_t[k] > 0) + int(s.stereo and n_s[k] > 0)
            n += int(s.stereo and n_s[k] > 0 and s.rig is not None and gate)
        return n

    def free(self):
        self.batch.free()
        for s in self.streams:
            for p in s.pyr + s.pyr_rs:
                p.free()
            if s.pyr_r is not None:
                s.pyr_r.free()
