"""The LK front-end loop on the device, for many camera streams at once.

Per stream a pool of features (positions, identities, ages; capacity `cap`)
lives on the GPU together with its count, so a step runs without a host
round trip:

  1. build the new frame's pyramids (left, and right for stereo) and track
     the pool from the previous left frame to the new one with the
     forward-backward check (one batched run; the task's point count is the
     pool's device-side count);
  2. carry-over: survivors keep their identity and age, thinned by age
     priority and min_dist (one launch for every stream), which also writes
     the detector mask;
  3. detect Shi-Tomasi corners on the new left frame away from the kept
     features, up to `cap`;
  4. stereo: track the new corners left -> right with the forward-backward
     check (a second batched run) -- only corners that pass it may enter
     the pool (Sec. V-A);
  5. spawn new tracks from the accepted corners until the pool is full (one
     launch for every stream).

Every step is one launch (or one batched run, or one detector call) for all
streams.
"""

from __future__ import annotations

import ctypes as C

from . import vt


class FrontEnd:
    def __init__(self, specs, params: vt.KltParams, cap: int, min_dist: float = 10.0,
                 detect: vt.GfttParams | None = None, device="cuda"):
        import torch

        self.torch = torch
        self.params = params
        self.cap = cap
        self.min_dist = float(min_dist)
        self.detect = detect or vt.GfttParams(max_corners=cap, quality=0.01, min_dist=int(min_dist), nms_radius=4,
                                              block_radius=1, border=10)
        self.detect.max_corners = cap
        self.specs = list(specs)
        self.frames_seen = 0
        z = lambda *shape, dt=torch.float32: torch.zeros(shape, dtype=dt, device=device)  # noqa: E731
        self.st = []
        for sp in self.specs:
            d = {
                "pyr": [vt.vt_pyramid_create(sp.w, sp.h, sp.levels) for _ in range(2)],
                "pyr_r": vt.vt_pyramid_create(sp.w, sp.h, sp.levels) if sp.stereo else None,
                "pool": vt.TrackPool(cap, device),
                "tracked": z(cap, 2), "status": z(cap, dt=torch.uint8),
                "mask": torch.full((cap, 2), float("nan"), device=device),
                "corners": z(cap, 2), "ncorners": z(1, dt=torch.int32),
                "right": z(cap, 2) if sp.stereo else None, "right_st": z(cap, dt=torch.uint8) if sp.stereo else None,
            }
            self.st.append(d)
        self.gftt = vt.vt_gftt_create_pixels(sum(sp.w * sp.h for sp in self.specs[:64]) if len(self.specs) <= 64
                                             else 64 * max(sp.w * sp.h for sp in self.specs))
        nf = sum(2 if sp.stereo else 1 for sp in self.specs)
        self.batch_a = vt.Batch(max(1, nf), max(1, len(self.specs)))
        self.batch_b = vt.Batch(1, max(1, len(self.specs)))

    def _cur(self, k):
        return self.st[k]["pyr"][(self.frames_seen + 1) % 2]

    def _prev(self, k):
        return self.st[k]["pyr"][self.frames_seen % 2]

    def step(self, lefts, rights, stream=None, graph=True):
        """One frame for every stream; lefts / rights: device uint8 images
        (rights[k] is None for mono streams)."""
        frames, tasks = [], []
        first = self.frames_seen == 0
        for k, sp in enumerate(self.specs):
            d = self.st[k]
            frames.append(vt.frame_job(lefts[k], self._cur(k)))
            if sp.stereo:
                frames.append(vt.frame_job(rights[k], d["pyr_r"]))
            if not first:
                p = d["pool"]
                prm_l = sp.levels
                tasks.append(vt.track_task(self._prev(k), self._cur(k), p.pts, d["tracked"], d["status"], fb=True,
                                           levels=prm_l, n_dev=p.count))
        self._run(self.batch_a, frames, tasks, stream, graph)
        if not first:
            vt.vt_tracks_carry([vt.carry_job(self.st[k]["pool"], self.st[k]["tracked"], self.st[k]["status"],
                                             self.st[k]["mask"]) for k in range(len(self.specs))], self.min_dist,
                               stream)
        jobs = [vt.gftt_job(self._cur(k), 0, d["corners"], d["ncorners"], self.cap, mask=d["mask"])
                for k, d in enumerate(self.st)]
        for c0 in range(0, len(jobs), 64):  # at most 64 frames per detector call
            vt.vt_gftt_detect_many(self.gftt, jobs[c0:c0 + 64], self.detect, stream)
        stereo_tasks = []
        for k, sp in enumerate(self.specs):
            if sp.stereo:
                d = self.st[k]
                stereo_tasks.append(vt.track_task(self._cur(k), d["pyr_r"], d["corners"], d["right"], d["right_st"],
                                                  fb=True, levels=sp.levels, n_dev=d["ncorners"]))
        if stereo_tasks:
            self._run(self.batch_b, [], stereo_tasks, stream, graph)
        vt.vt_tracks_spawn([vt.spawn_job(self.st[k]["pool"], self.st[k]["corners"], self.st[k]["ncorners"],
                                         self.st[k]["right_st"]) for k in range(len(self.specs))], stream)
        self.frames_seen += 1

    def _run(self, batch, frames, tasks, stream, graph):
        fa = (vt.vt_frame_job * max(1, len(frames)))(*frames)
        ta = (vt.vt_track_task * max(1, len(tasks)))(*tasks)
        prm = self.params.c()
        code = vt._lib.vt_batch_set(batch, fa, len(frames), vt.VT_GRAD_S16, ta, len(tasks), C.byref(prm))
        if code != vt.VT_OK:
            raise vt.VTError("vt_batch_set", code)
        if graph:
            vt.vt_batch_run_graph(batch, stream)
        else:
            vt.vt_batch_run(batch, stream)

    def launches_per_step(self):
        """Kernel launches of one step after the first (batched runs as
        reported by vt_batch_info; 7 per detector call)."""
        a = vt.vt_batch_info(self.batch_a)["launches_per_run"]
        b = vt.vt_batch_info(self.batch_b)["launches_per_run"] if any(sp.stereo for sp in self.specs) else 0
        return a + 1 + 7 * ((len(self.specs) + 63) // 64) + b + 1

    def pool(self, k):
        """(positions, identities, ages) of stream k's pool, on the host."""
        p = self.st[k]["pool"]
        n = int(p.count.item())
        return p.pts[:n].cpu().numpy(), p.ids[:n].cpu().numpy(), p.ages[:n].cpu().numpy()

    def free(self):
        self.batch_a.free()
        self.batch_b.free()
        for d in self.st:
            for p in d["pyr"]:
                p.free()
            if d["pyr_r"] is not None:
                d["pyr_r"].free()
        self.gftt.free()
