"""Streaming imager for host-resident snapshots (Section 4.1-4.4 pipeline).

Host snapshots (pinned memory) are copied to a depth-2 device staging ring
on a copy stream while the compute stream grids, images and runs tLISI on
the previous snapshot; CUDA events interlock the two streams so the host
never waits (Section 4.2), and each tLISI matrix is copied back to a pinned
host cube as soon as it exists.  This module only orders copies and library
calls; the computation is libtoi's.
"""
from __future__ import annotations

import torch

from .binding import Plan, TOI_CAND_PERIODIC, tlisi_candidates


class StreamingImager:
    def __init__(self, plan: Plan, n_bl: int, n_ch: int, n_pol: int, vis_dtype=torch.complex64,
                 weights: bool = False, depth: int = 2):
        self.plan = plan
        self.depth = depth
        self.copy_stream = torch.cuda.Stream()
        self.compute_stream = torch.cuda.current_stream()
        self.plan.set_stream(self.compute_stream)
        mk = lambda *shape, dtype: torch.empty(*shape, dtype=dtype, device="cuda")  # noqa: E731
        self.stage = []
        for _ in range(depth):
            self.stage.append(dict(
                uvw=mk(n_bl, 3, dtype=torch.float64), freq=mk(n_ch, dtype=torch.float64),
                vis=mk(n_bl, n_ch, n_pol, dtype=vis_dtype), flag=mk(n_bl, n_ch, n_pol, dtype=torch.uint8),
                weight=mk(n_bl, n_ch, n_pol, dtype=torch.float32) if weights else None))
        self.copied = [torch.cuda.Event() for _ in range(depth)]
        self.consumed = [torch.cuda.Event() for _ in range(depth)]
        self.h2d_bytes = 0
        self.d2h_bytes = 0

    def _h2d(self, i: int, snap):
        st = self.stage[i]
        with torch.cuda.stream(self.copy_stream):
            self.copy_stream.wait_event(self.consumed[i])
            for k in ("uvw", "freq", "vis", "flag", "weight"):
                if st[k] is not None and snap.get(k) is not None:
                    st[k].copy_(snap[k], non_blocking=True)
                    self.h2d_bytes += snap[k].numel() * snap[k].element_size()
            self.copied[i].record(self.copy_stream)

    def run(self, host_snapshots, n_snap: int, cube_dev, cube_host, tile: int,
            mode: int = TOI_CAND_PERIODIC):
        """Image snapshots host_snapshots[s % len] for s < n_snap; tLISI slices
        land in cube_dev and are copied to the pinned cube_host; returns the
        candidate search result on the cube."""
        nh = len(host_snapshots)
        self.plan.tlisi_reset()
        for i in range(min(self.depth, n_snap)):
            self._h2d(i, host_snapshots[i % nh])
        for s in range(n_snap):
            i = s % self.depth
            st = self.stage[i]
            self.compute_stream.wait_event(self.copied[i])
            self.plan.grid(st["uvw"], st["freq"], st["vis"], flag=st["flag"], weight=st["weight"])
            self.consumed[i].record(self.compute_stream)
            self.plan.image(0, None)
            out = cube_dev[s - 2] if s >= 2 else None
            if self.plan.tlisi_update(None, out):
                cube_host[s - 2].copy_(out, non_blocking=True)
                self.d2h_bytes += out.numel() * out.element_size()
            if s + self.depth < n_snap:
                self._h2d(i, host_snapshots[(s + self.depth) % nh])
        thr, boxes, n = tlisi_candidates(cube_dev, tile, mode, stream=self.compute_stream)
        self.d2h_bytes += 8 + 4 + 16 * len(boxes)
        return thr, boxes, n
