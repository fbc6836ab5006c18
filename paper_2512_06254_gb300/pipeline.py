"""Streaming imager for host-resident snapshots (Section 4.1-4.4 pipeline).

Host snapshots (pinned memory) are copied to a depth-2 device staging ring
while the compute stream grids, images and runs tLISI on earlier ones.
Each snapshot's visibilities are split by baseline rows over several copy
streams, so that several copy engines move one snapshot at once.  CUDA
events interlock copies and compute, so the host never waits on a copy
(Section 4.2), and each tLISI matrix is copied back to a pinned host cube
as soon as it exists.  With batch > 0 a staging slot holds a whole batch,
imaged by one toi_batch call.  This module only orders copies and library
calls; the computation is libtoi's.
"""
from __future__ import annotations

import torch

from .binding import Plan, TOI_CAND_PERIODIC, tlisi_candidates


class StreamingImager:
    def __init__(self, plan: Plan, n_bl: int, n_ch: int, n_pol: int, vis_dtype=torch.complex64,
                 weights: bool = False, depth: int = 2, batch: int = 0, copy_streams: int = 4):
        self.plan = plan
        self.depth = depth
        self.batch = batch
        self.copy_streams = [torch.cuda.Stream() for _ in range(max(1, copy_streams))]
        self.compute_stream = torch.cuda.current_stream()
        self.plan.set_stream(self.compute_stream)
        mk = lambda *shape, dtype: torch.empty(*shape, dtype=dtype, device="cuda")  # noqa: E731
        per_slot = max(1, batch)
        self.stage = []
        for _ in range(depth):
            self.stage.append([dict(
                uvw=mk(n_bl, 3, dtype=torch.float64), freq=mk(n_ch, dtype=torch.float64),
                vis=mk(n_bl, n_ch, n_pol, dtype=vis_dtype),
                flag=mk(n_bl, n_ch, n_pol, dtype=torch.uint8),
                weight=mk(n_bl, n_ch, n_pol, dtype=torch.float32) if weights else None)
                for _ in range(per_slot)])
        ncs = len(self.copy_streams)
        self.copied = [[torch.cuda.Event() for _ in range(ncs)] for _ in range(depth)]
        self.consumed = [torch.cuda.Event() for _ in range(depth)]
        self.h2d_bytes = 0
        self.d2h_bytes = 0

    def _copy(self, dst, src, k):
        """dst <- src, split along the first axis over the copy streams."""
        n = src.shape[0]
        ncs = len(self.copy_streams)
        if k not in ("vis", "flag", "weight") or n < ncs:
            with torch.cuda.stream(self.copy_streams[0]):
                dst.copy_(src, non_blocking=True)
        else:
            for j, cs in enumerate(self.copy_streams):
                lo, hi = n * j // ncs, n * (j + 1) // ncs
                with torch.cuda.stream(cs):
                    dst[lo:hi].copy_(src[lo:hi], non_blocking=True)
        self.h2d_bytes += src.numel() * src.element_size()

    def _h2d(self, i: int, snaps):
        """Copy host snapshots into staging slot i (after its last use)."""
        for cs in self.copy_streams:
            cs.wait_event(self.consumed[i])
        for st, snap in zip(self.stage[i], snaps):
            for k in ("uvw", "freq", "vis", "flag", "weight"):
                if st[k] is not None and snap.get(k) is not None:
                    self._copy(st[k], snap[k], k)
        for ev, cs in zip(self.copied[i], self.copy_streams):
            ev.record(cs)

    def _wait_copied(self, i: int):
        for ev in self.copied[i]:
            self.compute_stream.wait_event(ev)

    def run(self, host_snapshots, n_snap: int, cube_dev, cube_host, tile: int,
            mode: int = TOI_CAND_PERIODIC):
        """Image snapshots host_snapshots[s % len] for s < n_snap; tLISI slices
        land in cube_dev and are copied to the pinned cube_host; returns the
        candidate search result on the cube."""
        if self.batch > 0:
            self._run_batched(host_snapshots, n_snap, cube_dev, cube_host)
        else:
            self._run_single(host_snapshots, n_snap, cube_dev, cube_host)
        thr, boxes, n = tlisi_candidates(cube_dev, tile, mode, stream=self.compute_stream)
        self.d2h_bytes += 8 + 4 + 16 * len(boxes)
        return thr, boxes, n

    def _run_single(self, host_snapshots, n_snap, cube_dev, cube_host):
        nh = len(host_snapshots)
        self.plan.tlisi_reset()
        for i in range(min(self.depth, n_snap)):
            self._h2d(i, [host_snapshots[i % nh]])
        for s in range(n_snap):
            i = s % self.depth
            st = self.stage[i][0]
            self._wait_copied(i)
            self.plan.grid(st["uvw"], st["freq"], st["vis"], flag=st["flag"], weight=st["weight"])
            self.consumed[i].record(self.compute_stream)
            self.plan.image(0, None)
            out = cube_dev[s - 2] if s >= 2 else None
            if self.plan.tlisi_update(None, out):
                cube_host[s - 2].copy_(out, non_blocking=True)
                self.d2h_bytes += out.numel() * out.element_size()
            if s + self.depth < n_snap:
                self._h2d(i, [host_snapshots[(s + self.depth) % nh]])

    def _run_batched(self, host_snapshots, n_snap, cube_dev, cube_host):
        nh = len(host_snapshots)
        B = self.batch
        nb = (n_snap + B - 1) // B
        row = cube_dev[0].numel() * cube_dev.element_size()

        def batch_of(b):
            return [host_snapshots[s % nh] for s in range(b * B, min((b + 1) * B, n_snap))]

        self.plan.tlisi_reset()
        for b in range(min(self.depth, nb)):
            self._h2d(b, batch_of(b))
        for b in range(nb):
            i = b % self.depth
            lo, hi = b * B, min((b + 1) * B, n_snap)
            self._wait_copied(i)
            first = self.plan.batch(self.stage[i][:hi - lo],
                                    cube_dev.data_ptr() + (lo - 2) * row)
            self.consumed[i].record(self.compute_stream)
            r0, r1 = lo + first - 2, hi - 2
            if r1 > r0:
                cube_host[r0:r1].copy_(cube_dev[r0:r1], non_blocking=True)
                self.d2h_bytes += (r1 - r0) * row
            if b + self.depth < nb:
                self._h2d(i, batch_of(b + self.depth))
