"""Multi-rank host logic of the snapshot sharding (paper_2512_06254_gb300.shard)
on CPU with the gloo backend: the tLISI output blocks partition t = 2..S-1,
every rank's 2-snapshot halo makes its outputs identical to a single-rank
run, the all-gathered cube equals the single-rank cube (and so do the
candidates found in it), and the step time is the maximum over ranks.
The per-snapshot work here is the FP64 oracle (no GPU)."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import toi_oracle as O
from paper_2512_06254_gb300 import shard, synth

T_TILE = 16


@pytest.mark.parametrize("S", [2, 3, 4, 5, 10, 37, 1500])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_blocks_partition_the_outputs(S, world):
    owned = []
    for r in range(world):
        lo, hi = shard.tlisi_range(S, world, r)
        first, last = shard.image_range(S, world, r)
        assert 2 <= lo <= hi <= max(S, 2)
        if hi > lo:
            assert (first, last) == (lo - 2, hi)
        owned.extend(range(lo, hi))
        sizes = [shard.tlisi_range(S, world, q)[1] - shard.tlisi_range(S, world, q)[0]
                 for q in range(world)]
        assert max(sizes) - min(sizes) <= 1
    assert owned == list(range(2, S))


def _oracle_stream(w, snapshots):
    """Oracle images of the given snapshot indices (float32, as the library
    stores them)."""
    out = {}
    for s in snapshots:
        sn = synth.make_snapshot(w, s)
        h = {k: (v.numpy() if v is not None else None) for k, v in sn.items()}
        r = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], None, w.image_size,
                             w.cell_arcsec)
        out[s] = r["image"].astype(np.float32)
    return out


def _make_image_and_tlisi(images):
    ring = []

    def step(s, dst):
        ring.append(images[s])
        if len(ring) > 3:
            ring.pop(0)
        if len(ring) < 3:
            return False
        dst.copy_(torch.from_numpy(O.tlisi(ring[0], ring[1], ring[2], T_TILE).astype(np.float32)))
        return True
    return step


class _BatchedStream:
    """The batched engine's stream contract on the host: a batch of n
    snapshots extends the plan's image stream, first_valid = max(0, min(2 -
    images so far, n)), and entry i >= first_valid writes the tLISI of its
    three-image window to row i of the batch's output (earlier rows are left
    untouched)."""

    def __init__(self, images, out):
        self.images, self.out, self.ring, self.nimg = images, out, [], 0

    def __call__(self, s0, s1, row):
        fv = max(0, min(2 - self.nimg, s1 - s0))
        for i, s in enumerate(range(s0, s1)):
            self.ring = (self.ring + [self.images[s]])[-3:]
            if i >= fv:
                assert 0 <= row + i < self.out.shape[0], "a tLISI row outside the local block"
                self.out[row + i].copy_(torch.from_numpy(
                    O.tlisi(self.ring[0], self.ring[1], self.ring[2], T_TILE).astype(np.float32)))
        self.nimg += s1 - s0
        return fv


@pytest.mark.parametrize("S,world,batch", [(8, 2, 3), (8, 3, 2), (8, 2, 16), (37, 4, 5),
                                           (8, 1, 4), (8, 8, 2)])
def test_batched_shards_place_rows_like_one_rank(S, world, batch):
    """Each rank imaging [lo - 2, hi) in batches writes exactly its owned
    rows t = lo..hi-1, each equal to the single-rank per-snapshot output."""
    rng = np.random.default_rng(S + 10 * world + 100 * batch)
    n = 32
    images = {s: rng.normal(size=(n, n)).astype(np.float32) for s in range(S)}
    nt = n // T_TILE
    single = torch.zeros(S - 2, nt, nt)
    shard.run_shard(S, 1, 0, _make_image_and_tlisi(images), single)
    full = torch.full((S - 2, nt, nt), float("nan"))
    for r in range(world):
        lo, hi = shard.tlisi_range(S, world, r)
        local = torch.full((max(hi - lo, 1), nt, nt), float("nan"))
        assert shard.run_shard_batched(S, world, r, _BatchedStream(images, local), batch) == (lo, hi)
        full[lo - 2:hi - 2] = local[:hi - lo]
        assert torch.isnan(local[hi - lo:]).all()
    assert torch.equal(full, single)


def _rank_main(rank, world, port, outdir, batched=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.tiny_workload()
        S = w.n_snap
        nt = w.image_size // T_TILE
        first, hi = shard.image_range(S, world, rank)
        images = _oracle_stream(w, range(first, hi))
        width = -(-(S - 2) // world)
        local = torch.full((width, nt, nt), float("nan"))
        if batched:
            shard.run_shard_batched(S, world, rank, _BatchedStream(images, local), 4)
        else:
            shard.run_shard(S, world, rank, _make_image_and_tlisi(images), local)
        cube = shard.gather_cube(local, S, world, rank)
        t = shard.max_over_ranks(1.5 + rank)
        np.save(os.path.join(outdir, f"cube{rank}.npy"), cube.numpy())
        np.save(os.path.join(outdir, f"tmax{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


@pytest.mark.parametrize("batched", [False, True])
def test_two_ranks_match_one_rank(batched):
    world = 2
    w = synth.tiny_workload()
    S = w.n_snap
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d, batched), nprocs=world,
                           join=True, start_method="spawn")
        cubes = [np.load(os.path.join(d, f"cube{r}.npy")) for r in range(world)]
        tmax = [float(np.load(os.path.join(d, f"tmax{r}.npy"))[0]) for r in range(world)]
    assert tmax == [2.5, 2.5]
    images = _oracle_stream(w, range(S))
    nt = w.image_size // T_TILE
    single = torch.zeros(S - 2, nt, nt)
    shard.run_shard(S, 1, 0, _make_image_and_tlisi(images), single)
    for c in cubes:
        assert c.shape == (S - 2, nt, nt)
        assert np.array_equal(c, single.numpy())        # halos reproduce the outputs exactly
    a = O.candidates(cubes[0].astype(np.float64), T_TILE, O.MODE_NONPERIODIC)
    b = O.candidates(single.numpy().astype(np.float64), T_TILE, O.MODE_NONPERIODIC)
    assert a["threshold"] == b["threshold"] and a["boxes"] == b["boxes"]
