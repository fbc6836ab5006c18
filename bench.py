#!/usr/bin/env python
"""Throughput of the FIP-TOI hot path on the MeerKAT-shaped snapshot stream.

One step = one observation of 1500 snapshots (2016 baselines x 4096 channels
x 4 pols, 2048^2 image, 8 s dumps): for every snapshot the plane fit,
gridding, inverse FFT, grid correction, re-projection and tLISI (S1-S7),
then the periodic candidate search over the 1498-slice tLISI cube (S8).
Inputs are seeded synthetic snapshots resident in HBM (a pool of 40
distinct snapshots = one pulsar period, each 297 MB, larger than L2); the
metric is snapshots/s.  See the design doc for the roofline model.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "snapshots/s end-to-end (grid+iFFT+tLISI) at MeerKAT shape; % HBM roofline"
WORKLOAD = "meerkat-64ant-2016bl-4096ch-4pol-2048px-1500snap"

# Algorithmic HBM bytes per launch of each stage at this workload (minimum
# traffic: every input byte read once, every output byte written once).
N_BL, N_CH, N_POL, N_IMG = 2016, 4096, 4, 2048
G = 2 * N_IMG
VIS_B = N_BL * N_CH * N_POL * 8
FLAG_B = N_BL * N_CH * N_POL
HALF_GRID_B = (G // 2) * G * 8
ALG_BYTES = {
    "prep": FLAG_B,
    "bin": 0,
    "grid": VIS_B + FLAG_B + HALF_GRID_B,
    "fft_rows": HALF_GRID_B + (G // 2) * N_IMG * 8,
    "fft_cols": (G // 2) * N_IMG * 8 + N_IMG * N_IMG * 4,
    "reproject": N_IMG * N_IMG * 4 * 4,
    "tlisi": 64 * 64 * 4,
    # adjoint (not part of the timed step): dL/dI read, U and the column
    # pass written and read once, the half grid written and read, flags
    # read, grad_vis written
    "backward": (N_IMG * N_IMG * 4 * 3 + 2 * (G // 2) * N_IMG * 8 + 2 * HALF_GRID_B
                 + FLAG_B + VIS_B),
}



def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def make_pool(w, P, device):
    from paper_2512_06254_gb300 import synth
    pool = []
    for i in range(P):
        sn = synth.make_snapshot(w, i, device=device, uvw_index=i)
        sn.pop("weight")
        pool.append(sn)
    return pool


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth
    from paper_2512_06254_gb300 import shard
    from paper_2512_06254_gb300.pipeline import StreamingImager

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.meerkat_workload(n_snap=args.snapshots)
    S = args.snapshots
    T = 32
    nt = w.image_size // T
    pool = make_pool(w, args.pool, dev)
    plan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, tlisi_tile=T)
    cube = torch.empty(S - 2, nt, nt, dtype=torch.float32, device=dev)

    sharded = args.shard_observation and world > 1
    if sharded:
        # one observation split across ranks (2-snapshot halos, one all-gather)
        local = torch.empty(-(-(S - 2) // world), nt, nt, dtype=torch.float32, device=dev)

    def image_and_tlisi(s, dst):
        p = pool[s % len(pool)]
        plan.grid(p["uvw"], p["freq"], p["vis"], flag=p["flag"])
        plan.image(0, None)
        return plan.tlisi_update(None, dst)

    def step():
        plan.tlisi_reset()
        if sharded:
            shard.run_shard(S, world, rank, image_and_tlisi, local)
            full = shard.gather_cube(local, S, world, rank)
            return toi.tlisi_candidates(full, T, toi.TOI_CAND_PERIODIC)
        for s in range(S):
            image_and_tlisi(s, cube[s - 2] if s >= 2 else None)
        return toi.tlisi_candidates(cube, T, toi.TOI_CAND_PERIODIC)

    for _ in range(args.warmup):
        step()
    if plan.sync_status() != toi.TOI_OK:
        raise RuntimeError(plan.last_error())
    plan.profile_read()                       # reset counters
    plan.profile_enable(True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    found = None
    for _ in range(args.steps):
        found = step()
    t1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = plan.profile_read()
    plan.profile_enable(False)
    st = plan.sync_status()
    if st != toi.TOI_OK:
        raise RuntimeError(plan.last_error())
    ms = shard.max_over_ranks(ms, device=dev)
    snaps = S * args.steps * (1 if sharded else world)
    value = snaps / (ms / 1e3)
    launches = sum(v[1] for v in prof.values()) + 5 * args.steps

    # roofline of the dominant stage (CUDA events on the plan's stream)
    peak, peak_kind = load_peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    achieved = ALG_BYTES[dom] * dom_n / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    total_alg = sum(ALG_BYTES[k] * prof[k][1] for k in prof)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None, "alg_bytes_per_launch": ALG_BYTES[dom],
                "share": round(dom_ms / sum(v[0] for v in prof.values()), 3),
                "path_alg_gbs": round(total_alg / (ms / 1e3) / 1e9 * world / world, 1)}
    stages = {k: {"ms_per_launch": round(v[0] / max(v[1], 1), 4), "launches": v[1]}
              for k, v in prof.items()}

    # end to end through the streaming API from pinned host memory
    e2e = None
    if not args.no_e2e:
        hpool = []
        for p in pool[:args.host_pool]:
            hpool.append({k: v.cpu().pin_memory() for k, v in p.items()})
        cube_host = torch.empty(S - 2, nt, nt, dtype=torch.float32).pin_memory()
        si = StreamingImager(plan, w.n_bl, w.n_chan, w.n_pol)
        for _ in range(args.e2e_warmup):
            si.run(hpool, S, cube, cube_host, T)
        si.h2d_bytes = si.d2h_bytes = 0
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            si.run(hpool, S, cube, cube_host, T)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        es = time.perf_counter() - e0
        e2e = {"value": round(S * args.e2e_steps * world / es, 2), "unit": "snapshots/s",
               "h2d_bytes_per_step": si.h2d_bytes // args.e2e_steps,
               "d2h_bytes_per_step": si.d2h_bytes // args.e2e_steps,
               "host_pool_snapshots": args.host_pool}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    plan.close()
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 2), "unit": "snapshots/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
               "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded MeerKAT-shaped snapshots, resident pool)",
               "config": {"workload": WORKLOAD, "snapshots_per_step": S,
                          "resident_pool": args.pool, "image": N_IMG, "grid": G,
                          "tlisi_tile": T, "candidate_mode": "periodic",
                          "l2": "inputs larger than L2 (297 MB per snapshot, 40 distinct = one pulsar period)",
                          "parallelism": (f"snapshot-shards{world}" if sharded
                                          else f"replicas{world}")},
               "roofline": roofline, "stages": stages, "gpu_launches": int(launches),
               "candidates_found": found[2] if found else None,
               "clocks": ck, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


CPU_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_2512_06254_gb300 import synth
from oracle import toi_oracle as O
w = synth.meerkat_workload()
sn = synth.make_snapshot(w, {s})
h = {{k: (v.numpy() if v is not None else None) for k, v in sn.items()}}
rng = np.random.default_rng(0)
prev = [rng.normal(size=(w.image_size, w.image_size)) for _ in range(2)]
t0 = time.perf_counter()
r = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], None, w.image_size, w.cell_arcsec)
t = O.tlisi(prev[0], prev[1], r["image"], 32)
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt}}))
"""


def cpu_baseline(snap_index: int = 7):
    """The FP64 oracle, as it stands, imaging one MeerKAT-shaped snapshot
    (S1-S7) on one host core, in a fresh process."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = CPU_SNIPPET.format(root=ROOT, s=snap_index)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    sec = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    return {"value": round(1.0 / sec, 5), "unit": "snapshots/s", "cores": 1, "kind": "oracle",
            "sample": "1 MeerKAT-shaped snapshot (2016 bl x 4096 ch x 4 pol, 2048^2): S1-S6 "
                      "imaging + one tLISI matrix, FP64 numpy oracle, 1 thread",
            "seconds": round(sec, 2)}


def run_reference(args):
    """The oracle as the reference arm: each step images one MeerKAT-shaped
    snapshot (S1-S7) on the host; warm-up steps image one tiny snapshot."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from paper_2512_06254_gb300 import synth
    from oracle import toi_oracle as O
    tw = synth.tiny_workload()
    for i in range(args.warmup):
        sn = synth.make_snapshot(tw, i)
        h = {k: (v.numpy() if v is not None else None) for k, v in sn.items()}
        O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], None, tw.image_size, tw.cell_arcsec)
    secs = []
    for k in range(args.steps):
        cb = cpu_baseline(snap_index=k)
        if "error" in cb:
            print(json.dumps({"impl": "reference", "unavailable": cb["error"][-200:]}))
            return
        secs.append(cb["seconds"])
    total = sum(secs)
    value = args.steps / total
    cpu = {"value": round(value, 5), "unit": "snapshots/s", "cores": 1, "kind": "oracle",
           "sample": "1 MeerKAT-shaped snapshot per step (S1-S6 + one tLISI matrix), FP64 numpy"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(value, 5),
                      "unit": "snapshots/s", "n_gpus": world, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 1),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f64", "data": "synthetic (seeded MeerKAT-shaped snapshots)",
                      "config": {"workload": WORKLOAD, "snapshots_per_step": 1},
                      "cpu_baseline": cpu,
                      "e2e": {"value": round(value, 5), "unit": "snapshots/s",
                              "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def profile_case(args):
    """Small case for ncu captures: one MeerKAT-shaped snapshot resident on the
    device, `--profile-case` passes of toi_grid + toi_image + tlisi_update."""
    import torch

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth
    w = synth.meerkat_workload()
    p = synth.make_snapshot(w, 3, device="cuda", uvw_index=3)
    plan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol)
    out = torch.empty(w.image_size // 32, w.image_size // 32, device="cuda")
    for _ in range(args.profile_case):
        plan.grid(p["uvw"], p["freq"], p["vis"], flag=p["flag"])
        plan.image(0, None)
        plan.tlisi_update(None, out)
    torch.cuda.synchronize()
    st = plan.sync_status()
    print("profile case done, status", st)
    if st != toi.TOI_OK:
        raise SystemExit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--snapshots", type=int, default=1500)
    ap.add_argument("--pool", type=int, default=40)
    ap.add_argument("--host-pool", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--e2e-warmup", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard-observation", action="store_true",
                    help="with N > 1 ranks, split one observation across them (strong scaling) "
                         "instead of one observation per rank")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="run N imaging passes of one snapshot (for ncu) and exit")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
