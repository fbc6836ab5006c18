#!/usr/bin/env python
"""Throughput of the FIP-TOI hot path on the MeerKAT-shaped snapshot stream.

One step = one observation of 1500 snapshots (2016 baselines x 4096 channels
x 4 pols, 2048^2 image, 8 s dumps): for every snapshot the plane fit,
gridding, inverse FFT, grid correction, re-projection and tLISI (S1-S7),
then the periodic candidate search over the 1498-slice tLISI cube (S8).
Inputs are seeded synthetic snapshots resident in HBM (a pool of 40
distinct snapshots = one pulsar period, each 297 MB, larger than L2); the
metric is snapshots/s.  The roofline of the dominant stage divides its
algorithmic bytes (every input byte read once, every output byte written
once) by its CUDA-event time.  The end-to-end number streams the same
observation from pinned host memory through toi_stream_*.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  other workloads: --workload fp16 | uneven | adjoint | localise; --mode 3;
  --image-size N --fov-deg F --channels C; --batch B (default 32)
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
MODE3_HEIGHT_M = 16.4
WORKLOAD = "meerkat-64ant-2016bl-4096ch-4pol-2048px-1500snap"

# Algorithmic HBM bytes of each stage per snapshot (minimum traffic: every
# input byte read once, every output byte written once).
N_BL, N_CH, N_POL, N_IMG = 2016, 4096, 4, 2048
G = 2 * N_IMG


def alg_bytes(nbl=N_BL, nch=N_CH, npol=N_POL, N=N_IMG, T=32):
    g = 2 * N
    vis_b = nbl * nch * npol * 8
    flag_b = nbl * nch * npol
    half_grid_b = (g // 2) * g * 8
    return {
        "prep": flag_b,
        "bin": 0,
        "grid": vis_b + flag_b + half_grid_b,
        "fft_rows": half_grid_b + (g // 2) * N * 8,
        "fft_cols": (g // 2) * N * 8 + N * N * 4,
        "reproject": N * N * 4 * 4,
        "tlisi": (N // T) ** 2 * 4,
        # adjoint (not part of the timed step): dL/dI read, U and the column
        # pass written and read once, the half grid written and read, flags
        # read, grad_vis written
        "backward": N * N * 4 * 3 + 2 * (g // 2) * N * 8 + 2 * half_grid_b + flag_b + vis_b,
    }


ALG_BYTES = alg_bytes()


def scope_table_bytes(nbl=N_BL, nch=N_CH, npol=N_POL, N=N_IMG, vis_bytes=8):
    """The scope table's design-minimum byte model per snapshot, the roofline
    denominator: visibilities and flags read (flags twice: plane fit and
    gridding), the full G x G complex grid written once, two FFT passes (the
    second output-pruned to the N x N real tilted image), re-projection and
    tLISI each reading / writing two N x N float images.  At the MeerKAT
    shape: 264.2 + 2 x 33.0 + 134.2 + 268.4 + 151.0 + 33.6 + 33.6 = 951 MB.
    A design that moves fewer bytes (the half-plane grid, pruned passes)
    keeps this model and shows the saving as throughput above it."""
    g = 2 * N
    vis_b = nbl * nch * npol * vis_bytes
    flag_b = nbl * nch * npol
    grid_b = g * g * 8
    img_b = N * N * 4
    return {"prep": flag_b, "grid": vis_b + flag_b + grid_b, "fft_rows": 2 * grid_b,
            "fft_cols": grid_b + img_b, "reproject": 2 * img_b, "tlisi": 2 * img_b}


PATH_STAGES = ("prep", "grid", "fft_rows", "fft_cols", "reproject", "tlisi")

# DRAM bytes (read + write) per snapshot of the gridder, from an ncu capture
# of the profile case (dram__bytes_read.sum + dram__bytes_write.sum): the
# batched kernel over 16 references to one MeerKAT-shaped snapshot (5001.5 +
# 184.2 MB; each reference streams its visibilities again, L2 being smaller
# than them).  A launch's traffic is this times the snapshots it grids.  The
# single-snapshot kernel has not been captured in its current form.
GRID_DRAM_BYTES_PER_SNAPSHOT = {"batch": 5185.7e6 / 16, "single": None}


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


def parse_cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_host_to_gpu(index):
    """Run this process (and the threads it starts) on the CPU cores local to
    GPU `index`, so that pinned host buffers are first touched on the GPU's own
    memory node; returns the core list, or None when the topology is not
    exposed."""
    import torch
    try:
        prop = torch.cuda.get_device_properties(index)
        dom = getattr(prop, "pci_domain_id", 0)
        path = (f"/sys/bus/pci/devices/{dom:04x}:{prop.pci_bus_id:02x}:"
                f"{prop.pci_device_id:02x}.0/local_cpulist")
        with open(path) as f:
            text = f.read()
        cpus = parse_cpulist(text) & os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
            return text.strip()
    except (OSError, AttributeError, ValueError):
        pass
    return None


def fft_comparison(prof, per_launch, G, dev):
    """cuFFT (through torch.fft), timed with CUDA events on the same device, as
    the comparison baseline of the hand-written inverse transform (stage 4 of
    Section 4.1): a batch of G x G single-precision C2C inverse transforms,
    and the C2R form that, like the library, uses the Hermitian half plane.
    The library's figure is its row pass plus column pass (correction and
    normalisation fused), per snapshot, from the timed step."""
    import torch
    n = max(1, min(per_launch, 8))
    ours = (prof["fft_rows"][0] / max(prof["fft_rows"][1], 1) +
            prof["fft_cols"][0] / max(prof["fft_cols"][1], 1)) / per_launch * 1e3
    out = {"ours_us_per_snapshot": round(ours, 2), "grid": G, "batch": n}
    g = torch.Generator(device=dev).manual_seed(11)
    for name, shape, fn in (("cufft_c2c_us_per_snapshot", (n, G, G),
                             lambda x: torch.fft.ifft2(x)),
                            ("cufft_c2r_us_per_snapshot", (n, G, G // 2 + 1),
                             lambda x: torch.fft.irfft2(x, s=(G, G)))):
        x = torch.randn(*shape, dtype=torch.complex64, device=dev, generator=g)
        y = fn(x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            y = fn(x)
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / 5 / n * 1e3, 2)
        del x, y
        torch.cuda.empty_cache()
    return out


def headline_config(args, world):
    """The `config` object of the headline line (both arms print the same)."""
    snap_mb = N_BL * N_CH * N_POL * 9 / 1e6
    sharded = args.shard_observation and world > 1
    return {"workload": WORKLOAD, "snapshots_per_step": args.snapshots, "mode": args.mode,
            "engine": args.engine + (f"{args.batch}" if args.engine == "batch" else ""),
            "resident_pool": args.pool, "image": N_IMG, "grid": G, "cell_arcsec": 2.0,
            "tlisi_tile": 32, "candidate_mode": "periodic",
            "candidate_search": ("pipelined: observation k's search on a low-priority stream "
                                 "during observation k+1's imaging"
                                 if args.s8_overlap and args.engine == "batch" and not sharded
                                 else "after each observation's imaging"),
            "l2": (f"inputs larger than L2 ({snap_mb:.0f} MB per snapshot, {args.pool} distinct "
                   f"= {snap_mb * args.pool / 1e3:.1f} GB cycled; 40 = one pulsar period)"),
            "parallelism": f"snapshot-shards{world}" if sharded else f"replicas{world}"}


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
    host_cpus = bind_host_to_gpu(local)
    cell = args.fov_deg * 3600.0 / args.image_size if args.fov_deg else 2.0
    w = synth.meerkat_workload(n_snap=args.snapshots, n_chan=args.channels,
                               image_size=args.image_size, cell_arcsec=cell)
    default_shape = (args.image_size, args.channels, args.fov_deg) == (N_IMG, N_CH, None)
    workload = (WORKLOAD if default_shape else
                f"meerkat-64ant-2016bl-{w.n_chan}ch-4pol-{w.image_size}px-"
                f"fov{w.image_size * cell / 3600.0:g}deg-{args.snapshots}snap")
    ab = alg_bytes(w.n_bl, w.n_chan, w.n_pol, w.image_size)
    snap_mb = w.n_bl * w.n_chan * w.n_pol * 9 / 1e6
    if args.mode == 3:
        # antenna heights of ~16 m rms give this array Phi_max ~ 5 (one
        # slab, K = 16), the MeerKAT row of the paper's Table 2
        from dataclasses import replace as _replace
        w = _replace(w, height_sigma_m=MODE3_HEIGHT_M)
        args.engine = "single"
    S = args.snapshots
    T = 32
    nt = w.image_size // T
    pool = make_pool(w, args.pool, dev)
    B = args.batch if args.engine == "batch" else 0
    sharded = args.shard_observation and world > 1
    # Observations are pipelined as a streaming deployment runs them: the
    # candidate search (S8, float64, about 50 ms for 1498 x 64 x 64 on this
    # GPU) of observation k runs on its own low-priority stream while
    # observation k + 1 is imaged on a high-priority one; every step still
    # images its 1500 snapshots and searches its own cube, and the timed
    # region ends when the last search has finished.
    overlap = (args.s8_overlap and B > 0 and not sharded and args.mode == 2)
    lo_prio, hi_prio = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
    img_stream = torch.cuda.Stream(device=dev, priority=hi_prio) if overlap else None
    s8_stream = torch.cuda.Stream(device=dev, priority=lo_prio) if overlap else None
    if overlap:
        torch.cuda.set_stream(img_stream)
    plan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, tlisi_tile=T,
                    batch_max=B, mode=args.mode, grid_rows=args.grid_rows)
    cubes = [torch.empty(S - 2, nt, nt, dtype=torch.float32, device=dev)
             for _ in range(2 if overlap else 1)]
    cube = cubes[0]
    row_bytes = nt * nt * 4
    import concurrent.futures as _cf
    s8_pool = _cf.ThreadPoolExecutor(1) if overlap else None
    s8_pending = [None, None]
    s8_done = []

    def s8_job(c, ev):
        with torch.cuda.stream(s8_stream):          # the worker thread's current stream
            s8_stream.wait_event(ev)
            return toi.tlisi_candidates(c, T, toi.TOI_CAND_PERIODIC, stream=s8_stream)

    step_no = [0]
    if sharded:
        # one observation split across ranks (2-snapshot halos, one all-gather)
        local = torch.empty(-(-(S - 2) // world), nt, nt, dtype=torch.float32, device=dev)

    def image_and_tlisi(s, dst):
        p = pool[s % len(pool)]
        plan.grid(p["uvw"], p["freq"], p["vis"], flag=p["flag"])
        plan.image(0, None)
        return plan.tlisi_update(None, dst)

    def image_batched(first, last, out_base):
        """Snapshots [first, last) in batches of B; the tLISI of image t goes
        to row t - 2 of the cube whose first row is at out_base."""
        for lo in range(first, last, B):
            hi = min(lo + B, last)
            snaps = [pool[s % len(pool)] for s in range(lo, hi)]
            plan.batch(snaps, out_base + (lo - first - 2) * row_bytes)

    def step():
        plan.tlisi_reset()
        if overlap:
            k = step_no[0] % 2
            step_no[0] += 1
            if s8_pending[k] is not None:            # the search still reading this cube
                s8_done.append(s8_pending[k].result())
            image_batched(0, S, cubes[k].data_ptr())
            ev = torch.cuda.Event()
            ev.record(img_stream)
            s8_pending[k] = s8_pool.submit(s8_job, cubes[k], ev)
            return None
        if B and not sharded:
            image_batched(0, S, cube.data_ptr())
            return toi.tlisi_candidates(cube, T, toi.TOI_CAND_PERIODIC)
        if sharded:
            if B:   # this rank's [lo - 2, hi) through the batched engine
                def image_batch(s0, s1, row):
                    snaps = [pool[s % len(pool)] for s in range(s0, s1)]
                    return plan.batch(snaps, local.data_ptr() + row * row_bytes)
                shard.run_shard_batched(S, world, rank, image_batch, B)
            else:
                shard.run_shard(S, world, rank, image_and_tlisi, local)
            full = shard.gather_cube(local, S, world, rank)
            return toi.tlisi_candidates(full, T, toi.TOI_CAND_PERIODIC)
        for s in range(S):
            image_and_tlisi(s, cube[s - 2] if s >= 2 else None)
        return toi.tlisi_candidates(cube, T, toi.TOI_CAND_PERIODIC)

    def drain():
        out = None
        for k in (0, 1):
            if s8_pending[k] is not None:
                s8_done.append(s8_pending[k].result())
                s8_pending[k] = None
        if s8_done:
            out = s8_done[-1]
        return out

    for _ in range(args.warmup):
        step()
    drain()
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
    s8_done.clear()
    for _ in range(args.steps):
        found = step()
    if overlap:
        found = drain()                       # the last observations' searches
        assert len(s8_done) == args.steps
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
    # the plan's profiled stage launches, plus the periodic candidate search's
    # six kernels (mean, twiddles, centring, periodogram, harmonic sum, labels)
    # once per step
    launches = sum(v[1] for v in prof.values()) + 6 * args.steps

    # roofline of the dominant stage (CUDA events on the plan's stream)
    peak, peak_kind = load_peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0]
    if sharded:
        first, last = shard.image_range(S, world, rank)
        imaged = (last - first) * args.steps
    else:
        imaged = S * args.steps
    sb = scope_table_bytes(w.n_bl, w.n_chan, w.n_pol, w.image_size)
    dom_b = sb.get(dom, ab[dom])
    achieved = dom_b * imaged / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    design = ab[dom] * imaged / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    path_b = sum(sb[k] for k in PATH_STAGES)
    path_gbs = path_b * imaged / (ms / 1e3) / 1e9
    per_launch = args.batch if args.engine == "batch" else 1
    per_snap = GRID_DRAM_BYTES_PER_SNAPSHOT[args.engine]
    traffic = (per_snap * per_launch
               if per_snap and dom == "grid" and args.mode == 2 and default_shape else None)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "alg_bytes_per_launch": dom_b * per_launch,
                "byte_model": "scope table (full grid written once, flags read twice)",
                "share": round(dom_ms / sum(v[0] for v in prof.values()), 3),
                "path_alg_bytes_per_snapshot": path_b,
                "path_gbs": round(path_gbs, 1), "path_frac": round(path_gbs / peak, 4),
                "design_model": {"alg_bytes_per_launch": ab[dom] * per_launch,
                                 "achieved": round(design, 1),
                                 "frac": round(design / peak, 4),
                                 "note": "half-plane grid, flags read once per stage"}}
    stages = {k: {"ms_per_launch": round(v[0] / max(v[1], 1), 4), "launches": v[1]}
              for k, v in prof.items()}

    # end to end through the streaming API from pinned host memory
    # the Python batch pipeline (pipeline.StreamingImager): the end-to-end
    # number when sharded or asked for with --e2e-engine batch
    e2e = None
    use_native = args.e2e_engine == "native" and not sharded
    if not args.no_e2e and not use_native:
        hpool = []
        for p in pool[:args.host_pool]:
            hpool.append({k: v.cpu().pin_memory() for k, v in p.items()})
        cube_host = torch.empty(S - 2, nt, nt, dtype=torch.float32).pin_memory()
        si = StreamingImager(plan, w.n_bl, w.n_chan, w.n_pol, batch=B,
                             copy_streams=args.copy_streams, depth=args.e2e_depth)
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
               "host_pool_snapshots": args.host_pool, "copy_streams": args.copy_streams,
               "staging_depth": args.e2e_depth,
               "engine": args.engine + (f"{B}" if B else "")}

    # end to end through the native multi-stream runtime (toi_stream_*)
    if not args.no_e2e and use_native:
        nplan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, tlisi_tile=T,
                         grid_slots=3)
        hpool_n = []
        for p in pool[:args.host_pool]:
            hpool_n.append({k: v.cpu().pin_memory() for k, v in p.items()})
        sn = toi.Stream(nplan, host_depth=16, n_copy=args.copy_streams)
        row_host = torch.empty(nt, nt, dtype=torch.float32)

        def native_obs():
            h2d = d2h = 0
            for s_ in range(S):
                # the host row ring holds 16 rows: the oldest is popped when full
                while sn.pending_rows >= 15:
                    sn.pop(wait=True, out=row_host)
                    d2h += row_bytes
                hp = hpool_n[s_ % len(hpool_n)]
                sn.push(hp)
                h2d += sum(v.numel() * v.element_size() for v in hp.values())
                while sn.pop(wait=False, out=row_host) is not None:
                    d2h += row_bytes
            while sn.pop(wait=True, out=row_host) is not None:
                d2h += row_bytes
            return h2d, d2h

        for _ in range(args.e2e_warmup):
            native_obs()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(args.e2e_steps):
            a_, b_ = native_obs()
            h2d += a_
            d2h += b_
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        es = time.perf_counter() - e0
        sn.close()
        nplan.close()
        # the host link alone: pinned host -> device copies of one snapshot's bytes
        src_h = hpool_n[0]["vis"]
        dst_d = torch.empty_like(src_h, device=dev)
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            dst_d.copy_(src_h, non_blocking=True)
        l0.record()
        for _ in range(5):
            dst_d.copy_(src_h, non_blocking=True)
        l1.record()
        torch.cuda.synchronize()
        link_gbs = 5 * src_h.numel() * src_h.element_size() / (l0.elapsed_time(l1) / 1e3) / 1e9
        del dst_d
        e2e_gbs = h2d / es / 1e9          # all timed observations' host -> device bytes
        e2e = {"value": round(S * args.e2e_steps * world / es, 2), "unit": "snapshots/s",
               "h2d_bytes_per_step": h2d // args.e2e_steps,
               "d2h_bytes_per_step": d2h // args.e2e_steps,
               "h2d_gbs": round(e2e_gbs, 1), "link_h2d_gbs": round(link_gbs, 1),
               "link_frac": round(e2e_gbs / link_gbs, 3),
               "host_pool_snapshots": args.host_pool, "copy_streams": args.copy_streams,
               "host_cpus": host_cpus,
               "engine": "toi_stream (pipeline stages on their own CUDA streams, depth-3 "
                         "grid ring, depth-5 image ring)"}

    mode3_plan = plan.mode3_info() if args.mode == 3 else None
    fft_cmp = None
    if rank == 0 and args.mode == 2 and not args.no_fft_comparison:
        fft_cmp = fft_comparison(prof, per_launch, 2 * w.image_size, dev)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and default_shape:
        cpu = cpu_baseline()
    plan.close()
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 2), "unit": "snapshots/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
               "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded MeerKAT-shaped snapshots, resident pool)",
               "config": (headline_config(args, world) if default_shape and args.mode == 2 else
                          {"workload": workload + ("-3d-heights16m" if args.mode == 3 else ""),
                           "snapshots_per_step": S, "mode": args.mode,
                           "mode3_plan": mode3_plan,
                           "engine": args.engine + (f"{B}" if B else ""),
                           "resident_pool": args.pool, "image": w.image_size,
                           "grid": 2 * w.image_size, "cell_arcsec": round(cell, 6),
                           "tlisi_tile": T, "candidate_mode": "periodic",
                           "l2": (f"inputs larger than L2 ({snap_mb:.0f} MB per snapshot, "
                                  f"{args.pool} distinct = {snap_mb * args.pool / 1e3:.1f} GB "
                                  f"cycled)"),
                           "parallelism": (f"snapshot-shards{world}" if sharded
                                           else f"replicas{world}")}),
               "fft_comparison": fft_cmp,
               "roofline": roofline, "stages": stages, "gpu_launches": int(launches),
               "candidates_found": found[2] if found else None,
               "clocks": ck, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_uneven(args):
    """The batched uneven stream: 512 snapshots of the MeerKAT-shaped array
    with per-snapshot channel counts in {1024, 2048, 4096} (contiguous
    sub-bands), flag fractions uniform in [0, 0.6] and 1024^2 or 2048^2
    images, imaged in batches of --batch per image size (one plan per size,
    autotuned), optionally by replaying one captured batch launch."""
    import torch

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    S, B, P, T = 512, args.batch, args.pool, 32
    base = synth.meerkat_workload(n_snap=S)
    specs = synth.uneven_stream(base, S, seed=23, channel_choices=(1024, 2048, 4096),
                                flag_max=0.6, image_sizes=(1024, 2048))
    pool = []
    for i in range(P):
        sn = synth.make_snapshot(specs[i], i, device=dev, uvw_index=i)
        sn.pop("weight")
        pool.append(sn)
    sizes = sorted({specs[i].image_size for i in range(P)})
    stream = torch.cuda.Stream()
    plans, cubes, tuned = {}, {}, {}
    for N in sizes:
        plans[N] = toi.Plan(N, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol,
                            tlisi_tile=T, batch_max=B, stream=stream)
        count = sum(1 for s in range(S) if specs[s % P].image_size == N)
        cubes[N] = torch.empty(max(count - 2, 1), N // T, N // T, dtype=torch.float32, device=dev)
        sample = [pool[i] for i in range(P) if specs[i].image_size == N][:B]
        tuned[N] = plans[N].autotune(sample)
    graphs = {}

    def run_batch(N, idx, t0):
        plan = plans[N]
        snaps = [pool[s % P] for s in idx]
        row = (N // T) ** 2 * 4
        out = cubes[N].data_ptr() + (t0 - 2) * row
        if not args.graph:
            plan.batch(snaps, out)
            return
        stream.synchronize()
        plan.batch_prepare(snaps, out)
        if N not in graphs:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                plan.batch_run()
            graphs[N] = g
        with torch.cuda.stream(stream):
            graphs[N].replay()

    def step():
        pending = {N: [] for N in sizes}
        done = {N: 0 for N in sizes}
        for p in plans.values():
            p.tlisi_reset()
        for s in range(S):
            N = specs[s % P].image_size
            pending[N].append(s)
            if len(pending[N]) == B:
                run_batch(N, pending[N], done[N])
                done[N] += B
                pending[N] = []
        for N in sizes:
            if pending[N]:
                run_batch(N, pending[N], done[N])
                done[N] += len(pending[N])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for p in plans.values():
        if p.sync_status() != toi.TOI_OK:
            raise RuntimeError(p.last_error())
        p.profile_read()
        p.profile_enable(not args.graph)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = {}
    for p in plans.values():
        for k, v in p.profile_read().items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += v[0]
            a[1] += v[1]
        p.profile_enable(False)
        if p.sync_status() != toi.TOI_OK:
            raise RuntimeError(p.last_error())
    alg = {k: 0 for k in ALG_BYTES}
    for s in range(S):
        w = specs[s % P]
        for k, v in alg_bytes(base.n_bl, w.n_chan, base.n_pol, w.image_size).items():
            alg[k] += v * args.steps
    peak, peak_kind = load_peaks()
    roofline = None
    if prof and prof.get("grid", [0])[0] > 0:
        g_ms = prof["grid"][0]
        achieved = alg["grid"] / (g_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": "grid", "achieved": round(achieved, 1),
                    "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": None,
                    "share": round(g_ms / sum(v[0] for v in prof.values()), 3)}
    value = S * args.steps / (ms / 1e3)
    print(json.dumps({
        "metric": METRIC, "value": round(value, 2), "unit": "snapshots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded uneven MeerKAT-array snapshots, resident pool)",
        "config": {"workload": "meerkat-uneven-512snap-1024to4096ch-0to60pctflags-1024or2048px",
                   "batch": B, "graph": bool(args.graph), "resident_pool": P,
                   "autotuned_runs": {str(N): tuned[N][0] for N in sizes},
                   "l2": "inputs larger than L2"},
        "roofline": roofline,
        "stages": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]},
        "clocks": ck}))
    for p in plans.values():
        p.close()


def run_fp16(args):
    """The precision workload: one observation of 300 distinct snapshots of
    the faint-transient stream at the MeerKAT shape (two transients at 3 and
    5 sigma of the image noise in 10-snapshot windows, a pulsar ramping from
    1 to 2 Jy, 5 % flags), imaged by the batched engine with the visibilities
    stored as FP16 pairs with a per-channel FP32 scale (FP32 gridding and FFT,
    FP64 plane fit and coordinate factors), then the non-periodic candidate
    search (Section 6.3, 4 sigma).  The same observation stored as complex64
    is timed next to it, and the two pipelines' images are compared on every
    25th snapshot."""
    import torch

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    host_cpus = bind_host_to_gpu(0)
    S = args.snapshots if args.snapshots != 1500 else 300
    B, T = args.batch, 32
    w = synth.faint_transient_workload(n_snap=S)
    nt = w.image_size // T
    peak, peak_kind = load_peaks()
    sample = list(range(2, S, 25))
    results, images = {}, {}
    for storage in ("fp16", "c64"):
        snaps = []
        for s in range(S):
            sn = synth.make_snapshot(w, s, device=dev)
            sn.pop("weight")
            if storage == "fp16":
                q, scale = synth.to_fp16_channel_scaled(sn["vis"])
                sn["vis"], sn["chan_scale"] = q, scale
            snaps.append(sn)
        torch.cuda.synchronize()
        vdt = toi.TOI_VIS_C16_CHANSCALE if storage == "fp16" else toi.TOI_VIS_C64
        plan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, tlisi_tile=T,
                        batch_max=B, vis_dtype=vdt)
        cube = torch.empty(S, nt, nt, dtype=torch.float32, device=dev)

        def step(with_images=False):
            plan.tlisi_reset()
            for lo in range(0, S, B):
                hi = min(S, lo + B)
                group = snaps[lo:hi]
                if with_images:
                    group = [dict(g, image=images[storage][i]) if i in images[storage] else g
                             for i, g in zip(range(lo, hi), group)]
                plan.batch(group, cube[lo:hi])
            return toi.tlisi_candidates(cube[2:], T, toi.TOI_CAND_NONPERIODIC)

        images[storage] = {i: torch.empty(w.image_size, w.image_size, device=dev) for i in sample}
        step(with_images=True)
        for _ in range(args.warmup):
            step()
        if plan.sync_status() != toi.TOI_OK:
            raise RuntimeError(plan.last_error())
        plan.profile_read()
        plan.profile_enable(True)
        clocks = ClockSampler(0)
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
        ck = clocks.stop()
        ms = t0.elapsed_time(t1)
        prof = plan.profile_read()
        plan.profile_enable(False)
        if plan.sync_status() != toi.TOI_OK:
            raise RuntimeError(plan.last_error())
        n = S * args.steps
        sb = scope_table_bytes(w.n_bl, w.n_chan, w.n_pol, w.image_size,
                          vis_bytes=4 if storage == "fp16" else 8)
        g_ms = prof["grid"][0]
        g_gbs = sb["grid"] * n / (g_ms / 1e3) / 1e9
        path_b = sum(sb[k] for k in PATH_STAGES)
        path_gbs = path_b * n / (ms / 1e3) / 1e9
        results[storage] = {
            "value": round(n / (ms / 1e3), 2), "ms_per_step": round(ms / args.steps, 3),
            "candidates": found[2], "boxes": found[1], "threshold": found[0],
            "roofline": {"bound": "hbm", "kernel": "grid", "achieved": round(g_gbs, 1),
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": round(g_gbs / peak, 4), "traffic": None,
                         "alg_bytes_per_launch": sb["grid"] * B,
                         "share": round(g_ms / sum(v[0] for v in prof.values()), 3),
                         "path_alg_bytes_per_snapshot": path_b, "path_gbs": round(path_gbs, 1),
                         "path_frac": round(path_gbs / peak, 4)},
            "stages": {k: {"ms_per_launch": round(v[0] / max(v[1], 1), 4), "launches": v[1]}
                       for k, v in prof.items() if v[1]},
            # the non-periodic search: two kernels (scores, labels) per step
            "gpu_launches": int(sum(v[1] for v in prof.values()) + 2 * args.steps),
            "clocks": ck}
        plan.close()
        del snaps, cube
        torch.cuda.empty_cache()
    diffs = []
    for i in sample:
        a, b = images["fp16"][i], images["c64"][i]
        diffs.append(float((a - b).abs().max() / b.abs().max()))
    r16, r32 = results["fp16"], results["c64"]
    print(json.dumps({
        "metric": METRIC, "value": r16["value"], "unit": "snapshots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r16["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (visibilities stored f16 + per-channel f32 scale)",
        "data": "synthetic (seeded faint-transient MeerKAT-shaped stream, all snapshots distinct "
                "and resident)",
        "config": {"workload": f"meerkat-faint-transients-2016bl-4096ch-4pol-2048px-{S}snap-fp16",
                   "snapshots_per_step": S, "engine": f"batch{B}",
                   "candidate_mode": "nonperiodic (4 sigma)", "host_cpus": host_cpus,
                   "l2": "inputs larger than L2 (165 MB per FP16 snapshot, all distinct)"},
        "roofline": r16["roofline"], "stages": r16["stages"],
        "gpu_launches": r16["gpu_launches"], "clocks": r16["clocks"],
        "candidates": {"fp16": {"n": r16["candidates"], "boxes": r16["boxes"],
                                "threshold": r16["threshold"]},
                       "c64": {"n": r32["candidates"], "boxes": r32["boxes"],
                               "threshold": r32["threshold"]},
                       "same_boxes": r16["boxes"] == r32["boxes"]},
        "fp16_vs_c64_image_max_rel_err": {"max": max(diffs), "snapshots": sample,
                                          "per_snapshot": [round(d, 9) for d in diffs]},
        "c64_same_stream": {"value": r32["value"], "ms_per_step": r32["ms_per_step"],
                            "roofline": r32["roofline"], "stages": r32["stages"],
                            "clocks": r32["clocks"]},
        "e2e": None, "cpu_baseline": None}))


def run_adjoint(args):
    """Forward and reverse mode of the MeerKAT-shaped snapshot image: per
    snapshot toi_grid + toi_image, then toi_degrid_backward for a fixed
    image cotangent with the visibility and weight gradients."""
    import torch

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    S = args.snapshots
    w = synth.meerkat_workload(n_snap=S)
    pool = make_pool(w, args.pool, dev)
    N = w.image_size
    plan = toi.Plan(N, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol)
    g = torch.Generator(device=dev).manual_seed(5)
    grad_img = torch.randn(N, N, generator=g, device=dev)
    img = torch.empty(N, N, device=dev)
    gv = torch.empty(w.n_bl, w.n_chan, w.n_pol, dtype=torch.complex64, device=dev)
    gw = torch.empty(w.n_bl, w.n_chan, w.n_pol, dtype=torch.float32, device=dev)

    def step():
        for s in range(S):
            p = pool[s % len(pool)]
            plan.grid(p["uvw"], p["freq"], p["vis"], flag=p["flag"])
            plan.image(0, img)
            plan.degrid_backward(grad_img, image=img, grad_vis=gv, grad_weight=gw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if plan.sync_status() != toi.TOI_OK:
        raise RuntimeError(plan.last_error())
    plan.profile_read()
    plan.profile_enable(True)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = plan.profile_read()
    plan.close()
    n = S * args.steps
    bw_ms = prof["backward"][0]
    peak, peak_kind = load_peaks()
    achieved = ALG_BYTES["backward"] * n / (bw_ms / 1e3) / 1e9
    print(json.dumps({
        "metric": "snapshots/s forward image + reverse mode (grad vis and weights) at MeerKAT shape",
        "value": round(n / (ms / 1e3), 2), "unit": "snapshots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded MeerKAT-shaped snapshots, resident pool)",
        "config": {"workload": "meerkat-adjoint-" + str(S) + "snap", "resident_pool": args.pool},
        "roofline": {"bound": "hbm", "kernel": "backward", "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "alg_bytes_per_launch": ALG_BYTES["backward"]},
        "stages": {k: {"ms_per_snapshot": round(v[0] / n, 4)} for k, v in prof.items() if v[1]},
        "clocks": ck}))


def run_localise(args):
    """Differentiable localisation at MeerKAT shape (200 snapshots, 64
    windows of 32 x 32 per snapshot): per snapshot toi_grid + toi_image +
    tLISI, then (once three images exist) toi_localise_seed picks the 64
    smallest-tLISI tiles and toi_localise evaluates the point-source loss
    with its source and weight gradients."""
    import torch

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    S = args.snapshots if args.snapshots != 1500 else 200   # the localisation set: 200
    NW = args.windows
    w = synth.meerkat_workload(n_snap=S)
    pool = make_pool(w, args.pool, dev)
    N, T = w.image_size, 32
    nt = N // T
    plan = toi.Plan(N, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, tlisi_tile=T, max_windows=NW)
    row = torch.empty(nt, nt, device=dev)
    win = torch.empty(NW, 2, dtype=torch.int32, device=dev)
    src = torch.empty(NW, 3, dtype=torch.float64, device=dev)
    loss = torch.empty(NW, dtype=torch.float64, device=dev)
    gsrc = torch.empty(NW, 3, dtype=torch.float64, device=dev)
    gw = torch.empty(w.n_bl, w.n_chan, w.n_pol, dtype=torch.float32, device=dev)

    def step():
        plan.tlisi_reset()
        for s in range(S):
            p = pool[s % len(pool)]
            plan.grid(p["uvw"], p["freq"], p["vis"], flag=p["flag"])
            plan.image(0, None)
            if plan.tlisi_update(None, row):
                plan.localise_seed(row, NW, win=win, src=src)
                plan.localise(win, src, loss=loss, grad_src=gsrc, grad_weight=gw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if plan.sync_status() != toi.TOI_OK:
        raise RuntimeError("localisation status")
    plan.profile_read()
    plan.profile_enable(True)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = plan.profile_read()
    launches = sum(v[1] for v in prof.values())
    plan.close()
    n = S * args.steps
    nloc = (S - 2) * args.steps
    loc_ms = prof["localise"][0]
    # FP32 arithmetic of the facet passes: 64 taps x (2 FMA gridding + 2 FMA
    # degridding) per selected sample per window
    nsel = w.n_bl * w.n_chan * (1.0 - w.flag_frac ** 2)
    flops = nsel * NW * 64 * 8 * nloc
    sm_mhz = (ck or {}).get("sm_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (loc_ms / 1e3) / 1e12
    print(json.dumps({
        "metric": "snapshots/s of imaging + windowed point-source localisation (loss, d/d(l,m,S), "
                  "d/dweights) at MeerKAT shape",
        "value": round(n / (ms / 1e3), 2), "unit": "snapshots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded MeerKAT-shaped snapshots, resident pool)",
        "config": {"workload": f"meerkat-localise-{S}snap-{NW}windows-32px",
                   "resident_pool": args.pool, "windows_per_snapshot": NW,
                   "localised_snapshots_per_step": S - 2},
        "windows_per_s": round(NW * nloc / (ms / 1e3), 1),
        "roofline": {"bound": "alu", "kernel": "localise (facet gridding + degridding)",
                     "achieved": round(achieved, 2), "peak": round(peak, 1),
                     "peak_kind": f"FP32 FMA: {nsm} SMs x 128 lanes x 2 flop x median SM clock",
                     "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None},
        "stages": {k: {"ms_per_snapshot": round(v[0] / n, 4)} for k, v in prof.items() if v[1]},
        "gpu_launches": int(launches), "clocks": ck}))


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


POOL_SNIPPET = r"""
import concurrent.futures as cf, json, multiprocessing as mp, os, sys, time
sys.path.insert(0, {root!r})

def one(s):
    import numpy as np
    from paper_2512_06254_gb300 import synth
    from oracle import toi_oracle as O
    w = synth.meerkat_workload()
    sn = synth.make_snapshot(w, s)
    h = {{k: (v.numpy() if v is not None else None) for k, v in sn.items()}}
    rng = np.random.default_rng(s)
    prev = [rng.normal(size=(w.image_size, w.image_size)) for _ in range(2)]
    t0 = time.time()
    r = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], None, w.image_size,
                         w.cell_arcsec)
    O.tlisi(prev[0], prev[1], r["image"], 32)
    return t0, time.time()

if __name__ == "__main__":
    n, workers = {n}, {workers}
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        spans = list(ex.map(one, range(n)))
    print(json.dumps({{"seconds": max(b for _, b in spans) - min(a for a, _ in spans)}}))
"""


def mem_available_gb():
    """Host memory this process may still use: MemAvailable, capped by the
    cgroup's limit where one is set."""
    avail = 16.0
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) / 1e6
    except OSError:
        pass
    for lim_path, use_path in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                               ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                                "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            with open(lim_path) as f:
                lim = f.read().strip()
            with open(use_path) as f:
                use = int(f.read().strip())
            if lim.isdigit():
                avail = min(avail, (int(lim) - use) / 1e9)
            break
        except (OSError, ValueError):
            continue
    return avail


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def cpu_baseline(snap_index: int = 7, all_cores: bool = True):
    """The FP64 oracle, as it stands, imaging MeerKAT-shaped snapshots (S1-S7)
    in fresh processes: one snapshot on one host core, and (all_cores) 16
    snapshots over a pool of one single-threaded process per host core."""
    code = CPU_SNIPPET.format(root=ROOT, s=snap_index)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       env=_oracle_env(), timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    sec = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    ncores = len(os.sched_getaffinity(0))
    out = {"value": round(1.0 / sec, 5), "unit": "snapshots/s", "cores": 1, "kind": "oracle",
           "sample": "1 MeerKAT-shaped snapshot (2016 bl x 4096 ch x 4 pol, 2048^2): S1-S6 "
                     "imaging + one tLISI matrix, FP64 numpy oracle, 1 thread",
           "seconds": round(sec, 2), "cpu_model": cpu_model(), "nproc": os.cpu_count(),
           "host_cores_available": ncores}
    if all_cores:
        n = 16
        # about 3.5 GB of host memory per oracle process at this shape, more
        # with the interpreter and torch; halve the pool if a worker dies
        workers = max(1, min(n, ncores, int(mem_available_gb() // 6.0)))
        # the pool's worker function must be importable by the spawned
        # processes, so the script runs from a file, not from "-c"
        with tempfile.TemporaryDirectory() as tmp:
            script = os.path.join(tmp, "oracle_pool_timing.py")
            while True:
                with open(script, "w") as f:
                    f.write(POOL_SNIPPET.format(root=ROOT, n=n, workers=workers))
                r = subprocess.run([sys.executable, script], capture_output=True, text=True,
                                   env=_oracle_env(), timeout=1800)
                if r.returncode == 0 or workers == 1:
                    break
                workers = max(1, workers // 2)
        if r.returncode == 0:
            wall = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
            out["all_cores"] = {"value": round(n / wall, 4), "unit": "snapshots/s",
                                "cores": workers, "seconds": round(wall, 2),
                                "sample": f"{n} MeerKAT-shaped snapshots (S1-S6 + one tLISI "
                                          f"matrix each), one single-threaded oracle process "
                                          f"per core, wall time of the imaging"}
        else:
            out["all_cores"] = {"error": r.stderr[-300:]}
    return out


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
        cb = cpu_baseline(snap_index=k, all_cores=False)
        if "error" in cb:
            print(json.dumps({"impl": "reference", "unavailable": cb["error"][-200:]}))
            return
        secs.append(cb["seconds"])
    total = sum(secs)
    value = args.steps / total
    cpu = {"value": round(value, 5), "unit": "snapshots/s", "cores": 1, "kind": "oracle",
           "sample": "1 MeerKAT-shaped snapshot per step (S1-S6 + one tLISI matrix), FP64 numpy",
           "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(value, 5),
                      "unit": "snapshots/s", "n_gpus": world, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 1),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f64", "data": "synthetic (seeded MeerKAT-shaped snapshots)",
                      "config": headline_config(args, world),
                      "reference_sample": "each step images 1 MeerKAT-shaped snapshot of the "
                                          "workload with the FP64 oracle on 1 host core",
                      "cpu_baseline": cpu,
                      "e2e": {"value": round(value, 5), "unit": "snapshots/s",
                              "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def profile_case(args):
    """Small case for ncu captures: one MeerKAT-shaped snapshot resident on the
    device, `--profile-case` passes of toi_grid + toi_image + tlisi_update
    (--engine single) or of toi_batch over --batch references to it
    (--engine batch)."""
    import torch

    import paper_2512_06254_gb300 as toi
    from paper_2512_06254_gb300 import synth
    cell = args.fov_deg * 3600.0 / args.image_size if args.fov_deg else 2.0
    w = synth.meerkat_workload(n_chan=args.channels, image_size=args.image_size, cell_arcsec=cell)
    p = synth.make_snapshot(w, 3, device="cuda", uvw_index=3)
    batch = args.engine == "batch"
    B = args.batch if batch else 0
    plan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, batch_max=B)
    nt = w.image_size // 32
    out = torch.empty(max(B, 1), nt, nt, device="cuda")
    for _ in range(args.profile_case):
        if batch:   # one resident snapshot referenced B times: B launches' worth of work
            plan.batch([p] * B, out)
        else:
            plan.grid(p["uvw"], p["freq"], p["vis"], flag=p["flag"])
            plan.image(0, None)
            plan.tlisi_update(None, out[0])
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
    ap.add_argument("--no-fft-comparison", action="store_true",
                    help="skip the cuFFT comparison of the inverse transform")
    ap.add_argument("--s8-overlap", type=int, default=0, choices=[0, 1],
                    help="1: the candidate search of observation k runs on a low-priority stream "
                         "while observation k + 1 is imaged (batched engine)")
    ap.add_argument("--engine", default="batch", choices=["single", "batch"],
                    help="single: toi_grid + toi_image + tlisi_update per snapshot; batch: "
                         "toi_batch over --batch snapshots per launch")
    ap.add_argument("--batch", type=int, default=None,
                    help="snapshots per batched launch (default 32; 16 for --workload uneven, "
                         "the batched-stream configuration's B)")
    ap.add_argument("--grid-rows", type=int, default=0, choices=[0, 4, 8],
                    help="gridder window rows per lane (0: the library's default)")
    ap.add_argument("--mode", type=int, default=2, choices=[2, 3],
                    help="3: near-coplanar imaging (slabs + Chebyshev moments) of the stream "
                         "with antenna heights (single engine)")
    ap.add_argument("--image-size", type=int, default=N_IMG,
                    help="N of the MeerKAT-shaped stream (the paper's sweep: 2048 ... 10240)")
    ap.add_argument("--fov-deg", type=float, default=None,
                    help="field of view in degrees (cell = fov / N; default 2 arcsec cells)")
    ap.add_argument("--channels", type=int, default=N_CH,
                    help="channels per snapshot (the paper's MeerKAT set has 1024)")
    ap.add_argument("--e2e-engine", default="native", choices=["native", "batch"],
                    help="end-to-end path: toi_stream_* (native stage streams, default) or the "
                         "Python batch pipeline")
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="e2e: staging slots (of a batch each with the batch engine)")
    ap.add_argument("--copy-streams", type=int, default=4,
                    help="e2e: copy streams each snapshot's host-to-device copy is split over")
    ap.add_argument("--windows", type=int, default=64,
                    help="localise workload: candidate windows per snapshot")
    ap.add_argument("--workload", default="meerkat",
                    choices=["meerkat", "uneven", "adjoint", "localise", "fp16"],
                    help="meerkat: the headline stream; uneven: the batched uneven stream "
                         "(512 snapshots, 1024-4096 channels, 0-60%% flags, 1024/2048 px); "
                         "fp16: 300 faint-transient snapshots stored as FP16 + channel scale, "
                         "next to the same stream in complex64")
    ap.add_argument("--graph", action="store_true",
                    help="uneven workload: replay one captured toi_batch_run per batch")
    ap.add_argument("--shard-observation", action="store_true",
                    help="with N > 1 ranks, split one observation across them (strong scaling) "
                         "instead of one observation per rank")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="run N imaging passes of one snapshot (for ncu) and exit")
    args = ap.parse_args()
    if args.batch is None:
        args.batch = 16 if args.workload == "uneven" else 32
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "fp16":
        run_fp16(args)
    elif args.workload == "localise":
        run_localise(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
