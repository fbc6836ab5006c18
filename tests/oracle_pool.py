"""Oracle images of seeded snapshots, computed in a pool of host processes.

Each job names a synthetic workload, a snapshot index and options; the
worker regenerates that snapshot on the CPU from its seed (synth.py) and
images it with the FP64 oracle, so no large array crosses a process
boundary on the way in.  The pool uses the 'spawn' start method, so it is
safe to start after CUDA has been initialised in the parent.  Test
infrastructure only."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
from dataclasses import dataclass
from typing import List, Optional


@dataclass(frozen=True)
class Job:
    workload: object            # synth.Workload (frozen dataclass, picklable)
    snap: int                   # snapshot index s (sky schedule, noise and flag seeds)
    uvw_index: Optional[int] = None
    with_weights: bool = False
    keep: tuple = ("image",)    # keys of the oracle result to return
    fp16: bool = False          # also image the FP16-stored values (decoded) -> "image_dec",
                                # with the quantisation bound sum |dc| / (omega sum w) -> "bound"


def _run(job: Job):
    import numpy as np
    import torch
    from paper_2512_06254_gb300 import synth
    from oracle import toi_oracle as O
    w = job.workload
    sn = synth.make_snapshot(w, job.snap, with_weights=job.with_weights, uvw_index=job.uvw_index)
    h = {k: (v.numpy() if v is not None else None) for k, v in sn.items()}
    r = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], w.image_size,
                         w.cell_arcsec)
    out = {k: np.asarray(r[k]) for k in job.keep}
    if job.fp16:
        q, scale = synth.to_fp16_channel_scaled(sn["vis"])
        qd = q.double()
        dec = torch.complex(qd[..., 0], qd[..., 1]) * scale.double()[None, :, None]
        rd = O.image_snapshot(h["uvw"], h["freq"], dec.numpy(), h["flag"], h["weight"],
                              w.image_size, w.cell_arcsec)
        out["image_dec"] = np.asarray(rd["image"])
        pa, pb = O.parallel_hands(w.n_pol)
        d = (dec - sn["vis"].to(torch.complex128)).numpy()
        keep = (h["flag"] == 0)
        wts = h["weight"] if h["weight"] is not None else np.ones(keep.shape)
        dc = d[..., pa] * keep[..., pa] * wts[..., pa]
        if pb != pa:
            dc = dc + d[..., pb] * keep[..., pb] * wts[..., pb]
        out["bound"] = float(np.abs(dc).sum()) / (r["omega"] * r["sumw"])
    return out


def _init():
    # one BLAS / OpenMP thread per worker: the pool supplies the parallelism
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def oracle_images(jobs: List[Job], workers: Optional[int] = None):
    """Oracle results of every job, in order."""
    n = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    if n == 1:
        return [_run(j) for j in jobs]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=n, mp_context=ctx, initializer=_init) as ex:
        return list(ex.map(_run, jobs))
