"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
FP64 oracle on the same seeded inputs)."""
import numpy as np
import torch

import paper_2512_06254_gb300 as toi


def to_dev(snap):
    return {k: (v.cuda() if v is not None else None) for k, v in snap.items()}


def to_np(snap):
    return {k: (v.numpy() if v is not None else None) for k, v in snap.items()}


def plan_for(w, **kw):
    return toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, **kw)


def gpu_image(plan, dsnap, slot=0, out=True):
    """toi_grid + toi_image for one device snapshot; numpy outputs."""
    N = plan.N
    img = torch.empty(N, N, dtype=torch.float32, device="cuda") if out else None
    info = torch.empty(16, dtype=torch.float64, device="cuda")
    plan.grid(dsnap["uvw"], dsnap["freq"], dsnap["vis"], flag=dsnap["flag"],
              weight=dsnap.get("weight"), chan_scale=dsnap.get("chan_scale"), slot=slot)
    plan.image(slot, img, info)
    st = plan.sync_status()
    return dict(status=st, image=None if img is None else img.cpu().numpy(),
                info=info.cpu().numpy())


def rel_err(a, b):
    """max |a - b| / max |b|."""
    a = np.asarray(a)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
