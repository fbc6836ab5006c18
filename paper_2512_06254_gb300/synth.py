"""Seeded synthetic snapshot generator (inputs only).

This module builds interferometer snapshots with the shapes, value
distributions and structure of the workloads the FIP-TOI paper measures on
(MeerKAT-like arrays, Measurement-Set column layouts, flagged samples,
steady sources plus transients).  It predicts visibilities with the
van Cittert-Zernike measurement equation (Section 1, Eq. "vis") for point
sources and adds Gaussian noise.  It contains none of the imaging method:
no plane fitting, gridding, Fourier inversion, re-projection or tLISI.

Both the CUDA path and the FP64 checker consume what this module returns.
Every array is produced by torch on the requested device from an explicit
seed; tests generate on the CPU and copy the very same bytes to the GPU.

Layouts follow the Measurement-Set columns named in Section 3.5:
  uvw   float64 [n_bl, 3]            metres (UVW)
  freq  float64 [n_ch]               Hz (CHAN_FREQ), ascending
  vis   complex64 [n_bl, n_ch, n_pol] (DATA; linear feeds XX,XY,YX,YY)
  flag  uint8   [n_bl, n_ch, n_pol]  1 = flagged (FLAG)
  weight float32 [n_bl, n_ch, n_pol] or None (WEIGHT_SPECTRUM)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import torch

C_LIGHT = 299_792_458.0
SIDEREAL_DAY_S = 86_164.0905


@dataclass(frozen=True)
class Source:
    l: float          # direction cosine (east), radians
    m: float          # direction cosine (north), radians
    flux: float       # Jy
    kind: str = "steady"          # steady | window | periodic | ramp
    on_from: int = 0              # window: first snapshot on (inclusive)
    on_to: int = 0                # window: last snapshot on (exclusive)
    period: int = 0               # periodic: period in snapshots
    duty: int = 0                 # periodic: snapshots on per period
    ramp_to: float = 0.0          # ramp: flux at the last snapshot

    def flux_at(self, s: int, n_snap: int) -> float:
        if self.kind == "steady":
            return self.flux
        if self.kind == "window":
            return self.flux if self.on_from <= s < self.on_to else 0.0
        if self.kind == "periodic":
            return self.flux if (s % self.period) < self.duty else 0.0
        if self.kind == "ramp":
            frac = s / max(1, n_snap - 1)
            return self.flux + (self.ramp_to - self.flux) * frac
        raise ValueError(self.kind)


@dataclass(frozen=True)
class Workload:
    """One synthetic observation: array, band, image geometry and sky."""
    name: str
    n_ant: int
    layout: str                   # "disc" | "meerkat"
    n_chan: int
    f_lo_hz: float
    f_hi_hz: float
    n_pol: int
    n_snap: int
    image_size: int
    cell_arcsec: float
    noise_sigma: float            # Jy, per real / imaginary part
    flag_frac: float              # i.i.d. per (baseline, channel, pol)
    seed_layout: int = 1
    seed_sky: int = 2
    seed_flags: int = 3
    seed_noise: int = 1000
    lat_deg: float = -30.71
    dec_deg: float = -30.0
    ha0_hours: float = -0.5
    dump_s: float = 8.0
    layout_radius_m: float = 1000.0
    sources: tuple = field(default_factory=tuple)
    height_sigma_m: float = 0.0   # antenna heights ~ N(0, sigma) (non-coplanar array)
    curvature: bool = False       # antennas on the Earth's surface (height -(e^2+n^2)/2R)

    @property
    def n_bl(self) -> int:
        return self.n_ant * (self.n_ant - 1) // 2

    @property
    def fov_rad(self) -> float:
        return self.image_size * self.cell_arcsec * math.pi / 648000.0


# --------------------------------------------------------------------------
# Array layouts (local east/north/up metres)
# --------------------------------------------------------------------------

def layout_disc(n_ant: int, radius_m: float, seed: int) -> torch.Tensor:
    g = torch.Generator().manual_seed(seed)
    r = radius_m * torch.sqrt(torch.rand(n_ant, generator=g, dtype=torch.float64))
    th = 2 * math.pi * torch.rand(n_ant, generator=g, dtype=torch.float64)
    up = 2.0 * torch.rand(n_ant, generator=g, dtype=torch.float64)
    return torch.stack([r * torch.cos(th), r * torch.sin(th), up], 1)


def layout_meerkat(seed: int, n_core: int = 48, n_arm: int = 16,
                   core_sigma_m: float = 400.0, core_radius_m: float = 1000.0,
                   arm_radius_m: float = 4000.0) -> torch.Tensor:
    """Dense Gaussian core plus three spiral arms (MeerKAT-like, 8 km max)."""
    g = torch.Generator().manual_seed(seed)
    pos = []
    while len(pos) < n_core:
        e, n = (core_sigma_m * torch.randn(2, generator=g, dtype=torch.float64)).tolist()
        if e * e + n * n <= core_radius_m ** 2:
            pos.append((e, n))
    for k in range(n_arm):
        arm = k % 3
        frac = (k // 3 + 1) / (n_arm // 3 + 1)
        r = core_radius_m + (arm_radius_m - core_radius_m) * frac
        jitter = 0.05 * float(torch.rand(1, generator=g, dtype=torch.float64))
        th = 2 * math.pi * arm / 3 + 1.2 * math.log(r / core_radius_m) + jitter
        pos.append((r * math.cos(th), r * math.sin(th)))
    enu = torch.tensor(pos, dtype=torch.float64)
    up = 3.0 * torch.rand(len(pos), generator=g, dtype=torch.float64)
    return torch.cat([enu, up[:, None]], 1)


def array_layout(w: Workload) -> torch.Tensor:
    if w.layout == "disc":
        enu = layout_disc(w.n_ant, w.layout_radius_m, w.seed_layout)
    elif w.layout == "meerkat":
        enu = layout_meerkat(w.seed_layout)
    else:
        raise ValueError(w.layout)
    if w.height_sigma_m > 0.0 or w.curvature:
        enu = enu.clone()
        if w.height_sigma_m > 0.0:
            g = torch.Generator().manual_seed(w.seed_layout + 7)
            enu[:, 2] += w.height_sigma_m * torch.randn(enu.shape[0], generator=g,
                                                        dtype=enu.dtype)
        if w.curvature:
            enu[:, 2] -= (enu[:, 0] ** 2 + enu[:, 1] ** 2) / (2.0 * 6.371e6)
    return enu


def baseline_uvw(enu: torch.Tensor, lat_rad: float, dec_rad: float,
                 ha_rad: float) -> torch.Tensor:
    """UVW (metres) of every antenna pair i<j toward (ha, dec)."""
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    X = -math.sin(lat_rad) * n + math.cos(lat_rad) * u
    Y = e
    Z = math.cos(lat_rad) * n + math.sin(lat_rad) * u
    i, j = torch.triu_indices(enu.shape[0], enu.shape[0], 1)
    bx, by, bz = X[j] - X[i], Y[j] - Y[i], Z[j] - Z[i]
    sh, ch = math.sin(ha_rad), math.cos(ha_rad)
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    uu = sh * bx + ch * by
    vv = -sd * ch * bx + sd * sh * by + cd * bz
    ww = cd * ch * bx - cd * sh * by + sd * bz
    return torch.stack([uu, vv, ww], 1).contiguous()


def frequencies(w: Workload) -> torch.Tensor:
    if w.n_chan == 1:
        return torch.tensor([w.f_lo_hz], dtype=torch.float64)
    step = (w.f_hi_hz - w.f_lo_hz) / w.n_chan
    return w.f_lo_hz + step * torch.arange(w.n_chan, dtype=torch.float64)


def hour_angle(w: Workload, s: int) -> float:
    return (w.ha0_hours * 3600.0 + s * w.dump_s) * 2 * math.pi / SIDEREAL_DAY_S


# --------------------------------------------------------------------------
# Skies
# --------------------------------------------------------------------------

def steady_sources(n: int, s_min: float, s_max: float, fov_rad: float,
                   seed: int, powerlaw: bool) -> List[Source]:
    g = torch.Generator().manual_seed(seed)
    out = []
    for _ in range(n):
        l, m = ((torch.rand(2, generator=g, dtype=torch.float64) - 0.5) * 0.8 * fov_rad).tolist()
        x = float(torch.rand(1, generator=g, dtype=torch.float64))
        if powerlaw:   # dN/dS ~ S^-2 on [s_min, s_max]
            flux = 1.0 / (1.0 / s_min - x * (1.0 / s_min - 1.0 / s_max))
        else:
            flux = s_min + x * (s_max - s_min)
        out.append(Source(l, m, flux))
    return out


def random_position(fov_rad: float, seed: int):
    g = torch.Generator().manual_seed(seed)
    return ((torch.rand(2, generator=g, dtype=torch.float64) - 0.5) * 0.8 * fov_rad).tolist()


# --------------------------------------------------------------------------
# Named workloads (the shapes of the paper's measurements)
# --------------------------------------------------------------------------

def tiny_workload() -> Workload:
    """16 antennas within 1 km, 64 channels 1.0-1.1 GHz, Stokes I, 8
    snapshots, 128x128 pixels of 2 arcsec; 3 steady sources (1-5 Jy) and a
    0.5 Jy transient on in snapshots 3..5; noise 0.1 Jy; no flags."""
    w = Workload("tiny-16ant-64ch-128px", n_ant=16, layout="disc", n_chan=64,
                 f_lo_hz=1.0e9, f_hi_hz=1.1e9, n_pol=1, n_snap=8, image_size=128,
                 cell_arcsec=2.0, noise_sigma=0.1, flag_frac=0.0,
                 layout_radius_m=1000.0)
    src = steady_sources(3, 1.0, 5.0, w.fov_rad, w.seed_sky, powerlaw=False)
    l, m = random_position(w.fov_rad, w.seed_sky + 100)
    src.append(Source(l, m, 0.5, kind="window", on_from=3, on_to=6))
    return replace(w, sources=tuple(src))


def meerkat_workload(n_snap: int = 1500, n_chan: int = 4096,
                     image_size: int = 2048, cell_arcsec: float = 2.0) -> Workload:
    """64-antenna MeerKAT-like array (dense core, arms to 4 km radius), 2016
    baselines, 4096 channels 856-1712 MHz, 4 linear pols, 8 s dumps,
    2048x2048 pixels of 2 arcsec; 10 steady power-law sources (0.1-10 Jy),
    a 1 Jy pulsar on for 20 of every 40 snapshots; 5% flags.  Other image
    sizes and cells keep the sources inside their own field of view."""
    w = Workload(f"meerkat-64ant-{n_chan}ch-{image_size}px", n_ant=64,
                 layout="meerkat", n_chan=n_chan, f_lo_hz=856e6, f_hi_hz=1712e6,
                 n_pol=4, n_snap=n_snap, image_size=image_size, cell_arcsec=cell_arcsec,
                 noise_sigma=0.1, flag_frac=0.05)
    src = steady_sources(10, 0.1, 10.0, w.fov_rad, w.seed_sky, powerlaw=True)
    l, m = random_position(w.fov_rad, w.seed_sky + 100)
    src.append(Source(l, m, 1.0, kind="periodic", period=40, duty=20))
    return replace(w, sources=tuple(src))


def faint_transient_workload(n_snap: int = 300, n_chan: int = 4096, image_size: int = 2048,
                             cell_arcsec: float = 2.0) -> Workload:
    """MeerKAT shape with two faint transients (3 and 5 sigma of the image
    noise of this channel count) in disjoint 10-snapshot windows starting at
    n_snap // 3 and 40 snapshots later (100 and 140 for 300 snapshots), and a
    pulsar whose flux ramps from 1 to 2 Jy over the run."""
    base = meerkat_workload(n_snap=n_snap, n_chan=n_chan, image_size=image_size,
                            cell_arcsec=cell_arcsec)
    n_vis = base.n_bl * base.n_chan * 2 * (1 - base.flag_frac)
    sigma_img = base.noise_sigma / math.sqrt(n_vis)
    src = list(s for s in base.sources if s.kind == "steady")
    t0 = n_snap // 3
    for k, nsig in enumerate((3.0, 5.0)):
        l, m = random_position(base.fov_rad, base.seed_sky + 200 + k)
        src.append(Source(l, m, nsig * sigma_img, kind="window",
                          on_from=t0 + 40 * k, on_to=t0 + 10 + 40 * k))
    l, m = random_position(base.fov_rad, base.seed_sky + 100)
    src.append(Source(l, m, 1.0, kind="ramp", ramp_to=2.0))
    return replace(base, name="meerkat-faint-transients", sources=tuple(src))


def uneven_stream(base: Workload, n_snap: int, seed: int = 5,
                  channel_choices=(1024, 2048, 4096), flag_max: float = 0.6,
                  image_sizes=(1024, 2048)) -> List[Workload]:
    """Per-snapshot workloads of an uneven stream (the batched case): each
    snapshot s keeps the array, sky and noise of `base` but takes a channel
    count from `channel_choices` (a contiguous sub-band of base's channel
    grid at a random offset), a flag fraction uniform in [0, flag_max] and an
    image size from `image_sizes`, all drawn from a seeded generator."""
    g = torch.Generator().manual_seed(seed)
    step = (base.f_hi_hz - base.f_lo_hz) / base.n_chan
    out = []
    for _ in range(n_snap):
        nc = channel_choices[int(torch.randint(len(channel_choices), (1,), generator=g))]
        nc = min(nc, base.n_chan)
        off = int(torch.randint(base.n_chan - nc + 1, (1,), generator=g))
        ff = float(torch.rand(1, generator=g)) * flag_max
        N = image_sizes[int(torch.randint(len(image_sizes), (1,), generator=g))]
        f_lo = base.f_lo_hz + off * step
        out.append(replace(base, n_chan=nc, f_lo_hz=f_lo, f_hi_hz=f_lo + nc * step,
                           flag_frac=ff, image_size=N,
                           name=f"{base.name}-uneven-{nc}ch-{N}px"))
    return out


# --------------------------------------------------------------------------
# Snapshot synthesis
# --------------------------------------------------------------------------

def predict_vis(uvw: torch.Tensor, freq: torch.Tensor, sources, fluxes,
                chunk_bl: int = 256) -> torch.Tensor:
    """Point-source visibilities by the measurement equation (Section 1):
    V = sum_k S_k exp(-2 pi i (u l + v m + w (n - 1))), uvw in wavelengths."""
    dev = uvw.device
    nbl, nch = uvw.shape[0], freq.shape[0]
    out = torch.zeros(nbl, nch, dtype=torch.complex128, device=dev)
    scale = (freq / C_LIGHT).to(dev)
    for src, S in zip(sources, fluxes):
        if S == 0.0:
            continue
        n1 = math.sqrt(1.0 - src.l * src.l - src.m * src.m) - 1.0
        for b0 in range(0, nbl, chunk_bl):
            b1 = min(nbl, b0 + chunk_bl)
            d = (uvw[b0:b1, 0] * src.l + uvw[b0:b1, 1] * src.m + uvw[b0:b1, 2] * n1)
            ph = -2.0 * math.pi * d[:, None] * scale[None, :]
            out[b0:b1] += S * torch.polar(torch.ones_like(ph), ph)
    return out


def make_snapshot(w: Workload, s: int, device="cpu", with_weights: bool = False,
                  uvw_index: Optional[int] = None):
    """Snapshot s of workload w (uvw from hour angle of index uvw_index or s)."""
    dev = torch.device(device)
    enu = array_layout(w)
    si = s if uvw_index is None else uvw_index
    uvw = baseline_uvw(enu, math.radians(w.lat_deg), math.radians(w.dec_deg),
                       hour_angle(w, si)).to(dev)
    freq = frequencies(w).to(dev)
    fluxes = [src.flux_at(s, w.n_snap) for src in w.sources]
    sky = predict_vis(uvw, freq, w.sources, fluxes)
    nbl, nch, npol = w.n_bl, w.n_chan, w.n_pol
    gen = torch.Generator(device=dev).manual_seed(w.seed_noise + s)
    noise = torch.randn(nbl, nch, npol, 2, generator=gen, device=dev,
                        dtype=torch.float32) * w.noise_sigma
    vis = torch.view_as_complex(noise.contiguous())
    if npol == 1:
        vis[:, :, 0] += sky.to(torch.complex64)
    else:
        vis[:, :, 0] += sky.to(torch.complex64)
        vis[:, :, npol - 1] += sky.to(torch.complex64)
    if w.flag_frac > 0:
        genf = torch.Generator(device=dev).manual_seed(w.seed_flags * 100003 + s)
        flag = (torch.rand(nbl, nch, npol, generator=genf, device=dev) < w.flag_frac).to(torch.uint8)
    else:
        flag = torch.zeros(nbl, nch, npol, dtype=torch.uint8, device=dev)
    weight = None
    if with_weights:
        genw = torch.Generator(device=dev).manual_seed(w.seed_noise * 7 + s)
        weight = 0.5 + torch.rand(nbl, nch, npol, generator=genw, device=dev,
                                  dtype=torch.float32)
    return dict(uvw=uvw.contiguous(), freq=freq.contiguous(), vis=vis.contiguous(),
                flag=flag.contiguous(), weight=weight)


def to_fp16_channel_scaled(vis: torch.Tensor):
    """FP16 storage with a per-channel FP32 scale: scale_c = max|re,im| / 60000,
    stored = round_to_half(vis / scale_c).  Returns (half [nbl,nch,npol,2], scale [nch])."""
    ri = torch.view_as_real(vis)
    amax = ri.abs().amax(dim=(0, 2, 3)).to(torch.float32)
    scale = torch.where(amax > 0, amax / 60000.0, torch.ones_like(amax))
    q = (ri / scale[None, :, None, None]).to(torch.float16)
    return q.contiguous(), scale.contiguous()
