"""Pins of the oracle's reverse mode (adjoint of S2..S6 and the point-source
chain rule) against things other than itself: the transpose identity
<A x, y> = <x, A^T y> with the separately written forward routines, central
finite differences of the forward image, and the brute-force DFT adjoint of
the exact Section 3.2 image."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth


def _workload(n_ant=8, n_chan=24, N=64, n_pol=4, flag_frac=0.2):
    w = synth.tiny_workload()
    return replace(w, n_ant=n_ant, n_chan=n_chan, image_size=N, n_pol=n_pol,
                   flag_frac=flag_frac, cell_arcsec=2.0 * 128 / N)


def _snapshot(w, s=1, weights=True):
    sn = synth.make_snapshot(w, s, with_weights=weights)
    return {k: (v.numpy() if v is not None else None) for k, v in sn.items()}


def _loss(h, w, grad_image, vis=None, weight=None):
    r = O.image_snapshot(h["uvw"], h["freq"], h["vis"] if vis is None else vis, h["flag"],
                         h["weight"] if weight is None else weight, w.image_size,
                         w.cell_arcsec)
    return float((grad_image * r["image"]).sum())


def test_bilinear_adjoint_is_the_transpose():
    rng = np.random.default_rng(5)
    N = 12
    x = rng.normal(size=(N, N))
    j1 = rng.uniform(-1.5, N + 0.5, size=(N, N))
    j2 = rng.uniform(-1.5, N + 0.5, size=(N, N))
    j1[0, :4] = [0.0, N - 1.0, N - 1.0 - 1e-12, -1e-12]     # the edges of the rule
    j2[1, :4] = [0.0, N - 1.0, 5.5, N - 1.0]
    y = rng.normal(size=(N, N))
    lhs = (O.bilinear(x, j1, j2) * y).sum()
    rhs = (x * O.bilinear_adjoint(y, j1, j2)).sum()
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("n_pol,weights", [(1, False), (4, True)])
def test_image_adjoint_identity(n_pol, weights):
    """L = <grad_image, image(c)> is linear in the sample values, so it must
    equal sum_q Re(conj(g_q) c_q) = sum Re(conj(grad_vis) vis) exactly (up to
    rounding): pins the bilinear transpose, the correction, the direction and
    centring of the FFT and degridding against the forward routines."""
    w = _workload(n_pol=n_pol, flag_frac=0.2 if weights else 0.0)
    h = _snapshot(w, weights=weights)
    rng = np.random.default_rng(7)
    gimg = rng.normal(size=(w.image_size, w.image_size))
    a = O.image_snapshot_adjoint(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                                 w.image_size, w.cell_arcsec, gimg)
    L = float((gimg * a["image"]).sum())
    w_q, c_q = O.sample_weights_and_values(h["vis"], h["flag"], h["weight"])
    via_g = float((np.conj(a["g"]) * c_q).real.sum())
    via_vis = float((np.conj(a["grad_vis"]) * h["vis"]).real.sum())
    assert abs(via_g - L) <= 1e-11 * abs(L)
    assert abs(via_vis - L) <= 1e-11 * abs(L)
    assert np.all(a["g"][w_q == 0] == 0)


def test_weight_gradient_matches_finite_differences():
    """grad_weight (including the 1 / sum w normalisation term) against
    central differences of the forward image, step 1e-3 of the weight; a
    flagged polarisation and a cross hand have zero gradient."""
    w = _workload(n_pol=4, flag_frac=0.2)
    h = _snapshot(w, weights=True)
    rng = np.random.default_rng(9)
    gimg = rng.normal(size=(w.image_size, w.image_size))
    a = O.image_snapshot_adjoint(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                                 w.image_size, w.cell_arcsec, gimg)
    f = h["flag"].astype(bool)
    picks = []
    for p in (0, 3):
        ok = np.argwhere(~f[:, :, p])
        for i in rng.choice(len(ok), 3, replace=False):
            picks.append((int(ok[i][0]), int(ok[i][1]), p))
    flagged = np.argwhere(f[:, :, 0])[0]
    picks.append((int(flagged[0]), int(flagged[1]), 0))
    picks.append((2, 5, 1))                                  # a cross hand
    scale = np.abs(a["grad_weight"]).max()
    for (b, c, p) in picks:
        wt = h["weight"].astype(np.float64)
        step = 1e-3 * wt[b, c, p]
        wp = wt.copy(); wp[b, c, p] += step
        wm = wt.copy(); wm[b, c, p] -= step
        fd = (_loss(h, w, gimg, weight=wp) - _loss(h, w, gimg, weight=wm)) / (2 * step)
        assert abs(fd - a["grad_weight"][b, c, p]) <= 1e-7 * scale, (b, c, p)


def test_tilted_adjoint_matches_dft_adjoint():
    """Degridding of the grid cotangent equals the exact adjoint of the
    Section 3.2 dirty image, g_q = 1/(omega sum w) sum_j U_j exp(-i phase_qj),
    within the ES kernel's error."""
    w = _workload(n_ant=10, n_chan=16, N=64, n_pol=1, flag_frac=0.0)
    h = _snapshot(w, weights=False)
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], None)
    N, W = w.image_size, 8
    G, beta = 2 * N, O.es_beta(W)
    rng = np.random.default_rng(4)
    U = rng.normal(size=(N, N))
    g1, g2 = O.grid_coords(p["r"][:, 0], p["r"][:, 1], N, w.cell_arcsec)
    H = O.tilted_image_adjoint(U, G, W, beta, p["omega"], p["sumw"])
    g = O.degrid_es(H, g1, g2, W, beta)
    cell = w.cell_arcsec * O.ARCSEC
    j = np.arange(N) - N // 2
    t1 = -cell * j
    t2 = cell * j
    e1 = np.exp(-2j * np.pi * np.outer(p["r"][:, 0], t1))     # [q, j1]
    e2 = np.exp(-2j * np.pi * np.outer(p["r"][:, 1], t2))     # [q, j2]
    exact = np.einsum("qb,ba,qa->q", e2, U, e1) / (p["omega"] * p["sumw"])
    assert np.abs(g - exact).max() <= 1e-6 * np.abs(U).sum() / (p["omega"] * p["sumw"])


def test_point_source_gradient_matches_finite_differences():
    """dL/d(l, m, S) of L = <grad_image, image(point source)> through the
    adjoint and the chain rule, against central differences of the forward
    image (steps 1e-3 pixel in l and m, 1e-3 relative in S)."""
    w = _workload(n_pol=4, flag_frac=0.1)
    h = _snapshot(w, weights=True)
    N = w.image_size
    cell = w.cell_arcsec * O.ARCSEC
    l0, m0, S0 = 7.3 * cell, -4.1 * cell, 1.7
    rng = np.random.default_rng(12)
    gimg = rng.normal(size=(N, N))

    def L(l, m, S):
        return _loss(h, w, gimg, vis=O.point_source_vis(h["uvw"], h["freq"], 4, l, m, S))

    vis = O.point_source_vis(h["uvw"], h["freq"], 4, l0, m0, S0)
    a = O.image_snapshot_adjoint(h["uvw"], h["freq"], vis, h["flag"], h["weight"], N,
                                 w.cell_arcsec, gimg)
    gr = O.point_source_gradient(h["uvw"], h["freq"], a["grad_vis"], l0, m0, S0)
    dl = 1e-3 * cell
    fd_l = (L(l0 + dl, m0, S0) - L(l0 - dl, m0, S0)) / (2 * dl)
    fd_m = (L(l0, m0 + dl, S0) - L(l0, m0 - dl, S0)) / (2 * dl)
    dS = 1e-3 * S0
    fd_S = (L(l0, m0, S0 + dS) - L(l0, m0, S0 - dS)) / (2 * dS)
    assert abs(fd_l - gr["l"]) <= 1e-6 * abs(gr["l"])
    assert abs(fd_m - gr["m"]) <= 1e-6 * abs(gr["m"])
    assert abs(fd_S - gr["flux"]) <= 1e-8 * abs(gr["flux"])
