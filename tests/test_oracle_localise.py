"""Pins of the oracle's windowed point-source localisation against things
other than itself: central finite differences of the loss (steps 1e-3 pixel
in l and m, 1e-3 relative in S and in a weight), a zero loss and gradient at
the true source, the coplanar closed form (peak S / omega at the pixel that
source_of_pixel inverts), the transpose identity of the window image and its
adjoint, and the gridded full image (ES + FFT) on the window."""
from dataclasses import replace

import numpy as np

from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

SIZE = 16          # smaller windows keep the brute-force sums quick


def _workload(n_ant=8, n_chan=20, N=64, n_pol=4, flag_frac=0.15):
    w = synth.tiny_workload()
    return replace(w, n_ant=n_ant, n_chan=n_chan, image_size=N, n_pol=n_pol,
                   flag_frac=flag_frac, cell_arcsec=2.0 * 128 / N)


def _snapshot(w, s=1, weights=True):
    sn = synth.make_snapshot(w, s, with_weights=weights)
    return {k: (v.numpy() if v is not None else None) for k, v in sn.items()}


def _coplanar(h):
    """uvw projected onto their best-fit plane (r3 = 0 to rounding)."""
    uvw = h["uvw"]
    _, _, vt = np.linalg.svd(uvw - uvw.mean(0), full_matrices=False)
    n = vt[2]
    out = dict(h)
    out["uvw"] = uvw - np.outer(uvw @ n, n)
    return out


def _setup():
    w = _workload()
    h = _snapshot(w)
    cell = w.cell_arcsec * O.ARCSEC
    windows = np.array([[20, 26], [8, 40]])
    # a source near each window's centre, off the pixel grid
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"])
    src = []
    for (j2c, j1c), (d2, d1, S) in zip(windows, [(0.37, -0.21, 1.3), (-0.44, 0.18, 0.8)]):
        t1 = -cell * (j1c + SIZE // 2 + d1 - w.image_size // 2)
        t2 = cell * (j2c + SIZE // 2 + d2 - w.image_size // 2)
        l, m = O.source_of_pixel(t1, t2, p["V"])
        src.append((l, m, S))
    return w, h, windows, np.array(src), cell


def _loss(h, w, windows, src, weight=None):
    r = O.localise(h["uvw"], h["freq"], h["vis"], h["flag"],
                   h["weight"] if weight is None else weight, w.image_size, w.cell_arcsec,
                   windows, src, SIZE)
    return float(r["loss"].sum())


def test_source_gradient_matches_finite_differences():
    w, h, windows, src, cell = _setup()
    r = O.localise(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], w.image_size,
                   w.cell_arcsec, windows, src, SIZE)
    for i in range(len(windows)):
        for k, step in ((0, 1e-3 * cell), (1, 1e-3 * cell), (2, 1e-3 * src[i, 2])):
            sp, sm = src.copy(), src.copy()
            sp[i, k] += step
            sm[i, k] -= step
            fd = (_loss(h, w, windows, sp) - _loss(h, w, windows, sm)) / (2 * step)
            assert abs(fd - r["grad_src"][i, k]) <= 1e-6 * abs(r["grad_src"][i, k]), (i, k)


def test_weight_gradient_matches_finite_differences():
    """Both the data and the model depend on the weights (values and the
    1 / sum w normalisation); flagged and cross-hand records get 0."""
    w, h, windows, src, _ = _setup()
    r = O.localise(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], w.image_size,
                   w.cell_arcsec, windows, src, SIZE)
    f = h["flag"].astype(bool)
    rng = np.random.default_rng(3)
    scale = np.abs(r["grad_weight"]).max()
    picks = []
    for p in (0, 3):
        ok = np.argwhere(~f[:, :, p])
        for i in rng.choice(len(ok), 3, replace=False):
            picks.append((int(ok[i][0]), int(ok[i][1]), p))
    for (b, c, p) in picks:
        wt = h["weight"].astype(np.float64)
        step = 1e-3 * wt[b, c, p]
        wp = wt.copy(); wp[b, c, p] += step
        wm = wt.copy(); wm[b, c, p] -= step
        fd = (_loss(h, w, windows, src, wp) - _loss(h, w, windows, src, wm)) / (2 * step)
        assert abs(fd - r["grad_weight"][b, c, p]) <= 1e-7 * scale, (b, c, p)
    flagged = np.argwhere(f[:, :, 0])[0]
    assert r["grad_weight"][flagged[0], flagged[1], 0] == 0.0
    assert np.all(r["grad_weight"][:, :, 1] == 0.0) and np.all(r["grad_weight"][:, :, 2] == 0.0)


def test_true_source_gives_zero_loss_and_gradient():
    """Data that are exactly the model's visibilities fit with zero residual,
    so the loss and every gradient vanish."""
    w, h, windows, src, _ = _setup()
    vis = O.point_source_vis(h["uvw"], h["freq"], 4, *src[0])
    r = O.localise(h["uvw"], h["freq"], vis, h["flag"], h["weight"], w.image_size,
                   w.cell_arcsec, windows[:1], src[:1], SIZE)
    peak = np.abs(r["model"]).max()
    assert r["loss"][0] <= 1e-24 * peak * peak * SIZE * SIZE
    assert np.abs(r["grad_src"]).max() <= 1e-9 * peak
    assert np.abs(r["grad_weight"]).max() <= 1e-12 * peak


def test_coplanar_peak_is_flux_over_omega_at_the_named_pixel():
    """For coplanar samples the 2-D image of a point source is exactly
    S / (omega sum w) sum w_q = S / omega at tau = V (s - z); source_of_pixel
    inverts that map, so a source placed on a pixel centre images there to
    S / omega, the window's maximum."""
    w = _workload(flag_frac=0.0)
    h = _coplanar(_snapshot(w, weights=False))
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], None)
    cell = w.cell_arcsec * O.ARCSEC
    N = w.image_size
    j2, j1 = 30, 23
    l, m = O.source_of_pixel(-cell * (j1 - N // 2), cell * (j2 - N // 2), p["V"])
    S = 2.5
    vis = O.point_source_vis(h["uvw"], h["freq"], 4, l, m, S)
    pm = O.prepare(h["uvw"], h["freq"], vis, h["flag"], None)
    corner = (j2 - SIZE // 2, j1 - SIZE // 2)
    M = O.window_image_exact(pm, N, w.cell_arcsec, corner, SIZE)
    assert abs(M[SIZE // 2, SIZE // 2] - S / p["omega"]) <= 1e-9 * S
    assert np.unravel_index(np.argmax(M), M.shape) == (SIZE // 2, SIZE // 2)


def test_window_adjoint_is_the_transpose():
    w = _workload()
    h = _snapshot(w)
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"])
    rng = np.random.default_rng(8)
    c = rng.normal(size=p["c"].shape) + 1j * rng.normal(size=p["c"].shape)
    g = rng.normal(size=(SIZE, SIZE))
    q = dict(p, c=c)
    corner = (11, 37)
    lhs = float((g * O.window_image_exact(q, w.image_size, w.cell_arcsec, corner, SIZE)).sum())
    a = O.window_adjoint_exact(p, w.image_size, w.cell_arcsec, corner, g)
    rhs = float((np.conj(a) * c).real.sum())
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_window_equals_gridded_image_on_the_window():
    """The exact window equals the ES-gridded, FFT-imaged tilted image of the
    whole field on those pixels (a different route) within the ES error."""
    w, h, windows, src, _ = _setup()
    full = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                            w.image_size, w.cell_arcsec)["tilted"]
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"])
    for corner in windows:
        rows, cols = O.window_axes(corner, SIZE)
        win = O.window_image_exact(p, w.image_size, w.cell_arcsec, corner, SIZE)
        assert np.abs(win - full[np.ix_(rows, cols)]).max() <= 5e-7 * np.abs(full).max()
