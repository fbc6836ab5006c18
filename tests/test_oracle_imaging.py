"""Pins of the FP64 oracle's imaging steps (S1-S6) against things other than
itself: planted geometry, the brute-force dirty image of Section 3.2, point
source closed forms, the gridding/degridding adjoint identity, an
independent quadrature, and the two re-projection derivations (Section 3.3
and Appendix A)."""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth


def _tiny(s=3, **kw):
    w = synth.tiny_workload()
    snap = synth.make_snapshot(w, s, **kw)
    return w, {k: (v.numpy() if v is not None else None) for k, v in snap.items()}


# ---------------------------------------------------------------- S1 -------

def test_svd_planted_plane_normal():
    """Samples on the plane w = a u + b v: the third basis row is the plane
    normal (-a, -b, 1)/|.|, V is orthogonal with det +1, and xi = -a, eta = -b."""
    rng = np.random.default_rng(5)
    a, b = 0.21, -0.07
    u = rng.uniform(-5e3, 5e3, 3000)
    v = rng.uniform(-5e3, 5e3, 3000)
    B = np.stack([u, v, a * u + b * v + 17.0], 1)     # offset plane: centring removes it
    V = O.svd_basis(B)
    n = np.array([-a, -b, 1.0]) / math.sqrt(1 + a * a + b * b)
    assert np.allclose(V[2], n, atol=1e-12)
    assert np.allclose(V @ V.T, np.eye(3), atol=1e-13)
    assert abs(np.linalg.det(V) - 1.0) < 1e-13
    xi, eta = O.tilt_of(V)
    assert abs(xi + a) < 1e-12 and abs(eta + b) < 1e-12
    # omega equals V33 for a right-handed orthogonal V (cofactor identity)
    assert abs(O.omega_of(V) - V[2, 2]) < 1e-13
    # v1 keeps the u axis: its v component is zero (projection of e_u)
    assert abs(V[0, 1] - (-(n[0] * n[1]) / math.sqrt(1 - n[0] ** 2))) < 1e-12


def test_omega_is_the_cofactor_for_any_rotation():
    """Eq. 11 for a general basis: every entry of a rotation matrix equals its
    cofactor, so omega = |V11 V22 - V21 V12| = |V33| for any V with det +1.
    Random rotations have V21 != 0, which svd_basis's own convention (v1 in
    the u-w plane) never produces."""
    rng = np.random.default_rng(14)
    for _ in range(20):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        V = q if np.linalg.det(q) > 0 else -q
        assert abs(V[1, 0]) > 1e-3 or abs(V[0, 1]) > 1e-3
        assert O.omega_of(V) == pytest.approx(abs(V[2, 2]), abs=1e-14)


def test_svd_coplanar_identity():
    """Exactly coplanar baselines (all w = 0): V = I, omega = 1, xi = eta = 0."""
    rng = np.random.default_rng(6)
    B = np.stack([rng.normal(size=500), rng.normal(size=500), np.zeros(500)], 1)
    V = O.svd_basis(B)
    assert np.allclose(V, np.eye(3), atol=1e-14)
    assert O.omega_of(V) == pytest.approx(1.0, abs=1e-15)


def test_svd_degenerate_cloud_is_identity():
    """One sample, or samples on one line through the mean, fix no plane:
    the basis falls back to V = I (standard 2-D imaging)."""
    assert np.array_equal(O.svd_basis(np.array([[572.8, 636.5, 71.9]])), np.eye(3))
    t = np.linspace(1.0, 2.0, 50)[:, None]
    assert np.array_equal(O.svd_basis(t * np.array([[300.0, -20.0, 5.0]])), np.eye(3))


def test_svd_matches_covariance_eigenvectors():
    """The smallest-variance direction of the centred cloud (eigenvector of
    the 3x3 covariance) equals the third basis row."""
    w, s = _tiny()
    p = O.prepare(s["uvw"], s["freq"], s["vis"], s["flag"])
    B = O.wavelength_baselines(s["uvw"], s["freq"])[p["sel"]]
    C = np.cov(B.T)
    ev, evec = np.linalg.eigh(C)
    n = evec[:, 0] * np.sign(evec[2, 0])
    assert np.allclose(p["V"][2], n, atol=1e-9)


def test_flagged_samples_do_not_move_the_plane():
    """Section 3.5 (reading c4): only selected samples (w_q > 0) enter the
    plane fit, so a fully flagged baseline far off the plane leaves V the
    plane's own basis."""
    rng = np.random.default_rng(13)
    a, b = -0.12, 0.05
    u = rng.uniform(-3e3, 3e3, 40)
    v = rng.uniform(-3e3, 3e3, 40)
    uvw = np.stack([u, v, a * u + b * v], 1)          # a plane through the origin
    uvw[7] = [500.0, -800.0, 2500.0]                  # off the plane, fully flagged
    freq = np.linspace(1.0e9, 1.1e9, 6)
    vis = np.ones((40, 6, 1), np.complex64)
    flag = np.zeros((40, 6, 1), np.uint8)
    flag[7] = 1
    p = O.prepare(uvw, freq, vis, flag)
    n = np.array([-a, -b, 1.0]) / math.sqrt(1 + a * a + b * b)
    assert np.allclose(p["V"][2], n, atol=1e-12)
    assert p["n_vis"] == 39 * 6


def test_sample_weights_pol_average_by_hand():
    """Section 3.5 by hand: flags zero the weight; parallel hands averaged
    with their weights; c_q = w_q Vis_q."""
    vis = np.array([[[1 + 1j, 9, 9, 3 - 1j], [2, 9, 9, 4j]]], dtype=np.complex64)
    flag = np.array([[[0, 1, 1, 0], [0, 0, 0, 1]]], dtype=np.uint8)
    wt = np.array([[[2.0, 5, 5, 1.0], [0.5, 1, 1, 3.0]]], dtype=np.float32)
    w_q, c_q = O.sample_weights_and_values(vis, flag, wt)
    assert w_q[0, 0] == 3.0 and c_q[0, 0] == 2 * (1 + 1j) + 1 * (3 - 1j)
    assert w_q[0, 1] == 0.5 and c_q[0, 1] == 0.5 * 2


# ------------------------------------------------------------ S2..S5 -------

def test_gridded_image_matches_bruteforce_dft():
    """Gridding + FFT + correction reproduce the exact I_D^(2) of Section 3.2
    within the ES kernel's error (W = 8, sigma = 2: < 5e-7 of the peak)."""
    w, s = _tiny()
    r = O.image_snapshot(s["uvw"], s["freq"], s["vis"], s["flag"], None,
                         w.image_size, w.cell_arcsec)
    d = O.dirty_image_dft(r["r"][:, 0], r["r"][:, 1], r["c"], w.image_size,
                          w.cell_arcsec, r["omega"], r["sumw"])
    assert np.abs(d - r["tilted"]).max() <= 5e-7 * np.abs(d).max()


def test_point_source_at_phase_centre():
    """Noise-free unit-weight point source of flux S at the phase centre:
    the tilted image at t = 0 equals S / omega."""
    w = synth.tiny_workload()
    S = 2.5
    uvw = synth.baseline_uvw(synth.array_layout(w), math.radians(-30.71),
                             math.radians(-30.0), 0.3).numpy()
    freq = synth.frequencies(w).numpy()
    vis = np.full((uvw.shape[0], len(freq), 1), S, dtype=np.complex64)
    flag = np.zeros(vis.shape, np.uint8)
    r = O.image_snapshot(uvw, freq, vis, flag, None, w.image_size, w.cell_arcsec)
    N = w.image_size
    assert r["tilted"][N // 2, N // 2] == pytest.approx(S / r["omega"], rel=5e-7)
    assert r["omega"] < 1.0


def test_point_source_off_centre_closed_form():
    """A point source at s0 = (l0, m0, n0-1): b.s0 = r.t0 with t0 = V s0
    (Eq. 9-10), so the 2-D image is the PSF shifted to (t01, t02) with the
    residual phase r3 t03:  I(t) = S/(omega sum w) sum_q w_q
    cos 2 pi (r1 (t1 - t01) + r2 (t2 - t02) - r3 t03)."""
    w = synth.tiny_workload()
    N, cell = w.image_size, w.cell_arcsec
    beta = cell * O.ARCSEC
    l0, m0 = 17.3 * beta, -9.6 * beta
    src = synth.Source(l0, m0, 1.7)
    uvw = synth.baseline_uvw(synth.array_layout(w), math.radians(-30.71),
                             math.radians(-30.0), -0.4)
    freq = synth.frequencies(w)
    vis = synth.predict_vis(uvw, freq, [src], [1.7]).to(torch_c64())[:, :, None].numpy()
    flag = np.zeros(vis.shape, np.uint8)
    r = O.image_snapshot(uvw.numpy(), freq.numpy(), vis, flag, None, N, cell)
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    t0 = r["V"] @ np.array([l0, m0, n0 - 1])
    j = np.arange(N) - N // 2
    t1 = -beta * j
    t2 = beta * j
    R = r["r"]
    ph0 = R[:, 2] * t0[2]
    e1 = np.exp(2j * np.pi * np.outer(t1 - t0[0], R[:, 0]))
    e2 = np.exp(2j * np.pi * np.outer(t2 - t0[1], R[:, 1]))
    closed = ((e2 * np.exp(-2j * np.pi * ph0)[None, :]) @ e1.T).real * 1.7 / (r["omega"] * r["sumw"])
    assert np.abs(closed - r["tilted"]).max() <= 1e-6 * np.abs(closed).max()
    # the peak sits at the pixel nearest to t0 = (-beta (j1 - N/2), beta (j2 - N/2))
    pk = np.unravel_index(np.argmax(r["tilted"]), r["tilted"].shape)
    assert pk == (int(round(t0[1] / beta)) + N // 2, int(round(-t0[0] / beta)) + N // 2)


def torch_c64():
    import torch
    return torch.complex64


def test_gridding_degridding_adjoint():
    """<Grid(c), Y> = <c, Degrid(Y)> to 1e-12 (FP64): the degridder uses the
    very same taps as the gridder."""
    rng = np.random.default_rng(7)
    G, W = 64, 8
    beta = O.es_beta(W)
    g1 = rng.uniform(6, G - 6, 300)
    g2 = rng.uniform(6, G - 6, 300)
    c = rng.normal(size=300) + 1j * rng.normal(size=300)
    Y = rng.normal(size=(G, G)) + 1j * rng.normal(size=(G, G))
    lhs = np.vdot(Y, O.grid_es(g1, g2, c, G, W, beta))
    rhs = np.vdot(O.degrid_es(Y, g1, g2, W, beta), c)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_es_fourier_quadrature_vs_adaptive():
    """psi_hat by Gauss-Legendre equals an adaptive quadrature (scipy.quad)."""
    W = 8
    beta = O.es_beta(W)
    for f in (0.0, 0.1, 0.23, 0.25):
        ref, _ = scipy.integrate.quad(lambda x: float(O.es_kernel(x, W, beta)) *
                                      math.cos(2 * math.pi * x * f), -W / 2, W / 2,
                                      epsabs=0.0, epsrel=1e-13, limit=400)
        assert O.es_fourier([f], W, beta)[0] == pytest.approx(ref, rel=1e-12)


def test_es_kernel_values():
    """psi(0) = 1, psi(+-W/2) = exp(-beta), psi is even."""
    W = 8
    beta = O.es_beta(W)
    assert O.es_kernel(0.0, W, beta) == 1.0
    assert O.es_kernel(4.0, W, beta) == pytest.approx(math.exp(-beta), rel=1e-14)
    x = np.linspace(-4, 4, 81)
    assert np.array_equal(O.es_kernel(x, W, beta), O.es_kernel(-x, W, beta))


def test_hermitian_half_gives_real_image():
    """The inverse DFT of the Hermitian part equals Re of the full one."""
    rng = np.random.default_rng(8)
    G, N = 32, 16
    grid = np.zeros((G, G), complex)
    grid[4:28, 4:28] = rng.normal(size=(24, 24)) + 1j * rng.normal(size=(24, 24))
    H = O.hermitian_half(grid)
    full = np.zeros((G, G), complex)
    full[G // 2:, :] = H[:G // 2]
    idx = (G - np.arange(G)) % G
    for k2 in range(0, G // 2):
        full[k2, :] = np.conj(full[idx[k2], idx])
    full[0, :] = 0.5 * (grid[0, :] + np.conj(grid[0, idx]))
    a = O.ifft_centred(full, N)
    b = O.ifft_centred(grid, N)
    assert np.abs(a.imag).max() < 1e-12 * np.abs(b).max()
    assert np.abs(a.real - b.real).max() < 1e-12 * np.abs(b).max()


# ---------------------------------------------------------------- S6 -------

def test_reprojection_reduced_equals_wcs():
    """Section 3.3's reduced map and Appendix A's WCS route agree to 1e-10 px
    over a whole 2048 x 2048 image at a MeerKAT-like tilt."""
    N, cell = 2048, 2.0 / 3600
    j = np.arange(0, N, 7, dtype=np.float64) + 1
    p1, p2 = np.meshgrid(j, j)
    for xi, eta in ((-0.11, -0.016), (0.3, -0.2), (0.0, 0.0)):
        a1, a2 = O.reproject_map_reduced(p1, p2, N, cell, xi, eta)
        b1, b2 = O.reproject_map_wcs(p1, p2, N, cell, xi, eta)
        assert np.abs(a1 - b1).max() < 1e-10 and np.abs(a2 - b2).max() < 1e-10


def test_reprojection_identity_without_tilt():
    """xi = eta = 0: the map is the identity and so is the re-projection."""
    rng = np.random.default_rng(9)
    img = rng.normal(size=(64, 64))
    out = O.reproject(img, 2.0, 0.0, 0.0)
    assert np.array_equal(out, img)


def test_reprojection_gather_inverts_map():
    """The gathered source pixel p satisfies map(p) = p' (1e-9 px)."""
    N, cell = 512, 20.0 / 3600
    xi, eta = 0.25, -0.12
    j1, j2 = O.reproject_source_pixels(N, cell, xi, eta, iters=8)
    m1, m2 = O.reproject_map_reduced(j1 + 1, j2 + 1, N, cell, xi, eta)
    jo = np.arange(N, dtype=np.float64) + 1
    assert np.abs(m1 - jo[None, :]).max() < 1e-9
    assert np.abs(m2 - jo[:, None]).max() < 1e-9


def test_reproject_moves_a_point_where_the_wcs_route_maps_it():
    """reproject() as a whole, cell given in arcsec: a single bright tilted
    pixel lands, as the centroid of the gathered output, where Appendix A's
    WCS route maps that pixel (within 0.02 px; the shifts are up to ~1 px at
    this field and tilt)."""
    N, cell = 256, 60.0
    xi, eta = 0.3, -0.2
    yy, xx = np.mgrid[0:N, 0:N]
    largest = 0.0
    for j2, j1 in ((230, 20), (30, 200), (200, 140)):
        img = np.zeros((N, N))
        img[j2, j1] = 1.0
        out = O.reproject(img, cell, xi, eta)
        c2, c1 = (out * yy).sum() / out.sum(), (out * xx).sum() / out.sum()
        m1, m2 = O.reproject_map_wcs(j1 + 1.0, j2 + 1.0, N, cell / 3600.0, xi, eta)
        assert abs(c1 - (float(m1) - 1)) < 0.02 and abs(c2 - (float(m2) - 1)) < 0.02
        largest = max(largest, np.hypot(float(m1) - 1 - j1, float(m2) - 1 - j2))
    assert largest > 0.5


def test_bilinear_exact_on_planes():
    """Bilinear interpolation reproduces a linear function exactly inside."""
    N = 16
    yy, xx = np.mgrid[0:N, 0:N].astype(float)
    img = 3.0 * xx - 2.0 * yy + 0.5
    j1 = np.array([0.0, 3.25, 14.5, 15.0])
    j2 = np.array([0.0, 7.75, 2.5, 15.0])
    v = O.bilinear(img, j1, j2)
    assert np.allclose(v, 3.0 * j1 - 2.0 * j2 + 0.5, atol=1e-13)
    assert O.bilinear(img, np.array([-0.1]), np.array([3.0]))[0] == 0.0
