"""FP64 CPU oracle of the FIP-TOI hot path (TOI 2-D imaging + FITrig tLISI).

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or executes this module; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference legs of
``bench.py`` use it.  It shares no code with the CUDA path.

It is a plain, slow, step-by-step restatement of the method in float64:

  S1  Section 3 / 3.1 / 3.5  wavelength scaling, sample selection and weights,
                             SVD basis V of the centred baseline cloud, R = B V^T
  S2  Section 3.2            (r1, r2) -> continuous grid coordinates
  S3  Section 4.1 stage 3    convolutional gridding ("place visibilities on a
                             grid"; kernel = exponential of semicircle, reading c1)
  S4  Section 4.1 stage 4    inverse 2-D FFT (numpy.fft as the library step)
  S5  Section 3.2 Eq. 11     grid correction, crop, Re, 1/(omega sum w)
  S6  Section 3.3 / App. A   reduced SIN re-projection (and the WCS route)
  S7  Section 2 / 4.5        tLISI per tile from the three youngest images
                             (stand-in formula, reading c9: parity unpinned
                             against the paper, which does not print it)
  S8  Section 2, 6.2, 6.3    periodic / non-periodic scores, z-threshold,
                             connected tiles -> bounding boxes, in a fixed FP64
                             evaluation order so that another implementation
                             of the same order reproduces it bit for bit.
  3-D mode  Section 3.4, App. B, Table 2: t3 on the sphere, slabs,
                             Chebyshev moments (Jacobi-Anger), the order rule
  localisation              windowed point-source model, loss and its exact
                             gradients (candidate windows of Section 6)
  adjoint                   reverse mode of S2..S6 (Section 1 names the
                             adjoint route to gradients): bilinear transpose,
                             correction, forward DFT, ES degridding (the
                             exact adjoint of gridding); sample, visibility
                             and weight gradients with the plane fit fixed;
                             point-source chain rule

Exact-definition routines used as pins: ``dirty_image_dft`` (the 2-D dirty
image of Section 3.2 evaluated by brute force).

Parity status per function (pins live in tests/):
  wavelength/sample selection, svd_basis, grid_es, image pipeline: pinned
    (planted planes, brute-force DFT, point-source closed forms, adjoint).
  reproject_*: pinned (two derivations agree; identity at xi = eta = 0).
  tlisi: parity unpinned against the paper (its formula is not printed);
    pinned only by invariants of the stand-in definition.
  candidates_*: pinned by planted cubes and an independent FFT cross-check.
  t3_of, slab_plan, chebyshev_*, tilted_image_3d: pinned by Table 2's
    (Phi_max, N_slab, alpha_slab, K) rows, the sphere constraint of App. B.1,
    the Jacobi-Anger series, the brute-force I_D^(3) and the coplanar limit.
  *_adjoint, point_source_gradient: pinned by the adjoint identity
    <A x, y> = <x, A^T y> against the forward routines, central finite
    differences of the forward, and the brute-force DFT adjoint.
  window_*, source_of_pixel, localise: pinned by central finite differences
    of the loss (l, m, S and weights), a zero loss and gradient at the true
    source, the coplanar peak S / omega at the pixel source_of_pixel names,
    the window transpose identity and the gridded full image on the window.
  Pin strength: tests/test_oracle_mutations.py plants one plausible mistake
    at a time in these routines (a dropped term, a sign, an index, a
    transposed operand, a constant) and requires a named pin to fail on each.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Tuple

import numpy as np

C_LIGHT = 299_792_458.0
ARCSEC = math.pi / 648000.0


# ==========================================================================
# S1 — data handling (Section 3.5) and the SVD basis (Section 3.1)
# ==========================================================================

def parallel_hands(n_pol: int) -> Tuple[int, int]:
    """Indices of the parallel-hand polarisations (reading c13): linear feeds
    XX,XY,YX,YY -> (0, 3); two pols -> (0, 1); Stokes I only -> (0, 0)."""
    if n_pol == 4:
        return 0, 3
    if n_pol == 2:
        return 0, 1
    if n_pol == 1:
        return 0, 0
    raise ValueError("n_pol must be 1, 2 or 4")


def sample_weights_and_values(vis, flag, weight):
    """Section 3.5: flagged samples get zero weight; WEIGHT_SPECTRUM (or unit
    weights) is applied before gridding; the parallel hands are averaged with
    their weights.  Returns per (baseline, channel):
        w_q = w_a + w_b                  (the sample weight)
        c_q = w_a V_a + w_b V_b = w_q Vis_q   (the weighted visibility)
    For a single polarisation, w_q = w_0 and c_q = w_0 V_0."""
    vis = np.asarray(vis)
    n_pol = vis.shape[2]
    pa, pb = parallel_hands(n_pol)
    f = np.asarray(flag).astype(bool)
    if weight is None:
        wp = np.where(f, 0.0, 1.0)
    else:
        wp = np.where(f, 0.0, np.asarray(weight, dtype=np.float64))
    v = vis.astype(np.complex128)
    if pa == pb:
        w_q = wp[:, :, pa]
        c_q = wp[:, :, pa] * v[:, :, pa]
    else:
        w_q = wp[:, :, pa] + wp[:, :, pb]
        c_q = wp[:, :, pa] * v[:, :, pa] + wp[:, :, pb] * v[:, :, pb]
    return w_q, c_q


def wavelength_baselines(uvw_m, freq_hz):
    """Section 3: each UVW (metres) is converted to wavelengths for its channel,
    b_q = uvw * nu / c.  Shape [n_bl, n_ch, 3]."""
    uvw = np.asarray(uvw_m, dtype=np.float64)
    k = np.asarray(freq_hz, dtype=np.float64) / C_LIGHT
    return uvw[:, None, :] * k[None, :, None]


def svd_basis(B_sel: np.ndarray) -> np.ndarray:
    """Section 3.1: SVD of the centred baseline matrix B~ = B - mean(B).
    Rows of V are the basis vectors.  Sign / in-plane conventions (reading c5,
    the paper leaves them open): v3 = right singular vector of the smallest
    singular value with V33 > 0; v1 = e_u projected onto the plane and
    normalised (e_v if e_u is within 0.999 of the normal); v2 = v3 x v1, so
    (v1, v2, v3) is right-handed.  A sample cloud of rank <= 1 (second
    singular value <= 1e-6 of the first) fixes no plane: V = I."""
    Bt = B_sel - B_sel.mean(axis=0, keepdims=True)
    if Bt.shape[0] < 3:
        Bt = np.vstack([Bt, np.zeros((3 - Bt.shape[0], 3))])
    _, sv, Vt = np.linalg.svd(Bt, full_matrices=False)
    if not sv[1] > 1e-6 * sv[0]:
        return np.eye(3)
    v3 = Vt[2].copy()
    if v3[2] < 0:
        v3 = -v3
    e = np.array([1.0, 0.0, 0.0])
    if abs(e @ v3) > 0.999:
        e = np.array([0.0, 1.0, 0.0])
    v1 = e - (e @ v3) * v3
    v1 /= np.linalg.norm(v1)
    v2 = np.cross(v3, v1)
    return np.stack([v1, v2, v3])


def omega_of(V: np.ndarray) -> float:
    """Eq. 11: area Jacobian omega = |V11 V22 - V21 V12|."""
    return abs(V[0, 0] * V[1, 1] - V[1, 0] * V[0, 1])


def tilt_of(V: np.ndarray) -> Tuple[float, float]:
    """Section 3.3: xi = V31 / V33, eta = V32 / V33."""
    return V[2, 0] / V[2, 2], V[2, 1] / V[2, 2]


def prepare(uvw_m, freq_hz, vis, flag, weight=None) -> Dict:
    """S1 for one snapshot: selected samples (w_q > 0, reading c4), the basis
    V, R = B V^T (Section 3.1), omega, xi, eta and sum of weights."""
    w_q, c_q = sample_weights_and_values(vis, flag, weight)
    B = wavelength_baselines(uvw_m, freq_hz)
    sel = w_q > 0
    if not sel.any():
        raise ValueError("no unflagged sample with positive weight")
    Bs = B[sel]
    V = svd_basis(Bs)
    R = Bs @ V.T
    xi, eta = tilt_of(V)
    return dict(V=V, omega=omega_of(V), xi=xi, eta=eta, sumw=float(w_q[sel].sum()),
                r=R, c=c_q[sel], w=w_q[sel], sel=sel, n_vis=int(sel.sum()))


# ==========================================================================
# S2/S3 — gridding with the exponential-of-semicircle kernel (reading c1)
# ==========================================================================

def es_beta(W: int) -> float:
    """ES shape parameter for upsampling 2: beta = 2.30 W (Barnett, Magland &
    af Klinteberg 2019)."""
    return 2.30 * W


def es_kernel(x, W: int, beta: float):
    """psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) for |x| <= W/2, else 0."""
    z = 2.0 * np.asarray(x, dtype=np.float64) / W
    inside = np.abs(z) <= 1.0
    zz = np.where(inside, z, 0.0)
    return np.where(inside, np.exp(beta * (np.sqrt(1.0 - zz * zz) - 1.0)), 0.0)


def grid_coords(r1, r2, N: int, cell_arcsec: float, sigma: int = 2):
    """Section 3.2 with the pixel convention of Section 3.3 (reading c6):
    t1 = -beta (j1 - N/2), t2 = beta (j2 - N/2) (0-based j, beta in radians).
    The phase 2 pi (r1 t1 + r2 t2) is reproduced by a centred DFT over a
    G = sigma N grid when a sample sits at
        g1 = G/2 - r1 beta G,   g2 = G/2 + r2 beta G."""
    G = sigma * N
    beta = cell_arcsec * ARCSEC
    g1 = G / 2 - np.asarray(r1) * beta * G
    g2 = G / 2 + np.asarray(r2) * beta * G
    return g1, g2


def tap_start(g, W: int):
    """First tap index of a sample at continuous coordinate g: ceil(g - W/2)."""
    return np.ceil(g - W / 2.0).astype(np.int64)


def grid_es(g1, g2, c, G: int, W: int, beta: float) -> np.ndarray:
    """Convolutional gridding: Grid[k2, k1] = sum_q c_q psi(k1 - g1_q) psi(k2 - g2_q)
    over the W x W taps k = ceil(g - W/2) + 0..W-1 of every sample.  Full
    complex G x G grid, row index k2, column index k1."""
    g1 = np.asarray(g1, dtype=np.float64)
    g2 = np.asarray(g2, dtype=np.float64)
    c = np.asarray(c, dtype=np.complex128)
    k1 = tap_start(g1, W)
    k2 = tap_start(g2, W)
    if len(c) and (k1.min() < 0 or k2.min() < 0 or k1.max() + W > G or k2.max() + W > G):
        raise ValueError("a kernel footprint leaves the grid: reduce the cell size")
    re = np.zeros(G * G)
    im = np.zeros(G * G)
    wx = [es_kernel(k1 + a - g1, W, beta) for a in range(W)]
    wy = [es_kernel(k2 + b - g2, W, beta) for b in range(W)]
    for b in range(W):
        for a in range(W):
            idx = (k2 + b) * G + (k1 + a)
            val = c * (wx[a] * wy[b])
            re += np.bincount(idx, weights=val.real, minlength=G * G)
            im += np.bincount(idx, weights=val.imag, minlength=G * G)
    return (re + 1j * im).reshape(G, G)


def degrid_es(grid: np.ndarray, g1, g2, W: int, beta: float) -> np.ndarray:
    """Adjoint of grid_es: d_q = sum_k Grid[k2, k1] psi(k1 - g1_q) psi(k2 - g2_q)."""
    g1 = np.asarray(g1, dtype=np.float64)
    g2 = np.asarray(g2, dtype=np.float64)
    k1 = tap_start(g1, W)
    k2 = tap_start(g2, W)
    out = np.zeros(len(g1), dtype=np.complex128)
    for b in range(W):
        wy = es_kernel(k2 + b - g2, W, beta)
        for a in range(W):
            wx = es_kernel(k1 + a - g1, W, beta)
            out += grid[k2 + b, k1 + a] * (wx * wy)
    return out


# ==========================================================================
# S4/S5 — inverse FFT, grid correction, normalisation
# ==========================================================================

def ifft_centred(grid: np.ndarray, N: int) -> np.ndarray:
    """Section 4.1 stage 4: unnormalised inverse 2-D DFT with centred indices,
    I[j2', j1'] = sum_k' Grid[k'] exp(+2 pi i (k1' j1' + k2' j2') / G),
    k' = k - G/2, returning the central N x N block (j' = j - N/2)."""
    G = grid.shape[0]
    y = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(grid), norm="forward"))
    lo = G // 2 - N // 2
    return y[lo:lo + N, lo:lo + N]


def es_fourier(f, W: int, beta: float, nodes: int = 400) -> np.ndarray:
    """psi_hat(f) = integral_{-W/2}^{W/2} psi(x) cos(2 pi x f) dx by
    Gauss-Legendre quadrature (reading c1: correction by the kernel's
    numerically integrated Fourier transform)."""
    x, wts = np.polynomial.legendre.leggauss(nodes)
    x = x * (W / 2.0)
    wts = wts * (W / 2.0)
    psi = es_kernel(x, W, beta)
    f = np.asarray(f, dtype=np.float64)
    return (psi[None, :] * np.cos(2 * np.pi * np.outer(f, x)) * wts[None, :]).sum(1)


def correction_vector(N: int, G: int, W: int, beta: float) -> np.ndarray:
    j = np.arange(N) - N // 2
    return es_fourier(j / G, W, beta)


def tilted_image(grid: np.ndarray, N: int, W: int, beta: float, omega: float,
                 sumw: float) -> np.ndarray:
    """S4+S5: Re of the centred inverse FFT, divided by psi_hat(j1') psi_hat(j2')
    and by omega * sum w (Eq. 11 and reading c2, c3)."""
    G = grid.shape[0]
    img = ifft_centred(grid, N).real
    ph = correction_vector(N, G, W, beta)
    return img / (ph[:, None] * ph[None, :]) / (omega * sumw)


def dirty_image_dft(r1, r2, c, N: int, cell_arcsec: float, omega: float,
                    sumw: float, rows=None, cols=None) -> np.ndarray:
    """Exact 2-D dirty image of Section 3.2 by brute force:
    I(t1, t2) = 1/(omega sum w) Re sum_q c_q exp(i 2 pi (r1 t1 + r2 t2)),
    t1 = -beta (j1 - N/2), t2 = beta (j2 - N/2).  Optional pixel subsets."""
    beta = cell_arcsec * ARCSEC
    rows = np.arange(N) if rows is None else np.asarray(rows)
    cols = np.arange(N) if cols is None else np.asarray(cols)
    t1 = -beta * (cols - N // 2)
    t2 = beta * (rows - N // 2)
    r1 = np.asarray(r1)
    r2 = np.asarray(r2)
    c = np.asarray(c)
    e1 = np.exp(2j * np.pi * np.outer(t1, r1))        # [cols, q]
    e2 = np.exp(2j * np.pi * np.outer(t2, r2))        # [rows, q]
    img = (e2 * c[None, :]) @ e1.T                    # [rows, cols]
    return img.real / (omega * sumw)


# ==========================================================================
# S6 — re-projection (Section 3.3; Appendix A)
# ==========================================================================

def reproject_map_reduced(p1, p2, N: int, cell_deg: float, xi: float, eta: float):
    """Section 3.3 reduced pixel-to-pixel map of a tilted-plane pixel (p1, p2)
    (1-based) to the standard plane.  Sign of y' from Appendix A (reading c7):
    y' = y + r0 z eta (with z = 0 the map is then the identity)."""
    c0 = N / 2 + 1
    x = -cell_deg * (np.asarray(p1, dtype=np.float64) - c0)
    y = cell_deg * (np.asarray(p2, dtype=np.float64) - c0)
    h = np.sqrt(x * x + y * y)
    r0 = 180.0 / np.pi
    q = (h / r0) ** 2
    z = q / (1.0 + np.sqrt(1.0 - q))
    xp = x + r0 * z * xi
    yp = y + r0 * z * eta
    return -xp / cell_deg + c0, yp / cell_deg + c0


def reproject_map_wcs(p1, p2, N: int, cell_deg: float, xi: float, eta: float,
                      eps: float = 1e-10):
    """Appendix A: the conventional WCS route through native spherical
    coordinates (phi, theta) with the SIN tilt terms; angles in radians."""
    c0 = N / 2 + 1
    x = -(np.pi / 180) * cell_deg * (np.asarray(p1, dtype=np.float64) - c0)
    y = (np.pi / 180) * cell_deg * (np.asarray(p2, dtype=np.float64) - c0)
    x, y = np.broadcast_arrays(x, y)
    phi = np.where((x == 0) & (y <= 0), 0.0,
          np.where((x == 0) & (y > 0), np.pi,
          np.where((y == 0) & (x > 0), np.pi / 2,
          np.where((y == 0) & (x < 0), -np.pi / 2, np.arctan2(x, -y)))))
    r2 = x * x + y * y
    r = np.sqrt(r2)
    theta_small = np.where(r == 0, np.pi / 2,
                  np.where((r >= 1) & (r - 1 < eps), 0.0, np.arccos(np.minimum(r, 1.0))))
    s = np.sqrt(np.maximum(1.0 - r2, 0.0))
    theta_large = np.where(s == 0, 0.0,
                  np.where((s >= 1) & (s - 1 < eps), np.pi / 2, np.arcsin(np.minimum(s, 1.0))))
    theta = np.where(r2 < 0.5, theta_small, theta_large)
    xs = np.cos(theta) * np.sin(phi) + xi * (1 - np.sin(theta))
    ys = -(np.cos(theta) * np.cos(phi) - eta * (1 - np.sin(theta)))
    xd = xs * 180 / np.pi
    yd = ys * 180 / np.pi
    return -xd / cell_deg + c0, yd / cell_deg + c0


def reproject_source_pixels(N: int, cell_deg: float, xi: float, eta: float,
                            iters: int = 8):
    """Reading c8 (gather): for every output pixel p' find the tilted pixel p
    with map(p) = p' by fixed-point iteration p <- p' - (map(p) - p).  Returns
    0-based float source indices (j1, j2) as arrays [N, N] (row = j2)."""
    j2o, j1o = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64),
                           indexing="ij")
    return reproject_source_at(j1o, j2o, N, cell_deg, xi, eta, iters)


def reproject_source_at(j1o, j2o, N: int, cell_deg: float, xi: float, eta: float,
                        iters: int = 8):
    """The fixed point of reproject_source_pixels for given 0-based output
    pixels (j1o = column, j2o = row), any array shape."""
    p1o = np.asarray(j1o, dtype=np.float64) + 1
    p2o = np.asarray(j2o, dtype=np.float64) + 1
    p1, p2 = p1o.copy(), p2o.copy()
    for _ in range(iters):
        m1, m2 = reproject_map_reduced(p1, p2, N, cell_deg, xi, eta)
        p1 = p1o - (m1 - p1)
        p2 = p2o - (m2 - p2)
    return p1 - 1, p2 - 1


def bilinear(img: np.ndarray, j1, j2) -> np.ndarray:
    """Bilinear interpolation at 0-based (j1 = column, j2 = row); a source
    position outside [0, N-1] in either axis gives 0 (the missing corners);
    neighbours beyond the last row/column count as 0."""
    N = img.shape[0]
    out = np.zeros(np.shape(j1))
    ok = (j1 >= 0) & (j1 <= N - 1) & (j2 >= 0) & (j2 <= N - 1)
    a0 = np.floor(j1).astype(np.int64)
    b0 = np.floor(j2).astype(np.int64)
    fa = j1 - a0
    fb = j2 - b0
    pad = np.zeros((N + 1, N + 1))
    pad[:N, :N] = img
    a0c = np.clip(a0, 0, N - 1)
    b0c = np.clip(b0, 0, N - 1)
    v = ((1 - fb) * ((1 - fa) * pad[b0c, a0c] + fa * pad[b0c, a0c + 1]) +
         fb * ((1 - fa) * pad[b0c + 1, a0c] + fa * pad[b0c + 1, a0c + 1]))
    out[ok] = v[ok]
    return out


def reproject(img_tilted: np.ndarray, cell_arcsec: float, xi: float, eta: float,
              iters: int = 8) -> np.ndarray:
    """S6: standard-plane image from the tilted-plane image (reading c8)."""
    N = img_tilted.shape[0]
    j1, j2 = reproject_source_pixels(N, cell_arcsec / 3600.0, xi, eta, iters)
    return bilinear(img_tilted, j1, j2)


# ==========================================================================
# One snapshot: S1..S6
# ==========================================================================

def image_snapshot(uvw_m, freq_hz, vis, flag, weight, N: int, cell_arcsec: float,
                   W: int = 8, sigma: int = 2, keep_grid: bool = False) -> Dict:
    p = prepare(uvw_m, freq_hz, vis, flag, weight)
    G = sigma * N
    beta = es_beta(W)
    g1, g2 = grid_coords(p["r"][:, 0], p["r"][:, 1], N, cell_arcsec, sigma)
    grid = grid_es(g1, g2, p["c"], G, W, beta)
    tilted = tilted_image(grid, N, W, beta, p["omega"], p["sumw"])
    image = reproject(tilted, cell_arcsec, p["xi"], p["eta"])
    out = dict(V=p["V"], omega=p["omega"], xi=p["xi"], eta=p["eta"], sumw=p["sumw"],
               n_vis=p["n_vis"], tilted=tilted, image=image, g1=g1, g2=g2, c=p["c"],
               r=p["r"])
    if keep_grid:
        out["grid"] = grid
    return out


# ==========================================================================
# Adjoint of S2..S6: reverse-mode derivative of one snapshot's image
# (the "adjoint" the paper names as the route to gradients, Section 1)
# ==========================================================================
#
# Convention: for a real loss L and a complex quantity z the gradient is
# dL/dRe z + i dL/dIm z.  The plane fit of S1 (V, omega and the selection
# w_q > 0) is piecewise constant in the weights and not differentiated with
# respect to uvw, so it is held fixed.

def bilinear_adjoint(grad: np.ndarray, j1, j2) -> np.ndarray:
    """Transpose of bilinear(): every output cotangent is spread onto the four
    source pixels with the interpolation weights, under the same rules (a
    source position outside [0, N-1] contributes nothing; neighbours beyond
    the last row/column are dropped)."""
    N = grad.shape[0]
    ok = (j1 >= 0) & (j1 <= N - 1) & (j2 >= 0) & (j2 <= N - 1)
    a0 = np.floor(j1[ok]).astype(np.int64)
    b0 = np.floor(j2[ok]).astype(np.int64)
    fa = j1[ok] - a0
    fb = j2[ok] - b0
    g = grad[ok]
    out = np.zeros((N + 1, N + 1))
    np.add.at(out, (b0, a0), (1 - fb) * (1 - fa) * g)
    np.add.at(out, (b0, a0 + 1), (1 - fb) * fa * g)
    np.add.at(out, (b0 + 1, a0), fb * (1 - fa) * g)
    np.add.at(out, (b0 + 1, a0 + 1), fb * fa * g)
    return out[:N, :N]


def reproject_adjoint(grad_image: np.ndarray, cell_arcsec: float, xi: float, eta: float,
                      iters: int = 8) -> np.ndarray:
    """Transpose of reproject(): cotangent of the tilted-plane image."""
    N = grad_image.shape[0]
    j1, j2 = reproject_source_pixels(N, cell_arcsec / 3600.0, xi, eta, iters)
    return bilinear_adjoint(grad_image, j1, j2)


def tilted_image_adjoint(grad_tilted: np.ndarray, G: int, W: int, beta: float,
                         omega: float, sumw: float) -> np.ndarray:
    """Transpose of tilted_image() with respect to the complex grid: the
    tilted pixel j depends on Grid[k] through Re(Grid[k] e^{+i theta_kj}) s_j,
    s_j = 1 / (psi_hat psi_hat omega sum w), so
        dL/dGrid[k] = sum_j (dL/dT_j) s_j e^{-i theta_kj},
    a forward centred DFT of the scaled cotangent zero-padded to G x G."""
    N = grad_tilted.shape[0]
    ph = correction_vector(N, G, W, beta)
    U = grad_tilted / (ph[:, None] * ph[None, :]) / (omega * sumw)
    pad = np.zeros((G, G))
    lo = G // 2 - N // 2
    pad[lo:lo + N, lo:lo + N] = U
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(pad)))


def image_snapshot_adjoint(uvw_m, freq_hz, vis, flag, weight, N: int, cell_arcsec: float,
                           grad_image: np.ndarray, W: int = 8, sigma: int = 2) -> Dict:
    """Reverse mode of image_snapshot() for a loss L with dL/dImage =
    grad_image.  Per (baseline, channel) sample q:
      g[q]     = dL/dc_q, c_q = w_a V_a + w_b V_b (the gridded value): the
                 ES degridding of the grid cotangent at the sample
                 (degrid_es is the adjoint of grid_es); 0 outside the
                 selection.
      grad_vis = w_p g for the parallel hands p of selected samples, else 0.
      grad_weight[p] = Re(conj(g) V_p) - <grad_image, image> / sum w for the
                 unflagged parallel hands of selected samples (c_q is linear
                 in w_p and the image carries 1 / sum w), else 0.
    """
    r = image_snapshot(uvw_m, freq_hz, vis, flag, weight, N, cell_arcsec, W, sigma)
    G = sigma * N
    beta = es_beta(W)
    gt = reproject_adjoint(np.asarray(grad_image, dtype=np.float64), cell_arcsec,
                           r["xi"], r["eta"])
    H = tilted_image_adjoint(gt, G, W, beta, r["omega"], r["sumw"])
    g_sel = degrid_es(H, r["g1"], r["g2"], W, beta)
    vis = np.asarray(vis)
    nbl, nch, n_pol = vis.shape
    w_q, _ = sample_weights_and_values(vis, flag, weight)
    sel = w_q > 0
    g = np.zeros((nbl, nch), dtype=np.complex128)
    g[sel] = g_sel
    pa, pb = parallel_hands(n_pol)
    f = np.asarray(flag).astype(bool)
    wp = np.where(f, 0.0, 1.0 if weight is None else np.asarray(weight, dtype=np.float64))
    dot = float((np.asarray(grad_image, dtype=np.float64) * r["image"]).sum())
    grad_vis = np.zeros(vis.shape, dtype=np.complex128)
    grad_weight = np.zeros(vis.shape)
    for p in sorted({pa, pb}):
        use = sel & ~f[:, :, p]
        grad_vis[:, :, p] = np.where(sel, wp[:, :, p] * g, 0.0)
        gw = (np.conj(g) * vis[:, :, p].astype(np.complex128)).real - dot / r["sumw"]
        grad_weight[:, :, p] = np.where(use, gw, 0.0)
    return dict(g=g, grad_vis=grad_vis, grad_weight=grad_weight, image=r["image"],
                dot=dot, sumw=r["sumw"], omega=r["omega"])


def point_source_vis(uvw_m, freq_hz, n_pol: int, l: float, m: float, flux: float):
    """Measurement equation for one point source (Section 1): V = S exp(-2 pi
    i (u l + v m + w (n - 1))), n = sqrt(1 - l^2 - m^2), in every parallel
    hand (cross hands 0)."""
    k = np.asarray(freq_hz, dtype=np.float64) / C_LIGHT
    uvw = np.asarray(uvw_m, dtype=np.float64)
    n = math.sqrt(1.0 - l * l - m * m)
    ph = (uvw[:, 0:1] * l + uvw[:, 1:2] * m + uvw[:, 2:3] * (n - 1.0)) * k[None, :]
    v = flux * np.exp(-2j * np.pi * ph)
    out = np.zeros((uvw.shape[0], k.size, n_pol), dtype=np.complex128)
    pa, pb = parallel_hands(n_pol)
    out[:, :, pa] = v
    out[:, :, pb] = v
    return out


def point_source_gradient(uvw_m, freq_hz, grad_vis, l: float, m: float, flux: float):
    """Chain rule from grad_vis (dL/dRe V + i dL/dIm V per record) to the
    point-source parameters of point_source_vis: dL/dtheta = sum Re(conj(
    grad_vis) dV/dtheta), with dV/dS = V/S, dV/dl = -2 pi i k (u - w l / n) V,
    dV/dm = -2 pi i k (v - w m / n) V."""
    k = np.asarray(freq_hz, dtype=np.float64) / C_LIGHT
    uvw = np.asarray(uvw_m, dtype=np.float64)
    n = math.sqrt(1.0 - l * l - m * m)
    ph = (uvw[:, 0:1] * l + uvw[:, 1:2] * m + uvw[:, 2:3] * (n - 1.0)) * k[None, :]
    v = np.exp(-2j * np.pi * ph)                              # V / S
    gsum = np.asarray(grad_vis).sum(axis=2)                   # same V in each hand
    dl = -2j * np.pi * k[None, :] * (uvw[:, 0:1] - uvw[:, 2:3] * l / n) * flux * v
    dm = -2j * np.pi * k[None, :] * (uvw[:, 1:2] - uvw[:, 2:3] * m / n) * flux * v
    return dict(l=float((np.conj(gsum) * dl).real.sum()),
                m=float((np.conj(gsum) * dm).real.sum()),
                flux=float((np.conj(gsum) * v).real.sum()))


# ==========================================================================
# Windowed point-source localisation (Section 1's adjoint route to gradients,
# applied to sub-pixel positions of candidates, Section 6)
# ==========================================================================
#
# A candidate window is a LOC_WINDOW x LOC_WINDOW block of the tilted-plane
# image with corner (row j2c, column j1c).  Its model is the 2-D dirty image
# of Section 3.2 of one point source (l, m, S) (point_source_vis, with the
# data's flags and weights), restricted to the window.  The loss of a window
# is the squared residual between the data's tilted image and the model,
# summed over its pixels; the total loss sums the windows.  Every image value
# here is the exact brute-force sum (dirty_image_dft), not the gridded one.

LOC_WINDOW = 32


def window_axes(corner, size: int = LOC_WINDOW):
    """Rows and columns (0-based) of the window with corner (j2c, j1c)."""
    j2c, j1c = int(corner[0]), int(corner[1])
    return np.arange(j2c, j2c + size), np.arange(j1c, j1c + size)


def window_image_exact(p: Dict, N: int, cell_arcsec: float, corner,
                       size: int = LOC_WINDOW) -> np.ndarray:
    """The Section 3.2 dirty image of prepare()'s samples on one window."""
    rows, cols = window_axes(corner, size)
    return dirty_image_dft(p["r"][:, 0], p["r"][:, 1], p["c"], N, cell_arcsec, p["omega"],
                           p["sumw"], rows, cols)


def window_adjoint_exact(p: Dict, N: int, cell_arcsec: float, corner,
                         grad_window: np.ndarray) -> np.ndarray:
    """dL/dc_q (the complex convention above) of a loss whose cotangent on the
    window's image is grad_window:
        1/(omega sum w) sum_j g_j exp(-2 pi i (r1 t1_j + r2 t2_j)),
    the transpose of window_image_exact (the image is Re of the sum)."""
    size = grad_window.shape[0]
    rows, cols = window_axes(corner, size)
    beta = cell_arcsec * ARCSEC
    t1 = -beta * (cols - N // 2)
    t2 = beta * (rows - N // 2)
    e1 = np.exp(-2j * np.pi * np.outer(p["r"][:, 0], t1))     # [q, cols]
    e2 = np.exp(-2j * np.pi * np.outer(p["r"][:, 1], t2))     # [q, rows]
    return ((e2 @ grad_window) * e1).sum(axis=1) / (p["omega"] * p["sumw"])


def source_of_pixel(t1: float, t2: float, V: np.ndarray) -> Tuple[float, float]:
    """(l, m) of the point source whose 2-D image peaks at tilted-plane
    position (t1, t2): its phase b.(s - z) equals r.tau with tau = V (s - z),
    so s = V^T tau + z with tau3 the root of |s| = 1 nearest 0 (the t3 of
    App. B with t = tau)."""
    tau = np.array([t1, t2, float(t3_of(t1, t2, V))])
    s = V.T @ tau + np.array([0.0, 0.0, 1.0])
    return float(s[0]), float(s[1])


def localise(uvw_m, freq_hz, vis, flag, weight, N: int, cell_arcsec: float, windows,
             sources, size: int = LOC_WINDOW) -> Dict:
    """Loss, models and gradients of the windowed point-source fit.
    windows: [n_win, 2] corners (j2c, j1c); sources: [n_win, 3] (l, m, S).
    For window w with data image D and model M (both exact):
      L_w = sum (D - M)^2;  g^M = dL/dM = -2 (D - M);  g^D = -g^M;
      grad_src[w]  = d L / d(l, m, S) through point_source_gradient of
                     grad_vis = w_p dL/dc^M_q (the model's sample values);
      grad_weight[p] = sum_w Re(conj(dL/dc^M) V^M_p) + Re(conj(dL/dc^D) V_p)
                       - (<g^M, M> + <g^D, D>) / sum w
                     on the unflagged parallel hands of selected samples
                     (c = w_a V_a + w_b V_b is linear in w_p and both images
                     carry 1 / sum w), else 0."""
    vis = np.asarray(vis)
    nbl, nch, n_pol = vis.shape
    windows = np.asarray(windows, dtype=np.int64).reshape(-1, 2)
    sources = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    pd = prepare(uvw_m, freq_hz, vis, flag, weight)
    pa, pb = parallel_hands(n_pol)
    f = np.asarray(flag).astype(bool)
    wp = np.where(f, 0.0, 1.0 if weight is None else np.asarray(weight, dtype=np.float64))
    sel = pd["sel"]
    loss = np.zeros(len(windows))
    models = np.zeros((len(windows), size, size))
    data = np.zeros((len(windows), size, size))
    grad_src = np.zeros((len(windows), 3))
    grad_weight = np.zeros(vis.shape)
    for i, (corner, (l, m, S)) in enumerate(zip(windows, sources)):
        vm = point_source_vis(uvw_m, freq_hz, n_pol, l, m, S)
        pm = prepare(uvw_m, freq_hz, vm, flag, weight)
        D = window_image_exact(pd, N, cell_arcsec, corner, size)
        M = window_image_exact(pm, N, cell_arcsec, corner, size)
        R = D - M
        loss[i] = float((R * R).sum())
        models[i], data[i] = M, D
        gM = -2.0 * R
        gq_m = np.zeros((nbl, nch), dtype=np.complex128)
        gq_m[sel] = window_adjoint_exact(pm, N, cell_arcsec, corner, gM)
        gq_d = -gq_m                       # the data's cotangent is -g^M
        grad_vis = np.zeros(vis.shape, dtype=np.complex128)
        for p in sorted({pa, pb}):
            grad_vis[:, :, p] = np.where(sel, wp[:, :, p] * gq_m, 0.0)
        gs = point_source_gradient(uvw_m, freq_hz, grad_vis, l, m, S)
        grad_src[i] = (gs["l"], gs["m"], gs["flux"])
        dot = float((gM * M).sum() + (-gM * D).sum())
        for p in sorted({pa, pb}):
            use = sel & ~f[:, :, p]
            gw = ((np.conj(gq_m) * vm[:, :, p]).real +
                  (np.conj(gq_d) * vis[:, :, p].astype(np.complex128)).real - dot / pd["sumw"])
            grad_weight[:, :, p] += np.where(use, gw, 0.0)
    return dict(loss=loss, model=models, data=data, grad_src=grad_src,
                grad_weight=grad_weight, V=pd["V"], omega=pd["omega"], sumw=pd["sumw"])


# ==========================================================================
# Near-coplanar (3-D) mode (Section 3.4, Appendix B, Table 2)
# ==========================================================================

def t3_of(t1, t2, V):
    """Section 3.4 (derived in Appendix B.1): the t3 on the celestial sphere
    for image coordinates (t1, t2), the root that is 0 at t1 = t2 = 0,
        t3 = -V33 + sgn(V33) sqrt(1 - (t1 + V13)^2 - (t2 + V23)^2).
    Written without cancellation: with a = t1^2 + 2 t1 V13 + t2^2 + 2 t2 V23
    (using V13^2 + V23^2 + V33^2 = 1), t3 = -sgn(V33) a / (sqrt(V33^2 - a) + |V33|)."""
    t1 = np.asarray(t1, dtype=np.float64)
    t2 = np.asarray(t2, dtype=np.float64)
    a = t1 * t1 + 2.0 * t1 * V[0, 2] + t2 * t2 + 2.0 * t2 * V[1, 2]
    v33 = V[2, 2]
    return -np.sign(v33) * a / (np.sqrt(v33 * v33 - a) + abs(v33))


def pixel_t(N: int, cell_arcsec: float):
    """t1 (columns) and t2 (rows) of the N x N pixel centres (reading c6)."""
    beta = cell_arcsec * ARCSEC
    j = np.arange(N) - N // 2
    return -beta * j, beta * j


def t3_max(N: int, cell_arcsec: float, V) -> float:
    """max |t3| over the image's pixel centres (the valid region D); a pixel
    whose (t1, t2) is off the visible sphere (no real t3) is not valid."""
    t1, t2 = pixel_t(N, cell_arcsec)
    with np.errstate(invalid="ignore"):
        t3 = np.abs(t3_of(t1[None, :], t2[:, None], V))
    return float(np.nanmax(t3)) if np.isfinite(t3).any() else 0.0


def chebyshev_coeffs(alpha, K: int) -> np.ndarray:
    """Jacobi-Anger coefficients of exp(i alpha s) in Chebyshev polynomials
    (Appendix B.2): c_0 = J_0(alpha), c_k = 2 i^k J_k(alpha); shape
    alpha.shape + (K,).  scipy's Bessel J is the library step."""
    from scipy.special import jv
    alpha = np.asarray(alpha, dtype=np.float64)
    k = np.arange(K)
    J = jv(k, alpha[..., None])
    c = 2.0 * (1j ** k) * J
    c[..., 0] = J[..., 0]
    return c


def chebyshev_T(s, K: int) -> np.ndarray:
    """T_k(s) for k < K (shape s.shape + (K,)) by the three-term recurrence."""
    s = np.asarray(s, dtype=np.float64)
    T = np.empty(s.shape + (K,))
    T[..., 0] = 1.0
    if K > 1:
        T[..., 1] = s
    for k in range(2, K):
        T[..., k] = 2.0 * s * T[..., k - 1] - T[..., k - 2]
    return T


CHEB_ORDERS = (8, 16, 24, 32)
CHEB_GAMMA = 1e-2
ALPHA_TARGET = 10.0


def chebyshev_order(alpha_slab: float, n_alpha: int = 256, n_s: int = 257):
    """Section 3.4: the smallest K in {8, 16, 24, 32} whose maximum sampled
    error |exp(i alpha s) - sum_k c_k(alpha) T_k(s)| over 0 <= alpha <=
    alpha_slab, -1 <= s <= 1 is below 1e-2, else 32.  Reading: the samples
    are n_alpha uniform alphas and n_s uniform s, both ends included.
    Returns (K, error)."""
    a = np.linspace(0.0, alpha_slab, n_alpha)
    sv = np.linspace(-1.0, 1.0, n_s)
    exact = np.exp(1j * a[:, None] * sv[None, :])
    err = np.inf
    for K in CHEB_ORDERS:
        approx = np.einsum("ak,sk->as", chebyshev_coeffs(a, K), chebyshev_T(sv, K))
        err = float(np.abs(exact - approx).max())
        if err < CHEB_GAMMA:
            return K, err
    return CHEB_ORDERS[-1], err


def slab_plan(r3min: float, r3max: float, t3max: float, K=None) -> Dict:
    """Section 3.4, Eqs. (26)-(27): Phi_max = 2 pi t3max (r3max - r3min)/2,
    N_slab = max(1, ceil(Phi_max / alpha_target)), slabs of equal width
    2 dr3 over [r3min, r3max], alpha_slab = 2 pi t3max dr3 and K from
    chebyshev_order (or as given)."""
    phi = 2.0 * math.pi * t3max * (r3max - r3min) / 2.0
    n_slab = max(1, int(math.ceil(phi / ALPHA_TARGET)))
    dr3 = (r3max - r3min) / (2.0 * n_slab)
    centres = r3min + (2.0 * np.arange(n_slab) + 1.0) * dr3
    alpha_slab = 2.0 * math.pi * t3max * dr3
    if K is None:
        K, err = chebyshev_order(alpha_slab)
    else:
        err = None
    return dict(phi_max=phi, n_slab=n_slab, dr3=dr3, centres=centres, alpha_slab=alpha_slab,
                K=K, err=err, r3min=r3min)


def slab_of(r3, plan) -> Tuple[np.ndarray, np.ndarray]:
    """Slab index p and s_q = (r3_q - r3_p) / dr3 of every sample (the last
    slab is closed; a zero-width range gives s = 0)."""
    r3 = np.asarray(r3, dtype=np.float64)
    if plan["dr3"] <= 0.0:
        return np.zeros(r3.shape, dtype=np.int64), np.zeros(r3.shape)
    p = np.floor((r3 - plan["r3min"]) / (2.0 * plan["dr3"])).astype(np.int64)
    p = np.clip(p, 0, plan["n_slab"] - 1)
    s = (r3 - plan["centres"][p]) / plan["dr3"]
    return p, s


def tilted_image_3d(r, c, N: int, cell_arcsec: float, V, omega: float, sumw: float,
                    W: int = 8, sigma: int = 2, K=None) -> Dict:
    """Near-coplanar tilted image (Section 3.4): for every slab p and order
    k the Chebyshev moment M_pk (ES gridding of T_k(s_q) c_q, full complex
    centred inverse FFT, grid correction and 1/(omega sum w)), combined per
    pixel as Re sum_p exp(i 2 pi r3_p t3) sum_k c_k(2 pi dr3 t3) M_pk."""
    G = sigma * N
    beta_es = es_beta(W)
    r = np.asarray(r, dtype=np.float64)
    c = np.asarray(c, dtype=np.complex128)
    t1, t2 = pixel_t(N, cell_arcsec)
    with np.errstate(invalid="ignore"):
        T3 = t3_of(t1[None, :], t2[:, None], V)
    off = ~np.isfinite(T3)                     # pixels off the visible sphere: image 0
    T3 = np.where(off, 0.0, T3)
    t3m = t3_max(N, cell_arcsec, V)
    plan = slab_plan(float(r[:, 2].min()), float(r[:, 2].max()), t3m, K)
    p_of, s_of = slab_of(r[:, 2], plan)
    g1, g2 = grid_coords(r[:, 0], r[:, 1], N, cell_arcsec, sigma)
    ph = correction_vector(N, G, W, beta_es)
    corr = 1.0 / (ph[:, None] * ph[None, :]) / (omega * sumw)
    coef = chebyshev_coeffs(2.0 * math.pi * plan["dr3"] * T3, plan["K"])   # [N, N, K]
    out = np.zeros((N, N))
    for p in range(plan["n_slab"]):
        m = p_of == p
        if not m.any():
            continue
        Tk = chebyshev_T(s_of[m], plan["K"])
        slab_phase = np.exp(2j * math.pi * plan["centres"][p] * T3)
        acc = np.zeros((N, N), dtype=np.complex128)
        for k in range(plan["K"]):
            grid = grid_es(g1[m], g2[m], c[m] * Tk[:, k], G, W, beta_es)
            M = ifft_centred(grid, N) * corr
            acc += coef[:, :, k] * M
        out += (slab_phase * acc).real
    out[off] = 0.0
    return dict(tilted=out, plan=plan, t3=T3, t3max=t3m)


def dirty_image_3d_dft(r, c, N: int, cell_arcsec: float, V, omega: float, sumw: float,
                       rows=None, cols=None) -> np.ndarray:
    """Exact near-coplanar dirty image I_D^(3) of Section 3.4 by brute force:
    1/(omega sum w) Re sum_q c_q exp(i 2 pi (r1 t1 + r2 t2 + r3 t3(t1, t2)))."""
    t1, t2 = pixel_t(N, cell_arcsec)
    rows = np.arange(N) if rows is None else np.asarray(rows)
    cols = np.arange(N) if cols is None else np.asarray(cols)
    r = np.asarray(r)
    c = np.asarray(c)
    out = np.zeros((len(rows), len(cols)))
    for a, j2 in enumerate(rows):
        tt1 = t1[cols]
        tt2 = np.full_like(tt1, t2[j2])
        tt3 = t3_of(tt1, tt2, V)
        phase = 2 * np.pi * (np.outer(tt1, r[:, 0]) + np.outer(tt2, r[:, 1]) + np.outer(tt3, r[:, 2]))
        out[a] = (np.exp(1j * phase) @ c).real
    return out / (omega * sumw)


def image_snapshot_3d(uvw_m, freq_hz, vis, flag, weight, N: int, cell_arcsec: float,
                      W: int = 8, sigma: int = 2, K=None) -> Dict:
    """S1 + the near-coplanar S2-S5 + S6 for one snapshot."""
    p = prepare(uvw_m, freq_hz, vis, flag, weight)
    t = tilted_image_3d(p["r"], p["c"], N, cell_arcsec, p["V"], p["omega"], p["sumw"], W, sigma, K)
    image = reproject(t["tilted"], cell_arcsec, p["xi"], p["eta"])
    return dict(V=p["V"], omega=p["omega"], xi=p["xi"], eta=p["eta"], sumw=p["sumw"],
                r=p["r"], c=p["c"], tilted=t["tilted"], image=image, plan=t["plan"],
                t3max=t["t3max"])


def hermitian_half(grid: np.ndarray) -> np.ndarray:
    """S[k] = (Grid[k] + conj(Grid[-k])) / 2 (k' = k - G/2, -k' taken modulo
    G), returned for rows k2' = 0..G/2 (row k2' = G/2 is the periodic copy of
    k2' = -G/2).  The inverse DFT of S equals Re of the inverse DFT of Grid;
    this is a test helper for half-plane grid layouts."""
    G = grid.shape[0]
    idx = (G - np.arange(G)) % G
    S = 0.5 * (grid + np.conj(grid[idx][:, idx]))
    rows = (G // 2 + np.arange(G // 2 + 1)) % G
    return S[rows, :]


# ==========================================================================
# S7 — tLISI (stand-in definition, reading c9; parity unpinned vs the paper)
# ==========================================================================

def tlisi(I0: np.ndarray, I1: np.ndarray, I2: np.ndarray, T: int) -> np.ndarray:
    """tLISI of every T x T tile from the three youngest images (Section 2,
    Section 4.5): D_a = I1 - I0, D_b = I2 - I1.  With tile moments in float64
    (population moments over the n = T^2 pixels),
      S = ((2 mu_a mu_b + C1)(2 s_ab + C2)) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2)),
    C1 = (0.01 L)^2, C2 = (0.03 L)^2, tLISI = (1 + S) / 2 in [0, 1].
    L is the dynamic range of the three images, max |I| over all pixels of
    I0, I1, I2 (so a quiet tile stays near 1 whatever happens elsewhere, as
    Section 2 describes); L = 0 gives 1 everywhere."""
    a = np.asarray(I1, np.float64) - np.asarray(I0, np.float64)
    b = np.asarray(I2, np.float64) - np.asarray(I1, np.float64)
    N = a.shape[0]
    nt = N // T
    L = max(np.abs(I0).max(), np.abs(I1).max(), np.abs(I2).max())
    if L == 0:
        return np.ones((nt, nt))
    at = a.reshape(nt, T, nt, T).transpose(0, 2, 1, 3).reshape(nt, nt, T * T)
    bt = b.reshape(nt, T, nt, T).transpose(0, 2, 1, 3).reshape(nt, nt, T * T)
    n = T * T
    mu_a = at.sum(-1) / n
    mu_b = bt.sum(-1) / n
    va = (at * at).sum(-1) / n - mu_a * mu_a
    vb = (bt * bt).sum(-1) / n - mu_b * mu_b
    cab = (at * bt).sum(-1) / n - mu_a * mu_b
    C1 = (0.01 * L) ** 2
    C2 = (0.03 * L) ** 2
    S = ((2 * mu_a * mu_b + C1) * (2 * cab + C2)) / ((mu_a ** 2 + mu_b ** 2 + C1) * (va + vb + C2))
    return (1.0 + S) / 2.0


# ==========================================================================
# S8 — candidates (Sections 2, 6.2, 6.3) in a fixed FP64 evaluation order
# ==========================================================================
# Evaluation-order rules (readings c10-c12, written so a second implementation
# can reproduce every bit): IEEE binary64, round to nearest, every product and
# sum rounded separately (no fused multiply-add), sums sequential in the stated
# index order unless a pairwise tree is stated.

TAYLOR_TERMS = 13
PI_2 = 1.5707963267948966      # binary64 nearest to pi/2


def _inv_factorials():
    fact = [1.0]
    for n in range(1, 2 * TAYLOR_TERMS + 2):
        fact.append(fact[-1] * float(n))
    cos_c = [(1.0 if k % 2 == 0 else -1.0) / fact[2 * k] for k in range(TAYLOR_TERMS)]
    sin_c = [(1.0 if k % 2 == 0 else -1.0) / fact[2 * k + 1] for k in range(TAYLOR_TERMS)]
    return cos_c, sin_c


def twiddle(m: int, S: int) -> Tuple[float, float]:
    """cos, sin of 2 pi m / S: quadrant q = floor(4m / S), remainder
    a = 4m - qS, r = (PI_2 * a) / S in [0, pi/2), Taylor series in r^2
    (Horner from the highest of 13 terms), then the quadrant's swap/sign."""
    m %= S
    q = (4 * m) // S
    a = 4 * m - q * S
    r = (PI_2 * float(a)) / float(S)
    r2 = r * r
    cos_c, sin_c = _inv_factorials()
    c = cos_c[-1]
    s = sin_c[-1]
    for k in range(TAYLOR_TERMS - 2, -1, -1):
        c = c * r2 + cos_c[k]
        s = s * r2 + sin_c[k]
    s = s * r
    if q == 0:
        return c, s
    if q == 1:
        return -s, c
    if q == 2:
        return -c, -s
    return s, -c


def twiddle_table(S: int):
    cs = [twiddle(m, S) for m in range(S)]
    return np.array([x[0] for x in cs]), np.array([x[1] for x in cs])


def pairwise_sum(a, lo: int = 0, hi: Optional[int] = None) -> float:
    """Pairwise tree: sum(a[lo:hi]) = sum(a[lo:mid]) + sum(a[mid:hi]),
    mid = lo + (hi - lo) // 2; a single element is itself; empty is 0."""
    if hi is None:
        hi = len(a)
    n = hi - lo
    if n <= 0:
        return 0.0
    if n == 1:
        return float(a[lo])
    mid = lo + n // 2
    return pairwise_sum(a, lo, mid) + pairwise_sum(a, mid, hi)


HARMONICS = (1, 2, 4, 8)


def periodic_scores(cube: np.ndarray) -> np.ndarray:
    """Section 2 / 6.2: per tile, the tLISI series x_t (t = 0..S-1, mean
    removed) is Fourier transformed along time, P_f = A_f^2 + B_f^2 with
    A_f = sum_t x_t cos(2 pi f t / S), B_f = sum_t x_t sin(2 pi f t / S)
    (f = 1..F, F = floor(S/2)); harmonic sums H_h(f) = sum_{i=1..h, i f <= F}
    P_{i f} for h in (1, 2, 4, 8); score = max_{f,h} H_h(f) / sqrt(h).

    The series is real, so times t and S - t share their cosine and have
    opposite sines (2 pi f (S - t) / S = 2 pi f - 2 pi f t / S); the sums run
    over u_t = x_t + x_{S-t} and v_t = x_t - x_{S-t} for t = 1..floor((S-1)/2)
    with the twiddle of t, after A = x_0 cos(0) and before the middle time
    S/2 of an even S (reading c10's order); for an even S the frequencies f
    and S/2 - f are summed together from the even and odd times."""
    S = cube.shape[0]
    x = cube.reshape(S, -1).astype(np.float64)
    nt = x.shape[1]
    acc = np.zeros(nt)
    for t in range(S):
        acc = acc + x[t]
    mu = acc / float(S)
    xc = [x[t] - mu for t in range(S)]
    F = S // 2
    if F == 0:
        return np.zeros(nt)
    cos_t, sin_t = twiddle_table(S)
    Th = (S - 1) // 2
    u = [None] + [xc[t] + xc[S - t] for t in range(1, Th + 1)]
    v = [None] + [xc[t] - xc[S - t] for t in range(1, Th + 1)]
    P = np.zeros((F + 1, nt))
    half = S // 2
    singles = list(range(1, F + 1))
    if S % 2 == 0:
        # For an even S the frequencies f and g = S/2 - f share their
        # twiddles: 2 pi g t / S = pi t - 2 pi f t / S, so cos(2 pi g t / S) =
        # (-1)^t cos(2 pi f t / S) and sin(2 pi g t / S) = -(-1)^t sin(...).
        # Summing the even and odd times apart gives both transforms (g's
        # middle time S/2 keeps its own twiddle).
        NP = (half - 1) // 2
        for f in range(1, NP + 1):
            g = half - f
            Ae, Ao, Be, Bo = np.zeros(nt), np.zeros(nt), np.zeros(nt), np.zeros(nt)
            for t in range(1, Th + 1):
                m = (f * t) % S
                if t % 2 == 0:
                    Ae = Ae + u[t] * cos_t[m]
                    Be = Be + v[t] * sin_t[m]
                else:
                    Ao = Ao + u[t] * cos_t[m]
                    Bo = Bo + v[t] * sin_t[m]
            base = xc[0] * cos_t[0] + Ae
            Af, Ag = base + Ao, base - Ao
            Bf, Bg = Be + Bo, Bo - Be
            mf, mg = (f * half) % S, (g * half) % S
            Af = Af + xc[half] * cos_t[mf]
            Bf = Bf + xc[half] * sin_t[mf]
            Ag = Ag + xc[half] * cos_t[mg]
            Bg = Bg + xc[half] * sin_t[mg]
            P[f] = Af * Af + Bf * Bf
            P[g] = Ag * Ag + Bg * Bg
        singles = ([half // 2] if half % 2 == 0 else []) + [half]
    for f in singles:
        A = xc[0] * cos_t[0]
        B = np.zeros(nt)
        for t in range(1, Th + 1):
            m = (f * t) % S
            A = A + u[t] * cos_t[m]
            B = B + v[t] * sin_t[m]
        if S % 2 == 0:
            m = (f * half) % S
            A = A + xc[half] * cos_t[m]
            B = B + xc[half] * sin_t[m]
        P[f] = A * A + B * B
    best = np.zeros(nt)
    roots = {h: math.sqrt(float(h)) for h in HARMONICS}
    for f in range(1, F + 1):
        for h in HARMONICS:
            H = np.zeros(nt)
            for i in range(1, h + 1):
                if i * f > F:
                    break
                H = H + P[i * f]
            best = np.maximum(best, H / roots[h])
    return best


def nonperiodic_scores(cube: np.ndarray) -> np.ndarray:
    """Section 6.3: score = sum_t (1 - tLISI_t), sequential in t."""
    S = cube.shape[0]
    x = cube.reshape(S, -1).astype(np.float64)
    acc = np.zeros(x.shape[1])
    for t in range(S):
        acc = acc + (1.0 - x[t])
    return acc


def threshold(scores: np.ndarray, k: float) -> Tuple[float, float, float]:
    """Significance (reading c11): mean and population standard deviation over
    all tiles by the pairwise tree, thr = mean + k * std."""
    s = np.asarray(scores, dtype=np.float64).ravel()
    n = len(s)
    mu = pairwise_sum(s) / float(n)
    d = s - mu
    var = pairwise_sum(d * d) / float(n)
    sd = math.sqrt(var)
    return mu + k * sd, mu, sd


def connected_boxes(mask: np.ndarray, T: int):
    """Reading c12: 8-connected candidate tiles; a component's label is its
    first tile in raster order; box = [x0, y0, x1, y1) in 0-based pixels
    (tile bounds times T); boxes sorted by (y0, x0, label)."""
    nty, ntx = mask.shape
    lab = -np.ones((nty, ntx), dtype=np.int64)
    boxes = []
    for y in range(nty):
        for x in range(ntx):
            if not mask[y, x] or lab[y, x] >= 0:
                continue
            root = y * ntx + x
            stack = [(y, x)]
            lab[y, x] = root
            xs, ys = [x], [y]
            while stack:
                cy, cx = stack.pop()
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        ny, nx = cy + dy, cx + dx
                        if 0 <= ny < nty and 0 <= nx < ntx and mask[ny, nx] and lab[ny, nx] < 0:
                            lab[ny, nx] = root
                            stack.append((ny, nx))
                            xs.append(nx)
                            ys.append(ny)
            boxes.append((min(ys) * T, min(xs) * T, root,
                          [min(xs) * T, min(ys) * T, (max(xs) + 1) * T, (max(ys) + 1) * T]))
    boxes.sort(key=lambda b: (b[0], b[1], b[2]))
    return [b[3] for b in boxes], lab


MODE_PERIODIC = 0
MODE_NONPERIODIC = 1


def candidates(cube: np.ndarray, T: int, mode: int) -> Dict:
    """S8 on a tLISI cube [S, nty, ntx]: scores, threshold (5 sigma periodic,
    4 sigma non-periodic; Sections 2 and 6.3), candidate mask, boxes."""
    S, nty, ntx = cube.shape
    if mode == MODE_PERIODIC:
        sc = periodic_scores(cube)
        k = 5.0
    elif mode == MODE_NONPERIODIC:
        sc = nonperiodic_scores(cube)
        k = 4.0
    else:
        raise ValueError(mode)
    thr, mu, sd = threshold(sc, k)
    mask = (sc > thr).reshape(nty, ntx)
    boxes, lab = connected_boxes(mask, T)
    return dict(scores=sc.reshape(nty, ntx), threshold=thr, mean=mu, std=sd,
                mask=mask, boxes=boxes)
