"""Pins of the oracle's near-coplanar (3-D) mode (Section 3.4, Appendix B):
the slab and Chebyshev-order rule against the rows of Table 2, t3 against
the sphere constraint of Appendix B.1 and the printed root, the Jacobi-Anger
series against exp(i alpha s), the Chebyshev-moment image against the
brute-force I_D^(3), and the coplanar limit against the 2-D image."""
import math
import os

import numpy as np
import pytest

from oracle import toi_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_chebyshev.txt")


def _table2():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, phi, ns, a, K, nk = line.split()
            rows.append((name, float(phi), int(ns), float(a), int(K), int(nk)))
    return rows


@pytest.mark.parametrize("row", _table2(), ids=lambda r: r[0])
def test_table2_rows(row):
    name, phi, n_slab, alpha_slab, K, nk = row
    t3max = 1e-3                               # any t3max: the rule depends on Phi_max only
    span = phi / (math.pi * t3max)             # r3max - r3min giving this Phi_max
    plan = O.slab_plan(-0.3 * span, 0.7 * span, t3max)
    assert plan["phi_max"] == pytest.approx(phi, rel=1e-12)
    assert plan["n_slab"] == n_slab
    assert round(plan["alpha_slab"], 2) == alpha_slab
    assert plan["K"] == K
    assert plan["n_slab"] * plan["K"] == nk


def _random_V(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    V = q.T
    if V[2, 2] < 0:
        V[2] = -V[2]
    if np.linalg.det(V) < 0:
        V[1] = -V[1]
    return V


def test_t3_lies_on_the_sphere_and_matches_the_printed_root():
    rng = np.random.default_rng(1)
    for _ in range(20):
        V = _random_V(rng)
        if abs(V[2, 2]) < 0.8:      # keep every sampled (t1, t2) on the visible sphere
            continue
        t1 = rng.uniform(-0.05, 0.05, 50)
        t2 = rng.uniform(-0.05, 0.05, 50)
        t3 = O.t3_of(t1, t2, V)
        # Eqs. B1-B3: (l, m, n - 1) = V^T (t1, t2, t3)
        l = V[0, 0] * t1 + V[1, 0] * t2 + V[2, 0] * t3
        m = V[0, 1] * t1 + V[1, 1] * t2 + V[2, 1] * t3
        n = 1.0 + V[0, 2] * t1 + V[1, 2] * t2 + V[2, 2] * t3
        assert np.abs(l * l + m * m + n * n - 1.0).max() < 1e-13
        assert np.all(n > 0)                               # the visible hemisphere
        printed = -V[2, 2] + np.sign(V[2, 2]) * np.sqrt(
            1 - (t1 + V[0, 2]) ** 2 - (t2 + V[1, 2]) ** 2)
        assert np.abs(t3 - printed).max() < 1e-12
        assert O.t3_of(0.0, 0.0, V) == 0.0


def test_jacobi_anger_series():
    a = np.linspace(0.0, 10.0, 41)
    s = np.linspace(-1.0, 1.0, 33)
    approx = np.einsum("ak,sk->as", O.chebyshev_coeffs(a, 32), O.chebyshev_T(s, 32))
    assert np.abs(approx - np.exp(1j * a[:, None] * s[None, :])).max() < 1e-12
    # T_k(cos d) = cos(k d)
    d = np.linspace(0, np.pi, 17)
    assert np.abs(O.chebyshev_T(np.cos(d), 9) - np.cos(np.arange(9)[None, :] * d[:, None])).max() < 1e-13


def _noncoplanar_case(rng, N=64, cell=60.0, n=400, r3_span=4000.0):
    """Random R coordinates inside the gridder's reach with a wide r3 spread,
    point-source-like values, and a tilted basis V."""
    beta = cell * O.ARCSEC
    G = 2 * N
    lim = (G / 2 - 6) / (beta * G)
    r = np.stack([rng.uniform(-lim, lim, n), rng.uniform(-lim, lim, n),
                  rng.uniform(-0.5 * r3_span, 0.5 * r3_span, n)], 1)
    V = _random_V(rng)
    while abs(V[2, 2]) < 0.8:
        V = _random_V(rng)
    c = np.exp(-2j * np.pi * (r[:, 0] * 3 * beta + r[:, 1] * -5 * beta)) + 0.3 * (
        rng.normal(size=n) + 1j * rng.normal(size=n))
    return r, c, V


def test_moment_image_matches_the_exact_3d_dft():
    rng = np.random.default_rng(3)
    N, cell = 64, 60.0
    r, c, V = _noncoplanar_case(rng, N, cell)
    ref = O.dirty_image_3d_dft(r, c, N, cell, V, 1.0, float(len(c)))
    scale = np.abs(c).sum() / len(c)
    t = O.tilted_image_3d(r, c, N, cell, V, 1.0, float(len(c)), K=32)
    assert t["plan"]["n_slab"] > 1
    assert np.abs(t["tilted"] - ref).max() < 1e-6 * scale
    # with the automatic order the error stays within the sampled bound
    ta = O.tilted_image_3d(r, c, N, cell, V, 1.0, float(len(c)))
    bound = 2.0 * ta["plan"]["err"] * scale + 1e-6 * scale
    assert np.abs(ta["tilted"] - ref).max() < bound
    # and the 2-D image is far from it (the residual phase matters here)
    two_d = O.dirty_image_dft(r[:, 0], r[:, 1], c, N, cell, 1.0, float(len(c)))
    assert np.abs(two_d - ref).max() > 100 * np.abs(t["tilted"] - ref).max()


def test_coplanar_limit_equals_the_2d_image():
    rng = np.random.default_rng(4)
    N, cell = 64, 60.0
    r, c, V = _noncoplanar_case(rng, N, cell)
    r[:, 2] = 0.0
    t = O.tilted_image_3d(r, c, N, cell, V, 1.0, float(len(c)))
    g1, g2 = O.grid_coords(r[:, 0], r[:, 1], N, cell)
    grid = O.grid_es(g1, g2, c, 2 * N, 8, O.es_beta(8))
    two_d = O.tilted_image(grid, N, 8, O.es_beta(8), 1.0, float(len(c)))
    assert t["plan"]["n_slab"] == 1 and t["plan"]["dr3"] == 0.0
    assert np.abs(t["tilted"] - two_d).max() < 1e-12 * np.abs(two_d).max()


def test_slab_assignment():
    plan = O.slab_plan(-100.0, 300.0, 0.01)
    r3 = np.linspace(-100.0, 300.0, 1001)
    p, s = O.slab_of(r3, plan)
    assert p.min() == 0 and p.max() == plan["n_slab"] - 1
    assert np.all(np.abs(s) <= 1.0 + 1e-12)
    assert np.allclose(plan["centres"][p] + s * plan["dr3"], r3)
