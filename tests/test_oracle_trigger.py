"""Pins of the oracle's FITrig steps: tLISI invariants (its formula is a
stated stand-in, so parity against the paper is unpinned) and the candidate
search (Sections 2, 6.2, 6.3) against planted cubes, an independent FFT and
hand-made masks."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import toi_oracle as O


# --------------------------------------------------------------- tLISI -----

def _imgs(seed, N=64):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=(N, N)) for _ in range(3)]


def test_tlisi_identical_differences_is_one():
    a, b, _ = _imgs(1)
    I0, I1 = a, a + b
    I2 = I1 + b                     # D_a == D_b
    assert np.allclose(O.tlisi(I0, I1, I2, 16), 1.0, atol=1e-15)


def test_tlisi_range_reversal_scale():
    I0, I1, I2 = _imgs(2)
    t = O.tlisi(I0, I1, I2, 16)
    assert t.min() >= 0.0 and t.max() <= 1.0
    # time reversal swaps and negates the two differences: same tLISI
    assert np.allclose(O.tlisi(I2, I1, I0, 16), t, atol=1e-14)
    # scale invariance (C1, C2 scale with L^2)
    assert np.allclose(O.tlisi(3 * I0, 3 * I1, 3 * I2, 16), t, atol=1e-13)
    # a steady image that leaves the dynamic range unchanged changes nothing
    C = np.random.default_rng(3).uniform(-0.5, 0.5, size=I0.shape)
    C[0, 0] = 0.0
    big = np.zeros_like(I0)
    big[0, 0] = 100.0
    ref = O.tlisi(I0 + big, I1 + big, I2 + big, 16)
    assert np.allclose(O.tlisi(I0 + big + C, I1 + big + C, I2 + big + C, 16), ref, atol=1e-13)


def test_tlisi_transient_tile_low_quiet_tiles_stable():
    """A source switching on in one tile lowers that tile only; the quiet
    tiles' values do not depend on how bright the transient is (Section 2:
    the variation is confined to tiles that contain the transient)."""
    N, T = 64, 16
    rng = np.random.default_rng(4)
    sky = np.zeros((N, N))
    sky[50, 50] = 10.0                          # bright steady source sets L
    noise = [rng.normal(size=(N, N)) * 1e-3 for _ in range(3)]
    out = []
    for amp in (0.5, 2.0):
        I0 = sky + noise[0]
        I1 = sky + noise[1]
        I2 = sky + noise[2]
        I2 = I2.copy()
        I2[5:9, 20:24] += amp                   # transient turns on in tile (0, 1)
        out.append(O.tlisi(I0, I1, I2, T))
    a, b = out
    assert a[0, 1] < 0.9 and b[0, 1] < a[0, 1]
    quiet = np.ones_like(a, bool)
    quiet[0, 1] = False
    assert np.array_equal(a[quiet], b[quiet])
    assert a[quiet].min() > 0.999


def test_tlisi_hand_example_2x2_tiles():
    """4x4 image, 2x2 tiles, exact rationals: tile (0,0) holds a = (1,0,0,0),
    b = (0,1,0,0); L = 2 from another tile."""
    Da = np.zeros((4, 4))
    Db = np.zeros((4, 4))
    Da[0, 0] = 1
    Db[0, 1] = 1
    Da[3, 3] = 2
    I0 = np.zeros((4, 4))
    I0[2, 2] = -3.0                     # image range L = 3 (from I0)
    I1 = I0 + Da
    I2 = I1 + Db
    t = O.tlisi(I0, I1, I2, 2)
    n = Fraction(4)
    mua, mub = Fraction(1, 4), Fraction(1, 4)
    va = Fraction(1) / n - mua * mua
    vb = Fraction(1) / n - mub * mub
    cab = Fraction(0) / n - mua * mub
    L = Fraction(3)
    C1 = (Fraction(1, 100) * L) ** 2
    C2 = (Fraction(3, 100) * L) ** 2
    S = ((2 * mua * mub + C1) * (2 * cab + C2)) / ((mua ** 2 + mub ** 2 + C1) * (va + vb + C2))
    assert t[0, 0] == pytest.approx(float((1 + S) / 2), rel=1e-14)


# ---------------------------------------------------------- candidates -----

def test_twiddles_match_libm():
    for S in (1, 2, 3, 7, 40, 118, 1498):
        c, s = O.twiddle_table(S)
        m = np.arange(S)
        assert np.abs(c - np.cos(2 * np.pi * m / S)).max() < 2e-15
        assert np.abs(s - np.sin(2 * np.pi * m / S)).max() < 2e-15


@pytest.mark.parametrize("S", [37, 38, 40])
def test_periodogram_matches_fft(S):
    """P_f of the fixed-order DFT equals |rfft|^2 of the mean-removed series
    (odd S: every frequency on its own; even S: f and S/2 - f together, S/2
    odd or even)."""
    rng = np.random.default_rng(10)
    cube = rng.uniform(0.5, 1.0, size=(S, 3, 2)).astype(np.float32)
    S = cube.shape[0]
    x = cube.reshape(S, -1).astype(np.float64)
    x = x - x.mean(0)
    P_ref = np.abs(np.fft.rfft(x, axis=0)) ** 2
    # recompute the oracle's P via its public scores path: harmonic h=1 max
    best1 = P_ref[1:S // 2 + 1].max(0)
    sc = O.periodic_scores(cube)
    assert np.all(sc >= best1 * (1 - 1e-12))
    # with h in {1,2,4,8}, the score is the max over normalised harmonic sums
    F = S // 2
    ref = np.zeros(x.shape[1])
    for f in range(1, F + 1):
        for h in (1, 2, 4, 8):
            idx = [i * f for i in range(1, h + 1) if i * f <= F]
            ref = np.maximum(ref, P_ref[idx].sum(0) / math.sqrt(h))
    assert np.allclose(sc, ref, rtol=1e-11)


def test_periodic_score_at_the_highest_frequency():
    """A series alternating 5/8, 3/8 over an even S puts all its power at
    f = F = S/2: x_t - mean = (-1)^t / 8, so A_F = S/8, B_F = 0 and every other
    P_f = 0.  The best harmonic sum is then h = 1 at f = F, score (S/8)^2,
    exact in binary64 (the twiddles there are exactly +-1 and 0)."""
    S = 40
    t = np.arange(S)
    series = np.where(t % 2 == 0, 0.625, 0.375).astype(np.float32)
    cube = np.repeat(series[:, None, None], 6, axis=1).reshape(S, 2, 3)
    assert np.all(O.periodic_scores(cube) == (S / 8.0) ** 2)


def test_pairwise_sum_tree():
    a = [1e16, 1.0, -1e16, 1.0]
    # ((1e16 + 1) + (-1e16 + 1)) with binary64 rounding
    assert O.pairwise_sum(a) == (1e16 + 1.0) + (-1e16 + 1.0)
    # an odd count splits below the middle: 1 + (1e16 - 1e16) = 1, where the
    # other split would round 1 + 1e16 to 1e16 and give 0
    assert O.pairwise_sum([1.0, 1e16, -1e16]) == 1.0
    rng = np.random.default_rng(11)
    v = rng.normal(size=1001)
    assert O.pairwise_sum(v) == pytest.approx(math.fsum(v), abs=1e-12)
    assert O.pairwise_sum([]) == 0.0


def _planted_cube(S=120, nty=8, ntx=8, seed=12):
    rng = np.random.default_rng(seed)
    cube = (1.0 - np.abs(rng.normal(scale=0.02, size=(S, nty, ntx)))).astype(np.float32)
    return cube


def test_periodic_planted_tile_found():
    """A 40-snapshot square wave in tile (5, 2) and its 8-neighbour (6, 3)
    is the only candidate; one merged box."""
    cube = _planted_cube(nty=16, ntx=16)
    S = cube.shape[0]
    on = (np.arange(S) % 40) < 20
    cube[on, 5, 2] -= 0.3
    cube[on, 6, 3] -= 0.28
    r = O.candidates(cube, 32, O.MODE_PERIODIC)
    assert r["mask"].sum() == 2
    assert r["boxes"] == [[2 * 32, 5 * 32, 4 * 32, 7 * 32]]
    assert r["threshold"] == r["mean"] + 5.0 * r["std"]


def test_nonperiodic_dip_found():
    """A 10-snapshot drop in tile (1, 6) gives the only non-periodic candidate."""
    cube = _planted_cube(S=74)
    cube[30:40, 1, 6] -= 0.4
    r = O.candidates(cube, 32, O.MODE_NONPERIODIC)
    assert r["mask"].sum() == 1
    assert r["boxes"] == [[6 * 32, 1 * 32, 7 * 32, 2 * 32]]
    assert r["threshold"] == r["mean"] + 4.0 * r["std"]      # Section 6.3: 4 sigma


def test_connected_boxes_by_hand():
    m = np.zeros((6, 7), bool)
    m[0, 5] = m[1, 6] = True            # diagonal pair -> one component
    m[3, 1] = m[3, 2] = m[4, 2] = True  # L shape
    m[5, 0] = True                      # touches (4, 1)? no: (4,1) is False
    boxes, lab = O.connected_boxes(m, 4)
    assert boxes == [[20, 0, 28, 8], [4, 12, 12, 20], [0, 20, 4, 24]]
    assert lab[1, 6] == 0 * 7 + 5 and lab[4, 2] == 3 * 7 + 1


def test_threshold_by_hand():
    """Reading c11, population moments: scores 1, 2, 3, 4 have mean 5/2 and
    variance 5/4, so thr = 5/2 + k sqrt(5/4) (every step exact in binary64
    but the square root)."""
    thr, mu, sd = O.threshold(np.array([1.0, 2.0, 3.0, 4.0]), 5.0)
    assert mu == 2.5 and sd == math.sqrt(1.25)
    assert thr == 2.5 + 5.0 * math.sqrt(1.25)


def test_threshold_strict_and_flat():
    sc = np.ones(16)
    thr, mu, sd = O.threshold(sc, 5.0)
    assert thr == 1.0 and sd == 0.0
    assert not (sc > thr).any()
    # a flat cube has no outlier: every tile's score equals the threshold
    # (16 equal scores sum exactly), and a candidate must exceed it
    flat = np.full((12, 4, 4), 0.9, np.float32)
    for mode in (O.MODE_PERIODIC, O.MODE_NONPERIODIC):
        r = O.candidates(flat, 32, mode)
        assert r["std"] == 0.0 and r["mask"].sum() == 0 and r["boxes"] == []
