"""Pins for the oracle's gain estimation (reading C15).

The paper says only that a gain the user does not supply is estimated at
each iteration, and names a sigma-clipping helper; it prints no formula.
The oracle's reading: photon transfer on adjacent pixel pairs (columns 2m,
2m+1) of the iteration's image, both pixels unflagged and unsaturated, with
the pair differences d sigma-clipped at 3 population standard deviations
(exact integer test, at most 5 rounds, mean as centre) and the gain the
positive root of V g^2 - A g - 2 n rn^2 = 0 (V = sum (d - mean d)^2,
A = sum (a + b)).  The pins check it against things other than itself:
scipy's sigma clipping, the exact 3-sigma boundary worked out by hand, the
gain that truncated-normal moments predict on synthetic Poisson frames,
the undefined cases and invariants of the pair selection.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.stats import norm

import oracle


def _pairs_image(d: np.ndarray, base: int = 1000):
    """Image and mask whose unflagged pairs (columns 2m, 2m+1) are base + d, base."""
    d = np.asarray(d, np.int64)
    n = len(d)
    width = 64
    rows = -(-n // width)
    I = np.full((rows, 2 * width), float(base), np.float32)
    flat_a = I[:, 0::2].reshape(-1)
    flat_a[:n] = base + d
    I[:, 0::2] = flat_a.reshape(rows, width)
    M = np.zeros(I.shape, np.uint8)
    # pairs beyond n are excluded by flagging their first pixel
    Mv = M[:, 0::2].reshape(-1)
    Mv[n:] = 1
    M[:, 0::2] = Mv.reshape(rows, width)
    return I, M


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_clipping_keeps_what_scipy_sigmaclip_keeps(seed):
    # A bounded core (uniform integers, whose 3-sigma bound lies outside
    # their range) with wide outliers converges in a few rounds, so scipy's
    # loop without a round limit keeps the same set.
    rng = np.random.default_rng(seed)
    w = 3 + 4 * seed
    d = rng.integers(-w, w + 1, 3000)
    out = rng.choice(3000, 40, replace=False)
    d[out] += rng.integers(-900, 900, 40)
    I, M = _pairs_image(d)
    g, rounds, (n, s1, s2, a) = oracle.estimate_gain(I, M, np.zeros_like(M), 3.0)
    assert rounds < 5, "the case must converge for scipy's unbounded loop to be comparable"
    kept = stats.sigmaclip(d.astype(np.float64), 3.0, 3.0).clipped.astype(np.int64)
    assert n == len(kept)
    assert s1 == int(kept.sum()) and s2 == int((kept * kept).sum())
    assert a == int((2000 + kept).sum())
    assert g is not None and g > 0


def test_clipping_boundary_is_inclusive_and_exact():
    # Nine zeros and one x: (10x - x)^2 = 81 x^2 = 9 (10 x^2 - x^2), so x lies
    # exactly 3 population standard deviations from the mean and is kept.
    I, M = _pairs_image(np.array([0] * 9 + [7]))
    g, rounds, (n, s1, s2, a) = oracle.estimate_gain(I, M, np.zeros_like(M), 0.0)
    assert (n, s1, s2, rounds) == (10, 7, 49, 1)
    # Nineteen zeros and one x: (20x - x)^2 = 361 x^2 > 9 (20 x^2 - x^2) = 171 x^2.
    I, M = _pairs_image(np.array([0] * 19 + [7]))
    g, rounds, (n, s1, s2, a) = oracle.estimate_gain(I, M, np.zeros_like(M), 0.0)
    assert (n, s1, s2) == (19, 0, 0)
    assert g is None  # the survivors are all equal: V = 0


def test_gain_closed_forms():
    # Pairs (1, 0) and (0, 1), rn = 1: n = 2, d = +-1, V = 2, A = 2, so
    # 2 g^2 - 2 g - 2*2*1 = 0, i.e. (g - 2)(g + 1) = 0: g = 2 exactly.
    I = np.array([[1, 0, 0, 1]], np.float32)
    z = np.zeros(I.shape, np.uint8)
    g, rounds, st = oracle.estimate_gain(I, z, z, 1.0)
    assert st == (2, 0, 2, 2) and g == 2.0
    # Without read noise g = A / V: four pairs 101/100 alternating, V = 4, A = 804.
    I = np.array([[101, 100, 100, 101, 101, 100, 100, 101]], np.float32)
    z = np.zeros(I.shape, np.uint8)
    g, rounds, st = oracle.estimate_gain(I, z, z, 0.0)
    assert st == (4, 0, 4, 804) and g == 201.0


def test_clipping_stops_after_five_rounds():
    # 100 zero differences and outliers 2, 10, 50, 250, 1250, 6250, 31250
    # (ratio 5): in each round the largest survivor dominates the variance,
    # sigma ~ a_max / sqrt(n) ~ a_max / 10, so it alone lies beyond 3 sigma
    # (~0.3 a_max) while the next one (a_max / 5) stays inside.  One outlier
    # goes per round; after the fifth round {0 x 100, 2, 10} remain (n 102,
    # sum 12, sum of squares 104), although a sixth and seventh round would
    # still drop 10 and 2.
    I, M = _pairs_image(np.array([0] * 100 + [2, 10, 50, 250, 1250, 6250, 31250]))
    g, rounds, st = oracle.estimate_gain(I, M, np.zeros_like(M), 2.0)
    assert rounds == 5
    assert st == (102, 12, 104, 102 * 2000 + 12)
    assert g is not None


def _clip_variance_factor(rounds: int) -> float:
    """Variance of a unit normal after `rounds` progressive 3-sigma clips."""
    t, var = np.inf, 1.0
    for _ in range(rounds):
        t = min(t, 3.0 * np.sqrt(var))
        var = 1.0 - 2.0 * t * norm.pdf(t) / (2.0 * norm.cdf(t) - 1.0)
    return var


def _predicted_gain(g, rn, mu, rounds):
    # per pixel, in ADU^2: Poisson electrons / g^2, read noise, rounding to integers
    var_pix = mu / g + rn ** 2 / g ** 2 + 1.0 / 12.0
    V = _clip_variance_factor(rounds) * 2.0 * var_pix
    A = 2.0 * mu
    return (A + np.sqrt(A * A + 8.0 * rn ** 2 * V)) / (2.0 * V)


@pytest.mark.parametrize("g,rn,mu", [(2.0, 5.0, 1000.0), (0.5, 3.0, 200.0), (4.0, 20.0, 100.0),
                                     (1.0, 2.0, 5000.0), (8.0, 40.0, 30.0)])
def test_recovers_the_gain_of_synthetic_poisson_frames(g, rn, mu):
    # Photon transfer: the estimate matches what the model predicts after the
    # clipping's truncation (about +3%) within 1%; the statistical error of
    # 262144 pairs is about 0.3%.  Read-noise-dominated cases fail a dropped
    # or mis-scaled rn term; the bright case fails a wrong A.
    rng = np.random.default_rng(int(g * 100 + rn))
    e = rng.poisson(g * mu, (1024, 1024)) + rng.normal(0.0, rn, (1024, 1024))
    I = np.clip(np.rint(e / g), 0, 65535).astype(np.float32)
    z = np.zeros(I.shape, np.uint8)
    est, rounds, _ = oracle.estimate_gain(I, z, z, rn)
    assert abs(est / _predicted_gain(g, rn, mu, rounds) - 1.0) < 0.01
    # and the unclipped model is off by the truncation, so the clip matters
    assert abs(est / _predicted_gain(g, rn, mu, 0) - 1.0) > 0.01


def test_flagged_or_saturated_partner_removes_the_pair():
    rng = np.random.default_rng(7)
    I = np.rint(rng.normal(500.0, 25.0, (64, 96))).astype(np.float32)
    gone = (4, 5, 30, 31, 60, 61, 70, 71)
    kept_cols = [c for c in range(96) if c not in gone]
    z = np.zeros((64, 96 - len(gone)), np.uint8)
    ref = oracle.estimate_gain(I[:, kept_cols], z, z, 4.0)
    M = np.zeros(I.shape, np.uint8)
    sat = np.zeros(I.shape, np.uint8)
    M[:, 4] = 1     # the first pixel of pair (4, 5) flagged
    M[:, 61] = 1    # the second pixel of pair (60, 61) flagged
    sat[:, 31] = 1  # the second pixel of pair (30, 31) saturated
    sat[:, 70] = 1  # the first pixel of pair (70, 71) saturated
    assert oracle.estimate_gain(I, M, sat, 4.0) == ref


def test_undefined_estimates():
    z = np.zeros((8, 9), np.uint8)
    const = np.full((8, 9), 300.0, np.float32)
    assert oracle.estimate_gain(const, z, z, 2.0)[0] is None           # V = 0
    one_col = np.arange(8, dtype=np.float32).reshape(8, 1)
    assert oracle.estimate_gain(one_col, np.zeros((8, 1), np.uint8), np.zeros((8, 1), np.uint8), 2.0)[0] is None
    noisy = np.arange(72, dtype=np.float32).reshape(8, 9) % 7
    assert oracle.estimate_gain(noisy, np.ones((8, 9), np.uint8), z, 2.0)[0] is None  # all flagged
    with pytest.raises(ValueError):
        oracle.estimate_gain(noisy + 0.5, z, z, 2.0)                     # not integer ADU


def test_undefined_estimate_runs_with_unit_gain():
    f = np.full((40, 50), 120, np.uint16)
    f[10, 10] = 4000
    m0, c0, it0, nf0, g0, ok0 = oracle.run(f, 0.0, 3.0, niter=3, return_gain=True)
    m1, c1, it1, nf1 = oracle.run(f, 1.0, 3.0, niter=3)
    assert not ok0 and g0 == 1.0
    assert np.array_equal(m0, m1) and np.array_equal(c0.view(np.uint32), c1.view(np.uint32))
    assert (it0, nf0) == (it1, nf1)


def test_run_estimates_the_gain_at_every_iteration():
    # The loop with gain 0 equals iterations driven by hand, each with the
    # estimate from that iteration's image and the mask so far.
    rng = np.random.default_rng(11)
    e = rng.poisson(2.0 * 400.0, (96, 128)) + rng.normal(0.0, 6.0, (96, 128))
    f = np.clip(np.rint(e / 2.0), 0, 65535).astype(np.uint16)
    ys, xs = rng.integers(0, 96, 60), rng.integers(0, 128, 60)
    f[ys, xs] = np.minimum(65535, f[ys, xs].astype(np.int64) + rng.integers(300, 3000, 60)).astype(np.uint16)
    m, c, it, nf, g_last, ok = oracle.run(f, 0.0, 6.0, niter=4, return_gain=True)
    assert ok and it >= 2
    x0, sat = oracle.ingest(f, 65535.0)
    I, M = x0.copy(), np.zeros(f.shape, np.uint8)
    for k in range(1, 5):
        g, _, _ = oracle.estimate_gain(I, M, sat, 6.0)
        gk = float(np.float32(g))
        fresh, I, M, _ = oracle.iterate(x0, sat, I, M, gk, 6.0, 4.5, 0.3, 5.0)
        if fresh == 0:
            break
    assert k == it and gk == g_last
    assert np.array_equal(M, m) and np.array_equal(I.view(np.uint32), c.view(np.uint32))


def test_estimation_needs_a_uint16_frame():
    with pytest.raises(ValueError):
        oracle.run(np.full((8, 8), 10.0, np.float32), 0.0, 2.0)
    with pytest.raises(ValueError):
        oracle.run(np.full((8, 8), 10, np.uint16), -1.0, 2.0)
