"""Pins for the CPU oracle, checked against things other than the oracle itself.

The paper (dfcosmic, Methods / "Algorithm") lists the seven L.A.Cosmic steps
without equations and prints no worked numeric example, so every pin here
is one of: brute force with numpy/scipy on tiny frames, closed forms worked
out by hand, hand-derived fixtures under tests/golden/, or invariants of the
method.  Each is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong rank) fails.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view
from scipy import ndimage

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_median(a: np.ndarray, K: int) -> np.ndarray:
    r = K // 2
    p = np.pad(a, r, mode="edge")
    w = sliding_window_view(p, (K, K)).reshape(a.shape[0], a.shape[1], K * K)
    return np.sort(w, axis=-1)[..., (K * K - 1) // 2]


def literal_lplus(a: np.ndarray) -> np.ndarray:
    """Replicate 2x, convolve with the Laplacian, clip at 0, 2x2 block average (scipy)."""
    rep = np.repeat(np.repeat(a, 2, axis=0), 2, axis=1)
    k = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], dtype=a.dtype)
    conv = ndimage.convolve(rep, k, mode="nearest")
    conv = np.clip(conv, 0, None)
    ny, nx = a.shape
    return conv.reshape(ny, 2, nx, 2).mean(axis=(1, 3)).astype(a.dtype)


SHAPES = [(1, 1), (1, 5), (5, 1), (2, 3), (7, 7), (13, 9), (20, 17)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("K", [3, 5, 7])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_median_matches_full_sort(shape, K, precision):
    rng = np.random.default_rng(hash((shape, K)) % 2**32)
    T = np.float32 if precision == "f32" else np.float64
    for trial in range(3):
        if trial == 0:
            a = rng.normal(size=shape).astype(T)
        elif trial == 1:
            a = rng.integers(0, 4, size=shape).astype(T)  # many ties
        else:
            a = np.full(shape, 7.25, T)  # constant -> the constant
        got = oracle.median(a, K, precision)
        np.testing.assert_array_equal(got, brute_median(a, K))
        if trial == 2:
            assert np.all(got == T(7.25))


def test_median_is_a_rank_selection_not_a_mean():
    # 3x3 window with values 0..8 permuted: the median is 4, the mean also 4;
    # a skewed set separates them.
    a = np.array([[0, 0, 0], [0, 0, 100], [100, 100, 100]], np.float32)
    assert oracle.median(a, 3)[1, 1] == 0.0  # five zeros among nine


@pytest.mark.parametrize("shape", [(1, 1), (1, 6), (6, 1), (8, 8), (13, 9), (31, 40)])
def test_lplus_literal_pipeline_bit_exact_on_integers(shape):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    a = rng.integers(0, 65536, size=shape).astype(np.float32)
    fused = oracle.lplus(a)
    np.testing.assert_array_equal(fused, literal_lplus(a))
    np.testing.assert_array_equal(oracle.lplus(a, literal=True), literal_lplus(a))


def test_lplus_literal_pipeline_close_on_floats():
    rng = np.random.default_rng(3)
    a = (100 + 10 * rng.standard_normal((40, 33))).astype(np.float32)
    np.testing.assert_allclose(oracle.lplus(a), literal_lplus(a), rtol=0, atol=1e-3)
    a64 = a.astype(np.float64)
    np.testing.assert_allclose(oracle.lplus(a64, precision="f64"), literal_lplus(a64),
                               rtol=1e-12, atol=1e-9)


def test_lplus_closed_forms():
    # Constant -> 0.
    assert np.all(oracle.lplus(np.full((9, 11), 42.0, np.float32)) == 0)
    # Horizontal ramp I = alpha * j: interior L+ = |alpha| / 2.
    for alpha in (2.0, -6.0, 10.0):
        a = (alpha * np.arange(12, dtype=np.float32))[None, :].repeat(7, 0)
        L = oracle.lplus(a)
        assert np.all(L[:, 1:-1] == abs(alpha) / 2)
    # Vertical ramp: same by symmetry.
    a = (4.0 * np.arange(10, dtype=np.float32))[:, None].repeat(6, 1)
    assert np.all(oracle.lplus(a)[1:-1, :] == 2.0)
    # Delta of amplitude A on zero: 2A at the hit, 0 at every other pixel.
    a = np.zeros((9, 9), np.float32)
    a[4, 4] = 37.0
    L = oracle.lplus(a)
    assert L[4, 4] == 74.0
    L[4, 4] = 0
    assert np.all(L == 0)


def test_rebin_of_replicate_is_identity():
    rng = np.random.default_rng(11)
    x = rng.normal(size=(6, 5))
    rep = np.repeat(np.repeat(x, 2, 0), 2, 1)
    np.testing.assert_array_equal(rep.reshape(6, 2, 5, 2).mean(axis=(1, 3)), x)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 5), (12, 9)])
def test_dilation_matches_scipy(shape):
    rng = np.random.default_rng(shape[0] + 7 * shape[1])
    b = (rng.uniform(size=shape) < 0.15).astype(np.uint8)
    ref = ndimage.binary_dilation(b, structure=np.ones((3, 3), bool), border_value=0)
    np.testing.assert_array_equal(oracle.dilate3(b), ref.astype(np.uint8))


def brute_maskmed(x0, M, i, j):
    ny, nx = x0.shape
    for r in range(2, max(ny, nx) + 3):
        ys = np.clip(np.arange(i - r, i + r + 1), 0, ny - 1)
        xs = np.clip(np.arange(j - r, j + r + 1), 0, nx - 1)
        vals = [x0[y, x] for y in ys for x in xs if not M[y, x]]
        if vals:
            vals.sort()
            return vals[(len(vals) - 1) // 2]
    return None


def test_maskmed_brute_force_random():
    rng = np.random.default_rng(21)
    for trial in range(40):
        ny, nx = rng.integers(1, 12, 2)
        x0 = rng.integers(0, 9, size=(ny, nx)).astype(np.float32)
        M = (rng.uniform(size=(ny, nx)) < rng.uniform(0.1, 0.9)).astype(np.uint8)
        if M.all():
            M[0, 0] = 0
        for i in range(ny):
            for j in range(nx):
                assert oracle.maskmed(x0, M, i, j) == brute_maskmed(x0, M, i, j)


def test_maskmed_widening_on_flagged_block():
    # A 7x7 flagged block: its centre's 5x5 and 7x7 windows are fully flagged,
    # so the pool is the 9x9 ring of 32 unflagged pixels (values 1..32): the
    # lower median of 32 values is the 16th smallest, 16.
    x0 = np.zeros((15, 15), np.float32)
    M = np.zeros((15, 15), np.uint8)
    M[4:11, 4:11] = 1
    ring = [(y, x) for y in range(3, 12) for x in range(3, 12)
            if max(abs(y - 7), abs(x - 7)) == 4]
    assert len(ring) == 32
    perm = np.random.default_rng(0).permutation(32)
    for (y, x), v in zip(ring, perm + 1):
        x0[y, x] = v
    assert oracle.maskmed(x0, M, 7, 7) == 16.0
    # Even count -> lower median; odd count -> middle.
    x0 = np.arange(25, dtype=np.float32).reshape(5, 5)
    M = np.zeros((5, 5), np.uint8)
    M[2, 2] = 1  # pool at the centre = 24 values {0..24}\{12}: lower median 11
    assert oracle.maskmed(x0, M, 2, 2) == 11.0


def _load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_golden_single_hit(precision):
    """Hand-derived: flat sky s with one hit A; closed forms for N, S, S', F, the mask."""
    gd = _load_golden("single_hit.json")
    s, A, g, rn = gd["sky"], gd["amp"], gd["gain"], gd["readnoise"]
    ny, nx = gd["shape"]
    cy, cx = gd["hit"]
    T = np.float32 if precision == "f32" else np.float64
    x0 = np.full((ny, nx), s, T)
    x0[cy, cx] += A
    sat = np.zeros((ny, nx), np.uint8)
    fresh, I, M, d = oracle.iterate(x0, sat, x0, np.zeros_like(sat), g, rn, gd["sigclip"],
                                    gd["sigfrac"], gd["objlim"], precision=precision)
    exp = gd["expected"]
    assert d["L"][cy, cx] == exp["L_hit"]
    assert np.all(d["N"] == exp["N"])
    assert d["S"][cy, cx] == exp["S_hit"]
    assert d["Sp"][cy, cx] == exp["Sp_hit"]
    assert np.all(d["F"] == T(exp["F"]))
    assert fresh == 1 and M[cy, cx] == 1 and M.sum() == 1
    assert np.all(I == s)  # the hit is replaced by the sky


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_golden_flat_noise_model(precision):
    gd = _load_golden("flat_noise.json")
    T = np.float32 if precision == "f32" else np.float64
    for case in gd["cases"]:
        x0 = np.full((6, 7), case["sky"], T)
        sat = np.zeros(x0.shape, np.uint8)
        _, I, M, d = oracle.iterate(x0, sat, x0, sat, case["gain"], case["readnoise"], 4.5, 0.3,
                                    5.0, precision=precision)
        assert np.all(d["N"] == case["N"])
        assert np.all(d["S"] == 0) and np.all(d["Sp"] == 0)
        assert np.all(d["F"] == T(0.01))
        assert M.sum() == 0


def _noise_frame(seed, ny=128, nx=128, sky=100.0, gain=1.0, rn=1.5):
    rng = np.random.default_rng(seed)
    sig = math.sqrt(gain * sky + rn * rn) / gain
    return (sky + sig * rng.standard_normal((ny, nx))).astype(np.float32), sig


def test_noise_only_high_sigclip_no_detections():
    from paper_2602_17938_gb300 import synth
    spec = synth.FrameSpec(256, 256, "f32", (77, 0), n_stars=0, n_tracks=0, hot_frac=0.0)
    f = synth.make_frame(spec)
    m, c, it, nf = oracle.run(f, spec.gain, spec.readnoise, sigclip=20.0)
    assert nf == 0 and it == 1
    np.testing.assert_array_equal(c, f)


def test_isolated_hits_recovered_and_replaced_by_sky():
    f, sig = _noise_frame(5)
    rng = np.random.default_rng(6)
    hits = [(y, x) for y in range(8, 120, 16) for x in range(8, 120, 16)]
    for (y, x) in hits:
        f[y, x] += np.float32(rng.uniform(50, 80) * sig)  # A/N >= 10*sigclip
    m, c, it, nf = oracle.run(f, 1.0, 1.5)
    for (y, x) in hits:
        assert m[y, x] == 1
        win = f[y - 2:y + 3, x - 2:x + 3][m[y - 2:y + 3, x - 2:x + 3] == 0]
        assert c[y, x] in set(win.tolist())
        assert abs(c[y, x] - 100.0) < 5 * sig


def test_injected_tracks_recovered():
    # Straight horizontal/vertical/diagonal tracks, amplitude 20-60 sigma.
    f, sig = _noise_frame(8, 192, 192)
    rng = np.random.default_rng(9)
    truth = np.zeros(f.shape, bool)
    for k in range(30):
        y0, x0 = rng.integers(10, 170, 2)
        ln = rng.integers(2, 15)
        dy, dx = [(0, 1), (1, 0), (1, 1), (1, -1)][k % 4]
        amp = np.float32(rng.uniform(20, 60) * sig)
        for t in range(ln):
            y, x = y0 + t * dy, x0 + t * dx
            if 0 <= y < 192 and 0 <= x < 192 and not truth[y, x]:
                truth[y, x] = True
                f[y, x] += amp
    m, c, it, nf = oracle.run(f, 1.0, 1.5)
    recovered = (m.astype(bool) & truth).sum() / truth.sum()
    assert recovered >= 0.95


def test_isolated_stars_not_flagged():
    # Stars of FWHM 2.5 px on a 32-px grid (no blends), peaks log-uniform in
    # [500, 20000] ADU: the objlim test keeps their cores unflagged.
    rng = np.random.default_rng(5)
    f, _ = _noise_frame(5, 256, 256)
    yy, xx = np.mgrid[0:256, 0:256]
    cents = []
    s = 2.5 / 2.3548
    for cy in range(16, 256, 32):
        for cx in range(16, 256, 32):
            y0, x0 = cy + rng.uniform(-.5, .5), cx + rng.uniform(-.5, .5)
            pk = math.exp(rng.uniform(math.log(500), math.log(20000)))
            f += (pk * np.exp(-(((yy + .5) - y0) ** 2 + ((xx + .5) - x0) ** 2)
                              / (2 * s * s))).astype(np.float32)
            cents.append((cy, cx))
    m, c, it, nf = oracle.run(f, 1.0, 1.5)
    for cy, cx in cents:
        assert not m[cy - 3:cy + 4, cx - 3:cx + 4].any()


def test_saturated_pixels_never_flagged():
    f, sig = _noise_frame(12, 96, 96)
    f[20:23, 30:33] = 65535.0  # saturated block
    f[50, 50] = 65535.0  # a saturated "hit"
    f[60, 60] += 80 * sig  # an ordinary hit
    m, c, it, nf = oracle.run(f, 1.0, 1.5, satlevel=65535.0)
    assert not m[20:23, 30:33].any() and m[50, 50] == 0 and m[60, 60] == 1
    assert c[50, 50] == 65535.0
    # satlevel <= 0 disables the protection: the lone saturated spike is flagged.
    m2, *_ = oracle.run(f, 1.0, 1.5, satlevel=0.0)
    assert m2[50, 50] == 1


@pytest.mark.parametrize("r", [0, 1, 2, 3, 4])
def test_saturation_region_is_the_square_dilation(r):
    # Reading C16: the saturated set grown by the (2r+1)^2 square, inside the frame --
    # scipy's binary dilation with that structuring element and a zero border.
    rng = np.random.default_rng(100 + r)
    for shape in [(1, 1), (1, 9), (7, 1), (23, 31), (64, 50)]:
        B = (rng.random(shape) < 0.03).astype(np.uint8)
        B[0, 0] = 1  # a corner seed
        ref = ndimage.binary_dilation(B, structure=np.ones((2 * r + 1, 2 * r + 1), bool)) if r else B
        assert np.array_equal(oracle.dilate_square(B, r), ref.astype(np.uint8)), (shape, r)


def test_satgrow_zero_is_reading_c9():
    f, sig = _noise_frame(13, 96, 96)
    f[20:23, 30:33] = 65535.0
    f[40, 70] += 80 * sig
    a = oracle.run(f, 1.0, 1.5, satlevel=65535.0)
    b = oracle.run(f, 1.0, 1.5, satlevel=65535.0, satgrow=0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2:] == b[2:]


@pytest.mark.parametrize("r", [1, 2, 4])
def test_nothing_flagged_in_the_grown_saturated_region(r):
    rng = np.random.default_rng(7 * r)
    f, sig = _noise_frame(14 + r, 128, 128)
    for _ in range(6):  # saturated star cores
        y, x = rng.integers(8, 120, 2)
        f[y - 1:y + 2, x - 1:x + 2] = 65535.0
    hits = rng.integers(0, 128, (300, 2))
    f[hits[:, 0], hits[:, 1]] += rng.uniform(40, 400, 300) * sig
    sat0 = (f >= 65535.0).astype(np.uint8)
    m, c, it, nf = oracle.run(f, 1.0, 1.5, satlevel=65535.0, satgrow=r)
    grown = ndimage.binary_dilation(sat0, structure=np.ones((2 * r + 1, 2 * r + 1), bool))
    assert not (m.astype(bool) & grown).any()
    assert np.array_equal(c[grown], f[grown])  # never replaced
    assert nf > 0  # hits elsewhere are still found


def test_satgrow_protects_a_hit_next_to_a_saturated_core():
    f, sig = _noise_frame(15, 96, 96)
    f[40:43, 40:43] = 65535.0  # saturated star core
    f[41, 45] += 80 * sig  # an ordinary hit 3 px right of the core's edge column
    m0, *_ = oracle.run(f, 1.0, 1.5, satlevel=65535.0)
    m2, *_ = oracle.run(f, 1.0, 1.5, satlevel=65535.0, satgrow=2)
    m3, *_ = oracle.run(f, 1.0, 1.5, satlevel=65535.0, satgrow=3)
    assert m0[41, 45] == 1 and m2[41, 45] == 1  # distance 3 from the core: outside r = 2
    assert m3[41, 45] == 0


def _sep_median_numpy(A, K):
    r = K // 2
    P = np.pad(A, r, mode="edge")
    # row medians over columns j-r..j+r of every padded row, then medians over rows i-r..i+r
    rm = np.median(sliding_window_view(P, K, axis=1), axis=-1)  # (ny + 2r) x nx
    return np.median(sliding_window_view(rm, K, axis=0), axis=-1)


@pytest.mark.parametrize("K", [3, 5])
def test_separable_median_matches_numpy(K):
    # Reading C17: an independent numpy form (edge padding = clamped coordinates).
    rng = np.random.default_rng(60 + K)
    for shape in [(1, 1), (1, 7), (6, 1), (9, 13), (40, 33)]:
        A = rng.integers(0, 50, shape).astype(np.float32)  # many ties
        assert np.array_equal(oracle.median_sep(A, K), _sep_median_numpy(A, K).astype(np.float32)), shape


def test_separable_median_equals_true_median_on_row_constant_images():
    # A window of an image constant along each row holds each row value K times,
    # so the true median is the median of the row values -- the separable one.
    rng = np.random.default_rng(71)
    a = rng.normal(100, 20, 37).astype(np.float32)
    A = np.repeat(a[:, None], 29, axis=1)
    assert np.array_equal(oracle.median_sep(A, 5), oracle.median(A, 5))
    # and it differs from the true median on a generic image
    B = rng.normal(100, 20, (37, 29)).astype(np.float32)
    assert not np.array_equal(oracle.median_sep(B, 5), oracle.median(B, 5))


def test_sepmed_mode_changes_the_mask_on_star_fields():
    # The comparison mode swaps only the two 5x5 detection medians; on a field
    # of bright Gaussian stars (flat tops clipped at 65535) the two modes give
    # different masks.  (Which one flags more depends on the data: on these
    # synthetic stars the separable mode flags fewer star pixels.)
    from paper_2602_17938_gb300 import synth
    spec = synth.FrameSpec(256, 256, "f32", (17, 3), sky=300.0, gain=1.0, readnoise=3.0,
                           n_stars=40, star_peak=(1e5, 1e6), n_tracks=0, hot_frac=0.0, fwhm=3.5)
    f = np.minimum(synth.make_frame(spec), 65535.0).astype(np.float32)
    m_true, _, _, n_true = oracle.run(f, 1.0, 3.0, satlevel=65535.0)
    m_sep, _, _, n_sep = oracle.run(f, 1.0, 3.0, satlevel=65535.0, sepmed=True)
    assert n_true > 0 and n_sep > 0 and not np.array_equal(m_true, m_sep)
    assert not (m_sep.astype(bool) & (f >= 65535.0)).any()  # saturated pixels stay protected


def _config0():
    from paper_2602_17938_gb300 import synth
    spec = synth.config_specs(0)[0]
    return spec, synth.make_frame(spec)


def test_invariants_on_config0():
    spec, f = _config0()
    m, c, it, nf = oracle.run(f, spec.gain, spec.readnoise, niter=4)
    assert nf == m.sum() > 0
    np.testing.assert_array_equal(c[m == 0], f[m == 0])  # cleaned == input outside M
    x0 = f.astype(np.float32)
    ys, xs = np.nonzero(m)
    for y, x in list(zip(ys, xs))[::7]:  # cleaned value is an unflagged window member
        assert c[y, x] == brute_maskmed(x0, m, y, x)


def test_mask_monotone_early_stop_exact_and_niter0_identity():
    spec, f = _config0()
    x0, sat = oracle.ingest(f, spec.satlevel)
    I, M = x0.copy(), np.zeros(f.shape, np.uint8)
    history = []
    for k in range(6):
        fresh, I, Mn, _ = oracle.iterate(x0, sat, I, M, spec.gain, spec.readnoise, 4.5, 0.3, 5.0)
        assert np.all(Mn >= M)  # monotone
        assert fresh == int((Mn > M).sum())
        M = Mn
        history.append((fresh, M.copy(), I.copy()))
    # Once an iteration finds nothing new, every later iteration is identical.
    first_zero = next(k for k, h in enumerate(history) if h[0] == 0)
    for k in range(first_zero, 6):
        np.testing.assert_array_equal(history[k][1], history[first_zero][1])
        np.testing.assert_array_equal(history[k][2], history[first_zero][2])
    m6, c6, it6, _ = oracle.run(f, spec.gain, spec.readnoise, niter=6)
    assert it6 == first_zero + 1
    np.testing.assert_array_equal(m6, history[-1][1])
    np.testing.assert_array_equal(c6, history[-1][2])
    m0, c0, it0, nf0 = oracle.run(f, spec.gain, spec.readnoise, niter=0)
    assert it0 == 0 and nf0 == 0 and not m0.any()
    np.testing.assert_array_equal(c0, f)


def test_uint16_input_same_as_float_of_it():
    rng = np.random.default_rng(4)
    u = rng.integers(90, 110, size=(40, 50)).astype(np.uint16)
    u[10, 10] = 3000
    a = oracle.run(u, 1.0, 1.5)
    b = oracle.run(u.astype(np.float32), 1.0, 1.5)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_negative_zero_canonicalised_and_nonfinite_rejected():
    f = np.full((8, 8), 5.0, np.float32)
    f[2, 2] = -0.0
    x0, _ = oracle.ingest(f, 65535.0)
    assert not np.signbit(x0[2, 2])
    f[3, 3] = np.nan
    with pytest.raises(ValueError):
        oracle.run(f, 1.0, 1.5)


def test_fp64_flip_budget_on_config0():
    """FP32 vs FP64 per iteration from the same state: flips only near a threshold."""
    spec, f = _config0()
    x32, sat = oracle.ingest(f, spec.satlevel, "f32")
    x64 = x32.astype(np.float64)
    I, M = x32.copy(), np.zeros(f.shape, np.uint8)
    lo32 = np.float32(spec.sigfrac) * np.float32(spec.sigclip)
    total_flips = 0
    for k in range(spec.niter):
        f32, I32, M32, d32 = oracle.iterate(x32, sat, I, M, spec.gain, spec.readnoise,
                                            spec.sigclip, spec.sigfrac, spec.objlim)
        f64, I64, M64, d64 = oracle.iterate(x64, sat, I.astype(np.float64), M, spec.gain,
                                            spec.readnoise, spec.sigclip, spec.sigfrac,
                                            spec.objlim, precision="f64")
        diff = d32["g2"] != d64["g2"]
        total_flips += int(diff.sum())
        if diff.any():
            Sp, F = d64["Sp"], d64["F"]
            near = ((np.abs(Sp - spec.sigclip) <= 1e-5 * spec.sigclip) |
                    (np.abs(Sp - float(lo32)) <= 1e-5 * float(lo32)) |
                    (np.abs(Sp / F - spec.objlim) <= 1e-5 * spec.objlim))
            reach = ndimage.binary_dilation(near, np.ones((5, 5), bool))
            assert np.all(reach[diff])
        I, M = I32, M32
    assert total_flips <= max(1, int(1e-6 * f.size * spec.niter))


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_golden_checkerboard(precision):
    gd = _load_golden("checkerboard.json")
    T = np.float32 if precision == "f32" else np.float64
    ny, nx = gd["shape"]
    ii, jj = np.mgrid[0:ny, 0:nx]
    sign = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    x0 = (gd["sky"] + gd["amp"] * sign).astype(T)
    sat = np.zeros((ny, nx), np.uint8)
    _, _, _, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"], 4.5, 0.3, 5.0,
                                precision=precision)
    e = gd["expected"]
    inner = (slice(4, ny - 4), slice(4, nx - 4))
    hi = (sign > 0)[inner]
    for key, arr in (("N", d["N"]), ("L", d["L"]), ("S", d["S"])):
        a = arr[inner]
        if key == "N":
            assert np.all(a[hi] == e["N_high"]) and np.all(a[~hi] == e["N_low"])
        elif key == "L":
            assert np.all(a[hi] == e["L_high"]) and np.all(a[~hi] == 0)
        else:
            assert np.all(a[hi] == e["S_high"]) and np.all(a[~hi] == 0)
    assert np.all(d["Sp"][inner] == e["Sp"])
    assert np.all(d["F"][inner] == T(e["F"]))


@pytest.mark.parametrize("fnorm", [True, False])
def test_golden_blob_fine_structure(fnorm):
    gd = _load_golden("blob.json")
    ny, nx = gd["shape"]
    cy, cx = gd["centre"]
    x0 = np.full((ny, nx), gd["sky"], np.float32)
    x0[cy - 1:cy + 2, cx - 1:cx + 2] += gd["bump"]
    sat = np.zeros((ny, nx), np.uint8)
    _, _, _, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"], 4.5, 0.3, 5.0,
                                fnorm=fnorm)
    assert d["F"][cy, cx] == (gd["expected"]["F_norm"] if fnorm else gd["expected"]["F_raw"])


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_golden_growth_sigfrac(precision):
    gd = _load_golden("growth.json")
    T = np.float32 if precision == "f32" else np.float64
    ny, nx = gd["shape"]
    (py, px), (qy, qx) = gd["p"], gd["q"]
    for case in gd["cases"][:2]:
        x0 = np.full((ny, nx), gd["sky"], T)
        x0[py, px] += gd["amp_p"]
        x0[qy, qx] += case["b"]
        sat = np.zeros((ny, nx), np.uint8)
        fresh, I, M, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"],
                                        gd["sigclip"], gd["sigfrac"], gd["objlim"],
                                        precision=precision)
        assert d["Sp"][qy, qx] == T(case["Sp_q"])
        assert sorted(map(list, zip(*np.nonzero(M)))) == case["mask"]
        assert np.all(I[M == 1] == T(gd["sky"]))
        np.testing.assert_array_equal(I[M == 0], x0[M == 0])


def test_golden_blob5_med7_window():
    c = _load_golden("blob.json")["cases5"]
    ny, nx = c["shape"]
    cy, cx = c["centre"]
    h = c["half"]
    x0 = np.full((ny, nx), c["sky"], np.float32)
    x0[cy - h:cy + h + 1, cx - h:cx + h + 1] += c["bump"]
    sat = np.zeros((ny, nx), np.uint8)
    _, _, _, d = oracle.iterate(x0, sat, x0, sat, c["gain"], c["readnoise"], 4.5, 0.3, 5.0)
    assert d["F"][cy, cx] == c["F_norm"]


def test_golden_growth_third_pixel_not_reached():
    gd = _load_golden("growth.json")
    case = gd["cases"][2]
    ny, nx = gd["shape"]
    (py, px), (qy, qx), (ry, rx) = gd["p"], gd["q"], case["r"]
    x0 = np.full((ny, nx), gd["sky"], np.float32)
    x0[py, px] += gd["amp_p"]
    x0[qy, qx] += case["b"]
    x0[ry, rx] += case["c"]
    sat = np.zeros((ny, nx), np.uint8)
    _, _, M, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"], gd["sigclip"],
                                gd["sigfrac"], gd["objlim"])
    lo = np.float32(gd["sigfrac"]) * np.float32(gd["sigclip"])
    assert lo < d["Sp"][ry, rx] < gd["sigclip"] and lo < d["Sp"][qy, qx] < gd["sigclip"]
    assert sorted(map(list, zip(*np.nonzero(M)))) == case["mask"]


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_golden_stripes_objlim_uses_s_prime(precision):
    gd = _load_golden("stripes_objlim.json")
    T = np.float32 if precision == "f32" else np.float64
    ny, nx = gd["shape"]
    py, px = gd["p"]
    x0 = np.where(np.arange(nx)[None, :].repeat(ny, 0) % 2 == 0, gd["bright"], gd["dark"]).astype(T)
    x0[py, px] += gd["hit"]
    sat = np.zeros((ny, nx), np.uint8)
    for case in gd["cases"]:
        _, _, M, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"], gd["sigclip"],
                                    gd["sigfrac"], case["objlim"], precision=precision)
        assert abs(d["S"][py, px] - gd["S_p"]) < 1e-5 and abs(d["Sp"][py, px] - gd["Sp_p"]) < 1e-5
        assert d["F"][py, px] == T(0.01)
        assert sorted(map(list, zip(*np.nonzero(M)))) == case["mask"]


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_golden_noise_floor(precision):
    c = _load_golden("flat_noise.json")["floor_case"]
    x0 = np.full((6, 6), c["sky"], np.float32 if precision == "f32" else np.float64)
    sat = np.zeros(x0.shape, np.uint8)
    _, _, M, d = oracle.iterate(x0, sat, x0, sat, c["gain"], c["readnoise"], 4.5, 0.3, 5.0,
                                precision=precision)
    assert np.all(np.abs(d["N"] - c["N_approx"]) < 1e-7)
    assert np.all(d["S"] == 0) and M.sum() == 0


def test_golden_threshold_strictness():
    gd = _load_golden("growth.json")
    case = gd["cases"][3]
    ny, nx = gd["shape"]
    (py, px), (qy, qx), (ry, rx) = gd["p"], gd["q"], case["r"]
    x0 = np.full((ny, nx), gd["sky"], np.float32)
    x0[py, px] += case["amp_p"]
    x0[qy, qx] += case["b"]
    x0[ry, rx] += case["c"]
    sat = np.zeros((ny, nx), np.uint8)
    _, _, M, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"], gd["sigclip"],
                                gd["sigfrac"], gd["objlim"])
    assert d["Sp"][qy, qx] == np.float32(case["Sp_q"])
    assert sorted(map(list, zip(*np.nonzero(M)))) == case["mask"]


def test_golden_lower_threshold_strictness():
    # growth.json, fifth case: S'(q) equals sigfrac*sigclip exactly in float32;
    # q is grown only by a non-strict test.
    gd = _load_golden("growth.json")
    case = gd["cases"][4]
    ny, nx = gd["shape"]
    (py, px), (qy, qx) = gd["p"], gd["q"]
    x0 = np.full((ny, nx), gd["sky"], np.float32)
    x0[py, px] += gd["amp_p"]
    x0[qy, qx] += case["b"]
    sat = np.zeros((ny, nx), np.uint8)
    _, _, M, d = oracle.iterate(x0, sat, x0, sat, gd["gain"], gd["readnoise"], gd["sigclip"],
                                gd["sigfrac"], gd["objlim"])
    lo = np.float32(gd["sigfrac"]) * np.float32(gd["sigclip"])
    assert d["Sp"][qy, qx] == lo == np.float32(case["Sp_q"])
    assert sorted(map(list, zip(*np.nonzero(M)))) == case["mask"]


def test_saturated_pixel_seeds_no_growth():
    # Reading C9: a saturated pixel is never a candidate, so nothing grows from
    # it.  A sharp saturated pixel sits on the wing of a resolved star (FWHM 3,
    # peak 10000 ADU), two pixels from its centre.  Five of its neighbours have
    # S' > sigclip but fail the objlim test (the star is resolved: med3 - med7
    # is large there), so nothing is a candidate and nothing is flagged; a
    # saturated candidate would grow into those neighbours.
    yy, xx = np.mgrid[0:32, 0:32]
    s = 3.0 / 2.3548
    f = (100.0 + 10000.0 * np.exp(-((yy - 16) ** 2 + (xx - 16) ** 2) / (2 * s * s))).astype(np.float32)
    f[16, 18] = 65535.0
    sat = (f >= 60000.0).astype(np.uint8)
    _, _, M, d = oracle.iterate(f, sat, f, np.zeros(f.shape, np.uint8), 1.0, 1.5, 4.5, 0.3, 5.0)
    nb = [(16 + a, 18 + b) for a in (-1, 0, 1) for b in (-1, 0, 1) if (a, b) != (0, 0)]
    assert sum(d["Sp"][q] > 4.5 and d["Sp"][q] / d["F"][q] <= 5.0 for q in nb) >= 3  # fail objlim only
    assert d["Sp"][16, 18] > 4.5 and d["Sp"][16, 18] / d["F"][16, 18] > 5.0  # sharp: passes both tests
    assert d["cand"].sum() == 0 and M.sum() == 0
    m, _, _, nf = oracle.run(f, 1.0, 1.5, satlevel=60000.0, niter=4)
    assert nf == 0 and m.sum() == 0
