"""The two sparse tests of step 4-5 that the core kernel decides by rank.

The kernel never forms S' = S - med5(S) at an item that needs only the lo
test (S - med5 > lo), and never forms med7(med3) on a uint16 frame: a test
that is monotone in a median holds at the median iff it holds at enough of
the window's values (13 of 25, 25 of 49).  These tests state that lemma in
float32 arithmetic, with the kernel's operation order, against the same
tests evaluated at the median itself:

* the lo test, fl(S - x) > lo, falls as x grows;
* the objlim test, fl(S' / max(fl(d / N), 0.01)) > objlim with
  d = m3 - v (exact for integers below 2^16), rises with v when S' > 0;
  its threshold d* is taken from the real-number bound and confirmed with
  the float test at d* and d* + 1 (as the kernel does), and the search must
  settle within four steps.

The kernel's own arithmetic is checked bit for bit against the oracle by
the GPU parity tests; this pins the reasoning that makes the shortcut exact.
"""
import numpy as np
import pytest

f32 = np.float32


def objlim_at(sp, N, d, objlim, fnorm):
    """The objlim test with med3 - med7 = d (float32, the kernel's order)."""
    F = f32(0.01)
    if d > 0:
        F = f32(f32(d) / N) if fnorm else f32(d)
        F = f32(0.01) if F < f32(0.01) else F
    return bool(f32(sp / F) > objlim)


def objlim_by_median(sp, N, m3, w, objlim, fnorm):
    m7 = int(np.sort(w)[24])
    diff = f32(f32(m3) - f32(m7))  # the definition: a float difference
    F = f32(diff / N) if fnorm else diff
    F = f32(0.01) if F < f32(0.01) else F
    return bool(f32(sp / F) > objlim)


def objlim_by_rank(sp, N, m3, w, objlim, fnorm):
    """Returns (decision, steps) or (None, steps) when the search did not settle."""
    dlo, dhi = m3 - 65535, m3
    P = lambda d: objlim_at(sp, N, d, objlim, fnorm)
    steps = 0
    if not P(dlo):
        ds = dlo - 1
    elif P(dhi):
        ds = dhi
    else:
        x = f32(f32(sp / objlim) * N) if fnorm else f32(sp / objlim)
        d = dlo if not x > f32(dlo) else (dhi - 1 if x > f32(dhi) else int(np.ceil(x)) - 1)
        d = min(max(d, dlo), dhi - 1)
        ds = None
        for steps in range(1, 5):
            if not P(d):
                d -= 1
            elif P(d + 1):
                d += 1
            else:
                ds = d
                break
        if ds is None:
            return None, steps
    return bool((np.asarray(w) >= m3 - ds).sum() >= 25), steps


def lo_by_median(Sc, w, lo):
    return bool(f32(Sc - np.sort(w)[12]) > lo)


def lo_by_rank(Sc, w, lo):
    return int(sum(f32(Sc - v) > lo for v in w)) >= 13


def _window_u16(rng, m3):
    kind = rng.integers(0, 4)
    if kind == 0:
        return rng.integers(0, 65536, 49)
    if kind == 1:  # flat with ties
        return np.full(49, int(rng.integers(0, 65536)))
    return np.clip(m3 + rng.integers(-40, 40) + rng.integers(-25, 25, 49), 0, 65535)


@pytest.mark.parametrize("fnorm", [True, False])
@pytest.mark.parametrize("objlim", [5.0, 2.0, 0.5, 40.0, 1e-3, 0.0, -1.0])
def test_objlim_rank_equals_median(fnorm, objlim):
    rng = np.random.default_rng(abs(int(objlim * 1000)) + fnorm)
    objlim = f32(objlim)
    worst = 0
    for it in range(4000):
        m3 = int(rng.integers(0, 65536)) if it % 2 else int(rng.integers(0, 300))
        w = _window_u16(rng, m3)
        N = f32(rng.uniform(0.3, 40.0))
        sp = f32(rng.uniform(4.5, 800.0))
        if it % 3 == 1 and objlim > 0:  # S' placed on the test's boundary at the median, within an ulp
            d7 = f32(f32(m3) - f32(np.sort(w)[24]))
            F = f32(d7 / N) if fnorm else d7
            F = max(F, f32(0.01))
            sp = np.nextafter(f32(F * objlim), f32(np.inf if it % 2 else 0), dtype=f32)
            if not sp > 0:
                continue
        got, steps = objlim_by_rank(sp, N, m3, w, objlim, fnorm)
        worst = max(worst, steps)
        assert got is not None, (sp, N, m3, objlim, fnorm)
        assert got == objlim_by_median(sp, N, m3, w, objlim, fnorm), (sp, N, m3, objlim, fnorm)
    assert worst <= 3


def test_objlim_rank_extremes():
    # every med7 value passes, none passes, and the F floor (d <= 0.01 N)
    w = np.arange(49) * 1000
    assert objlim_by_rank(f32(1e6), f32(1.0), 65535, w, f32(5), True) == (True, 0)
    assert objlim_by_rank(f32(4.6), f32(1.0), 0, w, f32(1e4), True) == (False, 0)
    for m3 in (0, 1, 5, 65535):
        for sp in (f32(0.04), f32(0.05), f32(0.06), f32(5.0)):
            got, _ = objlim_by_rank(sp, f32(2.0), m3, w, f32(5.0), True)
            assert got == objlim_by_median(sp, f32(2.0), m3, w, f32(5.0), True)


def test_lo_rank_equals_median():
    rng = np.random.default_rng(3)
    lo = f32(1.35)
    for it in range(20000):
        w = rng.normal(0.0, 3.0, 25).astype(f32)
        if it % 3 == 0:
            w = (np.round(w * 4) / 4).astype(f32)  # ties
        if it % 7 == 0:
            w = np.full(25, f32(rng.normal()), dtype=f32)
        Sc = f32(rng.uniform(-2.0, 10.0))
        if it % 2:  # S - med5 on the threshold, within an ulp
            Sc = np.nextafter(f32(np.sort(w)[12] + lo), f32(rng.choice([-np.inf, np.inf])), dtype=f32)
        assert lo_by_rank(Sc, w, lo) == lo_by_median(Sc, w, lo), (Sc, w)


def test_a_slip_in_the_rank_is_caught():
    # The same check with the wrong rank (12 of 25 instead of 13) must fail somewhere,
    # so the tests above can tell a correct rank from a wrong one.
    rng = np.random.default_rng(5)
    lo = f32(1.35)
    wrong = 0
    for _ in range(2000):
        w = rng.normal(0.0, 3.0, 25).astype(f32)
        Sc = f32(np.sort(w)[12] + lo + f32(0.01))
        Sc = f32(np.sort(w)[11] + lo + f32(0.01)) if rng.integers(0, 2) else Sc
        wrong += (int(sum(f32(Sc - v) > lo for v in w)) >= 12) != lo_by_median(Sc, w, lo)
    assert wrong > 0


def _windows(A, r):
    """The (2r+1)^2 clamped-window values of every pixel of A, shape (K*K, ny, nx)."""
    P = np.pad(A, r, mode="edge")
    ny, nx = A.shape
    return np.stack([P[dy:dy + ny, dx:dx + nx] for dy in range(2 * r + 1) for dx in range(2 * r + 1)])


def test_rank_decisions_on_a_synthetic_frame():
    # Realistic value fields: a uint16 frame of the 61-Mpx recipe (stars, tracks, salt and pepper)
    # at its first level, S = L+ / (2N) with N from the exact 5x5 median, S' items where S
    # exceeds the lower threshold, med3 and the 7x7 median of med3 from the oracle.  At every
    # item the lo test by rank must equal the test at the oracle's med5(S), and at every fine
    # item with S' > sigclip the objlim test by rank must equal the test at its med7.
    import oracle
    from paper_2602_17938_gb300 import synth
    spec = synth.FrameSpec(**{**synth.config_specs(1)[0].__dict__, "ny": 192, "nx": 256, "seed": (1, 900),
                              "n_stars": 12, "n_tracks": 500})
    X = synth.make_frame(spec).astype(np.float32)
    g, rn2 = f32(spec.gain), f32(spec.readnoise) * f32(spec.readnoise)
    m5 = oracle.median(X, 5)
    N = (np.sqrt(np.maximum(g * m5, f32(1e-4)) + rn2) / g).astype(f32)
    S = (oracle.lplus(X) / (N + N)).astype(f32)
    lo, sigclip, objlim = f32(spec.sigfrac * spec.sigclip), f32(spec.sigclip), f32(spec.objlim)
    mS = oracle.median(S, 5)
    items = np.argwhere(S > min(lo, sigclip))
    assert len(items) > 2000
    W5 = _windows(S, 2)
    for y, x in items:
        assert lo_by_rank(S[y, x], W5[:, y, x], lo) == bool(f32(S[y, x] - mS[y, x]) > lo), (y, x)
    m3 = oracle.median(X, 3)
    m7 = oracle.median(m3, 7)
    W7 = _windows(m3, 3).astype(np.int64)
    fine = 0
    for y, x in items:
        sp = f32(S[y, x] - mS[y, x])
        if not (S[y, x] > sigclip and sp > sigclip):
            continue
        fine += 1
        got, steps = objlim_by_rank(sp, N[y, x], int(m3[y, x]), W7[:, y, x], objlim, True)
        assert got is not None and steps <= 3
        diff = f32(m3[y, x] - m7[y, x])
        F = max(f32(diff / N[y, x]), f32(0.01))
        assert got == bool(f32(sp / F) > objlim), (y, x)
    assert fine > 200
