"""Levels after the first recompute only the core tiles whose inputs changed.

A core tile's bit-planes at level k+1 depend on the mask only within 6
pixels of the tile (unless a replacement there needed a window wider than
5x5, which marks the tile for recomputation at every later level).  These
tests check that skipping the other tiles leaves every output bit-identical
to the float32 oracle, and that the skipping really happens (the profile's
px_core counts the tile pixels the core kernel computed).
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17938_gb300 import build, lacos
    build.build()
    return lacos


def _sky(ny, nx, seed, sky=200.0, gain=1.0, rn=2.0):
    rng = np.random.default_rng(seed)
    return sky + math.sqrt(gain * sky + rn * rn) / gain * rng.standard_normal((ny, nx)), rng


def _tracks(f, rng, n, length=(3, 14), amp=(300.0, 4000.0)):
    """Straight 1-2 px wide tracks: later levels grow into their wings."""
    ny, nx = f.shape
    for _ in range(n):
        y, x = rng.uniform(0, ny), rng.uniform(0, nx)
        a, L, A = rng.uniform(0, math.pi), rng.uniform(*length), rng.uniform(*amp)
        for t in np.linspace(0, L, int(2 * L) + 2):
            iy, ix = int(y + t * math.sin(a)), int(x + t * math.cos(a))
            if 0 <= iy < ny and 0 <= ix < nx:
                f[iy, ix] += A
                if rng.uniform() < 0.5 and ix + 1 < nx:
                    f[iy, ix + 1] += 0.6 * A


def _run(lacos, frame, gain, rn, niter):
    d = lacos.to_device(frame)
    m = torch.empty(frame.shape, dtype=torch.uint8, device="cuda")
    c = torch.empty(frame.shape, dtype=torch.float32, device="cuda")
    p = lacos.make_params(gain, rn, niter=niter)
    with lacos.Context(0) as ctx:
        ctx.set_profiling(True)
        r = ctx.wait(ctx.submit(d, p, m, c))
        prof = ctx.last_profile()
    torch.cuda.synchronize()
    return m.cpu().numpy(), c.cpu().numpy(), r, prof


def _assert_oracle(frame, gain, rn, niter, m, c, r):
    m_ref, c_ref, it, nf = oracle.run(frame, gain, rn, niter=niter)
    bad = np.argwhere(m != m_ref)
    assert bad.size == 0, f"{len(bad)} mask px differ, first at {bad[:5].tolist()}"
    badc = np.argwhere(c.view(np.uint32) != c_ref.view(np.uint32))
    assert badc.size == 0, f"{len(badc)} cleaned px differ, first at {badc[:5].tolist()}"
    assert r.status == 0 and r.iters_run == it and r.n_flagged == nf
    return it


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_sparse_tracks_skip_tiles_and_stay_exact(lib, dtype):
    # 640 x 1000 px = 20 x 16 tiles, a few dozen tracks: after level 1 most
    # tiles see no new flag within 6 px.
    f, rng = _sky(640, 1000, 5)
    _tracks(f, rng, 40)
    frame = np.clip(np.rint(f), 0, 65535).astype(np.uint16) if dtype == np.uint16 else f.astype(np.float32)
    m, c, r, prof = _run(lib, frame, 1.0, 2.0, niter=6)
    it = _assert_oracle(frame, 1.0, 2.0, 6, m, c, r)
    assert it >= 2, "the frame should need more than one level"
    npix = frame.size
    assert prof["px_iterations"] == npix * it
    assert npix <= prof["px_core"] < prof["px_iterations"], prof


def test_tracks_on_tile_borders(lib):
    # Tracks placed across the 32 x 64 tile grid lines, so that new flags of
    # later levels fall within 6 px of neighbouring tiles.
    f, rng = _sky(256, 512, 9)
    for y in (30, 31, 32, 33, 94, 160):
        for x in (60, 62, 63, 64, 65, 190, 320):
            f[y:y + 2, x:x + 3] += rng.uniform(500, 3000)
    frame = f.astype(np.float32)
    m, c, r, prof = _run(lib, frame, 1.0, 2.0, niter=6)
    _assert_oracle(frame, 1.0, 2.0, 6, m, c, r)


def test_wide_window_tile_recomputed_at_later_levels(lib):
    # One tile holds a block flagged almost entirely (5x5 windows with no
    # unflagged member: the widened replacement), the rest of the frame is
    # sparse; every level must reproduce the oracle.
    for seed in (3, 11):
        f, rng = _sky(192, 320, seed, sky=100.0, rn=1.5)
        f[70:85, 150:165] += rng.uniform(0, 20000, (15, 15))
        _tracks(f, rng, 6)
        frame = f.astype(np.float32)
        m, c, r, prof = _run(lib, frame, 1.0, 1.5, niter=5)
        _assert_oracle(frame, 1.0, 1.5, 5, m, c, r)
        assert prof["n_replace_wide"] > 0, "the frame no longer reaches the widened replacement"
