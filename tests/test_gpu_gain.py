"""Gain estimated at every iteration (gain 0, reading C15) on the GPU,
bit-identical to the float32 oracle: masks, cleaned frames, iteration counts
and the gain of the last iteration run.

Frames are seeded Poisson skies in electrons, read noise added, converted to
integer ADU with the true gain, plus cosmic-ray tracks: later levels flag
more pixels, so the pair set and the estimate change between levels (every
tile is then recomputed).  Shapes cover the 16-byte-load path (nx a multiple
of 8), the scalar path and an odd width (the last column has no partner).
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


def _frame(ny, nx, seed, g=2.0, rn=5.0, sky=400.0, ntracks=40):
    rng = np.random.default_rng(seed)
    e = rng.poisson(g * sky, (ny, nx)) + rng.normal(0.0, rn, (ny, nx))
    f = np.rint(e / g)
    for _ in range(ntracks):
        y, x = rng.uniform(0, ny), rng.uniform(0, nx)
        a, L, A = rng.uniform(0, math.pi), rng.uniform(2, 12), rng.uniform(300, 5000)
        for t in np.linspace(0, L, int(2 * L) + 2):
            iy, ix = int(y + t * math.sin(a)), int(x + t * math.cos(a))
            if 0 <= iy < ny and 0 <= ix < nx:
                f[iy, ix] += A
    return np.clip(f, 0, 65535).astype(np.uint16)


def _device_run(lacos, frame, params):
    d = lacos.to_device(frame)
    m = torch.empty(frame.shape, dtype=torch.uint8, device="cuda")
    c = torch.empty(frame.shape, dtype=torch.float32, device="cuda")
    with lacos.Context(0) as ctx:
        r = ctx.wait(ctx.submit(d, params, m, c))
    torch.cuda.synchronize()
    return m.cpu().numpy(), c.cpu().numpy(), r


def _assert_same(m, c, r, ref):
    m_ref, c_ref, it, nf, g_last, ok = ref
    bad = np.argwhere(m != m_ref)
    assert bad.size == 0, f"{len(bad)} mask px differ, first at {bad[:5].tolist()}"
    badc = np.argwhere(c.view(np.uint32) != c_ref.view(np.uint32))
    assert badc.size == 0, f"{len(badc)} cleaned px differ, first at {badc[:5].tolist()}"
    assert (r.iters_run, r.n_flagged) == (it, nf)
    assert r.gain == np.float32(g_last)


@pytest.mark.parametrize("ny,nx", [(256, 512), (300, 410), (517, 261)])
def test_estimated_gain_matches_oracle(lib, ny, nx):
    frame = _frame(ny, nx, ny + nx)
    p = lib.make_params(0.0, 5.0, niter=4)
    m, c, r = _device_run(lib, frame, p)
    ref = oracle.run(frame, 0.0, 5.0, niter=4, return_gain=True)
    assert ref[5] and ref[2] >= 2, "the frame should need several levels with a defined gain"
    assert r.status == 0
    _assert_same(m, c, r, ref)
    assert abs(r.gain / 2.0 - 1.0) < 0.08  # near the true gain (the clip biases it up ~3%)


@pytest.mark.parametrize("satgrow", [0, 2])
def test_estimated_gain_with_saturation(lib, satgrow):
    frame = _frame(200, 328, 21 + satgrow, sky=300.0)
    frame[50:56, 100:108] = 60000
    frame[150, 20] = 61000
    p = lib.make_params(0.0, 4.0, satlevel=50000.0, niter=4, satgrow=satgrow)
    m, c, r = _device_run(lib, frame, p)
    ref = oracle.run(frame, 0.0, 4.0, satlevel=50000.0, niter=4, satgrow=satgrow, return_gain=True)
    assert r.status == 0
    _assert_same(m, c, r, ref)


def test_undefined_estimate_reports_and_uses_unit_gain(lib):
    frame = np.full((64, 96), 150, np.uint16)
    frame[20, 30] = 5000
    p = lib.make_params(0.0, 3.0, niter=3)
    m, c, r = _device_run(lib, frame, p)
    ref = oracle.run(frame, 0.0, 3.0, niter=3, return_gain=True)
    assert not ref[5]
    assert r.status == lib.ENOGAIN and r.gain == 1.0
    _assert_same(m, c, r, ref)


def test_supplied_gain_is_reported(lib):
    frame = _frame(96, 128, 5)
    m, c, r = _device_run(lib, frame, lib.make_params(1.75, 5.0))
    assert r.status == 0 and r.gain == np.float32(1.75)


def test_estimation_rejects_float_frames_and_negative_gain(lib):
    f32 = lib.to_device(_frame(64, 64, 2).astype(np.float32))
    m = torch.empty(f32.shape, dtype=torch.uint8, device="cuda")
    c = torch.empty(f32.shape, dtype=torch.float32, device="cuda")
    u16 = lib.to_device(_frame(64, 64, 2))
    with lib.Context(0) as ctx:
        with pytest.raises(lib.LacosError) as e:
            ctx.submit(f32, lib.make_params(0.0, 3.0), m, c)
        assert e.value.code == lib.EINVAL
        with pytest.raises(lib.LacosError) as e:
            ctx.submit(u16, lib.make_params(-1.0, 3.0), m, c)
        assert e.value.code == lib.EINVAL


def test_batch_mixes_estimated_and_supplied_gains(lib):
    frames = [_frame(160, 200, 31), _frame(96, 352, 32), _frame(130, 140, 33).astype(np.float32)]
    gains = [0.0, 2.5, 2.0]
    params = [lib.make_params(g, 5.0, niter=4) for g in gains]
    d = [lib.to_device(f) for f in frames]
    ms = [torch.empty(f.shape, dtype=torch.uint8, device="cuda") for f in frames]
    cs = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in frames]
    with lib.Context(0) as ctx:
        t, per = ctx.submit_batch(d, params, ms, cs)
        ctx.wait(t)
    torch.cuda.synchronize()
    for i, f in enumerate(frames):
        ref = oracle.run(f, gains[i], 5.0, niter=4, return_gain=True)
        _assert_same(ms[i].cpu().numpy(), cs[i].cpu().numpy(), per[i], ref)


def test_static_entry_point_estimates_the_gain(lib):
    frame = _frame(192, 256, 41)
    d = lib.to_device(frame)
    m = torch.empty(frame.shape, dtype=torch.uint8, device="cuda")
    c = torch.empty(frame.shape, dtype=torch.float32, device="cuda")
    r = lib.run_static(d, lib.make_params(0.0, 5.0, niter=4), m, c)
    torch.cuda.synchronize()
    _assert_same(m.cpu().numpy(), c.cpu().numpy(), r, oracle.run(frame, 0.0, 5.0, niter=4, return_gain=True))


def test_histogram_bin_sums_wrap_and_extreme_differences(lib):
    # A bright, nearly flat uint16 frame (65500 ADU, 8% of pixels one higher) of 7200 x 7200
    # with the saturation guard off: on 152 SMs each histogram block sees about 36000 pairs
    # with d = 0, so that bin's sum of a + b (131000 per pair) passes 2^32 within one block
    # and the 32-bit shared sum must carry.  A few pairs (0, 65535) and (65535, 0) put
    # d = -65535 and +65535 in the outermost bins (clipped in the first round).  The level-1
    # gain must equal the oracle's estimate on the same image (reading C15), bit for bit
    # after rounding to float.
    ny = nx = 7200
    rng = np.random.default_rng(7200)
    f = np.full((ny, nx), 65500, np.int32) + (rng.random((ny, nx)) < 0.08)
    for y in range(100, 7100, 700):
        f[y, 100:104] = (0, 65535, 65535, 0)  # pairs (0, 65535) and (65535, 0) at even columns
    frame = f.astype(np.uint16)
    z = np.zeros(frame.shape, np.uint8)
    g_ref, rounds, stats = oracle.estimate_gain(frame.astype(np.float32), z, z, 2.0)
    assert g_ref is not None and rounds >= 1
    p = lib.make_params(0.0, 2.0, satlevel=0.0, niter=1)
    m, c, r = _device_run(lib, frame, p)
    assert r.status == 0 and r.iters_run == 1
    assert r.gain == np.float32(g_ref)
    keep = m == 0
    assert np.array_equal(c[keep], frame[keep].astype(np.float32))
