"""GPU (CUDA path, through the C ABI) vs the float32 CPU oracle: bit-exact.

The masks are compared byte for byte and the cleaned frames bit for bit;
iters_run and n_flagged must match too.  The 61-Mpx frame is compared on
every pixel with the oracle's whole-frame result (stored digests), and on
sampled crops against live oracle runs (a crop with a 64-pixel margin
reproduces the frame's result in its interior: one iteration reads at most
8 pixels away), plus properties that hold at any size.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_17938_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17938_gb300 import build, lacos
    build.build()
    c = lacos.Context(0)
    yield c
    c.close()


def gpu_run(ctx, frame, gain, rn, **kw):
    from paper_2602_17938_gb300 import lacos
    mask, clean, res = lacos.clean_frame(lacos.to_device(frame), gain, rn, ctx=ctx, **kw)
    torch.cuda.synchronize()
    return mask.cpu().numpy(), clean.cpu().numpy(), res


def assert_same(frame, gain, rn, gpu, **kw):
    m, c, res = gpu
    m_ref, c_ref, it_ref, nf_ref = oracle.run(frame, gain, rn, **kw)
    bad = np.argwhere(m != m_ref)
    assert bad.size == 0, f"{len(bad)} mask px differ, first at {bad[:5].tolist()}"
    badc = np.argwhere(c.view(np.uint32) != c_ref.view(np.uint32))
    assert badc.size == 0, f"{len(badc)} cleaned px differ, first at {badc[:5].tolist()}"
    assert res.status == 0
    assert res.iters_run == it_ref and res.n_flagged == nf_ref
    return m_ref, c_ref


def noisy_with_hits(ny, nx, seed, sky=100.0, gain=1.0, rn=1.5, n_hits=None, dtype=np.float32):
    rng = np.random.default_rng(seed)
    sig = math.sqrt(gain * sky + rn * rn) / gain
    f = sky + sig * rng.standard_normal((ny, nx))
    n_hits = max(1, ny * nx // 150) if n_hits is None else n_hits
    ys, xs = rng.integers(0, ny, n_hits), rng.integers(0, nx, n_hits)
    f[ys, xs] += rng.uniform(200, 3000, n_hits)
    if dtype == np.uint16:
        return np.clip(np.rint(f), 0, 65535).astype(np.uint16)
    return f.astype(np.float32)


def test_config0_bit_exact(ctx):
    spec = synth.config_specs(0)[0]
    f = synth.make_frame(spec)
    assert_same(f, spec.gain, spec.readnoise, gpu_run(ctx, f, spec.gain, spec.readnoise))


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (37, 1), (2, 2), (7, 7), (13, 9), (31, 33),
                                   (32, 32), (33, 65), (64, 64), (95, 129), (100, 37)])
def test_small_and_ragged_frames(ctx, shape):
    f = noisy_with_hits(*shape, seed=shape[0] * 1000 + shape[1])
    assert_same(f, 1.0, 1.5, gpu_run(ctx, f, 1.0, 1.5))


@pytest.mark.parametrize("shape", [(300, 433), (129, 64)])
def test_uint16_salt_and_pepper(ctx, shape):
    spec = synth.FrameSpec(shape[0], shape[1], "u16", (11, shape[0]), sky=300.0, gain=0.8,
                           readnoise=1.2, n_stars=10, n_tracks=150, hot_frac=0.005, salt_pepper=True)
    f = synth.make_frame(spec)
    assert_same(f, spec.gain, spec.readnoise, gpu_run(ctx, f, spec.gain, spec.readnoise))


@pytest.mark.parametrize("niter", [0, 1, 2, 6])
def test_niter_values(ctx, niter):
    f = noisy_with_hits(150, 170, seed=3)
    assert_same(f, 1.0, 1.5, gpu_run(ctx, f, 1.0, 1.5, niter=niter), niter=niter)


def test_unnormalised_fine_structure_variant(ctx):
    f = noisy_with_hits(120, 140, seed=4)
    assert_same(f, 1.0, 1.5, gpu_run(ctx, f, 1.0, 1.5, fine_norm=False), fnorm=False)


def test_negative_values_and_negative_zero(ctx):
    f = noisy_with_hits(90, 110, seed=5, sky=0.0)
    f[::7, ::5] = -0.0
    f[3, 3] = -500.0
    assert_same(f, 1.0, 1.5, gpu_run(ctx, f, 1.0, 1.5))


def test_saturation(ctx):
    f = noisy_with_hits(96, 96, seed=6)
    f[20:23, 30:33] = 65535.0
    f[50, 50] = 65535.0
    for sat in (65535.0, 0.0, 3000.0):
        assert_same(f, 1.0, 1.5, gpu_run(ctx, f, 1.0, 1.5, satlevel=sat), satlevel=sat)


def test_dense_hits_exercise_widened_replacement(ctx):
    # A 15x15 block of rough bright texture (uniform 0-20000 ADU added per
    # pixel) is flagged almost entirely, leaving 5x5 windows with no
    # unflagged member, so the replacement widens to 7x7 and beyond.
    for seed in (3, 11, 27):
        rng = np.random.default_rng(seed)
        f = (100 + 10 * rng.standard_normal((80, 90))).astype(np.float32)
        f[30:45, 30:45] += rng.uniform(0, 20000, (15, 15)).astype(np.float32)
        m_ref, _ = assert_same(f, 1.0, 1.5, gpu_run(ctx, f, 1.0, 1.5))
        from numpy.lib.stride_tricks import sliding_window_view
        full = sliding_window_view(np.pad(m_ref, 2, mode="edge"), (5, 5)).all(axis=(2, 3)) & (m_ref == 1)
        assert full.any(), "test frame no longer reaches the widened replacement"


@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_saturated_star_protection(ctx, r, dtype):
    # Saturated star cores, some on tile borders and frame edges, with hits
    # scattered around them: the grown protected region (reading C16) must
    # match the oracle bit for bit.
    rng = np.random.default_rng(40 + r)
    f = noisy_with_hits(150, 260, seed=90 + r, n_hits=400).astype(np.float64)
    for (y, x) in [(30, 62), (31, 130), (64, 5), (100, 200), (148, 258), (2, 100), (75, 64)]:
        f[max(0, y - 1):y + 2, max(0, x - 1):x + 2] = 65535.0
        for _ in range(6):  # hits around each core
            dy, dx = rng.integers(-6, 7, 2)
            yy, xx = min(max(y + dy, 0), 149), min(max(x + dx, 0), 259)
            if f[yy, xx] < 65535.0:
                f[yy, xx] += rng.uniform(400, 3000)
    frame = np.clip(np.rint(f), 0, 65535).astype(np.uint16) if dtype == np.uint16 else f.astype(np.float32)
    m_ref, _ = assert_same(frame, 1.0, 1.5, gpu_run(ctx, frame, 1.0, 1.5, satgrow=r), satgrow=r)
    m0, *_ = oracle.run(frame, 1.0, 1.5)
    assert (m0.astype(int) - m_ref.astype(int)).max() == 1, "the protection should remove some flags"


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_separable_median_mode(ctx, dtype):
    # The comparison mode (both 5x5 detection medians separable) against the
    # oracle's separable median, bit for bit: hits on noise plus bright stars.
    from paper_2602_17938_gb300 import synth
    for seed, shape in ((3, (200, 333)), (8, (129, 64))):
        spec = synth.FrameSpec(*shape, "f32", (30, seed), sky=300.0, gain=1.0, readnoise=3.0,
                               n_stars=12, star_peak=(1e4, 4e5), n_tracks=60, hot_frac=0.002, fwhm=3.0)
        f = np.minimum(synth.make_frame(spec), 65535.0)
        frame = np.rint(f).astype(np.uint16) if dtype == np.uint16 else f.astype(np.float32)
        m_ref, _ = assert_same(frame, 1.0, 3.0, gpu_run(ctx, frame, 1.0, 3.0, sepmed=True), sepmed=True)
        m_true, *_ = oracle.run(frame, 1.0, 3.0)
        assert not np.array_equal(m_ref, m_true)


def test_varied_parameters(ctx):
    f = noisy_with_hits(140, 160, seed=8)
    for kw in ({"sigclip": 3.0, "sigfrac": 0.5, "objlim": 2.0}, {"sigclip": 6.0, "sigfrac": 1.5, "objlim": 8.0},
               {"sigclip": 4.5, "sigfrac": 0.1, "objlim": 0.5}):
        assert_same(f, 2.5, 4.0, gpu_run(ctx, f, 2.5, 4.0, **kw), **kw)


def test_nonfinite_input_reported(ctx):
    f = noisy_with_hits(40, 40, seed=9)
    f[5, 5] = np.nan
    _, _, res = gpu_run(ctx, f, 1.0, 1.5)
    from paper_2602_17938_gb300 import lacos
    assert res.status == lacos.ENONFINITE


def test_argument_errors(ctx):
    from paper_2602_17938_gb300 import lacos
    f = lacos.to_device(noisy_with_hits(16, 16, seed=1))
    m = torch.empty((16, 16), dtype=torch.uint8, device="cuda")
    c = torch.empty((16, 16), dtype=torch.float32, device="cuda")
    # f is float32: gain 0 (estimate the gain) is for uint16 frames only
    for bad in (dict(gain=0.0), dict(gain=-1.0), dict(sigclip=0.0), dict(niter=-1), dict(niter=257),
                dict(readnoise=-1.0), dict(objlim=float("nan")), dict(satgrow=-1), dict(satgrow=5)):
        kw = dict(gain=1.0, readnoise=1.5)
        kw.update(bad)
        with pytest.raises(lacos.LacosError) as e:
            ctx.submit(f, lacos.make_params(**kw), m, c)
        assert e.value.code == lacos.EINVAL
    # a frame of 2^31 pixels or more is refused by the C ABI before any device access
    # (the call gets a small real buffer with the oversize dimensions)
    import ctypes
    lib = lacos.load_library()
    t = ctypes.c_ulonglong(0)
    p0 = lacos.make_params(1.0, 1.5)
    rc = lib.lacos_submit(ctx.h, ctypes.c_void_p(f.data_ptr()), lacos.LACOS_F32, 46341, 46341, ctypes.byref(p0),
                          ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(c.data_ptr()), None, ctypes.byref(t))
    assert rc == lacos.EINVAL
    for ny, nx in ((0, 16), (16, 0), (-1, 16)):  # empty and negative extents
        rc = lib.lacos_submit(ctx.h, ctypes.c_void_p(f.data_ptr()), lacos.LACOS_F32, ny, nx, ctypes.byref(p0),
                              ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(c.data_ptr()), None, ctypes.byref(t))
        assert rc == lacos.EINVAL, (ny, nx)
    p = lacos.make_params(1.0, 1.5)
    p.sepmed = 2  # only 0 or 1
    with pytest.raises(lacos.LacosError) as e:
        ctx.submit(f, p, m, c)
    assert e.value.code == lacos.EINVAL
    with pytest.raises(lacos.LacosError) as e:
        ctx.poll(123456789)
    assert e.value.code == lacos.EUNKNOWN_TICKET


def test_budget_and_slots(ctx):
    from paper_2602_17938_gb300 import lacos
    f = lacos.to_device(noisy_with_hits(64, 64, seed=2))
    m = torch.empty((64, 64), dtype=torch.uint8, device="cuda")
    c = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    p = lacos.make_params(1.0, 1.5)
    with lacos.Context(0, hbm_budget_bytes=1024, max_slots=1) as tiny:
        with pytest.raises(lacos.LacosError) as e:
            tiny.submit(f, p, m, c)
        assert e.value.code == lacos.ENOMEM
    with lacos.Context(0, max_slots=1) as one:
        t = one.submit(f, p, m, c)
        with pytest.raises(lacos.LacosError) as e:
            one.submit(f, p, m, c)  # the only slot is held until polled
        assert e.value.code == lacos.EAGAIN
        r = one.wait(t)
        assert r.status == 0
        t2 = one.submit(f, p, m, c)
        assert one.wait(t2).status == 0


def test_batch_equals_single_frames(ctx):
    from paper_2602_17938_gb300 import lacos
    frames = [noisy_with_hits(70, 90, seed=20), noisy_with_hits(33, 200, seed=21),
              noisy_with_hits(128, 64, seed=22, dtype=np.uint16), noisy_with_hits(5, 5, seed=23)]
    niters = [4, 1, 6, 2]
    gains = [1.0, 0.7, 1.3, 2.0]
    dev = [lacos.to_device(x) for x in frames]
    masks = [torch.empty(x.shape, dtype=torch.uint8, device="cuda") for x in frames]
    cleans = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in frames]
    ps = [lacos.make_params(g, 1.5, niter=n) for g, n in zip(gains, niters)]
    for reuse in (False, True, True):
        t, per = ctx.submit_batch(dev, ps, masks, cleans, reuse_graph=reuse)
        agg = ctx.wait(t)
        torch.cuda.synchronize()
        for i, x in enumerate(frames):
            m_ref, c_ref, it_ref, nf_ref = oracle.run(x, gains[i], 1.5, niter=niters[i])
            assert np.array_equal(masks[i].cpu().numpy(), m_ref)
            assert np.array_equal(cleans[i].cpu().numpy().view(np.uint32), c_ref.view(np.uint32))
            assert per[i].iters_run == it_ref and per[i].n_flagged == nf_ref
        assert agg.n_flagged == sum(p.n_flagged for p in per)


def test_batch_mixes_modes_per_frame(ctx):
    # One batched request whose frames use different modes (protection radius,
    # separable medians, dtypes): each frame equals the oracle with its own
    # parameters, through the graph-captured and replayed launches too.
    from paper_2602_17938_gb300 import lacos
    rng = np.random.default_rng(55)
    frames = []
    for i, (shape, dt) in enumerate([((90, 130), np.float32), ((70, 200), np.uint16),
                                      ((129, 64), np.uint16), ((40, 40), np.float32)]):
        f = noisy_with_hits(*shape, seed=60 + i).astype(np.float64)
        for _ in range(3):  # saturated cores with hits nearby
            y, x = int(rng.integers(2, shape[0] - 3)), int(rng.integers(2, shape[1] - 3))
            f[y - 1:y + 2, x - 1:x + 2] = 65535.0
            f[min(y + 3, shape[0] - 1), x] += 2000.0
        frames.append(np.clip(np.rint(f), 0, 65535).astype(np.uint16) if dt == np.uint16 else f.astype(np.float32))
    modes = [dict(satgrow=2), dict(sepmed=True), dict(satgrow=4, sepmed=True), dict()]
    dev = [lacos.to_device(x) for x in frames]
    masks = [torch.empty(x.shape, dtype=torch.uint8, device="cuda") for x in frames]
    cleans = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in frames]
    ps = [lacos.make_params(1.0, 1.5, niter=5, **m) for m in modes]
    for reuse in (False, True, True):
        t, per = ctx.submit_batch(dev, ps, masks, cleans, reuse_graph=reuse)
        ctx.wait(t)
        torch.cuda.synchronize()
        for i, x in enumerate(frames):
            m_ref, c_ref, it_ref, nf_ref = oracle.run(x, 1.0, 1.5, niter=5, **modes[i])
            assert np.array_equal(masks[i].cpu().numpy(), m_ref), i
            assert np.array_equal(cleans[i].cpu().numpy().view(np.uint32), c_ref.view(np.uint32)), i
            assert per[i].iters_run == it_ref and per[i].n_flagged == nf_ref


def _crop_check(frame, spec, mask, clean, boxes, margin=64):
    ny, nx = frame.shape
    for (y0, y1, x0, x1) in boxes:
        cy0, cy1 = max(0, y0 - margin), min(ny, y1 + margin)
        cx0, cx1 = max(0, x0 - margin), min(nx, x1 + margin)
        crop = np.ascontiguousarray(frame[cy0:cy1, cx0:cx1])
        m_ref, c_ref, _, _ = oracle.run(crop, spec.gain, spec.readnoise, niter=spec.niter)
        sy, sx = slice(y0 - cy0, y1 - cy0), slice(x0 - cx0, x1 - cx0)
        assert np.array_equal(mask[y0:y1, x0:x1], m_ref[sy, sx]), (y0, x0)
        assert np.array_equal(clean[y0:y1, x0:x1].view(np.uint32), c_ref[sy, sx].view(np.uint32)), (y0, x0)


def _sample_boxes(ny, nx, rng, n=10, size=48):
    boxes = [(0, size, 0, size), (ny - size, ny, nx - size, nx), (0, size, nx - size, nx),
             (ny - size, ny, 0, size)]
    for _ in range(n):
        y0, x0 = int(rng.integers(0, ny - size)), int(rng.integers(0, nx - size))
        boxes.append((y0, y0 + size, x0, x0 + size))
    return boxes


def test_full_size_61mpx_uint16_every_pixel(ctx):
    # Every pixel against the oracle's whole-frame run (stored digests), and
    # sampled boxes against live oracle runs on crops with a 64-pixel margin.
    from conftest import full_frame_digest_check
    spec = synth.config_specs(1)[0]
    f = synth.make_frame(spec)
    m, c, res = gpu_run(ctx, f, spec.gain, spec.readnoise, niter=spec.niter)
    assert res.status == 0 and res.n_flagged == int(m.sum()) > 0
    full_frame_digest_check(1, 0, f, m, c, res.iters_run, res.n_flagged)
    np.testing.assert_array_equal(c[m == 0], f[m == 0].astype(np.float32))
    _crop_check(f, spec, m, c, _sample_boxes(*f.shape, np.random.default_rng(1)))


def _variant_cases():
    """Frames that cross tile borders of every core-kernel tile shape (32 x 64,
    64 x 64, 32 x 128) with ragged edges, in both dtypes and the optional modes."""
    cases = [(noisy_with_hits(300, 517, seed=71), 1.0, 1.5, {}),
             (noisy_with_hits(97, 130, seed=72, dtype=np.uint16), 1.0, 1.5, {}),
             (noisy_with_hits(70, 61, seed=73), 1.0, 1.5, dict(sepmed=True))]
    spec = synth.FrameSpec(257, 389, "u16", (74, 0), sky=300.0, gain=0.8, readnoise=1.2, n_stars=12,
                           n_tracks=400, hot_frac=0.005, salt_pepper=True)
    sat = synth.make_frame(spec)
    sat[100:104, 127:131] = 65535  # a saturated core across a 128-column tile border
    cases.append((sat, spec.gain, spec.readnoise, dict(satgrow=2)))
    rng = np.random.default_rng(75)
    dense = (100 + 10 * rng.standard_normal((140, 200))).astype(np.float32)
    dense[58:72, 120:136] += rng.uniform(0, 20000, (14, 16)).astype(np.float32)  # widened windows at a border
    cases.append((dense, 1.0, 1.5, {}))
    return cases


def test_every_core_variant_bit_exact(ctx):
    # Every tile shape x occupancy variant the autotuner can pick gives the
    # oracle's result bit for bit.
    from paper_2602_17938_gb300 import lacos
    cases = _variant_cases()
    refs = [oracle.run(f, g, rn, **{"satgrow": kw.get("satgrow", 0), "sepmed": kw.get("sepmed", False)})
            for f, g, rn, kw in cases]
    v0 = ctx.core_variant()
    try:
        for v in range(lacos.CORE_VARIANTS):
            ctx.set_core_variant(v)
            for (f, g, rn, kw), (m_ref, c_ref, it_ref, nf_ref) in zip(cases, refs):
                m, c, res = gpu_run(ctx, f, g, rn, **kw)
                assert np.array_equal(m, m_ref), (v, f.shape, int((m != m_ref).sum()))
                assert np.array_equal(c.view(np.uint32), c_ref.view(np.uint32)), (v, f.shape)
                assert (res.status, res.iters_run, res.n_flagged) == (0, it_ref, nf_ref), (v, f.shape)
    finally:
        ctx.set_core_variant(v0)


def test_core_variants_on_the_batched_path(ctx):
    # A mixed batch (both dtypes) through each tile shape: the per-frame tile
    # ranges of the core and finalize queues differ when the core tile is not
    # 32 x 64.
    from paper_2602_17938_gb300 import lacos
    cases = _variant_cases()[:4]
    refs = [oracle.run(f, g, rn, **{"satgrow": kw.get("satgrow", 0), "sepmed": kw.get("sepmed", False)})
            for f, g, rn, kw in cases]
    d = [lacos.to_device(f) for f, _, _, _ in cases]
    ps = [lacos.make_params(g, rn, **kw) for _, g, rn, kw in cases]
    v0 = ctx.core_variant()
    try:
        for v in (3, 5, 7, 9):
            ctx.set_core_variant(v)
            masks = [torch.empty(f.shape, dtype=torch.uint8, device="cuda") for f in d]
            cleans = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in d]
            t, per = ctx.submit_batch(d, ps, masks, cleans)
            ctx.wait(t)
            torch.cuda.synchronize()
            for i, (m_ref, c_ref, it_ref, nf_ref) in enumerate(refs):
                assert np.array_equal(masks[i].cpu().numpy(), m_ref), (v, i)
                assert np.array_equal(cleans[i].cpu().numpy().view(np.uint32), c_ref.view(np.uint32)), (v, i)
                assert (per[i].iters_run, per[i].n_flagged) == (it_ref, nf_ref), (v, i)
    finally:
        ctx.set_core_variant(v0)


@pytest.mark.parametrize("dtype", [np.uint16, np.float32])
def test_unaligned_output_buffers(ctx, dtype):
    # The ABI takes any output pointers: a cleaned frame that is not 16-byte aligned and a mask
    # that is not 4-byte aligned (views one element into larger buffers) take the finalize
    # kernel's scalar stores and must give the same result as aligned buffers.
    from paper_2602_17938_gb300 import lacos
    ny, nx = 130, 256  # nx a multiple of 4: aligned outputs would take the vector stores
    f = noisy_with_hits(ny, nx, seed=77, dtype=dtype)
    cbuf = torch.empty(ny * nx + 1, dtype=torch.float32, device="cuda")
    mbuf = torch.empty(ny * nx + 1, dtype=torch.uint8, device="cuda")
    clean, mask = cbuf[1:].view(ny, nx), mbuf[1:].view(ny, nx)
    assert clean.data_ptr() % 16 != 0 and mask.data_ptr() % 4 != 0
    p = lacos.make_params(1.0, 1.5)
    res = ctx.wait(ctx.submit(lacos.to_device(f), p, mask, clean))
    torch.cuda.synchronize()
    assert_same(f, 1.0, 1.5, (mask.cpu().numpy(), clean.cpu().numpy(), res))
