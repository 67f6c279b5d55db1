"""Serving (continuous admission, overlapping requests) and the core-variant autotuner.

Every request's mask and cleaned frame must be identical -- bit for bit,
the tolerance of every GPU test here -- whether it runs alone or in a mix
of overlapping requests of other sizes, dtypes and parameters, and
whichever core-kernel variant runs it.
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


def _frame(ny, nx, seed, dtype=np.float32, sky=100.0):
    rng = np.random.default_rng(seed)
    f = sky + math.sqrt(sky + 2.25) * rng.standard_normal((ny, nx))
    n = max(1, ny * nx // 100)
    f[rng.integers(0, ny, n), rng.integers(0, nx, n)] += rng.uniform(200, 4000, n)
    if dtype == np.uint16:
        return np.clip(np.rint(f), 0, 65535).astype(np.uint16)
    return f.astype(np.float32)


def _mix(lacos):
    shapes = [(300, 410, np.float32), (517, 260, np.uint16), (96, 1000, np.float32),
              (640, 640, np.uint16), (33, 77, np.float32), (450, 455, np.uint16)]
    frames = [_frame(ny, nx, 40 + i, dt) for i, (ny, nx, dt) in enumerate(shapes)]
    params = [lacos.make_params(0.6 + 0.2 * i, 1.0 + 0.3 * i, niter=(1, 4, 6)[i % 3],
                                sigclip=(4.5, 4.0, 5.0)[i % 3]) for i in range(len(frames))]
    return frames, params


def test_each_result_same_alone_and_in_the_mix(lib):
    from paper_2602_17938_gb300 import serve
    lacos = lib
    frames, params = _mix(lacos)
    dev = [lacos.to_device(f) for f in frames]
    alone = []
    with lacos.Context(0) as ctx:
        for d, p in zip(dev, params):
            m = torch.empty(d.shape, dtype=torch.uint8, device="cuda")
            c = torch.empty(d.shape, dtype=torch.float32, device="cuda")
            r = ctx.wait(ctx.submit(d, p, m, c))
            alone.append((m.cpu(), c.cpu(), r))
    # 3 rounds of the 6 frames, all arriving at once: up to 18 requests overlap.
    reqs = [serve.Request(dev[i % 6], params[i % 6], 0.0) for i in range(18)]
    with serve.Server(0, hbm_budget_bytes=4 << 30, max_slots=18, keep_outputs=True) as srv:
        st = srv.run(reqs)
        torch.cuda.synchronize()
        assert st.n == 18 and st.max_in_flight > 1
        for rec in st.records:
            m, c, r = alone[rec.index % 6]
            assert rec.result.status == 0
            assert rec.result.n_flagged == r.n_flagged and rec.result.iters_run == r.iters_run
            assert torch.equal(rec.mask.cpu(), m)
            assert torch.equal(rec.clean.cpu().view(torch.int32), c.view(torch.int32))
    # and the alone results are the oracle's
    for f, p, (m, c, r) in zip(frames, params, alone):
        mr, cr, it, nf = oracle.run(f, p.gain, p.readnoise, p.satlevel, p.sigclip, p.sigfrac,
                                    p.objlim, p.niter)
        assert np.array_equal(m.numpy(), mr) and np.array_equal(c.numpy().view(np.uint32), cr.view(np.uint32))


def test_budget_limits_requests_in_flight(lib):
    from paper_2602_17938_gb300 import serve
    lacos = lib
    f = lacos.to_device(_frame(512, 512, 5))
    p = lacos.make_params(1.0, 1.5)
    with serve.Server(0, hbm_budget_bytes=1, max_slots=8) as srv:
        one = srv._request_bytes(512, 512, p)
    # room for one request at a time (plus the context's scratch for it)
    with serve.Server(0, hbm_budget_bytes=int(1.5 * one), max_slots=8) as srv:
        st = srv.run([serve.Request(f, p, 0.0) for _ in range(5)])
        assert st.n == 5 and st.max_in_flight == 1
    with serve.Server(0, hbm_budget_bytes=int(3.5 * one), max_slots=8) as srv:
        st = srv.run([serve.Request(f, p, 0.0) for _ in range(6)])
        assert st.n == 6 and 1 < st.max_in_flight <= 3


def test_poisson_stream_completes(lib):
    from paper_2602_17938_gb300 import serve
    lacos = lib
    frames, params = _mix(lacos)
    dev = [lacos.to_device(f) for f in frames]
    reqs = serve.poisson_requests(dev, params, rate_hz=400.0, n=24)
    with serve.Server(0, hbm_budget_bytes=4 << 30, max_slots=16) as srv:
        st = srv.run(reqs)
    assert st.n == 24 and all(r.result.status == 0 for r in st.records)
    assert 0 < st.p50_ms <= st.p99_ms and st.mpix_per_s > 0


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_every_core_variant_bit_exact_and_autotune(lib, dtype, tmp_path, monkeypatch):
    lacos = lib
    f = _frame(333, 517, 9, dtype)
    d = lacos.to_device(f)
    p = lacos.make_params(1.0, 1.5, niter=4)
    mr, cr, it, nf = oracle.run(f, 1.0, 1.5)
    m = torch.empty(f.shape, dtype=torch.uint8, device="cuda")
    c = torch.empty(f.shape, dtype=torch.float32, device="cuda")
    with lacos.Context(0) as ctx:
        for v in range(lacos.CORE_VARIANTS):
            ctx.set_core_variant(v)
            assert ctx.core_variant() == v
            r = ctx.wait(ctx.submit(d, p, m, c))
            assert r.iters_run == it and r.n_flagged == nf
            assert np.array_equal(m.cpu().numpy(), mr)
            assert np.array_equal(c.cpu().numpy().view(np.uint32), cr.view(np.uint32))
        monkeypatch.setenv("LACOS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
        from paper_2602_17938_gb300 import autotune
        best, ms = autotune.tune(ctx, d, p, m, c, reps=1)
        assert 0 <= best < lacos.CORE_VARIANTS and ctx.core_variant() == best and len(ms) == lacos.CORE_VARIANTS
        best2, ms2 = autotune.tune(ctx, d, p, m, c)  # from the cache
        assert best2 == best and ms2 is None


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_host_requests_match_device_requests(lib, dtype):
    lacos = lib
    frames = [_frame(ny, nx, 70 + i, dtype) for i, (ny, nx) in enumerate([(300, 410), (517, 260), (96, 1000)])]
    p = lacos.make_params(1.1, 1.4, niter=4)
    tdt = torch.uint16 if dtype == np.uint16 else torch.float32
    with lacos.Context(0) as ctx:
        ref = []
        for f in frames:
            d = lacos.to_device(f)
            m = torch.empty(f.shape, dtype=torch.uint8, device="cuda")
            c = torch.empty(f.shape, dtype=torch.float32, device="cuda")
            r = ctx.wait(ctx.submit(d, p, m, c))
            ref.append((m.cpu(), c.cpu(), r))
        h_frames = [torch.from_numpy(f.view(np.int16) if dtype == np.uint16 else f).pin_memory().view(tdt)
                    for f in frames]
        h_masks = [torch.zeros(f.shape, dtype=torch.uint8).pin_memory() for f in frames]
        h_cleans = [torch.zeros(f.shape, dtype=torch.float32).pin_memory() for f in frames]
        # one at a time, then streamed with two in flight (mixed sizes reuse the slots' buffers)
        for i in range(len(frames)):
            r = lacos.clean_host(h_frames[i], p, h_masks[i], h_cleans[i], ctx=ctx)
            assert r.status == 0 and r.n_flagged == ref[i][2].n_flagged
            assert torch.equal(h_masks[i], ref[i][0])
            assert torch.equal(h_cleans[i].view(torch.int32), ref[i][1].view(torch.int32))
            h_masks[i].zero_()
            h_cleans[i].zero_()
        order = [2, 0, 1, 2, 1, 0]
        res = lacos.clean_host_stream(ctx, [h_frames[j] for j in order], p,
                                      [h_masks[j] for j in order], [h_cleans[j] for j in order], depth=2)
        assert [r.n_flagged for r in res] == [ref[j][2].n_flagged for j in order]
        for i in range(len(frames)):
            assert torch.equal(h_masks[i], ref[i][0])
            assert torch.equal(h_cleans[i].view(torch.int32), ref[i][1].view(torch.int32))


def test_chained_and_concurrent_host_requests_match_device_requests(lib):
    # Host frames of 8 or more GPU waves of 32x64 tiles run their kernels one
    # request at a time (2688 x 4096 = 5376 tiles; 8 waves of 152 SMs x 4 CTAs
    # are 4864); the small frame runs concurrently beside them.
    lacos = lib
    specs = [(2688, 4096, np.uint16), (300, 410, np.float32), (2688, 4096, np.float32)]
    frames = [_frame(ny, nx, 90 + i, dt) for i, (ny, nx, dt) in enumerate(specs)]
    p = lacos.make_params(1.0, 1.5, niter=4)
    with lacos.Context(0) as ctx:
        ref = []
        for f in frames:
            d = lacos.to_device(f)
            m = torch.empty(f.shape, dtype=torch.uint8, device="cuda")
            c = torch.empty(f.shape, dtype=torch.float32, device="cuda")
            r = ctx.wait(ctx.submit(d, p, m, c))
            ref.append((m.cpu(), c.cpu(), r))
        h_frames = [torch.from_numpy(f.view(np.int16)).pin_memory().view(torch.uint16) if f.dtype == np.uint16
                    else torch.from_numpy(f).pin_memory() for f in frames]
        order = [0, 1, 2, 0, 2, 1, 0, 2]
        h_masks = [torch.zeros(frames[j].shape, dtype=torch.uint8).pin_memory() for j in order]
        h_cleans = [torch.zeros(frames[j].shape, dtype=torch.float32).pin_memory() for j in order]
        res = lacos.clean_host_stream(ctx, [h_frames[j] for j in order], p, h_masks, h_cleans, depth=3)
        for k, j in enumerate(order):
            assert res[k].status == 0 and res[k].n_flagged == ref[j][2].n_flagged, (k, j)
            assert torch.equal(h_masks[k], ref[j][0]), (k, j)
            assert torch.equal(h_cleans[k].view(torch.int32), ref[j][1].view(torch.int32)), (k, j)
