"""The no-allocation entry point against the regular one.

lacos_run_static serves callers that may not allocate device memory while
they run (a pipeline with a fixed up-front memory plan, a plugin whose host
owns the device allocator): its scratch is a fixed array inside the
library.  Here it must give the same mask and cleaned frame as lacos_submit
-- bit for bit, the tolerance of every GPU test in this suite -- on two
calls in a row (the array keeps the first call's contents, which the second
call must not see), and reject a frame whose scratch exceeds the array.
This file is collected last so a failure here stops a run only after every
other test has run; it also passes alone in a fresh process.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _frame(ny, nx, seed, dtype=np.float32):
    rng = np.random.default_rng(seed)
    sky, gain, rn = 120.0, 1.0, 1.5
    f = sky + math.sqrt(gain * sky + rn * rn) / gain * rng.standard_normal((ny, nx))
    n = ny * nx // 120
    f[rng.integers(0, ny, n), rng.integers(0, nx, n)] += rng.uniform(200, 4000, n)
    if dtype == np.uint16:
        return np.clip(np.rint(f), 0, 65535).astype(np.uint16)
    return f.astype(np.float32)


def test_static_entry_point_matches_submit_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17938_gb300 import build, lacos
    build.build()
    sat = _frame(300, 400, 3, np.uint16)
    sat[100:103, 200:203] = 65535  # a saturated core for the protection mode
    cases = [(_frame(700, 901, 1), 1.0, 4, {}), (_frame(513, 640, 2, np.uint16), 0.8, 6, {}),
             (sat, 1.0, 4, dict(satgrow=3)), (_frame(256, 320, 4), 1.2, 4, dict(sepmed=True))]
    with lacos.Context(0) as ctx:
        for frame, gain, niter, mode in cases:
            d = lacos.to_device(frame)
            p = lacos.make_params(gain, 1.5, niter=niter, **mode)
            m_ref = torch.empty(frame.shape, dtype=torch.uint8, device="cuda")
            c_ref = torch.empty(frame.shape, dtype=torch.float32, device="cuda")
            r_ref = ctx.wait(ctx.submit(d, p, m_ref, c_ref))
            m = torch.full(frame.shape, 7, dtype=torch.uint8, device="cuda")
            c = torch.full(frame.shape, -1.0, dtype=torch.float32, device="cuda")
            r = lacos.run_static(d, p, m, c)
            torch.cuda.synchronize()
            assert r.status == 0 and r_ref.status == 0
            assert r.iters_run == r_ref.iters_run and r.n_flagged == r_ref.n_flagged > 0
            assert torch.equal(m, m_ref)
            assert torch.equal(c.view(torch.int32), c_ref.view(torch.int32))
            assert r.latency_ms > 0.0  # host time of the blocking call
        # The first case also straight against the float32 CPU oracle.
        frame, gain, niter, _ = cases[0]
        d = lacos.to_device(frame)
        m = torch.empty(frame.shape, dtype=torch.uint8, device="cuda")
        c = torch.empty(frame.shape, dtype=torch.float32, device="cuda")
        r = lacos.run_static(d, lacos.make_params(gain, 1.5, niter=niter), m, c)
        m_o, c_o, it_o, nf_o = oracle.run(frame, gain, 1.5, niter=niter)
        assert r.status == 0 and r.iters_run == it_o and r.n_flagged == nf_o
        assert np.array_equal(m.cpu().numpy(), m_o)
        assert np.array_equal(c.cpu().numpy().view(np.uint32), c_o.view(np.uint32))


def test_static_entry_point_rejects_oversize_frames():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17938_gb300 import build, lacos
    build.build()
    ny, nx = 12000, 12000  # about 86 MiB of scratch > 64 MiB
    assert lacos.load_library().lacos_scratch_bytes(ny, nx) > lacos.STATIC_SCRATCH_BYTES
    d = torch.zeros((ny, nx), dtype=torch.uint16, device="cuda")
    m = torch.empty((ny, nx), dtype=torch.uint8, device="cuda")
    c = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    with pytest.raises(lacos.LacosError) as e:
        lacos.run_static(d, lacos.make_params(1.0, 1.5), m, c)
    assert e.value.code == lacos.ENOMEM


def test_static_limit_depends_on_the_saturation_plane():
    # A frame just inside the array with five bit-planes runs; with saturated-star
    # protection (a sixth plane) the same frame no longer fits and is rejected.
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2602_17938_gb300 import build, lacos
    build.build()
    lib = lacos.load_library()
    ny, nx = 10000, 9576
    p0, p1 = lacos.make_params(1.0, 1.5, niter=2), lacos.make_params(1.0, 1.5, niter=2, satgrow=1)
    assert lib.lacos_request_bytes(ny, nx, ctypes.byref(p0)) <= lacos.STATIC_SCRATCH_BYTES
    assert lib.lacos_request_bytes(ny, nx, ctypes.byref(p1)) > lacos.STATIC_SCRATCH_BYTES
    g = torch.Generator(device="cuda").manual_seed(10000)
    f = torch.randn((ny, nx), generator=g, device="cuda").mul_(11.0).add_(120.0)
    idx = torch.randint(0, ny * nx, (ny * nx // 200,), generator=g, device="cuda")
    f.view(-1).index_add_(0, idx, torch.rand(idx.numel(), generator=g, device="cuda").mul_(3000.0).add_(200.0))
    d = f.round_().clamp_(0, 65535).to(torch.int32).to(torch.int16).view(torch.uint16)
    del f, idx
    m = torch.empty((ny, nx), dtype=torch.uint8, device="cuda")
    c = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    r = lacos.run_static(d, p0, m, c)
    m_ref = torch.empty_like(m)
    c_ref = torch.empty_like(c)
    with lacos.Context(0) as ctx:
        r_ref = ctx.wait(ctx.submit(d, p0, m_ref, c_ref))
    torch.cuda.synchronize()
    assert r.status == 0 and r.n_flagged == r_ref.n_flagged > 0 and r.iters_run == r_ref.iters_run
    assert torch.equal(m, m_ref) and torch.equal(c.view(torch.int32), c_ref.view(torch.int32))
    with pytest.raises(lacos.LacosError) as e:
        lacos.run_static(d, p1, m, c)
    assert e.value.code == lacos.ENOMEM
