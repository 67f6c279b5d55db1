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
