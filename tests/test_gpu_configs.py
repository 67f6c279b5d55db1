"""Full-size workloads through the batched launch, checked against the oracle.

* The 64-frame batch (16x 2048x2048 f32, 16x 4096x3072 u16, 32x 9576x6388
  u16; per-frame gain and read noise) in one request, replayed from its
  CUDA graph.
* The stress set (9576x6388 u16, 5x the cosmic-ray rate, 1% hot pixels,
  saturated stars clipped at 65535, niter 1/4/6 per frame): a deterministic
  subset -- every 8th of the 256 frames, all three niter values -- in one
  batched request.

Outputs are compared bit for bit with the float32 oracle on sampled boxes
(the oracle runs a crop with a 64-pixel margin, more than six iterations
can reach), and every frame satisfies the any-size properties: cleaned
equals input outside the mask and the flagged count equals the mask's sum.
"""
import numpy as np
import pytest

import oracle
from paper_2602_17938_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lacos():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17938_gb300 import build, lacos as lc
    build.build()
    return lc


def _boxes(frame, rng, n=3, size=40, sat_box=False):
    ny, nx = frame.shape
    boxes = [(0, size, 0, size), (ny - size, ny, nx - size, nx)]
    for _ in range(n):
        y0, x0 = int(rng.integers(0, ny - size)), int(rng.integers(0, nx - size))
        boxes.append((y0, y0 + size, x0, x0 + size))
    if sat_box:
        ys, xs = np.nonzero(frame == 65535)
        if len(ys):
            y0 = int(np.clip(ys[0] - size // 2, 0, ny - size))
            x0 = int(np.clip(xs[0] - size // 2, 0, nx - size))
            boxes.append((y0, y0 + size, x0, x0 + size))
    return boxes


def _check(frame, spec, mask, clean, boxes, margin=64):
    ny, nx = frame.shape
    for (y0, y1, x0, x1) in boxes:
        cy0, cy1 = max(0, y0 - margin), min(ny, y1 + margin)
        cx0, cx1 = max(0, x0 - margin), min(nx, x1 + margin)
        crop = np.ascontiguousarray(frame[cy0:cy1, cx0:cx1])
        m_ref, c_ref, _, _ = oracle.run(crop, spec.gain, spec.readnoise, spec.satlevel, spec.sigclip,
                                        spec.sigfrac, spec.objlim, spec.niter)
        sy, sx = slice(y0 - cy0, y1 - cy0), slice(x0 - cx0, x1 - cx0)
        assert np.array_equal(mask[y0:y1, x0:x1], m_ref[sy, sx]), (spec.seed, y0, x0)
        assert np.array_equal(clean[y0:y1, x0:x1].view(np.uint32), c_ref[sy, sx].view(np.uint32)), \
            (spec.seed, y0, x0)


def _run_batch(lacos, frames, specs, reuse_graph):
    dev = [lacos.to_device(f) for f in frames]
    masks = [torch.empty(f.shape, dtype=torch.uint8, device="cuda") for f in frames]
    cleans = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in frames]
    ps = [lacos.make_params(s.gain, s.readnoise, s.satlevel, s.sigclip, s.sigfrac, s.objlim, s.niter)
          for s in specs]
    with lacos.Context(0, hbm_budget_bytes=32 << 30) as ctx:
        t, per = ctx.submit_batch(dev, ps, masks, cleans, reuse_graph=reuse_graph)
        ctx.wait(t)
        if reuse_graph:  # replay the captured graph and keep its outputs
            t, per = ctx.submit_batch(dev, ps, masks, cleans, reuse_graph=True)
            ctx.wait(t)
        torch.cuda.synchronize()
        results = [(p.status, p.iters_run, p.n_flagged) for p in per]
    del dev
    return masks, cleans, results


def _invariants(frame, mask, clean, result):
    status, iters, flagged = result
    assert status == 0 and flagged == int(mask.sum())
    keep = mask == 0
    assert np.array_equal(clean[keep], frame[keep].astype(np.float32))


def test_batch_of_64_mixed_frames(lacos):
    specs = synth.config_specs(2)
    frames = synth.make_frames_parallel(specs)
    masks, cleans, results = _run_batch(lacos, frames, specs, reuse_graph=True)
    rng = np.random.default_rng(202)
    for i, (f, sp) in enumerate(zip(frames, specs)):
        m, c = masks[i].cpu().numpy(), cleans[i].cpu().numpy()
        _invariants(f, m, c, results[i])
        if i in (0, 15, 16, 31, 32, 63):
            _check(f, sp, m, c, _boxes(f, rng))


def test_stress_subset_one_batched_launch(lacos):
    specs = synth.config_specs(4)[::8]
    assert {s.niter for s in specs} == {1, 4, 6}
    frames = synth.make_frames_parallel(specs)
    masks, cleans, results = _run_batch(lacos, frames, specs, reuse_graph=False)
    rng = np.random.default_rng(404)
    checked = set()
    for i, (f, sp) in enumerate(zip(frames, specs)):
        m, c = masks[i].cpu().numpy(), cleans[i].cpu().numpy()
        _invariants(f, m, c, results[i])
        assert results[i][1] <= sp.niter
        assert not m[f == 65535].any()  # saturated pixels are never flagged
        if sp.niter not in checked:
            checked.add(sp.niter)
            _check(f, sp, m, c, _boxes(f, rng, sat_box=True))
    assert checked == {1, 4, 6}
