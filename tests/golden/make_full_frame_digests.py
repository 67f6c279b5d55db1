#!/usr/bin/env python
"""Write full_frame_digests.json: the float32 oracle's results on whole frames.

For every frame of the full-size workloads -- the 61-Mpx uint16 frame, all 64
frames of the mixed batch, and every 8th frame of the 256-frame stress set
(all three niter values) -- this script draws the frame with the seeded
generator, runs the CPU oracle on the WHOLE frame (no crops, so no margin
argument is involved) and stores SHA-256 digests of the input, of the uint8
mask and of the float32 cleaned frame, with iters_run and n_flagged.  The GPU
tests hash their outputs the same way, so every pixel of every frame is
compared bit for bit with the oracle without re-running it.

Only the oracle and the input generator are called here; nothing comes from
the CUDA path.  Frames run one per process over all host cores (spawned
workers; a 61-Mpx frame holds about 3 GB in the oracle).  Entries already in
the output file are kept, so the script can be stopped and resumed.

    python tests/golden/make_full_frame_digests.py [--jobs N] [--only 1,2,4]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "full_frame_digests.json")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def frame_list(only=(1, 2, 4)):
    """(config index, frame index, spec) of the frames the digests cover."""
    from paper_2602_17938_gb300 import synth
    out = []
    for cfg in only:
        specs = synth.config_specs(cfg)
        idx = range(0, len(specs), 8) if cfg == 4 else range(len(specs))
        out += [(cfg, i, specs[i]) for i in idx]
    return out


def entry_key(cfg: int, i: int) -> str:
    return f"c{cfg}/{i}"


def sha256(a) -> str:
    return hashlib.sha256(memoryview(a).cast("B")).hexdigest()


def _one(job):
    cfg, i = job
    import numpy as np

    import oracle
    from paper_2602_17938_gb300 import synth
    spec = (synth.config_specs(cfg))[i]
    frame = synth.make_frame(spec)
    t0 = time.perf_counter()
    mask, clean, iters, nflag = oracle.run(frame, spec.gain, spec.readnoise, spec.satlevel, spec.sigclip,
                                           spec.sigfrac, spec.objlim, spec.niter)
    dt = time.perf_counter() - t0
    return entry_key(cfg, i), {
        "config": cfg, "frame": i, "seed": list(spec.seed), "ny": spec.ny, "nx": spec.nx, "dtype": spec.dtype,
        "gain": spec.gain, "readnoise": spec.readnoise, "satlevel": spec.satlevel, "sigclip": spec.sigclip,
        "sigfrac": spec.sigfrac, "objlim": spec.objlim, "niter": spec.niter,
        "input_sha256": sha256(np.ascontiguousarray(frame)),
        "mask_sha256": sha256(np.ascontiguousarray(mask)),
        "clean_sha256": sha256(np.ascontiguousarray(clean, dtype="<f4")),
        "iters_run": int(iters), "n_flagged": int(nflag), "oracle_s": round(dt, 1)}


def load(path=OUT) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default="1,2,4", help="config indices (1: 61-Mpx frame, 2: batch, 4: stress)")
    args = ap.parse_args()
    only = tuple(int(v) for v in args.only.split(","))
    import oracle
    oracle.build()
    have = load()
    todo = [(cfg, i, sp) for cfg, i, sp in frame_list(only) if entry_key(cfg, i) not in have]
    todo.sort(key=lambda t: -t[2].npix * t[2].niter)  # longest first
    print(f"{len(todo)} frames to run on {args.jobs} processes", flush=True)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(args.jobs) as pool:
        for key, ent in pool.imap_unordered(_one, [(c, i) for c, i, _ in todo]):
            have[key] = ent
            tmp = OUT + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(dict(sorted(have.items())), f, indent=1)
            os.replace(tmp, OUT)
            print(f"{key}: {ent['oracle_s']} s, {ent['n_flagged']} flagged, "
                  f"{time.perf_counter() - t0:.0f} s elapsed", flush=True)


if __name__ == "__main__":
    main()
