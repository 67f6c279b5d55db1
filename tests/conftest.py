import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def full_frame_digest_check(cfg, index, frame, mask, clean, iters_run, n_flagged):
    """Every pixel of a full-size workload frame against the float32 oracle run
    on the whole frame: tests/golden/full_frame_digests.json holds SHA-256
    digests of the oracle's uint8 mask and float32 cleaned frame, written by
    tests/golden/make_full_frame_digests.py (oracle and input generator only).
    The input's digest is checked first, so a generator that drew a different
    frame is reported as such."""
    import hashlib
    import json

    import numpy as np
    with open(os.path.join(ROOT, "tests", "golden", "full_frame_digests.json")) as f:
        ent = json.load(f)[f"c{cfg}/{index}"]
    h = lambda a: hashlib.sha256(memoryview(np.ascontiguousarray(a)).cast("B")).hexdigest()
    assert h(frame) == ent["input_sha256"], f"c{cfg}/{index}: the generator drew another input"
    assert (iters_run, n_flagged) == (ent["iters_run"], ent["n_flagged"]), f"c{cfg}/{index}"
    assert h(mask) == ent["mask_sha256"], f"c{cfg}/{index}: mask differs from the oracle's"
    assert h(np.ascontiguousarray(clean, dtype="<f4")) == ent["clean_sha256"], \
        f"c{cfg}/{index}: cleaned frame differs from the oracle's"
