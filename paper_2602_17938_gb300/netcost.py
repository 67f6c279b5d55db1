"""Static min/max operation counts of the selection networks the kernels run.

The detect kernel's "algorithmic" work, used for its ALU roofline, is the
number of two-input min/max operations its median networks perform per
output pixel and iteration (dense part) plus the data-dependent sparse parts
(S' = S - med5(S) where S exceeds the lower threshold, the fine-structure
image where S' exceeds sigclip, and masked-median replacements), each
counted from the generated network.  Halo recomputation is not counted.
"""
from __future__ import annotations

import functools
import importlib.util
import os

_GEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "gen_networks.py")


@functools.lru_cache(maxsize=1)
def counts() -> dict:
    spec = importlib.util.spec_from_file_location("gen_networks", _GEN)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    nets = gen.build_all()
    c = {name: gen.count_ops(d, o) for name, (d, o, _, _) in nets.items()}
    c["dense_med5_per_px"] = c["med5x5"]
    c["fine_per_px"] = 49 * c["med3x3"] + c["med7x7"]
    c["naive_med5_per_px"] = 25 * 24  # full sort by pairwise compare-exchange, for reference
    return c


def detect_minmax_ops(profile: dict) -> int:
    """Min/max operations of all detect launches of one request."""
    c = counts()
    return (profile["px_iterations"] * c["dense_med5_per_px"]
            + profile["n_sprime"] * c["med5x5"]
            + profile["n_fine"] * c["fine_per_px"]
            + profile["n_replace"] * c["med5x5"])
