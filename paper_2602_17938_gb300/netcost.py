"""Static min/max operation counts of the selection networks the kernels run.

The core kernel's "algorithmic" work, used for its ALU roofline, is the
number of two-input min/max operations its median networks perform per
output pixel and iteration -- the shared-block med5 (for N) and med3
networks, per output -- plus the data-dependent S' = S - med5(S) at the
pixels where S exceeds the lower threshold (standalone med5 network).
Halo recomputation is not counted.  The fine and replace kernels' work is
counted the same way from their networks.
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
    blk5 = nets["blk_med5_4x2"]
    blk3 = nets["blk_med3_8x2"]
    c["dense_med5_per_px"] = c["blk_med5_4x2"] / len(blk5[1])
    c["dense_med3_per_px"] = c["blk_med3_8x2"] / len(blk3[1])
    c["fine_per_px"] = c["med7x7"] + c["med5x5"]
    c["naive_med5_per_px"] = 25 * 24  # full sort by pairwise compare-exchange, for reference
    return c


def detect_minmax_ops(profile: dict) -> int:
    """Min/max operations of all detect launches of one request: the dense
    networks at the tile pixels the core kernel computed (a level skips the
    tiles whose inputs did not change) and med5 at each S' evaluation."""
    c = counts()
    px = profile.get("px_core", profile["px_iterations"])
    return int(px * (c["dense_med5_per_px"] + c["dense_med3_per_px"])
               + profile["n_sprime"] * c["med5x5"])


def detect_work(profile: dict, packed: bool) -> dict:
    """Algorithmic min/max work of the core launches of one request, split by
    kind and counted in instructions as well as element operations.

    * dense: the shared-block med5 (noise model) and med3 networks at every
      tile pixel the core kernel computed; on uint16 frames one packed
      min/max.u16x2 instruction serves two outputs (``packed``);
    * sprime: the standalone med5 of S at each S' evaluation (float keys);
    * fine: the med7 of med3 at each fine-structure evaluation (one lane).
    The masked-median replacement is not counted (its per-tile list includes
    the halo that neighbouring tiles recompute)."""
    c = counts()
    px = profile.get("px_core", profile["px_iterations"])
    dense = px * (c["dense_med5_per_px"] + c["dense_med3_per_px"])
    sprime = profile["n_sprime"] * c["med5x5"]
    fine = profile["n_fine"] * c["med7x7"]
    return {"dense_elem": dense, "dense_instr": dense / 2 if packed else dense,
            "sprime_instr": sprime, "fine_instr": fine,
            "instr": (dense / 2 if packed else dense) + sprime + fine}


def fine_minmax_ops(profile: dict) -> int:
    return int(profile["n_fine"] * counts()["fine_per_px"])


def replace_minmax_ops(profile: dict) -> int:
    return int(profile["n_replace"] * counts()["med5x5"])
