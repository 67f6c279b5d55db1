"""Static operation counts of the selection networks and rank tests the kernels run.

The core kernel's "algorithmic" work, used for its ALU roofline, is the
number of two-input min/max operations its median networks perform per
output pixel and iteration -- the shared-block med5 (for N) and med3
networks, per output -- plus the data-dependent sparse work: at each S'
item either the standalone med5 network (fine-structure items, and every
item in the separable-median mode) or the lo test decided by rank (one
comparison per window value, 25), and at each F evaluation either the med7
network (float32 frames) or the objlim test decided by rank (49
comparisons).  Halo recomputation is not counted.  The fine and replace
kernels' work is counted the same way from their networks.
"""
from __future__ import annotations

import functools
import importlib.util
import os

# Comparisons of a rank test: one per window value (5x5 for the lo test of S',
# 7x7 for the objlim test of F).
RANK_TEST_LO = 25
RANK_TEST_OBJLIM = 49

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


def detect_work(profile: dict, packed: bool) -> dict:
    """Algorithmic ALU work of the core launches of one request, split by
    kind and counted in instructions as well as element operations.

    * dense: the shared-block med5 (noise model) and med3 networks at every
      tile pixel the core kernel computed; on uint16 frames one packed
      min/max.u16x2 instruction serves two outputs (``packed``);
    * sprime: the standalone med5 of S at each S' evaluation that runs the
      network, and 25 comparisons at each one decided by rank (float keys);
    * fine: the med7 of med3 at each fine-structure evaluation that runs the
      network, and 49 comparisons at each one decided by rank (one lane).
    The masked-median replacement is not counted (its per-tile list includes
    the halo that neighbouring tiles recompute).  ``*_as_networks`` gives the
    same medians costed as if every one ran its network."""
    c = counts()
    px = profile.get("px_core", profile["px_iterations"])
    dense = px * (c["dense_med5_per_px"] + c["dense_med3_per_px"])
    n_s, n_f = profile["n_sprime"], profile["n_fine"]
    n_s_net = profile.get("n_sprime_net", n_s)
    n_f_net = profile.get("n_fine_net", n_f)
    sprime = n_s_net * c["med5x5"] + (n_s - n_s_net) * RANK_TEST_LO
    fine = n_f_net * c["med7x7"] + (n_f - n_f_net) * RANK_TEST_OBJLIM
    dense_i = dense / 2 if packed else dense
    return {"dense_elem": dense, "dense_instr": dense_i,
            "sprime_instr": sprime, "fine_instr": fine,
            "instr": dense_i + sprime + fine,
            "instr_as_networks": dense_i + n_s * c["med5x5"] + n_f * c["med7x7"]}
