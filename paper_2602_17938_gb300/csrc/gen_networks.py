"""Generator for the branch-free min/max selection networks used by the kernels.

Writes ``networks.cuh``.  Every network is straight-line code of two-input
``MN``/``MX`` (min/max) operations in SSA form, so the same text serves any
key type that defines them (float, 32-bit integers, packed u16x2).

Construction (standard results, written from their definitions):
  * K. E. Batcher's odd-even merge (1968) for merging sorted lists of any
    length, applied recursively to sort;
  * the separable "sort columns, then merge" median of Adams (2021, ACM TOG
    40(4), "Fast median filters using separable sorting networks"): a K x K
    median is the rank-(K*K-1)/2 element of the union of K sorted columns,
    and neighbouring outputs share column sorts and partial merges;
  * dead-code pruning: only operations that feed a requested output are
    emitted, a comparator whose max (or min) is unused costs one operation,
    and operations on +/-infinity sentinels are folded away.

Run as a script to regenerate the header; the tests re-run ``verify()``.
"""
from __future__ import annotations

import itertools
import os
import random
import sys

NEG, POS = "-inf", "+inf"


class Dag:
    """SSA min/max DAG with constant folding and common-subexpression reuse."""

    def __init__(self):
        self.ops = []  # (kind, a, b) ; node id = index + n_inputs offset via names
        self.memo = {}
        self.names = []  # node names: inputs are ("in", k)

    def inp(self, label):
        self.names.append(("in", label))
        return len(self.names) - 1

    def _op(self, kind, a, b):
        if a == b:
            return a
        if kind == "min":
            if a == NEG or b == NEG:
                return NEG
            if a == POS:
                return b
            if b == POS:
                return a
        else:
            if a == POS or b == POS:
                return POS
            if a == NEG:
                return b
            if b == NEG:
                return a
        key = (kind, min(a, b, key=str), max(a, b, key=str))
        if key in self.memo:
            return self.memo[key]
        self.names.append((kind, a, b))
        nid = len(self.names) - 1
        self.memo[key] = nid
        return nid

    def mn(self, a, b):
        return self._op("min", a, b)

    def mx(self, a, b):
        return self._op("max", a, b)

    def cmpx(self, lst, i, j):
        a, b = lst[i], lst[j]
        lst[i], lst[j] = self.mn(a, b), self.mx(a, b)

    # -- Batcher odd-even merge of two sorted lists (any lengths) ------------
    def merge(self, a, b):
        """Merge sorted lists a and b into one sorted list (Batcher)."""
        if not a:
            return list(b)
        if not b:
            return list(a)
        if len(a) == 1 and len(b) == 1:
            return [self.mn(a[0], b[0]), self.mx(a[0], b[0])]
        # pad both to a common power of two with +inf so the classic
        # recursion applies; the sentinels fold away.
        n = 1
        while n < max(len(a), len(b)):
            n *= 2
        A = list(a) + [POS] * (n - len(a))
        B = list(b) + [POS] * (n - len(b))
        out = self._merge_pow2(A, B)
        return out[:len(a) + len(b)]

    def _merge_pow2(self, A, B):
        n = len(A)
        if n == 1:
            return [self.mn(A[0], B[0]), self.mx(A[0], B[0])]
        ev = self._merge_pow2(A[0::2], B[0::2])
        od = self._merge_pow2(A[1::2], B[1::2])
        out = [ev[0]]
        for i in range(1, n):
            x, y = od[i - 1], ev[i]
            out += [self.mn(x, y), self.mx(x, y)]
        out.append(od[n - 1])
        return out

    def sort(self, lst):
        lst = list(lst)
        if len(lst) <= 1:
            return lst
        h = len(lst) // 2
        return self.merge(self.sort(lst[:h]), self.sort(lst[h:]))

    def sort5(self, v):
        """Optimal 9-comparator network for 5 keys (verified by the 0-1 principle)."""
        v = list(v)
        for i, j in ((0, 1), (3, 4), (2, 4), (2, 3), (1, 4), (0, 3), (0, 2), (1, 3), (1, 2)):
            self.cmpx(v, i, j)
        return v

    def sort3(self, v):
        v = list(v)
        for i, j in ((0, 1), (1, 2), (0, 1)):
            self.cmpx(v, i, j)
        return v

    def sortk(self, v):
        if len(v) == 3:
            return self.sort3(v)
        if len(v) == 5:
            return self.sort5(v)
        return self.sort(v)

    def select2(self, A, B, k):
        """Rank-k element of the union of sorted A and B, as the minimum over
        the k+1-element prefixes (i from A, k+1-i from B) of their largest
        member: min_i max(A[i-1], B[k-i])."""
        terms = []
        for i in range(0, len(A) + 1):
            j = k + 1 - i
            if j < 0 or j > len(B):
                continue
            a = A[i - 1] if i >= 1 else NEG
            b = B[j - 1] if j >= 1 else NEG
            terms.append(self.mx(a, b))
        out = terms[0]
        for t in terms[1:]:
            out = self.mn(out, t)
        return out

    def select_rank(self, lists, rank):
        """Element of rank ``rank`` (0-based) in the union of sorted lists."""
        lists = [l for l in lists if l]
        while len(lists) > 1:
            lists.sort(key=len)
            a, b = lists[0], lists[1]
            lists = lists[2:] + [self.merge(a, b)]
        return lists[0][rank]


def live_ops(dag: Dag, outputs):
    """Ids of operation nodes that feed ``outputs`` (after pruning)."""
    live = set()
    stack = [o for o in outputs if isinstance(o, int)]
    while stack:
        n = stack.pop()
        if n in live:
            continue
        live.add(n)
        nm = dag.names[n]
        if nm[0] != "in":
            for c in nm[1:]:
                if isinstance(c, int):
                    stack.append(c)
    return sorted(x for x in live if dag.names[x][0] != "in")


def count_ops(dag, outputs):
    return len(live_ops(dag, outputs))


def evaluate(dag: Dag, outputs, env):
    """Evaluate outputs with Python values; env maps input label -> value."""
    val = {}
    big = float("inf")

    def get(x):
        if x == NEG:
            return -big
        if x == POS:
            return big
        return val[x]

    for i, nm in enumerate(dag.names):
        if nm[0] == "in":
            val[i] = env[nm[1]]
    for i in live_ops(dag, outputs):
        k, a, b = dag.names[i]
        val[i] = min(get(a), get(b)) if k == "min" else max(get(a), get(b))
    return [get(o) for o in outputs]


# ---------------------------------------------------------------------------
# Networks
# ---------------------------------------------------------------------------

def window_median(K):
    """Standalone K x K median: sort columns, then select the middle rank.

    For K = 5 the four right-hand columns are merged pairwise, the two pairs
    merged, and the rank-12 element of that list and the first column is
    taken with ``select2``; other K use merges throughout."""
    d = Dag()
    cols = []
    for c in range(K):
        col = [d.inp((r, c)) for r in range(K)]
        cols.append(d.sortk(col))
    M = (K * K - 1) // 2
    if K == 5:
        q = d.merge(d.merge(cols[1], cols[2]), d.merge(cols[3], cols[4]))
        out = d.select2(q, cols[0], M)
    else:
        out = d.select_rank(cols, M)
    return d, [out]


def flat_median(n):
    """Median (rank (n-1)//2) of n loose keys: pruned Batcher sort."""
    d = Dag()
    v = [d.inp(i) for i in range(n)]
    s = d.sort(v)
    return d, [s[(n - 1) // 2]]


def emit_function(name, dag, outputs, in_shape, doc, loader=False):
    """Emit a __device__ template taking inputs v[...] and writing o[...].

    With ``loader`` the template (named ``<name>_ld``) takes a callable
    ``ld(i)`` instead of the array and fetches input i just before its first
    use, so only the inputs the network is working on need registers."""
    sig = (f"__device__ __forceinline__ void {name}_ld(const LD& ld, K* __restrict__ o) {{" if loader else
           f"__device__ __forceinline__ void {name}(const K* __restrict__ v, K* __restrict__ o) {{")
    lines = [f"// {doc}" + (" (inputs fetched at first use)" if loader else ""),
             f"// {count_ops(dag, outputs)} min/max operations.",
             "template <class K, class LD>" if loader else "template <class K>", sig]
    ids = live_ops(dag, outputs)
    names = {}
    in_idx = {}
    for i, nm in enumerate(dag.names):
        if nm[0] == "in":
            lab = nm[1]
            if isinstance(lab, tuple):
                idx = 0
                for k, dim in zip(lab, in_shape):
                    idx = idx * dim + k
            else:
                idx = lab
            names[i] = f"v{idx}" if loader else f"v[{idx}]"
            in_idx[i] = idx
    loaded = set()

    def ref(x):
        if x == NEG:
            return "lacos_net::neg_inf<K>()"
        if x == POS:
            return "lacos_net::pos_inf<K>()"
        if loader and x in in_idx and x not in loaded:
            loaded.add(x)
            lines.append(f"  const K v{in_idx[x]} = ld({in_idx[x]});")
        return names[x]

    for i in ids:
        k, a, b = dag.names[i]
        ra, rb = ref(a), ref(b)
        names[i] = f"t{i}"
        fn = "MN" if k == "min" else "MX"
        lines.append(f"  const K t{i} = {fn}({ra}, {rb});")
    if loader:
        for o in outputs:
            ref(o)
    for j, o in enumerate(outputs):
        lines.append(f"  o[{j}] = {ref(o)};")
    lines.append("}")
    return "\n".join(lines)


def block_median(K, W, R):
    """K x K medians of a W-wide, R-tall block of outputs sharing work.

    Inputs are v[(R+K-1) x (W+K-1)] (row-major); outputs o[R x W].  Each
    input column is sorted once per output row with vertical sharing (the
    rows common to all R windows are sorted once and the remaining rows
    merged in, halving recursively), created lazily left to right so the
    emitted code streams across the block.  Per output row the K sorted
    columns of a window are then combined:
      K = 3: the 3x3 median is med3(max of column minima, med3 of column
             medians, min of column maxima) (Paeth's construction), with the
             pairwise max/min terms shared between neighbouring outputs;
      K = 5: columns are merged in pairs shared by neighbouring output pairs,
             the two pairs merged (only the ranks that can be the median are
             kept by pruning) and the rank-12 element of that list and the
             fifth column taken with ``select2``.
    """
    d = Dag()
    ncol, nrow = W + K - 1, R + K - 1
    inp = [[d.inp((r, c)) for c in range(ncol)] for r in range(nrow)]
    colcache = {}

    def colsort(c, y):
        """Sorted column c over rows y..y+K-1, shared across the R rows."""
        if (c, y) not in colcache:
            def rec(lo, hi, core, core_rows):
                if hi - lo == 1:
                    extra = sorted(set(range(lo, lo + K)) - core_rows)
                    colcache[(c, lo)] = d.merge(core, d.sortk([inp[e][c] for e in extra])
                                                if len(extra) in (3, 5) else
                                                d.sort([inp[e][c] for e in extra]))
                    return
                mid = (lo + hi) // 2
                for a, b in ((lo, mid), (mid, hi)):
                    rows = set(range(b - 1, a + K))
                    extra = sorted(rows - core_rows)
                    rec(a, b, d.merge(core, d.sort([inp[e][c] for e in extra])), rows)
            rows = set(range(R - 1, K))
            core = d.sort([inp[e][c] for e in sorted(rows)]) if rows else []
            rec(0, R, core, rows)
        return colcache[(c, y)]

    M = (K * K - 1) // 2
    outs = [[None] * W for _ in range(R)]
    for x in range(W):
        for y in range(R):
            cols = [colsort(x + j, y) for j in range(K)]
            if K == 3:
                lo = [cc[0] for cc in cols]
                me = [cc[1] for cc in cols]
                hi = [cc[2] for cc in cols]
                # pair terms at even x are shared with x+1: max(lo1, lo2) etc.
                if x % 2 == 0:
                    a = d.mx(d.mx(lo[1], lo[2]), lo[0])
                    b = d.mn(d.mn(hi[1], hi[2]), hi[0])
                else:
                    a = d.mx(d.mx(lo[0], lo[1]), lo[2])
                    b = d.mn(d.mn(hi[0], hi[1]), hi[2])
                m = d.mx(d.mn(me[0], me[1]), d.mn(d.mx(me[0], me[1]), me[2]))
                outs[y][x] = d.mx(d.mn(a, m), d.mn(d.mx(a, m), b))
            elif K == 5:
                if x % 2 == 0:
                    q = d.merge(d.merge(cols[1], cols[2]), d.merge(cols[3], cols[4]))
                    outs[y][x] = d.select2(q, cols[0], M)
                else:
                    q = d.merge(d.merge(cols[0], cols[1]), d.merge(cols[2], cols[3]))
                    outs[y][x] = d.select2(q, cols[4], M)
            else:
                outs[y][x] = d.select_rank(cols, M)
    return d, [outs[y][x] for y in range(R) for x in range(W)]


BLOCKS = {"blk_med5_4x2": (5, 4, 2), "blk_med3_8x2": (3, 8, 2)}
# Separable K x K medians (the median over K rows of each row's K-tap median):
# the comparison mode of the detection medians.
SEP_BLOCKS = {"blk_sep5_4x2": (5, 4, 2)}


def _median_of(d, keys):
    s = d.sort(list(keys))
    return s[(len(keys) - 1) // 2]


def sep_window_median(K):
    """Separable K x K median of one window: K row medians, then their median."""
    d = Dag()
    v = [[d.inp((r, c)) for c in range(K)] for r in range(K)]
    rows = [_median_of(d, v[r]) for r in range(K)]
    return d, [_median_of(d, rows)]


def sep_block_median(K, W, R):
    """Separable K x K medians of a W-wide, R-tall block: each input row's
    K-tap medians at the W output columns are formed once and shared by the
    R output rows; then each output takes the median of its K row medians."""
    d = Dag()
    inp = [[d.inp((r, c)) for c in range(W + K - 1)] for r in range(R + K - 1)]
    rm = [[_median_of(d, inp[r][c:c + K]) for c in range(W)] for r in range(R + K - 1)]
    return d, [_median_of(d, [rm[y + a][x] for a in range(K)]) for y in range(R) for x in range(W)]


def sep_reference(env, win_rows):
    """Median over rows of the row medians, for a window given as rows of labels."""
    meds = sorted(sorted(env[lab] for lab in row)[(len(row) - 1) // 2] for row in win_rows)
    return meds[(len(meds) - 1) // 2]


def build_all():
    nets = {}
    nets["med3x3"] = window_median(3) + ((3, 3), "Median of a 3x3 window, v row-major.")
    nets["med5x5"] = window_median(5) + ((5, 5), "Median of a 5x5 window, v row-major.")
    nets["med7x7"] = window_median(7) + ((7, 7), "Median of a 7x7 window, v row-major.")
    for name, (K, W, R) in BLOCKS.items():
        d, o = block_median(K, W, R)
        nets[name] = (d, o, (R + K - 1, W + K - 1),
                      f"{K}x{K} medians of a {W}x{R} block (W x R); v is "
                      f"{R + K - 1}x{W + K - 1} row-major, o is {R}x{W} row-major.")
    nets["sep5x5"] = sep_window_median(5) + ((5, 5), "Separable median of a 5x5 window (median of "
                                                     "the row medians), v row-major.")
    for name, (K, W, R) in SEP_BLOCKS.items():
        d, o = sep_block_median(K, W, R)
        nets[name] = (d, o, (R + K - 1, W + K - 1),
                      f"Separable {K}x{K} medians of a {W}x{R} block (W x R); v is "
                      f"{R + K - 1}x{W + K - 1} row-major, o is {R}x{W} row-major.")
    return nets


def _window_rows(name, out_index):
    """Rows of input labels of the window behind an output (separable networks)."""
    if name in SEP_BLOCKS:
        K, W, R = SEP_BLOCKS[name]
        y, x = divmod(out_index, W)
        return [[(y + a, x + b) for b in range(K)] for a in range(K)]
    return [[(a, b) for b in range(5)] for a in range(5)]  # sep5x5


def block_window(name, out_index):
    """Input labels (row, col) of the window behind output ``out_index`` of a block."""
    K, W, R = BLOCKS[name] if name in BLOCKS else SEP_BLOCKS[name]
    y, x = divmod(out_index, W)
    return [(y + a, x + b) for a in range(K) for b in range(K)]


def _windows(name, dag, outs):
    labels = [nm[1] for nm in dag.names if nm[0] == "in"]
    if name in BLOCKS or name in SEP_BLOCKS:
        return [block_window(name, j) for j in range(len(outs))]
    return [labels]


def is_separable(name):
    return name == "sep5x5" or name in SEP_BLOCKS


def verify(nets=None, trials=2000, seed=1, exhaustive=True, max_exhaustive_outputs=None):
    """Check every network against a full sort of each output's window:
    random keys with many ties, and (for windows of up to 25 keys) every
    0-1 input of the window, bit-sliced with numpy (min = AND, max = OR),
    which by the 0-1 principle covers all inputs of a comparator network."""
    nets = nets or build_all()
    rng = random.Random(seed)
    for name, (dag, outs, shape, _) in nets.items():
        labels = [nm[1] for nm in dag.names if nm[0] == "in"]
        wins = _windows(name, dag, outs)
        for t in range(trials):
            hi = [1, 3, 1000][t % 3]
            env = {lab: rng.randint(0, hi) for lab in labels}
            got = evaluate(dag, outs, env)
            for j, win in enumerate(wins):
                if is_separable(name):
                    want = sep_reference(env, _window_rows(name, j))
                else:
                    vals = sorted(env[lab] for lab in win)
                    want = vals[(len(vals) - 1) // 2]
                if got[j] != want:
                    raise AssertionError(f"{name}: output {j} wrong on {env}")
        if exhaustive:
            for j, win in enumerate(wins[:max_exhaustive_outputs]):
                if len(win) <= 25:
                    _exhaustive01(dag, outs[j], win, labels,
                                  _window_rows(name, j) if is_separable(name) else None)
    return True


def _exhaustive01(dag, out, win, labels, rows=None):
    """Every 0-1 assignment of the window; the reference is the median of the
    window or, with ``rows``, the median of the row medians (both min/max
    formulas, which by the 0-1 principle agree everywhere if they agree on
    every 0-1 input)."""
    import numpy as np
    n = len(win)
    total = 1 << n
    idx = np.arange(total, dtype=np.uint64)
    val = {}
    inwin = {lab: k for k, lab in enumerate(win)}
    for i, nm in enumerate(dag.names):
        if nm[0] == "in":
            k = inwin.get(nm[1])
            val[i] = ((idx >> np.uint64(k)) & np.uint64(1)).astype(bool) if k is not None else None
    for i in live_ops(dag, [out]):
        kind, a, b = dag.names[i]
        va = {NEG: False, POS: True}.get(a) if not isinstance(a, int) else val[a]
        vb = {NEG: False, POS: True}.get(b) if not isinstance(b, int) else val[b]
        if va is None or vb is None:
            raise AssertionError("output depends on an input outside its window")
        val[i] = (va & vb) if kind == "min" else (va | vb)
    def bit(k):
        return ((idx >> np.uint64(k)) & np.uint64(1)).astype(np.int64)

    if rows is None:
        ones = sum(bit(k) for k in range(n))
        expect = ones >= (n + 1) // 2  # the median of n (odd) 0/1 keys is 1 iff #ones > n/2
    else:
        row_meds = [sum(bit(inwin[lab]) for lab in row) >= (len(row) + 1) // 2 for row in rows]
        expect = sum(m.astype(np.int64) for m in row_meds) >= (len(rows) + 1) // 2
    got = val[out] if isinstance(out, int) else np.full(total, out == POS)
    if not np.array_equal(np.asarray(got, dtype=bool), expect):
        raise AssertionError("0-1 exhaustive check failed")


HEADER = """// Generated by gen_networks.py -- do not edit.
// Branch-free min/max selection networks (see the generator for the
// construction and its sources).  MN/MX must be defined for the key type.
#pragma once
"""


# Networks also emitted in the fetch-at-first-use form.
LOADER_NETS = ("blk_med5_4x2", "blk_med3_8x2", "med5x5", "med7x7", "sep5x5", "blk_sep5_4x2")


def main(out_path):
    nets = build_all()
    verify(nets, trials=300)
    parts = [HEADER]
    for name, (dag, outs, shape, doc) in nets.items():
        parts.append(emit_function(name, dag, outs, shape, doc))
        if name in LOADER_NETS:
            parts.append(emit_function(name, dag, outs, shape, doc, loader=True))
    text = "\n\n".join(parts) + "\n"
    with open(out_path, "w") as f:
        f.write(text)
    for name, (dag, outs, shape, doc) in nets.items():
        print(f"{name}: {count_ops(dag, outs)} ops, {count_ops(dag, outs) / len(outs):.1f} per output")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else
         os.path.join(os.path.dirname(os.path.abspath(__file__)), "networks.cuh"))
