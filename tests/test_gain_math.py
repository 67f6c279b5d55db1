"""The library's gain-estimate arithmetic (csrc/gain_math.cuh), compiled for
the host with g++ and checked against exact integer arithmetic in Python and
against the oracle's estimate (reading C15)."""
import ctypes
import math
import os
import random
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def gm(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("gm") / "libgm.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    os.path.join(HERE, "gain_math_harness.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    u64, i64, d = ctypes.c_ulonglong, ctypes.c_longlong, ctypes.c_double
    P = ctypes.c_void_p
    lib.h_u128_to_double.argtypes = [u64, u64]
    lib.h_u128_to_double.restype = d
    lib.h_isqrt.argtypes = [u64, u64, P, P]
    lib.h_clip_interval.argtypes = [u64, i64, u64, P, P]
    lib.h_gain.argtypes = [u64, i64, u64, u64, ctypes.c_float, P]
    lib.h_gain.restype = ctypes.c_int
    return lib


def _split(v: int):
    return v >> 64, v & ((1 << 64) - 1)


def test_u128_to_double_rounds_to_nearest_even(gm):
    cases = [0, 1, (1 << 62) - 1, 1 << 62, (1 << 62) + 1, (1 << 63) + 1, (1 << 96) - 1,
             # exactly halfway between two doubles, both parities of the kept bit
             (1 << 70) + (1 << 17), (1 << 70) + (3 << 17), ((1 << 53) + 1) << 20 | (1 << 19),
             # just above and below halfway
             (1 << 70) + (1 << 17) + 1, (1 << 70) + (1 << 17) - 1]
    r = random.Random(0)
    for bits in range(1, 100):
        cases += [r.getrandbits(bits) for _ in range(20)]
    for v in cases:
        assert gm.h_u128_to_double(*_split(v)) == float(v), v


def test_isqrt(gm):
    rng = np.random.default_rng(1)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, (1 << 96) - 1, ((1 << 48) - 1) ** 2, ((1 << 48) - 1) ** 2 - 1]
    vals += [int(rng.integers(0, 1 << 62)) * int(rng.integers(1, 1 << 34)) for _ in range(500)]
    vals += [r * r + o for r in (int(x) for x in rng.integers(1, 1 << 47, 200)) for o in (-1, 0, 1)]
    for q in vals:
        hi, lo = ctypes.c_ulonglong(), ctypes.c_ulonglong()
        gm.h_isqrt(*_split(q), ctypes.byref(hi), ctypes.byref(lo))
        assert (hi.value << 64 | lo.value) == math.isqrt(q), q


def test_clip_interval_is_the_exact_3_sigma_set(gm):
    rng = np.random.default_rng(2)
    for _ in range(300):
        d = rng.integers(-int(rng.integers(1, 65536)), int(rng.integers(1, 65536)), int(rng.integers(1, 40)))
        n, s1, s2 = len(d), int(d.sum()), int((d.astype(object) ** 2).sum())
        lo, hi = ctypes.c_longlong(), ctypes.c_longlong()
        gm.h_clip_interval(n, s1, s2, ctypes.byref(lo), ctypes.byref(hi))
        q = 9 * (n * s2 - s1 * s1)
        inside = [x for x in range(-65536, 65537) if (n * x - s1) ** 2 <= q]
        assert (lo.value, hi.value) == (inside[0], inside[-1])
        assert len(inside) == inside[-1] - inside[0] + 1


def test_gain_matches_the_oracle_bit_for_bit(gm):
    rng = np.random.default_rng(3)
    for g, rn, mu in ((2.0, 5.0, 1000.0), (0.7, 11.0, 40.0), (3.0, 0.0, 20000.0), (1.3, 4.25, 3.0)):
        e = rng.poisson(g * mu, (300, 400)) + rng.normal(0.0, rn, (300, 400))
        I = np.clip(np.rint(e / g), 0, 65535).astype(np.float32)
        z = np.zeros(I.shape, np.uint8)
        est, _, (n, s1, s2, a) = oracle.estimate_gain(I, z, z, rn)
        out = ctypes.c_double()
        assert gm.h_gain(n, s1, s2, a, rn, ctypes.byref(out)) == 1
        assert out.value == est
    out = ctypes.c_double()
    assert gm.h_gain(1, 5, 25, 10, 2.0, ctypes.byref(out)) == 0      # one pair
    assert gm.h_gain(4, 8, 16, 100, 2.0, ctypes.byref(out)) == 0     # all d equal: V = 0
