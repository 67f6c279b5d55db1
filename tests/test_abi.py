"""The C-ABI library loads and exports every entry point include/lacos.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    out = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            out |= set(re.findall(r"\b(lacos_\w+)\s*\(", text))
    return out


@pytest.fixture(scope="module")
def lib():
    from paper_2602_17938_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert {"lacos_create", "lacos_submit", "lacos_poll", "lacos_destroy"} <= syms
    for s in sorted(syms):
        assert hasattr(lib, s), s


def test_host_only_entry_points(lib):
    lib.lacos_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lacos_version()
    lib.lacos_scratch_bytes.restype = ctypes.c_size_t
    lib.lacos_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    n = lib.lacos_scratch_bytes(6388, 9576)
    # five bit-planes (two mask buffers, three test planes): 5 * 6388 * ceil(9576/32) * 4,
    # the 65536-entry table of {2N, 1/(2N)} (float pairs) per uint16 med5 value, and three
    # level-mark bytes per tile of the smallest core tile, 32x32: 3 * ceil(6388/32) * ceil(9576/32)
    expect = 5 * 6388 * 300 * 4 + 65536 * 8 + 3 * 200 * 300
    assert expect <= n < expect + (1 << 20)
    assert lib.lacos_scratch_bytes(0, 5) == 0


def test_request_bytes_counts_the_saturation_plane(lib):
    from paper_2602_17938_gb300 import lacos
    lib.lacos_scratch_bytes.restype = ctypes.c_size_t
    lib.lacos_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.lacos_request_bytes.restype = ctypes.c_size_t
    lib.lacos_request_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    base = lib.lacos_scratch_bytes(6388, 9576)
    assert lib.lacos_request_bytes(6388, 9576, None) == base
    p = lacos.make_params(1.0, 1.5)
    assert lib.lacos_request_bytes(6388, 9576, ctypes.byref(p)) == base
    p = lacos.make_params(1.0, 1.5, satgrow=2)
    # one more bit-plane (6388 rows of 300 words), 256-byte aligned
    plane = (6388 * 300 * 4 + 255) // 256 * 256
    assert lib.lacos_request_bytes(6388, 9576, ctypes.byref(p)) == base + plane
    assert lib.lacos_request_bytes(0, 9576, ctypes.byref(p)) == 0


def test_batch_frame_count_limits_without_gpu(lib):
    # The per-frame kernels put frames on the grid's y dimension: 1 <= n <= 65535.
    # The count is checked before any pointer is read, so no context is needed.
    f = lib.lacos_submit_batch
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 8 + [ctypes.c_int, ctypes.c_void_p,
                                                                             ctypes.c_void_p]
    dummy = ctypes.c_void_p(16)
    args = [dummy] * 8
    for n in (0, -1, 65536, 1 << 30):
        assert f(None, n, *args, 0, None, dummy) == -1, n


def test_null_arguments_rejected_without_gpu(lib):
    lib.lacos_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_int]
    assert lib.lacos_create(None, 0, 0, 0) == -1
    lib.lacos_poll.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p]
    assert lib.lacos_poll(None, 1, None) == -1
    lib.lacos_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lacos_destroy(None) == -1


def test_networks_header_matches_generator_and_verifies():
    import importlib.util
    path = os.path.join(ROOT, "paper_2602_17938_gb300", "csrc", "gen_networks.py")
    spec = importlib.util.spec_from_file_location("gen_networks", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    nets = gen.build_all()
    # exhaustive 0-1 check of the first output of each network (all outputs:
    # run gen_networks.py), random keys with ties for every output
    assert gen.verify(nets, trials=200, max_exhaustive_outputs=1)
    text = open(os.path.join(ROOT, "paper_2602_17938_gb300", "csrc", "networks.cuh")).read()
    for name, (dag, outs, shape, doc) in nets.items():
        assert gen.emit_function(name, dag, outs, shape, doc) in text, name


def test_struct_layouts_match_the_binding(tmp_path):
    # The ctypes mirrors in the binding must have the header's sizes and field
    # offsets: a C program built against include/lacos.h prints them.
    import subprocess
    from paper_2602_17938_gb300 import lacos
    structs = {"lacos_params": lacos.Params, "lacos_result": lacos.Result, "lacos_profile": lacos.Profile}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lacos.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
