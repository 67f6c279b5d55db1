"""Python binding of the C ABI in include/lacos.h (argument marshalling only).

Every step of the detect-and-clean path runs in the CUDA library
``_build/liblacos.so``; this module only passes device pointers, sizes and
the stream.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblacos.so")

LACOS_F32, LACOS_U16 = 0, 1
OK, PENDING = 0, 1
EINVAL, EAGAIN, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNKNOWN_TICKET, ENOGAIN = -1, -2, -3, -4, -5, -6, -7, -8
MAX_NITER = 256
CORE_VARIANTS = 10  # LACOS_CORE_VARIANTS: core-kernel tile shape x occupancy variants
_ERRNAMES = {EINVAL: "EINVAL", EAGAIN: "EAGAIN", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
             ENONFINITE: "ENONFINITE", ETIMEOUT: "ETIMEOUT", EUNKNOWN_TICKET: "EUNKNOWN_TICKET",
             ENOGAIN: "ENOGAIN"}


class LacosError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed: {_ERRNAMES.get(code, code)}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_float), ("readnoise", ctypes.c_float),
                ("satlevel", ctypes.c_float), ("sigclip", ctypes.c_float),
                ("sigfrac", ctypes.c_float), ("objlim", ctypes.c_float),
                ("niter", ctypes.c_int), ("fine_norm", ctypes.c_int), ("satgrow", ctypes.c_int),
                ("sepmed", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int),
                ("core_ms", ctypes.c_float * MAX_NITER),
                ("grow_ms", ctypes.c_float * MAX_NITER),
                ("final_ms", ctypes.c_float), ("px_iterations", ctypes.c_longlong),
                ("n_sprime", ctypes.c_longlong), ("n_fine", ctypes.c_longlong),
                ("n_replace", ctypes.c_longlong), ("n_replace_wide", ctypes.c_longlong),
                ("px_core", ctypes.c_longlong), ("n_sprime_net", ctypes.c_longlong),
                ("n_fine_net", ctypes.c_longlong)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters_run", ctypes.c_int),
                ("n_flagged", ctypes.c_longlong), ("latency_ms", ctypes.c_double),
                ("gain", ctypes.c_float)]


def make_params(gain, readnoise, satlevel=65535.0, sigclip=4.5, sigfrac=0.3, objlim=5.0,
                niter=4, fine_norm=True, satgrow=0, sepmed=False) -> Params:
    """Frame parameters; gain 0 estimates the gain at every iteration (uint16 frames)."""
    return Params(gain, readnoise, satlevel, sigclip, sigfrac, objlim, int(niter), int(bool(fine_norm)),
                  int(satgrow), int(bool(sepmed)))


_lib = None


def load_library():
    """Load liblacos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, U64P = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)
        lib.lacos_create.argtypes = [ctypes.POINTER(P), I, ctypes.c_size_t, I]
        lib.lacos_submit.argtypes = [P, P, I, I, I, ctypes.POINTER(Params), P, P, P, U64P]
        lib.lacos_submit_batch.argtypes = [P, I, P, P, P, P, P, P, P, P, I, P, U64P]
        lib.lacos_poll.argtypes = [P, ctypes.c_ulonglong, ctypes.POINTER(Result)]
        lib.lacos_wait.argtypes = [P, ctypes.c_ulonglong, ctypes.POINTER(Result)]
        lib.lacos_destroy.argtypes = [P]
        lib.lacos_scratch_bytes.argtypes = [I, I]
        lib.lacos_scratch_bytes.restype = ctypes.c_size_t
        lib.lacos_request_bytes.argtypes = [I, I, ctypes.POINTER(Params)]
        lib.lacos_request_bytes.restype = ctypes.c_size_t
        lib.lacos_last_cuda_error.argtypes = [P]
        lib.lacos_version.restype = ctypes.c_char_p
        lib.lacos_set_profiling.argtypes = [P, I]
        lib.lacos_last_profile.argtypes = [P, ctypes.POINTER(Profile)]
        lib.lacos_run_static.argtypes = [P, I, I, I, ctypes.POINTER(Params), P, P, P,
                                         ctypes.POINTER(Result)]
        lib.lacos_run_static.restype = I
        lib.lacos_submit_async.argtypes = [P, P, I, I, I, ctypes.POINTER(Params), P, P, U64P]
        lib.lacos_set_core_variant.argtypes = [P, I]
        lib.lacos_get_core_variant.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        lib.lacos_autotune.argtypes = [P, P, I, I, I, ctypes.POINTER(Params), P, P, P, I,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        lib.lacos_selftest_division.argtypes = [ctypes.c_float, ctypes.c_float, U64P]
        lib.lacos_submit_host.argtypes = [P, P, I, I, I, ctypes.POINTER(Params), P, P, U64P]
        for name in ("lacos_submit_async", "lacos_set_core_variant", "lacos_get_core_variant",
                     "lacos_autotune", "lacos_selftest_division", "lacos_submit_host"):
            getattr(lib, name).restype = I
        for name in ("lacos_create", "lacos_submit", "lacos_submit_batch", "lacos_poll",
                     "lacos_wait", "lacos_destroy", "lacos_last_cuda_error",
                     "lacos_set_profiling", "lacos_last_profile"):
            getattr(lib, name).restype = I
        _lib = lib
    return _lib


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return LACOS_F32
    if t.dtype == torch.uint16:
        return LACOS_U16
    raise TypeError("frame must be torch.float32 or torch.uint16")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class FrameResult:
    status: int
    iters_run: int
    n_flagged: int
    latency_ms: float
    gain: float = 0.0  # the last iteration's gain (the estimate when the gain was 0)


class Context:
    """A library context (lacos_create / lacos_destroy)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_slots: int = 0):
        self.lib = load_library()
        self.h = ctypes.c_void_p()
        rc = self.lib.lacos_create(ctypes.byref(self.h), device, hbm_budget_bytes, max_slots)
        if rc != OK:
            raise LacosError(rc, "lacos_create")

    def submit(self, frame, params: Params, mask, clean, stream=None) -> int:
        """Queue one frame; returns a ticket.  Raises LacosError(EAGAIN) when full."""
        ny, nx = frame.shape
        for t in (frame, mask, clean):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("frame, mask and clean must be contiguous CUDA tensors")
        if tuple(mask.shape) != (ny, nx) or tuple(clean.shape) != (ny, nx):
            raise ValueError("mask and clean must have the frame's shape")
        t = ctypes.c_ulonglong(0)
        rc = self.lib.lacos_submit(self.h, ctypes.c_void_p(frame.data_ptr()), _dtype_code(frame),
                                   ny, nx, ctypes.byref(params), ctypes.c_void_p(mask.data_ptr()),
                                   ctypes.c_void_p(clean.data_ptr()), _stream_ptr(stream),
                                   ctypes.byref(t))
        if rc != OK:
            raise LacosError(rc, "lacos_submit")
        return t.value

    def submit_async(self, frame, params: Params, mask, clean) -> int:
        """Queue one frame on a stream of its own (requests overlap on the device).
        The frame must already be complete on the device.  Raises LacosError(EAGAIN)
        when no slot or budget is free."""
        ny, nx = frame.shape
        t = ctypes.c_ulonglong(0)
        rc = self.lib.lacos_submit_async(self.h, ctypes.c_void_p(frame.data_ptr()), _dtype_code(frame),
                                         ny, nx, ctypes.byref(params), ctypes.c_void_p(mask.data_ptr()),
                                         ctypes.c_void_p(clean.data_ptr()), ctypes.byref(t))
        if rc != OK:
            raise LacosError(rc, "lacos_submit_async")
        return t.value

    def submit_host(self, h_frame, params: Params, h_mask, h_clean) -> int:
        """Queue a host-to-host request (lacos_submit_host): CPU tensors, page-locked
        for overlap; the outputs are written when the request completes.  Raises
        LacosError(EAGAIN) when no slot or budget is free."""
        ny, nx = h_frame.shape
        t = ctypes.c_ulonglong(0)
        rc = self.lib.lacos_submit_host(self.h, ctypes.c_void_p(h_frame.data_ptr()), _dtype_code(h_frame),
                                        ny, nx, ctypes.byref(params), ctypes.c_void_p(h_mask.data_ptr()),
                                        ctypes.c_void_p(h_clean.data_ptr()), ctypes.byref(t))
        if rc != OK:
            raise LacosError(rc, "lacos_submit_host")
        return t.value

    def set_core_variant(self, v: int):
        rc = self.lib.lacos_set_core_variant(self.h, int(v))
        if rc != OK:
            raise LacosError(rc, "lacos_set_core_variant")

    def core_variant(self) -> int:
        v = ctypes.c_int(0)
        rc = self.lib.lacos_get_core_variant(self.h, ctypes.byref(v))
        if rc != OK:
            raise LacosError(rc, "lacos_get_core_variant")
        return v.value

    def autotune(self, frame, params: Params, mask, clean, reps: int = 2, stream=None):
        """Time every core-kernel variant on this frame and keep the fastest.
        Returns (best variant, [mean ms per variant])."""
        ny, nx = frame.shape
        best = ctypes.c_int(-1)
        ms = (ctypes.c_float * CORE_VARIANTS)()
        rc = self.lib.lacos_autotune(self.h, ctypes.c_void_p(frame.data_ptr()), _dtype_code(frame), ny, nx,
                                     ctypes.byref(params), ctypes.c_void_p(mask.data_ptr()),
                                     ctypes.c_void_p(clean.data_ptr()), _stream_ptr(stream), int(reps),
                                     ctypes.byref(best), ms)
        if rc != OK:
            raise LacosError(rc, "lacos_autotune")
        return best.value, list(ms)

    def submit_batch(self, frames, params, masks, cleans, stream=None, reuse_graph=False):
        """Queue a batch of frames (any sizes/dtypes); returns (ticket, per-frame result array)."""
        n = len(frames)
        ptr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        dts = (ctypes.c_int * n)(*[_dtype_code(f) for f in frames])
        nys = (ctypes.c_int * n)(*[f.shape[0] for f in frames])
        nxs = (ctypes.c_int * n)(*[f.shape[1] for f in frames])
        ps = (Params * n)(*params)
        per = (Result * n)()
        t = ctypes.c_ulonglong(0)
        keep = (ptr(frames), ptr(masks), ptr(cleans))
        rc = self.lib.lacos_submit_batch(self.h, n, keep[0], dts, nys, nxs, ps, keep[1], keep[2],
                                         _stream_ptr(stream), int(bool(reuse_graph)), per,
                                         ctypes.byref(t))
        if rc != OK:
            raise LacosError(rc, "lacos_submit_batch")
        self._keep = (keep, dts, nys, nxs, ps, per)
        return t.value, per

    def poll(self, ticket: int):
        r = Result()
        rc = self.lib.lacos_poll(self.h, ticket, ctypes.byref(r))
        if rc == PENDING:
            return None
        if rc != OK:
            raise LacosError(rc, "lacos_poll")
        return FrameResult(r.status, r.iters_run, r.n_flagged, r.latency_ms, r.gain)

    def wait(self, ticket: int) -> FrameResult:
        r = Result()
        rc = self.lib.lacos_wait(self.h, ticket, ctypes.byref(r))
        if rc != OK:
            raise LacosError(rc, "lacos_wait")
        return FrameResult(r.status, r.iters_run, r.n_flagged, r.latency_ms, r.gain)

    def set_profiling(self, on: bool):
        rc = self.lib.lacos_set_profiling(self.h, int(bool(on)))
        if rc != OK:
            raise LacosError(rc, "lacos_set_profiling")

    def last_profile(self) -> dict:
        p = Profile()
        rc = self.lib.lacos_last_profile(self.h, ctypes.byref(p))
        if rc != OK:
            raise LacosError(rc, "lacos_last_profile")
        n = p.n_levels
        return {"core_ms": list(p.core_ms[:n]), "grow_ms": list(p.grow_ms[:n]),
                "final_ms": p.final_ms,
                "px_iterations": p.px_iterations, "n_sprime": p.n_sprime, "n_fine": p.n_fine,
                "n_replace": p.n_replace, "n_replace_wide": p.n_replace_wide,
                "px_core": p.px_core, "n_sprime_net": p.n_sprime_net, "n_fine_net": p.n_fine_net}

    def last_cuda_error(self) -> int:
        return self.lib.lacos_last_cuda_error(self.h)

    def close(self):
        if self.h:
            rc = self.lib.lacos_destroy(self.h)
            self.h = ctypes.c_void_p()
            if rc != OK:
                raise LacosError(rc, "lacos_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def clean_frame(frame, gain, readnoise, satlevel=65535.0, sigclip=4.5, sigfrac=0.3, objlim=5.0,
                niter=4, fine_norm=True, ctx: Context | None = None, stream=None, satgrow=0,
                sepmed=False):
    """Detect and clean one device frame; returns (mask uint8, cleaned float32, FrameResult)."""
    import torch
    own = ctx is None
    ctx = ctx or Context(frame.device.index or 0)
    try:
        mask = torch.empty(frame.shape, dtype=torch.uint8, device=frame.device)
        clean = torch.empty(frame.shape, dtype=torch.float32, device=frame.device)
        p = make_params(gain, readnoise, satlevel, sigclip, sigfrac, objlim, niter, fine_norm, satgrow,
                        sepmed)
        t = ctx.submit(frame, p, mask, clean, stream)
        res = ctx.wait(t)
        return mask, clean, res
    finally:
        if own:
            ctx.close()


STATIC_SCRATCH_BYTES = 64 << 20


def selftest_division(gain: float, readnoise: float) -> int:
    """Pairs (numerator, table entry) where the uint16 path's division differs
    from IEEE float32 division for these parameters (lacos_selftest_division)."""
    lib = load_library()
    out = ctypes.c_ulonglong()
    rc = lib.lacos_selftest_division(float(gain), float(readnoise), ctypes.byref(out))
    if rc != OK:
        raise LacosError(rc, "lacos_selftest_division")
    return int(out.value)


def run_static(frame, params: Params, mask, clean, stream=None) -> FrameResult:
    """lacos_run_static: detect-and-clean one device frame with no device
    allocation (scratch in the library's fixed device array; frames whose
    scratch exceeds 64 MiB raise LacosError(ENOMEM)).  For callers that must
    not allocate device memory while running; blocks until the frame is done.
    Calls that overlap on the GPU share the array and must be serialised."""
    ny, nx = frame.shape
    for t in (frame, mask, clean):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("frame, mask and clean must be contiguous CUDA tensors")
    r = Result()
    rc = load_library().lacos_run_static(ctypes.c_void_p(frame.data_ptr()), _dtype_code(frame), ny, nx,
                                         ctypes.byref(params), ctypes.c_void_p(mask.data_ptr()),
                                         ctypes.c_void_p(clean.data_ptr()), _stream_ptr(stream),
                                         ctypes.byref(r))
    if rc != OK:
        raise LacosError(rc, "lacos_run_static")
    return FrameResult(r.status, r.iters_run, r.n_flagged, r.latency_ms, r.gain)


def clean_host(h_frame, params: Params, h_mask, h_clean, ctx: Context):
    """Host-to-host detect-and-clean of one frame through lacos_submit_host:
    the library copies the (page-locked) host frame in and the mask and cleaned
    frame out.  Returns FrameResult."""
    return ctx.wait(ctx.submit_host(h_frame, params, h_mask, h_clean))


def clean_host_stream(ctx: Context, frames, params: Params, masks, cleans, depth: int = 3):
    """Host-to-host detect-and-clean of a sequence of frames, up to ``depth``
    requests in flight (one frame's upload, another's compute and a third's
    download overlap).  Returns the FrameResults in order."""
    pending, results = [], [None] * len(frames)
    for i, (f, m, c) in enumerate(zip(frames, masks, cleans)):
        if len(pending) >= depth:
            j, t = pending.pop(0)
            results[j] = ctx.wait(t)
        pending.append((i, ctx.submit_host(f, params, m, c)))
    for j, t in pending:
        results[j] = ctx.wait(t)
    return results


def to_device(frame: np.ndarray, device="cuda"):
    import torch
    if frame.dtype == np.uint16:
        return torch.from_numpy(frame.view(np.int16)).to(device).view(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(frame, np.float32)).to(device)
