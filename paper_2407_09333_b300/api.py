"""ctypes binding of libhashbatch.so (C-ABI in include/hashbatch.h).

Argument marshalling only: every step of the hashing path runs in the CUDA
library.  Device buffers are torch tensors (torch supplies device memory and
streams); host-buffer entry points take numpy arrays or CPU tensors.  If the
library has not been built the first call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

MD5, SHA1, SM3 = 0, 1, 2
TUNE_MIXED = 3
ALL = 4                 # all three algorithms per message (hash_batch_all)
# The library's defaults for the ragged path (hash_tune_buckets,
# hash_tune_mixed_warps), which the autotuner keeps unless a candidate is
# clearly faster.
DEFAULT_BUCKETS = (6, 2)
DEFAULT_MIXED_WARPS = 8
ALL_RECORD_BYTES = 96
ALL_DIGEST_BYTES = 68
SLOT_BYTES = 32
ALG_NAMES = {MD5: "md5", SHA1: "sha1", SM3: "sm3"}
ALG_CODES = {v: k for k, v in ALG_NAMES.items()}

DEV_TIMEOUT = 0x1
DEV_BOUNDS = 0x2
DEV_SEGMENT = 0x4
SEG_MORE = 1 << 63

_PKG = os.path.dirname(os.path.abspath(__file__))
# HB_LIBRARY may name another build of the same library (e.g. an A/B variant).
LIB_PATH = os.environ.get("HB_LIBRARY") or os.path.join(_PKG, "libhashbatch.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "hashbatch.h")

_c_int, _c_u64, _c_u32, _vp = ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
_SIGNATURES = {
    "hash_digest_size": (ctypes.c_size_t, [_c_int]),
    "hash_strerror": (ctypes.c_char_p, [_c_int]),
    "hash_last_cuda_error": (ctypes.c_char_p, []),
    "hash_batch": (_c_int, [_c_int, _vp, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_batch_mixed": (_c_int, [_vp, _vp, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_batch_all": (_c_int, [_vp, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_batch_all_shape": (_c_int, [_vp, _vp, _vp, _c_u64, _vp, _c_int, _c_int, _vp]),
    "hash_batch_mixed_noalloc": (_c_int, [_vp, _vp, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_batch_segments": (_c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_batch_check_bounds": (_c_int, [_vp, _vp, _c_u64, _c_u64, _vp, _vp]),
    "hash_batch_host": (_c_int, [_c_int, _vp, _vp, _c_u64, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_batch_host_packed": (_c_int, [_c_int, _vp, _c_u64, _vp, _vp, _c_u64, _vp, _vp]),
    "hash_device_status": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "hash_release_device": (_c_int, []),
    "hash_tune_shapes": (_c_int, []),
    "hash_tune_shape": (_c_int, [_c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                 ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "hash_tune_set": (_c_int, [_c_int, _c_int]),
    "hash_tune_get": (_c_int, [_c_int]),
    "hash_tune_occupancy": (_c_int, [_c_int, _c_int]),
    "hash_tune_buckets": (_c_int, [_c_int, _c_int]),
    "hash_tune_mixed_warps": (_c_int, [_c_int]),
    "hash_tune_relay": (_c_int, [_c_int]),
    "hash_all_uses_relay": (_c_int, [_c_u64]),
    "hash_batch_shape": (_c_int, [_c_int, _vp, _vp, _vp, _c_u64, _vp, _c_int, _c_int, _vp]),
    "hash_batch_mixed_shape": (_c_int, [_vp, _vp, _vp, _vp, _c_u64, _vp, _c_int, _c_int, _vp]),
    "hash_int_peak": (_c_int, [_c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp]),
    "hash_int_peak_ops_per_iter": (_c_int, []),
    "hash_selftest_wait_timeout": (_c_int, [_c_u64, _vp]),
    "hash_set_wait_limit_ns": (_c_u64, [_c_u64]),
    "hash_plan_create": (_c_int, [_c_u64, ctypes.POINTER(_vp)]),
    "hash_plan_run": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_u64, _vp, _c_int, _vp]),
    "hash_plan_capture": (_c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _c_int]),
    "hash_plan_replay": (_c_int, [_vp, _c_u64, _vp]),
    "hash_plan_destroy": (_c_int, [_vp]),
    "hash_plan_configure": (_c_int, [_vp, _c_int, _c_int]),
    "hash_plan_set_completion": (_c_int, [_vp, _vp, _vp, _vp]),
    "hash_plan_set_segments": (_c_int, [_vp, _vp, _vp]),
    "hash_gather": (_c_int, [_vp, _c_u32, _vp]),
    "hash_digits": (_c_int, [_c_int, _c_u64, _c_u64, _vp, _vp]),
    "hash_set_host_memory_limit": (_c_u64, [_c_u64]),
    "hash_round_create": (_c_int, [_vp, _c_u32, _vp, _c_u64, ctypes.POINTER(_c_u32), _c_int,
                                   _c_int, ctypes.POINTER(_vp)]),
    "hash_round_launch": (_c_int, [_vp, _c_u64, _c_u64, _vp]),
    "hash_round_report": (_c_int, [_vp, ctypes.POINTER(_c_u64), ctypes.POINTER(_c_u64)]),
    "hash_round_destroy": (_c_int, [_vp]),
}

RING_FREE, RING_READY, RING_BUSY = 0, 1, 2


class HbRing(ctypes.Structure):
    """struct hb_ring of include/hashbatch.h."""
    _fields_ = [("capacity", _c_u64), ("src", _vp), ("prior", _vp), ("len", _vp),
                ("req", _vp), ("alg", _vp), ("state", _vp), ("slots", _vp),
                ("req_remaining", _vp), ("req_done", _vp), ("req_capacity", _c_u64)]

_lib = None


class HashBatchError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code in (-4, -5):
            detail = ": " + lib().hash_last_cuda_error().decode()
        super().__init__("%s failed: %s (%d)%s" % (where, strerror(code), code, detail))


def header_functions(path: str = HEADER_PATH) -> list[str]:
    """Names of the functions declared in include/hashbatch.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hash_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libhashbatch.so is not built (expected at %s); run "
                "paper_2407_09333_b300/build.py or __graft_entry__.build()" % LIB_PATH)
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def strerror(code: int) -> str:
    return lib().hash_strerror(int(code)).decode()


def digest_size(alg: int) -> int:
    return int(lib().hash_digest_size(int(alg)))


def _check(rc: int, where: str):
    if rc != 0:
        raise HashBatchError(rc, where)


# ---------------------------------------------------------------------------
# torch helpers

def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, itemsize: int, name: str):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.element_size() != itemsize:
        raise ValueError("%s must have %d-byte elements" % (name, itemsize))
    return ctypes.c_void_p(t.data_ptr())


def _out_tensor(out, n, device):
    torch = _torch()
    if out is None:
        return torch.empty((n, SLOT_BYTES), dtype=torch.uint8, device=device)
    if out.dtype != torch.uint8 or out.numel() < n * SLOT_BYTES or not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor of n*32 bytes")
    return out


def hash_batch(alg: int, packed, offsets, lengths, out=None, stream=None,
               shape: int = -1, grid: int = 0):
    """Digest slots (n, 32) uint8 of every message, one algorithm."""
    n = int(offsets.numel())
    if lengths.numel() != n:
        raise ValueError("offsets and lengths differ in length")
    out = _out_tensor(out, n, offsets.device)
    rc = lib().hash_batch_shape(
        int(alg), _dev_ptr(packed, 1, "packed"), _dev_ptr(offsets, 8, "offsets"),
        _dev_ptr(lengths, 4, "lengths"), n, _dev_ptr(out, 1, "out"),
        int(shape), int(grid), _stream_handle(stream))
    _check(rc, "hash_batch")
    return out


def hash_batch_all(packed, offsets, lengths, out=None, stream=None, shape: int = -1,
                   grid: int = 0):
    """Records (n, 96) uint8: MD5, SHA-1 and SM3 slots of every message,
    computed in one pass over the input."""
    torch = _torch()
    n = int(offsets.numel())
    if lengths.numel() != n:
        raise ValueError("offsets and lengths differ in length")
    if out is None:
        out = torch.empty((n, ALL_RECORD_BYTES), dtype=torch.uint8, device=offsets.device)
    elif out.dtype != torch.uint8 or out.numel() < n * ALL_RECORD_BYTES or not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor of n*96 bytes")
    rc = lib().hash_batch_all_shape(
        _dev_ptr(packed, 1, "packed"), _dev_ptr(offsets, 8, "offsets"),
        _dev_ptr(lengths, 4, "lengths"), n, _dev_ptr(out, 1, "out"), int(shape), int(grid),
        _stream_handle(stream))
    _check(rc, "hash_batch_all")
    return out


def hash_batch_mixed(algs, packed, offsets, lengths, out=None, stream=None,
                     shape: int = -1, grid: int = 0):
    """Digest slots (n, 32) uint8, per-message algorithm (ragged path)."""
    n = int(offsets.numel())
    if lengths.numel() != n or algs.numel() != n:
        raise ValueError("algs, offsets and lengths must have one entry per message")
    out = _out_tensor(out, n, offsets.device)
    rc = lib().hash_batch_mixed_shape(
        _dev_ptr(algs, 1, "algs"), _dev_ptr(packed, 1, "packed"),
        _dev_ptr(offsets, 8, "offsets"), _dev_ptr(lengths, 4, "lengths"), n,
        _dev_ptr(out, 1, "out"), int(shape), int(grid), _stream_handle(stream))
    _check(rc, "hash_batch_mixed")
    return out


def seg_words(prior, more):
    """Segment descriptors for hash_batch_segments: prior byte counts (a
    multiple of 64) with SEG_MORE set where more segments follow, as int64
    (the bit pattern of the C-ABI's uint64)."""
    prior = np.asarray(prior, dtype=np.uint64)
    more = np.asarray(more, dtype=bool)
    return (prior | np.where(more, np.uint64(SEG_MORE), np.uint64(0))).view(np.int64)


def hash_batch_segments(algs, packed, offsets, lengths, seg, slots, slot_index=None,
                        stream=None):
    """One call over message segments; `slots` (uint8, 32 bytes per slot)
    carries the chaining values between calls and receives the digests of
    messages whose last segment this is; message i uses slot slot_index[i]
    (CUDA int32 tensor) or, without it, slot i (see hash_batch_segments in
    the C header)."""
    n = int(offsets.numel())
    if lengths.numel() != n or algs.numel() != n or seg.numel() != n:
        raise ValueError("algs, offsets, lengths and seg must have one entry per message")
    if slot_index is None and slots.numel() < n * SLOT_BYTES:
        raise ValueError("slots must hold n*32 bytes")
    if slot_index is not None and slot_index.numel() != n:
        raise ValueError("slot_index must have one entry per message")
    if slots.dtype.itemsize != 1 or not slots.is_contiguous():
        raise ValueError("slots must be a contiguous uint8 tensor")
    rc = lib().hash_batch_segments(
        _dev_ptr(algs, 1, "algs"), _dev_ptr(packed, 1, "packed"),
        _dev_ptr(offsets, 8, "offsets"), _dev_ptr(lengths, 4, "lengths"),
        _dev_ptr(seg, 8, "seg"),
        None if slot_index is None else _dev_ptr(slot_index, 4, "slot_index"), n,
        _dev_ptr(slots, 1, "slots"), _stream_handle(stream))
    _check(rc, "hash_batch_segments")
    return slots


NOALLOC_MAX_MESSAGES = 1 << 20


def hash_batch_mixed_noalloc(algs, packed, offsets, lengths, out, stream=None):
    """hash_batch_mixed without any device allocation by the library.

    For callers that must not trigger cudaMalloc (device memory owned by
    someone else under a fixed budget, or a latency-critical loop): the
    bucketing scratch is a fixed array inside the library, so `out` must be
    supplied and n is limited to NOALLOC_MAX_MESSAGES.  Calls that overlap on
    the GPU share that array and must be ordered.
    """
    n = int(offsets.numel())
    if lengths.numel() != n or algs.numel() != n:
        raise ValueError("algs, offsets and lengths must have one entry per message")
    if out.dtype.itemsize != 1 or out.numel() < n * SLOT_BYTES or not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor of n*32 bytes")
    rc = lib().hash_batch_mixed_noalloc(
        _dev_ptr(algs, 1, "algs"), _dev_ptr(packed, 1, "packed"),
        _dev_ptr(offsets, 8, "offsets"), _dev_ptr(lengths, 4, "lengths"), n,
        _dev_ptr(out, 1, "out"), _stream_handle(stream))
    _check(rc, "hash_batch_mixed_noalloc")
    return out


DIGITS_COUNT = 10 ** 9


def hash_digits(alg: int, first: int, count: int, out=None, stream=None):
    """Digest slots (count, 32) of the 9-character decimal strings of
    first .. first + count - 1, generated on the device."""
    torch = _torch()
    out = _out_tensor(out, int(count), "cuda")
    _check(lib().hash_digits(int(alg), int(first), int(count), _dev_ptr(out, 1, "out"),
                             _stream_handle(stream)), "hash_digits")
    return out


def check_bounds(offsets, lengths, packed_len: int, status=None, stream=None):
    """Device int32 tensor: 0 when every message is inside packed_len."""
    torch = _torch()
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=offsets.device)
    rc = lib().hash_batch_check_bounds(
        _dev_ptr(offsets, 8, "offsets"), _dev_ptr(lengths, 4, "lengths"),
        int(offsets.numel()), int(packed_len), _dev_ptr(status, 4, "status"),
        _stream_handle(stream))
    _check(rc, "hash_batch_check_bounds")
    return status


def _host_ptr(a, name):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError("%s must be a host buffer" % name)
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def host_digest_bytes(alg, packed_digests: bool = False) -> int:
    """Bytes per message that hash_batch_host writes to `out`."""
    if packed_digests:
        return ALL_DIGEST_BYTES if alg == ALL else digest_size(alg)
    return ALL_RECORD_BYTES if alg == ALL else SLOT_BYTES


def hash_batch_host(alg, packed, offsets, lengths, out, algs=None, stream=None,
                    packed_digests: bool = False):
    """End-to-end call from host buffers (pinned for full speed).  `out`
    holds n 32-byte slots, or n 96-byte records for alg == ALL; with
    packed_digests, the digests back to back (16 / 20 / 32 bytes, 68 for
    ALL), which is what crosses the PCIe link."""
    n = int(len(offsets))
    packed_len = int(packed.numel() if hasattr(packed, "numel") else packed.size)
    if packed_digests and algs is not None:
        raise ValueError("packed digests need one algorithm (or ALL) for the whole batch")
    rec = host_digest_bytes(alg, packed_digests)
    out_bytes = int(out.numel() * out.element_size()) if hasattr(out, "numel") else int(out.nbytes)
    if out_bytes < n * rec or len(lengths) != n or (algs is not None and len(algs) != n):
        raise ValueError("out must hold %d bytes per message; offsets, lengths (and algs) "
                         "one entry per message" % rec)
    src = (_host_ptr(packed, "packed") if packed_len else None, packed_len,
           _host_ptr(offsets, "offsets"), _host_ptr(lengths, "lengths"), n,
           _host_ptr(out, "out"), _stream_handle(stream))
    a = -1 if alg is None else int(alg)
    if packed_digests:
        rc = lib().hash_batch_host_packed(a, *src)
    else:
        rc = lib().hash_batch_host(a, _host_ptr(algs, "algs"), *src)
    _check(rc, "hash_batch_host_packed" if packed_digests else "hash_batch_host")
    return out


def set_host_memory_limit(nbytes: int) -> int:
    """Device bytes hash_batch_host may use (0 = no limit); returns the old
    value.  Larger batches stream through two windows of nbytes/2."""
    return int(lib().hash_set_host_memory_limit(int(nbytes)))


def device_status(stream=None) -> int:
    v = ctypes.c_int(0)
    _check(lib().hash_device_status(_stream_handle(stream), ctypes.byref(v)), "hash_device_status")
    return int(v.value)


def release_device():
    _check(lib().hash_release_device(), "hash_release_device")


def set_wait_limit_ns(limit_ns: int) -> int:
    return int(lib().hash_set_wait_limit_ns(int(limit_ns)))


def selftest_wait_timeout(timeout_ns: int, stream=None):
    _check(lib().hash_selftest_wait_timeout(int(timeout_ns), _stream_handle(stream)),
           "hash_selftest_wait_timeout")


# ---------------------------------------------------------------------------
# plans (ragged path with private scratch; captured graphs)

class Plan:
    """A ragged-path plan for batches of up to `max_n` messages.

    run(...) hashes one batch on a stream with the plan's own scratch;
    capture(...) records the launch sequence as a CUDA graph for fixed
    buffers and replay(n) runs it for the first n messages of them.
    """

    def __init__(self, max_n: int, shape: int = -1, warps_per_sm: int = -1):
        h = ctypes.c_void_p()
        _check(lib().hash_plan_create(int(max_n), ctypes.byref(h)), "hash_plan_create")
        self._h = h
        self.max_n = int(max_n)
        self._keep = None
        if shape >= 0 or warps_per_sm >= 0:
            _check(lib().hash_plan_configure(h, int(shape), int(warps_per_sm)), "hash_plan_configure")

    def run(self, algs, packed, offsets, lengths, out, n=None, grid=0, stream=None):
        n = int(offsets.numel()) if n is None else int(n)
        _check(lib().hash_plan_run(self._h, _dev_ptr(algs, 1, "algs"), _dev_ptr(packed, 1, "packed"),
                                   _dev_ptr(offsets, 8, "offsets"), _dev_ptr(lengths, 4, "lengths"),
                                   n, _dev_ptr(out, 1, "out"), int(grid), _stream_handle(stream)),
               "hash_plan_run")
        return out

    def set_completion(self, msg_req, remaining, done_flags):
        """Per-request completion flags (see hash_plan_set_completion):
        msg_req and remaining are CUDA uint32/int32 tensors, done_flags a
        pinned CPU int32 tensor."""
        if done_flags.is_cuda or not done_flags.is_pinned():
            raise ValueError("done_flags must be pinned host memory")
        _check(lib().hash_plan_set_completion(self._h, _dev_ptr(msg_req, 4, "msg_req"),
                                              _dev_ptr(remaining, 4, "remaining"),
                                              ctypes.c_void_p(done_flags.data_ptr())),
               "hash_plan_set_completion")
        self._flags = (msg_req, remaining, done_flags)

    def set_segments(self, seg, slot_index=None):
        """Batches of this plan are message segments described by the CUDA
        int64 tensor `seg` (see seg_words), message i using slot
        slot_index[i] if given; before the first capture."""
        _check(lib().hash_plan_set_segments(
            self._h, _dev_ptr(seg, 8, "seg"),
            None if slot_index is None else _dev_ptr(slot_index, 4, "slot_index")),
            "hash_plan_set_segments")
        self._seg = (seg, slot_index)

    def capture(self, algs, packed, offsets, lengths, out, grid=0):
        _check(lib().hash_plan_capture(self._h, _dev_ptr(algs, 1, "algs"),
                                       _dev_ptr(packed, 1, "packed"), _dev_ptr(offsets, 8, "offsets"),
                                       _dev_ptr(lengths, 4, "lengths"), _dev_ptr(out, 1, "out"),
                                       int(grid)), "hash_plan_capture")
        self._keep = (algs, packed, offsets, lengths, out)   # buffers must outlive the graph

    def replay(self, n: int, stream=None):
        _check(lib().hash_plan_replay(self._h, int(n), _stream_handle(stream)), "hash_plan_replay")

    def close(self):
        if self._h:
            lib().hash_plan_destroy(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Round:
    """A streaming round over a message ring (hash_round_* in the C header).

    `ring` is a dict of tensors: src/prior (CUDA int64), len/req/state (CUDA
    int32), alg (CUDA uint8), slots (CUDA uint8, capacity x 32),
    req_remaining (CUDA int32) and req_done (pinned CPU int32); `staging` a
    CUDA uint8 tensor (16-byte aligned) of which the round uses
    staging_bytes from the start, or None to hash segments in place (then
    staging_bytes only caps the bytes a round claims).
    """

    def __init__(self, ring: dict, max_msgs: int, staging, staging_bytes: int,
                 segment_bytes, shape: int = -1, warps_per_sm: int = 0):
        """segment_bytes: one size for every algorithm, or (MD5, SHA-1, SM3)."""
        cap = int(ring["state"].numel())
        if ring["req_done"].is_cuda or not ring["req_done"].is_pinned():
            raise ValueError("req_done must be pinned host memory")
        if staging is not None and int(staging_bytes) > staging.numel():
            raise ValueError("staging_bytes exceeds the staging tensor")
        self._ring = HbRing(
            cap, _dev_ptr(ring["src"], 8, "src"), _dev_ptr(ring["prior"], 8, "prior"),
            _dev_ptr(ring["len"], 4, "len"), _dev_ptr(ring["req"], 4, "req"),
            _dev_ptr(ring["alg"], 1, "alg"), _dev_ptr(ring["state"], 4, "state"),
            _dev_ptr(ring["slots"], 1, "slots"), _dev_ptr(ring["req_remaining"], 4, "req_remaining"),
            ctypes.c_void_p(ring["req_done"].data_ptr()), int(ring["req_remaining"].numel()))
        if isinstance(segment_bytes, int):
            segment_bytes = (segment_bytes,) * 3
        seg = (_c_u32 * 3)(*[int(x) for x in segment_bytes])
        h = ctypes.c_void_p()
        _check(lib().hash_round_create(ctypes.byref(self._ring), int(max_msgs),
                                       None if staging is None else _dev_ptr(staging, 1, "staging"),
                                       int(staging_bytes),
                                       seg, int(shape), int(warps_per_sm),
                                       ctypes.byref(h)), "hash_round_create")
        self._h = h
        self._keep = (ring, staging)

    def launch(self, head: int, tail: int, stream=None):
        _check(lib().hash_round_launch(self._h, int(head), int(tail), _stream_handle(stream)),
               "hash_round_launch")

    def report(self) -> tuple[int, int]:
        seg, nb = _c_u64(0), _c_u64(0)
        _check(lib().hash_round_report(self._h, ctypes.byref(seg), ctypes.byref(nb)),
               "hash_round_report")
        return int(seg.value), int(nb.value)

    def close(self):
        if self._h:
            lib().hash_round_destroy(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gather(copies_dev, count: int, stream=None):
    """Device byte-range copies; copies_dev is a CUDA int64 tensor of shape
    (>= count, 3) holding (src address, dst address, bytes) per row."""
    _check(lib().hash_gather(_dev_ptr(copies_dev, 8, "copies"), int(count), _stream_handle(stream)),
           "hash_gather")


# ---------------------------------------------------------------------------
# tuning

def shapes() -> list[tuple[int, int, int, int]]:
    """Launch shapes: (warps per block, stages per warp, blocks per stage,
    cooperative copies 0/1)."""
    L = lib()
    out = []
    for i in range(L.hash_tune_shapes()):
        w, s, k, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(L.hash_tune_shape(i, ctypes.byref(w), ctypes.byref(s), ctypes.byref(k),
                                 ctypes.byref(c)), "hash_tune_shape")
        out.append((int(w.value), int(s.value), int(k.value), int(c.value)))
    return out


def tune_set(alg: int, shape: int):
    _check(lib().hash_tune_set(int(alg), int(shape)), "hash_tune_set")


def tune_get(alg: int) -> int:
    rc = int(lib().hash_tune_get(int(alg)))
    if rc < 0:
        raise HashBatchError(rc, "hash_tune_get")
    return rc


def tune_buckets(sub_log2: int, alg_major: int):
    """Ragged-path bucketing (hash_tune_buckets): 2^sub_log2 cost buckets per
    octave; alg_major 0 interleaved, 1 algorithm-major, 2 algorithm-major with
    MD5's two longest octaves served early."""
    _check(lib().hash_tune_buckets(int(sub_log2), int(alg_major)), "hash_tune_buckets")


def tune_mixed_warps(warps_per_sm: int):
    _check(lib().hash_tune_mixed_warps(int(warps_per_sm)), "hash_tune_mixed_warps")


def tune_relay(segment_blocks: int):
    """Segment length (64-byte blocks) of hash_batch_all's relay form for
    batches of few long messages; 0 turns it off (hash_tune_relay)."""
    _check(lib().hash_tune_relay(int(segment_blocks)), "hash_tune_relay")


def all_uses_relay(n: int) -> bool:
    """Whether hash_batch_all of n messages takes the relay form here."""
    rc = int(lib().hash_all_uses_relay(int(n)))
    _check(rc if rc < 0 else 0, "hash_all_uses_relay")
    return rc == 1


def tune_occupancy(alg: int, shape: int) -> int:
    rc = int(lib().hash_tune_occupancy(int(alg), int(shape)))
    if rc < 0:
        raise HashBatchError(rc, "hash_tune_occupancy")
    return rc


def int_peak(op_class: int, blocks: int, threads: int, iters: int, stream=None):
    """Runs the integer-issue microbenchmark; returns per-block SM cycles."""
    torch = _torch()
    cycles = torch.zeros(blocks, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib().hash_int_peak(int(op_class), int(blocks), int(threads), int(iters),
                               ctypes.c_void_p(cycles.data_ptr()), ctypes.c_void_p(sink.data_ptr()),
                               _stream_handle(stream)), "hash_int_peak")
    return cycles


def int_peak_ops_per_iter() -> int:
    return int(lib().hash_int_peak_ops_per_iter())


# ---------------------------------------------------------------------------
# convenience: move a workloads.Batch to the device

def to_device(batch, device="cuda"):
    """(packed, offsets, lengths[, algs]) as CUDA tensors from a workloads.Batch."""
    torch = _torch()
    packed = torch.from_numpy(np.ascontiguousarray(batch.packed)).to(device)
    if packed.numel() == 0:
        packed = torch.zeros(16, dtype=torch.uint8, device=device)
    offsets = torch.from_numpy(batch.offsets.view(np.int64)).to(device)
    lengths = torch.from_numpy(batch.lengths.view(np.int32)).to(device)
    algs = None
    if batch.algs is not None:
        algs = torch.from_numpy(batch.algs).to(device)
    return packed, offsets, lengths, algs
