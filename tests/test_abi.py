"""The C-ABI library loads and exports every symbol include/hashbatch.h
declares; argument checks that return before any CUDA call behave as
documented.  No GPU needed."""
import ctypes

import pytest

from paper_2407_09333_b300 import api


@pytest.fixture(scope="module")
def lib():
    from paper_2407_09333_b300 import build
    build.build()
    return api.lib()


def test_every_declared_function_is_exported(lib):
    names = api.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(api._SIGNATURES), set(names) - set(api._SIGNATURES)


def test_digest_sizes_and_strerror(lib):
    assert [api.digest_size(a) for a in (0, 1, 2, 3, -1)] == [16, 20, 32, 0, 0]
    for code in range(0, -11, -1):
        assert lib.hash_strerror(code)
    assert api.strerror(-1) == "invalid algorithm code"
    assert api.strerror(-99) == "unknown error code"


def test_argument_checks_before_cuda(lib):
    buf = ctypes.create_string_buffer(64)
    p = ctypes.c_void_p(ctypes.addressof(buf))
    # invalid algorithm
    assert lib.hash_batch(3, p, p, p, 1, p, None) == -1
    assert lib.hash_batch(-1, p, p, p, 1, p, None) == -1
    # empty batch is a no-op even with null pointers
    assert lib.hash_batch(0, None, None, None, 0, None, None) == 0
    assert lib.hash_batch_mixed(None, None, None, None, 0, None, None) == 0
    # null pointers
    assert lib.hash_batch(0, None, p, p, 1, p, None) == -2
    assert lib.hash_batch(1, p, None, p, 1, p, None) == -2
    assert lib.hash_batch(2, p, p, None, 1, p, None) == -2
    assert lib.hash_batch(2, p, p, p, 1, None, None) == -2
    assert lib.hash_batch_mixed(None, p, p, p, 1, p, None) == -2
    # digest slots must be 16-byte aligned
    odd = ctypes.c_void_p(((ctypes.addressof(buf) + 15) & ~15) + 4)
    assert lib.hash_batch(0, p, p, p, 1, odd, None) == -7
    # size limits
    assert lib.hash_batch(0, p, p, p, 1 << 40, p, None) == -3
    assert lib.hash_batch_mixed(p, p, p, p, 1 << 31, p, None) == -3
    # host path argument checks
    assert lib.hash_batch_host(5, None, p, 1, p, p, 1, p, None) == -1
    assert lib.hash_batch_host(0, None, p, 1, None, p, 1, p, None) == -2
    assert lib.hash_batch_host(0, None, None, 0, None, None, 0, None, None) == 0
    assert lib.hash_batch_host_packed(3, p, 1, p, p, 1, p, None) == -1
    assert lib.hash_batch_host_packed(0, p, 1, None, p, 1, p, None) == -2
    assert lib.hash_batch_host_packed(0, None, 0, None, None, 0, None, None) == 0


def test_tuning_shape_table(lib):
    n = lib.hash_tune_shapes()
    assert n >= 4
    w, s, k, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    refs = [ctypes.byref(x) for x in (w, s, k, c)]
    for i in range(n):
        assert lib.hash_tune_shape(i, *refs) == 0
        assert w.value in (1, 2, 4, 8, 16) and 2 <= s.value <= 4 and k.value in (1, 2, 4)
        assert c.value in (0, 1)
    assert lib.hash_tune_shape(n, *refs) == -10
    assert lib.hash_tune_set(0, n) == -10
    assert lib.hash_tune_set(7, 0) == -1


def test_int_peak_argument_checks(lib):
    assert lib.hash_int_peak(0, 1, 32, 1, None, None, None) == -2
    buf = ctypes.create_string_buffer(64)
    p = ctypes.c_void_p(ctypes.addressof(buf))
    assert lib.hash_int_peak(0, 0, 32, 1, p, p, None) == -10
    assert lib.hash_int_peak(0, 1, 2048, 1, p, p, None) == -10
    assert lib.hash_int_peak_ops_per_iter() == 32
    assert lib.hash_int_peak(19, 1, 32, 1, p, p, None) == -10


def test_product_path_does_not_import_oracle():
    import paper_2407_09333_b300
    import os
    pkg = os.path.dirname(paper_2407_09333_b300.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "hash_oracle" not in text and "liboracle" not in text, f


def test_segment_and_round_argument_checks(lib):
    buf = ctypes.create_string_buffer(256)
    p = ctypes.c_void_p((ctypes.addressof(buf) + 15) & ~15)
    # segments: empty batch, missing descriptors, missing buffers
    assert lib.hash_batch_segments(None, None, None, None, None, None, 0, None, None) == 0
    assert lib.hash_batch_segments(p, p, p, p, None, None, 1, p, None) == -2
    assert lib.hash_batch_segments(p, None, p, p, p, None, 1, p, None) == -2
    assert lib.hash_batch_segments(p, p, p, p, p, None, 1 << 31, p, None) == -3
    assert lib.hash_plan_set_segments(None, p, None) == -2
    # rounds: every check below returns before any CUDA call
    seg = (ctypes.c_uint32 * 3)(64, 64, 64)
    h = ctypes.c_void_p()
    assert lib.hash_round_create(None, 16, p, 4096, seg, -1, 0, ctypes.byref(h)) == -2
    ring = api.HbRing(64, p, p, p, p, p, p, p, p, p, 4)
    assert lib.hash_round_create(ctypes.byref(ring), 16, p, 4096, None, -1, 0, ctypes.byref(h)) == -2
    bad = api.HbRing(48, p, p, p, p, p, p, p, p, p, 4)           # not a power of two
    assert lib.hash_round_create(ctypes.byref(bad), 16, p, 4096, seg, -1, 0, ctypes.byref(h)) == -10
    nul = api.HbRing(64, p, p, p, p, p, None, p, p, p, 4)        # no state array
    assert lib.hash_round_create(ctypes.byref(nul), 16, p, 4096, seg, -1, 0, ctypes.byref(h)) == -2
    assert lib.hash_round_create(ctypes.byref(ring), 1 << 23, p, 4096, seg, -1, 0,
                                 ctypes.byref(h)) == -3
    odd = (ctypes.c_uint32 * 3)(64, 100, 64)                     # not a multiple of 64
    assert lib.hash_round_create(ctypes.byref(ring), 16, p, 4096, odd, -1, 0, ctypes.byref(h)) == -10
    mis = ctypes.c_void_p(p.value + 4)                           # staging not 16-byte aligned
    assert lib.hash_round_create(ctypes.byref(ring), 16, mis, 4096, seg, -1, 0, ctypes.byref(h)) == -7
    assert lib.hash_round_create(ctypes.byref(ring), 16, p, 4096, seg, 999, 0, ctypes.byref(h)) == -10
    assert lib.hash_round_launch(None, 0, 0, None) == -2
    assert lib.hash_round_report(None, None, None) == -2
    assert lib.hash_round_destroy(None) == 0


def test_digits_argument_checks(lib):
    buf = ctypes.create_string_buffer(64)
    p = ctypes.c_void_p((ctypes.addressof(buf) + 15) & ~15)
    assert lib.hash_digits(3, 0, 1, p, None) == -1
    assert lib.hash_digits(0, 0, 0, None, None) == 0
    assert lib.hash_digits(0, 10 ** 9, 1, p, None) == -3
    assert lib.hash_digits(0, 10 ** 9 - 1, 2, p, None) == -3
    assert lib.hash_digits(0, 0, 1, None, None) == -2
    assert lib.hash_digits(0, 0, 1, ctypes.c_void_p(p.value + 4), None) == -7


def test_host_digest_layouts():
    import numpy as np
    assert [api.host_digest_bytes(a) for a in (0, 1, 2, api.ALL)] == [32, 32, 32, 96]
    assert [api.host_digest_bytes(a, True) for a in (0, 1, 2, api.ALL)] == [16, 20, 32, 68]
    packed = np.zeros(64, np.uint8)
    off = np.zeros(2, np.uint64)
    ln = np.zeros(2, np.uint32)
    # these are refused before any library call
    with pytest.raises(ValueError):
        api.hash_batch_host(api.SHA1, packed, off, ln, np.zeros((2, 16), np.uint8), packed_digests=True)
    with pytest.raises(ValueError):
        api.hash_batch_host(None, packed, off, ln, np.zeros((2, 32), np.uint8),
                            algs=np.zeros(2, np.uint8), packed_digests=True)
    with pytest.raises(ValueError):
        api.hash_batch_host(api.ALL, packed, off, ln, np.zeros((2, 68), np.uint8))
