"""hash_batch_mixed_noalloc: the ragged path for callers that cannot allocate.

Some callers cannot let the library call cudaMalloc -- for example when their
device memory is owned by another component under a fixed budget, or inside a
latency-critical loop that must not meet an allocation's device-wide
synchronisation.  The no-allocation entry point keeps its bucketing scratch in
a fixed array inside the library.  These tests call it through the C-ABI and
check that its digest slots are byte-for-byte those of hash_batch_mixed, on
two calls in a row (the second, smaller batch runs on scratch that still holds
the first call's contents).  The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2407_09333_b300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09333_b300 import api, build
    build.build()
    api.lib()
    return api


def _reference_and_noalloc(hb, batch):
    packed, off, ln, algs = hb.to_device(batch)
    want = hb.hash_batch_mixed(algs, packed, off, ln)
    got = torch.full((batch.n, 32), 0xA5, dtype=torch.uint8, device="cuda")
    hb.hash_batch_mixed_noalloc(algs, packed, off, ln, got)
    torch.cuda.synchronize()
    return want.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_mixed_path_on_two_calls_in_a_row(hb):
    first = workloads.ragged(30000, seed=31, max_len=6000)
    second = workloads.ragged(7000, seed=32, max_len=2000)
    second.algs[::101] = 9            # unknown code: slot stays zero in both paths
    for batch in (first, second):
        want, got = _reference_and_noalloc(hb, batch)
        assert np.array_equal(got, want)


def test_noalloc_rejects_batches_above_its_limit(hb):
    n = hb.NOALLOC_MAX_MESSAGES + 1
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    algs = torch.zeros(n, dtype=torch.uint8, device="cuda")
    off = torch.zeros(n, dtype=torch.int64, device="cuda")
    ln = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(hb.HashBatchError) as e:
        hb.hash_batch_mixed_noalloc(algs, dummy, off, ln, out)
    assert e.value.code == -3
