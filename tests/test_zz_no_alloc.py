"""gj_self_join_noalloc: the self-join for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc during a join -- a service
whose device memory is reserved up front by a caching allocator, or a
latency-bound loop that must not enter the driver's allocator.  The
allocation-free entry point keeps its scratch in a fixed device array and
writes pairs straight into the caller's device buffer.  These tests call it
through the C ABI twice in a row (the second call finds the first call's
scratch contents) and check it against gj_self_join on the same index.  The
file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tests.parity import keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")


def _reference(ix, n):
    out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    st, m = gj.gj_self_join(ix.h, out)
    assert st == gj.GJ_OK and m == n
    return keys(out.cpu().numpy().view(np.uint32))


def test_noalloc_matches_gj_self_join_on_two_calls_in_a_row():
    X = synth.mixture(20_000, 18, 41)
    with gj.Index(X, 0.3, k=3) as ix:
        n = ix.count()
        ref = _reference(ix, n)
        for _ in range(2):
            out = torch.full((n + 64, 2), -1, dtype=torch.int32, device="cuda")
            st, m = gj.gj_self_join_noalloc(ix.h, out)
            assert st == gj.GJ_OK and m == n
            got = out[:m].cpu().numpy().view(np.uint32)
            assert np.array_equal(keys(got), ref)           # same pairs as gj_self_join
            assert int(out[m:].min().item()) == -1          # nothing written past |R|


def test_noalloc_count_capacity_and_parts():
    X = synth.uniform(12_000, 16, 42)
    with gj.Index(X, 0.85, k=2) as ix:
        n = ix.count()
        ref = _reference(ix, n)
        st, m = gj.gj_self_join_noalloc(ix.h, None)         # count only
        assert st == gj.GJ_OK and m == n
        small = torch.empty((n // 2, 2), dtype=torch.int32, device="cuda")
        st, m = gj.gj_self_join_noalloc(ix.h, small)
        assert st == gj.GJ_ERR_CAPACITY and m == n
        part_keys = []
        for p in range(3):
            cnt = gj.gj_self_join_noalloc(ix.h, None, part=p, nparts=3)[1]
            buf = torch.empty((max(cnt, 1), 2), dtype=torch.int32, device="cuda")
            st, m = gj.gj_self_join_noalloc(ix.h, buf, part=p, nparts=3)
            assert st == gj.GJ_OK and m == cnt
            part_keys.append(keys(buf[:m].cpu().numpy().view(np.uint32)))
        allk = np.sort(np.concatenate(part_keys))
        assert np.array_equal(allk, ref)


def test_noalloc_rejects_host_output_and_too_many_work_items():
    X = synth.uniform(2000, 4, 43)
    with gj.Index(X, 0.2, k=2) as ix:
        host = np.empty((10, 2), dtype=np.uint32)
        st, _ = gj.gj_self_join_noalloc(ix.h, host)
        assert st == gj.GJ_ERR_INVALID_ARG
    # one point per cell: 1.1 million work items, above the 1,048,512 the scratch holds
    P = np.arange(1_100_000, dtype=np.float64)[:, None]
    with gj.Index(P, 0.25, k=1) as ix:
        assert ix.info()["work_items"] > 1_048_512
        st, _ = gj.gj_self_join_noalloc(ix.h, None)
        assert st == gj.GJ_ERR_TOO_LARGE


def test_noalloc_rejects_a_tensor_core_index_and_counts_into_a_zero_capacity_buffer():
    X = synth.uniform(3000, 8, 44)
    with gj.Index(X, 0.3, k=2, flags=gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER) as ix:
        st, _ = gj.gj_self_join_noalloc(ix.h, None)
        assert st == gj.GJ_ERR_INVALID_ARG          # tensor-core indices use gj_self_join
    with gj.Index(X, 0.3, k=2) as ix:
        n = ix.count()
        assert n > 0
        buf = torch.full((1, 2), -1, dtype=torch.int32, device="cuda")
        cnt = C.c_uint64(0)
        st = gj.load().gj_self_join_noalloc(ix.h, 0, 1, buf.data_ptr(), 0, C.byref(cnt))
        assert st == gj.GJ_ERR_CAPACITY and cnt.value == n    # non-NULL, cap 0: counted, nothing written
        assert int(buf.min().item()) == -1


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second visible device")
def test_noalloc_rejects_another_devices_buffer():
    X = synth.uniform(2000, 4, 45)
    with gj.Index(X, 0.2, k=2) as ix:
        other = torch.empty((10, 2), dtype=torch.int32, device="cuda:1")
        st, _ = gj.gj_self_join_noalloc(ix.h, other)     # checked on the host, nothing launched
        assert st == gj.GJ_ERR_INVALID_ARG
