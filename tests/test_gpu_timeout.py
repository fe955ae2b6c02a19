"""Failure detection of the tensor-core join without any device fault.

Every wait inside the tensor-core kernel is bounded; when one runs out the
kernel records the expiry, tells its other warps to stop, lets its copies and
MMAs in flight land, frees its tensor memory and returns, and the join reports
GJ_ERR_TIMEOUT.  A diagnostic limit of 1 ns makes the waits run out on
purpose (a phase that has not completed yet is simply not waited for), for
both output forms; the next joins on the same context and index must then be
exact.  No trap, no bad address, no unbounded wait.
"""
import numpy as np
import pytest

import synth
from tests.parity import keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")

TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


def test_wait_expiry_reports_timeout_and_the_context_stays_usable():
    X = synth.uniform(20_000, 16, 71)
    eps = 0.45
    with gj.Index(X, eps, k=1) as ip:
        ref = keys(ip.join())
    n = len(ref)
    with gj.Index(X, eps, k=1, flags=TC) as it:
        dev = torch.empty((n + 8, 2), dtype=torch.int32, device="cuda")
        host = np.empty((n + 8, 2), dtype=np.uint32)
        try:
            gj.gj_debug_set_wait_limit(1)
            st, _ = gj.gj_self_join(it.h, dev)          # direct form, device output
            assert st == gj.GJ_ERR_TIMEOUT
            st, _ = gj.gj_self_join(it.h, None)         # count only
            assert st == gj.GJ_ERR_TIMEOUT
            st, _ = gj.gj_self_join(it.h, host)         # host output
            assert st == gj.GJ_ERR_TIMEOUT
        finally:
            gj.gj_debug_set_wait_limit(0)
        torch.cuda.synchronize()                       # the context is still usable
        for buf in (dev, host):
            st, m = gj.gj_self_join(it.h, buf)
            assert st == gj.GJ_OK and m == n
            got = buf[:m].cpu().numpy().view(np.uint32) if isinstance(buf, torch.Tensor) else buf[:m]
            assert np.array_equal(keys(got), ref)
    with gj.Index(X, eps, k=1, flags=TC | gj.GJ_HOST_BATCHED) as ib:
        host = np.empty((n + 8, 2), dtype=np.uint32)
        try:
            gj.gj_debug_set_wait_limit(1)
            st, _ = gj.gj_self_join(ib.h, host)         # staged form (result batches)
            assert st == gj.GJ_ERR_TIMEOUT
        finally:
            gj.gj_debug_set_wait_limit(0)
        st, m = gj.gj_self_join(ib.h, host)
        assert st == gj.GJ_OK and m == n and np.array_equal(keys(host[:m]), ref)
    with gj.Index(X, eps, k=1, flags=TC) as it2:           # and a new index on the same context
        assert np.array_equal(keys(it2.join()), ref)


def test_wait_expiry_in_the_tensor_core_similarity_join():
    E = synth.uniform(20_000, 16, 73)
    Q = synth.uniform(5_000, 16, 74)
    eps = 0.45
    with gj.Index(E, eps, k=1) as ip:
        st, m = gj.gj_join_qe(ip.h, Q, None)
        assert st == gj.GJ_OK
        ref = keys(ip.join_qe(Q))
    with gj.Index(E, eps, k=1, flags=TC) as it:
        out = torch.empty((m + 8, 2), dtype=torch.int32, device="cuda")
        try:
            gj.gj_debug_set_wait_limit(1)
            st, _ = gj.gj_join_qe(it.h, torch.from_numpy(Q).cuda(), out)
            assert st == gj.GJ_ERR_TIMEOUT
        finally:
            gj.gj_debug_set_wait_limit(0)
        torch.cuda.synchronize()
        st, m2 = gj.gj_join_qe(it.h, Q, out)
        assert st == gj.GJ_OK and m2 == m
        assert np.array_equal(keys(out[:m].cpu().numpy().view(np.uint32)), ref)
