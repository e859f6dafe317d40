"""The connection export that allocates nothing (sci_connections_noalloc).

Callers whose device memory is owned by a pooling allocator, or who cannot afford the
device-wide synchronisation of cudaFree, need an export that never allocates.  This
entry point keeps its scratch in a fixed array inside the library.  Here it is called
through the C ABI and checked against the allocating export, sci_connections(), on two
calls in a row (the scratch array is reused, so the second call must not see stale
contents), and its size limit is checked.  This file sorts last so that a failure here
stops a -x run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _call(ctx, rb, re, cap):
    L = sci.load()
    cnt = np.zeros(1, dtype=np.int64)
    rows = np.full(max(cap, 1), -7, dtype=np.int64)
    J = np.full(max(cap, 1), -7, dtype=np.int64)
    deg = np.zeros(max(cap, 1), dtype=np.int8)
    ph = np.zeros(max(cap, 1), dtype=np.int8)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    rc = L.sci_connections_noalloc(ctx, rb, re, p(cnt), p(rows), p(J), p(deg), p(ph), cap)
    n = int(cnt[0])
    return rc, n, (rows[:n], J[:n], deg[:n], ph[:n])


def test_noalloc_export_matches_allocating_export(gpu):
    w = W.selected_30o(M=60000)
    H = sci.Hamiltonian.from_workload(w)
    hf = int(np.searchsorted(w.keys, w.hf_key()))
    for rb, re in ((0, 100), (hf, hf + 1), (w.M - 300, w.M), (30000, 30150), (7, 7)):
        n_ref, ref = sci.sci_connections(H.ctx, rb, re, 0)
        n_ref, ref = sci.sci_connections(H.ctx, rb, re, n_ref)
        for _ in range(2):                      # two calls in a row on the shared scratch
            rc, n, got = _call(H.ctx, rb, re, n_ref)
            assert rc == sci.SCI_OK
            assert n == n_ref
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)


def test_noalloc_export_takes_no_device_memory(gpu):
    """The point of the entry point: a call changes the device's free memory by nothing,
    the first call on a fresh context included (its scratch was committed when the first
    context was created)."""
    torch = gpu
    w = W.selected_30o(M=60000)
    H = sci.Hamiltonian.from_workload(w)
    rb, re = 30000, 30150          # a range well inside the fixed scratch's 524,288 pairs
    n_ref, _ = sci.sci_connections(H.ctx, rb, re, 0)
    assert 0 < n_ref <= 524288
    torch.cuda.synchronize()
    for _ in range(3):
        free0 = torch.cuda.mem_get_info()[0]
        rc, n, _ = _call(H.ctx, rb, re, n_ref)
        free1 = torch.cuda.mem_get_info()[0]
        assert rc == sci.SCI_OK and n == n_ref
        assert free1 == free0, (free0, free1)


def test_noalloc_export_rejects_ranges_beyond_its_scratch(gpu):
    w = W.selected_30o(M=60000)
    H = sci.Hamiltonian.from_workload(w)
    total = H.count_pairs()
    assert total > 524288
    rc, n, _ = _call(H.ctx, 0, w.M, 16)
    assert rc == sci.SCI_ERR_OVERFLOW and n == total
    assert "split the range" in sci.sci_last_error(H.ctx)
    # the context and the scratch stay usable after the rejection
    n_ref, ref = sci.sci_connections(H.ctx, 10, 40, 1 << 20)
    rc, n, got = _call(H.ctx, 10, 40, n_ref)
    assert rc == sci.SCI_OK and n == n_ref and np.array_equal(got[1], ref[1])
