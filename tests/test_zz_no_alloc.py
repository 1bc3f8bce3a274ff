"""ivhd_eval_qnx_static: the allocation-free Q_NX entry point.

It serves callers that cannot let the library allocate device memory (see
its declaration in include/ivhd.h).  Its result must equal the allocating
ivhd_eval_qnx on the same inputs -- Q_NX is a ratio of integer hit counts, so
the tolerance is zero -- on two calls in a row, which share the fixed scratch
array, including a second call with fewer rows than the first.  Around every
call nothing may be allocated: the library's own allocation count and
PyTorch's allocation counters stay unchanged, and an allocation failure armed
before the call is still pending after it (the next allocating call consumes
it).  This file is collected last so that a run stopping at the first failure
has run everything else already.
"""
import contextlib
import ctypes
import gc

import numpy as np
import pytest
import torch

from paper_2303_05455_gb300 import _lib, ivhd, synth

pytestmark = pytest.mark.gpu


def _static_qnx(L, Y, knn, rows, lowd):
    q = ctypes.c_double()
    st = L.ivhd_eval_qnx_static(Y.data_ptr(), Y.shape[0], knn.data_ptr(), knn.shape[1],
                                rows.data_ptr(), rows.numel(),
                                lowd.data_ptr() if lowd is not None else None, ctypes.byref(q),
                                torch.cuda.current_stream().cuda_stream or None)
    return st, q.value


@contextlib.contextmanager
def _no_collection():
    """Objects of earlier tests are freed first, and not while counting (their
    destructors would lower the library's live-allocation count mid-call)."""
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()


def _alloc_counters(L):
    torch.cuda.synchronize()
    stats = torch.cuda.memory_stats()
    return (L.ivhd_test_live_allocs(), stats.get("allocation.all.allocated", 0),
            stats.get("num_alloc_retries", 0), torch.cuda.memory_reserved())


def test_static_qnx_matches_allocating_entry_point_on_consecutive_calls():
    L = _lib.load()
    M, k = 40_000, 5
    knn = torch.from_numpy(synth.random_knn_graph(M, k, 31)).cuda()
    Y = torch.from_numpy(synth.uniform_positions(M, 8)).cuda()
    Y[:4000] = torch.round(Y[:4000] * 16) / 16          # exact ties in the neighbour search
    for call, n in enumerate((30_000, 1_000)):          # second call: fewer rows, stale scratch
        rows = torch.from_numpy(synth.sample_rows(M, n, 100 + call)).cuda()
        low = torch.empty((n, k), dtype=torch.int32, device="cuda")
        with _no_collection():
            before = _alloc_counters(L)
            st, q = _static_qnx(L, Y, knn, rows, low)
            assert st == 0, st
            assert _alloc_counters(L) == before
        q_ref, low_ref = ivhd.eval_qnx(Y, knn, rows, return_lowd=True)
        assert q == q_ref
        assert torch.equal(low, low_ref)
        assert 0.0 <= q <= 1.0


def test_static_qnx_rejects_more_rows_than_its_scratch():
    L = _lib.load()
    M, k = 2000, 3
    knn = torch.from_numpy(synth.random_knn_graph(M, k, 2)).cuda()
    Y = torch.from_numpy(synth.uniform_positions(M, 1)).cuda()
    rows = torch.zeros(8192 * 128 + 1, dtype=torch.int64, device="cuda")
    st, _ = _static_qnx(L, Y, knn, rows, None)
    assert st == -1
    # the entry point stays usable after the rejection
    rows = torch.arange(M, dtype=torch.int64, device="cuda")
    st, q = _static_qnx(L, Y, knn, rows, None)
    assert st == 0 and q == ivhd.eval_qnx(Y, knn, rows)


def test_static_qnx_makes_no_allocation_request():
    """An allocation failure armed before the call is still pending after it."""
    L = _lib.load()
    M, k = 3000, 4
    knn = torch.from_numpy(synth.random_knn_graph(M, k, 3)).cuda()
    Y = torch.from_numpy(synth.uniform_positions(M, 4)).cuda()
    rows = torch.arange(M, dtype=torch.int64, device="cuda")
    q_ref = ivhd.eval_qnx(Y, knn, rows)
    try:
        L.ivhd_test_fail_alloc(0)                    # the next allocation request fails
        st, q = _static_qnx(L, Y, knn, rows, None)
        assert st == 0 and q == q_ref
        out = ctypes.c_double()
        st = L.ivhd_eval_qnx(Y.data_ptr(), M, knn.data_ptr(), k, rows.data_ptr(), M, None,
                             ctypes.byref(out), torch.cuda.current_stream().cuda_stream or None)
        assert st == -3                              # IVHD_ERR_OOM: the armed failure was pending
    finally:
        L.ivhd_test_fail_alloc(-1)
    st, q = _static_qnx(L, Y, knn, rows, None)
    assert st == 0 and q == q_ref


def test_static_qnx_rejects_row_ids_out_of_range():
    L = _lib.load()
    M, k = 2000, 3
    knn = torch.from_numpy(synth.random_knn_graph(M, k, 5)).cuda()
    Y = torch.from_numpy(synth.uniform_positions(M, 6)).cuda()
    for bad in (M, -1):
        rows = torch.arange(300, dtype=torch.int64, device="cuda")
        rows[137] = bad
        st, _ = _static_qnx(L, Y, knn, rows, None)
        assert st == -2, (bad, st)                   # IVHD_ERR_INDEX, nothing dereferenced
    rows = torch.arange(300, dtype=torch.int64, device="cuda")
    st, q = _static_qnx(L, Y, knn, rows, None)       # the scratch carries nothing over
    assert st == 0 and q == ivhd.eval_qnx(Y, knn, rows)
