"""The allocation-free dense-LU entry point, poro_lu_predict_static.

It exists for callers that cannot call cudaMalloc (a fixed device-memory
budget owned by an outer framework's allocator, or loops that must not take
the synchronisation cudaMalloc/cudaFree may imply); its factors live in a
64 MiB array inside the library.  Checked here through the C ABI against the
allocating path (poro_lu_factor + PORO_SOLVE_LU) on two calls in a row that
share the array, with the tolerance of the other predictor tests.  This file
is collected last so that a stop-at-first-failure run has already run every
other test.
"""
import numpy as np
import pytest

from _oracle_cases import population, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def test_static_lu_matches_allocating_path_on_two_calls(L):
    import torch

    N, n = 3, 12
    d = population(n, N, seed=900)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        q0 = torch.tensor(d["Q0"], device="cuda")
        B = q0.shape[2]
        stream = torch.cuda.current_stream().cuda_stream

        def buffers(k):
            return (torch.full((k, 13, B, N + 1), np.nan, dtype=torch.float64, device="cuda"),
                    torch.full((k, 13, B), np.nan, dtype=torch.float64, device="cuda"))

        # the existing (allocating) entry point on all elements
        L.poro_lu_factor(ctx, 0, n)
        ref_qt, ref_io = buffers(n)
        L.poro_predict_dev(ctx, 0, n, q0.data_ptr(), ref_qt.data_ptr(), ref_io.data_ptr(), L.PORO_SOLVE_LU, stream)
        L.poro_lu_release(ctx)
        # two calls in a row on the shared array: 7 elements (the most that fit
        # at N = 3), then 5 other elements over the first call's leftovers
        calls = [(2, 7), (0, 5)]
        outs = []
        for first, count in calls:
            qt, io = buffers(count)
            L.poro_lu_predict_static(ctx, first, count, q0[first:first + count].data_ptr(), qt.data_ptr(),
                                     io.data_ptr(), stream)
            torch.cuda.synchronize()
            outs.append((qt.cpu().numpy(), io.cpu().numpy()))
        rq, ri = ref_qt.cpu().numpy(), ref_io.cpu().numpy()
        for (first, count), (qt, io) in zip(calls, outs):
            for k in range(count):
                assert rel_l2(qt[k], rq[first + k]) <= TOL
                assert rel_l2(io[k], ri[first + k]) <= TOL
    finally:
        L.poro_destroy(ctx)


def test_static_lu_rejects_oversized_batches(L):
    import torch

    for N, count in ((3, 8), (5, 1)):
        d = population(count, N, seed=901)
        ctx = L.poro_create(0, N, L.PORO_FP64)
        try:
            L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
            q0 = torch.tensor(d["Q0"], device="cuda")
            with pytest.raises(L.PoroError) as ex:
                L.poro_lu_predict_static(ctx, 0, count, q0.data_ptr(), None, None)
            assert ex.value.status == L.PORO_EINVAL
            assert "static buffer holds" in str(ex.value)
        finally:
            L.poro_destroy(ctx)


def test_static_lu_one_element_n4_integrated_only_on_its_own_stream(L):
    """N = 4 with one element (the most that fits at N = 4), only the
    time-integrated output (Qt_dev = NULL), on a caller stream other than the
    context's, twice in a row; against poro_lu_factor + PORO_SOLVE_LU."""
    import torch

    N, n = 4, 3
    d = population(n, N, seed=902)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        q0 = torch.tensor(d["Q0"], device="cuda")
        B = q0.shape[2]
        L.poro_lu_factor(ctx, 0, n)
        ref_io = torch.full((n, 13, B), np.nan, dtype=torch.float64, device="cuda")
        L.poro_predict_dev(ctx, 0, n, q0.data_ptr(), None, ref_io.data_ptr(), L.PORO_SOLVE_LU, None)
        L.poro_sync(ctx)
        L.poro_lu_release(ctx)
        side = torch.cuda.Stream()
        outs = []
        for first in (2, 1):
            io = torch.full((1, 13, B), np.nan, dtype=torch.float64, device="cuda")
            # one N = 4 element is 13 x 35 doubles, not a multiple of 16 bytes:
            # the element's Q0 is passed from its own (aligned) buffer
            q1 = q0[first:first + 1].clone()
            L.poro_lu_predict_static(ctx, first, 1, q1.data_ptr(), None, io.data_ptr(), side.cuda_stream)
            side.synchronize()
            outs.append((first, io.cpu().numpy()[0]))
        ri = ref_io.cpu().numpy()
        for first, io in outs:
            assert rel_l2(io, ri[first]) <= TOL
    finally:
        L.poro_destroy(ctx)
