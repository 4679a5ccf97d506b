"""GPU parity of the dense-LU comparator (the approach the paper's
block-wise back-substitution replaces): assembled, equilibrated, factored
and solved on the device in binary64, against the oracle's dense LU and
against the block kernel.  Tolerance 1e-12 relative L2 per element."""
import numpy as np
import pytest

from _oracle_cases import oracle_predictor, population, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


@pytest.mark.parametrize("N,n", [(1, 21), (2, 21), (3, 9)])
def test_lu_matches_oracle(L, N, n):
    d = population(n, N, seed=500 + N)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_lu_factor(ctx, 0, n)
        L.poro_predict(ctx, -1, L.PORO_SOLVE_LU)
        qt_lu = L.poro_get_predictor(ctx, 0, n)
        io_lu = L.poro_get_integrated(ctx, 0, n)
        L.poro_predict(ctx, -1, L.PORO_SOLVE_BLOCK)
        qt_blk = L.poro_get_predictor(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)
    for i in range(n):
        ref = oracle_predictor(d, i, dense=True)
        assert rel_l2(qt_lu[i], ref) <= TOL
        assert rel_l2(qt_lu[i], qt_blk[i]) <= TOL
        np.testing.assert_allclose(io_lu[i], d["dt"][i] * qt_lu[i][:, :, 0], rtol=0, atol=1e-300)


def test_lu_one_cta_form_for_many_elements(L):
    """160 elements (at least one per SM): the triangular solves run one CTA
    per element (fewer elements take the blocked form tested above); against
    the block kernel on all, the dense oracle on three."""
    N, n = 2, 160
    d = population(n, N, seed=520)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_lu_factor(ctx, 0, n)
        L.poro_predict(ctx, -1, L.PORO_SOLVE_LU)
        qt_lu = L.poro_get_predictor(ctx, 0, n)
        L.poro_predict(ctx, -1, L.PORO_SOLVE_BLOCK)
        qt_blk = L.poro_get_predictor(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)
    for i in range(n):
        assert rel_l2(qt_lu[i], qt_blk[i]) <= TOL
    for i in (0, 77, 159):
        assert rel_l2(qt_lu[i], oracle_predictor(d, i, dense=True)) <= TOL


def test_lu_sub_batch_n6_matches_block(L):
    """N = 6 (s = 7,644, 467 MB of factors per element): a sub-batch of two
    elements in the middle of the population, through the device-pointer
    call, against the block kernel."""
    import torch

    N, n = 6, 6
    d = population(n, N, seed=77)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        assert L.poro_lu_bytes(N, 2) >= 2 * 7644 * 7644 * 8
        L.poro_lu_factor(ctx, 3, 2)
        q0 = torch.tensor(d["Q0"][3:5], device="cuda")
        B = q0.shape[2]
        out = {}
        for solver in (L.PORO_SOLVE_LU, L.PORO_SOLVE_BLOCK):
            qt = torch.empty((2, 13, B, N + 1), dtype=torch.float64, device="cuda")
            L.poro_predict_dev(ctx, 3, 2, q0.data_ptr(), qt.data_ptr(), None, solver,
                               torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            out[solver] = qt.cpu().numpy()
        for k in range(2):
            assert rel_l2(out[L.PORO_SOLVE_LU][k], out[L.PORO_SOLVE_BLOCK][k]) <= TOL
        with pytest.raises(L.PoroError) as ex:  # element 2 is not factored
            L.poro_predict_dev(ctx, 2, 2, q0.data_ptr(), None, None, L.PORO_SOLVE_LU)
        assert ex.value.status == L.PORO_ESTATE
        L.poro_lu_release(ctx)
        with pytest.raises(L.PoroError) as ex:
            L.poro_predict_dev(ctx, 3, 1, q0.data_ptr(), None, None, L.PORO_SOLVE_LU)
        assert ex.value.status == L.PORO_ESTATE
    finally:
        L.poro_destroy(ctx)


def test_lu_out_of_memory_is_reported(L):
    """Asking for more factors than HBM holds fails with PORO_ENOMEM and
    leaves the context usable."""
    N = 6
    d = population(3, N, seed=3)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, np.tile(d["vertices"], (300, 1, 1))[:900], np.tile(d["materials"], (300, 1))[:900],
                            np.tile(d["dt"], 300)[:900])
        with pytest.raises(L.PoroError) as ex:
            L.poro_lu_factor(ctx, 0, 900)  # 900 x 467 MB > HBM
        assert ex.value.status == L.PORO_ENOMEM
        L.poro_set_dofs(ctx, np.tile(d["Q0"], (300, 1, 1))[:900])
        L.poro_predict(ctx)
        qt = L.poro_get_predictor(ctx, 0, 1)
        assert rel_l2(qt[0], oracle_predictor(d, 0)) <= TOL
    finally:
        L.poro_destroy(ctx)
