"""GPU parity of the FP64 space-time predictor (Algorithm 3 kernel) against
the FP64 oracle, through the C ABI.

Tolerance: relative L2 over the 13 B (N+1) DOFs of every element
<= 1e-12 (FP64 GPU vs oracle).  Oracle: dense LU of Eq. stp-lineq on a
subset, Algorithm 3 as plain loops (pinned to the dense solve) on the rest.
"""
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


def _run_host(L, d, prec=0):
    ctx = L.poro_create(0, d["N"], prec)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        n = d["Q0"].shape[0]
        return L.poro_get_predictor(ctx, 0, n), L.poro_get_integrated(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)


@pytest.mark.parametrize("N,n,n_dense", [(1, 37, 37), (2, 37, 37), (3, 37, 12), (4, 21, 4), (5, 13, 2), (6, 9, 1)])
def test_fp64_predictor_matches_oracle(L, N, n, n_dense):
    d = population(n, N, seed=100 + N)
    qt, iout = _run_host(L, d)
    for i in range(n):
        ref = oracle_predictor(d, i, dense=i < n_dense)
        assert rel_l2(qt[i], ref) <= TOL, f"element {i}: {rel_l2(qt[i], ref):.3e}"
        # time integration over the own step: I = dt * Qt[:, :, 0]
        np.testing.assert_allclose(iout[i], d["dt"][i] * ref[:, :, 0], rtol=0,
                                   atol=TOL * np.abs(d["dt"][i] * ref[:, :, 0]).max())


@pytest.mark.parametrize("visc", [0.0, 100.0])
def test_fp64_inviscid_and_very_stiff(L, visc):
    """E = 0 (inviscid: no source) and a 100x stiffer Darcy term."""
    d = population(11, 4, seed=7, viscosity_scale=visc)
    qt, _ = _run_host(L, d)
    for i in range(11):
        assert rel_l2(qt[i], oracle_predictor(d, i)) <= TOL


def test_zero_input_gives_zero(L):
    d = population(5, 3, seed=1)
    d["Q0"] = np.zeros_like(d["Q0"])
    qt, iout = _run_host(L, d)
    assert np.all(qt == 0.0) and np.all(iout == 0.0)


def test_device_pointer_subrange_and_empty(L):
    """poro_predict_dev on a sub-range [first, first+count) with torch device
    buffers; count = 0 is a no-op."""
    import torch

    N, n = 3, 50
    d = population(n, N, seed=21)
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        first, count = 17, 23
        q0 = torch.tensor(d["Q0"][first:first + count], device="cuda")
        qt = torch.full((count, 13, q0.shape[2], N + 1), np.nan, dtype=torch.float64, device="cuda")
        io = torch.empty((count, 13, q0.shape[2]), dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        L.poro_predict_dev(ctx, first, count, q0.data_ptr(), qt.data_ptr(), io.data_ptr(),
                           stream=s.cuda_stream)
        L.poro_predict_dev(ctx, first, 0, q0.data_ptr(), qt.data_ptr(), io.data_ptr(), stream=s.cuda_stream)
        torch.cuda.synchronize()
        qt = qt.cpu().numpy()
        for k in range(count):
            assert rel_l2(qt[k], oracle_predictor(d, first + k)) <= TOL
        with pytest.raises(L.PoroError) as ex:
            L.poro_predict_dev(ctx, 40, 20, q0.data_ptr(), None, None)
        assert ex.value.status == L.PORO_EINVAL
    finally:
        L.poro_destroy(ctx)


def test_state_errors(L):
    ctx = L.poro_create(0, 2, L.PORO_FP64)
    try:
        with pytest.raises(L.PoroError) as ex:
            L.poro_predict(ctx)
        assert ex.value.status == L.PORO_ESTATE
        with pytest.raises(L.PoroError) as ex:
            L.poro_predict(ctx, cluster=3)
        assert ex.value.status == L.PORO_EINVAL
    finally:
        L.poro_destroy(ctx)
    with pytest.raises(L.PoroError) as ex:
        L.poro_create(0, 9, L.PORO_FP64)
    assert ex.value.status == L.PORO_EUNSUPPORTED


def test_full_size_sampled(L):
    """The benchmark workload (200,000 isolated elements at N = 6, the bench
    launch configuration): sampled elements against the oracle."""
    import torch

    N, n = 6, 200_000
    from paper_2108_10565_gb300 import inputs

    d = inputs.isolated_elements(n, N)
    dt = L.poro_cfl_dt(N, d["vertices"], d["materials"])
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], dt)
        q0 = torch.from_numpy(d["Q0"]).cuda()
        B = q0.shape[2]
        qt = torch.empty((n, 13, B, N + 1), dtype=torch.float64, device="cuda")
        io = torch.empty((n, 13, B), dtype=torch.float64, device="cuda")
        L.poro_predict_dev(ctx, 0, n, q0.data_ptr(), qt.data_ptr(), io.data_ptr(),
                           stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        rng = np.random.default_rng(0)
        idx = [0, n - 1] + list(rng.choice(n, 10, replace=False))
        from oracle import geometry
        for i in idx:
            dt_o = geometry.cfl_dt(d["vertices"][i], inputs.material_dict(d["materials"][i]), N)
            assert dt[i] == pytest.approx(dt_o, rel=1e-13)
            sub = {"N": N, "vertices": d["vertices"][i:i + 1], "materials": d["materials"][i:i + 1],
                   "Q0": d["Q0"][i:i + 1], "dt": np.array([dt_o])}
            ref = oracle_predictor(sub, 0, dense=(i == 0))
            got = qt[i].cpu().numpy()
            assert rel_l2(got, ref) <= TOL
            np.testing.assert_allclose(io[i].cpu().numpy(), dt_o * ref[:, :, 0], rtol=0,
                                       atol=TOL * np.abs(dt_o * ref[:, :, 0]).max())
        assert torch.isfinite(qt).all()
    finally:
        L.poro_destroy(ctx)


def test_sync_timeout_is_recoverable(L):
    """poro_sync with a zero budget right after queuing a large predictor
    reports PORO_ETIMEOUT without hanging; a later unbounded sync succeeds."""
    import torch

    N, n = 6, 20000
    d = population(64, N, seed=5)
    reps = n // 64
    vert = np.tile(d["vertices"], (reps, 1, 1))
    mat = np.tile(d["materials"], (reps, 1))
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, vert, mat, np.tile(d["dt"], reps))
        L.poro_set_dofs(ctx, np.tile(d["Q0"], (reps, 1, 1)))
        L.poro_predict(ctx)
        with pytest.raises(L.PoroError) as ex:
            L.poro_sync(ctx, 0)
        assert ex.value.status == L.PORO_ETIMEOUT
        L.poro_sync(ctx, -1)
        qt = L.poro_get_predictor(ctx, 64 * 3, 1)
        assert rel_l2(qt[0], oracle_predictor(d, 0)) <= TOL
    finally:
        L.poro_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("chunk", [0, 7, 1000])
def test_host_pipeline_matches_step_by_step(L, prec, chunk):
    """poro_predict_host (chunked copies overlapped with the kernels) gives
    bitwise the same I as set_dofs + predict + get_integrated, for automatic,
    ragged (7 elements, last chunk partial) and single-chunk sizes; the full
    predictor it leaves on the device matches too."""
    d = population(33, 4, seed=11)
    qt_ref, i_ref = _run_host(L, d, prec)
    ctx = L.poro_create(0, d["N"], prec)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        i_got = L.poro_predict_host(ctx, d["Q0"], chunk_elems=chunk)
        qt_got = L.poro_get_predictor(ctx, 0, 33)
    finally:
        L.poro_destroy(ctx)
    np.testing.assert_array_equal(i_got, i_ref)
    np.testing.assert_array_equal(qt_got, qt_ref)


@pytest.mark.parametrize("prec", [0, 2])
def test_host_pipeline_ramped_chunks(L, prec):
    """A population large enough for the automatic schedule's ramped first
    and last chunks (20,000 elements at N = 2: chunks 512, 1024, 2048, then
    about 4,096, then 2048, 1024, 512) gives bitwise the step-by-step I."""
    d = population(20000, 2, seed=13)
    qt_ref, i_ref = _run_host(L, d, prec)
    ctx = L.poro_create(0, d["N"], prec)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        i_got = L.poro_predict_host(ctx, d["Q0"])
        qt_got = L.poro_get_predictor(ctx, 0, 20000)
    finally:
        L.poro_destroy(ctx)
    np.testing.assert_array_equal(i_got, i_ref)
    np.testing.assert_array_equal(qt_got, qt_ref)


def test_host_pipeline_errors(L):
    d = population(5, 2, seed=12)
    ctx = L.poro_create(0, d["N"], 0)
    try:
        with pytest.raises(L.PoroError) as ex:
            L.poro_predict_host(ctx, d["Q0"])
        assert ex.value.status == L.PORO_ESTATE
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        with pytest.raises(L.PoroError) as ex:
            L.poro_predict_host(ctx, d["Q0"], chunk_elems=-1)
        assert ex.value.status == L.PORO_EINVAL
    finally:
        L.poro_destroy(ctx)
