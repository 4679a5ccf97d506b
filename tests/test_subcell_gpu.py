"""GPU parity of the sub-cell material predictor (Section "Limitations":
linearly varying Jacobians and source matrix inside an element, 3-tensor
stiffness) against the oracle's dense solve of the same system
(oracle/subcell.py, pinned in tests/test_oracle_subcell.py).  The kernel
iterates Q <- Y_0^{-1}(b - (Y - Y_0) Q) with Algorithm 3 on the mean
material; stopped at a relative change of 1e-14 it must match the dense
solve within 1e-12 relative L2 per element."""
import numpy as np
import pytest

from oracle import geometry, predictor, subcell
from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def _population(n, N, spread, seed, visc=1.0):
    d = inputs.subcell_isolated_elements(n, N, seed=seed, spread=spread)
    d["materials"] = d["materials"].copy()
    d["materials"][:, :, 9] *= visc
    d["dt"] = np.array([min(geometry.cfl_dt(d["vertices"][i], inputs.material_dict(m), N)
                            for m in d["materials"][i]) for i in range(n)])
    return d


def _oracle(d, i, N):
    mats = [inputs.material_dict(m) for m in d["materials"][i]]
    As, Es = subcell.element_operators(d["vertices"][i], mats, d["dt"][i])
    return subcell.predict_dense(N, As, Es, d["Q0"][i])


def _gpu(L, d, N, tol=1e-14, max_iter=200):
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated_subcell(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_subcell_tolerance(ctx, tol, max_iter)
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        n = d["Q0"].shape[0]
        qt, io = L.poro_get_predictor(ctx, 0, n), L.poro_get_integrated(ctx, 0, n)
        return qt, io, L.poro_get_subcell_iterations(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("spread", [0.05, 0.3])
def test_subcell_predictor_matches_dense_oracle(L, N, spread):
    n = 6 if N <= 3 else 2
    d = _population(n, N, spread, seed=1100 + N)
    qt, io, iters = _gpu(L, d, N)
    assert np.all(iters > 0), iters
    for i in range(n):
        ref = _oracle(d, i, N)
        err = np.linalg.norm(qt[i] - ref) / np.linalg.norm(ref)
        assert err <= 1e-12, (i, N, spread, err, iters[i])
        np.testing.assert_allclose(io[i], d["dt"][i] * qt[i][:, :, 0], rtol=0, atol=1e-300)
    print(f"N={N} spread={spread}: iterations {iters.tolist()}")


def test_subcell_stiff_and_n6(L):
    """10x and 100x viscosity (stiffer source, e ~ -1e3 .. -1e4) and N = 6
    (the dense oracle on one element, 7,644 unknowns)."""
    for visc, N in ((10.0, 3), (100.0, 3), (1.0, 6)):
        d = _population(1, N, 0.2, seed=1200 + N, visc=visc)
        qt, _, iters = _gpu(L, d, N)
        ref = _oracle(d, 0, N)
        err = np.linalg.norm(qt[0] - ref) / np.linalg.norm(ref)
        assert iters[0] > 0 and err <= 1e-12, (visc, N, err, iters)


def test_equal_vertex_materials_give_the_constant_material_predictor(L):
    """Four equal vertex materials: the variation terms vanish (to rounding)
    and the iteration stops after one step at the constant-material
    predictor of the FP64 kernel."""
    N = 4
    d = _population(8, N, 0.0, seed=1300)
    d["materials"][:] = d["materials"][:, :1, :]
    qt, _, iters = _gpu(L, d, N)
    assert np.all(iters == 1), iters
    ctx = L.poro_create(0, N, L.PORO_FP64)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"][:, 0, :], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        ref = L.poro_get_predictor(ctx, 0, 8)
    finally:
        L.poro_destroy(ctx)
    for i in range(8):
        assert np.linalg.norm(qt[i] - ref[i]) / np.linalg.norm(ref[i]) <= 1e-14


def test_subcell_iteration_limit_and_errors(L):
    d = _population(3, 2, 0.3, seed=1400)
    _, _, iters = _gpu(L, d, 2, tol=0.0, max_iter=3)
    assert np.all(iters == -3), iters  # tol 0 is never met: stopped at the limit
    ctx = L.poro_create(0, 2, L.PORO_FP64)
    try:
        with pytest.raises(L.PoroError) as ex:
            L.poro_get_subcell_iterations(ctx, 0, 1)
        assert ex.value.status == L.PORO_ESTATE
        bad = d["materials"].copy()
        bad[1, 2, 5] = 1.5  # porosity outside (0, 1) at one vertex
        with pytest.raises(L.PoroError) as ex:
            L.poro_set_isolated_subcell(ctx, d["vertices"], bad, d["dt"])
        assert ex.value.status == L.PORO_EINVAL
        L.poro_set_isolated_subcell(ctx, d["vertices"], d["materials"], d["dt"])
        with pytest.raises(L.PoroError) as ex:
            L.poro_lu_factor(ctx, 0, 1)
        assert ex.value.status == L.PORO_EUNSUPPORTED
        with pytest.raises(L.PoroError):
            L.poro_set_subcell_tolerance(ctx, -1.0, 10)
    finally:
        L.poro_destroy(ctx)
    ctx = L.poro_create(0, 2, L.PORO_FP32_REFINE)
    try:
        with pytest.raises(L.PoroError) as ex:
            L.poro_set_isolated_subcell(ctx, d["vertices"], d["materials"], d["dt"])
        assert ex.value.status == L.PORO_EUNSUPPORTED
    finally:
        L.poro_destroy(ctx)
