"""GPU parity of the binary64 Algorithm-3 predictor on the damped Maxwell
equations (the paper's second system with an upper-triangular source matrix,
Section "Other applications") against the oracle (oracle/maxwell.py with the
shape-generic dense LU and Algorithm 3 of oracle/predictor.py, pinned in
tests/test_oracle_maxwell.py).  Tolerance 1e-12 relative L2 per element."""
from math import factorial

import numpy as np
import pytest

from oracle import maxwell, predictor
from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def _population(n, N, sigma_scale, seed):
    d = inputs.maxwell_isolated_elements(n, N, seed=seed, sigma_scale=sigma_scale)
    d["dt"] = np.array([maxwell.cfl_dt(d["vertices"][i], inputs.maxwell_dict(d["materials"][i]), N)
                        for i in range(n)])
    return d


def _gpu(L, d, N):
    ctx = L.poro_create(0, N, L.PORO_FP64, system=L.PORO_SYSTEM_MAXWELL)
    try:
        assert L.poro_get_system(ctx) == (L.PORO_SYSTEM_MAXWELL, 6)
        L.poro_set_isolated_maxwell(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        n = d["Q0"].shape[0]
        return L.poro_get_predictor(ctx, 0, n), L.poro_get_integrated(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("sigma_scale", [0.0, 1.0, 1e3])
def test_maxwell_predictor_matches_oracle(L, N, sigma_scale):
    n = 9
    d = _population(n, N, sigma_scale, seed=700 + N)
    qt, io = _gpu(L, d, N)
    assert qt.shape == (n, 6, (N + 1) * (N + 2) * (N + 3) // 6, N + 1)
    for i in range(n):
        As, Es = maxwell.element_operators(d["vertices"][i], inputs.maxwell_dict(d["materials"][i]), d["dt"][i])
        fn = predictor.predict_dense if (i < 2 and N <= 5) else predictor.predict_alg3
        ref = fn(N, As, Es, d["Q0"][i])
        assert np.linalg.norm(qt[i] - ref) / np.linalg.norm(ref) <= 1e-12, (i, N, sigma_scale)
        np.testing.assert_allclose(io[i], d["dt"][i] * qt[i][:, :, 0], rtol=0, atol=1e-300)


def _pade_exp(k, m, z):
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("N", [3, 6])
def test_maxwell_stiff_conduction_is_radau_pade(L, N):
    """Mode-0 data: E decays by the (N, N+1) Pade approximant of exp (e down
    to about -1e6), H stays, higher modes stay zero."""
    for scale in (1.0, 1e3, 1e6):
        d = _population(4, N, scale, seed=800 + N)
        q0 = np.zeros_like(d["Q0"])
        q0[:, :, 0] = d["Q0"][:, :, 0]
        d["Q0"] = q0
        qt, _ = _gpu(L, d, N)
        assert np.abs(qt[:, :, 1:, :]).max() == 0.0
        for i in range(4):
            m = inputs.maxwell_dict(d["materials"][i])
            e = -m["sigma"] * d["dt"][i] / m["eps"]
            end = qt[i].sum(axis=2)
            R = _pade_exp(N, N + 1, e)
            sc = np.abs(q0[i, :, 0]).max()
            assert np.abs(end[:3, 0] - R * q0[i, :3, 0]).max() <= 1e-12 * sc, (scale, e)
            assert np.abs(end[3:, 0] - q0[i, 3:, 0]).max() <= 1e-13 * sc
