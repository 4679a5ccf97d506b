"""GPU parity of the binary64 Algorithm-3 predictor on viscoelastic
attenuation (3 relaxation mechanisms, 27 quantities; a system with an
upper-triangular source matrix named in the paper's Section "Other
applications") against the oracle (oracle/viscoelastic.py with the
shape-generic dense LU and Algorithm 3 of oracle/predictor.py, pinned in
tests/test_oracle_viscoelastic.py).  Tolerance 1e-12 relative L2 per
element."""
from math import factorial

import numpy as np
import pytest

from oracle import predictor, viscoelastic as ve
from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def _population(n, N, omega_scale, seed):
    d = inputs.viscoelastic_isolated_elements(n, N, seed=seed, omega_scale=omega_scale)
    d["dt"] = np.array([ve.cfl_dt(d["vertices"][i], inputs.viscoelastic_dict(d["materials"][i]), N)
                        for i in range(n)])
    return d


def _gpu(L, d, N):
    ctx = L.poro_create(0, N, L.PORO_FP64, system=L.PORO_SYSTEM_VISCOELASTIC)
    try:
        assert L.poro_get_system(ctx) == (L.PORO_SYSTEM_VISCOELASTIC, 27)
        L.poro_set_isolated_viscoelastic(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        n = d["Q0"].shape[0]
        return L.poro_get_predictor(ctx, 0, n), L.poro_get_integrated(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("omega_scale", [1.0, 1e3, 1e6])
def test_viscoelastic_predictor_matches_oracle(L, N, omega_scale):
    """omega_l dt from ~1e-4 (seismic band) to ~1e4 (stiff relaxation)."""
    n = 9
    d = _population(n, N, omega_scale, seed=900 + N)
    qt, io = _gpu(L, d, N)
    assert qt.shape == (n, 27, (N + 1) * (N + 2) * (N + 3) // 6, N + 1)
    for i in range(n):
        As, Es = ve.element_operators(d["vertices"][i], inputs.viscoelastic_dict(d["materials"][i]), d["dt"][i])
        fn = predictor.predict_dense if (i < 2 and N <= 3) else predictor.predict_alg3
        ref = fn(N, As, Es, d["Q0"][i])
        assert np.linalg.norm(qt[i] - ref) / np.linalg.norm(ref) <= 1e-12, (i, N, omega_scale)
        np.testing.assert_allclose(io[i], d["dt"][i] * qt[i][:, :, 0], rtol=0, atol=1e-300)


def _pade_exp(k, m, z):
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("N", [3, 6])
def test_viscoelastic_relaxation_is_radau_pade(L, N):
    """Mode-0 data: each anelastic function decays by the (N, N+1) Pade
    approximant R(e_l) of exp (e_l down to about -1e4), the stresses move by
    the couplings times (R(e_l) - 1) / e_l, the velocities stay, higher modes
    stay zero."""
    for scale in (1.0, 1e3, 1e6):
        d = _population(4, N, scale, seed=950 + N)
        q0 = np.zeros_like(d["Q0"])
        q0[:, :, 0] = d["Q0"][:, :, 0]
        d["Q0"] = q0
        qt, _ = _gpu(L, d, N)
        assert np.abs(qt[:, :, 1:, :]).max() == 0.0
        for i in range(4):
            m = inputs.viscoelastic_dict(d["materials"][i])
            Es = d["dt"][i] * ve.source_matrix(m)
            expect = q0[i, :, 0].copy()
            for l in range(ve.NMECH):
                e = -m["omega"][l] * d["dt"][i]
                R = _pade_exp(N, N + 1, e)
                for k in range(6):
                    expect[ve.th(l, k)] = R * q0[i, ve.th(l, k), 0]
                    for s in range(6):
                        expect[s] += Es[s, ve.th(l, k)] * (R - 1) / e * q0[i, ve.th(l, k), 0]
            end = qt[i].sum(axis=2)[:, 0]
            sc = np.abs(expect).max()
            assert np.abs(end - expect).max() <= 1e-12 * sc, (scale, N)


def test_viscoelastic_rejects_bad_input(L):
    d = _population(2, 2, 1.0, seed=3)
    ctx = L.poro_create(0, 2, L.PORO_FP64, system=L.PORO_SYSTEM_VISCOELASTIC)
    try:
        bad = d["materials"].copy()
        bad[1, 2] = -1.0  # mu_u <= 0
        with pytest.raises(L.PoroError):
            L.poro_set_isolated_viscoelastic(ctx, d["vertices"], bad, d["dt"])
        with pytest.raises(L.PoroError):
            L.poro_set_isolated(ctx, d["vertices"], np.tile(inputs.REFERENCE_MATERIAL, (2, 1)), d["dt"])
    finally:
        L.poro_destroy(ctx)
    with pytest.raises(L.PoroError):
        L.poro_create(0, 2, L.PORO_FP32_REFINE, system=L.PORO_SYSTEM_VISCOELASTIC)
