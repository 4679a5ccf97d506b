"""Pins of the damped Maxwell statement (oracle/maxwell.py; the paper's
second system with an upper-triangular source matrix, Section "Other
applications") against closed forms, and of the shape-generic predictor
functions on that 6-quantity system.  CPU only."""
from math import factorial

import numpy as np
import pytest
from scipy.special import eval_jacobi, roots_legendre

from oracle import basis, maxwell, predictor
from paper_2108_10565_gb300 import inputs


def _elements(n, N, sigma_scale, seed=3):
    d = inputs.maxwell_isolated_elements(n, N, seed=seed, sigma_scale=sigma_scale)
    out = []
    for i in range(n):
        m = inputs.maxwell_dict(d["materials"][i])
        dt = maxwell.cfl_dt(d["vertices"][i], m, N)
        As, Es = maxwell.element_operators(d["vertices"][i], m, dt)
        out.append((As, Es, d["Q0"][i], m, dt))
    return out


def test_characteristic_speeds():
    """n . (A, B, C) has eigenvalues +-1/sqrt(eps mu) (twice each) and 0
    (twice) for every unit direction n."""
    rng = np.random.default_rng(0)
    m = {"eps": 2.5, "mu": 1.3, "sigma": 0.7}
    A = maxwell.jacobians(m)
    c = 1 / np.sqrt(m["eps"] * m["mu"])
    for _ in range(5):
        nv = rng.standard_normal(3)
        nv /= np.linalg.norm(nv)
        ev = np.sort(np.linalg.eigvals(sum(nv[d] * A[d] for d in range(3))).real)
        np.testing.assert_allclose(ev, [-c, -c, 0, 0, c, c], atol=1e-14)


def test_damped_dispersion_relation():
    """Plane waves exp(i(k.x - w t)): four eigenvalues w of k.A + iE (the
    transverse waves) solve eps mu w^2 + i sigma mu w = |k|^2, the damped
    wave equation's dispersion relation; the two longitudinal modes are the
    static magnetic field (w = 0) and the relaxing charge (w = -i sigma/eps)."""
    m = {"eps": 1.7, "mu": 1.2, "sigma": 0.9}
    A = maxwell.jacobians(m)
    k = np.array([0.3, -1.1, 0.7])
    w = np.linalg.eigvals(sum(k[d] * A[d] for d in range(3)) + 1j * maxwell.source_matrix(m))
    res = np.abs(m["eps"] * m["mu"] * w ** 2 + 1j * m["sigma"] * m["mu"] * w - k @ k)
    trans = res < 1e-12
    assert trans.sum() == 4
    rest = np.sort_complex(w[~trans])
    np.testing.assert_allclose(rest, [-1j * m["sigma"] / m["eps"], 0.0], atol=1e-12)


def test_source_matrix_structure():
    E = maxwell.source_matrix({"eps": 2.0, "mu": 1.0, "sigma": 3.0})
    assert np.array_equal(E, np.triu(E)) and np.count_nonzero(E) == 3
    np.testing.assert_allclose(np.diag(E), [-1.5] * 3 + [0] * 3)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("sigma_scale", [0.0, 1e-2, 1.0])
def test_block_algorithms_equal_dense_maxwell(N, sigma_scale):
    """Algorithms 1-3 reach the dense LU solution for the 6-quantity system
    (e = -sigma dt / eps from 0 down to ~-5 here)."""
    for As, Es, q0, _, _ in _elements(2, N, sigma_scale):
        ref = predictor.predict_dense(N, As, Es, q0)
        for alg in (predictor.predict_alg1, predictor.predict_alg2, predictor.predict_alg3):
            assert np.linalg.norm(alg(N, As, Es, q0) - ref) / np.linalg.norm(ref) < 1e-13


def _pade_exp(k, m, z):
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("N", [1, 3, 6])
@pytest.mark.parametrize("sigma_scale", [1.0, 1e3, 1e6])
def test_stiff_conduction_is_radau_pade(N, sigma_scale):
    """Mode-0 data: E decays by the (N, N+1) Pade approximant R(e) of exp over
    the step (DG in time = Radau IIA), e = -sigma dt / eps; H stays."""
    As, Es, _, _, _ = _elements(1, N, sigma_scale)[0]
    B = basis.n_modes(N)
    q0 = np.zeros((6, B))
    q0[:, 0] = np.arange(1.0, 7.0)
    Qt = predictor.predict_alg3(N, As, Es, q0)
    end = Qt.sum(axis=2)
    e = Es[0, 0]
    R = _pade_exp(N, N + 1, e)
    np.testing.assert_allclose(end[:3, 0], R * q0[:3, 0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(end[3:, 0], q0[3:, 0], rtol=1e-14)
    assert np.abs(Qt[:, 1:, :]).max() == 0.0


@pytest.mark.parametrize("N", [1, 2, 3])
def test_lossless_predictor_is_ck_taylor_maxwell(N):
    """sigma = 0: the predictor equals the Cauchy-Kovalewski Taylor
    polynomial of the element-local solution, projected on the time basis."""
    As, Es, q0, _, _ = _elements(1, N, 0.0, seed=5)[0]
    assert np.count_nonzero(Es) == 0
    Kh = basis.khat_matrices(N)

    def D(Q):
        return -sum(As[j] @ Q @ Kh[j].T for j in range(3))

    terms = [q0]
    for k in range(1, N + 1):
        terms.append(D(terms[-1]) / k)
    x, w = roots_legendre(N + 2)
    tau, wt = (x + 1) / 2, w / 2
    Qt = np.zeros((6, basis.n_modes(N), N + 1))
    for tq, wq in zip(tau, wt):
        Qtau = sum(t * tq ** k for k, t in enumerate(terms))
        for s in range(N + 1):
            Qt[:, :, s] += (2 * s + 1) * wq * Qtau * eval_jacobi(s, 0, 0, 2 * tq - 1)
    got = predictor.predict_dense(N, As, Es, q0)
    assert np.linalg.norm(got - Qt) / np.linalg.norm(Qt) < 1e-12
