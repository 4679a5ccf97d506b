"""Pins of the viscoelastic statement (oracle/viscoelastic.py; a system with
an upper-triangular source matrix named in the paper's Section "Other
applications") against closed forms, and of the shape-generic predictor
functions on that 27-quantity system.  CPU only."""
from math import factorial

import numpy as np
import pytest
from scipy.special import eval_jacobi, roots_legendre

from oracle import basis, predictor, viscoelastic as ve
from paper_2108_10565_gb300 import inputs


def _elements(n, N, omega_scale=1.0, seed=3):
    d = inputs.viscoelastic_isolated_elements(n, N, seed=seed, omega_scale=omega_scale)
    out = []
    for i in range(n):
        m = inputs.viscoelastic_dict(d["materials"][i])
        dt = ve.cfl_dt(d["vertices"][i], m, N)
        As, Es = ve.element_operators(d["vertices"][i], m, dt)
        out.append((As, Es, d["Q0"][i], m, dt))
    return out


def _material(seed=0):
    return inputs.viscoelastic_dict(inputs.viscoelastic_isolated_elements(1, 1, seed=seed)["materials"][0])


def test_characteristic_speeds():
    """n . (A, B, C) has eigenvalues +-c_P, +-c_S (twice each) and 0 (21
    times: the anelastic functions and three stresses carry no flux) for
    every unit direction n, with the unrelaxed speeds."""
    rng = np.random.default_rng(0)
    m = _material()
    A = ve.jacobians(m)
    cp, cs = ve.speeds(m)
    for _ in range(5):
        nv = rng.standard_normal(3)
        nv /= np.linalg.norm(nv)
        ev = np.sort(np.linalg.eigvals(sum(nv[d] * A[d] for d in range(3))).real)
        np.testing.assert_allclose(ev, [-cp, -cs, -cs] + [0.0] * 21 + [cs, cs, cp], atol=1e-9 * cp)


def _dispersion_roots(m, kk, modulus, coef):
    """Roots w of rho w^2 = kk (M_u - sum_l Y_l omega_l / (omega_l - i w)),
    multiplied through by prod_l (omega_l - i w): a polynomial of degree
    2 + n in w."""
    P = np.polynomial.Polynomial
    om = np.asarray(m["omega"])
    fac = [P([o, -1j]) for o in om]
    prod = P([1.0 + 0j])
    for f in fac:
        prod = prod * f
    rest = P([0j])
    for l in range(len(om)):
        t = P([coef[l] * om[l] + 0j])
        for n_ in range(len(om)):
            if n_ != l:
                t = t * fac[n_]
        rest = rest + t
    return (P([0, 0, m["rho"]]) * prod - kk * (modulus * prod - rest)).roots()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dispersion_relation_complex_moduli(seed):
    """Plane waves exp(i(k.x - w t)): the 27 eigenvalues w of k.A + iE are the
    5 roots of rho w^2 = |k|^2 (lam(w) + 2 mu(w)) (P), the 5 roots of
    rho w^2 = |k|^2 mu(w) twice (two S polarisations), 0 three times and
    each -i omega_l three times (anelastic functions the wave does not
    drive), with the complex moduli of the generalised Maxwell body in
    closed form.  The wavenumber puts |k| c_P inside the relaxation band."""
    from scipy.optimize import linear_sum_assignment

    m = _material(seed)
    A = ve.jacobians(m)
    cp, _ = ve.speeds(m)
    rng = np.random.default_rng(seed)
    nv = rng.standard_normal(3)
    k = 3.0 * nv / np.linalg.norm(nv) / cp
    kk = k @ k
    w = np.linalg.eigvals(sum(k[d] * A[d] for d in range(3)) + 1j * ve.source_matrix(m))
    rp = _dispersion_roots(m, kk, m["lam"] + 2 * m["mu"], m["Ylam"] + 2 * m["Ymu"])
    rs = _dispersion_roots(m, kk, m["mu"], m["Ymu"])
    expect = np.concatenate([rp, rs, rs, np.zeros(3), np.repeat(-1j * np.asarray(m["omega"]), 3)])
    cost = np.abs(w[:, None] - expect[None, :])
    i, j = linear_sum_assignment(cost)
    assert cost[i, j].max() < 1e-8 * max(m["omega"]), np.sort(cost[i, j])[-5:]
    # the propagating pairs are there: two P roots with |Re w| ~ |k| c_P
    assert np.sum(np.abs(np.abs(rp.real) - np.sqrt(kk) * cp) < 0.1 * np.sqrt(kk) * cp) == 2


def test_source_matrix_structure():
    m = _material()
    E = ve.source_matrix(m)
    assert np.array_equal(E, np.triu(E))
    np.testing.assert_allclose(np.diag(E), [0.0] * 9 + list(np.repeat(-np.asarray(m["omega"]), 6)))
    # per mechanism 9 normal-block and 3 shear couplings into the stresses
    assert np.count_nonzero(E[:6]) == 3 * 12 and np.count_nonzero(E[6:9]) == 0


def test_relaxed_limit():
    """w -> 0: the moduli relax to lam_u - sum Ylam and mu_u - sum Ymu; w -> inf:
    the unrelaxed moduli."""
    m = _material()
    lam0, mu0 = ve.complex_moduli(m, 0.0)
    assert lam0 == pytest.approx(m["lam"] - m["Ylam"].sum(), rel=1e-14)
    assert mu0 == pytest.approx(m["mu"] - m["Ymu"].sum(), rel=1e-14)
    laminf, muinf = ve.complex_moduli(m, 1e12)
    assert laminf.real == pytest.approx(m["lam"], rel=1e-9) and muinf.real == pytest.approx(m["mu"], rel=1e-9)


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("omega_scale", [1.0, 30.0, 3e3])
def test_block_algorithms_equal_dense_viscoelastic(N, omega_scale):
    """Algorithms 1-3 reach the dense LU solution for the 27-quantity system
    (omega_l dt from ~1e-3 up to ~1e3 here)."""
    for As, Es, q0, _, _ in _elements(2, N, omega_scale):
        ref = predictor.predict_dense(N, As, Es, q0)
        for alg in (predictor.predict_alg1, predictor.predict_alg2, predictor.predict_alg3):
            assert np.linalg.norm(alg(N, As, Es, q0) - ref) / np.linalg.norm(ref) < 1e-12


def _pade_exp(k, m, z):
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("N", [1, 3, 5])
@pytest.mark.parametrize("omega_scale", [1.0, 1e3, 1e6])
def test_relaxation_is_radau_pade(N, omega_scale):
    """Mode-0 data: th_l decays by the (N, N+1) Pade approximant R(e_l) of exp
    over the step (e_l = -omega_l dt; DG in time = Radau IIA), the stresses
    move by sum_l g (R(e_l) - 1) / e_l th_l0 through each coupling g = E*[s, th],
    and the velocities stay."""
    As, Es, _, _, _ = _elements(1, N, omega_scale)[0]
    B = basis.n_modes(N)
    q0 = np.zeros((ve.NQ, B))
    q0[:, 0] = np.linspace(1.0, 2.0, ve.NQ)
    Qt = predictor.predict_alg3(N, As, Es, q0)
    end = Qt.sum(axis=2)
    expect = q0[:, 0].copy()
    for l in range(ve.NMECH):
        e = Es[ve.th(l, 0), ve.th(l, 0)]
        R = _pade_exp(N, N + 1, e)
        for k in range(6):
            expect[ve.th(l, k)] = R * q0[ve.th(l, k), 0]
            for s in range(6):
                expect[s] += Es[s, ve.th(l, k)] * (R - 1) / e * q0[ve.th(l, k), 0]
    np.testing.assert_allclose(end[:, 0], expect, rtol=1e-12, atol=1e-14)
    assert np.abs(Qt[:, 1:, :]).max() == 0.0


@pytest.mark.parametrize("N", [1, 2, 3])
def test_elastic_predictor_ignores_anelastic_data_without_coupling(N):
    """Ylam = Ymu = 0: the anelastic functions feed nothing back, so the
    stress and velocity predictor does not depend on their initial data."""
    As, _, q0, m, dt = _elements(1, N)[0]
    m = dict(m, Ylam=np.zeros(3), Ymu=np.zeros(3))
    Es = dt * ve.source_matrix(m)
    a = predictor.predict_alg3(N, As, Es, q0)
    q1 = q0.copy()
    q1[9:] = 0.0
    b = predictor.predict_alg3(N, As, Es, q1)
    np.testing.assert_array_equal(a[:9], b[:9])
    assert np.abs(a[9:] - b[9:]).max() > 0.0


@pytest.mark.parametrize("N", [1, 2, 3])
def test_lossless_predictor_is_ck_taylor_viscoelastic(N):
    """omega = 0 and no coupling (E = 0): the predictor equals the
    Cauchy-Kovalewski Taylor polynomial of the element-local solution,
    projected on the time basis (elastic waves)."""
    As0, _, q0, m, dt = _elements(1, N, seed=5)[0]
    d = inputs.viscoelastic_isolated_elements(1, N, seed=5)
    m = dict(m, omega=np.zeros(3), Ylam=np.zeros(3), Ymu=np.zeros(3))
    As, Es = ve.element_operators(d["vertices"][0], m, dt)
    assert np.count_nonzero(Es) == 0
    Kh = basis.khat_matrices(N)

    def D(Q):
        return -sum(As[j] @ Q @ Kh[j].T for j in range(3))

    terms = [q0]
    for k in range(1, N + 1):
        terms.append(D(terms[-1]) / k)
    x, w = roots_legendre(N + 2)
    tau, wt = (x + 1) / 2, w / 2
    Qt = np.zeros((ve.NQ, basis.n_modes(N), N + 1))
    for tq, wq in zip(tau, wt):
        Qtau = sum(t * tq ** k for k, t in enumerate(terms))
        for s in range(N + 1):
            Qt[:, :, s] += (2 * s + 1) * wq * Qtau * eval_jacobi(s, 0, 0, 2 * tq - 1)
    got = predictor.predict_dense(N, As, Es, q0)
    assert np.linalg.norm(got - Qt) / np.linalg.norm(Qt) < 1e-12
