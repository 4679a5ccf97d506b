"""Pins of the sub-cell material statement (oracle/subcell.py; the paper's
Section "Limitations": stiffness matrices become 3-tensors when the material
varies inside an element) against closed forms and independent routes.
CPU only."""
from math import factorial

import numpy as np
import pytest
from scipy.special import roots_legendre

from oracle import basis, geometry, predictor, subcell
from paper_2108_10565_gb300 import inputs
from test_oracle_pins import _interior_points, _phi_collapsed


def _vertex_materials(rng, spread=0.2, inviscid=False):
    mats = []
    for row in inputs.perturbed_materials(rng, 4, spread=spread):
        m = inputs.material_dict(row)
        if inviscid:
            m["nu"] = 0.0
        mats.append(m)
    return mats


def _element(N, seed, spread=0.2, inviscid=False):
    rng = np.random.default_rng(seed)
    d = inputs.isolated_elements(1, N, seed=seed)
    mats = _vertex_materials(rng, spread, inviscid)
    vert = d["vertices"][0]
    dt = min(geometry.cfl_dt(vert, m, N) for m in mats)
    As, Es = subcell.element_operators(vert, mats, dt)
    return vert, mats, dt, As, Es, d["Q0"][0]


@pytest.mark.parametrize("N", [1, 2, 3])
def test_constant_material_is_stp_lineq(N):
    """Four equal vertex materials: only the r = 0 terms remain, and Y and the
    predictor are those of Eq. stp-lineq."""
    rng = np.random.default_rng(N)
    d = inputs.isolated_elements(1, N, seed=N)
    m = _vertex_materials(rng)[0]
    vert = d["vertices"][0]
    dt = geometry.cfl_dt(vert, m, N)
    As, Es = subcell.element_operators(vert, [m] * 4, dt)
    assert np.abs(As[1:]).max() <= 1e-12 * np.abs(As[0]).max()
    A0, E0 = predictor.element_operators(vert, m, dt)
    np.testing.assert_allclose(As[0], A0, rtol=1e-13, atol=1e-13 * np.abs(A0).max())
    Y = subcell.assemble_dense(N, As, Es)
    Y0 = predictor.assemble_dense(N, A0, E0)
    assert np.abs(Y - Y0).max() <= 1e-13 * np.abs(Y0).max()
    q = subcell.predict_dense(N, As, Es, d["Q0"][0])
    q0 = predictor.predict_dense(N, A0, E0, d["Q0"][0])
    assert np.linalg.norm(q - q0) / np.linalg.norm(q0) < 1e-12


def test_interpolation_reproduces_vertex_jacobians():
    """sum_r A^{j*}_r phi_r(vertex v) = dt A^j(mat_v) at every reference
    vertex (the linear projection and the vertex order)."""
    vert, mats, dt, As, Es, _ = _element(2, 5)
    for v, x in enumerate(subcell.REF_VERTICES):
        phi = basis.eval_basis(1, *x)
        Av = np.einsum("r,rjpq->jpq", phi, As)
        Ev = np.einsum("r,rpq->pq", phi, Es)
        A0, E0 = predictor.element_operators(vert, mats[v], dt)
        np.testing.assert_allclose(Av, A0, rtol=1e-12, atol=1e-12 * np.abs(A0).max())
        np.testing.assert_allclose(Ev, E0, rtol=1e-12, atol=1e-12 * np.abs(E0).max())


@pytest.mark.parametrize("N", [1, 3])
def test_m3_by_collapsed_quadrature(N):
    """M3_r[k, l] = int phi_k phi_r phi_l against a collapsed Gauss product
    rule with the independent collapsed-coordinate evaluation."""
    M3, _ = subcell.tensors(N)
    triples = basis.mode_triples(N)
    x, w = roots_legendre(N + 3)
    Q = np.zeros((subcell.NR, len(triples), len(triples)))
    for a, wa in zip(x, w):
        for b, wb in zip(x, w):
            for c, wc in zip(x, w):
                xi = (1 + a) * (1 - b) * (1 - c) / 8
                eta = (1 + b) * (1 - c) / 4
                ze = (1 + c) / 2
                wt = wa * wb * wc * (1 - b) * (1 - c) ** 2 / 64
                ph = np.array([_phi_collapsed(i, j, k, xi, eta, ze) for (i, j, k) in triples])
                Q += wt * ph[None, :4, None, None].reshape(4, 1, 1) * np.outer(ph, ph)[None]
    for r in range(subcell.NR):
        np.testing.assert_allclose(M3[r], Q[r], rtol=0, atol=1e-13 * np.abs(Q[r]).max())


@pytest.mark.parametrize("N", [2, 4])
def test_k3_is_the_weighted_derivative(N):
    """M^{-1} K3^j_r c are the modal coefficients of phi_r d_j u, u = sum_l
    c_l phi_l: phi_r d_j u has degree <= N, so the L2 projection is exact.
    Checked pointwise with a 9-point central difference of the independent
    collapsed-coordinate evaluation."""
    rng = np.random.default_rng(N)
    c = rng.standard_normal(basis.n_modes(N))
    _, K3 = subcell.tensors(N)
    Minv = 1.0 / np.diag(basis.mass_matrix(N))
    triples = basis.mode_triples(N)
    wts = np.array([1 / 280, -4 / 105, 1 / 5, -4 / 5, 0.0, 4 / 5, -1 / 5, 4 / 105, -1 / 280])
    h = 0.01

    def u(x):
        return sum(cl * _phi_collapsed(i, j, k, *x) for cl, (i, j, k) in zip(c, triples))

    for x in _interior_points(rng, 2):
        phis = np.array([_phi_collapsed(i, j, k, *x) for (i, j, k) in triples])
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            du = sum(wk * u(x + (k - 4) * e) for k, wk in enumerate(wts)) / h
            for r in range(subcell.NR):
                got = phis @ (Minv * (K3[r][a] @ c))
                assert got == pytest.approx(phis[r] * du, rel=1e-8, abs=1e-8 * np.abs(c).sum())


def _pade_matrix(k, m, L):
    """(k, m) Pade approximant of exp at a matrix argument."""
    n = L.shape[0]
    P = np.zeros_like(L)
    Q = np.zeros_like(L)
    Lp = np.eye(n)
    for j in range(max(k, m) + 1):
        if j <= k:
            P += factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * Lp
        if j <= m:
            Q += factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (
                (-1) ** j * Lp)
        Lp = Lp @ L
    return np.linalg.solve(Q, P)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_linear_data_follow_the_pade_of_the_pointwise_operator(N):
    """Inviscid vertex materials (E = 0), linearly varying Jacobians and
    linear data: q_tau = -sum_j A^{j*}(xi) d_j q maps linear fields to linear
    fields, so the predictor keeps the degree-1 modes, the higher ones stay 0,
    and DG in time (Radau IIA) gives the end value R_{N,N+1}(L) c, L the
    52 x 52 operator of the PDE on {phi_0..phi_3} written out pointwise:
    coefficient s of -sum_j (sum_s A^{j*}_s phi_s)(sum_r c_r d_j phi_r)."""
    vert, mats, dt, As, Es, q0 = _element(N, 20 + N, spread=0.2, inviscid=True)
    assert np.abs(Es).max() == 0.0
    q0 = q0.copy()
    q0[:, subcell.NR:] = 0.0
    # d_j phi_r: constants (the linear modes' monomial coefficients)
    dphi = np.zeros((3, subcell.NR))
    for r, t in enumerate(basis.mode_triples(1)):
        for e, cf in basis.dubiner_poly(*t).items():
            if sum(e) == 1:
                dphi[e.index(1), r] = cf
    L = np.zeros((4 * 13, 4 * 13))
    for s in range(subcell.NR):
        for r in range(subcell.NR):
            L[s * 13:(s + 1) * 13, r * 13:(r + 1) * 13] = -sum(As[s, j] * dphi[j, r] for j in range(3))
    c = q0[:, :subcell.NR].T.reshape(-1)  # index r * 13 + p
    end = _pade_matrix(N, N + 1, L) @ c
    Qt = subcell.predict_dense(N, As, Es, q0)
    got = Qt[:, :subcell.NR, :].sum(axis=2).T.reshape(-1)  # chi_s(1) = 1
    np.testing.assert_allclose(got, end, rtol=0, atol=1e-11 * np.abs(end).max())
    if Qt.shape[1] > subcell.NR:
        assert np.abs(Qt[:, subcell.NR:, :]).max() <= 1e-11 * np.abs(Qt).max()


@pytest.mark.parametrize("N", [1, 2])
def test_varying_source_follows_the_pade_of_its_galerkin_operator(N):
    """No flux (A* = 0) and a linearly varying source matrix: the predictor is
    DG in time for Q' = G Q with G the Galerkin operator of E*(xi),
    G[(p,k),(q,l)] = M_kk^{-1} int phi_k E*_pq(xi) phi_l, so its end value is
    R_{N,N+1}(G) Q0.  G is built here by a collapsed Gauss rule with E*(xi)
    interpolated from the vertices by barycentric coordinates and the
    independent collapsed-coordinate basis evaluation."""
    vert, mats, dt, As, Es, q0 = _element(N, 40 + N, spread=0.3)
    Ev = np.stack([dt * predictor.material.source_matrix(m) for m in mats])
    triples = basis.mode_triples(N)
    B = len(triples)
    Mdiag = np.diag(basis.mass_matrix(N))
    x, w = roots_legendre(N + 3)
    G = np.zeros((13, B, 13, B))
    for a, wa in zip(x, w):
        for b, wb in zip(x, w):
            for c, wc in zip(x, w):
                xi = (1 + a) * (1 - b) * (1 - c) / 8
                eta = (1 + b) * (1 - c) / 4
                ze = (1 + c) / 2
                wt = wa * wb * wc * (1 - b) * (1 - c) ** 2 / 64
                lam = np.array([1 - xi - eta - ze, xi, eta, ze])
                Ex = np.einsum("v,vpq->pq", lam, Ev)
                ph = np.array([_phi_collapsed(i, j, k, xi, eta, ze) for (i, j, k) in triples])
                G += wt * np.einsum("pq,k,l->pkql", Ex, ph, ph)
    G = (G / Mdiag[None, :, None, None]).reshape(13 * B, 13 * B)
    end = _pade_matrix(N, N + 1, G) @ q0.reshape(-1)
    Qt = subcell.predict_dense(N, np.zeros_like(As), Es, q0)
    got = Qt.sum(axis=2).reshape(-1)
    np.testing.assert_allclose(got, end, rtol=0, atol=1e-11 * np.abs(end).max())
