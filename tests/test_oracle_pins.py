"""Pins of the oracle against facts the paper and the mathematics fix.

Every test here checks the oracle against something other than itself:
values printed in the paper (tests/golden), closed forms, textbook
identities, or an independent evaluation route.  CPU only.
"""
import os
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest
from scipy.special import eval_jacobi, roots_legendre

from oracle import basis, flops, geometry, material, predictor, timebasis
from paper_2108_10565_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- P5: Table flop-count
def test_flop_table_exact():
    for row in _golden("flop_count.txt"):
        N = int(row[0])
        assert flops.unknowns(N) == int(row[1])
        assert flops.lu_flops(N) == int(row[2])
        assert flops.stp_flops_bound(N) == int(row[3])
        assert flops.lu_storage_mib(N) == pytest.approx(float(row[4]), rel=1e-15)
        assert flops.stp_storage_mib(N) == pytest.approx(float(row[5]), rel=1e-15)


def test_unknowns_match_basis():
    for N in range(2, 7):
        assert flops.unknowns(N) == 13 * basis.n_modes(N) * (N + 1)


# ---------------------------------------------------------------- P6: wave speeds
def _table_material(row):
    K_S, rho_S, lam, mu, phi, kappa, T, K_F, rho_F, nu = map(float, row[:10])
    return dict(K_S=K_S, rho_S=rho_S, lambda_M=lam, mu_M=mu, kappa=kappa, phi=phi, T=T,
                K_F=K_F, rho_F=rho_F, nu=nu)


def test_fast_p_speed_two_halfspaces():
    """Fast P speeds printed for Table material_heterogeneous."""
    for row in _golden("wave_speeds_two_halfspaces.txt"):
        mat = _table_material(row)
        assert geometry.max_wave_speed(mat) == pytest.approx(float(row[10]), abs=1e-6)


def _biot_speeds_closed_form(mat):
    """Textbook inviscid Biot speeds: c_S^2 = mu / (rho - rho_F^2 / m), and the
    two P speeds are the roots of
    det [[H - rho c^2, C - rho_F c^2], [C - rho_F c^2, M - m c^2]] = 0,
    H = K_M + 4/3 mu + alpha^2 M, C = alpha M (Biot's dispersion relation)."""
    K_S, K_F, phi = mat["K_S"], mat["K_F"], mat["phi"]
    lam, mu = mat["lambda_M"], mat["mu_M"]
    rho = phi * mat["rho_F"] + (1 - phi) * mat["rho_S"]
    rf = mat["rho_F"]
    m = rf * mat["T"] / phi
    K_M = lam + 2 * mu / 3
    alpha = 1 - K_M / K_S
    M = K_S / ((1 - K_M / K_S) - phi * (1 - K_S / K_F))
    H = K_M + 4 * mu / 3 + alpha ** 2 * M
    C = alpha * M
    # (H - rho x)(M - m x) - (C - rf x)^2 = 0, x = c^2
    a = rho * m - rf ** 2
    b = -(H * m + rho * M - 2 * C * rf)
    c = H * M - C ** 2
    x = np.roots([a, b, c])
    return np.sqrt(mu / (rho - rf ** 2 / m)), np.sqrt(np.sort(x.real))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_wave_speeds_closed_form(seed):
    rng = np.random.default_rng(seed)
    mat = inputs.material_dict(inputs.perturbed_materials(rng, 1)[0])
    mat["nu"] = 0.0
    cs, (cp2, cp1) = _biot_speeds_closed_form(mat)
    for n in ([1, 0, 0], [0, 1, 0], [0, 0, 1], np.array([1, 2, -2]) / 3.0):
        sp = material.wave_speeds(mat, n)
        # 13 eigenvalues: +-cp1, +-cs (x2), +-cp2, 5 zeros
        assert sp[0] == pytest.approx(cp1, rel=1e-12)
        assert sp[2] == pytest.approx(cs, rel=1e-12)
        assert sp[4] == pytest.approx(cs, rel=1e-12)
        assert sp[6] == pytest.approx(cp2, rel=1e-12)
        assert np.all(sp[8:] < 1e-6 * cp1)


def test_source_matrix_structure_and_momentum():
    """E upper triangular, 6 non-zeros, G (strict upper part) 3 non-zeros
    (Section "Structure of the system matrix"); the Darcy friction exchanges
    momentum between solid and fluid only: rho E[u,:] + rho_F E[uf,:] = 0."""
    mat = inputs.material_dict(inputs.REFERENCE_MATERIAL)
    E = material.source_matrix(mat)
    assert np.count_nonzero(E) == 6
    assert np.count_nonzero(np.tril(E, -1)) == 0
    assert np.count_nonzero(np.triu(E, 1)) == 3
    d = material.derived(mat)
    for v_, f_ in ((material.U, material.UF), (material.V, material.VF), (material.W, material.WF)):
        assert d["rho"] * E[v_, f_] + mat["rho_F"] * E[f_, f_] == pytest.approx(0.0, abs=1e-9 * abs(E[f_, f_]))
    # relative velocity decays at rate b rho / D (closed form of the Darcy term)
    assert -E[material.UF, material.UF] == pytest.approx(d["b"] * d["rho"] / d["D"], rel=1e-15)


def test_jacobian_sparsity():
    """Union pattern of the Jacobians: 18 non-zeros each, 54 for A+B+C
    (figure sparsity_jacobians)."""
    mat = inputs.material_dict(inputs.REFERENCE_MATERIAL)
    A, B, C = material.jacobians(mat)
    assert [np.count_nonzero(J) for J in (A, B, C)] == [18, 18, 18]
    assert np.count_nonzero(np.abs(A) + np.abs(B) + np.abs(C)) == 54


# ---------------------------------------------------------------- P2: spatial basis
def _collapsed(xi, eta, zeta):
    L = 1.0 - eta - zeta
    return 2.0 * xi / L - 1.0, 2.0 * eta / (1.0 - zeta) - 1.0, 2.0 * zeta - 1.0


def _phi_collapsed(i, j, k, xi, eta, zeta):
    """Independent evaluation of phi_ijk through collapsed coordinates and
    scipy's Jacobi polynomials."""
    r, s, t = _collapsed(xi, eta, zeta)
    return (eval_jacobi(i, 0, 0, r) * ((1 - s) / 2) ** i * eval_jacobi(j, 2 * i + 1, 0, s)
            * ((1 - t) / 2) ** (i + j) * eval_jacobi(k, 2 * i + 2 * j + 2, 0, t))


def _interior_points(rng, n):
    p = rng.dirichlet([2.0, 2.0, 2.0, 2.0], n)[:, 1:]
    return p


@pytest.mark.parametrize("N", [1, 3, 6])
def test_basis_matches_collapsed_evaluation(N):
    rng = np.random.default_rng(10 + N)
    for x in _interior_points(rng, 5):
        ref = np.array([_phi_collapsed(i, j, k, *x) for (i, j, k) in basis.mode_triples(N)])
        np.testing.assert_allclose(basis.eval_basis(N, *x), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", range(1, 7))
def test_mass_matrix_closed_form(N):
    """M diagonal (orthogonal basis, Section "Structure of the system
    matrix"), with the Jacobi-weight closed form
    int phi_ijk^2 = 1 / ((2i+1)(2i+2j+2)(2(i+j+k)+3))."""
    assert basis.mass_exact_offdiag_max(N) == 0
    for (i, j, k), m in zip(basis.mode_triples(N), basis.mass_exact_diag(N)):
        assert m == Fraction(1, (2 * i + 1) * (2 * i + 2 * j + 2) * (2 * (i + j + k) + 3))


def test_monomial_integral_formula():
    """int_E xi^a eta^b zeta^c against a collapsed Gauss product rule."""
    x, w = roots_legendre(12)
    for (a, b, c) in [(0, 0, 0), (2, 1, 0), (1, 3, 2), (0, 0, 5)]:
        tot = 0.0
        for r, wr in zip(x, w):
            for s, ws in zip(x, w):
                for t, wt in zip(x, w):
                    xi = (1 + r) * (1 - s) * (1 - t) / 8
                    eta = (1 + s) * (1 - t) / 4
                    ze = (1 + t) / 2
                    tot += wr * ws * wt * (1 - s) * (1 - t) ** 2 / 64 * xi ** a * eta ** b * ze ** c
        assert float(basis.monomial_integral(a, b, c)) == pytest.approx(tot, rel=1e-13)


@pytest.mark.parametrize("N", range(1, 7))
def test_lemma1_zero_blocks(N):
    """Lemma 1: K^alpha_ij = 0 whenever deg(phi_i) >= deg(phi_j)."""
    deg = np.array([i + j + k for (i, j, k) in basis.mode_triples(N)])
    for K in basis.khat_matrices(N) + basis.stiffness_matrices(N):
        mask = deg[:, None] >= deg[None, :]
        assert np.all(K[mask] == 0.0)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_khat_is_the_derivative(N):
    """sum_k phi_k(x) (Khat^alpha c)_k equals d_alpha (sum_l c_l phi_l)(x):
    Khat^alpha = M^{-1} K^alpha is the L2 projection of the derivative, exact
    for polynomials.  The derivative is taken by a 9-point central
    difference of the independent collapsed-coordinate evaluation (exact for
    degree <= 8 up to rounding)."""
    rng = np.random.default_rng(N)
    c = rng.standard_normal(basis.n_modes(N))
    Kh = basis.khat_matrices(N)
    triples = basis.mode_triples(N)
    wts = np.array([1 / 280, -4 / 105, 1 / 5, -4 / 5, 0.0, 4 / 5, -1 / 5, 4 / 105, -1 / 280])
    h = 0.01

    def u(x):
        return sum(cl * _phi_collapsed(i, j, k, *x) for cl, (i, j, k) in zip(c, triples))

    for x in _interior_points(rng, 3):
        phis = np.array([_phi_collapsed(i, j, k, *x) for (i, j, k) in triples])
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = sum(wk * u(x + (k - 4) * e) for k, wk in enumerate(wts)) / h
            got = phis @ (Kh[a] @ c)
            assert got == pytest.approx(fd, rel=1e-8, abs=1e-8 * np.abs(c).sum())


def khat_row_fractions(K, max_den=10**6):
    """Rows of one Khat^alpha as (numerators, common denominator), or None
    where an entry is not a rational with a denominator <= max_den."""
    from math import lcm

    out = []
    for row in K:
        nz = np.nonzero(row)[0]
        fr = [Fraction(float(x)).limit_denominator(max_den) for x in row[nz]]
        if any(abs(float(f) - x) > 1e-14 * abs(x) for f, x in zip(fr, row[nz])):
            return None
        d = 1
        for f in fr:
            d = lcm(d, f.denominator)
        out.append(([int(f * d) for f in fr], d))
    return out


# largest common denominator of a Khat row, N = 1..6
KHAT_MAX_DENOMINATOR = {1: 1, 2: 6, 3: 90, 4: 360, 5: 3150, 6: 103950}


@pytest.mark.parametrize("N", range(1, 7))
def test_khat_rows_are_small_rationals(N):
    """Khat^alpha = M^{-1} K^alpha with the closed-form rational mass matrix
    and polynomial integrals of a basis with rational recurrence
    coefficients, so each row is an integer row over a small common
    denominator (a wrong normalisation factor, e.g. a stray sqrt(2), breaks
    this).  The mixed-precision residual stores Khat in exactly this form:
    numerators below 2^23 (packable with a 7-bit column), and each row's sum
    of |numerators| below 2^22, so that its products with 22-bit fixed-point
    values sum exactly below 2^44 in 64-bit integers."""
    worst_den, worst_num, worst_sum = 1, 0, 0
    for K in basis.khat_matrices(N):
        rows = khat_row_fractions(K)
        assert rows is not None
        for nums, d in rows:
            worst_den = max(worst_den, d)
            worst_num = max([worst_num] + [abs(c) for c in nums])
            worst_sum = max(worst_sum, sum(abs(c) for c in nums))
    assert worst_den == KHAT_MAX_DENOMINATOR[N]
    assert worst_num < 2**23
    assert worst_sum < 2**22


# ---------------------------------------------------------------- time matrices
@pytest.mark.parametrize("N", range(0, 7))
def test_time_matrices_closed_form(N):
    """Shifted Legendre on [0,1]: W_rs = 1, w_r = (-1)^r, S_rs = d_rs/(2r+1),
    K^tau_rs = 2 if r > s and r - s odd (derivative of P_r expands in P_s,
    s = r-1, r-3, ... with weight 2s+1)."""
    W, w, S, Kt = timebasis.time_matrices(N)
    T = N + 1
    np.testing.assert_allclose(W, np.ones((T, T)), atol=1e-15)
    np.testing.assert_allclose(w, [(-1) ** r for r in range(T)], atol=1e-15)
    np.testing.assert_allclose(S, np.diag([1.0 / (2 * r + 1) for r in range(T)]), atol=1e-15)
    Kref = np.array([[2.0 if (r > s and (r - s) % 2 == 1) else 0.0 for s in range(T)] for r in range(T)])
    np.testing.assert_allclose(Kt, Kref, atol=1e-13)


# ---------------------------------------------------------------- P1: algorithms = dense solve
def _element(N, seed, stiff=1.0):
    d = inputs.isolated_elements(1, N, seed=seed)
    mat = inputs.material_dict(d["materials"][0])
    mat["nu"] *= stiff
    v = d["vertices"][0]
    dt = geometry.cfl_dt(v, mat, N)
    As, Es = predictor.element_operators(v, mat, dt)
    return As, Es, d["Q0"][0], dt


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("stiff", [0.0, 1.0, 10.0])
def test_block_algorithms_equal_dense(N, stiff):
    """Algorithms 1, 2, 3 (block back-substitution) reach the dense LU
    solution of Eq. stp-lineq: exact algebra, so agreement to rounding."""
    for seed in (1, 2):
        As, Es, q0, _ = _element(N, seed, stiff)
        ref = predictor.predict_dense(N, As, Es, q0)
        nrm = np.linalg.norm(ref)
        for alg in (predictor.predict_alg1, predictor.predict_alg2, predictor.predict_alg3):
            assert np.linalg.norm(alg(N, As, Es, q0) - ref) / nrm < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_batched_algorithm3_equals_dense(N):
    """The batched Algorithm 3 that the time-stepping oracle (GTS and LTS)
    calls reaches the dense LU solution of Eq. stp-lineq for every element
    of one batch that mixes materials: inviscid, the reference viscosity,
    10x and 100x stiff (e down to ~-2e4).  Every degree block g >= 3 takes the
    green update, so an index slip there fails this pin."""
    from oracle import corrector

    scales = (0.0, 1.0, 10.0, 100.0) if N <= 4 else ((0.0, 100.0) if N == 5 else (100.0,))
    d = inputs.isolated_elements(len(scales), N, seed=40 + N)
    ops = []
    for i, s in enumerate(scales):
        mat = inputs.material_dict(d["materials"][i])
        mat["nu"] *= s
        dt = geometry.cfl_dt(d["vertices"][i], mat, N)
        ops.append(predictor.element_operators(d["vertices"][i], mat, dt))
    As = np.stack([o[0] for o in ops])
    Es = np.stack([o[1] for o in ops])
    Qb = corrector.predict_alg3_batch(N, As, Es, d["Q0"])
    for i in range(len(scales)):
        ref = predictor.predict_dense(N, As[i], Es[i], d["Q0"][i])
        # at N >= 5 the 100x stiff system is the worst conditioned (|Qt| ~
        # 1e7 |r|): dense LU and back-substitution then differ by ~6e-13,
        # both within their rounding bound
        tol = 1e-12 if (N >= 5 and scales[i] >= 100.0) else 1e-13
        assert np.linalg.norm(Qb[i] - ref) / np.linalg.norm(ref) < tol, (N, scales[i])
        # and the batch takes the same steps as the per-element Algorithm 3
        q3 = predictor.predict_alg3(N, As[i], Es[i], d["Q0"][i])
        assert np.linalg.norm(Qb[i] - q3) / np.linalg.norm(q3) < 1e-14
    if N == 6:
        # the fastest Darcy mode of the batch reaches the stiff range
        assert Es[0][material.UF, material.UF] < -1e3


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_c_algorithm3_equals_dense(N):
    """The plain-loop C statement of Algorithm 3 (oracle/alg3_loop.c: the timed
    CPU baseline) reaches the dense LU solution of Eq. stp-lineq for a batch
    mixing inviscid to 100x stiff elements, with 1 and with 3 threads (the
    element loop's schedule changes nothing)."""
    from oracle import alg3_c

    scales = (0.0, 1.0, 10.0, 100.0) if N <= 4 else (1.0, 100.0)
    d = inputs.isolated_elements(len(scales), N, seed=60 + N)
    ops = []
    for i, s in enumerate(scales):
        mat = inputs.material_dict(d["materials"][i])
        mat["nu"] *= s
        dt = geometry.cfl_dt(d["vertices"][i], mat, N)
        ops.append(predictor.element_operators(d["vertices"][i], mat, dt))
    As = np.stack([o[0] for o in ops])
    Es = np.stack([o[1] for o in ops])
    q1 = alg3_c.predict_alg3_c(N, As, Es, d["Q0"], threads=1)
    q3 = alg3_c.predict_alg3_c(N, As, Es, d["Q0"], threads=3)
    assert np.array_equal(q1, q3)
    for i in range(len(scales)):
        ref = predictor.predict_dense(N, As[i], Es[i], d["Q0"][i])
        # the 100x stiff systems are the worst conditioned (|Qt| ~ 1e7 |r|):
        # dense LU and back-substitution differ there by up to a few 1e-13
        tol = 1e-12 if scales[i] >= 100.0 else 1e-13
        assert np.linalg.norm(q1[i] - ref) / np.linalg.norm(ref) < tol, (N, scales[i])


# ---------------------------------------------------------------- P3: stiff source path
def _pade_exp(k, m, z):
    """(k, m) Pade approximant of exp(z) (closed form)."""
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("stiff", [0.1, 1.0, 10.0])
def test_stiff_source_is_radau_pade(N, stiff):
    """Constant-in-space data (mode 0 only): the spatial terms vanish and the
    predictor is DG in time for q' = E* q.  Its end value is the (N, N+1)
    subdiagonal Pade approximant of exp (DG in time = Radau IIA):
    uf(1) = R(e) uf0 and, through the coupling g = E*[u, uf],
    u(1) = u0 + g/e (R(e) - 1) uf0; quantities without source stay constant."""
    As, Es, _, _ = _element(N, 3, stiff)
    B, T = basis.n_modes(N), N + 1
    q0 = np.zeros((13, B))
    q0[:, 0] = np.arange(1.0, 14.0)
    for fn in (predictor.predict_dense, predictor.predict_alg3):
        Qt = fn(N, As, Es, q0)
        end = Qt.sum(axis=2)  # chi_s(1) = 1
        for v_, f_ in ((material.U, material.UF), (material.V, material.VF), (material.W, material.WF)):
            e, g = Es[f_, f_], Es[v_, f_]
            R = _pade_exp(N, N + 1, e)
            assert end[f_, 0] == pytest.approx(R * q0[f_, 0], rel=1e-12, abs=1e-14)
            assert end[v_, 0] == pytest.approx(q0[v_, 0] + g / e * (R - 1) * q0[f_, 0], rel=1e-12)
        for q in (0, 1, 2, 3, 4, 5, 9):
            np.testing.assert_allclose(Qt[q, 0], [q0[q, 0]] + [0.0] * N, atol=1e-12)
        # exact zeros by back-substitution; rounding of pivoted LU otherwise
        bound = 0.0 if fn is predictor.predict_alg3 else 1e-13 * np.abs(q0).max()
        assert np.abs(Qt[:, 1:, :]).max() <= bound


def test_stiff_limit_l_stable():
    """R_{N,N+1}(e) -> 0 as e -> -inf (L-stability of the stiff solve)."""
    for N in (1, 3, 6):
        assert abs(_pade_exp(N, N + 1, -1e6)) < 1e-5


# ---------------------------------------------------------------- P4: hyperbolic part (CK Taylor)
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_inviscid_predictor_is_ck_taylor(N):
    """E = 0: the element-local solution of q_t + sum_j A^j d_j q = 0 from a
    degree-N polynomial is the Cauchy-Kovalewski Taylor polynomial
    sum_k tau^k/k! D^k Q0 (Eq. taylor), D Q = -sum_j A^{j*} Q Khat^{jT}
    nilpotent; it lies in the time space, so the predictor equals its
    Legendre projection.  Independent of the DG-in-time matrices."""
    As, Es, q0, _ = _element(N, 4, stiff=0.0)
    assert np.count_nonzero(Es) == 0
    Kh = basis.khat_matrices(N)

    def D(Q):
        return -sum(As[j] @ Q @ Kh[j].T for j in range(3))

    terms = [q0]
    for k in range(1, N + 1):
        terms.append(D(terms[-1]) / k)
    assert np.abs(D(terms[-1])).max() < 1e-9 * np.abs(q0).max()
    x, w = roots_legendre(N + 2)
    tau, wt = (x + 1) / 2, w / 2
    Qt = np.zeros((13, basis.n_modes(N), N + 1))
    for tq, wq in zip(tau, wt):
        Qtau = sum(t * tq ** k for k, t in enumerate(terms))
        for s in range(N + 1):
            Qt[:, :, s] += (2 * s + 1) * wq * Qtau * eval_jacobi(s, 0, 0, 2 * tq - 1)
    for fn in (predictor.predict_dense, predictor.predict_alg3):
        got = fn(N, As, Es, q0)
        assert np.linalg.norm(got - Qt) / np.linalg.norm(Qt) < 1e-12


# ---------------------------------------------------------------- time integration
def test_time_integration_sub_intervals():
    """int_a^b chi_s against Gauss quadrature; [0,1] picks mode 0 only."""
    N = 5
    x, w = roots_legendre(8)
    for a, b in ((0.0, 1.0), (0.0, 0.5), (0.5, 1.0), (0.25, 0.75)):
        tq = a + (b - a) * (x + 1) / 2
        ref = [(b - a) / 2 * np.sum(w * eval_jacobi(s, 0, 0, 2 * tq - 1)) for s in range(N + 1)]
        np.testing.assert_allclose(timebasis.chi_integrals(N, a, b), ref, atol=1e-15)
    np.testing.assert_allclose(timebasis.chi_integrals(N, 0, 1), [1.0] + [0.0] * N, atol=1e-15)


def test_cfl_regular_tet():
    """Regular tetrahedron of edge a: insphere diameter a / sqrt(6)."""
    a = 2.0
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(8) * a
    assert geometry.insphere_diameter(v) == pytest.approx(a / np.sqrt(6), rel=1e-14)
    mat = inputs.material_dict(inputs.REFERENCE_MATERIAL)
    assert geometry.cfl_dt(v, mat, 3) == pytest.approx(0.5 / 7 * a / np.sqrt(6) / geometry.max_wave_speed(mat))
