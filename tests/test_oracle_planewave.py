"""Pin P7 (full scheme order) on the oracle: plane waves of the Biot system
on a periodic mesh (paper, Section "Convergence").  The analytic solution is
checked against the PDE itself; the oracle's ADER-DG run (predictor,
corrector, periodic Godunov flux, source term) must converge to it at the
optimal order N + 1."""
import numpy as np
import pytest

from oracle import basis, corrector, material, planewave
from paper_2108_10565_gb300 import inputs

K_CUBE = np.array([np.pi, np.pi, np.pi])


def _modes(k):
    return planewave.plane_wave_modes(inputs.material_dict(inputs.REFERENCE_MATERIAL), k, 3)


def test_plane_wave_solves_the_pde():
    """q_t + A q_x + B q_y + C q_z - E q = 0 for the real plane-wave field,
    by central differences in space and time at random points (independent
    of the eigen-decomposition that produced it)."""
    md = inputs.material_dict(inputs.REFERENCE_MATERIAL)
    A = material.jacobians(md)
    E = material.source_matrix(md)
    modes = _modes(K_CUBE)
    rng = np.random.default_rng(7)
    for _ in range(4):
        x = rng.uniform(-1, 1, 3)
        t = rng.uniform(0, 1e-4)
        hx, ht = 1e-4, 1e-9
        q = lambda y, s: planewave.plane_wave(y[None, :], s, K_CUBE, modes)[0]
        dq_dt = (q(x, t + ht) - q(x, t - ht)) / (2 * ht)
        res = dq_dt - E @ q(x, t)
        scale = np.abs(dq_dt) + np.abs(E @ q(x, t))
        for d in range(3):
            e = np.zeros(3)
            e[d] = hx
            g = (q(x + e, t) - q(x - e, t)) / (2 * hx)
            res += A[d] @ g
            scale += np.abs(A[d] @ g)
        assert np.max(np.abs(res) / np.max(scale)) < 1e-6
    # the selected modes: fast P first, then the two S waves (equal speeds)
    w = [m[0] for m in modes]
    assert w[0].real > w[1].real > 0 and abs(w[1].real - w[2].real) < 1e-6 * w[1].real
    assert all(m[0].imag <= 0 for m in modes)  # the source term only dissipates


@pytest.mark.parametrize("n", [2, 4, 6])
def test_tet_quadrature_integrates_monomials(n):
    pts, wts = planewave.tet_quadrature(n)
    deg = 2 * n - 3
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                exact = float(basis.monomial_integral(a, b, c))
                got = np.sum(wts * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert got == pytest.approx(exact, rel=1e-13, abs=1e-16)


def test_projection_reproduces_polynomials():
    """The DG projection is exact for fields of degree <= N."""
    N = 3
    mesh = inputs.kuhn_box_mesh(3, lo=(-1, -1, -1), hi=(1, 1, 1))
    v = mesh["vertices"][mesh["tets"]]
    f = lambda x: np.stack([x[:, 0] ** 3 - 2 * x[:, 1] * x[:, 2] + p for p in range(13)], axis=1)
    Q = planewave.project(v, N, f)
    pts = np.array([[0.1, 0.2, 0.3], [0.25, 0.25, 0.25], [0.6, 0.1, 0.2]])
    phi = corrector.basis_values(N, pts)
    for e in (0, 17, 101):
        x0 = v[e][0]
        J = np.stack([v[e][1] - x0, v[e][2] - x0, v[e][3] - x0], axis=1)
        np.testing.assert_allclose(Q[e] @ phi.T, f(x0[None] + pts @ J.T).T, atol=1e-12)


@pytest.mark.parametrize("N", [1, 2])
def test_oracle_converges_at_order_n_plus_1(N):
    """Plane wave along x (k = (pi, 0, 0)) on the periodic cube [-1, 1]^3
    with (8, 3, 3) and (16, 3, 3) Kuhn boxes, one common time step (the
    coarse mesh's CFL step, halved on the fine mesh) and the same final
    time: the error of the oracle's GTS run against the projected exact
    solution falls at the optimal rate N + 1 (within 0.25)."""
    k = np.array([np.pi, 0.0, 0.0])
    modes = _modes(k)
    sims = []
    for nx in (8, 16):
        mesh = inputs.kuhn_box_mesh((nx, 3, 3), lo=(-1, -1, -1), hi=(1, 1, 1))
        mats = np.tile(inputs.REFERENCE_MATERIAL, (len(mesh["tets"]), 1))
        sims.append((mesh, corrector.GTSSimulation(mesh, mats, N)))
    dtc = min(sims[0][1].dt, 2 * sims[1][1].dt)
    errs = []
    for i, (mesh, sim) in enumerate(sims):
        sim.dt = dtc / (1 + i)
        steps = 6 * (1 + i)
        v = mesh["vertices"][mesh["tets"]]
        Q0 = planewave.project(v, N, lambda x: planewave.plane_wave(x, 0.0, k, modes))
        Q, _ = sim.run(Q0, steps)
        Qref = planewave.project(v, N, lambda x: planewave.plane_wave(x, steps * sim.dt, k, modes))
        e, r = planewave.dg_error(v, N, Q, Qref)
        errs.append(e / r)
    rate = np.log2(errs[0] / errs[1])
    assert errs[1] < 0.01
    assert abs(rate - (N + 1)) < 0.25, (errs, rate)


def test_error_norms_of_a_known_offset():
    """error_norms against a closed form: the exact projection of a degree-N
    polynomial field, compared with that field plus a constant c in one
    quantity, differs by exactly c everywhere: L1 = |c| vol, L2 = |c|
    sqrt(vol), Linf = |c|; and a field compared with its own projection
    (degree <= N) has zero error."""
    N = 2
    mesh = inputs.kuhn_box_mesh(3, lo=(0, 0, 0), hi=(1.5, 1.5, 1.5))
    v = mesh["vertices"][mesh["tets"]]
    vol = 1.5 ** 3

    def poly(x):
        q = np.zeros((len(x), 13))
        q[:, 0] = 1 + x[:, 0] * x[:, 1] - 2 * x[:, 2] ** 2
        q[:, 9] = x[:, 0] - 3 * x[:, 1] * x[:, 2]
        return q

    c = 0.25
    Q = planewave.project(v, N, poly)
    r = planewave.error_norms(v, N, Q, poly)
    assert max(r["err"]) < 1e-12

    def shifted(x):
        q = poly(x)
        q[:, 4] += c
        return q

    r = planewave.error_norms(v, N, Q, shifted)
    np.testing.assert_allclose(r["err"], (c * vol, c * np.sqrt(vol), c), rtol=1e-12)
