"""Plane-wave solutions of the Biot system and DG projections (test
infrastructure, part of the oracle: only tests, the smoke check and the
bench's CPU legs may use it).

Paper, Section "Convergence" (plane-wave test on a periodic cube): for
q_t + A q_x + B q_y + C q_z = E q, the ansatz q = q^ exp(i (k.x - w t)) gives
    (k_x A + k_y B + k_z C + i E) q^ = w q^,
so every eigenpair (w, q^) of that complex 13 x 13 matrix is an exact
solution; Im w <= 0 because E only dissipates.  The real solution used here
is a sum of the selected modes, q(x, t) = Re sum_m q^_m exp(i (k.x - w_m t)),
with each eigenvector scaled to unit 2-norm and its largest component made
real and positive.

The DG projection onto an element is the L2 projection in the element's
basis: Q_pl = (int_ref q_p(x(xi)) phi_l(xi) dxi) / M_ll, with a collapsed
Gauss product rule on the reference tetrahedron.
"""
import numpy as np
from scipy.special import roots_legendre

from . import basis, geometry, material
from .corrector import basis_values


def plane_wave_modes(mat, k, count=3):
    """The `count` eigenpairs (w, q^) of k.A + i E with the largest Re w
    (fast P, then the two S waves for count = 3)."""
    A = material.jacobians(mat)
    KA = sum(float(k[d]) * A[d] for d in range(3)) + 1j * material.source_matrix(mat)
    w, V = np.linalg.eig(KA)
    order = np.argsort(-w.real)
    modes = []
    for idx in order[:count]:
        v = V[:, idx] / np.linalg.norm(V[:, idx])
        big = np.argmax(np.abs(v))
        v = v * (np.abs(v[big]) / v[big])  # largest component real positive
        modes.append((complex(w[idx]), v))
    return modes


def plane_wave(x, t, k, modes):
    """Real plane-wave field q(x, t) at points x [n][3] -> [n][13]."""
    x = np.atleast_2d(np.asarray(x, float))
    phase = x @ np.asarray(k, float)
    q = np.zeros((x.shape[0], 13))
    for w, v in modes:
        q += np.real(np.exp(1j * (phase[:, None] - w * t)) * v[None, :])
    return q


def tet_quadrature(n):
    """Collapsed (Duffy) Gauss-Legendre product rule with n points per
    direction on the reference tetrahedron {xi, eta, zeta >= 0, sum <= 1}:
    xi = u, eta = v (1 - u), zeta = w (1 - u)(1 - v), Jacobian
    (1 - u)^2 (1 - v).  Weights sum to 1/6."""
    r, wr = roots_legendre(n)
    g, wg = (r + 1) / 2, wr / 2
    pts, wts = [], []
    for u, wu in zip(g, wg):
        for v, wv in zip(g, wg):
            for s, ws in zip(g, wg):
                pts.append((u, v * (1 - u), s * (1 - u) * (1 - v)))
                wts.append(wu * wv * ws * (1 - u) ** 2 * (1 - v))
    return np.array(pts), np.array(wts)


def project(vertices, N, field, qn=None, chunk=4096):
    """L2 projection of field(x [n][3]) -> [n][13] onto the DG basis of
    every element; vertices [ne][4][3] -> Q [ne][13][B]."""
    qn = qn or N + 4
    pts, wts = tet_quadrature(qn)
    phi = basis_values(N, pts)                                   # [nq][B]
    M = np.diag(basis.mass_matrix(N))
    vertices = np.asarray(vertices, float)
    out = np.zeros((len(vertices), 13, basis.n_modes(N)))
    for c0 in range(0, len(vertices), chunk):
        v = vertices[c0:c0 + chunk]
        x0 = v[:, 0, :]                                          # [ne][3]
        J = np.stack([v[:, 1] - x0, v[:, 2] - x0, v[:, 3] - x0], axis=2)  # [ne][3][3], columns
        x = x0[:, None, :] + np.einsum("qj,edj->eqd", pts, J)   # [ne][nq][3]
        q = field(x.reshape(-1, 3)).reshape(len(v), len(pts), 13)
        out[c0:c0 + chunk] = np.einsum("eqp,q,ql->epl", q, wts, phi) / M[None, None, :]
    return out


def dg_error(vertices, N, Q, Qref):
    """Discrete L2 norm of Q - Qref, sum_e |J_e| sum_l M_ll |Q - Qref|_pl^2
    (the L2 norm of the difference of the two DG fields), and the same norm
    of Qref; returns (error, reference)."""
    M = np.diag(basis.mass_matrix(N))
    v = np.asarray(vertices, float)
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    dj = np.abs(np.linalg.det(J))
    err = np.einsum("e,l,epl->", dj, M, (np.asarray(Q) - Qref) ** 2)
    ref = np.einsum("e,l,epl->", dj, M, np.asarray(Qref) ** 2)
    return float(np.sqrt(err)), float(np.sqrt(ref))


def error_norms(vertices, N, Q, field, t=None, qn=None, chunk=4096):
    """L1, L2 and L-infinity norms of the DG field Q minus the exact field,
    over all 13 quantities: at the points of the collapsed Gauss rule of
    every element, e(x) = sum_l Q_pl phi_l(xi) - q_p(x);
      L1 = sum_e |J_e| sum_q w_q sum_p |e_p|,
      L2 = (sum_e |J_e| sum_q w_q sum_p e_p^2)^(1/2),
      Linf = max over points and p of |e_p|.
    Returns dict(err=(L1, L2, Linf), ref=(the same norms of q))."""
    qn = qn or N + 4
    pts, wts = tet_quadrature(qn)
    phi = basis_values(N, pts)                                   # [nq][B]
    vertices = np.asarray(vertices, float)
    e1 = e2 = einf = r1 = r2 = rinf = 0.0
    for c0 in range(0, len(vertices), chunk):
        v = vertices[c0:c0 + chunk]
        x0 = v[:, 0, :]
        J = np.stack([v[:, 1] - x0, v[:, 2] - x0, v[:, 3] - x0], axis=2)
        dj = np.abs(np.linalg.det(J))
        x = x0[:, None, :] + np.einsum("qj,edj->eqd", pts, J)
        q = field(x.reshape(-1, 3)).reshape(len(v), len(pts), 13)
        qh = np.einsum("epl,ql->eqp", np.asarray(Q[c0:c0 + chunk]), phi)
        d = qh - q
        w = dj[:, None] * wts[None, :]
        e1 += float(np.einsum("eq,eqp->", w, np.abs(d)))
        e2 += float(np.einsum("eq,eqp->", w, d * d))
        einf = max(einf, float(np.abs(d).max()))
        r1 += float(np.einsum("eq,eqp->", w, np.abs(q)))
        r2 += float(np.einsum("eq,eqp->", w, q * q))
        rinf = max(rinf, float(np.abs(q).max()))
    return {"err": (e1, float(np.sqrt(e2)), einf), "ref": (r1, float(np.sqrt(r2)), rinf)}
