"""Sub-cell material variation in the space-time predictor (test
infrastructure, part of the oracle).

Paper, Section "Limitations": with material parameters that vary inside an
element, the second integral of the weak form has to be evaluated with the
varying Jacobians, and the stiffness matrices become 3-tensors.  Reading of
this build: the Jacobians A_d(x) and the source matrix E(x) vary linearly
inside each tetrahedron, interpolating their values for four vertex
materials, A_d(x) = sum_v lambda_v(x) A_d(mat_v) with lambda_v the
barycentric coordinates.  In the modal basis a linear field is
f(xi) = sum_{r<4} f_r phi_r(xi) (phi_0..phi_3 the Dubiner modes of degree
<= 1), and the predictor system of Eq. stp-lineq becomes

    Y = I (x) M (x) (W - K^tau) - sum_r E*_r (x) M3_r (x) S
        + sum_j sum_r A^{j*}_r (x) K3^j_r (x) S

with the 3-tensors M3_r[k, l] = int phi_k phi_r phi_l and
K3^j_r[k, l] = int phi_k phi_r d_j phi_l (exact rationals, rounded once).
With r = 0 alone (constant material) this is Eq. stp-lineq.  The oracle's
solution is the dense LU of this Y.
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial

import numpy as np
import scipy.linalg as sla

from . import basis, geometry, material, predictor, timebasis

NR = 4  # modes of a linear field

REF_VERTICES = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))


def _poly_coeffs(polys, monos):
    idx = {m: t for t, m in enumerate(monos)}
    C = np.zeros((len(polys), len(monos)), dtype=object)
    C[:] = 0
    for a, p in enumerate(polys):
        for e, c in p.items():
            C[a, idx[e]] += c
    return C


def _derivative(p, ax):
    out = {}
    for e, c in p.items():
        if e[ax] > 0:
            e2 = list(e)
            e2[ax] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0) + c * e[ax]
    return out


@lru_cache(maxsize=None)
def _exact_tensors(N):
    """Integer matrices D * M3_r and D * K3^j_r (D = (2N+4)!) for r < 4."""
    triples = basis.mode_triples(N)
    phis = [basis.dubiner_poly(*t) for t in triples]
    lin = phis[:NR]
    monos_n = basis._monomials(N)
    monos_n1 = basis._monomials(N + 1)
    C = _poly_coeffs(phis, monos_n)
    dC = [_poly_coeffs([_derivative(p, ax) for p in phis], monos_n) for ax in range(3)]
    D = factorial(2 * N + 4)
    G = np.zeros((len(monos_n1), len(monos_n)), dtype=object)
    for a, ma in enumerate(monos_n1):
        for b, mb in enumerate(monos_n):
            v = basis.monomial_integral(ma[0] + mb[0], ma[1] + mb[1], ma[2] + mb[2]) * D
            assert v.denominator == 1
            G[a, b] = v.numerator
    M3, K3 = [], []
    for r in range(NR):
        Cr = _poly_coeffs([basis._pmul(p, lin[r]) for p in phis], monos_n1)  # phi_k phi_r
        CG = Cr.dot(G)
        M3.append(CG.dot(C.T))
        K3.append([CG.dot(d.T) for d in dC])
    return M3, K3, D


def tensors(N):
    """M3[r] (B x B) and K3[r][j] (B x B), float64, r < 4, j = xi, eta, zeta."""
    M3i, K3i, D = _exact_tensors(N)

    def f(A):
        return np.array([[float(Fraction(v, D)) for v in row] for row in A])

    return [f(m) for m in M3i], [[f(k) for k in kr] for kr in K3i]


@lru_cache(maxsize=None)
def linear_projection():
    """P (4 x 4): the modal coefficients f_r = sum_v P[r, v] f_v of the linear
    field with values f_v at the reference vertices (0,0,0), (1,0,0), (0,1,0),
    (0,0,1); P = V^{-1}, V[v, r] = phi_r(vertex v), exact."""
    lin = [basis.dubiner_poly(*t) for t in basis.mode_triples(1)]
    V = [[Fraction(sum(c * Fraction(x) ** e[0] * Fraction(y) ** e[1] * Fraction(z) ** e[2]
                       for e, c in p.items())) for p in lin] for (x, y, z) in REF_VERTICES]
    Vm = sla.inv(np.array([[float(v) for v in row] for row in V]))
    return Vm


def element_operators(vert, mats, dt):
    """A^{j*}_r (4 x 3 x 13 x 13) and E*_r (4 x 13 x 13) of the linear
    interpolation of the four vertex materials' Jacobians and source
    matrices (vertex v of `vert` carries mats[v])."""
    P = linear_projection()
    Av = np.stack([np.stack(geometry.reference_jacobians(vert, m)) for m in mats])   # [v][j]
    Ev = np.stack([material.source_matrix(m) for m in mats])
    Astar = dt * np.einsum("rv,vjpq->rjpq", P, Av)
    Estar = dt * np.einsum("rv,vpq->rpq", P, Ev)
    return Astar, Estar


def assemble_dense(N, Astar, Estar):
    """Y with the unrolling (p, k, s) -> (p*B + k)*T + s."""
    M = basis.mass_matrix(N)
    M3, K3 = tensors(N)
    W, _, S, Kt = timebasis.time_matrices(N)
    nq = Estar.shape[1]
    Y = np.kron(np.eye(nq), np.kron(M, W - Kt))
    for r in range(NR):
        Y -= np.kron(Estar[r], np.kron(M3[r], S))
        for j in range(3):
            Y += np.kron(Astar[r, j], np.kron(K3[r][j], S))
    return Y


def predict_dense(N, Astar, Estar, Q0):
    """Qt[q, l, s] by equilibrated dense LU of Y (the definition)."""
    B, T, nq = basis.n_modes(N), N + 1, Estar.shape[1]
    Y = assemble_dense(N, Astar, Estar)
    R, C = predictor.equilibrate(Y)
    lu = sla.lu_factor(Y * R[:, None] * C[None, :], check_finite=True)
    return (C * sla.lu_solve(lu, R * predictor.rhs_dense(N, Q0))).reshape(nq, B, T)
