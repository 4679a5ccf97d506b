"""Damped Maxwell equations in the first-order form of the space-time
predictor (test infrastructure, part of the oracle).

Paper, Section "Other applications": the predictor and Algorithm 3 apply to
any linear hyperbolic system with a possibly stiff source term whose source
matrix is upper triangular; the damped Maxwell equations are one such system:
    eps dE/dt = curl H - sigma E,     mu dH/dt = - curl E.
Reading: the paper prints the second equation with + curl E; with that sign
the system is not hyperbolic (E_tt = -(1/(eps mu)) Laplace E for divergence-free
fields), so Faraday's law with - curl E is used.

Quantities in the order (E_x, E_y, E_z, H_x, H_y, H_z).  With the curl
expanded, q_t + A q_x + B q_y + C q_z = E q where every Jacobian couples
the electric and magnetic components through +-1/eps and +-1/mu and
E = diag(-sigma/eps x 3, 0 x 3) (diagonal, so upper triangular with G = 0).
Material parameters: dict with keys eps, mu, sigma (consistent units).
"""
import numpy as np

from . import geometry

NQ = 6
EX, EY, EZ, HX, HY, HZ = range(6)


def jacobians(mat):
    """A, B, C of q_t + A q_x + B q_y + C q_z = E q."""
    ie, im = 1.0 / mat["eps"], 1.0 / mat["mu"]
    A, B, C = (np.zeros((6, 6)) for _ in range(3))
    # eps E_t = curl H: (d_y Hz - d_z Hy, d_z Hx - d_x Hz, d_x Hy - d_y Hx)
    B[EX, HZ], C[EX, HY] = -ie, +ie
    C[EY, HX], A[EY, HZ] = -ie, +ie
    A[EZ, HY], B[EZ, HX] = -ie, +ie
    # mu H_t = -curl E
    B[HX, EZ], C[HX, EY] = +im, -im
    C[HY, EX], A[HY, EZ] = +im, -im
    A[HZ, EY], B[HZ, EX] = +im, -im
    return [A, B, C]


def source_matrix(mat):
    E = np.zeros((6, 6))
    for p in (EX, EY, EZ):
        E[p, p] = -mat["sigma"] / mat["eps"]
    return E


def speed(mat):
    """Largest characteristic speed 1 / sqrt(eps mu)."""
    return 1.0 / np.sqrt(mat["eps"] * mat["mu"])


def element_operators(vert, mat, dt):
    """A^{j*} = dt sum_d (d xi_j / d x_d) A_d and E* = dt E (Section
    "Space-Time predictor")."""
    _, _, Jinv = geometry.affine(vert)
    Ad = jacobians(mat)
    Astar = np.stack([dt * sum(Jinv[j, d] * Ad[d] for d in range(3)) for j in range(3)])
    return Astar, dt * source_matrix(mat)


def cfl_dt(vert, mat, N, c=0.5):
    """dt = c / (2N + 1) d / v with v = 1 / sqrt(eps mu)."""
    return c / (2 * N + 1) * geometry.insphere_diameter(vert) / speed(mat)
