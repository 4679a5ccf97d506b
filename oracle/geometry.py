"""Affine element map, reference Jacobians and the CFL time step.

Paper, Section "Spatial discretisation": an affine map takes each tetrahedron
to the reference element; the reference Jacobians are
    A* = A xi_x + B xi_y + C xi_z,  B* = A eta_x + ...,  C* = A zeta_x + ...,
constant on each element.  Section "Space-Time predictor": the predictor uses
A^{j*} = dt * A^j and E* = dt * E.  Section "Temporal discretisation with
ADER": dt <= C(N) d / v with C(N) = 0.5 / (2N + 1), d the insphere diameter
and v the largest wave speed of the element.
"""
import numpy as np

from . import material


def affine(vert):
    """x = x0 + J xi with J = [x1-x0, x2-x0, x3-x0] (columns); returns
    (x0, J, Jinv) where Jinv[j, d] = d xi_j / d x_d."""
    vert = np.asarray(vert, dtype=float)
    x0 = vert[0]
    J = np.stack([vert[1] - x0, vert[2] - x0, vert[3] - x0], axis=1)
    return x0, J, np.linalg.inv(J)


def volume(vert):
    _, J, _ = affine(vert)
    return abs(np.linalg.det(J)) / 6.0


def face_areas(vert):
    """Areas of the 4 faces; face i is opposite vertex i."""
    vert = np.asarray(vert, dtype=float)
    out = []
    for i in range(4):
        a, b, c = [vert[k] for k in range(4) if k != i]
        out.append(0.5 * np.linalg.norm(np.cross(b - a, c - a)))
    return np.array(out)


def insphere_diameter(vert):
    return 6.0 * volume(vert) / face_areas(vert).sum()


def reference_jacobians(vert, mat):
    """A^j (j = xi, eta, zeta): sum_d (d xi_j / d x_d) A_d, without dt."""
    _, _, Jinv = affine(vert)
    Ad = material.jacobians(mat)
    return [sum(Jinv[j, d] * Ad[d] for d in range(3)) for j in range(3)]


def max_wave_speed(mat):
    """Largest characteristic speed; isotropic, so direction x suffices."""
    return float(material.wave_speeds(mat)[0])


def cfl_dt(vert, mat, N, c=0.5):
    """dt = C(N) d / v, C(N) = c / (2N + 1)."""
    return c / (2 * N + 1) * insphere_diameter(vert) / max_wave_speed(mat)
