"""Isotropic viscoelastic attenuation in the first-order form of the
space-time predictor (test infrastructure, part of the oracle).

Paper, Section "Other applications": Algorithm 3 applies to linear
hyperbolic systems whose source matrix is upper triangular, and viscoelastic
attenuation is named as one.  The paper gives no equations for it; this
module states the usual anelastic-function form of a generalised Maxwell
body with n relaxation mechanisms (reading of this build):

    d sigma/dt = lam_u tr(D) I + 2 mu_u D - sum_l (Ylam_l tr(th_l) I + 2 Ymu_l th_l)
    rho dv/dt  = div sigma
    d th_l/dt  = omega_l (D - th_l),                  l = 1..n

with D = (grad v + grad v^T) / 2 the strain rate, lam_u, mu_u the unrelaxed
Lame moduli, omega_l the relaxation frequencies and Ylam_l, Ymu_l the
anelastic coefficients.  A plane wave exp(i(k.x - w t)) sees the complex
moduli

    lam(w) = lam_u - sum_l Ylam_l omega_l / (omega_l - i w)    (mu alike),

so rho w^2 = |k|^2 (lam(w) + 2 mu(w)) for P waves and rho w^2 = |k|^2 mu(w)
for S waves (used as a pin).

Quantities (27 for n = 3), in this order: the 6 stresses (xx, yy, zz, xy,
yz, xz), the 3 velocities, then th_1 (6 components, same order), th_2,
th_3.  With q_t + A q_x + B q_y + C q_z = E q, E has -omega_l on the
diagonal of th_l and -(Ylam_l delta + 2 Ymu_l) couplings from th_l into the
stresses, all right of the diagonal: E is upper triangular, and the time
solves of Algorithm 3 are: th rows with (Z + omega_l dt I)^{-1}, then the
stresses after adding E* th, velocities with Z^{-1}.

Material: dict with rho, lam (unrelaxed), mu (unrelaxed), and arrays omega,
Ylam, Ymu of length n (consistent units).
"""
import numpy as np

from . import geometry

NMECH = 3
NQ = 9 + 6 * NMECH
SXX, SYY, SZZ, SXY, SYZ, SXZ, U, V, W = range(9)


def th(l, k):
    """Index of component k (0..5, stress order) of mechanism l."""
    return 9 + 6 * l + k


def jacobians(mat):
    """A, B, C of q_t + A q_x + B q_y + C q_z = E q."""
    lam, mu, rho = mat["lam"], mat["mu"], mat["rho"]
    A, B, C = (np.zeros((NQ, NQ)) for _ in range(3))
    J = (A, B, C)
    vel = (U, V, W)
    normal = (SXX, SYY, SZZ)
    # stresses: sigma_ii,t = lam div v + 2 mu d_i v_i; sigma_ij,t = mu (d_j v_i + d_i v_j)
    for i in range(3):
        for d in range(3):
            J[d][normal[i], vel[d]] = -(lam + 2 * mu) if d == i else -lam
    for s, (a, b) in ((SXY, (0, 1)), (SYZ, (1, 2)), (SXZ, (0, 2))):
        J[b][s, vel[a]] = -mu   # d_b v_a
        J[a][s, vel[b]] = -mu   # d_a v_b
    # momentum: rho v_i,t = sum_j d_j sigma_ij
    sig = np.array([[SXX, SXY, SXZ], [SXY, SYY, SYZ], [SXZ, SYZ, SZZ]])
    for i in range(3):
        for d in range(3):
            J[d][vel[i], sig[i, d]] = -1.0 / rho
    # anelastic functions: th_l,t = omega_l D + ... (D_ii = d_i v_i, D_ab = (d_b v_a + d_a v_b) / 2)
    for l in range(NMECH):
        w = mat["omega"][l]
        for i in range(3):
            J[i][th(l, i), vel[i]] = -w
        for k, (a, b) in ((3, (0, 1)), (4, (1, 2)), (5, (0, 2))):
            J[b][th(l, k), vel[a]] = -w / 2
            J[a][th(l, k), vel[b]] = -w / 2
    return [A, B, C]


def source_matrix(mat):
    E = np.zeros((NQ, NQ))
    for l in range(NMECH):
        yl, ym = mat["Ylam"][l], mat["Ymu"][l]
        for k in range(6):
            E[th(l, k), th(l, k)] = -mat["omega"][l]
        for i in range(3):
            for k in range(3):
                E[i, th(l, k)] = -(yl + 2 * ym) if i == k else -yl
        for k in (3, 4, 5):
            E[k, th(l, k)] = -2 * ym
    return E


def complex_moduli(mat, w):
    """lam(w), mu(w) of a plane wave of angular frequency w (complex)."""
    om = np.asarray(mat["omega"], dtype=float)
    f = om / (om - 1j * w)
    return (mat["lam"] - np.sum(np.asarray(mat["Ylam"]) * f), mat["mu"] - np.sum(np.asarray(mat["Ymu"]) * f))


def speeds(mat):
    """Unrelaxed (high-frequency) P and S speeds."""
    return np.sqrt((mat["lam"] + 2 * mat["mu"]) / mat["rho"]), np.sqrt(mat["mu"] / mat["rho"])


def element_operators(vert, mat, dt):
    """A^{j*} = dt sum_d (d xi_j / d x_d) A_d and E* = dt E (Section
    "Space-Time predictor")."""
    _, _, Jinv = geometry.affine(vert)
    Ad = jacobians(mat)
    Astar = np.stack([dt * sum(Jinv[j, d] * Ad[d] for d in range(3)) for j in range(3)])
    return Astar, dt * source_matrix(mat)


def cfl_dt(vert, mat, N, c=0.5):
    """dt = c / (2N + 1) d / v_P with the unrelaxed P speed."""
    return c / (2 * N + 1) * geometry.insphere_diameter(vert) / speeds(mat)[0]
