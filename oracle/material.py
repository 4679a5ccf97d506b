"""Biot material -> Jacobians A, B, C and source matrix E (13 x 13, float64).

Paper, Section "Governing equations":
  * quantity vector q = (s_xx, s_yy, s_zz, s_xy, s_yz, s_xz, u, v, w, p, uf, vf, wf)
    and the system q_t + A q_x + B q_y + C q_z = E q  (Eq. poroelastic-wave);
  * rho = phi rho_F + (1 - phi) rho_S, K_M = lambda_M + 2/3 mu_M,
    M = K_S / ((1 - K_M/K_S) - phi (1 - K_S/K_F)), alpha = 1 - K_M/K_S
    (Section "Constitutive behaviour");
  * the constitutive matrix relating (sigma, -p) to (eps^M, -zeta);
  * the equations of motion with Darcy's term (Eq. biot-dynamic).
The paper does not print A, B, C, E (it defers them to another work); they are
derived here.  Readings taken:
  * off-diagonal "lambda" of the constitutive matrix is lambda_M, so the
    undrained coefficient is lambda_c = lambda_M + M alpha^2;
  * shear rows are engineering shear: d/dt s_xy = mu (d_x v + d_y u);
  * the second row of Eq. biot-dynamic carries rho_F (not rho) in front of
    dv/dt, i.e. the symmetric Biot mass matrix [[rho, rho_F], [rho_F, m]],
    m = rho_F T / phi;
  * zeta_t = -div(v^F) with v^F the relative fluid velocity.
Inverting the mass matrix (D = rho m - rho_F^2, b = nu / kappa) gives
    v_t  = ( m div(sigma) + rho_F grad p + rho_F b v^F) / D
    vF_t = (-rho_F div(sigma) - rho grad p - rho b v^F) / D
and the constitutive law in rate form gives
    s_ii_t = (lambda_c + 2 mu) d_i v_i + lambda_c sum_{j!=i} d_j v_j + M alpha div(v^F)
    s_ij_t = mu (d_i v_j + d_j v_i),     p_t = -M alpha div(v) - M div(v^F).
"""
import numpy as np

# quantity indices (paper order)
SXX, SYY, SZZ, SXY, SYZ, SXZ, U, V, W, P, UF, VF, WF = range(13)
NQ = 13

PARAM_NAMES = ("K_S", "rho_S", "lambda_M", "mu_M", "kappa", "phi", "T", "K_F", "rho_F", "nu")


def derived(mat):
    """Derived Biot quantities from the 10 parameters of Table
    poroelastic_parameters (dict keyed by PARAM_NAMES)."""
    K_S, rho_S, lam, mu = mat["K_S"], mat["rho_S"], mat["lambda_M"], mat["mu_M"]
    kappa, phi, T, K_F, rho_F, nu = (mat["kappa"], mat["phi"], mat["T"], mat["K_F"],
                                     mat["rho_F"], mat["nu"])
    rho = phi * rho_F + (1.0 - phi) * rho_S
    K_M = lam + 2.0 / 3.0 * mu
    M = K_S / ((1.0 - K_M / K_S) - phi * (1.0 - K_S / K_F))
    alpha = 1.0 - K_M / K_S
    lam_c = lam + M * alpha * alpha
    m = rho_F * T / phi
    D = rho * m - rho_F * rho_F
    b = nu / kappa if nu != 0.0 else 0.0
    return dict(rho=rho, K_M=K_M, M=M, alpha=alpha, lam_c=lam_c, m=m, D=D, b=b, mu=mu)


def jacobians(mat):
    """A, B, C: x-, y-, z-direction Jacobians (Eq. poroelastic-wave)."""
    d = derived(mat)
    lam_c, mu, M, alpha = d["lam_c"], d["mu"], d["M"], d["alpha"]
    m, D, rho, rho_F = d["m"], d["D"], d["rho"], mat["rho_F"]
    # per direction x_i: normal stress row, the two shear stresses touching i,
    # solid and fluid velocity components
    normal = (SXX, SYY, SZZ)
    vel = (U, V, W)
    fvel = (UF, VF, WF)
    shear = {(0, 1): SXY, (1, 2): SYZ, (0, 2): SXZ}

    def sh(a, b):
        return shear[(min(a, b), max(a, b))]

    out = []
    for i in range(3):
        J = np.zeros((NQ, NQ))
        # stresses: s_kk_t - (lam_c + 2mu delta_ik) d_i u_i - M alpha d_i uf_i = 0
        for k in range(3):
            J[normal[k], vel[i]] = -(lam_c + 2.0 * mu) if k == i else -lam_c
            J[normal[k], fvel[i]] = -M * alpha
        # shear: s_ij_t - mu (d_i v_j + d_j v_i) = 0 -> in direction i, s_ij row hits v_j
        for j in range(3):
            if j != i:
                J[sh(i, j), vel[j]] = -mu
        # pressure: p_t + M alpha d_i u_i + M d_i uf_i = 0
        J[P, vel[i]] = M * alpha
        J[P, fvel[i]] = M
        # velocities: direction i derivative of sigma_{k i} enters row k
        for k in range(3):
            s_ki = normal[i] if k == i else sh(k, i)
            J[vel[k], s_ki] = -m / D
            J[fvel[k], s_ki] = rho_F / D
        J[vel[i], P] = -rho_F / D
        J[fvel[i], P] = rho / D
        out.append(J)
    return out


def source_matrix(mat):
    """E: the Darcy (reactive) source term, E q on the right of
    Eq. poroelastic-wave.  Upper triangular with 6 non-zeros."""
    d = derived(mat)
    E = np.zeros((NQ, NQ))
    for v_, f_ in ((U, UF), (V, VF), (W, WF)):
        E[v_, f_] = mat["rho_F"] * d["b"] / d["D"]
        E[f_, f_] = -d["rho"] * d["b"] / d["D"]
    return E


def wave_speeds(mat, n=(1.0, 0.0, 0.0)):
    """Sorted non-negative real parts of the eigenvalues of the normal
    Jacobian n_x A + n_y B + n_z C (the characteristic speeds)."""
    A, B, C = jacobians(mat)
    An = n[0] * A + n[1] * B + n[2] * C
    ev = np.linalg.eigvals(An)
    return np.sort(np.abs(ev.real))[::-1]


def biot_frequency(mat):
    """f_c = nu phi / (2 pi T kappa rho_F) (Section "Equations of motion")."""
    return mat["nu"] * mat["phi"] / (2.0 * np.pi * mat["T"] * mat["kappa"] * mat["rho_F"])


def check_physical(mat):
    """Raise ValueError for materials outside the model's domain."""
    d = derived(mat)
    if not (0.0 < mat["phi"] < 1.0):
        raise ValueError("porosity outside (0, 1)")
    if mat["nu"] > 0.0 and mat["kappa"] <= 0.0:
        raise ValueError("non-positive permeability with viscous fluid")
    if d["M"] <= 0.0:
        raise ValueError("non-positive coupling modulus M")
    if d["D"] <= 0.0:
        raise ValueError("indefinite Biot mass matrix")
    if mat["mu_M"] <= 0.0 or mat["rho_S"] <= 0.0 or mat["rho_F"] <= 0.0:
        raise ValueError("non-positive modulus or density")
