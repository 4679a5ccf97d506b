"""Godunov numerical flux of the poroelastic system (exact Riemann solver).

Paper, Section "Spatial discretisation": the numerical flux F^j across face j
is Godunov's flux from exact Riemann problems; Sections "Homogeneous
full-space" (absorbing boundaries), "Free surface" (sigma n = 0, p = 0) and
"Planar wave convergence analysis" (periodic boundaries).  The paper gives
only the names; the construction here is the reading:

For a face with unit normal n pointing from the element L out to R, let
A_n = n_x A + n_y B + n_z C of each side.  The Riemann solution keeps the
outgoing characteristics of each side and adds the waves that enter it:
    q*_L = q_L + R_L^- alpha     (the 4 eigenvectors of A_n^L with speed < 0)
    q*_R = q_R + R_R^+ beta      (the 4 eigenvectors of A_n^R with speed > 0)
with alpha, beta fixed by the 8 open-pore interface conditions: continuity
of the traction sigma.n (3), the pore pressure p (1), the solid velocity
(3) and the normal relative fluid velocity v^F.n (1).  The flux into L is
A_n^L q*_L = F^- q_L + F^+ q_R (two 13 x 13 "flux solver" matrices).
  * free surface: q*_L = q_L + R_L^- alpha with sigma.n = 0, p = 0;
  * absorbing: no incoming waves, F^- = A_n^+ (positive part), F^+ = 0;
  * periodic: an interior face with the wrapped neighbour.
"""
import numpy as np

from . import material

SIG = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (1, 2): 4, (2, 1): 4, (0, 2): 5, (2, 0): 5}


def normal_jacobian(mat, n):
    A, B, C = material.jacobians(mat)
    return n[0] * A + n[1] * B + n[2] * C


def _impedance_scaling(mat):
    """Diagonal D with stresses and pressure in units of the impedance
    rho c_max and velocities unscaled: D^{-1} A_n D has entries of the order
    of the wave speeds (A_n itself mixes ~1e10 and ~1e-4)."""
    d = material.derived(mat)
    c = float(material.wave_speeds(mat)[0])
    z = d["rho"] * c
    s = np.ones(13)
    s[[0, 1, 2, 3, 4, 5, material.P]] = z
    return s


def _projectors(An, s):
    """Real spectral projectors of A_n (scaled by s) onto its negative and
    positive speeds.  The eigen-decomposition runs in complex arithmetic: the
    degenerate speeds (S waves, the 5-fold zero) may come back with complex
    eigenvectors, and only the projectors are real."""
    As = An * s[None, :] / s[:, None]
    lam, V = np.linalg.eig(As)
    Vi = np.linalg.inv(V)
    tol = 1e-6 * np.abs(lam).max()

    def proj(mask, weights=None):
        w = mask.astype(float) if weights is None else np.where(mask, weights, 0.0)
        return ((V * w[None, :]) @ Vi).real      # in the scaled frame

    return lam.real, tol, proj


def _basis(P, k, s):
    """k columns spanning the range of the rank-k projector P (given in the
    scaled frame), returned in physical units."""
    U = np.linalg.svd(P)[0][:, :k]
    return U * s[:, None]


def _eig_split(An, s):
    """(R^-, R^+): real bases of the invariant subspaces of A_n with negative
    and positive speeds."""
    lam, tol, proj = _projectors(An, s)
    neg, pos = lam < -tol, lam > tol
    return _basis(proj(neg), int(neg.sum()), s), _basis(proj(pos), int(pos.sum()), s)


def traction_pressure_rows(n):
    """4 x 13: (sigma.n)_x, (sigma.n)_y, (sigma.n)_z, p."""
    C = np.zeros((4, 13))
    for i in range(3):
        for j in range(3):
            C[i, SIG[(i, j)]] += n[j]
    C[3, material.P] = 1.0
    return C


def interface_rows(n):
    """8 x 13: traction (3), p, solid velocity (3), v^F . n."""
    C = np.zeros((8, 13))
    C[:4] = traction_pressure_rows(n)
    C[4, material.U] = C[5, material.V] = C[6, material.W] = 1.0
    C[7, material.UF], C[7, material.VF], C[7, material.WF] = n
    return C


def positive_part(An, mat):
    """(A_n^+, A_n^-): the parts of A_n with positive / negative speeds."""
    sc = _impedance_scaling(mat)
    lam, tol, proj = _projectors(An, sc)
    back = sc[:, None] / sc[None, :]
    return proj(lam > tol, lam) * back, proj(lam < -tol, lam) * back


def _solve_scaled(M, rhs, rows_scale):
    """Solve M x = rhs with the rows divided by rows_scale first."""
    r = rhs / (rows_scale[:, None] if rhs.ndim == 2 else rows_scale)
    return np.linalg.solve(M / rows_scale[:, None], r)


def flux_matrices(matL, matR, n, kind="interior"):
    """(F^-, F^+) with A_n^L q*_L = F^- q_L + F^+ q_R.  kind: 'interior'
    (also periodic), 'free_surface', 'absorbing'."""
    n = np.asarray(n, float)
    AL = normal_jacobian(matL, n)
    sL = _impedance_scaling(matL)
    if kind == "absorbing":
        Ap, _ = positive_part(AL, matL)
        return Ap, np.zeros((13, 13))
    RLm, _ = _eig_split(AL, sL)
    assert RLm.shape[1] == 4, "expected 4 waves entering the element"
    z = sL[0]
    if kind == "free_surface":
        Cf = traction_pressure_rows(n)
        G = _solve_scaled(Cf @ RLm, Cf, np.full(4, z))          # alpha = -G q_L
        return AL @ (np.eye(13) - RLm @ G), np.zeros((13, 13))
    AR = normal_jacobian(matR, n)
    _, RRp = _eig_split(AR, _impedance_scaling(matR))
    assert RRp.shape[1] == 4
    C = interface_rows(n)
    rs = np.array([z, z, z, z, 1.0, 1.0, 1.0, 1.0])
    # [C R_L^-, -C R_R^+] [alpha; beta] = C (q_R - q_L)
    M = np.hstack([C @ RLm, -C @ RRp])
    Galpha = _solve_scaled(M, C, rs)[:4]                        # alpha = Galpha (q_R - q_L)
    K = RLm @ Galpha
    return AL @ (np.eye(13) - K), AL @ K


def godunov_states(matL, matR, n, qL, qR):
    """(q*_L, q*_R) of the interior Riemann problem (for the pins)."""
    n = np.asarray(n, float)
    AL, AR = normal_jacobian(matL, n), normal_jacobian(matR, n)
    RLm = _eig_split(AL, _impedance_scaling(matL))[0]
    RRp = _eig_split(AR, _impedance_scaling(matR))[1]
    C = interface_rows(n)
    z = _impedance_scaling(matL)[0]
    rs = np.array([z, z, z, z, 1.0, 1.0, 1.0, 1.0])
    M = np.hstack([C @ RLm, -C @ RRp])
    ab = _solve_scaled(M, C @ (qR - qL), rs)
    return qL + RLm @ ab[:4], qR + RRp @ ab[4:]
