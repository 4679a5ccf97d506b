"""The element-local space-time predictor: the plain definition and the
paper's three back-substitution algorithms, in float64.

Paper, Section "Space-Time predictor", Eq. stp-lineq: for one element the
predictor Qt[q, l, s] (quantity q, spatial mode l, time mode s) solves

  ( d_pq W_rs M_kl - d_pq Kt_rs M_kl - E*_pq S_rs M_kl
    + sum_j A^{j*}_pq S_rs K^j_kl ) Qt[q, l, s] = d_pq w_r M_kl Q0[q, l]

(Eq. linear_system: Y Qt = r).  `predict_dense` assembles Y densely and solves
it by LU with partial pivoting (LAPACK getrf/getrs): this is the definition
every other path is checked against.

Section "Block-wise back-substitution": Algorithms 1, 2 and 3 solve the same
system by exploiting its block-triangular structure.  They are written here
as plain loops, only to be checked against the dense solve.
"""
import numpy as np
import scipy.linalg as sla

from . import basis, geometry, material, timebasis

NQ = material.NQ


def element_operators(vert, mat, dt):
    """A^{j*} = dt A^j (3 x 13 x 13) and E* = dt E (Section "Space-Time
    predictor")."""
    Aj = geometry.reference_jacobians(vert, mat)
    Astar = np.stack([dt * a for a in Aj])
    Estar = dt * material.source_matrix(mat)
    return Astar, Estar


def assemble_dense(N, Astar, Estar):
    """Y of Eq. stp-lineq with the unrolling (p, k, r) -> (p*B + k)*T + r
    (any number of quantities: the size of E*)."""
    M = basis.mass_matrix(N)
    K = basis.stiffness_matrices(N)
    W, w, S, Kt = timebasis.time_matrices(N)
    Y = np.kron(np.eye(Estar.shape[0]), np.kron(M, W - Kt))
    Y -= np.kron(Estar, np.kron(M, S))
    for j in range(3):
        Y += np.kron(Astar[j], np.kron(K[j], S))
    return Y


def rhs_dense(N, Q0):
    """r_{pkr} = w_r M_kk Q0[p, k]."""
    M = basis.mass_matrix(N)
    _, w, _, _ = timebasis.time_matrices(N)
    return (np.diag(M)[None, :, None] * Q0[:, :, None] * w[None, None, :]).reshape(-1)


def equilibrate(Y):
    """Row then column scale factors, exact powers of two, that bring the
    largest entry of every row and column of Y to about 1 (the equilibration
    of LAPACK's getrf drivers).  Y mixes stress rows (entries ~ dt * modulus /
    h, up to ~1e5) with velocity rows (~1e-10); without equilibration a
    pivoted LU of Y loses ~5 digits at N >= 4.  Power-of-two factors change
    no rounding of the scaled system's entries."""
    R = 2.0 ** (-np.round(np.log2(np.abs(Y).max(axis=1))))
    C = 2.0 ** (-np.round(np.log2((np.abs(Y) * R[:, None]).max(axis=0))))
    return R, C


def predict_dense(N, Astar, Estar, Q0, return_factors=False):
    """Qt[q, l, s] by dense LU of Y (the oracle's definition): solve
    (R Y C) z = R r by LU with partial pivoting, Qt = C z."""
    B, T, nq = basis.n_modes(N), N + 1, Estar.shape[0]
    Y = assemble_dense(N, Astar, Estar)
    R, C = equilibrate(Y)
    lu = sla.lu_factor(Y * R[:, None] * C[None, :], check_finite=True)
    x = C * sla.lu_solve(lu, R * rhs_dense(N, Q0))
    if return_factors:
        return x.reshape(nq, B, T), (lu, R, C)
    return x.reshape(nq, B, T)


def _common(N):
    B, T = basis.n_modes(N), N + 1
    Kh = basis.khat_matrices(N)
    W, w, S, Kt = timebasis.time_matrices(N)
    Sinv_w = np.linalg.solve(S, w)
    Z = np.linalg.solve(S, W - Kt)
    return B, T, Kh, Sinv_w, Z


def predict_alg1(N, Astar, Estar, Q0):
    """Algorithm 1: for m = B..1 solve the Q(N+1) system
    (d_pq Z_us - E*_pq d_us) Qt[q, m, s] = b[p, m, u], with b pulled from the
    already solved modes l > m through Eq. b_pmu."""
    B, T, Kh, Sinv_w, Z = _common(N)
    nq = Estar.shape[0]
    Qt = np.zeros((nq, B, T))
    Ablk = np.kron(np.eye(nq), Z) - np.kron(Estar, np.eye(T))
    for m in range(B - 1, -1, -1):
        b = np.outer(Q0[:, m], Sinv_w)
        for l in range(m + 1, B):
            for j in range(3):
                b -= Kh[j][m, l] * (Astar[j] @ Qt[:, l, :])
        Qt[:, m, :] = np.linalg.solve(Ablk, b.reshape(-1)).reshape(nq, T)
    return Qt


def predict_alg2(N, Astar, Estar, Q0):
    """Algorithm 2: unrolled over modes m and quantities p; E* = F + G with
    F diagonal and G strictly upper triangular."""
    B, T, Kh, Sinv_w, Z = _common(N)
    nq = Estar.shape[0]
    F = np.diag(Estar)
    G = Estar - np.diag(F)
    b = Q0[:, :, None] * Sinv_w[None, None, :]
    Qt = np.zeros((nq, B, T))
    for m in range(B - 1, -1, -1):
        for p in range(nq - 1, -1, -1):
            Qt[p, m, :] = np.linalg.solve(Z - F[p] * np.eye(T), b[p, m, :])
            for o in range(p):
                if G[o, p] != 0.0:
                    b[o, m, :] += G[o, p] * Qt[p, m, :]
        for n in range(m):
            for j in range(3):
                b[:, n, :] -= Kh[j][n, m] * (Astar[j] @ Qt[:, m, :])
    return Qt


def predict_alg3(N, Astar, Estar, Q0):
    """Algorithm 3: Algorithm 2 with the modes of one polynomial degree fused
    (degree blocks g = N..0, modes [o_g, o_g + d_g)); the green update is the
    pair of n-mode products A^{j*} x_1 Qt[:, blk, :] x_2 Khat^j[:, blk]."""
    B, T, Kh, Sinv_w, Z = _common(N)
    nq = Estar.shape[0]
    F = np.diag(Estar)
    G = Estar - np.diag(F)
    b = Q0[:, :, None] * Sinv_w[None, None, :]
    Qt = np.zeros((nq, B, T))
    for g in range(N, -1, -1):
        blk = slice(basis.block_offset(g), basis.block_offset(g) + basis.block_size(g))
        for p in range(nq - 1, -1, -1):
            Zinv_T = np.linalg.inv(Z - F[p] * np.eye(T)).T
            Qt[p, blk, :] = b[p, blk, :] @ Zinv_T
            for o in range(p):
                if G[o, p] != 0.0:
                    b[o, blk, :] += G[o, p] * Qt[p, blk, :]
        if g > 0:
            for j in range(3):
                b -= np.einsum("pq,lm,qmu->plu", Astar[j], Kh[j][:, blk], Qt[:, blk, :])
    return Qt


def time_integrated(N, Qt, dt, a=0.0, b=1.0):
    """I[q, l] = dt * sum_s Qt[q, l, s] int_a^b chi_s (time integration of the
    predictor over [t_i + a dt, t_i + b dt]; Section "Temporal
    discretisation with ADER").  With a=0, b=1 this is dt * Qt[:, :, 0]."""
    return dt * np.einsum("qls,s->ql", Qt, timebasis.chi_integrals(N, a, b))


def residual(N, Astar, Estar, Q0, Qt):
    """r - Y Qt for the dense system (used to state conditioning in tests)."""
    Y = assemble_dense(N, Astar, Estar)
    return rhs_dense(N, Q0) - Y @ Qt.reshape(-1)
