"""Time basis and time matrices of the space-time predictor.

Paper, Section "Space-Time predictor": on the reference time interval [0, 1]
the predictor uses Jacobi polynomials chi_s of the same degree N as space,
and the matrices
    W_rs = chi_r(1) chi_s(1),  w_r = chi_r(0),
    S_rs = int_0^1 chi_r chi_s,  K^tau_rs = int_0^1 chi_r' chi_s.
Section "Block-wise back-substitution": Z = S^{-1} (W - K^tau).
Reading: the Jacobi parameters are not given; the figure caption of the
sparsity plot calls S_rs diagonal, which holds on [0, 1] only for the
Legendre family, so chi_s(tau) = P_s(2 tau - 1) (shifted Legendre).
The matrices are computed here by integrating numpy Legendre series exactly
(products of degree <= 2N are integrated by the antiderivative).
"""
import numpy as np
from numpy.polynomial import legendre as L


def _chi(s):
    c = np.zeros(s + 1)
    c[s] = 1.0
    return c  # Legendre series in x = 2 tau - 1


def _integral_01(c):
    """int_0^1 f(tau) dtau for f given as a Legendre series in x = 2tau-1."""
    ci = L.legint(c)
    return 0.5 * (L.legval(1.0, ci) - L.legval(-1.0, ci))


def time_matrices(N):
    T = N + 1
    W = np.zeros((T, T))
    w = np.zeros(T)
    S = np.zeros((T, T))
    Kt = np.zeros((T, T))
    for r in range(T):
        w[r] = L.legval(-1.0, _chi(r))
        for s in range(T):
            W[r, s] = L.legval(1.0, _chi(r)) * L.legval(1.0, _chi(s))
            S[r, s] = _integral_01(L.legmul(_chi(r), _chi(s)))
            # d/dtau chi_r = 2 d/dx P_r
            dr = 2.0 * L.legder(_chi(r)) if r > 0 else np.zeros(1)
            Kt[r, s] = _integral_01(L.legmul(dr, _chi(s)))
    return W, w, S, Kt


def z_matrix(N):
    W, _, S, Kt = time_matrices(N)
    return np.linalg.solve(S, W - Kt)


def chi_values(N, tau):
    """chi_s(tau) for s = 0..N."""
    return np.array([L.legval(2.0 * tau - 1.0, _chi(s)) for s in range(N + 1)])


def chi_integrals(N, a, b):
    """int_a^b chi_s(tau) dtau for s = 0..N (sub-interval integrals used by
    time integration)."""
    out = np.zeros(N + 1)
    for s in range(N + 1):
        ci = L.legint(_chi(s))
        out[s] = 0.5 * (L.legval(2.0 * b - 1.0, ci) - L.legval(2.0 * a - 1.0, ci))
    return out
