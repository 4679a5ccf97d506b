"""Dubiner modal basis on the reference tetrahedron, in exact rational
arithmetic, and the spatial matrices of the space-time predictor.

Paper, Section "Spatial discretisation": the solution is expanded in
orthogonal Dubiner polynomials phi_l on the reference tetrahedron
E = {xi, eta, zeta >= 0, xi + eta + zeta <= 1}, ordered by non-decreasing
degree; B(N) = C(N+3, 3) functions span the polynomials of degree <= N and
each degree g adds C(g+2, 2) of them.
Section "Space-Time predictor": M_kl = int phi_k phi_l and
K^alpha_kl = int phi_k d(phi_l)/d(alpha).
Section "Block-wise back-substitution": Khat^alpha = M^{-1} K^alpha.

Reading (the paper fixes neither normalisation nor the order inside one
degree): the unnormalised Koornwinder/Dubiner form

    phi_ijk = [L^i P_i(r)] [(1-zeta)^j P_j^(2i+1,0)(s)] P_k^(2i+2j+2,0)(t),
    L = 1 - eta - zeta,  r = 2 xi / L - 1,  s = 2 eta / (1 - zeta) - 1,
    t = 2 zeta - 1,

ordered by total degree g = i + j + k, then k ascending, then j ascending.
With this normalisation every phi has integer monomial coefficients, so M
and K are computed exactly as rationals from the monomial integrals
int xi^a eta^b zeta^c = a! b! c! / (a + b + c + 3)! and rounded once to
float64 at the end.  No quadrature rule is involved.
"""
from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import numpy as np


def n_modes(N: int) -> int:
    """B(N) = C(N+3, 3): number of basis functions of degree <= N."""
    return comb(N + 3, 3)


def block_size(g: int) -> int:
    """d_g = C(g+2, 2): number of basis functions of exact degree g."""
    return comb(g + 2, 2)


def block_offset(g: int) -> int:
    """o_g = C(g+2, 3): index of the first basis function of degree g."""
    return comb(g + 2, 3)


def mode_triples(N: int):
    """(i, j, k) of every basis function in basis order."""
    out = []
    for g in range(N + 1):
        for k in range(g + 1):
            for j in range(g - k + 1):
                out.append((g - j - k, j, k))
    return out


# --- exact polynomial arithmetic: dict {(a, b, c): int} over xi, eta, zeta ---

def _pmul(p, q):
    r = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            r[e] = r.get(e, 0) + ca * cb
    return {e: c for e, c in r.items() if c != 0}


def _padd(p, q):
    r = dict(p)
    for e, c in q.items():
        r[e] = r.get(e, 0) + c
    return {e: c for e, c in r.items() if c != 0}


def _ppow(p, n):
    r = {(0, 0, 0): 1}
    for _ in range(n):
        r = _pmul(r, p)
    return r


def _pscale(p, s):
    return {e: c * s for e, c in p.items() if c * s != 0}


_ONE = {(0, 0, 0): 1}
_XI = {(1, 0, 0): 1}
_ETA = {(0, 1, 0): 1}
_ZETA = {(0, 0, 1): 1}


def _jacobi_homogenised(n, alpha, lo, hi):
    """hi-weighted Jacobi polynomial in homogeneous form.

    With x = 2 u / w - 1 (u = `hi`, w a linear form), the Jacobi polynomial
    P_n^(alpha,0)(x) = sum_m C(n+alpha, n-m) C(n, m) ((x-1)/2)^m ((x+1)/2)^(n-m)
    times w^n equals sum_m C(n+alpha, n-m) C(n, m) (u - w)^m u^(n-m);
    `lo` is the polynomial u - w.
    """
    r = {}
    for m in range(n + 1):
        c = comb(n + alpha, n - m) * comb(n, m)
        r = _padd(r, _pscale(_pmul(_ppow(lo, m), _ppow(hi, n - m)), c))
    return r


@lru_cache(maxsize=None)
def dubiner_poly(i, j, k):
    """Monomial expansion (integer coefficients) of phi_ijk.  The returned
    dict is cached and shared: callers read it and never modify it."""
    L = _padd(_ONE, _pscale(_padd(_ETA, _ZETA), -1))          # 1 - eta - zeta
    f1 = _jacobi_homogenised(i, 0, _padd(_XI, _pscale(L, -1)), _XI)
    L2 = _padd(_ONE, _pscale(_ZETA, -1))                       # 1 - zeta
    f2 = _jacobi_homogenised(j, 2 * i + 1, _padd(_ETA, _pscale(L2, -1)), _ETA)
    f3 = _jacobi_homogenised(k, 2 * i + 2 * j + 2, _padd(_ZETA, _pscale(_ONE, -1)), _ZETA)
    return _pmul(_pmul(f1, f2), f3)


def _monomials(deg):
    return [(a, b, c) for g in range(deg + 1) for c in range(g + 1)
            for b in range(g - c + 1) for a in [g - b - c]]


def monomial_integral(a, b, c) -> Fraction:
    """int_E xi^a eta^b zeta^c dV = a! b! c! / (a+b+c+3)!  (exact)."""
    return Fraction(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))


@lru_cache(maxsize=None)
def _exact_matrices(N):
    """Exact M (diagonal entries and full matrix) and K^alpha as Fractions."""
    triples = mode_triples(N)
    monos = _monomials(N)
    midx = {m: t for t, m in enumerate(monos)}
    B, nm = len(triples), len(monos)
    C = np.zeros((B, nm), dtype=object)
    C[:] = 0
    dC = [np.zeros((B, nm), dtype=object) for _ in range(3)]
    for d in dC:
        d[:] = 0
    for l, (i, j, k) in enumerate(triples):
        for e, c in dubiner_poly(i, j, k).items():
            C[l, midx[e]] += c
            for ax in range(3):
                if e[ax] > 0:
                    e2 = list(e)
                    e2[ax] -= 1
                    dC[ax][l, midx[tuple(e2)]] += c * e[ax]
    # integer Gram matrix of the monomials, scaled by D = (2N+3)!
    D = factorial(2 * N + 3)
    G = np.zeros((nm, nm), dtype=object)
    for a, ma in enumerate(monos):
        for b, mb in enumerate(monos):
            s = (ma[0] + mb[0], ma[1] + mb[1], ma[2] + mb[2])
            v = monomial_integral(*s) * D
            assert v.denominator == 1
            G[a, b] = v.numerator
    CG = C.dot(G)
    Mint = CG.dot(C.T)
    Kint = [CG.dot(d.T) for d in dC]
    return Mint, Kint, D


def mass_matrix(N):
    """M_kl = int_E phi_k phi_l (float64, correctly rounded from exact)."""
    Mint, _, D = _exact_matrices(N)
    return np.array([[float(Fraction(v, D)) for v in row] for row in Mint])


def stiffness_matrices(N):
    """K^alpha_kl = int_E phi_k d_alpha phi_l, alpha = xi, eta, zeta."""
    _, Kint, D = _exact_matrices(N)
    return [np.array([[float(Fraction(v, D)) for v in row] for row in K]) for K in Kint]


def khat_matrices(N):
    """Khat^alpha = M^{-1} K^alpha (M diagonal), exact then rounded."""
    Mint, Kint, _ = _exact_matrices(N)
    B = Mint.shape[0]
    out = []
    for K in Kint:
        out.append(np.array([[float(Fraction(K[k, l], Mint[k, k])) for l in range(B)]
                             for k in range(B)]))
    return out


def khat_exact(N):
    """Khat^alpha as exact Fractions (used by the pins)."""
    Mint, Kint, _ = _exact_matrices(N)
    B = Mint.shape[0]
    return [[[Fraction(K[k, l], Mint[k, k]) for l in range(B)] for k in range(B)] for K in Kint]


def mass_exact_diag(N):
    Mint, _, D = _exact_matrices(N)
    return [Fraction(Mint[k, k], D) for k in range(Mint.shape[0])]


def mass_exact_offdiag_max(N):
    """Largest |M_kl| over k != l, exactly (0 for an orthogonal basis)."""
    Mint, _, _ = _exact_matrices(N)
    B = Mint.shape[0]
    return max((abs(Mint[k, l]) for k in range(B) for l in range(B) if k != l), default=0)


@lru_cache(maxsize=None)
def _polys(N):
    return [dubiner_poly(*t) for t in mode_triples(N)]


def eval_basis(N, xi, eta, zeta):
    """phi_l(xi, eta, zeta) for all l: the exact polynomial evaluated at the
    (exactly converted) float64 point, rounded once."""
    x, y, z = Fraction(xi), Fraction(eta), Fraction(zeta)
    out = np.empty(n_modes(N))
    for l, p in enumerate(_polys(N)):
        out[l] = float(sum(c * x ** e[0] * y ** e[1] * z ** e[2] for e, c in p.items()))
    return out
