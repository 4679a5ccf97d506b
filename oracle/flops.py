"""Operation and storage model of the paper's Table flop-count.

Paper, Section "Block-wise back-substitution":
  * LU with precomputed factors: two triangular solves, 2 s^2 flops, with
    s = Q B (N+1) unknowns; storage of the two triangles s (s+1) doubles;
  * Algorithm 3, upper bound
      2B (Q (N+1)^2 + 3(N+1) + 3(N+1) Q^2 + 3(N+1) Q B) + 3 Q B (N+1)^2;
  * Algorithm 3 storage: 13 matrices (Z - E*_pp I)^{-1} of size (N+1)^2, the
    three 13 x 13 matrices A*, B*, C* and the 6 non-zeros of E*.
Storage is reported in MiB (2^20 bytes) of float64, as in the table.
"""
from math import comb

NQ = 13


def unknowns(N):
    return NQ * comb(N + 3, 3) * (N + 1)


def lu_flops(N):
    s = unknowns(N)
    return 2 * s * s


def stp_flops_bound(N):
    B, T = comb(N + 3, 3), N + 1
    return 2 * B * (NQ * T * T + 3 * T + 3 * T * NQ * NQ + 3 * T * NQ * B) + 3 * NQ * B * T * T


def lu_storage_mib(N):
    s = unknowns(N)
    return s * (s + 1) * 8 / 2 ** 20


def stp_storage_mib(N):
    T = N + 1
    return (NQ * T * T + 3 * NQ * NQ + 6) * 8 / 2 ** 20
