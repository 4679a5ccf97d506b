// Device building blocks of the degree-block back-substitution (Section
// "Block-wise back-substitution", Algorithm 3), templated on the arithmetic
// type so the binary64 kernel and the binary32 sweeps of the refinement
// kernel run the same code.
//
// Shared-memory layout of one element's b / Q tensor: quantity p at offset
// p * QS, mode l at l * T, time mode u at u, where the quantity stride QS is
// B * T padded so that QS = T (mod 32): the 13 T lanes (p, u) of one mode then
// fall on consecutive 4-byte banks (conflict-free).  The star products X use
// the same rule with the block size d_g in place of B.
#pragma once

#include <cuda_runtime.h>

#include "poro_internal.h"

namespace poro {

__host__ __device__ constexpr int bank_stride(int n, int T) { return n + ((T - n % 32) + 32) % 32; }

template <int T, class Real>
__device__ __forceinline__ void solve_row(Real* row, const Real* Zi);

// The linear system of the predictor: its quantities, the union pattern of
// its reference Jacobians and the structure of its source matrix E (upper
// triangular, Section "Block-wise back-substitution"): per mode the time
// solves are NPLAIN rows with Z^{-1} (E_pp = 0), NSHIFT rows with
// (Z - e I)^{-1} and no coupling, and NPAIR pairs: src solved with
// (Z - e I)^{-1}, then b_dst += g Q_src, then dst with Z^{-1}.
// Per-element constants (in this order): star[3][NNZ], NSHM shifted time
// matrices (Z - e I)^{-1}, NSC scalars with dt at DT_SC; TWO_PHASE systems
// solve their blocks with solve_block (below) instead of the kinds above.
struct BiotSystem {  // Biot's equations: G couples u_f -> u, v_f -> v, w_f -> w
    static constexpr int NQ = poro::NQ, NNZ = STAR_NNZ, NPLAIN = 7, NSHIFT = 0, NPAIR = 3;
    static constexpr int NSHM = 1, NSC = 4, DT_SC = 2;
    static constexpr bool TWO_PHASE = false;
    PORO_HD static constexpr int row(int n) { return star_row(n); }
    PORO_HD static constexpr int col(int n) { return star_col(n); }
    PORO_HD static constexpr int plain(int k) { return k < 6 ? k : QP; }
    PORO_HD static constexpr int shifted(int) { return 0; }
    PORO_HD static constexpr int pair_src(int i) { return QUF + i; }
    PORO_HD static constexpr int pair_dst(int i) { return QU + i; }
};
struct MaxwellSystem {  // damped Maxwell: E diagonal, -sigma/eps on the electric rows
    static constexpr int NQ = maxwell::NQ, NNZ = maxwell::STAR_NNZ, NPLAIN = 3, NSHIFT = 3, NPAIR = 0;
    static constexpr int NSHM = 1, NSC = 4, DT_SC = 2;
    static constexpr bool TWO_PHASE = false;
    PORO_HD static constexpr int row(int n) { return maxwell::star_row(n); }
    PORO_HD static constexpr int col(int n) { return maxwell::star_col(n); }
    PORO_HD static constexpr int plain(int k) { return 3 + k; }
    PORO_HD static constexpr int shifted(int k) { return k; }
    PORO_HD static constexpr int pair_src(int) { return 0; }
    PORO_HD static constexpr int pair_dst(int) { return 0; }
};
// Viscoelastic attenuation: per mode, phase 1 solves the velocities with
// Z^{-1} and mechanism l's six anelastic functions with (Z - e_l I)^{-1};
// after a barrier, phase 2 adds to each stress its couplings to the solved
// functions (E* strictly upper part) and solves it with Z^{-1}.
struct ViscoSystem {
    static constexpr int NQ = visco::NQ, NNZ = visco::STAR_NNZ, NPLAIN = 0, NSHIFT = 0, NPAIR = 0;
    static constexpr int NSHM = visco::NMECH, NSC = visco::NSC, DT_SC = visco::sc_dt();
    static constexpr bool TWO_PHASE = true;
    PORO_HD static constexpr int row(int n) { return visco::star_row(n); }
    PORO_HD static constexpr int col(int n) { return visco::star_col(n); }
    PORO_HD static constexpr int plain(int) { return 0; }
    PORO_HD static constexpr int shifted(int) { return 0; }
    PORO_HD static constexpr int pair_src(int) { return 0; }
    PORO_HD static constexpr int pair_dst(int) { return 0; }
    // modes [o, o + d) of one degree block; zsh: NMECH matrices (Z - e_l I)^{-1};
    // cp: per mechanism the couplings (normal diagonal, normal off-diagonal,
    // shear) of E*.  The caller's barrier follows.
    template <int T, int NT, int QS, class Real>
    __device__ static void solve_block(Real* bq, int o, int d, const Real* zin, const Real* zsh, const Real* cp) {
        const int tid = threadIdx.x;
        constexpr int NM = visco::NMECH;
        for (int it = tid; it < (3 + 6 * NM) * d; it += NT) {
            const int kind = it / d, m = o + it % d;
            if (kind < 3) solve_row<T>(bq + (6 + kind) * QS + m * T, zin);
            else solve_row<T>(bq + (9 + (kind - 3)) * QS + m * T, zsh + ((kind - 3) / 6) * T * T);
        }
        __syncthreads();
        for (int it = tid; it < 6 * d; it += NT) {
            const int c = it / d, m = o + it % d;
            Real* row = bq + c * QS + m * T;
#pragma unroll
            for (int l = 0; l < NM; ++l) {
                const Real* th = bq + (9 + 6 * l) * QS + m * T;
                if (c < 3) {
                    // normal stress c: (Ylam + 2 Ymu) on th_cc, Ylam on the other two
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const Real g = k == c ? cp[3 * l] : cp[3 * l + 1];
#pragma unroll
                        for (int u = 0; u < T; ++u) row[u] = fma(g, th[k * QS + u], row[u]);
                    }
                } else {
                    const Real g = cp[3 * l + 2];
#pragma unroll
                    for (int u = 0; u < T; ++u) row[u] = fma(g, th[c * QS + u], row[u]);
                }
            }
            solve_row<T>(row, zin);
        }
    }
};

template <int N, int NQ_ = NQ>
struct Alg3Shape {
    static constexpr int B = n_modes(N);
    static constexpr int T = N + 1;
    static constexpr int QBT = NQ_ * B * T;                // dense size (global layout)
    static constexpr int QS = bank_stride(B * T, T);       // shared quantity stride
    static constexpr int SQ = NQ_ * QS;                    // shared size of b / Q
    static constexpr int DMAX = block_size(N);
    static constexpr int XSMAX = bank_stride(DMAX * T, T);
    static constexpr int PT = NQ_ * T;                     // (p, u) pairs of one mode
    static constexpr int PUL = (PT + 31) / 32;             // pairs per lane
};

// Khat^j block CSR (rows l < o_g, columns m_local of block g) for one precision
template <class Real>
struct KhatBlocks {
    const Real* val;
    const int32_t* col;
    const int32_t* row;
    int32_t row_base[MAX_N + 1][3];
    // optional (one direction per pass): block (g, j)'s rows dealt to the
    // warps, [warps + 1] starts then the lists, at lists + list_base[g][j]
    const int32_t* lists = nullptr;
    int32_t list_base[MAX_N + 1][3];
};

template <int T, class Real>
__device__ __forceinline__ void solve_row(Real* row, const Real* Zi) {
    Real x[T];
#pragma unroll
    for (int s = 0; s < T; ++s) x[s] = row[s];
#pragma unroll
    for (int u = 0; u < T; ++u) {
        Real acc = Real(0);
#pragma unroll
        for (int s = 0; s < T; ++s) acc = fma(Zi[u * T + s], x[s], acc);
        row[u] = acc;
    }
}

// b[p,l,u] = (S^{-1} w)_u q0[p,l] with (S^{-1} w)_u = (2u+1)(-1)^u
template <int N, int NT, class Real, class In, int NQ_ = NQ>
__device__ __forceinline__ void init_rhs(Real* bq, const In* q0) {
    using S = Alg3Shape<N, NQ_>;
    for (int i = threadIdx.x; i < NQ_ * S::B; i += NT) {
        const Real v = (Real)q0[i];
        const int p = i / S::B, l = i % S::B;
        Real* row = bq + p * S::QS + l * S::T;
#pragma unroll
        for (int u = 0; u < S::T; ++u) row[u] = Real((2 * u + 1) * ((u & 1) ? -1 : 1)) * v;
    }
}

// In-place sweep: on entry bq holds b, on exit the solution Q.  X is a
// scratch area of JX * Sys::NQ * XSMAX values in shared memory; star[3][NNZ]
// the element's reference Jacobians on the union pattern; zuf = (Z - e I)^{-1},
// zin = Z^{-1}; gcoup = the coupling entry g of E* (Biot: E*_{u,uf}); for
// two-phase systems zuf holds their NSHM shifted matrices and cpl their
// couplings.  JX
// directions are handled per pass (1 or 3).  Ends with a barrier.
template <int N, int NT, class Real, int JX, class Sys = BiotSystem>
__device__ void alg3_sweep(Real* bq, Real* X, const Real* star, const Real* zuf, const Real* zin,
                           const Real gcoup, const KhatBlocks<Real>& K, const Real* cpl = nullptr) {
    constexpr int NQ = Sys::NQ, STAR_NNZ = Sys::NNZ;
    using S = Alg3Shape<N, NQ>;
    constexpr int T = S::T, QS = S::QS, PT = S::PT, PUL = S::PUL, NW = NT / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int lp[PUL], lu[PUL];
#pragma unroll
    for (int k = 0; k < PUL; ++k) {
        const int pu = lane + 32 * k;
        lp[k] = pu < PT ? pu / T : 0;
        lu[k] = pu < PT ? pu % T : 0;
    }
#pragma unroll 1
    for (int g = N; g >= 0; --g) {
        const int o = block_offset(g), d = block_size(g);
        // time solves of block g, per mode: the plain rows, the shifted rows,
        // and the coupled pairs (Biot: 6 stresses and p; u_f then u, v_f
        // then v, w_f then w)
        constexpr int NKIND = Sys::NPLAIN + Sys::NSHIFT + Sys::NPAIR;
        if constexpr (Sys::TWO_PHASE) {
            Sys::template solve_block<T, NT, QS, Real>(bq, o, d, zin, zuf, cpl);
        } else {
          for (int it = tid; it < NKIND * d; it += NT) {
            const int kind = it / d, m = o + it % d;
            if (kind < Sys::NPLAIN) {
                solve_row<T>(bq + Sys::plain(kind) * QS + m * T, zin);
            } else if (kind < Sys::NPLAIN + Sys::NSHIFT) {
                solve_row<T>(bq + Sys::shifted(kind - Sys::NPLAIN) * QS + m * T, zuf);
            } else {
                const int i = kind - Sys::NPLAIN - Sys::NSHIFT;
                Real* rf = bq + Sys::pair_src(i) * QS + m * T;
                Real* rv = bq + Sys::pair_dst(i) * QS + m * T;
                solve_row<T>(rf, zuf);
#pragma unroll
                for (int u = 0; u < T; ++u) rv[u] = fma(gcoup, rf[u], rv[u]);
                solve_row<T>(rv, zin);
            }
          }
        }
        __syncthreads();
        if (g == 0) break;
        const int XS = bank_stride(d * T, T);
#pragma unroll 1
        for (int jb = 0; jb < 3; jb += JX) {
            // X^j[p, ml, u] = sum_q A^{j*}_pq Q[q, o+ml, u]
            for (int it = tid; it < d * T; it += NT) {
                const int ml = it / T, u = it % T;
                Real qv[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) qv[q] = bq[q * QS + (o + ml) * T + u];
#pragma unroll
                for (int jj = 0; jj < JX; ++jj) {
                    const Real* sj = star + (jb + jj) * STAR_NNZ;
                    Real acc[NQ];
#pragma unroll
                    for (int p = 0; p < NQ; ++p) acc[p] = Real(0);
#pragma unroll
                    for (int n = 0; n < STAR_NNZ; ++n)
                        acc[Sys::row(n)] = fma(sj[n], qv[Sys::col(n)], acc[Sys::row(n)]);
                    Real* xj = X + jj * NQ * S::XSMAX + ml * T + u;
#pragma unroll
                    for (int p = 0; p < NQ; ++p) xj[p * XS] = acc[p];
                }
            }
            __syncthreads();
            // b[p, l, u] -= sum_j sum_m Khat^j[l, o+m] X^j[p, m, u], l < o;
            // one warp per row l, each lane owns PUL (p, u) pairs
            int xo[PUL];
#pragma unroll
            for (int k = 0; k < PUL; ++k) xo[k] = lp[k] * XS + lu[k];
            auto row = [&](int l) {
                Real acc[PUL];
#pragma unroll
                for (int k = 0; k < PUL; ++k) acc[k] = Real(0);
#pragma unroll
                for (int jj = 0; jj < JX; ++jj) {
                    const int32_t* rp = K.row + K.row_base[g][jb + jj] + l;
                    const int n0 = __ldg(rp), n1 = __ldg(rp + 1);
                    const Real* xj = X + jj * NQ * S::XSMAX;
                    int n = n0;
                    for (; n + 1 < n1; n += 2) {
                        const Real v0 = __ldg(K.val + n), v1 = __ldg(K.val + n + 1);
                        const int m0 = __ldg(K.col + n) * T, m1 = __ldg(K.col + n + 1) * T;
#pragma unroll
                        for (int k = 0; k < PUL; ++k) {
                            acc[k] = fma(v0, xj[xo[k] + m0], acc[k]);
                            acc[k] = fma(v1, xj[xo[k] + m1], acc[k]);
                        }
                    }
                    if (n < n1) {
                        const Real v0 = __ldg(K.val + n);
                        const int m0 = __ldg(K.col + n) * T;
#pragma unroll
                        for (int k = 0; k < PUL; ++k) acc[k] = fma(v0, xj[xo[k] + m0], acc[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < PUL; ++k)
                    if (lane + 32 * k < PT) bq[lp[k] * QS + l * T + lu[k]] -= acc[k];
            };
            if (JX == 1 && K.lists) {
                // this warp's rows of the block, dealt so that the warps' work is balanced
                const int32_t* L = K.lists + K.list_base[g][jb];
                const int i0 = __ldg(L + warp), i1 = __ldg(L + warp + 1);
                for (int i = i0; i < i1; ++i) row(__ldg(L + NW + 1 + i));
            } else {
                for (int l = warp; l < o; l += NW) row(l);
            }
            __syncthreads();
        }
    }
}

}  // namespace poro
