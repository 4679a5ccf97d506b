/* Algorithm 3 (Section "Block-wise back-substitution") as plain C loops,
 * binary64, one element after another, OpenMP over elements.
 *
 * TEST INFRASTRUCTURE of the oracle: the timed CPU baseline and a second
 * statement of Algorithm 3 checked against the dense LU solve (the oracle's
 * definition).  No BLAS, no blocking beyond the algorithm's own degree
 * blocks; built with -ffp-contract=off so every product and sum rounds as
 * written.  The reference matrices (Khat^j, Z, S^{-1} w) come from the Python
 * oracle (oracle/basis.py, oracle/timebasis.py); this file holds only the
 * algorithm's steps.
 *
 * For one element, with b[p][l][u] = (S^{-1} w)_u Q0[p][l] and degree blocks
 * g = N .. 0 (modes [o_g, o_g + d_g)):
 *   time solves, p = 12 .. 0:  (Z - E*_pp I) Qt[p][m][:] = b[p][m][:]
 *                              for the modes m of block g; then the coupling
 *                              b[o][m][:] += E*_op Qt[p][m][:] for o < p;
 *   green update (g > 0):      b[p][l][u] -= sum_j sum_{m in block g}
 *                              Khat^j[l][m] (sum_q A^{j*}_pq Qt[q][m][u]),
 *                              over the rows l < o_g (the other rows of the
 *                              block's columns are zero, Lemma 1).
 * Zero entries of A^{j*} and Khat^j are skipped.
 *
 * Layouts (row-major): Astar[n][3][13][13], Estar[n][13][13], Q0[n][13][B],
 * Khat[3][B][B], Z[T][T], sinv_w[T], Qt[n][13][B][T].
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 13
#define TMAX 8

/* x = A^{-1} y for a T x T matrix A (Gaussian elimination with partial
 * pivoting on a copy); returns 0 if a pivot is zero */
static int solve_small(int T, const double* A, double* x) {
    double a[TMAX][TMAX];
    for (int r = 0; r < T; ++r)
        for (int c = 0; c < T; ++c) a[r][c] = A[r * T + c];
    for (int k = 0; k < T; ++k) {
        int piv = k;
        for (int r = k + 1; r < T; ++r)
            if ((a[r][k] < 0 ? -a[r][k] : a[r][k]) > (a[piv][k] < 0 ? -a[piv][k] : a[piv][k])) piv = r;
        if (a[piv][k] == 0.0) return 0;
        if (piv != k) {
            for (int c = 0; c < T; ++c) {
                double t = a[k][c];
                a[k][c] = a[piv][c];
                a[piv][c] = t;
            }
            double t = x[k];
            x[k] = x[piv];
            x[piv] = t;
        }
        for (int r = k + 1; r < T; ++r) {
            double f = a[r][k] / a[k][k];
            for (int c = k; c < T; ++c) a[r][c] -= f * a[k][c];
            x[r] -= f * x[k];
        }
    }
    for (int k = T - 1; k >= 0; --k) {
        double s = x[k];
        for (int c = k + 1; c < T; ++c) s -= a[k][c] * x[c];
        x[k] = s / a[k][k];
    }
    return 1;
}

static int predict_one(int N, int B, const double* As, const double* Es, const double* q0, const double* Kh,
                       const double* Z, const double* sinv_w, double* Qt, double* b, double* X) {
    const int T = N + 1;
    double Zp[TMAX * TMAX];
    for (int p = 0; p < NQ; ++p)
        for (int l = 0; l < B; ++l)
            for (int u = 0; u < T; ++u) b[(p * B + l) * T + u] = sinv_w[u] * q0[p * B + l];
    memset(Qt, 0, sizeof(double) * NQ * B * T);
    for (int g = N; g >= 0; --g) {
        const int o = g * (g + 1) * (g + 2) / 6, d = (g + 1) * (g + 2) / 2;
        for (int p = NQ - 1; p >= 0; --p) {
            for (int r = 0; r < T; ++r)
                for (int c = 0; c < T; ++c) Zp[r * T + c] = Z[r * T + c] - (r == c ? Es[p * NQ + p] : 0.0);
            for (int m = o; m < o + d; ++m) {
                double* x = Qt + (p * B + m) * T;
                for (int u = 0; u < T; ++u) x[u] = b[(p * B + m) * T + u];
                if (!solve_small(T, Zp, x)) return 0;
                for (int oq = 0; oq < p; ++oq) {
                    const double G = Es[oq * NQ + p];
                    if (G == 0.0) continue;
                    for (int u = 0; u < T; ++u) b[(oq * B + m) * T + u] += G * x[u];
                }
            }
        }
        if (g == 0) break;
        for (int j = 0; j < 3; ++j) {
            const double* A = As + j * NQ * NQ;
            /* X[p][m][u] = sum_q A^{j*}_pq Qt[q][m][u], modes m of block g */
            for (int p = 0; p < NQ; ++p)
                for (int ml = 0; ml < d; ++ml)
                    for (int u = 0; u < T; ++u) {
                        double s = 0.0;
                        for (int q = 0; q < NQ; ++q) {
                            const double a = A[p * NQ + q];
                            if (a != 0.0) s += a * Qt[(q * B + o + ml) * T + u];
                        }
                        X[(p * d + ml) * T + u] = s;
                    }
            /* b[p][l][u] -= sum_m Khat^j[l][m] X[p][m][u], rows l < o_g */
            const double* K = Kh + (size_t)j * B * B;
            for (int l = 0; l < o; ++l)
                for (int ml = 0; ml < d; ++ml) {
                    const double k = K[l * B + o + ml];
                    if (k == 0.0) continue;
                    for (int p = 0; p < NQ; ++p)
                        for (int u = 0; u < T; ++u) b[(p * B + l) * T + u] -= k * X[(p * d + ml) * T + u];
                }
        }
    }
    return 1;
}

/* Predictor of n elements with `threads` OpenMP threads (<= 0: the
 * runtime's default).  Returns the number of elements solved (n unless a
 * time-matrix pivot was zero, which the system never produces for e <= 0). */
int64_t oracle_alg3_predict(int N, int64_t n, const double* Astar, const double* Estar, const double* Q0,
                            const double* Khat, const double* Z, const double* sinv_w, double* Qt, int threads) {
    if (N < 0 || N + 1 > TMAX) return 0;
    const int B = (N + 1) * (N + 2) * (N + 3) / 6, T = N + 1;
    const int dmax = (N + 1) * (N + 2) / 2;
    int64_t ok = 0;
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt) reduction(+ : ok)
    {
        double* b = (double*)malloc(sizeof(double) * NQ * B * T);
        double* X = (double*)malloc(sizeof(double) * NQ * dmax * T);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < n; ++e)
            ok += predict_one(N, B, Astar + e * 3 * NQ * NQ, Estar + e * NQ * NQ, Q0 + e * NQ * B, Khat, Z, sinv_w,
                              Qt + e * NQ * B * T, b, X);
        free(b);
        free(X);
    }
    return ok;
}

/* Threads a call with `threads` <= 0 uses. */
int oracle_alg3_default_threads(void) { return omp_get_max_threads(); }
