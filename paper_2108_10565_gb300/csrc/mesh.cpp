// Host set-up of the corrector: Godunov flux matrices, face matrices of the
// Dubiner basis, mesh faces (neighbour face, vertex permutation, normal,
// area), point location and basis values at points.
//
// Flux (Section "Spatial discretisation": Godunov's flux from exact Riemann
// problems; boundary types of Sections "Homogeneous full-space", "Free
// surface", "Planar wave convergence analysis"): the invariant subspaces of
// the normal Jacobian A_n with incoming / outgoing speeds are obtained from
// the matrix sign function sign(A_n -+ sigma I) (Newton iteration with
// determinant scaling), A_n scaled by the impedance first; the Godunov state
// keeps the outgoing characteristics of each side and is fixed by continuity
// of traction, pore pressure, solid velocity and normal relative fluid
// velocity (free surface: zero traction and pressure; absorbing: no incoming
// waves).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "poro_internal.h"

namespace poro {

namespace {
using ld = double;  // the scaled Jacobians are well conditioned; double keeps set-up fast on every host

// small dense helpers (row-major n x n, long double)
void matmul(int n, const ld* a, const ld* b, ld* c) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            ld s = 0;
            for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
            c[i * n + j] = s;
        }
}

bool inverse_ld(int n, const ld* a, ld* inv, ld* det_out = nullptr) {
    std::vector<ld> m(2 * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            m[i * 2 * n + j] = a[i * n + j];
            m[i * 2 * n + n + j] = (i == j) ? 1 : 0;
        }
    ld det = 1;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(m[r * 2 * n + c]) > std::fabs(m[piv * 2 * n + c])) piv = r;
        if (m[piv * 2 * n + c] == 0) return false;
        if (piv != c) {
            for (int j = 0; j < 2 * n; ++j) std::swap(m[c * 2 * n + j], m[piv * 2 * n + j]);
            det = -det;
        }
        ld d = m[c * 2 * n + c];
        det *= d;
        for (int j = 0; j < 2 * n; ++j) m[c * 2 * n + j] /= d;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                ld f = m[r * 2 * n + c];
                if (f != 0)
                    for (int j = 0; j < 2 * n; ++j) m[r * 2 * n + j] -= f * m[c * 2 * n + j];
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = m[i * 2 * n + n + j];
    if (det_out) *det_out = det;
    return true;
}

// sign(X) by the scaled Newton iteration X <- (mu X + (mu X)^{-1}) / 2
bool matrix_sign(int n, std::vector<ld>& X) {
    std::vector<ld> inv(n * n), nxt(n * n);
    for (int it = 0; it < 100; ++it) {
        ld det;
        if (!inverse_ld(n, X.data(), inv.data(), &det)) return false;
        ld mu = std::pow(std::fabs(det), -1.0 / n);
        if (!std::isfinite((double)mu) || it > 12) mu = 1;
        ld diff = 0, norm = 0;
        for (int i = 0; i < n * n; ++i) {
            nxt[i] = 0.5L * (mu * X[i] + inv[i] / mu);
            diff = std::max(diff, std::fabs(nxt[i] - X[i]));
            norm = std::max(norm, std::fabs(nxt[i]));
        }
        X.swap(nxt);
        if (diff <= 4e-16 * norm && it > 2) return true;
    }
    return false;
}

// k columns spanning the range of the rank-k matrix P (n x n), by
// Gram-Schmidt with column pivoting (columns are returned orthonormal)
void range_basis(int n, const std::vector<ld>& P, int k, std::vector<ld>& R) {
    std::vector<ld> cols(P);  // column j = P[:, j]
    R.assign(n * k, 0);
    std::vector<bool> used(n, false);
    for (int c = 0; c < k; ++c) {
        int best = -1;
        ld bn = -1;
        for (int j = 0; j < n; ++j) {
            if (used[j]) continue;
            ld s = 0;
            for (int i = 0; i < n; ++i) s += cols[i * n + j] * cols[i * n + j];
            if (s > bn) { bn = s; best = j; }
        }
        used[best] = true;
        ld nr = std::sqrt(bn);
        for (int i = 0; i < n; ++i) R[i * k + c] = cols[i * n + best] / nr;
        // remove the new direction from the remaining columns
        for (int j = 0; j < n; ++j) {
            if (used[j]) continue;
            ld d = 0;
            for (int i = 0; i < n; ++i) d += R[i * k + c] * cols[i * n + j];
            for (int i = 0; i < n; ++i) cols[i * n + j] -= d * R[i * k + c];
        }
    }
}

struct Scaled {
    std::vector<ld> A;  // scaled normal Jacobian S^{-1} A_n S
    ld s[NQ];           // scaling
    ld An[NQ * NQ];     // physical A_n
};

bool scaled_normal_jacobian(const poro_material& m, const double n[3], Scaled& out, ld& sigma, std::string& err) {
    double abc[3][NQ][NQ], E[NQ][NQ];
    if (!material_jacobians(m, abc, E, err)) return false;
    double cmax;
    if (!max_wave_speed(m, cmax, err)) return false;
    // slowest non-zero speed: slow P (smaller root of Biot's quadratic) and S
    const double K_M = m.lambda_M + 2.0 * m.mu_M / 3.0, alpha = 1.0 - K_M / m.K_S;
    const double M = m.K_S / ((1.0 - K_M / m.K_S) - m.phi * (1.0 - m.K_S / m.K_F));
    const double rho = m.phi * m.rho_F + (1.0 - m.phi) * m.rho_S, mm = m.rho_F * m.tortuosity / m.phi;
    const double D = rho * mm - m.rho_F * m.rho_F;
    const double H = m.lambda_M + M * alpha * alpha + 2.0 * m.mu_M, C = alpha * M;
    const double a = D, b = -(H * mm + rho * M - 2.0 * C * m.rho_F), c = H * M - C * C;
    const double cslow = std::sqrt((-b - std::sqrt(b * b - 4 * a * c)) / (2 * a));
    const double cs = std::sqrt(m.mu_M * mm / D);
    sigma = 0.5L * std::min(cslow, cs);
    const ld z = (ld)rho * cmax;
    for (int q = 0; q < NQ; ++q) out.s[q] = (q <= SXZ || q == QP) ? z : 1.0L;
    out.A.assign(NQ * NQ, 0);
    for (int i = 0; i < NQ; ++i)
        for (int j = 0; j < NQ; ++j) {
            ld v = (ld)n[0] * abc[0][i][j] + (ld)n[1] * abc[1][i][j] + (ld)n[2] * abc[2][i][j];
            out.An[i * NQ + j] = v;
            out.A[i * NQ + j] = v * out.s[j] / out.s[i];
        }
    return true;
}

// spectral projector (scaled frame) on speeds > 0 (pos) or < 0 (!pos)
bool projector(const Scaled& S, ld sigma, bool pos, std::vector<ld>& P) {
    std::vector<ld> X(S.A);
    for (int i = 0; i < NQ; ++i) X[i * NQ + i] += pos ? -sigma : sigma;
    if (!matrix_sign(NQ, X)) return false;
    P.assign(NQ * NQ, 0);
    for (int i = 0; i < NQ * NQ; ++i) P[i] = pos ? 0.5L * X[i] : -0.5L * X[i];
    for (int i = 0; i < NQ; ++i) P[i * NQ + i] += 0.5L;
    return true;
}

void traction_rows(const double n[3], ld C[][NQ], int& rows, bool full) {
    const int sig[3][3] = {{SXX, SXY, SXZ}, {SXY, SYY, SYZ}, {SXZ, SYZ, SZZ}};
    for (int r = 0; r < 8; ++r)
        for (int q = 0; q < NQ; ++q) C[r][q] = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i][sig[i][j]] += n[j];
    C[3][QP] = 1;
    rows = 4;
    if (full) {
        C[4][QU] = C[5][QV] = C[6][QW] = 1;
        C[7][QUF] = n[0];
        C[7][QVF] = n[1];
        C[7][QWF] = n[2];
        rows = 8;
    }
}
}  // namespace

bool flux_solver(const poro_material& mL, const poro_material* mR, const double n[3], int kind, double* Fm,
                 double* Fp, std::string& err) {
    Scaled SL;
    ld sigL;
    if (!scaled_normal_jacobian(mL, n, SL, sigL, err)) return false;
    std::memset(Fp, 0, sizeof(double) * NQ * NQ);
    if (kind == PORO_FACE_ABSORBING) {
        std::vector<ld> P;
        if (!projector(SL, sigL, true, P)) { err = "flux: sign iteration failed"; return false; }
        // A_n^+ = A_n P^+ (physical frame: S (A_s P_s) S^{-1})
        std::vector<ld> AP(NQ * NQ);
        matmul(NQ, SL.A.data(), P.data(), AP.data());
        for (int i = 0; i < NQ; ++i)
            for (int j = 0; j < NQ; ++j) Fm[i * NQ + j] = (double)(AP[i * NQ + j] * SL.s[i] / SL.s[j]);
        return true;
    }
    std::vector<ld> Pm, RmL;
    if (!projector(SL, sigL, false, Pm)) { err = "flux: sign iteration failed"; return false; }
    range_basis(NQ, Pm, 4, RmL);
    for (int i = 0; i < NQ; ++i)
        for (int c = 0; c < 4; ++c) RmL[i * 4 + c] *= SL.s[i];  // physical frame
    ld C[8][NQ];
    int rows;
    const bool interior = (kind == PORO_FACE_INTERIOR);
    traction_rows(n, C, rows, interior);
    const ld z = SL.s[0];
    std::vector<ld> RpR;
    if (interior) {
        Scaled SR;
        ld sigR;
        if (!mR || !scaled_normal_jacobian(*mR, n, SR, sigR, err)) {
            if (err.empty()) err = "flux: interior face without neighbour material";
            return false;
        }
        std::vector<ld> Pp;
        if (!projector(SR, sigR, true, Pp)) { err = "flux: sign iteration failed"; return false; }
        range_basis(NQ, Pp, 4, RpR);
        for (int i = 0; i < NQ; ++i)
            for (int c = 0; c < 4; ++c) RpR[i * 4 + c] *= SR.s[i];
    }
    // system M x = C (q_R - q_L) (interior) or M alpha = -C q_L (free surface),
    // rows of traction / pressure divided by the impedance
    const int nu = rows;  // unknowns: 4 (free surface) or 8 (interior)
    std::vector<ld> Mx(nu * nu, 0), Minv(nu * nu), Cs(nu * NQ);
    for (int r = 0; r < nu; ++r) {
        const ld rs = r < 4 ? 1.0L / z : 1.0L;
        for (int c = 0; c < 4; ++c) {
            ld s = 0;
            for (int q = 0; q < NQ; ++q) s += C[r][q] * RmL[q * 4 + c];
            Mx[r * nu + c] = s * rs;
        }
        if (interior)
            for (int c = 0; c < 4; ++c) {
                ld s = 0;
                for (int q = 0; q < NQ; ++q) s += C[r][q] * RpR[q * 4 + c];
                Mx[r * nu + 4 + c] = -s * rs;
            }
        for (int q = 0; q < NQ; ++q) Cs[r * NQ + q] = C[r][q] * rs;
    }
    if (!inverse_ld(nu, Mx.data(), Minv.data())) { err = "flux: singular interface system"; return false; }
    // G = first 4 rows of M^{-1} C  (alpha = G (q_R - q_L), or alpha = -G q_L)
    ld G[4][NQ];
    for (int a = 0; a < 4; ++a)
        for (int q = 0; q < NQ; ++q) {
            ld s = 0;
            for (int r = 0; r < nu; ++r) s += Minv[a * nu + r] * Cs[r * NQ + q];
            G[a][q] = s;
        }
    // K = R_L^- G ;  F^- = A_n (I - K),  F^+ = A_n K (interior)
    ld K[NQ][NQ];
    for (int i = 0; i < NQ; ++i)
        for (int q = 0; q < NQ; ++q) {
            ld s = 0;
            for (int a = 0; a < 4; ++a) s += RmL[i * 4 + a] * G[a][q];
            K[i][q] = s;
        }
    for (int i = 0; i < NQ; ++i)
        for (int q = 0; q < NQ; ++q) {
            ld am = 0, ap = 0;
            for (int k = 0; k < NQ; ++k) {
                const ld a = SL.An[i * NQ + k];
                am += a * ((k == q ? 1.0L : 0.0L) - K[k][q]);
                ap += a * K[k][q];
            }
            Fm[i * NQ + q] = (double)am;
            if (interior) Fp[i * NQ + q] = (double)ap;
        }
    return true;
}

// ------------------------------------------------------------ basis at points
namespace {
// L^n P_n^(a,b)(x/L), homogeneous three-term recurrence (no division by L)
ld hjacobi(int n, int a, int b, ld x, ld L) {
    if (n == 0) return 1;
    ld p0 = 1, p1 = (a + 1) * L + (a + b + 2) * (x - L) / 2;
    for (int k = 1; k < n; ++k) {
        const ld c = 2.0L * k + a + b;
        const ld a1 = 2.0L * (k + 1) * (k + a + b + 1) * c;
        const ld p2 = ((c + 1) * ((c + 2) * c * x + ((ld)a * a - (ld)b * b) * L) * p1 -
                       2.0L * (k + a) * (k + b) * (c + 2) * L * L * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}
}  // namespace

void basis_at(int N, const double xi[3], double* phi) {
    const ld x = xi[0], y = xi[1], z = xi[2];
    const ld L = 1 - y - z, L2 = 1 - z;
    int l = 0;
    for (int g = 0; g <= N; ++g)
        for (int k = 0; k <= g; ++k)
            for (int j = 0; j <= g - k; ++j) {
                const int i = g - j - k;
                const ld v = hjacobi(i, 0, 0, 2 * x - L, L) * hjacobi(j, 2 * i + 1, 0, 2 * y - L2, L2) *
                             hjacobi(k, 2 * i + 2 * j + 2, 0, 2 * z - 1, 1);
                phi[l++] = (double)v;
            }
}

// ------------------------------------------------------------ face matrices
namespace {
const double REFV[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

void face_vertices(int f, int v[3]) {
    int n = 0;
    for (int k = 0; k < 4; ++k)
        if (k != f) v[n++] = k;
}

// point of reference face f with face barycentrics (l0, l1, l2) on its
// vertices in increasing local order
void face_point(int f, const double lam[3], double xi[3]) {
    int v[3];
    face_vertices(f, v);
    for (int d = 0; d < 3; ++d) xi[d] = lam[0] * REFV[v[0]][d] + lam[1] * REFV[v[1]][d] + lam[2] * REFV[v[2]][d];
}

// triangle rule: collapsed Gauss-Legendre with N + 3 points per direction
void triangle_rule(int N, std::vector<double>& a, std::vector<double>& b, std::vector<double>& w) {
    const int n = N + 3;
    std::vector<long double> x(n), wx(n);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = std::cos(pi * (i + 0.75L) / (n + 0.5L));
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            long double dp = n * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-19L) {
                x[i] = z;
                wx[i] = 2 / ((1 - z * z) * dp * dp);
                break;
            }
        }
    }
    a.clear();
    b.clear();
    w.clear();
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            a.push_back((double)((1 + x[i]) * (1 - x[j]) / 4));
            b.push_back((double)((1 + x[j]) / 2));
            w.push_back((double)(wx[i] * wx[j] * (1 - x[j]) / 8));
        }
}
}  // namespace

// Face trace operators.  With {psi_a} orthonormal on the reference triangle
// under the quadrature weights (d_f = (N+1)(N+2)/2 functions, from the
// Cholesky factor of the monomial Gram matrix), the trace of every basis
// function on a face is a polynomial of degree <= N in the face parameters, so
//   phi_k(chi_f(t)) = sum_a Pf[f][a][k] psi_a(t)   exactly, and
//   Floc[f] = Pf[f]^T Pf[f],  Fnb[f,h,s] = Pf[f]^T Pnb[f,h,s]
// with Pnb the neighbour's trace seen in this face's parameters.
void face_traces(int N, std::vector<double>& Pf, std::vector<double>& Pnb) {
    const int B = n_modes(N), df = (N + 1) * (N + 2) / 2;
    std::vector<double> qa, qb, qw;
    triangle_rule(N, qa, qb, qw);
    const int nq = (int)qw.size();
    // psi at the quadrature points: [nq][df]; the starting functions are the
    // collapsed-coordinate (Dubiner) polynomials of the triangle, already
    // orthogonal, so the Cholesky step only normalises them
    std::vector<long double> m((size_t)nq * df), G((size_t)df * df, 0.0L), Lc((size_t)df * df, 0.0L);
    for (int q = 0; q < nq; ++q) {
        int i = 0;
        const long double a = qa[q], b = qb[q];
        for (int g = 0; g <= N; ++g)
            for (int e = 0; e <= g; ++e) {
                const int ii = g - e, jj = e;
                m[(size_t)q * df + i++] = hjacobi(ii, 0, 0, 2 * a - (1 - b), 1 - b) * hjacobi(jj, 2 * ii + 1, 0, 2 * b - 1, 1);
            }
    }
    for (int q = 0; q < nq; ++q)
        for (int i = 0; i < df; ++i)
            for (int j = 0; j < df; ++j) G[i * df + j] += qw[q] * m[(size_t)q * df + i] * m[(size_t)q * df + j];
    for (int j = 0; j < df; ++j) {
        long double d = G[j * df + j];
        for (int k = 0; k < j; ++k) d -= Lc[j * df + k] * Lc[j * df + k];
        Lc[j * df + j] = std::sqrt(d);
        for (int i = j + 1; i < df; ++i) {
            long double v = G[i * df + j];
            for (int k = 0; k < j; ++k) v -= Lc[i * df + k] * Lc[j * df + k];
            Lc[i * df + j] = v / Lc[j * df + j];
        }
    }
    std::vector<long double> psi((size_t)nq * df);
    for (int q = 0; q < nq; ++q)
        for (int i = 0; i < df; ++i) {
            long double v = m[(size_t)q * df + i];
            for (int k = 0; k < i; ++k) v -= Lc[i * df + k] * psi[(size_t)q * df + k];
            psi[(size_t)q * df + i] = v / Lc[i * df + i];
        }
    std::vector<long double> acc((size_t)4 * df * B, 0.0L), accn((size_t)96 * df * B, 0.0L);
    std::vector<double> ph(B);
    for (int q = 0; q < nq; ++q) {
        const double lam[3] = {1 - qa[q] - qb[q], qa[q], qb[q]};
        for (int f = 0; f < 4; ++f) {
            double xi[3];
            face_point(f, lam, xi);
            basis_at(N, xi, ph.data());
            for (int a = 0; a < df; ++a) {
                const long double c = qw[q] * psi[(size_t)q * df + a];
                for (int k = 0; k < B; ++k) acc[((size_t)f * df + a) * B + k] += c * ph[k];
            }
            for (int h = 0; h < 4; ++h)
                for (int s = 0; s < 6; ++s) {
                    double mu[3];
                    for (int i = 0; i < 3; ++i) mu[PERM[s][i]] = lam[i];
                    double xr[3];
                    face_point(h, mu, xr);
                    basis_at(N, xr, ph.data());
                    const size_t t = ((size_t)f * 4 + h) * 6 + s;
                    for (int a = 0; a < df; ++a) {
                        const long double c = qw[q] * psi[(size_t)q * df + a];
                        for (int l = 0; l < B; ++l) accn[(t * df + a) * B + l] += c * ph[l];
                    }
                }
        }
    }
    Pf.assign(acc.begin(), acc.end());
    Pnb.assign(accn.begin(), accn.end());
}

void face_matrices(int N, std::vector<double>& Floc, std::vector<double>& Fnb) {
    const int B = n_modes(N);
    std::vector<double> qa, qb, qw;
    triangle_rule(N, qa, qb, qw);
    const int nq = (int)qw.size();
    Floc.assign((size_t)4 * B * B, 0.0);
    Fnb.assign((size_t)4 * 4 * 6 * B * B, 0.0);
    std::vector<double> phL(B), phR(B);
    for (int q = 0; q < nq; ++q) {
        const double lam[3] = {1 - qa[q] - qb[q], qa[q], qb[q]};
        for (int f = 0; f < 4; ++f) {
            double xi[3];
            face_point(f, lam, xi);
            basis_at(N, xi, phL.data());
            double* Fl = Floc.data() + (size_t)f * B * B;
            for (int k = 0; k < B; ++k)
                for (int l = 0; l < B; ++l) Fl[k * B + l] += qw[q] * phL[k] * phL[l];
            for (int h = 0; h < 4; ++h)
                for (int s = 0; s < 6; ++s) {
                    // local face vertex i sits on neighbour face vertex PERM[s][i]
                    double mu[3];
                    for (int i = 0; i < 3; ++i) mu[PERM[s][i]] = lam[i];
                    double xr[3];
                    face_point(h, mu, xr);
                    basis_at(N, xr, phR.data());
                    double* Fn = Fnb.data() + (((size_t)f * 4 + h) * 6 + s) * B * B;
                    for (int k = 0; k < B; ++k)
                        for (int l = 0; l < B; ++l) Fn[k * B + l] += qw[q] * phL[k] * phR[l];
                }
        }
    }
}

int face_permutation_index(const int p[3]) {
    for (int s = 0; s < 6; ++s)
        if (PERM[s][0] == p[0] && PERM[s][1] == p[1] && PERM[s][2] == p[2]) return s;
    return -1;
}

}  // namespace poro
