// Host set-up of libporoader: Biot Jacobians, reference matrices of the
// Dubiner basis, time matrices, element geometry and per-element constants.
//
// Independent route from any test reference: the spatial matrices are
// integrated numerically with a collapsed (Duffy) Gauss-Legendre product rule
// of N+2 points per direction, exact for the polynomial integrands; basis
// values and derivatives are evaluated through the collapsed coordinates with
// Jacobi three-term recurrences.
#include <cmath>
#include <cstring>
#include <limits>
#include <string>

#include "poro_internal.h"

namespace poro {

// ------------------------------------------------------------ materials
// Section "Governing equations": constitutive law and Eq. biot-dynamic.
// Rates of (sigma, p) are linear in the velocity gradients; rates of the
// velocities follow from the Biot mass matrix [[rho, rho_F], [rho_F, m]],
// m = rho_F T / phi, applied to (div sigma, -grad p - b v^F), b = nu/kappa.
namespace {
struct Biot {
    double rho, lam_c, mu, M, alpha, m, D, b, rho_F;
};

bool biot_constants(const poro_material& p, Biot& c, std::string& err) {
    const double vals[10] = {p.K_S, p.rho_S, p.lambda_M, p.mu_M, p.kappa,
                             p.phi, p.tortuosity, p.K_F, p.rho_F, p.nu};
    for (double v : vals)
        if (!std::isfinite(v)) { err = "material: non-finite parameter"; return false; }
    if (!(p.phi > 0.0 && p.phi < 1.0)) { err = "material: porosity outside (0,1)"; return false; }
    if (p.nu < 0.0) { err = "material: negative viscosity"; return false; }
    if (p.nu > 0.0 && !(p.kappa > 0.0)) { err = "material: kappa <= 0 with viscous fluid"; return false; }
    if (!(p.mu_M > 0.0 && p.K_S > 0.0 && p.K_F > 0.0 && p.rho_S > 0.0 && p.rho_F > 0.0 &&
          p.tortuosity > 0.0)) {
        err = "material: non-positive modulus, density or tortuosity";
        return false;
    }
    const double K_M = p.lambda_M + 2.0 * p.mu_M / 3.0;
    c.alpha = 1.0 - K_M / p.K_S;
    c.M = p.K_S / ((1.0 - K_M / p.K_S) - p.phi * (1.0 - p.K_S / p.K_F));
    c.rho = p.phi * p.rho_F + (1.0 - p.phi) * p.rho_S;
    c.lam_c = p.lambda_M + c.M * c.alpha * c.alpha;
    c.mu = p.mu_M;
    c.m = p.rho_F * p.tortuosity / p.phi;
    c.D = c.rho * c.m - p.rho_F * p.rho_F;
    c.b = p.nu > 0.0 ? p.nu / p.kappa : 0.0;
    c.rho_F = p.rho_F;
    if (!(c.M > 0.0)) { err = "material: coupling modulus M <= 0"; return false; }
    if (!(c.D > 0.0)) { err = "material: Biot mass matrix not positive definite"; return false; }
    return true;
}

// symmetric stress index of (k, l)
int sig(int k, int l) {
    if (k == l) return k;  // SXX, SYY, SZZ
    int a = k < l ? k : l, b = k < l ? l : k;
    if (a == 0 && b == 1) return SXY;
    if (a == 1 && b == 2) return SYZ;
    return SXZ;
}
}  // namespace

bool material_jacobians(const poro_material& mat, double abc[3][NQ][NQ], double e[NQ][NQ],
                        std::string& err) {
    Biot c;
    if (!biot_constants(mat, c, err)) return false;
    std::memset(abc, 0, sizeof(double) * 3 * NQ * NQ);
    std::memset(e, 0, sizeof(double) * NQ * NQ);
    // inverse Biot mass matrix
    const double mi00 = c.m / c.D, mi01 = -c.rho_F / c.D, mi11 = c.rho / c.D;
    for (int d = 0; d < 3; ++d) {
        auto& A = abc[d];
        // d/dt sigma_kl = lam_c d_kl div v + mu (d_k v_l + d_l v_k) + M alpha d_kl div vF
        for (int k = 0; k < 3; ++k)
            for (int l = k; l < 3; ++l)
                for (int m = 0; m < 3; ++m) {
                    double cv = (k == l && d == m ? c.lam_c : 0.0) +
                                c.mu * ((k == d && l == m ? 1.0 : 0.0) + (l == d && k == m ? 1.0 : 0.0));
                    double cf = (k == l && d == m) ? c.M * c.alpha : 0.0;
                    if (cv != 0.0) A[sig(k, l)][QU + m] -= cv;
                    if (cf != 0.0) A[sig(k, l)][QUF + m] -= cf;
                }
        // d/dt p = -M alpha div v - M div vF
        A[QP][QU + d] += c.M * c.alpha;
        A[QP][QUF + d] += c.M;
        // [v; vF]_t = Minv [(div sigma)_m; -d_m p]
        for (int m = 0; m < 3; ++m) {
            A[QU + m][sig(m, d)] -= mi00;
            A[QUF + m][sig(m, d)] -= mi01;
        }
        A[QU + d][QP] += mi01;
        A[QUF + d][QP] += mi11;
    }
    // source: -b vF in the fluid momentum balance
    for (int m = 0; m < 3; ++m) {
        e[QU + m][QUF + m] = -mi01 * c.b;
        e[QUF + m][QUF + m] = -mi11 * c.b;
    }
    return true;
}

bool max_wave_speed(const poro_material& mat, double& v, std::string& err) {
    // Biot's P-wave dispersion relation (inviscid limit, which bounds the
    // characteristic speeds of the hyperbolic part):
    // det [[H - rho c^2, C - rho_F c^2], [C - rho_F c^2, M - m c^2]] = 0
    Biot c;
    if (!biot_constants(mat, c, err)) return false;
    const double H = c.lam_c + 2.0 * c.mu, C = c.alpha * c.M;
    const double a = c.rho * c.m - c.rho_F * c.rho_F;
    const double b = -(H * c.m + c.rho * c.M - 2.0 * C * c.rho_F);
    const double cc = H * c.M - C * C;
    const double disc = b * b - 4.0 * a * cc;
    if (!(disc >= 0.0)) { err = "material: complex wave speeds"; return false; }
    const double x = (-b + std::sqrt(disc)) / (2.0 * a);
    v = std::sqrt(x);
    return std::isfinite(v) && v > 0.0;
}

// ------------------------------------------------------------ quadrature
namespace {
// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration.
void gauss_legendre(int n, std::vector<long double>& x, std::vector<long double>& w) {
    x.assign(n, 0.0L);
    w.assign(n, 0.0L);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double z = std::cos(pi * (i + 0.75L) / (n + 0.5L)), dp = 0.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0L; }
            dp = n * (z * p1 - p0) / (z * z - 1.0L);
            long double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-19L) break;
        }
        long double p0 = 1.0L, p1 = z;
        for (int k = 2; k <= n; ++k) {
            long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0L; }
        dp = n * (z * p1 - p0) / (z * z - 1.0L);
        x[i] = z;
        w[i] = 2.0L / ((1.0L - z * z) * dp * dp);
    }
}

// Jacobi polynomial P_n^(a,b)(x) by the three-term recurrence.
long double jacobi(int n, int a, int b, long double x) {
    if (n == 0) return 1.0L;
    long double p0 = 1.0L, p1 = (a + 1) + (a + b + 2) * (x - 1.0L) / 2.0L;
    for (int k = 1; k < n; ++k) {
        long double c = 2.0L * k + a + b;
        long double a1 = 2.0L * (k + 1) * (k + a + b + 1) * c;
        long double a2 = (c + 1) * ((c + 2) * c * x + (long double)a * a - (long double)b * b);
        long double a3 = 2.0L * (k + a) * (k + b) * (c + 2);
        long double p2 = (a2 * p1 - a3 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

long double jacobi_d(int n, int a, int b, long double x) {
    if (n == 0) return 0.0L;
    return 0.5L * (n + a + b + 1) * jacobi(n - 1, a + 1, b + 1, x);
}

long double ipow(long double x, int k) {
    long double r = 1.0L;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

// value and reference-coordinate gradient of phi_ijk at collapsed (r, s, t)
void dubiner(int i, int j, int k, long double r, long double s, long double t, long double& val,
             long double grad[3]) {
    const long double f = jacobi(i, 0, 0, r), fr = jacobi_d(i, 0, 0, r);
    const long double hs = (1.0L - s) / 2.0L, ht = (1.0L - t) / 2.0L;
    const long double Pj = jacobi(j, 2 * i + 1, 0, s), dPj = jacobi_d(j, 2 * i + 1, 0, s);
    const long double Pk = jacobi(k, 2 * i + 2 * j + 2, 0, t), dPk = jacobi_d(k, 2 * i + 2 * j + 2, 0, t);
    const long double g = ipow(hs, i) * Pj;
    const long double gs = (i > 0 ? -0.5L * i * ipow(hs, i - 1) * Pj : 0.0L) + ipow(hs, i) * dPj;
    const long double h = ipow(ht, i + j) * Pk;
    const long double ht_ = (i + j > 0 ? -0.5L * (i + j) * ipow(ht, i + j - 1) * Pk : 0.0L) +
                            ipow(ht, i + j) * dPk;
    val = f * g * h;
    const long double om = (1.0L - s) * (1.0L - t);
    grad[0] = fr * g * h * 8.0L / om;
    grad[1] = fr * g * h * 4.0L * (1.0L + r) / om + f * gs * h * 4.0L / (1.0L - t);
    grad[2] = fr * g * h * 4.0L * (1.0L + r) / om + f * gs * h * 2.0L * (1.0L + s) / (1.0L - t) +
              f * g * ht_ * 2.0L;
}
}  // namespace

bool invert_small(int n, const double* a, double* ainv) {
    // Gauss-Jordan with partial pivoting in extended precision
    std::vector<long double> m(2 * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            m[i * 2 * n + j] = a[i * n + j];
            m[i * 2 * n + n + j] = (i == j) ? 1.0L : 0.0L;
        }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(m[r * 2 * n + c]) > std::fabs(m[piv * 2 * n + c])) piv = r;
        if (m[piv * 2 * n + c] == 0.0L) return false;
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) std::swap(m[c * 2 * n + j], m[piv * 2 * n + j]);
        long double d = m[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) m[c * 2 * n + j] /= d;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                long double f = m[r * 2 * n + c];
                if (f != 0.0L)
                    for (int j = 0; j < 2 * n; ++j) m[r * 2 * n + j] -= f * m[c * 2 * n + j];
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) ainv[i * n + j] = (double)m[i * 2 * n + n + j];
    return true;
}

bool reference_data(int N, ReferenceData& R, std::string& err) {
    if (N < 1 || N > MAX_N) { err = "degree N outside 1..6"; return false; }
    R.N = N;
    R.B = n_modes(N);
    R.T = N + 1;
    const int B = R.B, T = R.T;
    // basis index -> (i, j, k): degree g, then k, then j ascending
    std::vector<int> ti, tj, tk;
    for (int g = 0; g <= N; ++g)
        for (int k = 0; k <= g; ++k)
            for (int j = 0; j <= g - k; ++j) {
                ti.push_back(g - j - k);
                tj.push_back(j);
                tk.push_back(k);
            }
    std::vector<long double> xg, wg;
    gauss_legendre(N + 2, xg, wg);
    const int nq = N + 2;
    std::vector<long double> M(B, 0.0L), K(3 * B * B, 0.0L);
    std::vector<long double> val(B), grad(3 * B);
    for (int a = 0; a < nq; ++a)
        for (int b = 0; b < nq; ++b)
            for (int c = 0; c < nq; ++c) {
                const long double r = xg[a], s = xg[b], t = xg[c];
                const long double w = wg[a] * wg[b] * wg[c] * (1.0L - s) * (1.0L - t) * (1.0L - t) / 64.0L;
                for (int l = 0; l < B; ++l) dubiner(ti[l], tj[l], tk[l], r, s, t, val[l], &grad[3 * l]);
                for (int k = 0; k < B; ++k) {
                    M[k] += w * val[k] * val[k];
                    for (int l = 0; l < B; ++l)
                        for (int d = 0; d < 3; ++d) K[(d * B + k) * B + l] += w * val[k] * grad[3 * l + d];
                }
            }
    R.mass_diag.resize(B);
    R.khat.assign(3 * B * B, 0.0);
    long double kmax = 0.0L;
    for (int i = 0; i < 3 * B * B; ++i) kmax = std::max(kmax, std::fabs(K[i]));
    for (int k = 0; k < B; ++k) R.mass_diag[k] = (double)M[k];
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < B; ++k)
            for (int l = 0; l < B; ++l) {
                long double v = K[(d * B + k) * B + l];
                // entries at the rounding level of the quadrature are exact
                // zeros of the basis (orthogonality); the smallest true
                // non-zero of K is ~1e-5 of the largest
                if (std::fabs(v) <= 1e-13L * kmax) v = 0.0L;
                R.khat[(d * B + k) * B + l] = (double)(v / M[k]);
            }
    // time matrices of the shifted Legendre basis (closed forms):
    // W_rs = 1, w_r = (-1)^r, S = diag(1/(2r+1)), K^tau_rs = 2 for r > s, r-s odd
    R.z.assign(T * T, 0.0);
    R.sinv_w.assign(T, 0.0);
    for (int u = 0; u < T; ++u) {
        R.sinv_w[u] = (2 * u + 1) * ((u % 2) ? -1.0 : 1.0);
        for (int s = 0; s < T; ++s) {
            double kt = (u > s && ((u - s) % 2 == 1)) ? 2.0 : 0.0;
            R.z[u * T + s] = (2 * u + 1) * (1.0 - kt);
        }
    }
    R.zinv.assign(T * T, 0.0);
    if (!invert_small(T, R.z.data(), R.zinv.data())) { err = "Z singular"; return false; }
    // CSR of Khat^j restricted to each degree block's columns
    R.blocks.assign((N + 1) * 3, KhatBlockCSR());
    R.khat_block_nnz = 0;
    for (int g = 1; g <= N; ++g) {
        const int o = block_offset(g), d = block_size(g);
        for (int j = 0; j < 3; ++j) {
            KhatBlockCSR& C = R.blocks[g * 3 + j];
            C.row_ptr.assign(1, 0);
            for (int l = 0; l < o; ++l) {
                for (int m = 0; m < d; ++m) {
                    double v = R.khat[(j * B + l) * B + o + m];
                    if (v != 0.0) {
                        C.col.push_back(m);
                        C.val.push_back(v);
                    }
                }
                C.row_ptr.push_back((int32_t)C.col.size());
            }
            R.khat_block_nnz += (int64_t)C.col.size();
        }
    }
    return true;
}

// ------------------------------------------------------------ geometry
bool tet_geometry(const double* v, double jinv[3][3], double& volume, double& insphere_d,
                  std::string& err) {
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(v[i])) { err = "element: non-finite vertex"; return false; }
    double J[3][3];
    for (int d = 0; d < 3; ++d)
        for (int c = 0; c < 3; ++c) J[d][c] = v[3 * (c + 1) + d] - v[d];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double scale = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int c = 0; c < 3; ++c) scale = std::max(scale, std::fabs(J[d][c]));
    if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) { err = "element: degenerate tetrahedron"; return false; }
    // inverse by cofactors: jinv[j][d] = d xi_j / d x_d
    jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    volume = std::fabs(det) / 6.0;
    double area = 0.0;
    for (int f = 0; f < 4; ++f) {
        int idx[3], n = 0;
        for (int k = 0; k < 4; ++k)
            if (k != f) idx[n++] = k;
        double a[3], b[3];
        for (int d = 0; d < 3; ++d) {
            a[d] = v[3 * idx[1] + d] - v[3 * idx[0] + d];
            b[d] = v[3 * idx[2] + d] - v[3 * idx[0] + d];
        }
        double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
        area += 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    insphere_d = 6.0 * volume / area;
    return true;
}

bool element_constants(const ReferenceData& ref, const double* v12, const poro_material& mat,
                       double dt, double* out, std::string& err) {
    if (!(dt > 0.0) || !std::isfinite(dt)) { err = "element: time step must be positive"; return false; }
    double jinv[3][3], vol, dins;
    if (!tet_geometry(v12, jinv, vol, dins, err)) return false;
    double abc[3][NQ][NQ], E[NQ][NQ];
    if (!material_jacobians(mat, abc, E, err)) return false;
    const int T = ref.T;
    const int stride = elem_const_stride(ref.N);
    std::memset(out, 0, sizeof(double) * stride);
    for (int j = 0; j < 3; ++j)
        for (int p = 0; p < NQ; ++p)
            for (int n = star_row_ptr(p); n < star_row_ptr(p + 1); ++n) {
                const int q = star_col(n);
                double s = 0.0;
                for (int d = 0; d < 3; ++d) s += jinv[j][d] * abc[d][p][q];
                out[j * STAR_NNZ + n] = dt * s;
            }
    const double e = dt * E[QUF][QUF], g = dt * E[QU][QUF];
    std::vector<double> zm(ref.z);
    for (int u = 0; u < T; ++u) zm[u * T + u] -= e;
    if (!invert_small(T, zm.data(), out + ec_zinv(ref.N))) { err = "element: singular time block"; return false; }
    double* sc = out + ec_scalars(ref.N);
    sc[0] = e;
    sc[1] = g;
    sc[2] = dt;
    return true;
}

// Damped Maxwell (Section "Other applications"): the Jacobians of
// q_t + A q_x + B q_y + C q_z = E q with q = (E_x, E_y, E_z, H_x, H_y, H_z),
// eps E_t = curl H - sigma E and mu H_t = -curl E.  M[d][p][q] is the
// coefficient of d_d q_q in the equation of q_p moved to the left side.
static void maxwell_jacobians(double eps, double mu, double M[3][6][6]) {
    std::memset(M, 0, sizeof(double) * 3 * 36);
    const double ie = 1.0 / eps, im = 1.0 / mu;
    // E_x: -(1/eps)(d_y H_z - d_z H_y), E_y: -(1/eps)(d_z H_x - d_x H_z), E_z: -(1/eps)(d_x H_y - d_y H_x)
    M[1][0][5] = -ie; M[2][0][4] = ie;
    M[2][1][3] = -ie; M[0][1][5] = ie;
    M[0][2][4] = -ie; M[1][2][3] = ie;
    // H: +(1/mu) curl E
    M[1][3][2] = im; M[2][3][1] = -im;
    M[2][4][0] = im; M[0][4][2] = -im;
    M[0][5][1] = im; M[1][5][0] = -im;
}

bool maxwell_element_constants(const ReferenceData& ref, const double* v12, const double mat[3], double dt,
                               double* out, std::string& err) {
    if (!(dt > 0.0) || !std::isfinite(dt)) { err = "element: time step must be positive"; return false; }
    const double eps = mat[0], mu = mat[1], sigma = mat[2];
    if (!(eps > 0.0) || !(mu > 0.0) || !(sigma >= 0.0) || !std::isfinite(eps) || !std::isfinite(mu) ||
        !std::isfinite(sigma)) {
        err = "element: need eps > 0, mu > 0, sigma >= 0";
        return false;
    }
    double jinv[3][3], vol, dins;
    if (!tet_geometry(v12, jinv, vol, dins, err)) return false;
    double M[3][6][6];
    maxwell_jacobians(eps, mu, M);
    const int T = ref.T;
    std::memset(out, 0, sizeof(double) * maxwell::elem_const_stride(ref.N));
    for (int j = 0; j < 3; ++j)
        for (int n = 0; n < maxwell::STAR_NNZ; ++n) {
            const int p = maxwell::star_row(n), q = maxwell::star_col(n);
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += jinv[j][d] * M[d][p][q];
            out[j * maxwell::STAR_NNZ + n] = dt * s;
        }
    const double e = -dt * sigma / eps;
    std::vector<double> zm(ref.z);
    for (int u = 0; u < T; ++u) zm[u * T + u] -= e;
    double* zi = out + 3 * maxwell::STAR_NNZ;
    if (!invert_small(T, zm.data(), zi)) { err = "element: singular time block"; return false; }
    double* sc = zi + T * T;
    sc[0] = e;
    sc[1] = 0.0;
    sc[2] = dt;
    return true;
}

// Reference Jacobians of the viscoelastic system (the form of q_t + A q_x +
// B q_y + C q_z = E q): sigma_ii,t = lam_u div v + 2 mu_u d_i v_i, sigma_ab,t =
// mu_u (d_b v_a + d_a v_b), rho v_i,t = sum_d d_d sigma_id, th_ii,t = omega
// d_i v_i, th_ab,t = omega (d_b v_a + d_a v_b) / 2 (plus the source terms).
static void visco_jacobians(const double* mat, double M[3][visco::NQ][visco::NQ]) {
    std::memset(M, 0, sizeof(double) * 3 * visco::NQ * visco::NQ);
    const double rho = mat[0], lam = mat[1], mu = mat[2];
    const int vel[3] = {6, 7, 8};
    const int shear[3][3] = {{3, 0, 1}, {4, 1, 2}, {5, 0, 2}};  // component, a, b
    const int sig[3][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}};
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) M[d][i][vel[d]] = -(d == i ? lam + 2.0 * mu : lam);
    for (const auto& sh : shear) {
        M[sh[2]][sh[0]][vel[sh[1]]] = -mu;
        M[sh[1]][sh[0]][vel[sh[2]]] = -mu;
    }
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) M[d][vel[i]][sig[i][d]] = -1.0 / rho;
    for (int l = 0; l < visco::NMECH; ++l) {
        const double w = mat[3 + l];
        const int base = 9 + 6 * l;
        for (int i = 0; i < 3; ++i) M[i][base + i][vel[i]] = -w;
        for (const auto& sh : shear) {
            M[sh[2]][base + sh[0]][vel[sh[1]]] = -0.5 * w;
            M[sh[1]][base + sh[0]][vel[sh[2]]] = -0.5 * w;
        }
    }
}

bool visco_element_constants(const ReferenceData& ref, const double* v12, const double mat[12], double dt,
                             double* out, std::string& err) {
    if (!(dt > 0.0) || !std::isfinite(dt)) { err = "element: time step must be positive"; return false; }
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(mat[i])) { err = "element: non-finite material parameter"; return false; }
    if (!(mat[0] > 0.0) || !(mat[2] > 0.0) || !(mat[1] + 2.0 * mat[2] / 3.0 > 0.0)) {
        err = "element: need rho > 0, mu_u > 0 and a positive unrelaxed bulk modulus";
        return false;
    }
    for (int l = 0; l < visco::NMECH; ++l)
        if (!(mat[3 + l] >= 0.0)) { err = "element: relaxation frequencies must be >= 0"; return false; }
    double jinv[3][3], vol, dins;
    if (!tet_geometry(v12, jinv, vol, dins, err)) return false;
    static thread_local double M[3][visco::NQ][visco::NQ];
    visco_jacobians(mat, M);
    const int T = ref.T;
    std::memset(out, 0, sizeof(double) * visco::elem_const_stride(ref.N));
    for (int j = 0; j < 3; ++j)
        for (int n = 0; n < visco::STAR_NNZ; ++n) {
            const int p = visco::star_row(n), q = visco::star_col(n);
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += jinv[j][d] * M[d][p][q];
            out[j * visco::STAR_NNZ + n] = dt * s;
        }
    double* zi = out + 3 * visco::STAR_NNZ;
    double* sc = zi + visco::NMECH * T * T;
    for (int l = 0; l < visco::NMECH; ++l) {
        const double e = -dt * mat[3 + l];
        std::vector<double> zm(ref.z);
        for (int u = 0; u < T; ++u) zm[u * T + u] -= e;
        if (!invert_small(T, zm.data(), zi + l * T * T)) { err = "element: singular time block"; return false; }
        const double ylam = mat[6 + l], ymu = mat[9 + l];
        sc[3 * l + 0] = -dt * (ylam + 2.0 * ymu);
        sc[3 * l + 1] = -dt * ylam;
        sc[3 * l + 2] = -dt * 2.0 * ymu;
        sc[3 * visco::NMECH + l] = e;
    }
    sc[visco::sc_dt()] = dt;
    return true;
}

// ------------------------------------------------------------ sub-cell material
// Section "Limitations": with Jacobians and source matrix that vary linearly
// inside the element, the stiffness becomes the 3-tensor
// int phi_k phi_r d_j phi_l = (M3_r Khat^j)[k, l] (d_j phi_l lies in the
// basis) with the mass 3-tensor M3_r[k, l] = int phi_k phi_r phi_l, r < 4.
bool subcell_mass_tensors(const ReferenceData& R, std::vector<int32_t>& row, std::vector<int32_t>& col,
                          std::vector<double>& val, std::string& err) {
    const int N = R.N, B = R.B;
    if (B < 4) { err = "sub-cell material needs N >= 1"; return false; }
    std::vector<int> ti, tj, tk;
    for (int g = 0; g <= N; ++g)
        for (int k = 0; k <= g; ++k)
            for (int j = 0; j <= g - k; ++j) {
                ti.push_back(g - j - k);
                tj.push_back(j);
                tk.push_back(k);
            }
    // integrands of degree <= 2N + 1, times the collapsed weight: N + 3 points
    std::vector<long double> xg, wg;
    gauss_legendre(N + 3, xg, wg);
    const int nq = N + 3;
    std::vector<long double> T3(3 * (size_t)B * B, 0.0L), val_q(B), grad(3 * B);
    for (int a = 0; a < nq; ++a)
        for (int b = 0; b < nq; ++b)
            for (int c = 0; c < nq; ++c) {
                const long double r = xg[a], s = xg[b], t = xg[c];
                const long double w = wg[a] * wg[b] * wg[c] * (1.0L - s) * (1.0L - t) * (1.0L - t) / 64.0L;
                for (int l = 0; l < B; ++l) dubiner(ti[l], tj[l], tk[l], r, s, t, val_q[l], &grad[3 * l]);
                for (int m = 1; m < 4; ++m)
                    for (int k = 0; k < B; ++k) {
                        const long double wk = w * val_q[k] * val_q[m];
                        for (int l = 0; l < B; ++l) T3[((size_t)(m - 1) * B + k) * B + l] += wk * val_q[l];
                    }
            }
    long double tmax = 0.0L;
    for (long double v : T3) tmax = std::max(tmax, std::fabs(v));
    row.assign(3 * (size_t)(B + 1), 0);
    col.clear();
    val.clear();
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < B; ++k) {
            row[(size_t)m * (B + 1) + k] = (int32_t)col.size();
            for (int l = 0; l < B; ++l) {
                const long double v = T3[((size_t)m * B + k) * B + l];
                // exact zeros of the orthogonal basis sit at the rounding level
                if (std::fabs(v) <= 1e-13L * tmax) continue;
                col.push_back(l);
                val.push_back((double)(v / (long double)R.mass_diag[k]));
            }
            row[(size_t)m * (B + 1) + B] = (int32_t)col.size();
        }
    return true;
}

bool subcell_projection(double P[4][4], std::string& err) {
    const double verts[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double V[16], Pi[16];
    for (int v = 0; v < 4; ++v) basis_at(1, verts[v], V + 4 * v);  // V[v][r] = phi_r(vertex v)
    if (!invert_small(4, V, Pi)) { err = "sub-cell projection singular"; return false; }
    for (int r = 0; r < 4; ++r)
        for (int v = 0; v < 4; ++v) P[r][v] = Pi[r * 4 + v];
    return true;
}

bool subcell_element_constants(const ReferenceData& ref, const double P[4][4], const double* v12,
                               const poro_material mats[4], double dt, double* mean_out, double* var_out,
                               std::string& err) {
    if (!(dt > 0.0) || !std::isfinite(dt)) { err = "element: time step must be positive"; return false; }
    double jinv[3][3], vol, dins;
    if (!tet_geometry(v12, jinv, vol, dins, err)) return false;
    static thread_local double abc[4][3][NQ][NQ], E[4][NQ][NQ];
    for (int v = 0; v < 4; ++v)
        if (!material_jacobians(mats[v], abc[v], E[v], err)) {
            err = "vertex " + std::to_string(v) + ": " + err;
            return false;
        }
    const int T = ref.T;
    std::memset(mean_out, 0, sizeof(double) * elem_const_stride(ref.N));
    std::memset(var_out, 0, sizeof(double) * subcell_var_stride());
    double e[4], g[4];
    for (int r = 0; r < 4; ++r) {
        double* star = r == 0 ? mean_out : var_out + (r - 1) * 3 * STAR_NNZ;
        for (int j = 0; j < 3; ++j)
            for (int n = 0; n < STAR_NNZ; ++n) {
                const int p = star_row(n), q = star_col(n);
                double s = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double a = 0.0;
                    for (int v = 0; v < 4; ++v) a += P[r][v] * abc[v][d][p][q];
                    s += jinv[j][d] * a;
                }
                star[j * STAR_NNZ + n] = dt * s;
            }
        e[r] = g[r] = 0.0;
        for (int v = 0; v < 4; ++v) {
            e[r] += P[r][v] * E[v][QUF][QUF];
            g[r] += P[r][v] * E[v][QU][QUF];
        }
        e[r] *= dt;
        g[r] *= dt;
    }
    std::vector<double> zm(ref.z);
    for (int u = 0; u < T; ++u) zm[u * T + u] -= e[0];
    if (!invert_small(T, zm.data(), mean_out + ec_zinv(ref.N))) { err = "element: singular time block"; return false; }
    double* sc = mean_out + ec_scalars(ref.N);
    sc[0] = e[0];
    sc[1] = g[0];
    sc[2] = dt;
    for (int r = 1; r < 4; ++r) {
        var_out[3 * 3 * STAR_NNZ + 2 * (r - 1)] = e[r];
        var_out[3 * 3 * STAR_NNZ + 2 * (r - 1) + 1] = g[r];
    }
    return true;
}

}  // namespace poro
