/*
 * poroader.h -- C ABI of libporoader: the element-local space-time predictor
 * of ADER-DG for Biot's poroelastic equations on one NVIDIA GB300 (sm_103a).
 *
 * Paper: Wolf, Galis, Uphoff, Gabriel, Moczo, Gregor, Bader, "An Efficient
 * ADER-DG Local Time Stepping Scheme for 3D HPC Simulation of Seismic Waves
 * in Poroelastic Media" (arXiv 2108.10565).
 *
 * Conventions (all calls):
 *  - SI units.  Quantity order q = (s_xx, s_yy, s_zz, s_xy, s_yz, s_xz,
 *    u, v, w, p, u_f, v_f, w_f) (Section "Governing equations").
 *  - Degree N in 1..6; B = (N+1)(N+2)(N+3)/6 spatial modes, T = N+1 time
 *    modes.  Host arrays are row-major: DOFs [elem][13][B], predictor
 *    [elem][13][B][T], time-integrated DOFs [elem][13][B].
 *  - The spatial basis is the unnormalised Dubiner basis ordered by total
 *    degree g, then k, then j (phi_ijk, i = g - j - k); the time basis is the
 *    shifted Legendre family chi_s(tau) = P_s(2 tau - 1) on [0, 1].
 *  - Every call returns a poro_status; 0 is success, negative is an error.
 *    No call aborts or throws across the ABI.  poro_last_error() gives a
 *    text for the last failing call on that context.
 *  - Host pointers passed in are read during the call only (inputs are
 *    copied); the caller keeps ownership.  Output host buffers are written
 *    by the call and owned by the caller.  Device pointers passed to *_dev
 *    calls are neither copied nor freed by the library; they must stay valid
 *    until the work queued on the given stream has finished.
 *  - Work is queued asynchronously on a CUDA stream; device-side errors
 *    surface at the next synchronising call (poro_sync, poro_get_*).
 */
#ifndef PORO_ADER_H
#define PORO_ADER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t poro_status;
enum {
    PORO_OK = 0,
    PORO_EINVAL = -1,       /* bad argument: NULL, size, degenerate element, unphysical material */
    PORO_ENOMEM = -2,       /* device or host allocation failed */
    PORO_ECUDA = -3,        /* a CUDA runtime call or kernel failed */
    PORO_ETIMEOUT = -4,     /* poro_sync gave up waiting; the context stays usable */
    PORO_ESTATE = -5,       /* calls in the wrong order (e.g. predict before set_isolated) */
    PORO_ENUMERIC = -6,     /* non-finite value in input */
    PORO_EUNSUPPORTED = -7  /* degree outside 1..6, precision or solver not built */
};

typedef struct poro_ctx poro_ctx;

/* The 10 Biot parameters of Table poroelastic_parameters:
 * solid bulk modulus K_S [Pa], solid density rho_S [kg/m^3], matrix Lame
 * parameters lambda_M, mu_M [Pa], permeability kappa [m^2], porosity phi,
 * tortuosity T, fluid bulk modulus K_F [Pa], fluid density rho_F [kg/m^3],
 * fluid viscosity nu [Pa s].  Memory layout: 10 consecutive doubles. */
typedef struct {
    double K_S, rho_S, lambda_M, mu_M, kappa, phi, tortuosity, K_F, rho_F, nu;
} poro_material;

typedef enum {
    PORO_FP64 = 0,          /* every step in IEEE binary64 */
    PORO_FP32_REFINE = 1,   /* binary32 back-substitution + refinement against an
                               FP64-accurate residual of the predictor system */
    PORO_BF16X3_REFINE = 2  /* as PORO_FP32_REFINE with the tensor-core split products
                               in bf16 (hi + lo, ~16 significant bits per product);
                               one refinement sweep by default, as for FP32_REFINE */
} poro_precision;

typedef enum {
    PORO_FACE_INTERIOR = 0,     /* interior or periodic face (a neighbour is given) */
    PORO_FACE_FREE_SURFACE = 1, /* sigma n = 0, p = 0 (Section "Free surface") */
    PORO_FACE_ABSORBING = 2     /* no incoming waves (Section "Homogeneous full-space") */
} poro_face;

/* The linear hyperbolic system of a context.  Section "Other applications":
 * the predictor and Algorithm 3 apply to any such system whose source matrix
 * E is upper triangular; besides Biot's equations the library builds, for
 * the isolated-element predictor in binary64:
 *  - the damped Maxwell equations (eps E_t = curl H - sigma E, mu H_t =
 *    -curl E, quantities (E_x, E_y, E_z, H_x, H_y, H_z), E = diag(-sigma/eps
 *    x 3, 0 x 3));
 *  - viscoelastic attenuation with 3 relaxation mechanisms (anelastic
 *    functions th_l: sigma_t = lam_u tr(D) I + 2 mu_u D - sum_l (Ylam_l tr(th_l)
 *    I + 2 Ymu_l th_l), rho v_t = div sigma, th_l,t = omega_l (D - th_l), D the
 *    strain rate; 27 quantities: stresses xx yy zz xy yz xz, velocities u v w,
 *    then th_1, th_2, th_3 in the stress order; E upper triangular with
 *    -omega_l on th_l's diagonal). */
typedef enum {
    PORO_SYSTEM_BIOT = 0,         /* 13 quantities, the paper's poroelastic system */
    PORO_SYSTEM_MAXWELL = 1,      /* 6 quantities, damped Maxwell */
    PORO_SYSTEM_VISCOELASTIC = 2  /* 27 quantities, viscoelastic attenuation */
} poro_system;

typedef enum {
    PORO_SOLVE_BLOCK = 0,   /* Algorithm 3: degree-block back-substitution */
    PORO_SOLVE_LU = 1       /* dense LU of the whole predictor system (comparator) */
} poro_solver;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device` for degree `degree_N` (1..6) and
 * arithmetic `precision`.  Allocates a CUDA stream and the device-resident
 * reference matrices (Khat^alpha = M^{-1} K^alpha, Section "Block-wise
 * back-substitution"; Z = S^{-1}(W - K^tau)).  *out receives the handle, or
 * NULL on error.  Errors: PORO_EINVAL (out NULL), PORO_EUNSUPPORTED,
 * PORO_ECUDA, PORO_ENOMEM, and PORO_ENUMERIC for a mixed-precision context
 * whose Khat rows are not integer rows over a common denominator with a sum
 * of |numerators| below 2^22 (the exact integer residual needs that). */
poro_status poro_create(int device, int degree_N, poro_precision precision, poro_ctx** out);

/* poro_create for a given system.  PORO_SYSTEM_MAXWELL and
 * PORO_SYSTEM_VISCOELASTIC contexts support PORO_FP64 and the
 * isolated-element calls (poro_set_isolated_maxwell or
 * poro_set_isolated_viscoelastic, poro_set_dofs, poro_predict*,
 * poro_get_predictor, poro_get_integrated, poro_flop_count); DOF arrays then
 * have 6 or 27 quantities ([n][Q][B] and [n][Q][B][N+1]).  Meshes, the LU
 * comparator and the autotuner return PORO_EUNSUPPORTED on them.  Errors: as
 * poro_create, PORO_EUNSUPPORTED (unknown system, a mixed precision for a
 * system other than Biot's). */
poro_status poro_create_system(int device, int degree_N, poro_precision precision, poro_system system,
                               poro_ctx** out);

/* System and number of quantities of the context. */
poro_status poro_get_system(const poro_ctx* ctx, int32_t* system, int32_t* n_quantities);

/* Release every device and host resource of the context (waits for queued
 * work first).  NULL is accepted and ignored. */
poro_status poro_destroy(poro_ctx* ctx);

/* Text of the last error on `ctx`; owned by the context, valid until the
 * next call on it.  For ctx == NULL: the last error of a call that had no
 * context (e.g. a failed poro_create), thread-local. */
const char* poro_last_error(const poro_ctx* ctx);

/* Number of refinement sweeps of a mixed-precision context (0, 1 or 2;
 * default 1).  The binary32 solution is first rounded onto a fixed-point grid
 * per quantity (integers of at most 22 bits times a power of two set by the
 * quantity's largest entry).  Each sweep then forms the residual of the
 * predictor system for that solution, binary64-accurate:
 *   - the Khat and time-matrix products as exact integer sums;
 *   - the star, E* and coupling products in double-binary32 arithmetic
 *     (error-free products and sums, ~2^-48 relative).
 * It solves for the correction with the low-precision back-substitution.
 * The result is the rounded solution plus the corrections, in binary64.
 * Errors: PORO_EUNSUPPORTED for a PORO_FP64 context, PORO_EINVAL. */
poro_status poro_set_refinement(poro_ctx* ctx, int32_t sweeps);

/* Limit of the bounded waits of a mixed-precision context's predictor (the
 * tensor-core and bulk-copy completions of its low-precision sweeps), in SM
 * clock cycles; 0 restores the default (2e9 cycles, about 1 s).  The paper has
 * no counterpart: every wait in the library's kernels gives up after its
 * limit instead of spinning forever.  When a wait gives up, the CTA stops,
 * waits with the default limit for its own copies and MMAs still in flight,
 * frees its tensor memory and raises the context's device status; CTAs of the
 * context that start an element after that skip it.  The next synchronising
 * call (poro_sync, poro_get_*, poro_advance, poro_predict_host) then returns
 * PORO_ETIMEOUT once and clears the status; the context stays usable.  A
 * limit of 1 makes every wait that finds its operation unfinished give up at
 * once (tests use it to exercise that path).
 * Errors: PORO_EUNSUPPORTED for a PORO_FP64 context, PORO_EINVAL (negative). */
poro_status poro_set_wait_limit(poro_ctx* ctx, int64_t cycles);

/* Degree and precision the context was created with; n_elem after
 * poro_set_isolated (0 before). */
poro_status poro_get_info(const poro_ctx* ctx, int32_t* degree_N, int32_t* precision, int64_t* n_elem);

/* ------------------------------------------------------ host-only queries */
/* These touch no GPU; they expose the library's own set-up arithmetic. */

/* Reference matrices of degree N (Section "Space-Time predictor"):
 * mass_diag[B] = M_kk (M is diagonal), khat[3][B][B] = Khat^alpha_kl for
 * alpha = xi, eta, zeta (row-major).  Either pointer may be NULL. */
poro_status poro_reference_matrices(int degree_N, double* mass_diag, double* khat);

/* Jacobians of Eq. poroelastic-wave for one material: abc[3][13][13] holds
 * A, B, C; e[13][13] holds E.  Errors: PORO_EINVAL for an unphysical
 * material (phi outside (0,1), kappa <= 0 with nu > 0, M <= 0,
 * rho m - rho_F^2 <= 0, non-positive moduli or densities). */
poro_status poro_material_jacobians(const poro_material* mat, double* abc, double* e);

/* Largest characteristic speed of the material (fast P wave) [m/s]. */
poro_status poro_max_wave_speed(const poro_material* mat, double* speed);

/* CFL step of each element (Section "Temporal discretisation with ADER"):
 * dt[i] = cfl_c / (2N + 1) * d_i / v_i, d_i the insphere diameter of
 * tetrahedron i (vert[n][4][3]) and v_i the fast P speed of mat[i].
 * cfl_c = 0.5 in the paper.  Errors: PORO_EINVAL for a degenerate element. */
poro_status poro_cfl_dt(int degree_N, int64_t n, const double* vert, const poro_material* mat,
                        double cfl_c, double* dt);

/* poro_cfl_dt for a system's material rows (host): mat[n][3] (eps, mu, sigma)
 * for PORO_SYSTEM_MAXWELL with v = 1 / sqrt(eps mu), mat[n][12] (rho, lam_u,
 * mu_u, ...) for PORO_SYSTEM_VISCOELASTIC with the unrelaxed P speed
 * v = sqrt((lam_u + 2 mu_u) / rho), poro_material rows for PORO_SYSTEM_BIOT.
 * Errors: PORO_EINVAL (degenerate element or material), PORO_EUNSUPPORTED. */
poro_status poro_cfl_dt_system(poro_system system, int degree_N, int64_t n, const double* vert,
                               const double* mat, double cfl_c, double* dt);

/* ------------------------------------------------------ isolated elements */

/* Load n_elem unconnected tetrahedra (the population of the paper's
 * performance proxy, Section "Roofline model"): vertices vert[n][4][3],
 * one material per element, one time step dt[n] per element.  Computes on
 * the host, per element, the reference Jacobians A^{j*} = dt A^j (Section
 * "Space-Time predictor"), E* = dt E, and (Z - E*_pp I)^{-1}, and uploads
 * them.  Replaces a previous population.  Errors: PORO_EINVAL (degenerate
 * tetrahedron, unphysical material, dt <= 0), PORO_ENOMEM. */
poro_status poro_set_isolated(poro_ctx* ctx, int64_t n_elem, const double* vert,
                              const poro_material* mat, const double* dt);

/* Isolated damped-Maxwell elements (Section "Other applications"): like
 * poro_set_isolated with mat[n][3] = (eps, mu, sigma) per element (eps > 0,
 * mu > 0, sigma >= 0; host, copied).  Per element the library builds
 * A^{j*} = dt sum_d (d xi_j / d x_d) A_d on the 12-entry pattern of the curl
 * operator, e = -sigma dt / eps and (Z - e I)^{-1}.  Errors: PORO_EINVAL
 * (degenerate element or material), PORO_EUNSUPPORTED (not a Maxwell
 * context). */
poro_status poro_set_isolated_maxwell(poro_ctx* ctx, int64_t n, const double* vert, const double* mat,
                                      const double* dt);

/* Isolated tetrahedra with sub-cell material variation (Section
 * "Limitations": with material varying inside an element the stiffness
 * matrices become 3-tensors).  mat[n][4] holds one material per vertex
 * (vertex v of vert[i] carries mat[4 i + v]); the Jacobians A_d(x) and the
 * source matrix E(x) are the linear interpolation of the four vertex
 * materials' (a reading: the paper does not say how the material varies).
 * The predictor system is then Y = Y_0 + sum_{r=1..3} Mh3_r (sum_j Khat^j
 * A^{j*}_r - E*_r), Y_0 the constant-material operator of the mode-0 (mean)
 * Jacobians and Mh3_r = M^{-1} int phi_k phi_r phi_l; a material of degree 1
 * couples modes of equal degree, so Algorithm 3 does not solve Y directly.
 * poro_predict then iterates Q <- Y_0^{-1} (b - (Y - Y_0) Q) per element
 * (Richardson iteration preconditioned by Algorithm 3 on the mean
 * material, binary64) until max |change| <= tol max |Q| (see
 * poro_set_subcell_tolerance); the contraction factor is about the
 * material's relative variation inside the element.  Biot FP64 contexts
 * only; the LU comparator and the autotuners return PORO_EUNSUPPORTED on
 * such a population.  dt[n] as in poro_set_isolated (the CFL step of the
 * fastest vertex material is the safe choice).  Errors: PORO_EINVAL
 * (degenerate element or vertex material), PORO_EUNSUPPORTED, PORO_ENOMEM. */
poro_status poro_set_isolated_subcell(poro_ctx* ctx, int64_t n_elem, const double* vert,
                                      const poro_material* mat, const double* dt);

/* Stopping rule of the sub-cell iteration: relative change tol (>= 0,
 * default 1e-13) and at most max_iter iterations (1..100000, default 100).
 * Errors: PORO_EINVAL. */
poro_status poro_set_subcell_tolerance(poro_ctx* ctx, double tol, int32_t max_iter);

/* Iterations each element of [first, first + count) took in the last
 * sub-cell predictor (synchronises the context stream; after a
 * poro_predict_dev on another stream, synchronise that stream first): k > 0 converged
 * after k iterations, -k stopped at max_iter = k without converging or on a
 * non-finite iterate, 0 not run.  Errors: PORO_ESTATE (no sub-cell
 * population), PORO_EINVAL, PORO_ECUDA. */
poro_status poro_get_subcell_iterations(poro_ctx* ctx, int64_t first, int64_t count, int32_t* out);

/* Isolated viscoelastic elements (Section "Other applications"): like
 * poro_set_isolated with mat[n][12] = (rho, lam_u, mu_u, omega_1..3,
 * Ylam_1..3, Ymu_1..3) per element (host, copied; rho > 0, mu_u > 0, unrelaxed
 * bulk modulus > 0, omega_l >= 0).  Per element the library builds A^{j*} on
 * the 51-entry union pattern of the system's Jacobians, e_l = -omega_l dt,
 * the three (Z - e_l I)^{-1} and the couplings of E* into the stresses.
 * Errors: PORO_EINVAL (degenerate element or material), PORO_EUNSUPPORTED
 * (not a viscoelastic context). */
poro_status poro_set_isolated_viscoelastic(poro_ctx* ctx, int64_t n, const double* vert, const double* mat,
                                           const double* dt);

/* Copy DOFs Q[n_elem][13][B] (host) into the context.  Errors: PORO_ESTATE
 * before poro_set_isolated. */
poro_status poro_set_dofs(poro_ctx* ctx, const double* Q);

/* Space-time predictor of every element from the context's DOFs (Eq.
 * stp-lineq), solved by `solver`, followed by the time integration
 * I = dt * int_0^1 Qt dtau (= dt * Qt[..][0] for the shifted Legendre basis).
 * `cluster` must be -1 (all elements) for an isolated population.
 * Asynchronous on the context stream.  Errors: PORO_ESTATE,
 * PORO_EUNSUPPORTED (solver not available for this precision), PORO_ECUDA. */
poro_status poro_predict(poro_ctx* ctx, int32_t cluster, poro_solver solver);

/* Copy elements [first, first+count) of the last predictor to the host:
 * Qt_out[count][13][B][T].  Synchronises the context stream. */
poro_status poro_get_predictor(poro_ctx* ctx, int64_t first, int64_t count, double* Qt_out);

/* Copy the time-integrated DOFs I_out[count][13][B] of elements
 * [first, first+count).  Synchronises the context stream. */
poro_status poro_get_integrated(poro_ctx* ctx, int64_t first, int64_t count, double* I_out);

/* Wait for the context stream, polling, at most timeout_ms milliseconds
 * (< 0: no limit).  PORO_ETIMEOUT if the work is still running; the context
 * remains valid and a later poro_sync may succeed. */
poro_status poro_sync(poro_ctx* ctx, int32_t timeout_ms);

/* Device-pointer form of poro_predict for callers that keep DOFs resident:
 * Q0_dev[n_elem][13][B] (read), Qt_dev[n_elem][13][B][T] (written; may be
 * NULL to skip storing the full predictor), I_dev[n_elem][13][B] (written;
 * may be NULL).  All three are device pointers aligned to 16 bytes.
 * `stream` is a cudaStream_t (NULL: the context stream).  The element range
 * is [first, first + count) of the loaded population; row 0 of each buffer
 * is element `first`.  Errors: PORO_EINVAL, PORO_ESTATE, PORO_ECUDA. */
poro_status poro_predict_dev(poro_ctx* ctx, int64_t first, int64_t count, const double* Q0_dev,
                             double* Qt_dev, double* I_dev, poro_solver solver, void* stream);

/* End-to-end predictor from host buffers: Q0 of every element in, I out, with
 * the host<->device copies overlapped with the kernels.  The population is
 * cut into chunks of `chunk_elems` elements (0: automatic, about 16 chunks
 * of at least 4096 elements, the first three and last three smaller);
 * chunk i's Q0 copy, predictor (solver as in poro_predict) and I copy run on
 * three streams, so one chunk's copies run under another chunk's kernel.
 * q0_host[n_elem][Q][B] is read and becomes the context's DOFs;
 * I_out[n_elem][Q][B] is written (Q the system's quantities); the full predictor stays on the device
 * (poro_get_predictor).  Pinned host memory gives the overlap; pageable
 * memory works without it.  Synchronous: returns when I_out is complete.
 * (The paper has no counterpart: it is the host boundary of a batched GPU
 * predictor.)  Errors: PORO_EINVAL, PORO_ESTATE (no population),
 * PORO_EUNSUPPORTED, PORO_ECUDA, PORO_ETIMEOUT (a bounded device wait gave up). */
poro_status poro_predict_host(poro_ctx* ctx, const double* q0_host, double* I_out, int64_t chunk_elems,
                              poro_solver solver);

/* ------------------------------------------------------ meshes, corrector, time stepping */
/* A conforming tetrahedral mesh (Section "Spatial discretisation"):
 * xyz[n_vert][3] vertex coordinates, tet[n_elem][4] vertex ids, nb[n_elem][4]
 * the element across face i (the face opposite local vertex i) or -1 on a
 * boundary, face_tag[n_elem][4] a poro_face value (boundary faces must be
 * PORO_FACE_FREE_SURFACE or PORO_FACE_ABSORBING; periodicity is expressed
 * through nb, the faces of periodic neighbours matching up to a translation).
 * Inputs are copied.  Replaces any previous population.  Errors: PORO_EINVAL. */
poro_status poro_set_mesh(poro_ctx* ctx, int64_t n_vert, const double* xyz, int64_t n_elem, const int64_t* tet,
                          const int64_t* nb, const int32_t* face_tag);

/* One material per element (constant per element, Section "Spatial
 * discretisation").  Errors: PORO_ESTATE (no mesh), PORO_EINVAL. */
poro_status poro_set_materials(poro_ctx* ctx, const poro_material* mat);

/* Time steps (Section "Temporal discretisation with ADER"): every element's
 * CFL step dt_e = cfl_c/(2N+1) d/v (cfl_c = 0.5 in the paper).  Clustered
 * local time stepping with rate 2: element e joins cluster
 * c_e = min(max_clusters - 1, floor(log2(dt_e / dt_min))) and steps with
 * 2^c_e dt_min; max_clusters = 1 is global time stepping with dt_min.
 * Builds the element constants, the face data (neighbour face, vertex
 * permutation, outward normal, area), the Godunov flux solvers of every face
 * and the buffers of the cluster interfaces, and zeroes the DOFs.
 * dt_min_out (nullable) receives dt_min, cluster_out[n_elem] (nullable) the
 * cluster of each element.  Errors: PORO_ESTATE, PORO_EINVAL
 * (non-conforming face, max_clusters outside 1..16). */
poro_status poro_set_clusters(poro_ctx* ctx, double cfl_c, int32_t max_clusters, double* dt_min_out,
                              int32_t* cluster_out);

/* Point source with a Ricker wavelet s(t) = A (1 - 2a^2) exp(-a^2),
 * a = pi f0 (t - t0), acting on the quantities with weights w[13]
 * (Section "Homogeneous full-space"); located in the lowest-numbered element
 * containing xyz.  Each step adds w_p phi_k(xi_s) / (|J| M_kk) times the
 * exact integral of s over the step.  After poro_set_clusters.
 * Errors: PORO_EINVAL (outside the mesh), PORO_ESTATE. */
poro_status poro_add_point_source(poro_ctx* ctx, const double xyz[3], const double w[13], double f0, double t0,
                                  double amplitude);

/* Receiver at xyz: q_p(x_r) = sum_l Q_pl phi_l(xi_r) sampled at the end of
 * every step.  *id_out receives its index. */
poro_status poro_add_receiver(poro_ctx* ctx, const double xyz[3], int32_t* id_out);

/* Advance by whole steps of the largest cluster (2^(C-1) dt_min) while
 * t <= t_end.  Ticks k of dt_min: (A) the clusters whose step starts at k
 * predict (the context's precision, Algorithm 3) and add their
 * time-integrated predictor to the buffers of larger neighbours; (B) the
 * clusters whose step ends at k + 1 correct (Eq. semi_discrete over their
 * step: volume, Darcy source term, Godunov flux with each neighbour's trace
 * integrated over the same interval: its own integral, the buffered sum of
 * its sub-steps, or its predictor integrated over the sub-interval), then
 * point sources (over the element's own step) and receivers (sampled at
 * the end of every step of their element).  Synchronises at the end and
 * collects the new seismogram samples. */
poro_status poro_advance(poro_ctx* ctx, double t_end);

/* poro_advance without CUDA graphs, timing every cluster's launches: the
 * same cycles and results, and ms_out[C] (caller-owned, C = the context's
 * cluster count) receives the GPU milliseconds spent in each cluster's
 * predictor, buffer, corrector, source and receiver launches (CUDA events
 * around each cluster's group of launches on the context stream).  The
 * paper reports only whole-run LTS times (Section "Scaling"); this splits
 * them.  Errors: as poro_advance, PORO_EINVAL (NULL ms_out). */
poro_status poro_cluster_times(poro_ctx* ctx, double t_end, double* ms_out);

/* Replay a CUDA graph of one cycle (default on) or enqueue every cycle's
 * launches from the host (off); results are identical. */
poro_status poro_set_graphs(poro_ctx* ctx, int32_t on);

/* One corrector pass of all elements from the last predictor (low-level). */
poro_status poro_correct(poro_ctx* ctx, int32_t cluster);

/* DOFs Q_out[n_elem][13][B] (synchronises). */
poro_status poro_get_dofs(poro_ctx* ctx, double* Q_out);

/* Samples of receiver rec: up to cap times t_out[cap] and values
 * q_out[cap][13]; *n_out = number of samples recorded. */
poro_status poro_get_seismogram(poro_ctx* ctx, int32_t rec, int64_t cap, double* t_out, double* q_out,
                                int64_t* n_out);

/* Current simulation time and step. */
poro_status poro_get_time(const poro_ctx* ctx, double* t, double* dt);

/* Host-only: the Godunov flux solver matrices of one face with unit outward
 * normal n[3] (A_n^L q* = Fm q_L + Fp q_R, both [13][13] row-major); kind a
 * poro_face value; mR is required for PORO_FACE_INTERIOR. */
poro_status poro_flux_matrices(const poro_material* mL, const poro_material* mR, const double n[3], int32_t kind,
                               double* Fm, double* Fp);

/* ------------------------------------------------------ dense-LU comparator */
/* The approach Section "Block-wise back-substitution" replaces: the whole
 * predictor system of an element (s = 13 B (N+1) unknowns) factored once,
 * P Y = L U with partial pivoting in binary64 after power-of-two row and
 * column equilibration, then two triangular solves per predictor (2 s^2
 * flops, s^2 doubles of factors per element; Table flop-count). */

/* Device bytes poro_lu_factor needs for `count` elements of degree N. */
poro_status poro_lu_bytes(int degree_N, int64_t count, size_t* bytes);

/* Assemble, equilibrate and factor the predictor systems of elements
 * [first, first + count) (count <= 65535) into a context-owned device buffer
 * (replaces a previous factorisation; synchronous).  Afterwards
 * poro_predict / poro_predict_dev with PORO_SOLVE_LU solve those elements.
 * Errors: PORO_ENOMEM (factors do not fit), PORO_ENUMERIC (zero pivot),
 * PORO_ESTATE, PORO_EINVAL. */
poro_status poro_lu_factor(poro_ctx* ctx, int64_t first, int64_t count);

/* Free the factor buffer. */
poro_status poro_lu_release(poro_ctx* ctx);

/* Dense-LU predictor without any allocation.  The paper has no counterpart:
 * this is a service for callers that cannot call cudaMalloc (for example code
 * working inside a fixed device-memory budget handed out by an outer
 * framework's allocator, or loops that must not take the device
 * synchronisation cudaMalloc/cudaFree may imply), which poro_lu_factor
 * excludes because it allocates its factor buffer on every call.
 * Factors and solves elements [first, first + count) of the loaded population
 * in one asynchronous call on `stream` (NULL: the context stream), with the
 * same kernels as poro_lu_factor + PORO_SOLVE_LU; Q0_dev, Qt_dev (nullable),
 * I_dev (nullable) as in poro_predict_dev (device pointers, 16-byte aligned,
 * row 0 = element `first`).
 * The factors live in one 64 MiB array inside the library (every GPU that
 * loads libporoader holds it until the process exits); the call allocates
 * nothing.  A batch needing more than 64 MiB of factors (s^2 doubles plus 24 s
 * bytes per element, s = 13 B (N+1): at most 7 elements at N = 3, 1 at
 * N = 4, none at N >= 5) is rejected with PORO_EINVAL and a message giving the
 * bytes needed.  The first call for a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process, so do not use the library across a cudaDeviceReset of that
 * device.  The caller's current device is restored before the call returns.
 * Every call shares the one array and each
 * call zeroes what must start at zero (factor area, zero-pivot flag) before
 * use; calls whose work overlaps on the GPU (different streams, or a second
 * call before the first finished on another stream) race on the array.
 * A zero pivot is not reported (use poro_lu_factor for the checked path).
 * Errors: PORO_EINVAL, PORO_ESTATE (no population), PORO_ECUDA. */
poro_status poro_lu_predict_static(poro_ctx* ctx, int64_t first, int64_t count, const double* Q0_dev,
                                   double* Qt_dev, double* I_dev, void* stream);

/* Autotuner of the predictor kernels: times the CTA-size variants (0: 256
 * threads at N >= 5, 128 at N = 4, 64 at N <= 3; 1: the alternative) on the
 * first `sample` elements of the loaded population (<= 0: all), three timed
 * runs after two warm-ups each, and keeps the fastest for this context.
 * *variant_out (nullable) receives the choice, ms_out[2] (nullable) the
 * mean milliseconds per run of each variant.  The DOFs are not changed; the
 * context's predictor buffers are overwritten.  The paper has no counterpart
 * (its kernels are generated per architecture). */
poro_status poro_autotune(poro_ctx* ctx, int64_t sample, int32_t* variant_out, double* ms_out);

/* Select a predictor CTA-size variant explicitly (0 or 1). */
poro_status poro_set_variant(poro_ctx* ctx, int32_t variant);

/* Tile choices of the predictor kernels: choice = 6 * cta + layout, with cta
 * the CTA-size variant (as poro_set_variant) and layout capping the operand
 * buffers of the mixed kernel's tensor-core sweeps per degree block
 * (A-tile buffers, Khat image slots): 0 (3, 3) = as many as fit (default),
 * 1 (2, 3), 2 (1, 3), 3 (2, 2), 4 (1, 2), 5 (1, 1).  Fewer buffers serialise
 * the star products, image copies and MMAs of the three directions; more
 * buffers take shared memory the block may not have, so the kernel still
 * uses only what fits.  Every choice gives bitwise the same predictor.
 * Available: FP64 contexts layouts 0 only (choices 0 and 6), the bf16 form
 * cta 0 only (choices 0..5), the tf32 form all 12; layouts 1..5 with one
 * refinement sweep (the default) only. */
#define PORO_TILE_CHOICES 12

/* Autotuner over the available tile choices: times each on the first
 * `sample` elements of the loaded population (<= 0: all; two warm-ups,
 * three timed runs) and keeps the fastest for this context.  *choice_out
 * (nullable) receives it, ms_out[PORO_TILE_CHOICES] (nullable) the mean
 * milliseconds per run of each choice (-1 for choices not available).  The
 * DOFs are kept; the predictor buffers are overwritten.  The paper has no
 * counterpart (its kernels are generated per architecture).
 * Errors: PORO_ESTATE (no population), PORO_EUNSUPPORTED (not Biot). */
poro_status poro_autotune_tiles(poro_ctx* ctx, int64_t sample, int32_t* choice_out, double* ms_out);

/* Select a tile choice explicitly.  Errors: PORO_EINVAL (not available). */
poro_status poro_set_tiles(poro_ctx* ctx, int32_t choice);

/* Floating-point operations one predictor of this context performs, counted
 * from the structural non-zeros the kernels touch (Khat blocks, the 54-entry
 * star pattern, the (N+1)^2 time solves): used for rooflines.  flops_out[0]
 * = FP64 operations (PORO_FP64), flops_out[1] = low-precision operations
 * (refinement modes), flops_out[2] = residual operations (refinement modes,
 * per sweep). */
poro_status poro_flop_count(const poro_ctx* ctx, int32_t refine_sweeps, double* flops_out);

/* ------------------------------------------------------ serving */
/* Continuous-batching server for ensembles of independent simulations (the
 * paper has no counterpart; it runs one simulation per job).  Requests are
 * admitted in arrival order while a slot is free and the sum of the admitted
 * requests' device-memory footprints (poro_footprint_bytes) fits the
 * budget; each admitted request runs on its own context and CUDA stream on a
 * worker thread, so requests admitted while others run overlap with them on
 * the device.  A failing request (invalid input, footprint above the whole
 * budget, an error in its own calls) ends in PORO_REQ_FAILED without
 * affecting the others.  All calls are thread-safe. */
typedef struct poro_server poro_server;

enum { PORO_REQ_QUEUED = 0, PORO_REQ_RUNNING = 1, PORO_REQ_DONE = 2, PORO_REQ_FAILED = 3, PORO_REQ_CANCELLED = 4 };

/* One simulation: the arguments of poro_set_mesh, poro_set_materials,
 * poro_set_clusters, poro_add_point_source (n_sources of them) and
 * poro_add_receiver (n_receivers), optional initial DOFs Q0 (nullable), run
 * from t = 0 by whole steps of the largest cluster to t_end.  All arrays are
 * copied by poro_submit. */
typedef struct {
    int32_t degree_N, precision, refine_sweeps, max_clusters;
    double cfl_c, t_end;
    int64_t n_vert;
    const double* xyz;
    int64_t n_elem;
    const int64_t* tet;
    const int64_t* nb;
    const int32_t* face_tag;
    const poro_material* mat;
    const double* Q0;
    int32_t n_sources, n_receivers;
    const double* src_xyz;    /* [n_sources][3] */
    const double* src_w;      /* [n_sources][13] */
    const double* src_f0;     /* [n_sources] */
    const double* src_t0;     /* [n_sources] */
    const double* src_amp;    /* [n_sources] */
    const double* rec_xyz;    /* [n_receivers][3] */
} poro_scenario;

/* Server on `device` with a device-memory budget in bytes and at most
 * max_slots concurrently running requests. */
poro_status poro_server_create(int device, size_t hbm_budget, int32_t max_slots, poro_server** out);

/* Execution mode for requests admitted after the call.  on != 0 (the
 * default): batched.  One executor thread advances the running requests in
 * groups of equal degree, precision, refinement and cluster count; every
 * tick's predictors of a group's requests are one kernel launch over all of
 * their due elements, followed by each request's buffers, correctors, sources
 * and receivers, one cycle captured as a CUDA graph and replayed; groups of
 * different degrees run concurrently on their own streams.  on == 0: each
 * request advances on its own thread, context and stream.  Results are
 * identical in both modes and alone.  Errors: PORO_EINVAL (NULL server). */
poro_status poro_server_set_batching(poro_server* s, int32_t on);
/* Cancel queued and running requests, wait for the workers, free. */
poro_status poro_server_destroy(poro_server* srv);
const char* poro_server_last_error(poro_server* srv);
/* Copy the scenario and queue it; *ticket identifies the request. */
poro_status poro_submit(poro_server* srv, const poro_scenario* sc, uint64_t* ticket);
/* State (PORO_REQ_*) and simulated time reached. */
poro_status poro_poll(poro_server* srv, uint64_t ticket, int32_t* state, double* sim_time);
/* Block until the request finished (DONE, FAILED or CANCELLED) or timeout_ms
 * passed (< 0: no limit; PORO_ETIMEOUT then). */
poro_status poro_wait(poro_server* srv, uint64_t ticket, int32_t timeout_ms, int32_t* state);
/* Seismogram of receiver rec of a DONE request (as poro_get_seismogram). */
poro_status poro_fetch(poro_server* srv, uint64_t ticket, int32_t rec, int64_t cap, double* t_out, double* q_out,
                       int64_t* n_out);
/* Wall-clock seconds from submission to admission, from admission to the
 * end, and in total (time to seismogram) of a finished request. */
poro_status poro_request_times(poro_server* srv, uint64_t ticket, double* queued_s, double* run_s, double* total_s);
/* Error text of a FAILED request. */
poro_status poro_request_error(poro_server* srv, uint64_t ticket, char* buf, size_t cap);
/* Cancel: a queued request is dropped, a running one stops at its next chunk. */
poro_status poro_cancel(poro_server* srv, uint64_t ticket);
/* Device bytes the server reserves for a request of this size. */
poro_status poro_footprint_bytes(int degree_N, int64_t n_elem, int32_t max_clusters, int32_t n_receivers, size_t* bytes);

#ifdef __cplusplus
}
#endif
#endif /* PORO_ADER_H */
