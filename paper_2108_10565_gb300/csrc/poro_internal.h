// Internal declarations shared by the host set-up, the C ABI and the kernels
// of libporoader.  Not part of the public interface (include/poroader.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/poroader.h"

// the CUDA runtime's graph-exec handle (cudaGraphExec_t points to it),
// declared here for the host translation units built without CUDA headers
struct CUgraphExec_st;

namespace poro {

constexpr int NQ = 13;
constexpr int MAX_N = 6;
// quantity indices, paper order (Section "Governing equations")
enum { SXX, SYY, SZZ, SXY, SYZ, SXZ, QU, QV, QW, QP, QUF, QVF, QWF };

constexpr int n_modes(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
constexpr int block_size(int g) { return (g + 1) * (g + 2) / 2; }
constexpr int block_offset(int g) { return g * (g + 1) * (g + 2) / 6; }
// tensor-core tile of degree block g's Khat product: N extent (rows l < o_g,
// a multiple of 16, at least 16) and K extent (columns of the block, a
// multiple of the MMA's K step: 8 for tf32 words, 16 for bf16)
constexpr int tc_np(int g) { return block_offset(g) <= 16 ? 16 : (block_offset(g) + 15) / 16 * 16; }
constexpr int tc_kp(int g, bool bf16 = false) {
    return bf16 ? (block_size(g) + 15) / 16 * 16 : (block_size(g) + 7) / 8 * 8;
}

// Union sparsity pattern of A*, B*, C* (54 entries): for every row p the
// columns q with a structurally non-zero Jacobian entry.  Rows are stored
// contiguously; star_row_ptr(p) .. star_row_ptr(p+1) index star_col().
#ifdef __CUDACC__
#define PORO_HD __host__ __device__
#else
#define PORO_HD
#endif
constexpr int STAR_NNZ = 54;
PORO_HD constexpr int star_row_ptr(int p) {
    constexpr int t[NQ + 1] = {0, 6, 12, 18, 20, 22, 24, 28, 32, 36, 42, 46, 50, 54};
    return t[p];
}
PORO_HD constexpr int star_row(int n) {
    return n < 18 ? n / 6 : n < 24 ? 3 + (n - 18) / 2 : n < 36 ? 6 + (n - 24) / 4 : n < 42 ? 9 : 10 + (n - 42) / 4;
}
PORO_HD constexpr int star_col(int n) {
    constexpr int t[STAR_NNZ] = {
        QU, QV, QW, QUF, QVF, QWF,   // s_xx
        QU, QV, QW, QUF, QVF, QWF,   // s_yy
        QU, QV, QW, QUF, QVF, QWF,   // s_zz
        QU, QV,                      // s_xy
        QV, QW,                      // s_yz
        QU, QW,                      // s_xz
        SXX, SXY, SXZ, QP,           // u
        SYY, SXY, SYZ, QP,           // v
        SZZ, SXZ, SYZ, QP,           // w
        QU, QV, QW, QUF, QVF, QWF,   // p
        SXX, SXY, SXZ, QP,           // u_f
        SYY, SXY, SYZ, QP,           // v_f
        SZZ, SXZ, SYZ, QP};          // w_f
    return t[n];
}

// Damped Maxwell equations (Section "Other applications"): 6 quantities
// (E_x, E_y, E_z, H_x, H_y, H_z), eps E_t = curl H - sigma E, mu H_t =
// -curl E.  Union pattern of the reference Jacobians: row p couples the two
// field components of the other kind that its curl row involves.
namespace maxwell {
constexpr int NQ = 6;
constexpr int STAR_NNZ = 12;
PORO_HD constexpr int star_row(int n) { return n / 2; }
PORO_HD constexpr int star_col(int n) {
    constexpr int t[STAR_NNZ] = {4, 5, 3, 5, 3, 4, 1, 2, 0, 2, 0, 1};
    return t[n];
}
// per-element constants: star[3][12], (Z - e I)^{-1} [T][T], e, 0, dt, pad
PORO_HD constexpr int elem_const_stride(int N) { return (3 * STAR_NNZ + (N + 1) * (N + 1) + 4 + 1) & ~1; }
}  // namespace maxwell

// Viscoelastic attenuation (Section "Other applications": upper-triangular
// source matrix), anelastic-function form with NMECH relaxation mechanisms:
// 27 quantities (6 stresses xx yy zz xy yz xz, velocities u v w, then six
// anelastic functions per mechanism in the stress order).  E* holds
// -omega_l dt on the diagonal of mechanism l's functions and the couplings
// -(Ylam_l + 2 Ymu_l) dt, -Ylam_l dt (normal block) and -2 Ymu_l dt (shear)
// from them into the stresses.  Union pattern of the reference Jacobians
// (51 entries a direction): normal stresses <- u v w, shear stresses <- their
// two velocities, velocities <- the three stresses of their row of sigma,
// anelastic functions <- the velocities of their strain-rate component.
namespace visco {
constexpr int NMECH = 3;
constexpr int NQ = 9 + 6 * NMECH;
constexpr int STAR_NNZ = 15 + 9 + 9 * NMECH;
// row-major pattern of the first 24 (stress and velocity rows) and of one
// mechanism's 9 (functions xx yy zz xy yz xz), columns as quantity indices
PORO_HD constexpr int star_row(int n) {
    constexpr int r[24] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 4, 4, 5, 5, 6, 6, 6, 7, 7, 7, 8, 8, 8};
    constexpr int m[9] = {0, 1, 2, 3, 3, 4, 4, 5, 5};
    return n < 24 ? r[n] : 9 + 6 * ((n - 24) / 9) + m[(n - 24) % 9];
}
PORO_HD constexpr int star_col(int n) {
    constexpr int c[24] = {6, 7, 8, 6, 7, 8, 6, 7, 8, 6, 7, 7, 8, 6, 8, 0, 3, 5, 3, 1, 4, 5, 4, 2};
    constexpr int m[9] = {6, 7, 8, 6, 7, 7, 8, 6, 8};
    return n < 24 ? c[n] : m[(n - 24) % 9];
}
// per-element constants: star[3][51], (Z - e_l I)^{-1} [NMECH][T][T], then
// 14 scalars: per mechanism (-(Ylam+2Ymu) dt, -Ylam dt, -2 Ymu dt), e_l
// (NMECH), dt, pad
constexpr int NSC = 3 * NMECH + NMECH + 2;
PORO_HD constexpr int sc_dt() { return 4 * NMECH; }
PORO_HD constexpr int elem_const_stride(int N) {
    return (3 * STAR_NNZ + NMECH * (N + 1) * (N + 1) + NSC + 1) & ~1;
}
}  // namespace visco

// Per-element constants, in doubles, in this order:
//   star[3][54]       A^{j*} = dt A^j on the union pattern
//   zinv_uf[T][T]     (Z - e I)^{-1}, e = E*_{uf,uf} (row-major, [u][s])
//   e, g, dt, pad     E*_{uf,uf}, E*_{u,uf}, time step
PORO_HD constexpr int elem_const_stride(int N) {
    // keep 16-byte alignment of every element's block
    return (3 * STAR_NNZ + (N + 1) * (N + 1) + 4 + 1) & ~1;
}
PORO_HD constexpr int ec_zinv(int) { return 3 * STAR_NNZ; }
PORO_HD constexpr int ec_scalars(int N) { return 3 * STAR_NNZ + (N + 1) * (N + 1); }

// Khat^j restricted to the columns of one degree block g, in CSR over the
// rows l < o_g (the only rows Lemma 1 leaves non-zero); entries
// (m_local, value) with m_local < d_g.
struct KhatBlockCSR {
    std::vector<int32_t> row_ptr;    // [o_g + 1]
    std::vector<int32_t> col;        // m_local
    std::vector<double> val;
};

struct ReferenceData {
    int N = 0, B = 0, T = 0;
    std::vector<double> mass_diag;     // [B]
    std::vector<double> khat;          // [3][B][B]
    std::vector<double> zinv;          // [T][T]  Z^{-1}
    std::vector<double> z;             // [T][T]  Z = S^{-1}(W - K^tau)
    std::vector<double> sinv_w;        // [T]     S^{-1} w
    std::vector<KhatBlockCSR> blocks;  // [(N+1)*3], index g*3 + j (block 0 empty)
    int64_t khat_block_nnz = 0;        // structural non-zeros of all Khat blocks
};

// ----- host set-up (setup.cpp) -----
bool reference_data(int N, ReferenceData& out, std::string& err);
bool material_jacobians(const poro_material& m, double abc[3][NQ][NQ], double e[NQ][NQ],
                        std::string& err);
bool max_wave_speed(const poro_material& m, double& v, std::string& err);
bool tet_geometry(const double* v12, double jinv[3][3], double& volume, double& insphere_d,
                  std::string& err);
bool invert_small(int n, const double* a, double* ainv);
// fills one element's constants block (elem_const_stride(N) doubles)
bool element_constants(const ReferenceData& ref, const double* v12, const poro_material& mat,
                       double dt, double* out, std::string& err);
// the same for a damped-Maxwell element, mat = (eps, mu, sigma)
// (maxwell::elem_const_stride(N) doubles)
bool maxwell_element_constants(const ReferenceData& ref, const double* v12, const double mat[3], double dt,
                               double* out, std::string& err);
// One viscoelastic element: mat = rho, lam_u, mu_u, omega[3], Ylam[3],
// Ymu[3]; out gets visco::elem_const_stride(N) doubles
bool visco_element_constants(const ReferenceData& ref, const double* v12, const double mat[12], double dt,
                             double* out, std::string& err);

// ----- sub-cell material (setup.cpp, subcell.cu) -----
// Per element, besides the mean-material constants (elem_const_stride
// layout, from the mode-0 Jacobians): star_r[3][54] for the variation modes
// r = 1..3 of the linearly interpolated Jacobians, then (e_r, g_r) of E*_r.
PORO_HD constexpr int subcell_var_stride() { return (3 * 3 * STAR_NNZ + 6 + 1) & ~1; }
// Mh3_r = M^{-1} int phi_k phi_r phi_l, r = 1..3, as CSR over all rows k:
// row pointers [3][B + 1] absolute into col / val (device)
struct SubcellReference {
    int32_t* m3_row = nullptr;
    int32_t* m3_col = nullptr;
    double* m3_val = nullptr;
};
// host: the three tensors by the collapsed Gauss rule of reference_data
bool subcell_mass_tensors(const ReferenceData& R, std::vector<int32_t>& row, std::vector<int32_t>& col,
                          std::vector<double>& val, std::string& err);
// host: P[r][v], the modal coefficients f_r = sum_v P[r][v] f_v of the linear
// field with values f_v at the reference vertices
bool subcell_projection(double P[4][4], std::string& err);
// host: one element with vertex materials mats[4] (vertex v of v12 carries
// mats[v]); mean constants into mean_out, variation block into var_out
bool subcell_element_constants(const ReferenceData& ref, const double P[4][4], const double* v12,
                               const poro_material mats[4], double dt, double* mean_out, double* var_out,
                               std::string& err);

// ----- corrector set-up (mesh.cpp) -----
// Godunov flux solver matrices of one face: A_n^L q* = Fm q_L + Fp q_R.
// kind: PORO_FACE_INTERIOR (mR required), PORO_FACE_FREE_SURFACE, PORO_FACE_ABSORBING.
bool flux_solver(const poro_material& mL, const poro_material* mR, const double n[3], int kind, double* Fm,
                 double* Fp, std::string& err);
// phi_l(xi) for all l (singularity-free homogenised recurrences)
void basis_at(int N, const double xi[3], double* phi);
// Floc[4][B][B] = int_face phi_k phi_l, Fnb[4][4][6][B][B] = int_face phi_k(L) phi_l(R)
// for local face f, neighbour face h, vertex permutation s
void face_matrices(int N, std::vector<double>& Floc, std::vector<double>& Fnb);
// Pf[4][df][B], Pnb[96][df][B] with Floc[f] = Pf^T Pf, Fnb[f,h,s] = Pf^T Pnb,
// df = (N+1)(N+2)/2 (traces in a basis orthonormal on the reference triangle)
void face_traces(int N, std::vector<double>& Pf, std::vector<double>& Pnb);
int face_permutation_index(const int p[3]);

// ----- device side (kernels) -----
struct DeviceReference {
    int N = 0;
    double* khat_val = nullptr;   // concatenated CSR values of all (g, j) blocks
    int32_t* khat_col = nullptr;  // concatenated CSR columns (m_local)
    int32_t* khat_row = nullptr;  // concatenated row pointers, absolute into val/col
    int32_t row_base[MAX_N + 1][3] = {};  // start of block (g, j)'s row pointers in khat_row
    double* zinv = nullptr;       // [T][T]
    // rows l < o_g of block (g, j) with Khat entries, dealt to 2, 4, 8 warps
    // (index 0, 1, 2): at lists[w] + list_base[w][g][j], [warps + 1] list
    // starts, then the lists
    int32_t* lists[3] = {nullptr, nullptr, nullptr};
    int32_t list_base[3][MAX_N + 1][3] = {};
};

// Extra device data of the mixed-precision (refinement) path.
struct MixedReference {
    const DeviceReference* base = nullptr;
    bool bf16 = false;              // sweeps' split products in bf16 (else tf32)
    float* res_inv = nullptr;       // [3][B][2] 1 / d_jl as (hi, lo) binary32 words
    // residual rows dealt to 8, 4 and 2 warps (longest work first, each row to
    // the least loaded warp): [warps + 1] list starts, then the lists
    int32_t* res_order8 = nullptr;
    int32_t* res_order4 = nullptr;
    int32_t* res_order2 = nullptr;
    float* zinv_f32 = nullptr;      // [T][T]
    // tensor-core images of Khat^j restricted to block g (rows l < o_g, columns
    // of the block), K-major core-matrix layout of tc_np(g) x tc_kp(g) words
    // (tf32 in 32-bit words, or bf16), hi image then lo image; tc_off[g][j] in
    // bytes
    float* khat_tc = nullptr;
    int32_t tc_off[MAX_N + 1][3] = {};
    int32_t* status = nullptr;      // device word: 1 after a bounded wait gave up
    long long wait_limit = 0;       // SM clocks a wait of the sweeps may take (0: about 1 s)
    // operand layout of the tensor-core sweeps (the autotuner's tile choice):
    // at most cap_a A-tile buffers and cap_b Khat image slots per degree block
    // (3, 3: as many as fit in the operand region)
    int cap_a = 3, cap_b = 3;
};

// Fill the constant-memory residual table of degree N on the current device
// (row pointers relative to the entries); idempotent, same data for every
// context of that degree.
int upload_residual_table(int N, const int32_t* rows, const int32_t* entries, int n_entries);

// Per-run buffers of a predictor launch that covers the elements of several
// simulations of the same degree and precision (the server's batched mode):
// item i of the launch is element elems[i] of run item_run[i], read from and
// written to that run's buffers.
struct RunPtrs {
    const double* q0;      // [ne][13][B]
    const double* econst;  // [ne][stride]
    double* qt;            // [ne][13][B][T] or nullptr
    double* iout;          // [ne][13][B] or nullptr
};

// Launch the mixed-precision predictor (binary32 sweeps, `refine` residual
// corrections in double-binary32) for `count` elements.  With `runs`
// (device array) and `item_run`, the items come from several runs and q0,
// econst, qt, iout are ignored.
int launch_stp_mixed(const MixedReference& ref, int refine, const int32_t* elems, int64_t count,
                     const double* q0, const double* econst, double* qt, double* iout, void* stream,
                     int variant = 0, const RunPtrs* runs = nullptr, const int32_t* item_run = nullptr);

// Dense-LU comparator: reference data and per-batch scratch (factors,
// pivots, permutation, equilibration factors, singularity flag).
struct LUReference {
    int N = 0;
    double* z = nullptr;       // [T][T] Z = S^{-1}(W - K^tau)
    int32_t* krow = nullptr;   // [3][B+1] full-row CSR of Khat^j, absolute offsets
    int32_t* kcol = nullptr;
    double* kval = nullptr;
};
struct LUScratch {
    double* A = nullptr;       // [count][s][s] factors L\U of P R Y' C
    int32_t* piv = nullptr;    // [count][s]
    int32_t* perm = nullptr;   // [count][s]
    double* R = nullptr;       // [count][s]
    double* C = nullptr;       // [count][s]
    int32_t* bad = nullptr;    // 1 if a zero pivot occurred
    double* x = nullptr;       // [count][s] solution scratch of the blocked solve (nullable: one CTA per element)
    // the blocked solve's launches captured as a CUDA graph, valid for the
    // pointers and counts in key
    CUgraphExec_st* exec = nullptr;  // a cudaGraphExec_t
    const void* key[10] = {};
};
size_t lu_scratch_bytes(int N, int64_t count);
int launch_lu_factor(const LUReference& ref, int64_t count, const double* econst, LUScratch& w, void* stream);
int launch_lu_solve(const LUReference& ref, int64_t count, LUScratch& w, int64_t offset, const double* q0,
                    const double* econst, double* qt, double* iout, void* stream);

// Read-only view of the context fields the allocation-free LU entry point
// needs (defined in api.cu).
struct CtxView {
    int device = 0, N = 0;
    int64_t n_elem = 0;
    int stride = 0;
    const double* econst = nullptr;
    const LUReference* lref = nullptr;
    void* stream = nullptr;
};
bool ctx_view(const poro_ctx* c, CtxView& v);
void ctx_set_error(poro_ctx* c, const std::string& msg);

// Corrector (Eq. semi_discrete integrated over one step) for `count`
// elements starting at `first` of the mesh.
struct CorrectorData {
    int N = 0;
    const double* econst = nullptr;   // [ne][stride] (stars with dt, e, g, dt)
    const double* iout = nullptr;     // [ne][13][B] time-integrated predictor
    double* q = nullptr;              // [ne][13][B] DOFs, updated in place
    const int32_t* nb = nullptr;      // [ne][4]
    const int32_t* tab = nullptr;     // [ne][4] neighbour table index f*24 + h*6 + s, or -1
    const double* fc = nullptr;       // [ne][4] 2 |S_f| / |J|
    const double* fF = nullptr;       // [ne][4][2][169] flux solver matrices
    const int32_t* vrow = nullptr;    // volume CSR rows [3][B+1] (absolute)
    const int32_t* vcol = nullptr;
    const double* vval = nullptr;     // Kv^j_kl = M_ll Khat^j_lk / M_kk
    const double* minv = nullptr;     // [B] 1 / M_kk
    // face traces (df = (N+1)(N+2)/2): Floc^f = Pf^T Pf, Fnb^{f,h,s} = Pf^T Pnb
    const double* Pf = nullptr;       // [4][df][B]
    const double* Pnb = nullptr;      // [96][df][B]
    // double-binary32 (hi, lo) copies for the mixed-precision form (dw = true:
    // the corrector runs in double-binary32 and fF is not needed)
    bool dw = false;
    const float* fF2 = nullptr;       // [ne][4][2][169] pairs
    const float* Pf2 = nullptr;       // [4][df][B] pairs
    const float* Pnb2 = nullptr;      // [96][df][B] pairs
    const float* vval2 = nullptr;     // Kv^j values, pairs
    // clustered local time stepping (all nullptr / 1 for global time stepping)
    int C = 1;                        // number of clusters
    const int32_t* cl = nullptr;      // [ne] cluster of each element
    const int32_t* slot = nullptr;    // [ne][C] buffer slot of (element, larger level) or -1
    const double* buf = nullptr;      // [slots][13][B] buffered sub-step integrals
    const double* qt = nullptr;       // [ne][13][B][T] full predictors (larger neighbours)
    int64_t tick = 0;                 // tick k of the correction (interval ends at k + 1)
};
int launch_lts_buffers(int N, int C, const int32_t* elems, int64_t count, const int32_t* slot, const double* iout,
                       double* buf, int64_t tick, void* stream);
// `runs` (device array, nullable) / `item_run`: a launch over several runs;
// item i is element elems[i] of the run whose data is runs[item_run[i]] (d
// then only selects the precision and degree)
int launch_corrector(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream,
                     const CorrectorData* runs = nullptr, const int32_t* item_run = nullptr);
int launch_corrector_dw(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream,
                        const CorrectorData* runs = nullptr, const int32_t* item_run = nullptr);
int launch_point_source(int N, double* q, int64_t elem, const double* coef, double amp, void* stream);
// One point source or receiver of one run, for the launches of a batched
// group that serve all its runs' sources (then receivers) of a tick.
// Source: q[elem] += (S(t1) - S(t0)) coef over the step [(k+1-len) dt,
// (k+1) dt], k = *tick + k_rel.  Receiver: out[*counter] = Q[elem] phi, then
// ++*counter.
struct TickItem {
    double* q = nullptr;
    const double* vec = nullptr;     // coef (source) or phi (receiver)
    double* out = nullptr;           // receiver samples
    int32_t* counter = nullptr;      // receiver sample counter
    const int64_t* tick = nullptr;   // the run's tick counter (source)
    int64_t elem = 0, len = 1, k_rel = 0;
    double f0 = 0.0, tc = 0.0, dt = 0.0;
};
int launch_tick_sources(int N, const TickItem* items, int64_t count, void* stream);
int launch_tick_receivers(int N, const TickItem* items, int64_t count, void* stream);
// *ticks[i] += n for i < count (the tick counters of a group's runs)
int launch_ticks_advance(int64_t* const* ticks, int count, int64_t n, void* stream);
int launch_point_source_tick(int N, double* q, int64_t elem, const double* coef, double f0, double tc, double dt,
                             int64_t len, int64_t k_rel, const int64_t* tick, void* stream);
int launch_receiver_count(int N, const double* q, int64_t elem, const double* phi, double* out, int32_t* counter,
                          void* stream);
int launch_tick_advance(int64_t* tick, int64_t n, void* stream);
int launch_receivers(int N, const double* q, int32_t nrec, const int64_t* elems, const double* phi, double* out,
                     int64_t stride_out, void* stream);

// Batched advance of several simulations (the server): runs of one degree,
// precision, refinement, CTA variant and cluster count, each at the end of a
// cycle.  Every tick's predictors of all runs are one launch; each run's
// results are those it gets when advanced alone.  group_enqueue queues
// n_cycles cycles on the group's own stream; group_finish waits for them and
// appends the receiver samples.  The runs must not be used otherwise while
// the group exists.
struct RunGroup;
RunGroup* group_create(poro_ctx* const* runs, int n, std::string& err);
int group_enqueue(RunGroup* g, int64_t n_cycles, std::string& err);
poro_status group_finish(RunGroup* g, std::string& err);
void group_destroy(RunGroup* g);

// Launch the FP64 Algorithm-3 predictor for `count` elements.
// q0[count][13][B], econst[count][stride], qt (nullable), iout (nullable).
// `elems` (nullable): element index list; outputs are indexed by element.
// `variant` selects the CTA size (0: default, 1: the alternative the
// autotuner may pick).  `runs` / `item_run`: items of several runs, as for
// launch_stp_mixed.
int launch_stp_fp64(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
                    const double* econst, double* qt, double* iout, void* stream, int variant = 0,
                    const RunPtrs* runs = nullptr, const int32_t* item_run = nullptr);
// The same kernel for the damped Maxwell system (q0 [count][6][B], econst
// [count][maxwell::elem_const_stride(N)], qt [count][6][B][T]).
int launch_stp_fp64_maxwell(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
                            const double* econst, double* qt, double* iout, void* stream);
// Sub-cell material predictor (subcell.cu): evar [count][subcell_var_stride()],
// iters [count] (iterations of each element, negative if not converged).
int launch_stp_subcell(const DeviceReference& ref, const SubcellReference& sub, int64_t count, const double* q0,
                       const double* econst, const double* evar, double* qt, double* iout, int32_t* iters,
                       double tol, int max_iter, void* stream);
// ... and for the viscoelastic system (q0 [count][27][B], econst
// [count][visco::elem_const_stride(N)], qt [count][27][B][T]).
int launch_stp_fp64_visco(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
                          const double* econst, double* qt, double* iout, void* stream);

}  // namespace poro
