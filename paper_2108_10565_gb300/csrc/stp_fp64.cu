// K1: the space-time predictor of one element per CTA, in IEEE binary64,
// by the degree-block back-substitution of the paper (Section "Block-wise
// back-substitution", Algorithm 3).
//
// Per element the CTA keeps b (13 x B x T) in shared memory and overwrites it
// in place with the predictor Qt: once the modes of degree block g are solved,
// their b entries are dead.  For g = N .. 0:
//   S3  time solves: Q[p,m,:] = Zinv_p b[p,m,:] for the modes m of block g,
//       Zinv_p = (Z - E*_pp I)^{-1}; E*_pp != 0 only for u_f, v_f, w_f, and the
//       strictly upper part G of E* couples u_f -> u, v_f -> v, w_f -> w, so a
//       thread solves u_f, adds g Q_uf to b_u, then solves u.
//   S4  green update (g > 0), one direction j at a time:
//       X[p,m,u] = sum_q A^{j*}_pq Q[q,m,u]          (54-entry star pattern)
//       b[p,l,u] -= sum_m Khat^j_lm X[p,m,u], l < o_g (sparse rows of Khat^j)
// then the time integration I = dt Qt[:, :, 0] (int_0^1 chi_s = delta_s0).
//
// GB300's binary64 pipe is narrow, so the design minimises binary64
// instructions: only structural non-zeros of Khat and of the stars are
// touched, and the Khat row index is warp-uniform (lanes run over the 13 T
// (p, u) pairs of one row, padded to a multiple of 32) so every lane of a
// warp-wide FMA does useful work.
#include <cuda_runtime.h>

#include "alg3_device.cuh"

namespace poro {
namespace {

struct K1Params {
    const int32_t* elems;  // optional element index list (LTS clusters); nullptr: elements 0..count-1
    const double* q0;
    const double* econst;
    double* qt;
    double* iout;
    int64_t count;
    int stride;
    KhatBlocks<double> khat;
    const double* zinv;
    const RunPtrs* runs;       // items of several runs (nullptr: the pointers above)
    const int32_t* item_run;
};

// CTA sizes the autotuner chooses from (index 0 is the default)
template <int N>
struct K1Sizes {
    static constexpr int NT0 = N >= 5 ? 256 : (N == 4 ? 128 : 64);
    static constexpr int NT1 = N >= 5 ? 128 : (N == 4 ? 256 : 128);
};

template <int N, int NT_, class Sys = BiotSystem>
struct K1Shape : Alg3Shape<N, Sys::NQ> {
    using A = Alg3Shape<N, Sys::NQ>;
    static constexpr int NT = NT_;
    static constexpr int T_ = N + 1;
    // shared layout (doubles): bq[NQ*QS] | X[NQ*XSMAX] | star[3*NNZ] |
    // zsh[NSHM*T*T] | sc[NSC] | zin[T*T]; star .. sc are the element's
    // constants in their global order (EC words)
    static constexpr int OFF_X = A::SQ;
    static constexpr int OFF_STAR = OFF_X + Sys::NQ * A::XSMAX;
    static constexpr int OFF_ZUF = OFF_STAR + 3 * Sys::NNZ;
    static constexpr int OFF_SC = OFF_ZUF + Sys::NSHM * T_ * T_;
    static constexpr int OFF_ZIN = OFF_SC + Sys::NSC;
    static constexpr int EC = OFF_ZIN - OFF_STAR;
    static constexpr int SMEM_DOUBLES = OFF_ZIN + T_ * T_;
};

template <int N, int NT_, class Sys = BiotSystem>
__global__ void __launch_bounds__(NT_) stp_fp64_kernel(const K1Params P) {
    using S = K1Shape<N, NT_, Sys>;
    constexpr int NQ = Sys::NQ;
    constexpr int B = S::B, T = S::T, NT = S::NT, QS = S::QS;
    extern __shared__ double sm[];
    double* bq = sm;
    double* X = sm + S::OFF_X;
    double* star = sm + S::OFF_STAR;
    double* zuf = sm + S::OFF_ZUF;
    double* sc = sm + S::OFF_SC;
    double* zin = sm + S::OFF_ZIN;
    const int tid = threadIdx.x;

    for (int64_t it = blockIdx.x; it < P.count; it += gridDim.x) {
        const int64_t e = P.elems ? (int64_t)P.elems[it] : it;
        RunPtrs R{P.q0, P.econst, P.qt, P.iout};
        if (P.runs) R = P.runs[P.item_run[it]];
        const double* q0 = R.q0 + e * (int64_t)(NQ * B);
        const double* ec = R.econst + e * (int64_t)P.stride;
        // element constants: stars, shifted time matrices and scalars are contiguous
        for (int i = tid; i < S::EC; i += NT) star[i] = ec[i];
        for (int i = tid; i < T * T; i += NT) zin[i] = P.zinv[i];
        init_rhs<N, NT, double, double, NQ>(bq, q0);
        __syncthreads();
        alg3_sweep<N, NT, double, 1, Sys>(bq, X, star, zuf, zin, sc[1], P.khat, sc);
        // time integration and outputs (global layout [p][l][u], dense)
        const double dt = sc[Sys::DT_SC];
        if (R.iout) {
            double* io = R.iout + e * (int64_t)(NQ * B);
            for (int i = tid; i < NQ * B; i += NT) io[i] = dt * bq[(i / B) * QS + (i % B) * T];
        }
        if (R.qt) {
            double* qo = R.qt + e * (int64_t)S::QBT;
            for (int i = tid; i < S::QBT; i += NT) qo[i] = bq[(i / (B * T)) * QS + i % (B * T)];
        }
        __syncthreads();
    }
}

template <int N, int NT_, class Sys = BiotSystem>
int launch_nt(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
              const double* econst, double* qt, double* iout, void* stream, const RunPtrs* runs,
              const int32_t* item_run) {
    using S = K1Shape<N, NT_, Sys>;
    K1Params P;
    P.elems = elems;
    P.q0 = q0;
    P.econst = econst;
    P.qt = qt;
    P.iout = iout;
    P.count = count;
    P.stride = Sys::NQ == NQ ? elem_const_stride(N)
               : Sys::NQ == maxwell::NQ ? maxwell::elem_const_stride(N) : visco::elem_const_stride(N);
    P.khat.val = ref.khat_val;
    P.khat.col = ref.khat_col;
    P.khat.row = ref.khat_row;
    for (int g = 0; g <= MAX_N; ++g)
        for (int j = 0; j < 3; ++j) P.khat.row_base[g][j] = ref.row_base[g][j];
    constexpr int W = NT_ == 256 ? 2 : (NT_ == 128 ? 1 : 0);  // lists for NT_ / 32 warps
    static_assert(NT_ == 64 || NT_ == 128 || NT_ == 256, "2, 4 or 8 warps");
    P.khat.lists = ref.lists[W];
    for (int g = 0; g <= MAX_N; ++g)
        for (int j = 0; j < 3; ++j) P.khat.list_base[g][j] = ref.list_base[W][g][j];
    P.zinv = ref.zinv;
    P.runs = runs;
    P.item_run = item_run;
    const size_t smem = sizeof(double) * S::SMEM_DOUBLES;
    cudaError_t err = cudaFuncSetAttribute(stp_fp64_kernel<N, NT_, Sys>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    if (count <= 0) return 0;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    stp_fp64_kernel<N, NT_, Sys><<<(unsigned)grid, S::NT, smem, (cudaStream_t)stream>>>(P);
    return (int)cudaGetLastError();
}

template <int N>
int launch_n(const DeviceReference& ref, int variant, const int32_t* elems, int64_t count, const double* q0,
             const double* econst, double* qt, double* iout, void* stream, const RunPtrs* runs,
             const int32_t* item_run) {
    if (variant == 1)
        return launch_nt<N, K1Sizes<N>::NT1>(ref, elems, count, q0, econst, qt, iout, stream, runs, item_run);
    return launch_nt<N, K1Sizes<N>::NT0>(ref, elems, count, q0, econst, qt, iout, stream, runs, item_run);
}

}  // namespace

int launch_stp_fp64_maxwell(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
                            const double* econst, double* qt, double* iout, void* stream) {
    // 6 quantities: 2 warps cover the 6 T (p, u) pairs of a mode at every N
    switch (ref.N) {
        case 1: return launch_nt<1, 64, MaxwellSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 2: return launch_nt<2, 64, MaxwellSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 3: return launch_nt<3, 64, MaxwellSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 4: return launch_nt<4, 128, MaxwellSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr,
                                                        nullptr);
        case 5: return launch_nt<5, 128, MaxwellSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr,
                                                        nullptr);
        case 6: return launch_nt<6, 128, MaxwellSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr,
                                                        nullptr);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_stp_fp64_visco(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
                          const double* econst, double* qt, double* iout, void* stream) {
    // 27 quantities: the (p, u) pairs of a mode span 1 to 6 lanes per warp
    switch (ref.N) {
        case 1: return launch_nt<1, 64, ViscoSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 2: return launch_nt<2, 64, ViscoSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 3: return launch_nt<3, 128, ViscoSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 4: return launch_nt<4, 128, ViscoSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 5: return launch_nt<5, 256, ViscoSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        case 6: return launch_nt<6, 256, ViscoSystem>(ref, elems, count, q0, econst, qt, iout, stream, nullptr, nullptr);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_stp_fp64(const DeviceReference& ref, const int32_t* elems, int64_t count, const double* q0,
                    const double* econst, double* qt, double* iout, void* stream, int variant, const RunPtrs* runs,
                    const int32_t* item_run) {
    switch (ref.N) {
        case 1: return launch_n<1>(ref, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 2: return launch_n<2>(ref, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 3: return launch_n<3>(ref, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 4: return launch_n<4>(ref, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 5: return launch_n<5>(ref, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 6: return launch_n<6>(ref, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace poro
