// K11: the space-time predictor with sub-cell material variation (Section
// "Limitations": material varying inside an element turns the stiffness
// matrices into 3-tensors), in binary64, one element per CTA.
//
// The element's Jacobians and source matrix vary linearly inside it:
// A^{j*}(xi) = sum_r A^{j*}_r phi_r(xi), E*(xi) = sum_r E*_r phi_r(xi) over the
// four Dubiner modes of degree <= 1.  With the M^{-1}-scaled mass 3-tensor
// Mh3_r[k, l] = int phi_k phi_r phi_l / M_kk, the weighted derivative tensor is
// Mh3_r Khat^j (d_j phi_l lies in the basis), so the system is
//   Y Q = Y_0 Q + sum_{r>=1} Mh3_r (sum_j Khat^j (A^{j*}_r Q) - E*_r Q) = b0,
// Y_0 the constant-material operator of the mode-0 (mean) Jacobians, which
// Algorithm 3 solves.  A material of degree 1 couples modes of equal degree,
// so Lemma 1's block structure does not hold for Y itself; the kernel iterates
//   Q_{k+1} = Y_0^{-1} (b0 - Delta Q_k),  Delta = Y - Y_0,
// (Richardson iteration preconditioned by Algorithm 3 on the mean material)
// until max |Q_{k+1} - Q_k| <= tol max |Q_{k+1}|, at most max_iter times.
// The contraction factor is about the relative variation of the material
// inside the element.
//
// Shared memory (doubles): U (iterate), V (right-hand side, then the next
// iterate) and W (one variation term) in the b / Q layout of Algorithm 3, the
// star scratch X, the mean element constants, the variation stars and the
// reduction words.
#include <cuda_runtime.h>

#include "alg3_device.cuh"

namespace poro {
namespace {

struct SubParams {
    const double* q0;
    const double* econst;  // mean-material constants (the layout of the FP64 predictor)
    const double* evar;    // per element: star_r[3][3][54] for r = 1..3, then (e_r, g_r) for r = 1..3
    double* qt;
    double* iout;
    int32_t* iters;        // per element: iterations, negative if not converged
    int64_t count;
    int stride, vstride;
    KhatBlocks<double> khat;
    const double* zinv;
    const int32_t* m3_row;  // [3][B + 1], absolute into m3_col / m3_val
    const int32_t* m3_col;
    const double* m3_val;
    double tol;
    int max_iter;
};

constexpr int NVAR = 3;  // variation modes r = 1..3

template <int N, int NT_>
struct SubShape : Alg3Shape<N> {
    using A = Alg3Shape<N>;
    static constexpr int NT = NT_, NW = NT_ / 32;
    static constexpr int T_ = N + 1;
    static constexpr int OFF_V = A::SQ;
    static constexpr int OFF_W = 2 * A::SQ;
    static constexpr int OFF_X = 3 * A::SQ;
    static constexpr int OFF_STAR = OFF_X + NQ * A::XSMAX;       // mean constants: star, zuf, sc (EC words)
    static constexpr int EC = 3 * STAR_NNZ + T_ * T_ + 4;
    static constexpr int OFF_ZIN = OFF_STAR + EC;
    static constexpr int OFF_VAR = OFF_ZIN + T_ * T_;             // variation stars and (e_r, g_r)
    static constexpr int VAR = NVAR * 3 * STAR_NNZ + 2 * NVAR;
    static constexpr int OFF_RED = OFF_VAR + VAR;                 // 2 NW reduction words
    static constexpr int SMEM_DOUBLES = OFF_RED + 2 * NW;
};

// W <- -E*_r U (source variation): u_f rows e_r U_uf, u rows g_r U_uf
template <int N, int NT>
__device__ void source_term(double* W, const double* U, double e, double g) {
    using S = Alg3Shape<N>;
    constexpr int QS = S::QS, BT = S::B * S::T;
    for (int i = threadIdx.x; i < NQ * BT; i += NT) {
        const int p = i / BT, m = i - p * BT;
        double v = 0.0;
        if (p >= QUF) v = -e * U[p * QS + m];
        else if (p >= QU && p <= QW) v = -g * U[(p + QUF - QU) * QS + m];
        W[p * QS + m] = v;
    }
}

// W += sum_j Khat^j (A^{j*}_r U) over all degree blocks (strictly upper in
// degree: rows l < o_g take column block g); ends with a barrier
template <int N, int NT>
__device__ void flux_term(double* W, double* X, const double* U, const double* starr, const KhatBlocks<double>& K) {
    using S = Alg3Shape<N>;
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
    for (int g = 1; g <= N; ++g) {
        const int o = block_offset(g), d = block_size(g);
        const int XS = bank_stride(d * T, T);
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            const double* sj = starr + j * STAR_NNZ;
            for (int it = tid; it < d * T; it += NT) {
                const int ml = it / T, u = it % T;
                double qv[NQ], acc[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) qv[q] = U[q * QS + (o + ml) * T + u];
#pragma unroll
                for (int p = 0; p < NQ; ++p) acc[p] = 0.0;
#pragma unroll
                for (int n = 0; n < STAR_NNZ; ++n) acc[star_row(n)] = fma(sj[n], qv[star_col(n)], acc[star_row(n)]);
#pragma unroll
                for (int p = 0; p < NQ; ++p) X[p * XS + ml * T + u] = acc[p];
            }
            __syncthreads();
            for (int l = warp; l < o; l += NW) {
                const int32_t* rp = K.row + K.row_base[g][j] + l;
                const int n0 = __ldg(rp), n1 = __ldg(rp + 1);
                double acc[PUL];
#pragma unroll
                for (int k = 0; k < PUL; ++k) acc[k] = 0.0;
                for (int n = n0; n < n1; ++n) {
                    const double v = __ldg(K.val + n);
                    const int m = __ldg(K.col + n) * T;
#pragma unroll
                    for (int k = 0; k < PUL; ++k) acc[k] = fma(v, X[lp[k] * XS + lu[k] + m], acc[k]);
                }
#pragma unroll
                for (int k = 0; k < PUL; ++k)
                    if (lane + 32 * k < PT) W[lp[k] * QS + l * T + lu[k]] += acc[k];
            }
            __syncthreads();
        }
    }
}

// V -= Mh3_r W (all rows k); ends with a barrier
template <int N, int NT>
__device__ void mass_term(double* V, const double* W, const int32_t* row, const int32_t* col, const double* val) {
    using S = Alg3Shape<N>;
    constexpr int B = S::B, T = S::T, QS = S::QS, PT = S::PT, PUL = S::PUL, NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k < B; k += NW) {
        const int n0 = __ldg(row + k), n1 = __ldg(row + k + 1);
        double acc[PUL];
#pragma unroll
        for (int q = 0; q < PUL; ++q) acc[q] = 0.0;
        for (int n = n0; n < n1; ++n) {
            const double v = __ldg(val + n);
            const int l = __ldg(col + n) * T;
#pragma unroll
            for (int q = 0; q < PUL; ++q) {
                const int pu = lane + 32 * q;
                if (pu < PT) acc[q] = fma(v, W[(pu / T) * QS + l + pu % T], acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < PUL; ++q) {
            const int pu = lane + 32 * q;
            if (pu < PT) V[(pu / T) * QS + k * T + pu % T] -= acc[q];
        }
    }
    __syncthreads();
}

template <int N, int NT_>
__global__ void __launch_bounds__(NT_) stp_subcell_kernel(const SubParams P) {
    using S = SubShape<N, NT_>;
    constexpr int B = S::B, T = S::T, NT = S::NT, NW = S::NW, QS = S::QS, BT = B * T;
    extern __shared__ double sm[];
    double* bufs[2] = {sm, sm + S::OFF_V};
    double* W = sm + S::OFF_W;
    double* X = sm + S::OFF_X;
    double* star = sm + S::OFF_STAR;
    double* zuf = star + 3 * STAR_NNZ;
    double* sc = zuf + T * T;
    double* zin = sm + S::OFF_ZIN;
    double* var = sm + S::OFF_VAR;
    double* red = sm + S::OFF_RED;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int64_t e = blockIdx.x; e < P.count; e += gridDim.x) {
        const double* q0 = P.q0 + e * (int64_t)(NQ * B);
        const double* ec = P.econst + e * (int64_t)P.stride;
        const double* ev = P.evar + e * (int64_t)P.vstride;
        for (int i = tid; i < S::EC; i += NT) star[i] = ec[i];
        for (int i = tid; i < T * T; i += NT) zin[i] = P.zinv[i];
        for (int i = tid; i < S::VAR; i += NT) var[i] = ev[i];
        double* U = bufs[0];
        double* V = bufs[1];
        init_rhs<N, NT, double, double>(U, q0);
        __syncthreads();
        alg3_sweep<N, NT, double, 1>(U, X, star, zuf, zin, sc[1], P.khat);  // Q_0 = Y_0^{-1} b0
        int it = 0;
        bool converged = false, stop = false;
        while (it < P.max_iter && !stop) {
            ++it;
            init_rhs<N, NT, double, double>(V, q0);
            for (int r = 0; r < NVAR; ++r) {
                source_term<N, NT>(W, U, var[NVAR * 3 * STAR_NNZ + 2 * r], var[NVAR * 3 * STAR_NNZ + 2 * r + 1]);
                __syncthreads();
                flux_term<N, NT>(W, X, U, var + r * 3 * STAR_NNZ, P.khat);
                mass_term<N, NT>(V, W, P.m3_row + r * (B + 1), P.m3_col, P.m3_val);
            }
            alg3_sweep<N, NT, double, 1>(V, X, star, zuf, zin, sc[1], P.khat);  // Q_{k+1}
            // max |Q_{k+1} - Q_k| and max |Q_{k+1}| over the element
            double dmax = 0.0, vmax = 0.0;
            for (int i = tid; i < NQ * BT; i += NT) {
                const int p = i / BT, m = i - p * BT;
                const double v = V[p * QS + m];
                dmax = fmax(dmax, fabs(v - U[p * QS + m]));
                vmax = fmax(vmax, fabs(v));
            }
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, s));
                vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, s));
            }
            if (lane == 0) {
                red[warp] = dmax;
                red[NW + warp] = vmax;
            }
            __syncthreads();
            dmax = 0.0;
            vmax = 0.0;
            for (int w = 0; w < NW; ++w) {
                dmax = fmax(dmax, red[w]);
                vmax = fmax(vmax, red[NW + w]);
            }
            // a non-finite iterate stops the loop unconverged (and is written out as it is)
            const bool finite = isfinite(dmax) && isfinite(vmax);
            converged = finite && dmax <= P.tol * vmax;
            stop = converged || !finite;
            double* t = U;
            U = V;
            V = t;
            __syncthreads();
        }
        const double dt = sc[2];
        double* io = P.iout ? P.iout + e * (int64_t)(NQ * B) : nullptr;
        double* qo = P.qt ? P.qt + e * (int64_t)S::QBT : nullptr;
        if (io)
            for (int i = tid; i < NQ * B; i += NT) io[i] = dt * U[(i / B) * QS + (i % B) * T];
        if (qo)
            for (int i = tid; i < S::QBT; i += NT) qo[i] = U[(i / BT) * QS + i % BT];
        if (tid == 0 && P.iters) P.iters[e] = converged ? it : -it;
        __syncthreads();
    }
}

template <int N, int NT_>
int launch_sub(const DeviceReference& ref, const SubcellReference& sub, int64_t count, const double* q0,
               const double* econst, const double* evar, double* qt, double* iout, int32_t* iters, double tol,
               int max_iter, void* stream) {
    using S = SubShape<N, NT_>;
    SubParams P;
    P.q0 = q0;
    P.econst = econst;
    P.evar = evar;
    P.qt = qt;
    P.iout = iout;
    P.iters = iters;
    P.count = count;
    P.stride = elem_const_stride(N);
    P.vstride = subcell_var_stride();
    P.khat.val = ref.khat_val;
    P.khat.col = ref.khat_col;
    P.khat.row = ref.khat_row;
    for (int g = 0; g <= MAX_N; ++g)
        for (int j = 0; j < 3; ++j) P.khat.row_base[g][j] = ref.row_base[g][j];
    P.khat.lists = nullptr;
    P.zinv = ref.zinv;
    P.m3_row = sub.m3_row;
    P.m3_col = sub.m3_col;
    P.m3_val = sub.m3_val;
    P.tol = tol;
    P.max_iter = max_iter;
    const size_t smem = sizeof(double) * S::SMEM_DOUBLES;
    cudaError_t err = cudaFuncSetAttribute(stp_subcell_kernel<N, NT_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return (int)err;
    if (count <= 0) return 0;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    stp_subcell_kernel<N, NT_><<<(unsigned)grid, NT_, smem, (cudaStream_t)stream>>>(P);
    return (int)cudaGetLastError();
}

}  // namespace

int launch_stp_subcell(const DeviceReference& ref, const SubcellReference& sub, int64_t count, const double* q0,
                       const double* econst, const double* evar, double* qt, double* iout, int32_t* iters,
                       double tol, int max_iter, void* stream) {
    switch (ref.N) {
        case 1: return launch_sub<1, 128>(ref, sub, count, q0, econst, evar, qt, iout, iters, tol, max_iter, stream);
        case 2: return launch_sub<2, 128>(ref, sub, count, q0, econst, evar, qt, iout, iters, tol, max_iter, stream);
        case 3: return launch_sub<3, 128>(ref, sub, count, q0, econst, evar, qt, iout, iters, tol, max_iter, stream);
        case 4: return launch_sub<4, 256>(ref, sub, count, q0, econst, evar, qt, iout, iters, tol, max_iter, stream);
        case 5: return launch_sub<5, 256>(ref, sub, count, q0, econst, evar, qt, iout, iters, tol, max_iter, stream);
        case 6: return launch_sub<6, 256>(ref, sub, count, q0, econst, evar, qt, iout, iters, tol, max_iter, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace poro
