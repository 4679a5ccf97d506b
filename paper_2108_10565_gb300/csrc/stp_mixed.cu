// K2: mixed-precision space-time predictor with iterative refinement.
//
// Solves the predictor system of one element (Eq. stp-lineq, in the scaled
// form of Section "Block-wise back-substitution":
//   (Z (x) I - E* + sum_j A^{j*} (x) Khat^j) Q = (S^{-1} w) o Q0 )
// as
//   Q1 = Alg3_f32(b0)                      binary32 back-substitution
//   r  = b0 - Y Q1                         residual, double-binary32 exact
//   d  = Alg3_f32(fl32(r));  Q = Q1 + d    (one sweep; a second repeats with
//                                           Q1 + d in the residual)
// The binary32 sweeps are Algorithm 3 (degree blocks, time solves with
// (Z - E*_pp I)^{-1}, G coupling, star and Khat products) in float.  The
// residual needs ~47 significant bits because Y Q1 cancels b0 to ~1e-7; GB300
// issues binary64 FMAs at ~1/60 of its binary32 rate, so the residual runs on
// the binary32 pipe with error-free transformations: FMA-based exact products
// (p + e = a*b) and Knuth's TwoSum, accumulating pairs (hi, lo) as in the
// double-word dot product of Ogita, Rump and Oishi (2005).  Every product of
// the residual is formed exactly from double-word operands (Khat, A*, E* split
// into hi + lo binary32 words; Z's entries are small integers, exact).
//
// Residual layout: one warp per Khat row l (rows round-robin over warps).
//   R1: lanes over the 13 T (q, u) pairs: Y^j[q,u] = sum_m Khat^j[l,m] Q[q,m,u]
//   R2: lanes over the (p, u) pairs: r[p,l,u] = b0 - sum_s Z_us Q[p,l,s]
//       + E*_pp Q[p,l,u] + G Q[uf,l,u] - sum_j sum_q A^{j*}_pq Y^j[q,u]
#include <cuda_runtime.h>

#include "alg3_device.cuh"

namespace poro {
namespace {

struct K2Params {
    const int32_t* elems;     // optional element index list (LTS clusters)
    const double* q0;
    const double* econst;
    double* qt;
    double* iout;
    int64_t count;
    int stride;
    KhatBlocks<float> khat;   // block CSR, binary32 values (for the sweeps)
    const int32_t* res_row;   // [3][B+1] full-row CSR of Khat^j (absolute offsets)
    const int32_t* res_col;   // column m
    const float2* res_val;    // Khat value split (hi, lo)
    const float* zinv;        // Z^{-1} [T][T] binary32
};

// star pattern tables for lane-varying lookups (copied to shared memory)
__constant__ int c_star_tab[NQ + 1 + STAR_NNZ] = {
    0, 6, 12, 18, 20, 22, 24, 28, 32, 36, 42, 46, 50, 54,
    QU, QV, QW, QUF, QVF, QWF, QU, QV, QW, QUF, QVF, QWF, QU, QV, QW, QUF, QVF, QWF,
    QU, QV, QV, QW, QU, QW,
    SXX, SXY, SXZ, QP, SYY, SXY, SYZ, QP, SZZ, SXZ, SYZ, QP,
    QU, QV, QW, QUF, QVF, QWF,
    SXX, SXY, SXZ, QP, SYY, SXY, SYZ, QP, SZZ, SXZ, SYZ, QP};

// ------------------------------------------------ error-free double-word ops
// Explicit round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the transformations.
__device__ __forceinline__ void dw_mac(float& h, float& l, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(er, e));
}

// acc += a * b with b a single binary32 word
__device__ __forceinline__ void dw_mac1(float& h, float& l, float ah, float al, float b) {
    const float p = __fmul_rn(ah, b);
    float e = __fmaf_rn(ah, b, -p);
    e = __fmaf_rn(al, b, e);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(er, e));
}

__device__ __forceinline__ float2 dw_split(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// CTA sizes the autotuner chooses from (index 0 is the default)
template <int N>
struct K2Sizes {
    static constexpr int NT0 = N >= 5 ? 256 : (N == 4 ? 128 : 64);
    static constexpr int NT1 = N >= 5 ? 128 : (N == 4 ? 256 : 128);
};

template <int N, int REF, int NT_>
struct K2Shape : Alg3Shape<N> {
    using A = Alg3Shape<N>;
    static constexpr int NT = NT_;
    static constexpr int NW = NT / 32;
    static constexpr int T_ = N + 1;
    static constexpr int R4(int x) { return (x + 3) & ~3; }
    static constexpr int MAX2(int a, int b) { return a > b ? a : b; }
    // shared layout in floats; the star products X of the sweeps (3 directions)
    // and the per-warp Y buffers of the residual share one region
    static constexpr int OFF_W = 0;
    static constexpr int OFF_Q1 = R4(A::SQ);
    static constexpr int OFF_D1 = OFF_Q1 + R4(A::SQ);
    static constexpr int OFF_XY = OFF_D1 + (REF == 2 ? R4(A::SQ) : 0);
    static constexpr int XY_SIZE = R4(MAX2(3 * NQ * A::XSMAX, NW * 3 * A::PT * 2));
    static constexpr int OFF_B0 = OFF_XY + XY_SIZE;
    static constexpr int OFF_SH = OFF_B0 + R4(2 * NQ * A::B);
    static constexpr int OFF_SL = OFF_SH + R4(3 * STAR_NNZ);
    static constexpr int OFF_ZIN = OFF_SL + R4(3 * STAR_NNZ);
    static constexpr int OFF_ZUF = OFF_ZIN + R4(T_ * T_);
    static constexpr int OFF_ZI = OFF_ZUF + R4(T_ * T_);
    static constexpr int OFF_TAB = OFF_ZI + R4(T_ * T_);   // ints: row_ptr[14], col[54]
    static constexpr int SMEM_FLOATS = OFF_TAB + R4(NQ + 1 + STAR_NNZ);
};

template <int N, int REF, int NT_>
__device__ void residual(float* W, const float* Q1, const float* D1, const float2* b0, const float* sh,
                         const float* sl, const float* zi, const int* tab, float2 e_dw, float2 g_dw, float2* Yall,
                         const K2Params& P) {
    using S = K2Shape<N, REF, NT_>;
    constexpr int B = S::B, T = S::T, PT = S::PT, PUL = S::PUL, QS = S::QS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* Y = Yall + warp * 3 * PT;
    const int* srp = tab;
    const int* scol = tab + NQ + 1;
#pragma unroll 1
    for (int l = warp; l < B; l += S::NW) {
        // R1: Y^j[q, u] = sum_m Khat^j[l, m] Q[q, m, u]
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            float yh[PUL], yl[PUL];
            int off[PUL];
#pragma unroll
            for (int k = 0; k < PUL; ++k) {
                yh[k] = yl[k] = 0.f;
                const int pu = lane + 32 * k;
                const int q = pu / T, u = pu % T;
                off[k] = pu < PT ? q * QS + u : 0;
            }
            const int n0 = __ldg(P.res_row + j * (B + 1) + l), n1 = __ldg(P.res_row + j * (B + 1) + l + 1);
            for (int n = n0; n < n1; ++n) {
                const float2 kv = __ldg(P.res_val + n);
                const int mo = __ldg(P.res_col + n) * T;
#pragma unroll
                for (int k = 0; k < PUL; ++k) {
                    const int a = off[k] + mo;
                    if (REF == 2)
                        dw_mac(yh[k], yl[k], kv.x, kv.y, Q1[a], D1[a]);
                    else
                        dw_mac1(yh[k], yl[k], kv.x, kv.y, Q1[a]);
                }
            }
#pragma unroll
            for (int k = 0; k < PUL; ++k) {
                const int pu = lane + 32 * k;
                if (pu < PT) Y[j * PT + pu] = make_float2(yh[k], yl[k]);
            }
        }
        __syncwarp();
        // R2: assemble r[p, l, u]
#pragma unroll
        for (int k = 0; k < PUL; ++k) {
            const int pu = lane + 32 * k;
            if (pu < PT) {
                const int p = pu / T, u = pu % T;
                const int base = p * QS + l * T;
                float h = 0.f, lo = 0.f;
                const float2 bv = b0[p * B + l];
                const float sw = (float)((2 * u + 1) * ((u & 1) ? -1 : 1));
                dw_mac(h, lo, sw, 0.f, bv.x, bv.y);
                // - sum_s Z_us Q[p, l, s]   (Z entries are exact small integers)
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    if (REF == 2)
                        dw_mac(h, lo, -zi[u * T + s], 0.f, Q1[base + s], D1[base + s]);
                    else
                        dw_mac1(h, lo, -zi[u * T + s], 0.f, Q1[base + s]);
                }
                // + E*_pp Q[p, l, u] (u_f rows) and + G Q[u_f, l, u] (u rows)
                if (p >= QUF || (p >= QU && p <= QW)) {
                    const int src = p >= QUF ? base + u : (p + 4) * QS + l * T + u;
                    const float2 c = p >= QUF ? e_dw : g_dw;
                    if (REF == 2)
                        dw_mac(h, lo, c.x, c.y, Q1[src], D1[src]);
                    else
                        dw_mac1(h, lo, c.x, c.y, Q1[src]);
                }
                // - sum_j sum_q A^{j*}_pq Y^j[q, u]
                const int r0 = srp[p], r1 = srp[p + 1];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
#pragma unroll
                    for (int t = 0; t < 6; ++t) {
                        const int idx = r0 + t;
                        if (idx < r1) {
                            const float2 yv = Y[j * PT + scol[idx] * T + u];
                            dw_mac(h, lo, -sh[j * STAR_NNZ + idx], -sl[j * STAR_NNZ + idx], yv.x, yv.y);
                        }
                    }
                }
                W[base + u] = __fadd_rn(h, lo);
            }
        }
        __syncwarp();
    }
}

template <int N, int REF, int NT_>
__global__ void __launch_bounds__(NT_, (REF == 2 || NT_ > 256) ? 1 : 2) stp_mixed_kernel(const K2Params P) {
    using S = K2Shape<N, REF, NT_>;
    constexpr int B = S::B, T = S::T, NT = S::NT, QBT = S::QBT, QS = S::QS;
    extern __shared__ float smf[];
    float* W = smf + S::OFF_W;
    float* Q1 = smf + S::OFF_Q1;
    float* D1 = smf + S::OFF_D1;
    float* X = smf + S::OFF_XY;
    float2* Yall = reinterpret_cast<float2*>(smf + S::OFF_XY);
    float2* b0 = reinterpret_cast<float2*>(smf + S::OFF_B0);
    float* sh = smf + S::OFF_SH;
    float* sl = smf + S::OFF_SL;
    float* zin = smf + S::OFF_ZIN;
    float* zuf = smf + S::OFF_ZUF;
    float* zi = smf + S::OFF_ZI;
    int* tab = reinterpret_cast<int*>(smf + S::OFF_TAB);
    const int tid = threadIdx.x;

    for (int i = tid; i < T * T; i += NT) {
        zin[i] = P.zinv[i];
        const int u = i / T, s = i % T;
        zi[i] = (float)((2 * u + 1) * ((u > s && ((u - s) & 1)) ? -1 : 1));  // Z = S^{-1}(W - K^tau)
    }
    for (int i = tid; i < NQ + 1 + STAR_NNZ; i += NT) tab[i] = c_star_tab[i];

    for (int64_t it = blockIdx.x; it < P.count; it += gridDim.x) {
        const int64_t e = P.elems ? (int64_t)P.elems[it] : it;
        const double* q0 = P.q0 + e * (int64_t)(NQ * B);
        const double* ec = P.econst + e * (int64_t)P.stride;
        for (int i = tid; i < 3 * STAR_NNZ; i += NT) {
            const float2 v = dw_split(ec[i]);
            sh[i] = v.x;
            sl[i] = v.y;
        }
        for (int i = tid; i < T * T; i += NT) zuf[i] = (float)ec[ec_zinv(N) + i];
        const double* scal = ec + 3 * STAR_NNZ + T * T;
        const float2 e_dw = dw_split(scal[0]), g_dw = dw_split(scal[1]);
        const double dt = scal[2];
        for (int i = tid; i < NQ * B; i += NT) b0[i] = dw_split(q0[i]);
        __syncthreads();
        // Q1 = Alg3_f32(b0)
        for (int i = tid; i < NQ * B; i += NT) {
            const float v = b0[i].x;
            float* row = W + (i / B) * QS + (i % B) * T;
#pragma unroll
            for (int u = 0; u < T; ++u) row[u] = (float)((2 * u + 1) * ((u & 1) ? -1 : 1)) * v;
        }
        __syncthreads();
        alg3_sweep<N, NT, float, 3>(W, X, sh, zuf, zin, g_dw.x, P.khat);
        for (int i = tid; i < S::SQ; i += NT) {
            Q1[i] = W[i];
            if (REF == 2) D1[i] = 0.f;
        }
        __syncthreads();
#pragma unroll 1
        for (int sweep = 1; sweep <= REF; ++sweep) {
            residual<N, REF, NT_>(W, Q1, D1, b0, sh, sl, zi, tab, e_dw, g_dw, Yall, P);
            __syncthreads();
            alg3_sweep<N, NT, float, 3>(W, X, sh, zuf, zin, g_dw.x, P.khat);
            if (REF == 2 && sweep == 1) {
                for (int i = tid; i < S::SQ; i += NT) D1[i] = W[i];
                __syncthreads();
            }
        }
        // Q = Q1 (+ d1) (+ d2) in binary64; time integration
        if (P.qt || P.iout) {
            double* qo = P.qt ? P.qt + e * (int64_t)QBT : nullptr;
            double* io = P.iout ? P.iout + e * (int64_t)(NQ * B) : nullptr;
            for (int i = tid; i < QBT; i += NT) {
                const int si = (i / (B * T)) * QS + i % (B * T);
                double v = (double)Q1[si];
                if (REF == 2) v += (double)D1[si];
                if (REF >= 1) v += (double)W[si];
                if (qo) qo[i] = v;
                if (io && (i % T) == 0) io[i / T] = dt * v;
            }
        }
        __syncthreads();
    }
}

template <int N, int REF, int NT_>
int launch_nr(const MixedReference& ref, const int32_t* elems, int64_t count, const double* q0, const double* econst,
              double* qt, double* iout, void* stream) {
    using S = K2Shape<N, REF, NT_>;
    K2Params P;
    P.elems = elems;
    P.q0 = q0;
    P.econst = econst;
    P.qt = qt;
    P.iout = iout;
    P.count = count;
    P.stride = elem_const_stride(N);
    P.khat.val = ref.khat_val_f32;
    P.khat.col = ref.base->khat_col;
    P.khat.row = ref.base->khat_row;
    for (int g = 0; g <= MAX_N; ++g)
        for (int j = 0; j < 3; ++j) P.khat.row_base[g][j] = ref.base->row_base[g][j];
    P.res_row = ref.res_row;
    P.res_col = ref.res_col;
    P.res_val = reinterpret_cast<const float2*>(ref.res_val);
    P.zinv = ref.zinv_f32;
    const size_t smem = sizeof(float) * S::SMEM_FLOATS;
    cudaError_t err = cudaFuncSetAttribute(stp_mixed_kernel<N, REF, NT_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return (int)err;
    if (count <= 0) return 0;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    stp_mixed_kernel<N, REF, NT_><<<(unsigned)grid, S::NT, smem, (cudaStream_t)stream>>>(P);
    return (int)cudaGetLastError();
}

template <int N, int NT_>
int launch_nv(const MixedReference& ref, int refine, const int32_t* elems, int64_t count, const double* q0,
              const double* econst, double* qt, double* iout, void* stream) {
    switch (refine) {
        case 0: return launch_nr<N, 0, NT_>(ref, elems, count, q0, econst, qt, iout, stream);
        case 1: return launch_nr<N, 1, NT_>(ref, elems, count, q0, econst, qt, iout, stream);
        case 2: return launch_nr<N, 2, NT_>(ref, elems, count, q0, econst, qt, iout, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <int N>
int launch_n(const MixedReference& ref, int refine, int variant, const int32_t* elems, int64_t count,
             const double* q0, const double* econst, double* qt, double* iout, void* stream) {
    if (variant == 1)
        return launch_nv<N, K2Sizes<N>::NT1>(ref, refine, elems, count, q0, econst, qt, iout, stream);
    return launch_nv<N, K2Sizes<N>::NT0>(ref, refine, elems, count, q0, econst, qt, iout, stream);
}

}  // namespace

int launch_stp_mixed(const MixedReference& ref, int refine, const int32_t* elems, int64_t count, const double* q0,
                     const double* econst, double* qt, double* iout, void* stream, int variant) {
    switch (ref.base->N) {
        case 1: return launch_n<1>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream);
        case 2: return launch_n<2>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream);
        case 3: return launch_n<3>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream);
        case 4: return launch_n<4>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream);
        case 5: return launch_n<5>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream);
        case 6: return launch_n<6>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace poro
