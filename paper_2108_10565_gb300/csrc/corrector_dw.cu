// Corrector of the ADER-DG scheme in double-binary32 arithmetic (contexts of
// the mixed-precision form).  Same operator as the binary64 corrector
// (Eq. semi_discrete integrated over one step, Section "Temporal
// discretisation with ADER"):
//   dQ_pk = sum_j sum_l Kv^j_kl (A^j I)_pl + (E I)_pk
//         - sum_f c_f / M_kk [ sum_l Floc^f_kl (F^- I^e)_pl
//                            + sum_l Fnb^{f,h,s}_kl (F^+ I^nb)_pl ]
// with every operand split into (hi, lo) binary32 words and every product and
// sum done by the error-free transformations of dw_device.cuh (about 48
// significant bits).  The work is the same as in binary64, but it runs on the
// binary32 pipe, which GB300 issues ~60x faster than binary64.  The DOFs are
// updated in binary64: Q += hi + lo.
//
// The face terms go through face traces (Floc^f = Pf^T Pf, Fnb = Pf^T Pnb with
// df = (N+1)(N+2)/2 rows): u_f = c_f (F^- (I Pf^T) + F^+ (I^nb Pnb^T)), then
// dQ -= M^{-1} sum_f Pf^T u_f, half the multiply-adds of dense face matrices.
#include <cuda_runtime.h>

#include "dw_device.cuh"
#include "poro_internal.h"

namespace poro {
namespace {

constexpr int DNT = 128;

template <int N, bool BATCH>
__global__ void __launch_bounds__(DNT, 4) corrector_dw_kernel(const CorrectorData D1, const int32_t* elems,
                                                             int64_t count, const CorrectorData* runs,
                                                             const int32_t* item_run) {
    constexpr int B = n_modes(N), QB = NQ * B;
    constexpr int stride = elem_const_stride(N);
    constexpr int DF = (N + 1) * (N + 2) / 2, FQ = NQ * DF;
    extern __shared__ float2 sm2[];
    float2* I = sm2;        // [13][B]
    float2* Y = I + QB;     // [13][B]
    float2* dQ = Y + QB;    // [13][B]
    float2* In = dQ + QB;   // [13][B]
    float2* tL = In + QB;   // [4][13][DF] traces of I
    float2* tR = tL + 4 * FQ;  // [13][DF] neighbour trace
    float2* U = tR + FQ;    // [4][13][DF] flux values
    __shared__ float2 F[2 * NQ * NQ];
    __shared__ float2 st[3 * STAR_NNZ];  // A^j = A^{j*} / dt
    __shared__ double wts[MAX_N + 1];
    const int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        // one run's data (D1), or item it's run of a batched launch over
        // several runs (their tables in global memory)
        const CorrectorData& D = BATCH ? runs[item_run[it]] : D1;
        const int64_t e = elems ? elems[it] : it;
        const double* ec = D.econst + e * stride;
        const double dt = ec[ec_scalars(N) + 2];
        const float2 ev = dw_split(ec[ec_scalars(N)] / dt), gv = dw_split(ec[ec_scalars(N) + 1] / dt);
        for (int i = tid; i < QB; i += DNT) {
            I[i] = dw_split(D.iout[e * QB + i]);
            dQ[i] = make_float2(0.f, 0.f);
        }
        for (int i = tid; i < 3 * STAR_NNZ; i += DNT) st[i] = dw_split(ec[i] / dt);
        __syncthreads();
        // volume: X^j = A^j I (54-entry star pattern), dQ += Kv^j X^j
        for (int j = 0; j < 3; ++j) {
            const float2* sj = st + j * STAR_NNZ;
            for (int l = tid; l < B; l += DNT) {
                float2 qv[NQ];
                float ah[NQ], al[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    qv[q] = I[q * B + l];
                    ah[q] = al[q] = 0.f;
                }
#pragma unroll
                for (int n = 0; n < STAR_NNZ; ++n)
                    dw_mac(ah[star_row(n)], al[star_row(n)], sj[n].x, sj[n].y, qv[star_col(n)].x, qv[star_col(n)].y);
#pragma unroll
                for (int p = 0; p < NQ; ++p) Y[p * B + l] = make_float2(ah[p], al[p]);
            }
            __syncthreads();
            const int32_t* vr = D.vrow + j * (B + 1);
            for (int i = tid; i < QB; i += DNT) {
                const int p = i / B, k = i - (i / B) * B;
                float h = 0.f, lo = 0.f;
                for (int n = __ldg(vr + k); n < __ldg(vr + k + 1); ++n) {
                    const float2 v = __ldg(reinterpret_cast<const float2*>(D.vval2) + n);
                    const float2 y = Y[p * B + __ldg(D.vcol + n)];
                    dw_mac(h, lo, v.x, v.y, y.x, y.y);
                }
                dQ[i] = dw_add(dQ[i], make_float2(h, lo));
            }
            __syncthreads();
        }
        // Darcy source term E I: u rows from u_f, u_f rows from u_f
        for (int i = tid; i < 6 * B; i += DNT) {
            const int r = i / B, k = i - (i / B) * B;
            const float2 x = I[(QUF + (r % 3)) * B + k];
            const float2 c = r < 3 ? gv : ev;
            float h = 0.f, lo = 0.f;
            dw_mac(h, lo, c.x, c.y, x.x, x.y);
            float2& d = dQ[(r < 3 ? QU + r : QUF + r - 3) * B + k];
            d = dw_add(d, make_float2(h, lo));
        }
        __syncthreads();
        // traces of I on the four faces: tL[f][p][a] = sum_k Pf[f][a][k] I[p][k];
        // a thread takes one row (f, a) and all 13 quantities (one load, 13 MACs)
        for (int t = tid; t < 4 * DF; t += DNT) {
            const int f = t / DF, a = t - f * DF;
            const float2* row = reinterpret_cast<const float2*>(D.Pf2) + ((size_t)f * DF + a) * B;
            float h[NQ], lo[NQ];
#pragma unroll
            for (int p = 0; p < NQ; ++p) h[p] = lo[p] = 0.f;
            for (int k = 0; k < B; ++k) {
                const float2 pv = __ldg(row + k);
#pragma unroll
                for (int p = 0; p < NQ; ++p) {
                    const float2 x = I[p * B + k];
                    dw_mac(h[p], lo[p], pv.x, pv.y, x.x, x.y);
                }
            }
#pragma unroll
            for (int p = 0; p < NQ; ++p) tL[f * FQ + p * DF + a] = make_float2(h[p], lo[p]);
        }
        __syncthreads();
        for (int f = 0; f < 4; ++f) {
            const int64_t nbr = D.nb[e * 4 + f];
            const bool inner = nbr >= 0;
            const float2* Fm = reinterpret_cast<const float2*>(D.fF2) + ((e * 4 + f) * 2) * NQ * NQ;
            for (int i = tid; i < (inner ? 2 : 1) * NQ * NQ; i += DNT) F[i] = Fm[i];
            if (inner) {
                // the neighbour's trace integrated over this element's interval
                const int c = D.cl ? D.cl[e] : 0, cr = D.cl ? D.cl[nbr] : 0;
                if (cr == c) {
                    for (int i = tid; i < QB; i += DNT) In[i] = dw_split(D.iout[nbr * QB + i]);
                } else if (cr < c) {
                    const double* b = D.buf + (int64_t)D.slot[nbr * D.C + c] * QB;
                    for (int i = tid; i < QB; i += DNT) In[i] = dw_split(b[i]);
                } else {
                    // larger neighbour: dt_r sum_s Qt_s int_a^b chi_s over the sub-interval
                    constexpr int T = N + 1;
                    if (tid == 0) {
                        const int64_t ks = D.tick + 1 - ((int64_t)1 << c);
                        const int64_t m = (ks >> cr) << cr;
                        const double a = (double)(ks - m) / (double)((int64_t)1 << cr);
                        const double bb = (double)(D.tick + 1 - m) / (double)((int64_t)1 << cr);
                        // int_a^b P_s(2 tau - 1) dtau = (1/2) [ (P_{s+1} - P_{s-1}) / (2s+1) ]_{2a-1}^{2b-1}
                        double P0[MAX_N + 3], P1[MAX_N + 3];
                        const double x0 = 2 * a - 1, x1 = 2 * bb - 1;
                        P0[0] = 1;
                        P0[1] = x0;
                        P1[0] = 1;
                        P1[1] = x1;
                        for (int n = 1; n <= T; ++n) {
                            P0[n + 1] = ((2 * n + 1) * x0 * P0[n] - n * P0[n - 1]) / (n + 1);
                            P1[n + 1] = ((2 * n + 1) * x1 * P1[n] - n * P1[n - 1]) / (n + 1);
                        }
                        wts[0] = 0.5 * (x1 - x0);
                        for (int sidx = 1; sidx < T; ++sidx)
                            wts[sidx] = 0.5 * ((P1[sidx + 1] - P1[sidx - 1]) - (P0[sidx + 1] - P0[sidx - 1])) /
                                        (2 * sidx + 1);
                    }
                    __syncthreads();
                    const double dtr = D.econst[nbr * stride + ec_scalars(N) + 2];
                    const double* qr = D.qt + nbr * (int64_t)QB * T;
                    for (int i = tid; i < QB; i += DNT) {
                        double acc = 0.0;
                        for (int sidx = 0; sidx < T; ++sidx) acc = fma(qr[i * T + sidx], wts[sidx], acc);
                        In[i] = dw_split(dtr * acc);
                    }
                }
                __syncthreads();
                const float2* Pn = reinterpret_cast<const float2*>(D.Pnb2) + (size_t)D.tab[e * 4 + f] * DF * B;
                // one row a and a group of 4 quantities per thread
                constexpr int RG = 4, NRG = (NQ + RG - 1) / RG;
                for (int t = tid; t < NRG * DF; t += DNT) {
                    const int a = t % DF, p0 = (t / DF) * RG;
                    const float2* row = Pn + (size_t)a * B;
                    float h[RG], lo[RG];
#pragma unroll
                    for (int g = 0; g < RG; ++g) h[g] = lo[g] = 0.f;
                    for (int k = 0; k < B; ++k) {
                        const float2 pv = __ldg(row + k);
#pragma unroll
                        for (int g = 0; g < RG; ++g) {
                            if (p0 + g < NQ) {
                                const float2 x = In[(p0 + g) * B + k];
                                dw_mac(h[g], lo[g], pv.x, pv.y, x.x, x.y);
                            }
                        }
                    }
#pragma unroll
                    for (int g = 0; g < RG; ++g)
                        if (p0 + g < NQ) tR[(p0 + g) * DF + a] = make_float2(h[g], lo[g]);
                }
            }
            __syncthreads();
            // U = c_f (F^- tL + F^+ tR)
            const float2 cf = dw_split(D.fc[e * 4 + f]);
            for (int t = tid; t < FQ; t += DNT) {
                const int p = t / DF, a = t - p * DF;
                float h = 0.f, lo = 0.f;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float2 fv = F[p * NQ + q], x = tL[f * FQ + q * DF + a];
                    dw_mac(h, lo, fv.x, fv.y, x.x, x.y);
                }
                if (inner) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float2 fv = F[NQ * NQ + p * NQ + q], x = tR[q * DF + a];
                        dw_mac(h, lo, fv.x, fv.y, x.x, x.y);
                    }
                }
                float uh = 0.f, ul = 0.f;
                dw_mac(uh, ul, cf.x, cf.y, h, lo);
                U[f * FQ + t] = make_float2(uh, ul);
            }
            __syncthreads();
        }
        // dQ[p][k] -= M_kk^{-1} sum_f sum_a Pf[f][a][k] U[f][p][a]; a thread takes
        // one column k and all 13 quantities
        for (int k = tid; k < B; k += DNT) {
            float h[NQ], lo[NQ];
#pragma unroll
            for (int p = 0; p < NQ; ++p) h[p] = lo[p] = 0.f;
#pragma unroll 1
            for (int f = 0; f < 4; ++f) {
                const float2* col = reinterpret_cast<const float2*>(D.Pf2) + (size_t)f * DF * B + k;
                for (int a = 0; a < DF; ++a) {
                    const float2 pv = __ldg(col + (size_t)a * B);
#pragma unroll
                    for (int p = 0; p < NQ; ++p) {
                        const float2 x = U[f * FQ + p * DF + a];
                        dw_mac(h[p], lo[p], pv.x, pv.y, x.x, x.y);
                    }
                }
            }
            const float2 mi = dw_split(-D.minv[k]);
#pragma unroll
            for (int p = 0; p < NQ; ++p) {
                float sh = 0.f, sl = 0.f;
                dw_mac(sh, sl, mi.x, mi.y, h[p], lo[p]);
                dQ[p * B + k] = dw_add(dQ[p * B + k], make_float2(sh, sl));
            }
        }
        __syncthreads();
        for (int i = tid; i < QB; i += DNT) {
            const float2 d = dQ[i];
            D.q[e * QB + i] += (double)d.x + (double)d.y;
        }
        __syncthreads();
    }
}

template <int N>
int launch_n(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream, const CorrectorData* runs,
             const int32_t* item_run) {
    auto* kern = runs ? corrector_dw_kernel<N, true> : corrector_dw_kernel<N, false>;
    constexpr int B = n_modes(N);
    constexpr int DF = (N + 1) * (N + 2) / 2;
    const size_t smem = sizeof(float2) * (4 * NQ * B + 9 * NQ * DF);
    cudaError_t err =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    kern<<<(unsigned)grid, DNT, smem, (cudaStream_t)stream>>>(d, elems, count, runs, item_run);
    return (int)cudaGetLastError();
}

}  // namespace

int launch_corrector_dw(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream,
                        const CorrectorData* runs, const int32_t* item_run) {
    if (count <= 0) return 0;
    switch (d.N) {
        case 1: return launch_n<1>(d, elems, count, stream, runs, item_run);
        case 2: return launch_n<2>(d, elems, count, stream, runs, item_run);
        case 3: return launch_n<3>(d, elems, count, stream, runs, item_run);
        case 4: return launch_n<4>(d, elems, count, stream, runs, item_run);
        case 5: return launch_n<5>(d, elems, count, stream, runs, item_run);
        case 6: return launch_n<6>(d, elems, count, stream, runs, item_run);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace poro
