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
// The dense face products (13 x B x B per face side, most of the work) give
// each thread one row k of the face matrix and a group of quantities p (5 or 7
// at N = 5, 6), so one load of F_kl serves that many multiply-adds.
#include <cuda_runtime.h>

#include "dw_device.cuh"
#include "poro_internal.h"

namespace poro {
namespace {

constexpr int DNT = 128;
// quantities per thread in the face products: groups of PG cover the 13
// quantities, (groups x B) tasks fill the CTA's 128 threads in about whole rounds
__host__ __device__ constexpr int face_pg(int N) { return N == 6 ? 5 : (N == 5 ? 7 : (N == 4 ? 5 : (N == 3 ? 3 : 2))); }

template <int N>
__global__ void __launch_bounds__(DNT, 4) corrector_dw_kernel(const CorrectorData D, const int32_t* elems,
                                                             int64_t count) {
    constexpr int B = n_modes(N), QB = NQ * B;
    constexpr int stride = elem_const_stride(N);
    constexpr int PG = face_pg(N), NG = (NQ + PG - 1) / PG;
    extern __shared__ float2 sm2[];
    float2* I = sm2;        // [13][B]
    float2* Y = I + QB;     // [13][B]
    float2* dQ = Y + QB;    // [13][B]
    float2* In = dQ + QB;   // [13][B]
    __shared__ float2 F[NQ * NQ];
    __shared__ float2 st[3 * STAR_NNZ];  // A^j = A^{j*} / dt
    __shared__ double wts[MAX_N + 1];
    const int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
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
        // faces
        for (int f = 0; f < 4; ++f) {
            const int64_t nbr = D.nb[e * 4 + f];
            const double cf = D.fc[e * 4 + f];
            const float2* Fm = reinterpret_cast<const float2*>(D.fF2) + ((e * 4 + f) * 2) * NQ * NQ;
            for (int side = 0; side < (nbr >= 0 ? 2 : 1); ++side) {
                const float2* src = I;
                if (side == 1) {
                    // the neighbour's trace integrated over this element's interval
                    const int c = D.cl ? D.cl[e] : 0, cr = D.cl ? D.cl[nbr] : 0;
                    if (cr == c) {
                        for (int i = tid; i < QB; i += DNT) In[i] = dw_split(D.iout[nbr * QB + i]);
                    } else if (cr < c) {
                        const double* b = D.buf + (int64_t)D.slot[nbr * D.C + c] * QB;
                        for (int i = tid; i < QB; i += DNT) In[i] = dw_split(b[i]);
                    } else {
                        // larger neighbour: dt_r sum_s Qt_s int_a^b chi_s over the sub-interval
                        const int T = N + 1;
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
                    src = In;
                }
                for (int i = tid; i < NQ * NQ; i += DNT) F[i] = Fm[side * NQ * NQ + i];
                __syncthreads();
                // Y = F src
                for (int i = tid; i < QB; i += DNT) {
                    const int p = i / B, l = i - (i / B) * B;
                    float h = 0.f, lo = 0.f;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float2 fv = F[p * NQ + q], x = src[q * B + l];
                        dw_mac(h, lo, fv.x, fv.y, x.x, x.y);
                    }
                    Y[i] = make_float2(h, lo);
                }
                __syncthreads();
                // dQ[p, k] -= c_f / M_kk sum_l Fmat_kl Y[p, l]; thread = (row k, 7 quantities)
                const float2* Fmat = side == 0
                                         ? reinterpret_cast<const float2*>(D.Floc2) + (size_t)f * B * B
                                         : reinterpret_cast<const float2*>(D.Fnb2) + (size_t)D.tab[e * 4 + f] * B * B;
                for (int t = tid; t < NG * B; t += DNT) {
                    const int k = t % B, p0 = (t / B) * PG;
                    float h[PG], lo[PG];
#pragma unroll
                    for (int g = 0; g < PG; ++g) h[g] = lo[g] = 0.f;
                    const float2* row = Fmat + (size_t)k * B;
                    // four entries of the row in flight per step (the face matrices
                    // live in L2 at N = 6)
                    constexpr int U = 4, BU = B / U * U;
                    for (int l0 = 0; l0 < BU; l0 += U) {
                        float2 fm[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) fm[u] = __ldg(row + l0 + u);
#pragma unroll
                        for (int u = 0; u < U; ++u)
#pragma unroll
                            for (int g = 0; g < PG; ++g) {
                                if (p0 + g < NQ) {
                                    const float2 y = Y[(p0 + g) * B + l0 + u];
                                    dw_mac(h[g], lo[g], fm[u].x, fm[u].y, y.x, y.y);
                                }
                            }
                    }
                    for (int l = BU; l < B; ++l) {
                        const float2 fm = __ldg(row + l);
#pragma unroll
                        for (int g = 0; g < PG; ++g) {
                            if (p0 + g < NQ) {
                                const float2 y = Y[(p0 + g) * B + l];
                                dw_mac(h[g], lo[g], fm.x, fm.y, y.x, y.y);
                            }
                        }
                    }
                    const float2 s = dw_split(-cf * D.minv[k]);
#pragma unroll
                    for (int g = 0; g < PG; ++g) {
                        if (p0 + g < NQ) {
                            float sh = 0.f, sl = 0.f;
                            dw_mac(sh, sl, s.x, s.y, h[g], lo[g]);
                            float2& d = dQ[(p0 + g) * B + k];
                            d = dw_add(d, make_float2(sh, sl));
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < QB; i += DNT) {
            const float2 d = dQ[i];
            D.q[e * QB + i] += (double)d.x + (double)d.y;
        }
        __syncthreads();
    }
}

template <int N>
int launch_n(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream) {
    constexpr int B = n_modes(N);
    const size_t smem = sizeof(float2) * 4 * NQ * B;
    cudaError_t err =
        cudaFuncSetAttribute(corrector_dw_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    corrector_dw_kernel<N><<<(unsigned)grid, DNT, smem, (cudaStream_t)stream>>>(d, elems, count);
    return (int)cudaGetLastError();
}

}  // namespace

int launch_corrector_dw(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream) {
    if (count <= 0) return 0;
    switch (d.N) {
        case 1: return launch_n<1>(d, elems, count, stream);
        case 2: return launch_n<2>(d, elems, count, stream);
        case 3: return launch_n<3>(d, elems, count, stream);
        case 4: return launch_n<4>(d, elems, count, stream);
        case 5: return launch_n<5>(d, elems, count, stream);
        case 6: return launch_n<6>(d, elems, count, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace poro
