// Corrector of the ADER-DG scheme (Eq. semi_discrete integrated over one
// time step, Section "Temporal discretisation with ADER"), point source and
// receivers, binary64.
//
// For element e with time-integrated predictor I (13 x B):
//   dQ_pk = sum_j sum_l Kv^j_kl (A^j I)_pl              volume, Kv^j = M^{-1} K^{jT}
//         + (E I)_pk                                    Darcy source term
//         - sum_f c_f / M_kk [ sum_l Floc^f_kl (F^- I^e)_pl
//                            + sum_l Fnb^{f,h,s}_kl (F^+ I^nb)_pl ]   Godunov flux
// with A^j = A^{j*} / dt and E = E* / dt from the element constants,
// c_f = 2 |S_f| / |J|, Floc^f / Fnb the face mass matrices of the local face
// and of the (neighbour face h, vertex permutation s) pair.  One CTA per
// element; the DOFs are updated in place (neighbours read I only).
#include <cuda_runtime.h>

#include "poro_internal.h"

namespace poro {
namespace {

constexpr int CNT = 128;

// the neighbour's trace source, integrated over this element's interval:
// its own I (same cluster), the buffered sum of its sub-steps (smaller
// neighbour) or its predictor integrated over the sub-interval (larger
// neighbour); written to In[13][B]
template <int N>
__device__ void neighbour_integral(const CorrectorData& D, int64_t e, int64_t nbr, double* In, double* wts) {
    constexpr int B = n_modes(N), QB = NQ * B, T = N + 1;
    const int c = D.cl ? D.cl[e] : 0, cr = D.cl ? D.cl[nbr] : 0;
    if (cr == c) {
        for (int i = threadIdx.x; i < QB; i += CNT) In[i] = D.iout[nbr * QB + i];
    } else if (cr < c) {
        const double* b = D.buf + (int64_t)D.slot[nbr * D.C + c] * QB;
        for (int i = threadIdx.x; i < QB; i += CNT) In[i] = b[i];
    } else {
        // larger neighbour: dt_r sum_s Qt_s int_a^b chi_s over the sub-interval
        if (threadIdx.x == 0) {
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
                wts[sidx] = 0.5 * ((P1[sidx + 1] - P1[sidx - 1]) - (P0[sidx + 1] - P0[sidx - 1])) / (2 * sidx + 1);
        }
        __syncthreads();
        const int stride = elem_const_stride(N);
        const double dtr = D.econst[nbr * stride + ec_scalars(N) + 2];
        const double* qr = D.qt + nbr * (int64_t)QB * T;
        for (int i = threadIdx.x; i < QB; i += CNT) {
            double acc = 0.0;
            for (int sidx = 0; sidx < T; ++sidx) acc = fma(qr[i * T + sidx], wts[sidx], acc);
            In[i] = dtr * acc;
        }
    }
}

// Face terms through face traces.  Floc^f = Pf^T Pf and Fnb^{f,h,s} = Pf^T Pnb
// with Pf, Pnb of df = (N+1)(N+2)/2 rows (traces in a basis orthonormal on
// the reference triangle), so per face
//   u_f = c_f (F^- (I Pf^T) + F^+ (I^nb Pnb^T))          [13 x df]
//   dQ -= M^{-1} sum_f Pf^T u_f                          (one pass over all faces)
template <int N, bool BATCH>
__global__ void __launch_bounds__(CNT) corrector_kernel(const CorrectorData D1, const int32_t* elems, int64_t count,
                                                        const CorrectorData* runs, const int32_t* item_run) {
    constexpr int B = n_modes(N), QB = NQ * B, DF = (N + 1) * (N + 2) / 2, FQ = NQ * DF;
    constexpr int stride = elem_const_stride(N);
    extern __shared__ double sm[];
    double* I = sm;             // [13][B]
    double* Y = I + QB;         // [13][B]
    double* dQ = Y + QB;        // [13][B]
    double* In = dQ + QB;       // [13][B]
    double* tL = In + QB;       // [4][13][DF] traces of I
    double* tR = tL + 4 * FQ;   // [13][DF] neighbour trace
    double* U = tR + FQ;        // [4][13][DF] flux values
    __shared__ double F[2 * NQ * NQ];
    __shared__ double wts[MAX_N + 1];
    const int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        // one run's data (D1), or item it's run of a batched launch over
        // several runs (their tables in global memory)
        const CorrectorData& D = BATCH ? runs[item_run[it]] : D1;
        const int64_t e = elems ? elems[it] : it;
        const double* ec = D.econst + e * stride;
        const double dt = ec[ec_scalars(N) + 2];
        const double ev = ec[ec_scalars(N)] / dt, gv = ec[ec_scalars(N) + 1] / dt;
        for (int i = tid; i < QB; i += CNT) {
            I[i] = D.iout[e * QB + i];
            dQ[i] = 0.0;
        }
        __syncthreads();
        // volume: X^j = A^j I (54-entry star pattern), dQ += Kv^j X^j
        for (int j = 0; j < 3; ++j) {
            const double* sj = ec + j * STAR_NNZ;
            for (int l = tid; l < B; l += CNT) {
                double qv[NQ], acc[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    qv[q] = I[q * B + l];
                    acc[q] = 0.0;
                }
#pragma unroll
                for (int n = 0; n < STAR_NNZ; ++n) acc[star_row(n)] = fma(sj[n], qv[star_col(n)], acc[star_row(n)]);
#pragma unroll
                for (int p = 0; p < NQ; ++p) Y[p * B + l] = acc[p] / dt;
            }
            __syncthreads();
            const int32_t* vr = D.vrow + j * (B + 1);
            for (int i = tid; i < QB; i += CNT) {
                const int p = i / B, k = i - (i / B) * B;
                double acc = 0.0;
                for (int n = vr[k]; n < vr[k + 1]; ++n) acc = fma(D.vval[n], Y[p * B + D.vcol[n]], acc);
                dQ[i] += acc;
            }
            __syncthreads();
        }
        // Darcy source term E I: u rows from u_f, u_f rows from u_f
        for (int i = tid; i < 6 * B; i += CNT) {
            const int r = i / B, k = i - (i / B) * B;
            if (r < 3) dQ[(QU + r) * B + k] += gv * I[(QUF + r) * B + k];
            else dQ[(QUF + r - 3) * B + k] += ev * I[(QUF + r - 3) * B + k];
        }
        // traces of I on the four faces: tL[f][p][a] = sum_k Pf[f][a][k] I[p][k]
        for (int t = tid; t < 4 * FQ; t += CNT) {
            const int f = t / FQ, r = t - f * FQ, p = r / DF, a = r - p * DF;
            const double* row = D.Pf + ((size_t)f * DF + a) * B;
            double acc = 0.0;
#pragma unroll 4
            for (int k = 0; k < B; ++k) acc = fma(__ldg(row + k), I[p * B + k], acc);
            tL[t] = acc;
        }
        __syncthreads();
        for (int f = 0; f < 4; ++f) {
            const int64_t nbr = D.nb[e * 4 + f];
            const double cf = D.fc[e * 4 + f];
            const double* Fm = D.fF + ((e * 4 + f) * 2) * NQ * NQ;
            const bool inner = nbr >= 0;
            for (int i = tid; i < (inner ? 2 : 1) * NQ * NQ; i += CNT) F[i] = Fm[i];
            if (inner) {
                neighbour_integral<N>(D, e, nbr, In, wts);
                __syncthreads();
                const double* Pn = D.Pnb + (size_t)D.tab[e * 4 + f] * DF * B;
                for (int t = tid; t < FQ; t += CNT) {
                    const int p = t / DF, a = t - p * DF;
                    const double* row = Pn + (size_t)a * B;
                    double acc = 0.0;
#pragma unroll 4
                    for (int k = 0; k < B; ++k) acc = fma(__ldg(row + k), In[p * B + k], acc);
                    tR[t] = acc;
                }
            }
            __syncthreads();
            // u = c_f (F^- tL + F^+ tR)
            for (int t = tid; t < FQ; t += CNT) {
                const int p = t / DF, a = t - p * DF;
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc = fma(F[p * NQ + q], tL[f * FQ + q * DF + a], acc);
                if (inner) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) acc = fma(F[NQ * NQ + p * NQ + q], tR[q * DF + a], acc);
                }
                U[f * FQ + t] = cf * acc;
            }
            __syncthreads();
        }
        // dQ[p][k] -= M_kk^{-1} sum_f sum_a Pf[f][a][k] U[f][p][a], then Q += dQ
        for (int i = tid; i < QB; i += CNT) {
            const int p = i / B, k = i - (i / B) * B;
            double acc = 0.0;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const double* col = D.Pf + (size_t)f * DF * B + k;
                const double* u = U + f * FQ + p * DF;
#pragma unroll 4
                for (int a = 0; a < DF; ++a) acc = fma(__ldg(col + (size_t)a * B), u[a], acc);
            }
            D.q[e * QB + i] += dQ[i] - D.minv[k] * acc;
        }
        __syncthreads();
    }
}

// buffers of the sub-step integrals for larger neighbours: level L restarts
// at ticks that are multiples of 2^L
__global__ void lts_buffer_kernel(int QB, int C, const int32_t* elems, int64_t count, const int32_t* slot,
                                  const double* iout, double* buf, int64_t tick) {
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        const int64_t e = elems[it];
        for (int L = 0; L < C; ++L) {
            const int sl = slot[e * C + L];
            if (sl < 0) continue;
            const bool reset = (tick & (((int64_t)1 << L) - 1)) == 0;
            double* b = buf + (int64_t)sl * QB;
            const double* I = iout + e * QB;
            for (int i = threadIdx.x; i < QB; i += blockDim.x) b[i] = reset ? I[i] : b[i] + I[i];
        }
    }
}

// point source with the amplitude of the step computed on the device:
// int_{t0}^{t1} s dt = S(t1) - S(t0), S(t) = (t - tc) exp(-(pi f0 (t - tc))^2),
// the step [ (k+1-len) dt, (k+1) dt ], k = *tick + k_rel
__global__ void point_source_tick_kernel(int QB, double* q, int64_t elem, const double* coef, double f0, double tc,
                                         double dt, int64_t len, int64_t k_rel, const int64_t* tick) {
    const int64_t k = *tick + k_rel;
    const double t1 = (double)(k + 1) * dt, t0 = (double)(k + 1 - len) * dt;
    const double a1 = 3.14159265358979323846 * f0 * (t1 - tc), a0 = 3.14159265358979323846 * f0 * (t0 - tc);
    const double amp = (t1 - tc) * exp(-a1 * a1) - (t0 - tc) * exp(-a0 * a0);
    for (int i = threadIdx.x; i < QB; i += blockDim.x) q[elem * QB + i] += amp * coef[i];
}

// receiver sample at the position given by a device counter
__global__ void receiver_count_kernel(int B, const double* q, int64_t elem, const double* phi, double* out,
                                      int32_t* counter) {
    const int p = threadIdx.x;
    const int32_t idx = *counter;
    if (p < NQ) {
        const double* qe = q + elem * (int64_t)(NQ * B) + p * B;
        double acc = 0.0;
        for (int l = 0; l < B; ++l) acc = fma(qe[l], phi[l], acc);
        out[(int64_t)idx * NQ + p] = acc;
    }
    __syncthreads();
    if (p == 0) *counter = idx + 1;
}

__global__ void tick_advance_kernel(int64_t* tick, int64_t n) { *tick += n; }

__global__ void ticks_advance_kernel(int64_t* const* ticks, int count, int64_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) *ticks[i] += n;
}

// one CTA per source item of a batched group: the arithmetic of
// point_source_tick_kernel
__global__ void source_items_kernel(int QB, const TickItem* items) {
    const TickItem& it = items[blockIdx.x];
    const int64_t k = *it.tick + it.k_rel;
    const double t1 = (double)(k + 1) * it.dt, t0 = (double)(k + 1 - it.len) * it.dt;
    const double a1 = 3.14159265358979323846 * it.f0 * (t1 - it.tc), a0 = 3.14159265358979323846 * it.f0 * (t0 - it.tc);
    const double amp = (t1 - it.tc) * exp(-a1 * a1) - (t0 - it.tc) * exp(-a0 * a0);
    double* q = it.q + it.elem * QB;
    for (int i = threadIdx.x; i < QB; i += blockDim.x) q[i] += amp * it.vec[i];
}

// one CTA per receiver item: the arithmetic of receiver_count_kernel
__global__ void receiver_items_kernel(int B, const TickItem* items) {
    const TickItem& it = items[blockIdx.x];
    const int p = threadIdx.x;
    const int32_t idx = *it.counter;
    if (p < NQ) {
        const double* qe = it.q + it.elem * (int64_t)(NQ * B) + p * B;
        double acc = 0.0;
        for (int l = 0; l < B; ++l) acc = fma(qe[l], it.vec[l], acc);
        it.out[(int64_t)idx * NQ + p] = acc;
    }
    __syncthreads();
    if (p == 0) *it.counter = idx + 1;
}

__global__ void point_source_kernel(int QB, double* q, int64_t elem, const double* coef, double amp) {
    for (int i = threadIdx.x; i < QB; i += blockDim.x) q[elem * QB + i] += amp * coef[i];
}

// out[r * stride_out + p] = sum_l Q[e_r][p][l] phi_r[l]
__global__ void receiver_kernel(int B, const double* q, int32_t nrec, const int64_t* elems, const double* phi,
                                double* out, int64_t stride_out) {
    const int r = blockIdx.x, p = threadIdx.x;
    if (r >= nrec || p >= NQ) return;
    const double* qe = q + elems[r] * (int64_t)(NQ * B) + p * B;
    double acc = 0.0;
    for (int l = 0; l < B; ++l) acc = fma(qe[l], phi[r * B + l], acc);
    out[r * stride_out + p] = acc;
}

template <int N>
int launch_corr_n(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream, const CorrectorData* runs,
                  const int32_t* item_run) {
    constexpr int B = n_modes(N), DF = (N + 1) * (N + 2) / 2;
    const size_t smem = sizeof(double) * (4 * NQ * B + 9 * NQ * DF);
    auto* kern = runs ? corrector_kernel<N, true> : corrector_kernel<N, false>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    kern<<<(unsigned)grid, CNT, smem, (cudaStream_t)stream>>>(d, elems, count, runs, item_run);
    return (int)cudaGetLastError();
}

}  // namespace

int launch_corrector(const CorrectorData& d, const int32_t* elems, int64_t count, void* stream,
                     const CorrectorData* runs, const int32_t* item_run) {
    if (count <= 0) return 0;
    if (d.dw) return launch_corrector_dw(d, elems, count, stream, runs, item_run);
    switch (d.N) {
        case 1: return launch_corr_n<1>(d, elems, count, stream, runs, item_run);
        case 2: return launch_corr_n<2>(d, elems, count, stream, runs, item_run);
        case 3: return launch_corr_n<3>(d, elems, count, stream, runs, item_run);
        case 4: return launch_corr_n<4>(d, elems, count, stream, runs, item_run);
        case 5: return launch_corr_n<5>(d, elems, count, stream, runs, item_run);
        case 6: return launch_corr_n<6>(d, elems, count, stream, runs, item_run);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_lts_buffers(int N, int C, const int32_t* elems, int64_t count, const int32_t* slot, const double* iout,
                       double* buf, int64_t tick, void* stream) {
    if (count <= 0) return 0;
    const int64_t grid = count < 65536 ? count : 65536;
    lts_buffer_kernel<<<(unsigned)grid, 128, 0, (cudaStream_t)stream>>>(NQ * n_modes(N), C, elems, count, slot, iout,
                                                                       buf, tick);
    return (int)cudaGetLastError();
}

int launch_point_source_tick(int N, double* q, int64_t elem, const double* coef, double f0, double tc, double dt,
                             int64_t len, int64_t k_rel, const int64_t* tick, void* stream) {
    point_source_tick_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(NQ * n_modes(N), q, elem, coef, f0, tc, dt, len,
                                                                  k_rel, tick);
    return (int)cudaGetLastError();
}

int launch_receiver_count(int N, const double* q, int64_t elem, const double* phi, double* out, int32_t* counter,
                          void* stream) {
    receiver_count_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(n_modes(N), q, elem, phi, out, counter);
    return (int)cudaGetLastError();
}

int launch_tick_sources(int N, const TickItem* items, int64_t count, void* stream) {
    if (count <= 0) return 0;
    source_items_kernel<<<(unsigned)count, 256, 0, (cudaStream_t)stream>>>(NQ * n_modes(N), items);
    return (int)cudaGetLastError();
}

int launch_tick_receivers(int N, const TickItem* items, int64_t count, void* stream) {
    if (count <= 0) return 0;
    receiver_items_kernel<<<(unsigned)count, 32, 0, (cudaStream_t)stream>>>(n_modes(N), items);
    return (int)cudaGetLastError();
}

int launch_ticks_advance(int64_t* const* ticks, int count, int64_t n, void* stream) {
    if (count <= 0) return 0;
    ticks_advance_kernel<<<(unsigned)((count + 127) / 128), 128, 0, (cudaStream_t)stream>>>(ticks, count, n);
    return (int)cudaGetLastError();
}

int launch_tick_advance(int64_t* tick, int64_t n, void* stream) {
    tick_advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(tick, n);
    return (int)cudaGetLastError();
}

int launch_point_source(int N, double* q, int64_t elem, const double* coef, double amp, void* stream) {
    point_source_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(NQ * n_modes(N), q, elem, coef, amp);
    return (int)cudaGetLastError();
}

int launch_receivers(int N, const double* q, int32_t nrec, const int64_t* elems, const double* phi, double* out,
                     int64_t stride_out, void* stream) {
    if (nrec <= 0) return 0;
    receiver_kernel<<<nrec, 32, 0, (cudaStream_t)stream>>>(n_modes(N), q, nrec, elems, phi, out, stride_out);
    return (int)cudaGetLastError();
}

}  // namespace poro
