// K3: the comparator of the paper's Section "Block-wise back-substitution":
// the predictor system of each element solved as one dense s x s system,
// s = 13 B (N+1), with precomputed LU factors (the approach the paper
// replaces; two triangular solves cost 2 s^2 flops and the factors s^2
// doubles per element).
//
// Assembly uses the row-scaled form of Eq. stp-lineq (every row (p,k,r)
// divided by M_kk S_rr, which leaves the solution unchanged):
//   Y'[(p,k,r),(q,l,s)] = d_pq d_kl Z_rs - E*_pq d_kl d_rs + sum_j A^{j*}_pq d_rs Khat^j_kl
//   r'[(p,k,r)]         = (S^{-1} w)_r Q0[p,k]
// with the unrolling (p,k,r) -> (p B + k) T + r.  Rows and columns are then
// equilibrated by exact powers of two and factored P Y = L U (partial
// pivoting, binary64), right-looking: per column one pivot kernel (one CTA
// per element) and one trailing rank-1 update kernel over all elements.
#include <cuda_runtime.h>

#include <cmath>

#include "poro_internal.h"

namespace poro {
namespace {

__device__ __forceinline__ double pow2_inverse_of(double m) {
    // 2^(-round(log2 m)) for m > 0 (exactly representable scaling)
    if (!(m > 0.0)) return 1.0;
    int ex;
    const double f = frexp(m, &ex);  // m = f 2^ex, f in [0.5, 1)
    const int r = f >= 0.70710678118654752 ? ex : ex - 1;
    return ldexp(1.0, -r);
}

// one thread per row: scatter the non-zeros of row (p,k,r) of Y' into a
// zeroed dense row
__global__ void lu_assemble_kernel(int N, int64_t count, const double* econst, int stride, const double* z,
                                   const int32_t* krow, const int32_t* kcol, const double* kval, double* A) {
    const int B = n_modes(N), T = N + 1, s = NQ * B * T;
    const int64_t e = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count || i >= s) return;
    const double* ec = econst + e * stride;
    const double* star = ec;
    const double ev = ec[ec_scalars(N)], gv = ec[ec_scalars(N) + 1];
    const int p = i / (B * T), k = (i / T) % B, r = i % T;
    double* row = A + (size_t)e * s * s + (size_t)i * s;
    // time block: Z_rs, and -E*_pp on the diagonal (u_f rows)
    for (int t = 0; t < T; ++t) row[(p * B + k) * T + t] = z[r * T + t];
    if (p >= QUF) row[(p * B + k) * T + r] -= ev;
    // strictly upper part of E*: u row couples to u_f
    if (p >= QU && p <= QW) row[((p + 4) * B + k) * T + r] -= gv;
    // star (x) Khat: columns (q, l, r)
    for (int j = 0; j < 3; ++j) {
        const int32_t* rp = krow + j * (B + 1) + k;
        for (int n = star_row_ptr(p); n < star_row_ptr(p + 1); ++n) {
            const int q = star_col(n);
            const double a = star[j * STAR_NNZ + n];
            for (int m = rp[0]; m < rp[1]; ++m) row[(q * B + kcol[m]) * T + r] += a * kval[m];
        }
    }
}

__global__ void lu_row_scale_kernel(int s, int64_t count, double* A, double* R) {
    const int64_t e = blockIdx.y;
    const int i = blockIdx.x;
    const double* row = A + (size_t)e * s * s + (size_t)i * s;
    double m = 0.0;
    for (int j = threadIdx.x; j < s; j += blockDim.x) m = fmax(m, fabs(row[j]));
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) R[e * s + i] = pow2_inverse_of(red[0]);
}

__global__ void lu_col_scale_kernel(int s, int64_t count, const double* A, const double* R, double* C) {
    const int64_t e = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s) return;
    const double* Ae = A + (size_t)e * s * s;
    const double* Re = R + e * s;
    double m = 0.0;
    for (int i = 0; i < s; ++i) m = fmax(m, fabs(Ae[(size_t)i * s + j]) * Re[i]);
    C[e * s + j] = pow2_inverse_of(m);
}

__global__ void lu_apply_scale_kernel(int s, int64_t count, double* A, const double* R, const double* C) {
    const int64_t e = blockIdx.y;
    const size_t n = (size_t)s * s;
    double* Ae = A + (size_t)e * n;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / s), j = (int)(t % s);
        Ae[t] *= R[e * s + i] * C[e * s + j];
    }
}

// column k: pivot search over rows k..s-1, row swap, multipliers
__global__ void lu_pivot_kernel(int s, int k, double* A, int32_t* piv, int32_t* bad) {
    const int64_t e = blockIdx.x;
    double* Ae = A + (size_t)e * s * s;
    __shared__ double bv[256];
    __shared__ int bi[256];
    double best = -1.0;
    int besti = k;
    for (int i = k + threadIdx.x; i < s; i += blockDim.x) {
        const double v = fabs(Ae[(size_t)i * s + k]);
        if (v > best) { best = v; besti = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double o = bv[threadIdx.x + w];
            const int oi = bi[threadIdx.x + w];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int pr = bi[0];
    if (threadIdx.x == 0) {
        piv[e * s + k] = pr;
        if (!(bv[0] > 0.0)) atomicExch(bad, 1);
    }
    if (pr != k)
        for (int j = threadIdx.x; j < s; j += blockDim.x) {
            const double t = Ae[(size_t)k * s + j];
            Ae[(size_t)k * s + j] = Ae[(size_t)pr * s + j];
            Ae[(size_t)pr * s + j] = t;
        }
    __syncthreads();
    const double d = Ae[(size_t)k * s + k];
    if (d != 0.0)
        for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) Ae[(size_t)i * s + k] /= d;
}

// trailing update A[i, j] -= A[i, k] A[k, j] for i, j > k
__global__ void lu_update_kernel(int s, int k, double* A) {
    const int64_t e = blockIdx.z;
    double* Ae = A + (size_t)e * s * s;
    const int j = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s) return;
    const double ukj = Ae[(size_t)k * s + j];
    const int rows_per = (s - k - 1 + gridDim.y - 1) / gridDim.y;
    const int i0 = k + 1 + blockIdx.y * rows_per, i1 = min(s, i0 + rows_per);
    for (int i = i0; i < i1; ++i) Ae[(size_t)i * s + j] = fma(-Ae[(size_t)i * s + k], ukj, Ae[(size_t)i * s + j]);
}

// final row permutation of every element: perm[i] = original row of row i of P Y
__global__ void lu_perm_kernel(int s, int64_t count, const int32_t* piv, int32_t* perm) {
    const int64_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    int32_t* pe = perm + e * s;
    for (int i = 0; i < s; ++i) pe[i] = i;
    for (int k = 0; k < s; ++k) {
        const int pr = piv[e * s + k];
        const int32_t t = pe[k];
        pe[k] = pe[pr];
        pe[pr] = t;
    }
}

// two triangular solves per element, one CTA (1024 threads) per element,
// the solution vector in shared memory; rows in blocks of 32: a GEMV of the
// block against the solved part (one warp per row), then the 32 x 32
// triangle by one warp
constexpr int SOLVE_NT = 1024;

__global__ void __launch_bounds__(SOLVE_NT) lu_solve_kernel(int N, const double* A, const int32_t* perm,
                                                            const double* R, const double* C, const double* q0,
                                                            const double* econst, int stride, double* qt,
                                                            double* iout) {
    extern __shared__ double x[];
    const int B = n_modes(N), T = N + 1, s = NQ * B * T;
    const int64_t e = blockIdx.x;
    const double* Ae = A + (size_t)e * s * s;
    const int32_t* pe = perm + e * s;
    const double* Re = R + e * s;
    const double* Ce = C + e * s;
    const double* q = q0 + e * (int64_t)(NQ * B);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NW = SOLVE_NT / 32;
    __shared__ double part[32];
    // x = P (R r'),  r'[(p,k,r)] = (2r+1)(-1)^r Q0[p,k]
    for (int i = threadIdx.x; i < s; i += SOLVE_NT) {
        const int o = pe[i];
        const int r = o % T;
        x[i] = Re[o] * (double)((2 * r + 1) * ((r & 1) ? -1 : 1)) * q[o / T];
    }
    __syncthreads();
    // forward: L unit lower
    for (int rb = 0; rb < s; rb += 32) {
        const int nr = min(32, s - rb);
        for (int rr = warp; rr < nr; rr += NW) {
            const double* row = Ae + (size_t)(rb + rr) * s;
            double acc = 0.0;
            for (int j = lane; j < rb; j += 32) acc = fma(row[j], x[j], acc);
            for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
            if (lane == 0) part[rr] = acc;
        }
        __syncthreads();
        if (warp == 0) {
            double xi = lane < nr ? x[rb + lane] - part[lane] : 0.0;
            for (int t = 0; t < nr; ++t) {
                const double xt = __shfl_sync(0xffffffffu, xi, t);
                if (lane > t && lane < nr) xi = fma(-Ae[(size_t)(rb + lane) * s + rb + t], xt, xi);
            }
            if (lane < nr) x[rb + lane] = xi;
        }
        __syncthreads();
    }
    // backward: U upper with diagonal
    for (int re = s; re > 0; re -= 32) {
        const int rb = max(0, re - 32), nr = re - rb;
        for (int rr = warp; rr < nr; rr += NW) {
            const double* row = Ae + (size_t)(rb + rr) * s;
            double acc = 0.0;
            for (int j = re + lane; j < s; j += 32) acc = fma(row[j], x[j], acc);
            for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
            if (lane == 0) part[rr] = acc;
        }
        __syncthreads();
        if (warp == 0) {
            double xi = lane < nr ? x[rb + lane] - part[lane] : 0.0;
            for (int t = nr - 1; t >= 0; --t) {
                if (lane == t) xi = xi / Ae[(size_t)(rb + t) * s + rb + t];
                const double xt = __shfl_sync(0xffffffffu, xi, t);
                if (lane < t) xi = fma(-Ae[(size_t)(rb + lane) * s + rb + t], xt, xi);
            }
            if (lane < nr) x[rb + lane] = xi;
        }
        __syncthreads();
    }
    // Qt = C z, I = dt Qt[..][0]
    const double dt = econst[e * stride + ec_scalars(N) + 2];
    for (int i = threadIdx.x; i < s; i += SOLVE_NT) {
        const double v = Ce[i] * x[i];
        if (qt) qt[e * (int64_t)s + i] = v;
        if (iout && (i % T) == 0) iout[e * (int64_t)(NQ * B) + i / T] = dt * v;
    }
}

// ---- blocked triangular solves over many CTAs (large systems).  One CTA
// per element reads its s^2 factor entries at the bandwidth of one SM; the
// blocked form reads them with every SM: the solution vector x[count][s]
// stays in global memory and, per block of BS unknowns, one launch solves
// the block's triangle (one CTA per element, the block staged in shared
// memory) and one launch subtracts the block's columns from all remaining
// rows (row chunks of every element spread over the GPU).  The launches
// follow each other on the stream, so no CTA waits for another.
constexpr int BS = 128;      // unknowns per block
constexpr int PANEL_ROWS = 16;  // rows per CTA of the panel update (two per warp)

// x = P (R r'),  r'[(p,k,r)] = (2r+1)(-1)^r Q0[p,k]
__global__ void lu_bsolve_init(int N, const int32_t* perm, const double* R, const double* q0, double* x) {
    const int B = n_modes(N), T = N + 1, s = NQ * B * T;
    const int64_t e = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s) return;
    const int o = perm[e * s + i], r = o % T;
    x[e * s + i] = R[e * s + o] * (double)((2 * r + 1) * ((r & 1) ? -1 : 1)) * q0[e * (int64_t)(NQ * B) + o / T];
}

// the triangle of block [rb, rb + nr): unit lower (forward) or upper with
// its diagonal (backward).  BS threads stage the block into shared memory
// with asynchronous 8-byte copies (all in flight at once); then one warp
// solves it, each lane holding rows lane + 32 i in registers and the solved
// value broadcast by shuffles, with no CTA barrier per row.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}

__global__ void __launch_bounds__(BS) lu_bsolve_diag(int s, int rb, int nr, bool lower, const double* A, double* x) {
    extern __shared__ double blk[];  // [BS][BS + 1]
    constexpr int RPL = BS / 32;     // rows per lane
    const int64_t e = blockIdx.x;
    const double* Ae = A + (size_t)e * s * s;
    double* xe = x + e * (int64_t)s;
    const int t = threadIdx.x;
    if (t < nr)
        for (int r = 0; r < nr; ++r) cp_async8(blk + r * (BS + 1) + t, Ae + (size_t)(rb + r) * s + rb + t);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (t >= 32) return;
    double xv[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) xv[i] = t + 32 * i < nr ? xe[rb + t + 32 * i] : 0.0;
    if (lower) {
        for (int k = 0; k < nr; ++k) {
            const int slot = k >> 5;
            double own = xv[0];
#pragma unroll
            for (int i = 1; i < RPL; ++i) own = slot == i ? xv[i] : own;
            const double xk = __shfl_sync(0xffffffffu, own, k & 31);
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                const int r = t + 32 * i;
                if (r > k && r < nr) xv[i] = fma(-blk[r * (BS + 1) + k], xk, xv[i]);
            }
        }
    } else {
        for (int k = nr - 1; k >= 0; --k) {
            const int slot = k >> 5;
            double own = xv[0];
#pragma unroll
            for (int i = 1; i < RPL; ++i) own = slot == i ? xv[i] : own;
            if ((k & 31) == t) own = own / blk[k * (BS + 1) + k];
            const double xk = __shfl_sync(0xffffffffu, own, k & 31);
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                const int r = t + 32 * i;
                if (r == k) xv[i] = xk;
                else if (r < k) xv[i] = fma(-blk[r * (BS + 1) + k], xk, xv[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i)
        if (t + 32 * i < nr) xe[rb + t + 32 * i] = xv[i];
}

// x[i] -= sum_{j < nr} A[i, rb + j] x[rb + j] for the rows [r0, r1) of every
// element: one warp per row, the block's solved values in shared memory
__global__ void __launch_bounds__(256) lu_bsolve_panel(int s, int rb, int nr, int r0, int r1, const double* A,
                                                       double* x) {
    __shared__ double ys[BS];
    const int64_t e = blockIdx.y;
    const double* Ae = A + (size_t)e * s * s;
    double* xe = x + e * (int64_t)s;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t < nr) ys[t] = xe[rb + t];
    __syncthreads();
    const int i0 = r0 + blockIdx.x * PANEL_ROWS, i1 = min(r1, i0 + PANEL_ROWS);
    for (int i = i0 + warp; i < i1; i += 8) {
        const double* row = Ae + (size_t)i * s + rb;
        double acc = 0.0;
        for (int j = lane; j < nr; j += 32) acc = fma(row[j], ys[j], acc);
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if (lane == 0) xe[i] -= acc;
    }
}

// Qt = C z, I = dt Qt[..][0]
__global__ void lu_bsolve_out(int N, const double* C, const double* x, const double* econst, int stride, double* qt,
                              double* iout) {
    const int B = n_modes(N), T = N + 1, s = NQ * B * T;
    const int64_t e = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s) return;
    const double v = C[e * s + i] * x[e * s + i];
    if (qt) qt[e * (int64_t)s + i] = v;
    if (iout && (i % T) == 0) iout[e * (int64_t)(NQ * B) + i / T] = econst[e * stride + ec_scalars(N) + 2] * v;
}

int enqueue_lu_bsolve(int N, int64_t count, const LUScratch& w, int64_t offset, const double* q0, const double* econst,
                      double* qt, double* iout, cudaStream_t st) {
    const int B = n_modes(N), T = N + 1, s = NQ * B * T;
    const double* A = w.A + (size_t)offset * s * s;
    double* x = w.x;  // [count][s]
    const size_t smem = sizeof(double) * BS * (BS + 1);
    const dim3 gv((s + 255) / 256, (unsigned)count);
    lu_bsolve_init<<<gv, 256, 0, st>>>(N, w.perm + offset * s, w.R + offset * s, q0, x);
    const int nb = (s + BS - 1) / BS;
    for (int b = 0; b < nb; ++b) {  // forward, L unit lower
        const int rb = b * BS, nr = min(BS, s - rb);
        lu_bsolve_diag<<<(unsigned)count, BS, smem, st>>>(s, rb, nr, true, A, x);
        const int r0 = rb + nr;
        if (r0 < s)
            lu_bsolve_panel<<<dim3((s - r0 + PANEL_ROWS - 1) / PANEL_ROWS, (unsigned)count), 256, 0, st>>>(
                s, rb, nr, r0, s, A, x);
    }
    for (int b = nb - 1; b >= 0; --b) {  // backward, U upper with its diagonal
        const int rb = b * BS, nr = min(BS, s - rb);
        lu_bsolve_diag<<<(unsigned)count, BS, smem, st>>>(s, rb, nr, false, A, x);
        if (rb > 0)
            lu_bsolve_panel<<<dim3((rb + PANEL_ROWS - 1) / PANEL_ROWS, (unsigned)count), 256, 0, st>>>(s, rb, nr, 0,
                                                                                                     rb, A, x);
    }
    lu_bsolve_out<<<gv, 256, 0, st>>>(N, w.C + offset * s, x, econst, elem_const_stride(N), qt, iout);
    return (int)cudaGetLastError();
}

// The 4 * ceil(s / BS) launches of a blocked solve (240 at N = 6) as one CUDA
// graph (captured on a private stream, re-captured when a pointer or the count
// changes), launched on st.
int launch_lu_bsolve(int N, int64_t count, LUScratch& w, int64_t offset, const double* q0, const double* econst,
                     double* qt, double* iout, cudaStream_t st) {
    const int B = n_modes(N), T = N + 1, s = NQ * B * T;
    cudaError_t err = cudaFuncSetAttribute(lu_bsolve_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * BS * (BS + 1)));
    if (err != cudaSuccess) return (int)err;
    const void* key[10] = {w.A + (size_t)offset * s * s, w.x, w.perm + offset * s, w.R + offset * s,
                           w.C + offset * s, q0, econst, qt, iout, (const void*)(intptr_t)count};
    bool same = w.exec != nullptr;
    for (int i = 0; i < 10 && same; ++i) same = key[i] == w.key[i];
    if (!same) {
        if (w.exec) cudaGraphExecDestroy(w.exec);
        w.exec = nullptr;
        cudaStream_t cs = nullptr;
        cudaGraph_t graph = nullptr;
        err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (err == cudaSuccess) {
            const int rc = enqueue_lu_bsolve(N, count, w, offset, q0, econst, qt, iout, cs);
            const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            err = rc != 0 ? (cudaError_t)rc : e2;
        }
        if (err == cudaSuccess) err = cudaGraphInstantiate(&w.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (err != cudaSuccess) {
            w.exec = nullptr;
            return (int)err;
        }
        for (int i = 0; i < 10; ++i) w.key[i] = key[i];
    }
    return (int)cudaGraphLaunch(w.exec, st);
}

}  // namespace

size_t lu_scratch_bytes(int N, int64_t count) {
    const size_t s = (size_t)NQ * n_modes(N) * (N + 1);
    return (size_t)count * (s * s * sizeof(double) + s * (2 * sizeof(int32_t) + 3 * sizeof(double)));
}

int launch_lu_factor(const LUReference& ref, int64_t count, const double* econst, LUScratch& w, void* stream) {
    const int N = ref.N, B = n_modes(N), T = N + 1, s = NQ * B * T;
    cudaStream_t st = (cudaStream_t)stream;
    if (count <= 0) return 0;
    cudaError_t err = cudaMemsetAsync(w.A, 0, (size_t)count * s * s * sizeof(double), st);
    if (err != cudaSuccess) return (int)err;
    err = cudaMemsetAsync(w.bad, 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return (int)err;
    dim3 ga((s + 127) / 128, (unsigned)count);
    lu_assemble_kernel<<<ga, 128, 0, st>>>(N, count, econst, elem_const_stride(N), ref.z, ref.krow, ref.kcol, ref.kval,
                                           w.A);
    lu_row_scale_kernel<<<dim3(s, (unsigned)count), 256, 0, st>>>(s, count, w.A, w.R);
    lu_col_scale_kernel<<<dim3((s + 127) / 128, (unsigned)count), 128, 0, st>>>(s, count, w.A, w.R, w.C);
    lu_apply_scale_kernel<<<dim3(1024, (unsigned)count), 256, 0, st>>>(s, count, w.A, w.R, w.C);
    for (int k = 0; k < s - 1; ++k) {
        lu_pivot_kernel<<<(unsigned)count, 256, 0, st>>>(s, k, w.A, w.piv, w.bad);
        const int rem = s - k - 1;
        const int gy = rem >= 512 ? 32 : (rem >= 64 ? 8 : 1);
        lu_update_kernel<<<dim3((rem + 127) / 128, gy, (unsigned)count), 128, 0, st>>>(s, k, w.A);
    }
    // last pivot: record and flag a zero
    lu_pivot_kernel<<<(unsigned)count, 256, 0, st>>>(s, s - 1, w.A, w.piv, w.bad);
    lu_perm_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(s, count, w.piv, w.perm);
    return (int)cudaGetLastError();
}

int launch_lu_solve(const LUReference& ref, int64_t count, LUScratch& w, int64_t offset, const double* q0,
                    const double* econst, double* qt, double* iout, void* stream) {
    const int N = ref.N, B = n_modes(N), T = N + 1, s = NQ * B * T;
    if (count <= 0) return 0;
    // fewer elements than SMs (one CTA per element would leave most SMs idle)
    // and a solution scratch: the blocked solve over all SMs.  Measured on
    // GB300: N = 6, 4 elements 578 element-solves/s against 191 with one CTA
    // per element; N = 3, 1,024 elements 97k against 130k, so many elements
    // keep the one-CTA form.
    if (w.x && s > 2 * BS && count < 152)
        return launch_lu_bsolve(N, count, w, offset, q0, econst, qt, iout, (cudaStream_t)stream);
    const size_t smem = (size_t)s * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(lu_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    lu_solve_kernel<<<(unsigned)count, SOLVE_NT, smem, (cudaStream_t)stream>>>(
        N, w.A + (size_t)offset * s * s, w.perm + offset * s, w.R + offset * s, w.C + offset * s, q0, econst,
        elem_const_stride(N), qt, iout);
    return (int)cudaGetLastError();
}

}  // namespace poro
