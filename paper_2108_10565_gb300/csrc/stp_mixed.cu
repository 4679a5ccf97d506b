// K2: mixed-precision space-time predictor with iterative refinement.
//
// Solves the predictor system of one element (Eq. stp-lineq, in the scaled
// form of Section "Block-wise back-substitution":
//   (Z (x) I - E* + sum_j A^{j*} (x) Khat^j) Q = (S^{-1} w) o Q0 )
// as
//   Q1 = Alg3_lo(b0)                       binary32 back-substitution
//   Q1' = Q1 on a fixed-point grid          integers |v| <= 2^22 times 2^-s_p
//   r  = b0 - Y Q1'                        residual, binary64-accurate
//   d  = Alg3_lo(fl32(r));  Q = Q1' + d    (one sweep; a second repeats with
//                                           Q1' + d in the residual)
// The low-precision sweeps are Algorithm 3 (degree blocks, time solves with
// (Z - E*_pp I)^{-1}, G coupling, star and Khat products).  Their dominant
// step, b[p, l, u] -= sum_j sum_m Khat^j[l, m] X^j[p, m, u] over the rows
// l < o_g of degree block g, is a dense contraction whose left operand Khat is
// the same for every element: it runs on the tensor cores (tcgen05.mma,
// accumulator in TMEM) with both operands split into hi + lo words (tf32, or
// bf16 for the bf16 form) and the three products hi*hi + hi*lo + lo*hi
// accumulated.  One MMA tile per (g, j): M = 128 rows (p, u) of the element,
// N = rows l (o_g rounded up to 16), K = columns m of the block.  X^j (A
// operand) is written by the star-product threads straight into shared memory
// in the K-major core-matrix layout; the Khat^j block images (B operand,
// prebuilt on the host in the same layout) arrive by bulk copy, prefetched
// during the previous block (tc_layout says which buffers fit per block).
//
// The residual needs ~47 significant bits because Y Q1' cancels b0 to ~1e-7,
// and GB300 issues binary64 FMAs at ~1/60 of its binary32 rate.  So:
//   - the Khat rows are integer rows over a common denominator d_jl and Q1' is
//     integer, so sum_m c_jlm Q1'[q,m,u] is an exact 64-bit integer sum (R1),
//     and so is the time-matrix term sum_s Z_us Q1'[p,l,s] (Z is integer);
//   - the star, E* and coupling products use double-binary32 arithmetic on
//     the FP32 pipe: FMA-based exact products (p + e = a*b) and Knuth's
//     TwoSum, accumulating pairs (hi, lo) as in the double-word dot product of
//     Ogita, Rump and Oishi (2005).
//
// Residual layout: each warp takes its rows l from a balanced list.
//   R1: lanes over the 13 T (q, u) pairs: Y^j[q,u] = (1/d_jl) sum_m c_jlm Q'[q,m,u]
//   R2: lanes over the (p, u) pairs, dealt by star-row width:
//       r[p,l,u] = b0 - sum_s Z_us Q'[p,l,s] + E*_pp Q'[p,l,u] + G Q'[uf,l,u]
//                  - sum_j sum_q A^{j*}_pq Y^j[q,u]
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "alg3_device.cuh"
#include "dw_device.cuh"
#include "tc_device.cuh"

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
    const float2* res_inv;    // [3][B] 1 / d_jl as (hi, lo)
    const int32_t* res_order; // [warps + 1] list starts, then each warp's residual rows
    const float* zinv;        // Z^{-1} [T][T] binary32
    const float* khat_tc;     // tensor-core images of the Khat^j blocks (hi then lo)
    int32_t tc_off[MAX_N + 1][3];
    int32_t* status;          // set to 1 if a bounded wait gave up
    long long wait_limit;     // SM clocks after which a wait of the sweeps gives up (> 0)
    const RunPtrs* runs;      // items of several runs (nullptr: q0, econst, qt, iout above)
    const int32_t* item_run;
    int cap_a, cap_b;         // at most this many A buffers / Khat image slots per block (1..3)
};

// Residual CSR of every degree in constant memory: the table depends only on
// N (the reference matrices), so all contexts of one device share it.  Per N:
// [3][B+1] row pointers (relative to the entries), then the packed entries.
constexpr int res_words(int N) {
    return N == 1 ? 21 : N == 2 ? 79 : N == 3 ? 265 : N == 4 ? 755 : N == 5 ? 1879 : 4175;
}
constexpr int res_base(int N) { return N <= 1 ? 0 : res_base(N - 1) + res_words(N - 1); }
constexpr int RES_CONST_WORDS = res_base(MAX_N) + res_words(MAX_N);
__constant__ int32_t c_res[RES_CONST_WORDS];

// residual star terms per row p: 3 directions x 6 slots (rows have 2, 4 or 6
// entries; unused slots carry a zero coefficient)
constexpr int STAR_SLOTS = 18;

// star pattern tables for lane-varying lookups (copied to shared memory)
__constant__ int c_star_tab[NQ + 1 + STAR_NNZ] = {
    0, 6, 12, 18, 20, 22, 24, 28, 32, 36, 42, 46, 50, 54,
    QU, QV, QW, QUF, QVF, QWF, QU, QV, QW, QUF, QVF, QWF, QU, QV, QW, QUF, QVF, QWF,
    QU, QV, QV, QW, QU, QW,
    SXX, SXY, SXZ, QP, SYY, SXY, SYZ, QP, SZZ, SXZ, SYZ, QP,
    QU, QV, QW, QUF, QVF, QWF,
    SXX, SXY, SXZ, QP, SYY, SXY, SYZ, QP, SZZ, SXZ, SYZ, QP};

// CTA sizes the autotuner chooses from (index 0 is the default)
template <int N>
struct K2Sizes {
    static constexpr int NT0 = N >= 5 ? 256 : (N == 4 ? 128 : 64);
    static constexpr int NT1 = N >= 5 ? 128 : (N == 4 ? 256 : 128);
};

template <int N, int REF, int NT_, int BF = 0>
struct K2Shape : Alg3Shape<N> {
    using A = Alg3Shape<N>;
    static constexpr int NT = NT_;
    static constexpr int NW = NT / 32;
    static constexpr int T_ = N + 1;
    static constexpr int R4(int x) { return (x + 3) & ~3; }
    static constexpr int R32(int x) { return (x + 31) & ~31; }
    static constexpr int MAX2(int a, int b) { return a > b ? a : b; }
    // tensor-core operand tiles: A (X^j, hi and lo) with ceil(13 T / 8) row
    // groups of the widest block, then the Khat^j image (hi and lo).  The MMA
    // reads 16 row groups of each A tile; the rows past 13 T only feed
    // accumulator rows that are never read, so they may overlap what follows.
    // (sizes in floats; operand words are 4 bytes for tf32, 2 for bf16)
    static constexpr int ES = BF ? 2 : 4;
    static constexpr int KPM = tc_kp(N, BF != 0);
    static constexpr int SBOMAX = KPM * 8 * ES / 4;
    static constexpr int AH = (A::PT + 7) / 8 * SBOMAX;
    static constexpr int BIMG = 2 * tc_np(N) * KPM * ES / 4;
    // at least one A tile pair and one Khat image; the bf16 form gets the
    // room of the tf32 form, where the Khat images of all three directions fit
    // beside one A pair at every degree (tf32: up to degree 4)
    static constexpr int TC1 = MAX2(2 * AH + BIMG, AH + 16 * SBOMAX);
    static constexpr int TC_SIZE = BF ? MAX2(TC1, 2 * AH + 3 * BIMG) : TC1;
    // shared layout in floats; the tensor-core tiles of the sweeps and the
    // per-warp Y buffers of the residual share the first region
    static constexpr int OFF_XY = 0;
    static constexpr int XY_SIZE = R32(MAX2(TC_SIZE, NW * 3 * A::PT * 2));
    static constexpr int OFF_W = OFF_XY + XY_SIZE;
    static constexpr int Q1S = A::PT;                       // mode stride of Q1 / D1
    static constexpr int Q1SIZE = R4(A::B * Q1S + 32);       // + slack read by idle lanes
    static constexpr int OFF_Q1 = OFF_W + R4(A::SQ);
    static constexpr int OFF_D1 = OFF_Q1 + (REF >= 1 ? Q1SIZE : 0);
    static constexpr int OFF_SH = OFF_D1 + (REF == 2 ? Q1SIZE : 0);
    static constexpr int OFF_SL = OFF_SH + R4(3 * STAR_NNZ);
    static constexpr int OFF_ZIN = OFF_SL + R4(3 * STAR_NNZ);  // [T][8]
    static constexpr int OFF_ZUF = OFF_ZIN + 8 * T_;            // [T][8]
    static constexpr int OFF_ZI = OFF_ZUF + 8 * T_;
    static constexpr int OFF_TAB = OFF_ZI + R4(T_ * T_);   // ints: row_ptr[14], col[54]
    static constexpr int OFF_STAB = OFF_TAB + R4(NQ + 1 + STAR_NNZ);  // float4 [13][STAR_SLOTS]
    static constexpr int OFF_SC = OFF_STAB + 4 * NQ * STAR_SLOTS;  // ints: Q1 exponents [16], D1 exponents [16]
    static constexpr int OFF_BAR = OFF_SC + 32;  // 5 mbarriers, wait limit, TMEM slot, abort, non-finite, dirty, drain mask
    static constexpr int SMEM_FLOATS = OFF_BAR + 18;
    static constexpr int TMEM_COLS = tc_np(N) <= 32 ? 32 : (tc_np(N) <= 64 ? 64 : 128);
    static_assert(A::PT <= 32 * (NW < 4 ? NW : 4), "every accumulator row (p, u) needs a reading warp");
    static_assert(NW == 2 || NW == 4 || NW == 8, "2, 4 or 8 warps");
};

// row[0..T) <- Zi row[0..T), Zi stored with row stride 8 (two 16-byte loads a row)
template <int T>
__device__ __forceinline__ void solve_row8(float* row, const float* Zi) {
    float x[T];
#pragma unroll
    for (int s = 0; s < T; ++s) x[s] = row[s];
#pragma unroll
    for (int u = 0; u < T; ++u) {
        const float4 a = *reinterpret_cast<const float4*>(Zi + 8 * u);
        float z[8] = {a.x, a.y, a.z, a.w, 0.f, 0.f, 0.f, 0.f};
        if constexpr (T > 4) {
            const float4 b = *reinterpret_cast<const float4*>(Zi + 8 * u + 4);
            z[4] = b.x;
            z[5] = b.y;
            z[6] = b.z;
            z[7] = b.w;
        }
        float acc = 0.f;
#pragma unroll
        for (int s = 0; s < T; ++s) acc = fmaf(z[s], x[s], acc);
        row[u] = acc;
    }
}

// Tensor-core state of one CTA (shared addresses, barrier phases).  Thread 0
// issues every MMA commit and the Khat copies needed inside a block; thread
// 96 (a warp with no epilogue rows) issues the next block's copies once the
// block's MMAs are done.  An issuing thread issues only while all of its own
// waits have succeeded.  Thread 0 waits for every copy before the MMAs that
// read it, and thread 96's copies follow MMAs that thread 0 issued only after
// such waits, so no barrier ever gets a second operation while an earlier one
// may still be in flight.
// Each thread keeps in `pend` the barriers it gave work that it has not seen
// complete: bits 0, 1 MMA commits (cleared by the successful wait), bits 2-4
// Khat copies into slots 0-2 (cleared by thread 0's wait on the copy, and by
// every thread once the block's last MMAs are done, which implies that every
// copy of the block was consumed); bit 31 records that one of the thread's
// waits gave up.  The abort path merges the masks of threads 0 and 96.
struct TcState {
    float* xy;      // operand region: A tiles (tf32 words, or bf16 values in the same bytes), then Khat images
    uint32_t xy_s;  // its shared address
    int xy_floats;  // its size
    uint32_t bar_s;     // mbarriers: MMAs done reading A buffer 0, 1; Khat image in slot 0, 1, 2
    uint32_t tmem;
    uint32_t mph, lph;  // phase parity of each barrier (bit b for MMA barrier b, bit 2 + s for slot s)
    uint32_t pend;      // barriers given work not seen complete; bit 31: a wait gave up
    volatile int* abort;
};
constexpr uint32_t GAVE_UP = 1u << 31;

// A wait that gives up keeps its phase, so that the abort path can still
// wait (with the full limit) for the operation it was waiting for
__device__ __forceinline__ void tc_wait(TcState& S, uint32_t bit) {
    const uint32_t par = ((bit < 2 ? S.mph : S.lph) >> bit) & 1u;
    // the wait limit is the 64-bit word after the five mbarriers
    if (tc::mbar_wait_s(S.bar_s + 8u * bit, par, S.bar_s + 40u)) {
        if (bit < 2)
            S.mph ^= 1u << bit;
        else
            S.lph ^= 1u << bit;
        S.pend &= ~(1u << bit);
    } else {
        *S.abort = 1;
        S.pend |= GAVE_UP;
    }
}

// abort path (thread 0, after a CTA barrier, with `mask` the union of the
// issuing threads' records): a wait with the full limit on every barrier
// given work not seen complete, so that copies and MMAs still in flight have
// landed before the CTA frees its TMEM and exits.  Barriers with nothing in
// flight are skipped.  (A copy of thread 96 that thread 0 consumed before an
// MMA wait gave up stays in thread 96's record; its barrier then has no
// pending phase and the wait runs out its limit: bounded, and only on this
// path.)
__device__ __forceinline__ void tc_drain(TcState& S, uint32_t mask) {
    for (uint32_t bit = 0; bit < 5; ++bit)
        if ((mask >> bit) & 1u) tc::mbar_wait(S.bar_s + 8u * bit, ((bit < 2 ? S.mph : S.lph) >> bit) & 1u);
}

// Operand layout of degree block g in the region (floats): nA A buffers (hi
// tile, lo tile), then nB Khat image slots (hi image, lo image).  Direction j
// uses A buffer j % nA and slot j % nB.  An MMA reads 16 row groups of an A
// tile; the rows past 13 T feed accumulator rows that are never read and
// stay inside the region.  As many slots as fit (all three directions' images
// can then be in flight before the block starts), then a second A buffer if
// it fits (the star products of direction j overlap the MMAs of j - 1).
struct TcLayout {
    int KP, NP, ahf, bif, nA, nB;
    uint32_t sbo, half;  // bytes: 8-row group stride; one Khat image (hi or lo)
};
template <int PT, int BF, bool CAPS>
__device__ __forceinline__ TcLayout tc_layout(int g, int xy_floats, int cap_a, int cap_b) {
    constexpr int ES = BF ? 2 : 4;
    TcLayout L;
    L.KP = tc_kp(g, BF != 0);
    L.NP = tc_np(g);
    L.sbo = (uint32_t)L.KP * 8u * ES;
    L.half = (uint32_t)(L.NP * L.KP) * ES;
    L.ahf = (PT + 7) / 8 * (int)(L.sbo / 4);
    L.bif = (int)(2u * L.half / 4u);
    const int over = 16 * (int)(L.sbo / 4) - L.ahf;
    auto fits = [&](int na, int nb) { return 2 * na * L.ahf + nb * L.bif <= xy_floats && (2 * na - 1) * L.ahf + 16 * (int)(L.sbo / 4) <= xy_floats && over >= 0; };
    L.nB = fits(1, 3) ? 3 : (fits(1, 2) ? 2 : 1);
    if (CAPS) L.nB = L.nB < cap_b ? L.nB : cap_b;
    // direction j >= nB loads once the MMAs of j - nB are done, known at step
    // j - nB + nA: that is no later than step j only if nA <= nB.  With three
    // A buffers (and three slots) the block runs all directions in one pass.
    L.nA = (L.nB == 3 && fits(3, 3)) ? 3 : ((L.nB >= 2 && fits(2, L.nB)) ? 2 : 1);
    if (CAPS) L.nA = L.nA < cap_a ? L.nA : cap_a;
    return L;
}

// bulk copy of direction j's Khat image of block g into its slot (one
// thread, unless one of its waits gave up)
template <int PT, int BF>
__device__ __forceinline__ void tc_load_khat(TcState& S, const TcLayout& L, const K2Params& P, int g, int j) {
    if (S.pend & GAVE_UP) return;
    const int slot = j % L.nB;
    S.pend |= 4u << slot;
    const uint32_t bar = S.bar_s + 16u + 8u * (uint32_t)slot;
    const uint32_t dst = S.xy_s + 4u * (uint32_t)(2 * L.nA * L.ahf + slot * L.bif);
    tc::fence_async_smem();
    tc::mbar_expect_tx(bar, 2u * L.half);
    tc::bulk_g2s(dst, reinterpret_cast<const char*>(P.khat_tc) + P.tc_off[g][j], 2u * L.half, bar);
}

// star products of one item (ml, u) of block g (modes o + ml) for direction
// j's 54 coefficients: acc[p] = sum_q A^{j*}_pq Q[q, o+ml, u]
template <int T, int QS>
__device__ __forceinline__ void star_item(const float* bq, const float* sj, int o, int it, float acc[NQ]) {
    const int ml = it / T, u = it % T;
    float qv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        qv[q] = bq[q * QS + (o + ml) * T + u];
        acc[q] = 0.f;
    }
#pragma unroll
    for (int n = 0; n < STAR_NNZ; ++n) acc[star_row(n)] = fmaf(sj[n], qv[star_col(n)], acc[star_row(n)]);
}

// store one item's 13 values as hi + lo (tf32 words, or bf16) into the A tiles
template <int T, int BF>
__device__ __forceinline__ void store_item(float* ah, float* al, int it, int KP, const float acc[NQ]) {
    const int ml = it / T, u = it % T;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (BF) {
            const int at = tc::kmajor_offset16(q * T + u, ml, KP);
            const uint16_t h = tc::bf16_bits(acc[q]);
            reinterpret_cast<uint16_t*>(ah)[at] = h;
            reinterpret_cast<uint16_t*>(al)[at] = tc::bf16_bits(acc[q] - tc::bf16_value(h));
        } else {
            const int at = tc::kmajor_offset(q * T + u, ml, KP);
            const float h = tc::to_tf32(acc[q]);
            ah[at] = h;
            al[at] = acc[q] - h;
        }
    }
}

// One binary32 sweep of Algorithm 3 with the Khat products on the tensor
// cores.  On entry bq holds b, on exit Q.  Returns false (uniformly across the
// CTA) if a bounded wait gave up.
template <int N, int NT, int BF, bool CAPS>
__device__ bool alg3_sweep_tc(float* bq, const float* star, const float* zuf, const float* zin, const float gcoup,
                              const K2Params& P, TcState& S) {
    using A = Alg3Shape<N>;
    constexpr int T = A::T, QS = A::QS, PT = A::PT, NW = NT / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the first block's Khat images load while its time solves run
    if (tid == 0 && N >= 1) {
        const TcLayout L0 = tc_layout<PT, BF, CAPS>(N, S.xy_floats, P.cap_a, P.cap_b);
        for (int j = 0; j < L0.nB; ++j) tc_load_khat<PT, BF>(S, L0, P, N, j);
    }
#pragma unroll 1
    for (int g = N; g >= 0; --g) {
        const int o = block_offset(g), d = block_size(g);
        // time solves of block g: 7 plain rows (6 stresses, p) and 3 coupled
        // pairs (u_f then u, v_f then v, w_f then w) per mode
        for (int it = tid; it < 10 * d; it += NT) {
            const int kind = it / d, m = o + it % d;
            if (kind < 7) {
                const int p = kind < 6 ? kind : QP;
                solve_row8<T>(bq + p * QS + m * T, zin);
            } else {
                const int i = kind - 7;
                float* rf = bq + (QUF + i) * QS + m * T;
                float* rv = bq + (QU + i) * QS + m * T;
                solve_row8<T>(rf, zuf);
#pragma unroll
                for (int u = 0; u < T; ++u) rv[u] = fmaf(gcoup, rf[u], rv[u]);
                solve_row8<T>(rv, zin);
            }
        }
        __syncthreads();
        if (g == 0) break;
        constexpr int KSTEP = BF ? 16 : 8;
        const TcLayout L = tc_layout<PT, BF, CAPS>(g, S.xy_floats, P.cap_a, P.cap_b);
        const int KP = L.KP, NP = L.NP;
        const uint32_t sbo = L.sbo, half = L.half;
        if (L.nA == 3) {
            // small block: the star products of all three directions in one
            // pass, one barrier, then every direction's MMAs and one commit
            for (int it = tid; it < 3 * d * T; it += NT) {
                const int j = it / (d * T), r = it - j * (d * T);
                float acc[NQ];
                star_item<T, QS>(bq, star + j * STAR_NNZ, o, r, acc);
                store_item<T, BF>(S.xy + 2 * j * L.ahf, S.xy + (2 * j + 1) * L.ahf, r, KP, acc);
            }
            tc::fence_async_smem();
            __syncthreads();
            if (*S.abort) return false;
            if (tid == 0) {
                for (int j = 0; j < 3; ++j) tc_wait(S, 2u + (uint32_t)j);
            }
            if (tid == 0 && !(S.pend & GAVE_UP)) {
                tc::fence_after_sync();
                const uint32_t id = BF ? tc::idesc_bf16(128, NP) : tc::idesc_tf32(128, NP);
                const int nk = KP / KSTEP;
                constexpr int MAXK = tc_kp(N, BF != 0) / KSTEP;
                for (int j = 0; j < 3; ++j) {
                    const uint32_t ah_s = S.xy_s + 4u * (uint32_t)(2 * j * L.ahf), al_s = ah_s + 4u * (uint32_t)L.ahf;
                    const uint32_t b_s = S.xy_s + 4u * (uint32_t)(6 * L.ahf + j * L.bif);
                    const uint64_t dal = tc::smem_desc(al_s, sbo), dah = tc::smem_desc(ah_s, sbo);
                    const uint64_t dbh = tc::smem_desc(b_s, sbo), dbl = tc::smem_desc(b_s + half, sbo);
#pragma unroll
                    for (int kk = 0; kk < MAXK; ++kk) {
                        if (kk < nk) {
                            const uint64_t k16 = 16ull * (uint64_t)kk;
                            if (BF) {
                                tc::mma_bf16(S.tmem, dal + k16, dbh + k16, id, (j | kk) != 0);
                                tc::mma_bf16(S.tmem, dah + k16, dbl + k16, id, 1u);
                                tc::mma_bf16(S.tmem, dah + k16, dbh + k16, id, 1u);
                            } else {
                                tc::mma_tf32(S.tmem, dal + k16, dbh + k16, id, (j | kk) != 0);
                                tc::mma_tf32(S.tmem, dah + k16, dbl + k16, id, 1u);
                                tc::mma_tf32(S.tmem, dah + k16, dbh + k16, id, 1u);
                            }
                        }
                    }
                }
                tc::mma_commit(S.bar_s);
                S.pend |= 1u;
            }
            tc_wait(S, 0u);
            // the block's MMAs are done: every copy of the block was consumed
            if (!(S.pend & GAVE_UP)) S.pend &= ~0x1Cu;
        } else {
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            const int abuf = j % L.nA, slot = j % L.nB;
            const uint32_t mma_bar = S.bar_s + 8u * (uint32_t)abuf;
            if (j >= L.nA) {  // the MMAs of direction j - nA (and all before) are done
                tc_wait(S, (uint32_t)abuf);
                // their slots are free: load the images not yet in flight
                if (tid == 0)
                    for (int k = L.nB; k < 3; ++k)
                        if (k - L.nB <= j - L.nA && k - L.nB > j - 1 - L.nA) tc_load_khat<PT, BF>(S, L, P, g, k);
            }
            float* ah = S.xy + 2 * abuf * L.ahf;
            float* al = ah + L.ahf;
            const uint32_t ah_s = S.xy_s + 4u * (uint32_t)(2 * abuf * L.ahf), al_s = ah_s + 4u * (uint32_t)L.ahf;
            const uint32_t b_s = S.xy_s + 4u * (uint32_t)(2 * L.nA * L.ahf + slot * L.bif);
            // X^j[p, ml, u] = sum_q A^{j*}_pq Q[q, o+ml, u], stored as hi + lo
            // (tf32 words, or bf16)
            const float* sj = star + j * STAR_NNZ;
            for (int it = tid; it < d * T; it += NT) {
                float acc[NQ];
                star_item<T, QS>(bq, sj, o, it, acc);
                store_item<T, BF>(ah, al, it, KP, acc);
            }
            tc::fence_async_smem();
            __syncthreads();
            if (*S.abort) return false;
            if (tid == 0) tc_wait(S, 2u + (uint32_t)slot);
            if (tid == 0 && !(S.pend & GAVE_UP)) {
                tc::fence_after_sync();
                const uint32_t id = BF ? tc::idesc_bf16(128, NP) : tc::idesc_tf32(128, NP);
                // one K step = two core matrices along K, 256 B further: 16
                // units of the descriptors' start-address field (no carry,
                // shared addresses are below 2^18)
                const uint64_t dal = tc::smem_desc(al_s, sbo), dah = tc::smem_desc(ah_s, sbo);
                const uint64_t dbh = tc::smem_desc(b_s, sbo), dbl = tc::smem_desc(b_s + half, sbo);
                const int nk = KP / KSTEP;
                constexpr int MAXK = tc_kp(N, BF != 0) / KSTEP;
#pragma unroll
                for (int kk = 0; kk < MAXK; ++kk) {
                    if (kk < nk) {
                        const uint64_t k16 = 16ull * (uint64_t)kk;
                        if (BF) {
                            tc::mma_bf16(S.tmem, dal + k16, dbh + k16, id, (j | kk) != 0);
                            tc::mma_bf16(S.tmem, dah + k16, dbl + k16, id, 1u);
                            tc::mma_bf16(S.tmem, dah + k16, dbh + k16, id, 1u);
                        } else {
                            tc::mma_tf32(S.tmem, dal + k16, dbh + k16, id, (j | kk) != 0);
                            tc::mma_tf32(S.tmem, dah + k16, dbl + k16, id, 1u);
                            tc::mma_tf32(S.tmem, dah + k16, dbh + k16, id, 1u);
                        }
                    }
                }
                tc::mma_commit(mma_bar);
                S.pend |= 1u << abuf;
            }
        }
        // wait for the commits not yet waited for (directions 3 - nA .. 2);
        // the last one covers every MMA of the block
#pragma unroll 1
        for (int j = 3 - L.nA; j < 3; ++j) {
            tc_wait(S, (uint32_t)(j % L.nA));
        }
        // the block's MMAs are done: every copy of the block was consumed
        if (!(S.pend & GAVE_UP)) S.pend &= ~0x1Cu;
        }
        // the region is free: the next block's Khat images load during this
        // block's epilogue and the next time solves (issued by lane 0 of warp
        // 3, whose TMEM lane quarter holds no rows: 13 T <= 96)
        if (tid == (NW >= 4 ? 96 : 0) && g > 1) {
            const TcLayout Ln = tc_layout<PT, BF, CAPS>(g - 1, S.xy_floats, P.cap_a, P.cap_b);
            for (int j = 0; j < Ln.nB; ++j) tc_load_khat<PT, BF>(S, Ln, P, g - 1, j);
        }
        tc::fence_after_sync();
        // b[p, l, u] -= D[(p, u), l]: warp w reads TMEM lanes 32 (w % 4) ...,
        // with 8 warps the two warps of a lane quarter split the columns
        {
            const int sp = warp & 3;
            const int ncol = NW == 8 ? NP / 2 : NP;
            const int c_begin = NW == 8 ? (warp >> 2) * ncol : 0;
            // a warp with a lane whose wait gave up reads no TMEM (the MMAs
            // may still be writing it); the CTA leaves the sweep below
            const bool skip = __any_sync(0xffffffffu, (S.pend & GAVE_UP) != 0u);
            if (sp * 32 < PT && !skip) {
                const int r = sp * 32 + lane;
                const int p = r / T, u = r - (r / T) * T;
                float* dst = bq + p * QS + u;
                const int c_end = min(c_begin + ncol, o);
#pragma unroll 1
                for (int c0 = c_begin; c0 < c_end; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(S.tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)c0, v);
                    if (r < PT) {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (c0 + q < c_end) dst[(c0 + q) * T] -= v[q];
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (*S.abort) return false;
    }
    return true;
}

// Residual lanes by star width: the 13 T pairs (p, u) ordered as rows
// {sxx, syy, szz, p} (6 entries per direction), {u, v, w, uf, vf, wf} (4),
// {sxy, syz, sxz} (2); slot s -> p * T + u, or -1 past the last pair
__host__ __device__ constexpr int r2_class(int T, int s) { return s < 4 * T ? 0 : (s < 10 * T ? 1 : 2); }
__host__ __device__ constexpr int r2_slot(int T, int s) {
    return s >= NQ * T ? -1
           : s < 4 * T ? ((s / T) < 3 ? s / T : QP) * T + s % T
           : s < 10 * T ? (((s - 4 * T) / T) < 3 ? QU + (s - 4 * T) / T : QUF + (s - 4 * T) / T - 3) * T + (s - 4 * T) % T
                        : (SXY + (s - 10 * T) / T) * T + (s - 10 * T) % T;
}

// Q1 / D1 of the residual: fixed-point integers, mode-major,
// Q[m * Q1S + p * T + u] (the (q, u) lanes of one mode are consecutive
// words); the value is Q * 2^-sq[p] with |Q| <= 2^22
template <int N, int REF, int NT_>
__device__ void residual(float* W, const int* Q1, const int* D1, const int* sq, const int* sd, const float4* stab,
                         const int* zneg, float2 e_dw, float2 g_dw, float2* Yall, const K2Params& P) {
    using S = K2Shape<N, REF, NT_>;
    constexpr int B = S::B, T = S::T, PT = S::PT, PUL = S::PUL, QS = S::QS, Q1S = S::Q1S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* Y = Yall + warp * 3 * PT;
    const int i0 = __ldg(P.res_order + warp), i1 = __ldg(P.res_order + warp + 1);
#pragma unroll 1
    for (int i = i0; i < i1; ++i) {
        const int l = __ldg(P.res_order + S::NW + 1 + i);  // this warp's rows (balanced lists)
        // R1: Y^j[q, u] = (1 / d_jl) sum_m c_jlm Q[q, m, u]: integer numerators
        // times integer Q, summed exactly in 64 bits (sum_m |c_jlm| < 2^22 and
        // |Q| <= 2^22, so |sum| <= 2^44)
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            long long ya[PUL], yd[PUL];
#pragma unroll
            for (int k = 0; k < PUL; ++k) ya[k] = yd[k] = 0;
            const int32_t* cr = c_res + res_base(N);
            const int32_t* ce = cr + 3 * (B + 1);
            const int n0 = cr[j * (B + 1) + l], n1 = cr[j * (B + 1) + l + 1];
#pragma unroll 4
            for (int n = n0; n < n1; ++n) {
                const int kv = ce[n];
                const long long cv = (long long)(kv >> 7);
                const int mo = (kv & 127) * Q1S + lane;
#pragma unroll
                for (int k = 0; k < PUL; ++k) {
                    ya[k] += cv * Q1[mo + 32 * k];
                    if (REF == 2) yd[k] += cv * D1[mo + 32 * k];
                }
            }
            const float2 inv = __ldg(P.res_inv + j * B + l);
#pragma unroll
            for (int k = 0; k < PUL; ++k) {
                const int pu = lane + 32 * k;
                const int q = pu < PT ? pu / T : 0;
                float yh, yl;
                int_to_dw(ya[k], yh, yl);
                const float f = pow2f(-sq[q]);
                float2 y = make_float2(__fmul_rn(yh, f), __fmul_rn(yl, f));
                if (REF == 2) {
                    int_to_dw(yd[k], yh, yl);
                    const float fd = pow2f(-sd[q]);
                    y = dw_add(y, make_float2(__fmul_rn(yh, fd), __fmul_rn(yl, fd)));
                }
                float h = 0.f, lo = 0.f;
                dw_mac(h, lo, inv.x, inv.y, y.x, y.y);
                if (pu < PT) Y[j * PT + pu] = make_float2(h, lo);
            }
        }
        // R2 lanes are dealt by the width of row p's star pattern (6, 4 or 2
        // entries per direction), so a warp's padded star loop is as short as
        // its widest row: slot s -> (p, u) via r2_slot
        // b0[p, l] (hi, lo) sits in W[p, l, 0..1]; read before row l is written
        float2 bv[PUL];
#pragma unroll
        for (int k = 0; k < PUL; ++k) {
            const int pu = r2_slot(T, lane + 32 * k);
            const int p = pu >= 0 ? pu / T : 0;
            bv[k] = make_float2(W[p * QS + l * T], W[p * QS + l * T + 1]);
        }
        __syncwarp();
        // R2: assemble r[p, l, u]
#pragma unroll
        for (int k = 0; k < PUL; ++k) {
            const int pu = r2_slot(T, lane + 32 * k);
            constexpr int WID[3] = {6, 4, 2};
            const int wk = WID[r2_class(T, 32 * k)];  // widest row of this slot
            if (pu >= 0) {
                const int p = pu / T, u = pu % T;
                const int bq = l * Q1S + p * T;
                // - sum_s Z_us Q[p, l, s]: Z's entries are small integers, so the
                // sum is an exact integer (|sum| < 2^29)
                int za = 0, zd = 0;
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    za += zneg[u * T + s] * Q1[bq + s];
                    if (REF == 2) zd += zneg[u * T + s] * D1[bq + s];
                }
                float h, lo;
                {
                    float zh, zl;
                    int_to_dw(za, zh, zl);
                    const float f = pow2f(-sq[p]);
                    h = __fmul_rn(zh, f);
                    lo = __fmul_rn(zl, f);
                    if (REF == 2) {
                        int_to_dw(zd, zh, zl);
                        const float fd = pow2f(-sd[p]);
                        const float2 z2 = dw_add(make_float2(h, lo), make_float2(__fmul_rn(zh, fd), __fmul_rn(zl, fd)));
                        h = z2.x;
                        lo = z2.y;
                    }
                }
                const float sw = (float)((2 * u + 1) * ((u & 1) ? -1 : 1));
                dw_mac_x2(h, lo, sw, bv[k].x, bv[k].y);
                // + E*_pp Q[p, l, u] (u_f rows) and + G Q[u_f, l, u] (u rows)
                if (p >= QUF || (p >= QU && p <= QW)) {
                    const int ps = p >= QUF ? p : p + (QUF - QU);
                    const int src = l * Q1S + ps * T + u;
                    const float2 c = p >= QUF ? e_dw : g_dw;
                    const float qv = __fmul_rn(small_int_to_float(Q1[src]), pow2f(-sq[ps]));
                    if (REF == 2)
                        dw_mac(h, lo, c.x, c.y, qv, __fmul_rn(small_int_to_float(D1[src]), pow2f(-sd[ps])));
                    else
                        dw_mac1(h, lo, c.x, c.y, qv);
                }
                // - sum_j sum_q A^{j*}_pq Y^j[q, u]: row p's entries of each
                // direction, padded to the slot width
                // (-coef hi, -coef lo, offset of Y^j[q, 0])
                const float4* st = stab + p * STAR_SLOTS;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int t = 0; t < 6; ++t) {
                        if (t < wk) {
                            const float4 c = st[j * 6 + t];
                            const float2 yv = Y[__float_as_int(c.z) + u];
                            dw_mac(h, lo, c.x, c.y, yv.x, yv.y);
                        }
                    }
                W[p * QS + l * T + u] = __fadd_rn(h, lo);
            }
        }
        __syncwarp();
    }
    // the Y buffers share memory with the tensor-core tiles that bulk copies
    // and MMAs touch next
    tc::fence_async_smem();
}

// Save the sweep result W into dst as fixed-point integers and put the
// double-binary32 split of b0 = q0 into W[p, l, 0..1] for the residual.
// Quantity p is rounded to the grid 2^-sc[p] with sc[p] chosen from
// max_{l,u} |W[p, l, u]| so that every integer has |v| <= 2^22: the residual
// then takes exact integer products, and the refinement corrects the rounding
// (~2^-23 of the quantity's largest entry) like any other error of the sweep.
// A non-finite value raises *nonfinite, which turns the element's output into
// NaN.
template <int N, int REF, int NT_>
__device__ void stash_sweep(int* dst, int* sc, int* nonfinite, float* W, const double* q0) {
    using S = K2Shape<N, REF, NT_>;
    constexpr int B = S::B, T = S::T, QS = S::QS, Q1S = S::Q1S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int p = warp; p < NQ; p += S::NW) {
        uint32_t m = 0;
        for (int i = lane; i < B * T; i += 32) m = max(m, __float_as_uint(W[p * QS + i]) & 0x7FFFFFFFu);
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) {
            const int e = (int)(m >> 23) - 127;  // max in [2^e, 2^(e+1)), so max 2^sc < 2^22
            sc[p] = min(21 - e, 126);
            if (e == 128) *nonfinite = 1;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NQ * B; i += NT_) {
        const int p = i / B, l = i - (i / B) * B;
        float* w = W + p * QS + l * T;
        int* d = dst + l * Q1S + p * T;
        const float f = pow2f(sc[p]);
#pragma unroll
        for (int u = 0; u < T; ++u) d[u] = round_to_int(w[u], f);
        const float2 b = dw_split(q0[i]);
        w[0] = b.x;
        w[1] = b.y;
    }
}

template <int N, int REF, int NT_, int BF, bool CAPS>
__global__ void __launch_bounds__(NT_, (REF == 2 || NT_ > 256) ? 1 : 2) stp_mixed_kernel(const K2Params P) {
    using S = K2Shape<N, REF, NT_, BF>;
    constexpr int B = S::B, T = S::T, NT = S::NT, QBT = S::QBT, QS = S::QS;
    extern __shared__ __align__(1024) float smf[];
    float* W = smf + S::OFF_W;
    int* Q1 = reinterpret_cast<int*>(smf + S::OFF_Q1);
    int* D1 = reinterpret_cast<int*>(smf + S::OFF_D1);
    int* sq = reinterpret_cast<int*>(smf + S::OFF_SC);
    int* sd = sq + 16;
    float2* Yall = reinterpret_cast<float2*>(smf + S::OFF_XY);
    float* sh = smf + S::OFF_SH;
    float* sl = smf + S::OFF_SL;
    float* zin = smf + S::OFF_ZIN;
    float* zuf = smf + S::OFF_ZUF;
    int* zneg = reinterpret_cast<int*>(smf + S::OFF_ZI);
    int* tab = reinterpret_cast<int*>(smf + S::OFF_TAB);
    float4* stab = reinterpret_cast<float4*>(smf + S::OFF_STAB);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smf + S::OFF_BAR);
    long long* wlimit = reinterpret_cast<long long*>(smf + S::OFF_BAR + 10);  // wait limit (SM clocks)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smf + S::OFF_BAR + 12);
    volatile int* abort = reinterpret_cast<volatile int*>(smf + S::OFF_BAR + 13);
    int* nonfinite = reinterpret_cast<int*>(smf + S::OFF_BAR + 14);
    int* dirty = reinterpret_cast<int*>(smf + S::OFF_BAR + 15);  // a result was not finite
    uint32_t* drain_mask = reinterpret_cast<uint32_t*>(smf + S::OFF_BAR + 16);  // thread 96's record, at exit
    const int tid = threadIdx.x;

    TcState tcs;
    tcs.xy = smf + S::OFF_XY;
    tcs.xy_s = tc::smem_addr(tcs.xy);
    tcs.xy_floats = S::XY_SIZE;
    tcs.bar_s = tc::smem_addr(bars);
    tcs.mph = tcs.lph = 0;
    tcs.pend = 0;
    tcs.abort = abort;

    // operand region starts finite (K padding of A meets zeros of B)
    for (int i = tid; i < S::XY_SIZE; i += NT) smf[S::OFF_XY + i] = 0.f;
    for (int i = tid; i < T * T; i += NT) {
        const int u = i / T, s = i % T;
        zin[8 * u + s] = P.zinv[i];
        zneg[i] = -(2 * u + 1) * ((u > s && ((u - s) & 1)) ? -1 : 1);  // -Z, Z = S^{-1}(W - K^tau)
    }
    for (int i = tid; i < NQ + 1 + STAR_NNZ; i += NT) tab[i] = c_star_tab[i];
    if (tid == 0) {
        *wlimit = P.wait_limit;
        *abort = 0;
        *dirty = 0;
        for (int b = 0; b < 5; ++b) tc::mbar_init(tcs.bar_s + 8u * (uint32_t)b, 1);
        tc::mbar_init_fence();
    }
    if (tid < 32) tc::tmem_alloc(tc::smem_addr(tslot), S::TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tcs.tmem = *tslot;

    for (int64_t it = blockIdx.x; it < P.count; it += gridDim.x) {
        const int64_t e = P.elems ? (int64_t)P.elems[it] : it;
        const double* q0 = (P.runs ? P.runs[P.item_run[it]].q0 : P.q0) + e * (int64_t)(NQ * B);
        const double* ec = (P.runs ? P.runs[P.item_run[it]].econst : P.econst) + e * (int64_t)P.stride;
        // a wait of another CTA of this context gave up: skip the remaining
        // elements (the launch's results are reported as failed anyway)
        const int failed = (tid == 0 && P.status) ? *reinterpret_cast<volatile const int32_t*>(P.status) : 0;
        if (tid == 0) *nonfinite = 0;  // read after the barriers below
        for (int i = tid; i < 3 * STAR_NNZ; i += NT) {
            const float2 v = dw_split(ec[i]);
            sh[i] = v.x;
            sl[i] = v.y;
        }
        for (int i = tid; i < T * T; i += NT) zuf[8 * (i / T) + i % T] = (float)ec[ec_zinv(N) + i];
        if (REF >= 1)
            for (int i = tid; i < NQ * STAR_SLOTS; i += NT) {
                const int p = i / STAR_SLOTS, t = i % STAR_SLOTS, j = t / 6, idx = tab[p] + t % 6;
                float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
                if (idx < tab[p + 1]) {
                    const float2 v = dw_split(ec[j * STAR_NNZ + idx]);
                    c = make_float4(-v.x, -v.y, __int_as_float(j * S::PT + tab[NQ + 1 + idx] * T), 0.f);
                }
                stab[i] = c;
            }
        const double* scal = ec + 3 * STAR_NNZ + T * T;
        const float2 e_dw = dw_split(scal[0]), g_dw = dw_split(scal[1]);
        const double dt = scal[2];
        // Q1 = Alg3_f32(b0), b0[p, l, u] = (S^{-1} w)_u q0[p, l]
        for (int i = tid; i < NQ * B; i += NT) {
            const float v = (float)q0[i];
            float* row = W + (i / B) * QS + (i % B) * T;
#pragma unroll
            for (int u = 0; u < T; ++u) row[u] = (float)((2 * u + 1) * ((u & 1) ? -1 : 1)) * v;
        }
        if (failed) *abort = 1;
        __syncthreads();
        if (*abort) break;
        if (!alg3_sweep_tc<N, NT, BF, CAPS>(W, sh, zuf, zin, g_dw.x, P, tcs)) break;
        if (REF >= 1) {
            stash_sweep<N, REF, NT_>(Q1, sq, nonfinite, W, q0);
            if (REF == 2) {
                for (int i = tid; i < S::Q1SIZE; i += NT) D1[i] = 0;
                if (tid < NQ) sd[tid] = 0;
            }
            __syncthreads();
        }
        bool ok = true;
#pragma unroll 1
        for (int sweep = 1; sweep <= REF && ok; ++sweep) {
            residual<N, REF, NT_>(W, Q1, D1, sq, sd, stab, zneg, e_dw, g_dw, Yall, P);
            __syncthreads();
            ok = alg3_sweep_tc<N, NT, BF, CAPS>(W, sh, zuf, zin, g_dw.x, P, tcs);
            if (ok && REF == 2 && sweep == 1) {
                stash_sweep<N, REF, NT_>(D1, sd, nonfinite, W, q0);
                __syncthreads();
            }
        }
        if (!ok) break;
        // Q = Q1 (+ d1) (+ d2) in binary64; time integration
        double* qtb = P.runs ? P.runs[P.item_run[it]].qt : P.qt;
        double* iob = P.runs ? P.runs[P.item_run[it]].iout : P.iout;
        if (qtb || iob) {
            double* qo = qtb ? qtb + e * (int64_t)QBT : nullptr;
            double* io = iob ? iob + e * (int64_t)(NQ * B) : nullptr;
            // one (p, l) row of T time modes per thread
            bool bad = false;
            for (int i = tid; i < NQ * B; i += NT) {
                const int p = i / B, l = i - (i / B) * B;
                const float* w = W + p * QS + l * T;
                const int* q1 = Q1 + l * S::Q1S + p * T;
                const int* d1 = D1 + l * S::Q1S + p * T;
                const float fq = REF >= 1 ? pow2f(-sq[p]) : 0.f, fd = REF == 2 ? pow2f(-sd[p]) : 0.f;
#pragma unroll
                for (int u = 0; u < T; ++u) {
                    bad |= (__float_as_uint(w[u]) & 0x7F800000u) == 0x7F800000u;
                    double v;
                    if (REF == 0) {
                        v = __longlong_as_double((long long)f2d_bits(w[u]));
                    } else {
                        float sv, ev;
                        two_sum(__fmul_rn(small_int_to_float(q1[u]), fq), w[u], sv, ev);
                        if (REF == 2) {
                            float s2, e2;
                            two_sum(sv, __fmul_rn(small_int_to_float(d1[u]), fd), s2, e2);
                            ev = __fadd_rn(ev, e2);
                            sv = __fadd_rn(s2, ev);  // renormalise: |ev| <= ulp(sv) / 2
                            ev = __fsub_rn(ev, __fsub_rn(sv, s2));
                        }
                        v = pair_to_double(sv, ev);
                        if (*nonfinite) v = __longlong_as_double(0x7FF8000000000000LL);
                    }
                    if (qo) qo[(int64_t)i * T + u] = v;
                    if (io && u == 0) io[i] = dt * v;
                }
            }
            if (bad) *dirty = 1;
        }
        __syncthreads();
        // a non-finite result may have left non-finite words in the operand
        // region, where the next element's A-tile padding (multiplied by the
        // zero padding of the Khat images) would turn them into NaN: clear it
        if (*dirty || (REF >= 1 && *nonfinite)) {
            for (int i = tid; i < S::XY_SIZE; i += NT) smf[S::OFF_XY + i] = 0.f;
            tc::fence_async_smem();  // before the bulk copies into the region
            __syncthreads();
            if (tid == 0) *dirty = 0;
        }
    }
    // the issuing threads' records of work not seen complete (empty unless a
    // wait gave up: every copy and commit is waited for otherwise)
    if (tid == (S::NW >= 4 ? 96 : 0)) *drain_mask = tcs.pend & 0x1Fu;
    __syncthreads();
    if (tid == 0) {
        const uint32_t mask = (tcs.pend | *drain_mask) & 0x1Fu;
        if (mask) tc_drain(tcs, mask);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort && P.status) atomicExch(P.status, 1);
    if (tid < 32) tc::tmem_dealloc(tcs.tmem, S::TMEM_COLS);
}

template <int N, int REF, int NT_, int BF>
int launch_nr(const MixedReference& ref, const int32_t* elems, int64_t count, const double* q0, const double* econst,
              double* qt, double* iout, void* stream, const RunPtrs* runs, const int32_t* item_run) {
    using S = K2Shape<N, REF, NT_, BF>;
    K2Params P;
    P.elems = elems;
    P.q0 = q0;
    P.econst = econst;
    P.qt = qt;
    P.iout = iout;
    P.count = count;
    P.stride = elem_const_stride(N);
    P.res_inv = reinterpret_cast<const float2*>(ref.res_inv);
    P.res_order = NT_ == 256 ? ref.res_order8 : (NT_ == 128 ? ref.res_order4 : ref.res_order2);
    P.zinv = ref.zinv_f32;
    P.khat_tc = ref.khat_tc;
    for (int g = 0; g <= MAX_N; ++g)
        for (int j = 0; j < 3; ++j) P.tc_off[g][j] = ref.tc_off[g][j];
    P.status = ref.status;
    P.wait_limit = ref.wait_limit > 0 ? ref.wait_limit : tc::WAIT_LIMIT_CYCLES;
    P.runs = runs;
    P.item_run = item_run;
    P.cap_a = ref.cap_a;
    P.cap_b = ref.cap_b;
    // one CTA per element; every resident CTA holds TMEM_COLS columns of the
    // SM's 512, so the shared-memory request is raised where needed to keep
    // at most 512 / TMEM_COLS CTAs of this kernel resident on an SM (so no
    // CTA of this kernel waits for TMEM behind another one of it).  Kernels
    // of different degrees running concurrently on other streams (the
    // server's requests) can together ask for more than 512 columns; a CTA
    // then waits in tcgen05.alloc until a CTA of the other kernel exits and
    // frees its columns.  That CTA depends on nothing of this one and all of
    // its waits are bounded, so the allocation wait ends too.
    int dev = 0, sm_smem = 0, reserved = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (err != cudaSuccess) return (int)err;
    size_t smem = sizeof(float) * S::SMEM_FLOATS;
    const size_t floor_smem = (size_t)sm_smem / (512 / S::TMEM_COLS + 1) + 64;
    if (smem + (size_t)reserved < floor_smem) smem = floor_smem - (size_t)reserved;
    // the default layout (as many buffers as fit) runs the kernel without caps;
    // the autotuner's capped layouts run a second instantiation, built for one
    // refinement sweep (the default) only
    const bool caps = REF == 1 && (P.cap_a < 3 || P.cap_b < 3);
    auto* kern = caps ? stp_mixed_kernel<N, REF, NT_, BF, REF == 1> : stp_mixed_kernel<N, REF, NT_, BF, false>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    if (count <= 0) return 0;
    const int64_t grid = count < (int64_t)(1u << 30) ? count : (int64_t)(1u << 30);
    kern<<<(unsigned)grid, S::NT, smem, (cudaStream_t)stream>>>(P);
    return (int)cudaGetLastError();
}

template <int N, int NT_, int BF>
int launch_nv(const MixedReference& ref, int refine, const int32_t* elems, int64_t count, const double* q0,
              const double* econst, double* qt, double* iout, void* stream, const RunPtrs* runs,
              const int32_t* item_run) {
    switch (refine) {
        case 0: return launch_nr<N, 0, NT_, BF>(ref, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 1: return launch_nr<N, 1, NT_, BF>(ref, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 2: return launch_nr<N, 2, NT_, BF>(ref, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <int N>
int launch_n(const MixedReference& ref, int refine, int variant, const int32_t* elems, int64_t count,
             const double* q0, const double* econst, double* qt, double* iout, void* stream, const RunPtrs* runs,
             const int32_t* item_run) {
    // the bf16 form is built for the default CTA size only
    if (ref.bf16)
        return launch_nv<N, K2Sizes<N>::NT0, 1>(ref, refine, elems, count, q0, econst, qt, iout, stream, runs,
                                                 item_run);
    if (variant == 1)
        return launch_nv<N, K2Sizes<N>::NT1, 0>(ref, refine, elems, count, q0, econst, qt, iout, stream, runs,
                                                 item_run);
    return launch_nv<N, K2Sizes<N>::NT0, 0>(ref, refine, elems, count, q0, econst, qt, iout, stream, runs, item_run);
}

}  // namespace

int upload_residual_table(int N, const int32_t* rows, const int32_t* entries, int n_entries) {
    const int B = n_modes(N);
    if (N < 1 || N > MAX_N || 3 * (B + 1) + n_entries != res_words(N)) return (int)cudaErrorInvalidValue;
    // once per (device, N): later contexts find the same data in place
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, N})) return 0;
    const int base = res_base(N);
    e = cudaMemcpyToSymbol(c_res, rows, sizeof(int32_t) * 3 * (B + 1), sizeof(int32_t) * base);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_res, entries, sizeof(int32_t) * n_entries, sizeof(int32_t) * (base + 3 * (B + 1)));
    if (e == cudaSuccess) done.insert({dev, N});
    return (int)e;
}

int launch_stp_mixed(const MixedReference& ref, int refine, const int32_t* elems, int64_t count, const double* q0,
                     const double* econst, double* qt, double* iout, void* stream, int variant, const RunPtrs* runs,
                     const int32_t* item_run) {
    switch (ref.base->N) {
        case 1: return launch_n<1>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 2: return launch_n<2>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 3: return launch_n<3>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 4: return launch_n<4>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 5: return launch_n<5>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        case 6: return launch_n<6>(ref, refine, variant, elems, count, q0, econst, qt, iout, stream, runs, item_run);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace poro
