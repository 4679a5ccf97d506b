// C ABI of libporoader (declared in include/poroader.h).  Argument checks,
// context state, device memory and the dispatch to the kernels.  No compute
// on the host beyond the per-element set-up of constants.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "poro_internal.h"
#include "tc_device.cuh"

using poro::NQ;

struct poro_ctx {
    int device = 0;
    int N = 0, B = 0, T = 0;
    int system = PORO_SYSTEM_BIOT;
    int nq = NQ;                   // quantities of the system (13 Biot, 6 damped Maxwell)
    poro_precision prec = PORO_FP64;
    cudaStream_t stream = nullptr;
    // copy streams and chunk events of poro_predict_host (created on first use)
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_k;
    poro::ReferenceData ref;
    poro::DeviceReference dref;
    poro::MixedReference mref;
    poro::LUReference lref;
    poro::LUScratch lu;
    int64_t lu_first = 0, lu_count = 0;
    int refine = 1;
    int variant = 0;   // predictor CTA-size variant (poro_autotune)
    int64_t n_elem = 0;
    int stride = 0;
    double* d_econst = nullptr;
    double* d_q0 = nullptr;
    double* d_qt = nullptr;
    double* d_iout = nullptr;
    bool have_dofs = false, have_pred = false;
    // ---- sub-cell material population (poro_set_isolated_subcell)
    bool subcell = false;
    double* d_evar = nullptr;                  // [n][subcell_var_stride()]
    int32_t* d_iters = nullptr;                // [n] iterations of the last predictor
    poro::SubcellReference sub;                // mass 3-tensors (built on first use)
    double sub_tol = 1e-13;
    int sub_max_iter = 100;
    std::string err;
    // ---- mesh mode (corrector, sources, receivers, time stepping)
    bool mesh_mode = false, have_mat = false, ready = false;
    std::vector<double> h_xyz;
    std::vector<int64_t> h_tet, h_nb;
    std::vector<int32_t> h_tag;
    std::vector<poro_material> h_mat;
    double dt = 0.0, t = 0.0;
    poro::CorrectorData cd;
    int32_t *d_nb = nullptr, *d_tab = nullptr, *d_vrow = nullptr, *d_vcol = nullptr;
    double *d_fc = nullptr, *d_fF = nullptr, *d_Pf = nullptr, *d_Pnb = nullptr, *d_vval = nullptr,
           *d_minv = nullptr;
    float *d_fF2 = nullptr, *d_Pf2 = nullptr, *d_Pnb2 = nullptr, *d_vval2 = nullptr;  // (hi, lo) pairs
    struct Source {
        int64_t elem;
        double* d_coef;
        double f0, t0;
    };
    std::vector<Source> sources;
    std::vector<int64_t> rec_elem;
    std::vector<double> rec_phi;
    std::vector<std::vector<double>> seis_q;   // per receiver [n][13]
    std::vector<std::vector<double>> seis_t;   // per receiver sample times
    // clustered local time stepping
    int C = 1;
    int64_t tick = 0;                          // ticks of dt (the smallest step) done
    std::vector<int32_t> h_cl;                 // cluster of each element
    std::vector<std::vector<int32_t>> cl_elems;
    std::vector<int32_t*> d_cl_elems;
    int32_t *d_cl = nullptr, *d_slot = nullptr;
    double* d_buf = nullptr;
    std::vector<char> cl_has_slot;             // a cluster with elements that buffer for a larger neighbour
    bool use_graphs = true;
    int64_t* d_tick = nullptr;                 // device copy of the tick counter (graph replays)
    // persistent receiver buffers (no allocation in steady-state advances)
    double *d_rp = nullptr, *d_seis = nullptr;
    int32_t* d_cnt = nullptr;
    int64_t seis_cap = 0;                      // samples per receiver d_seis holds
    size_t rp_n = 0;                           // receivers uploaded to d_rp
    std::vector<double> h_seis;                // staging for the D2H copy
};

namespace {
thread_local std::string g_err;

poro_status fail(poro_ctx* c, poro_status s, const std::string& msg) {
    if (c) c->err = msg; else g_err = msg;
    return s;
}

poro_status cuda_fail(poro_ctx* c, cudaError_t e, const char* where) {
    return fail(c, PORO_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

cudaError_t upload(void** dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMalloc(dst, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) return e;
    if (bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return e;
}

void free_lu(poro_ctx* c);

void free_mesh_device(poro_ctx* c) {
    dfree(c->d_nb);
    dfree(c->d_tab);
    dfree(c->d_vrow);
    dfree(c->d_vcol);
    dfree(c->d_fc);
    dfree(c->d_fF);
    dfree(c->d_Pf);
    dfree(c->d_Pnb);
    dfree(c->d_vval);
    dfree(c->d_minv);
    dfree(c->d_fF2);
    dfree(c->d_Pf2);
    dfree(c->d_Pnb2);
    dfree(c->d_vval2);
    for (auto& s : c->sources) dfree(s.d_coef);
    c->sources.clear();
    for (auto& p : c->d_cl_elems) dfree(p);
    c->d_cl_elems.clear();
    dfree(c->d_cl);
    dfree(c->d_slot);
    dfree(c->d_buf);
    dfree(c->d_tick);
    dfree(c->d_rp);
    dfree(c->d_seis);
    dfree(c->d_cnt);
    c->seis_cap = 0;
    c->rp_n = 0;
    c->ready = false;
}

void free_population(poro_ctx* c) {
    free_lu(c);
    free_mesh_device(c);
    dfree(c->d_evar);
    dfree(c->d_iters);
    c->subcell = false;
    dfree(c->d_econst);
    dfree(c->d_q0);
    dfree(c->d_qt);
    dfree(c->d_iout);
    c->n_elem = 0;
    c->have_dofs = c->have_pred = false;
}

void free_lu(poro_ctx* c) {
    dfree(c->lu.A);
    dfree(c->lu.piv);
    dfree(c->lu.perm);
    dfree(c->lu.R);
    dfree(c->lu.C);
    dfree(c->lu.bad);
    dfree(c->lu.x);
    if (c->lu.exec) cudaGraphExecDestroy(c->lu.exec);
    c->lu.exec = nullptr;
    c->lu_first = c->lu_count = 0;
}

void free_reference(poro_ctx* c) {
    dfree(c->lref.z);
    dfree(c->lref.krow);
    dfree(c->lref.kcol);
    dfree(c->lref.kval);

    dfree(c->mref.res_inv);
    dfree(c->mref.res_order8);
    dfree(c->mref.res_order4);
    dfree(c->mref.res_order2);
    dfree(c->mref.khat_tc);
    dfree(c->mref.status);
    dfree(c->mref.zinv_f32);
    dfree(c->sub.m3_row);
    dfree(c->sub.m3_col);
    dfree(c->sub.m3_val);
    dfree(c->dref.khat_val);
    dfree(c->dref.khat_col);
    dfree(c->dref.khat_row);
    for (int w = 0; w < 3; ++w) dfree(c->dref.lists[w]);
    dfree(c->dref.zinv);
}

}  // namespace

namespace poro {
bool ctx_view(const poro_ctx* c, CtxView& v) {
    if (!c || !c->d_econst || c->system != PORO_SYSTEM_BIOT || c->subcell) return false;
    v.device = c->device;
    v.N = c->N;
    v.n_elem = c->n_elem;
    v.stride = c->stride;
    v.econst = c->d_econst;
    v.lref = &c->lref;
    v.stream = c->stream;
    return true;
}
void ctx_set_error(poro_ctx* c, const std::string& msg) {
    if (c) c->err = msg; else g_err = msg;
}
}  // namespace poro

extern "C" {

const char* poro_last_error(const poro_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

// Rows dealt to `warps` lists, longest first, each to the least loaded list
// (ties to the lower index); rows of zero cost are left out when `drop_free`.
// Layout: [warps + 1] list starts, then the lists one after another.
static std::vector<int32_t> deal_rows(const std::vector<int64_t>& cost, int warps, bool drop_free) {
    std::vector<int> order;
    for (int l = 0; l < (int)cost.size(); ++l)
        if (!drop_free || cost[l] > 0) order.push_back(l);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int32_t>> lists(warps);
    std::vector<int64_t> load(warps, 0);
    for (int l : order) {
        int best = 0;
        for (int k = 1; k < warps; ++k)
            if (load[k] < load[best]) best = k;
        load[best] += cost[l];
        lists[best].push_back(l);
    }
    std::vector<int32_t> out(warps + 1, 0);
    for (int k = 0; k < warps; ++k) out[k + 1] = out[k] + (int32_t)lists[k].size();
    for (int k = 0; k < warps; ++k) out.insert(out.end(), lists[k].begin(), lists[k].end());
    return out;
}

// x = num / den with den <= 10^6 (continued-fraction convergents), if x is
// such a rational to 1e-14 relative
static bool rational_of(double x, int64_t& num, int64_t& den) {
    const double ax = std::fabs(x);
    int64_t h0 = 0, h1 = 1, k0 = 1, k1 = 0;
    double r = ax;
    for (int it = 0; it < 64; ++it) {
        const double a = std::floor(r);
        if (a > 9.0e15) break;
        const int64_t ai = (int64_t)a;
        const int64_t h2 = ai * h1 + h0, k2 = ai * k1 + k0;
        if (k2 > 1000000) break;
        h0 = h1;
        h1 = h2;
        k0 = k1;
        k1 = k2;
        if (std::fabs((double)h1 / (double)k1 - ax) <= 1e-14 * ax) {
            num = x < 0 ? -h1 : h1;
            den = k1;
            return true;
        }
        const double f = r - a;
        if (f <= 0.0) break;
        r = 1.0 / f;
    }
    return false;
}

poro_status poro_create(int device, int degree_N, poro_precision precision, poro_ctx** out) {
    return poro_create_system(device, degree_N, precision, PORO_SYSTEM_BIOT, out);
}

poro_status poro_create_system(int device, int degree_N, poro_precision precision, poro_system system,
                               poro_ctx** out) {
    if (!out) return fail(nullptr, PORO_EINVAL, "poro_create: out is NULL");
    *out = nullptr;
    if (system != PORO_SYSTEM_BIOT && system != PORO_SYSTEM_MAXWELL && system != PORO_SYSTEM_VISCOELASTIC)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_create: unknown system");
    if (system != PORO_SYSTEM_BIOT && precision != PORO_FP64)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_create: systems other than Biot's are built in FP64 only");
    if (degree_N < 1 || degree_N > poro::MAX_N)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_create: degree N must be in 1..6");
    if (precision != PORO_FP64 && precision != PORO_FP32_REFINE && precision != PORO_BF16X3_REFINE)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_create: unknown precision");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "poro_create: cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(nullptr, PORO_EINVAL, "poro_create: no such device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "poro_create: cudaSetDevice");
    poro_ctx* c = new poro_ctx();
    c->device = device;
    c->N = degree_N;
    c->prec = precision;
    c->system = system;
    c->nq = system == PORO_SYSTEM_MAXWELL ? poro::maxwell::NQ : system == PORO_SYSTEM_VISCOELASTIC ? poro::visco::NQ : NQ;
    c->refine = 1;  // one sweep reaches the 1e-10 goal in both mixed forms (measured)
    std::string err;
    if (!poro::reference_data(degree_N, c->ref, err)) {
        delete c;
        return fail(nullptr, PORO_EINVAL, "poro_create: " + err);
    }
    c->B = c->ref.B;
    c->T = c->ref.T;
    c->stride = system == PORO_SYSTEM_MAXWELL        ? poro::maxwell::elem_const_stride(degree_N)
                : system == PORO_SYSTEM_VISCOELASTIC ? poro::visco::elem_const_stride(degree_N)
                                                     : poro::elem_const_stride(degree_N);
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(nullptr, e, "poro_create: cudaStreamCreate");
    }
    // concatenate the (g, j) CSR blocks of Khat
    std::vector<double> val;
    std::vector<int32_t> col, row;
    c->dref.N = degree_N;
    for (int g = 1; g <= degree_N; ++g)
        for (int j = 0; j < 3; ++j) {
            const poro::KhatBlockCSR& C = c->ref.blocks[g * 3 + j];
            c->dref.row_base[g][j] = (int32_t)row.size();
            const int32_t base = (int32_t)val.size();
            for (int32_t r : C.row_ptr) row.push_back(base + r);
            val.insert(val.end(), C.val.begin(), C.val.end());
            col.insert(col.end(), C.col.begin(), C.col.end());
        }
    // per block (g, j): its rows l < o_g dealt to 2, 4 and 8 warps by Khat
    // entries (rows without entries in the block are left out)
    std::vector<int32_t> blists[3];
    for (int w = 0; w < 3; ++w)
        for (int g = 1; g <= degree_N; ++g)
            for (int j = 0; j < 3; ++j) {
                const poro::KhatBlockCSR& C = c->ref.blocks[g * 3 + j];
                std::vector<int64_t> cost(C.row_ptr.size() - 1);
                for (size_t l = 0; l + 1 < C.row_ptr.size(); ++l) cost[l] = C.row_ptr[l + 1] - C.row_ptr[l];
                c->dref.list_base[w][g][j] = (int32_t)blists[w].size();
                const std::vector<int32_t> d = deal_rows(cost, 2 << w, true);
                blists[w].insert(blists[w].end(), d.begin(), d.end());
            }
    if ((e = upload((void**)&c->dref.lists[0], blists[0].data(), blists[0].size() * sizeof(int32_t))) != cudaSuccess ||
        (e = upload((void**)&c->dref.lists[1], blists[1].data(), blists[1].size() * sizeof(int32_t))) != cudaSuccess ||
        (e = upload((void**)&c->dref.lists[2], blists[2].data(), blists[2].size() * sizeof(int32_t))) != cudaSuccess ||
        (e = upload((void**)&c->dref.khat_val, val.data(), val.size() * sizeof(double))) != cudaSuccess ||
        (e = upload((void**)&c->dref.khat_col, col.data(), col.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = upload((void**)&c->dref.khat_row, row.data(), row.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = upload((void**)&c->dref.zinv, c->ref.zinv.data(), c->ref.zinv.size() * sizeof(double))) !=
            cudaSuccess) {
        free_reference(c);
        cudaStreamDestroy(c->stream);
        delete c;
        return e == cudaErrorMemoryAllocation ? fail(nullptr, PORO_ENOMEM, "poro_create: out of device memory")
                                              : cuda_fail(nullptr, e, "poro_create: upload");
    }
    {
        // full-row CSR of Khat^j in binary64 and Z for the dense-LU comparator
        const int B = c->B;
        std::vector<int32_t> lrow, lcol;
        std::vector<double> lval;
        for (int j = 0; j < 3; ++j) {
            lrow.push_back((int32_t)lcol.size());
            for (int l = 0; l < B; ++l) {
                for (int m = 0; m < B; ++m) {
                    const double v = c->ref.khat[((size_t)j * B + l) * B + m];
                    if (v != 0.0) {
                        lcol.push_back(m);
                        lval.push_back(v);
                    }
                }
                lrow.push_back((int32_t)lcol.size());
            }
        }
        c->lref.N = degree_N;
        if ((e = upload((void**)&c->lref.z, c->ref.z.data(), c->ref.z.size() * sizeof(double))) != cudaSuccess ||
            (e = upload((void**)&c->lref.krow, lrow.data(), lrow.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->lref.kcol, lcol.data(), lcol.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->lref.kval, lval.data(), lval.size() * sizeof(double))) != cudaSuccess) {
            free_reference(c);
            cudaStreamDestroy(c->stream);
            delete c;
            return cuda_fail(nullptr, e, "poro_create: upload (LU)");
        }
    }
    if (precision != PORO_FP64) {
        // Residual CSR of Khat^j (all rows): every row l of every Khat^j is an
        // integer row over a common denominator d (the reference matrices are
        // rational with small denominators), so an entry is packed as
        // (numerator << 7) | column and the row carries 1/d as a
        // double-binary32 pair.  The kernel multiplies the numerators with
        // 21-bit fixed-point values and sums in 64-bit integers, exact while a
        // row's sum of |numerators| stays below 2^22 (3.6e6 at N = 6).
        const int B = c->B;
        std::vector<float> zf(c->ref.zinv.begin(), c->ref.zinv.end());
        std::vector<int32_t> rrow, rint;
        std::vector<float> rinv;
        std::string rerr;
        for (int j = 0; j < 3 && rerr.empty(); ++j) {
            rrow.push_back((int32_t)rint.size());
            for (int l = 0; l < B && rerr.empty(); ++l) {
                const double* row = c->ref.khat.data() + ((size_t)j * B + l) * B;
                int64_t d = 1;
                for (int m = 0; m < B; ++m) {
                    int64_t num = 0, den = 1;
                    if (row[m] == 0.0) continue;
                    if (!rational_of(row[m], num, den)) {
                        rerr = "Khat entry is not a small-denominator rational";
                        break;
                    }
                    d = d / std::gcd(d, den) * den;
                    if (d > (1 << 30)) {
                        rerr = "Khat row denominator too large";
                        break;
                    }
                }
                int64_t abs_sum = 0;  // the residual's 64-bit integer sums need sum |c| < 2^22
                for (int m = 0; m < B && rerr.empty(); ++m) {
                    if (row[m] == 0.0) continue;
                    const double cv = row[m] * (double)d;
                    const int64_t ci = std::llround(cv);
                    abs_sum += std::llabs(ci);
                    if (std::fabs(cv - (double)ci) > 1e-6 || std::llabs(ci) >= (1 << 23) || abs_sum >= (1 << 22)) {
                        rerr = "Khat numerator out of range";
                        break;
                    }
                    rint.push_back((int32_t)(((uint32_t)(int32_t)ci << 7) | (uint32_t)m));
                }
                const double inv = 1.0 / (double)d;
                const float ih = (float)inv;
                rinv.push_back(ih);
                rinv.push_back((float)(inv - (double)ih));
                rrow.push_back((int32_t)rint.size());
            }
        }
        // residual row order per warp count: a row costs its Khat entries (all
        // directions) plus a fixed share for the star and time terms
        auto deal = [&](int warps) {
            std::vector<int64_t> cost(B);
            for (int l = 0; l < B; ++l) {
                cost[l] = 40;
                for (int j = 0; j < 3; ++j) cost[l] += rrow[j * (B + 1) + l + 1] - rrow[j * (B + 1) + l];
            }
            return deal_rows(cost, warps, false);
        };
        const std::vector<int32_t> ord8 = deal(8), ord4 = deal(4), ord2 = deal(2);
        if (!rerr.empty()) {
            free_reference(c);
            cudaStreamDestroy(c->stream);
            delete c;
            return fail(nullptr, PORO_ENUMERIC, "poro_create: " + rerr);
        }
        // tensor-core images of the blocks, hi image then lo image in the
        // K-major core-matrix layout: tf32 words, or bf16 for the bf16 form
        const bool bf16 = precision == PORO_BF16X3_REFINE;
        c->mref.bf16 = bf16;
        auto tf32 = [](float x) {
            uint32_t b;
            std::memcpy(&b, &x, 4);
            b = (b + 0x1000u) & 0xFFFFE000u;  // nearest, ties away from zero
            std::memcpy(&x, &b, 4);
            return x;
        };
        std::vector<uint8_t> tci;  // bytes
        for (int g = 1; g <= degree_N; ++g) {
            const int NP = poro::tc_np(g), KP = poro::tc_kp(g, bf16), o = poro::block_offset(g),
                      d = poro::block_size(g);
            const size_t es = bf16 ? 2 : 4, img = (size_t)NP * KP * es;
            for (int j = 0; j < 3; ++j) {
                const size_t base = tci.size();
                c->mref.tc_off[g][j] = (int32_t)base;
                tci.resize(base + 2 * img, 0);
                for (int l = 0; l < o; ++l)
                    for (int m = 0; m < d; ++m) {
                        const double v = c->ref.khat[((size_t)j * B + l) * B + o + m];
                        if (bf16) {
                            const uint16_t h = poro::tc::bf16_bits((float)v);
                            const uint16_t lo = poro::tc::bf16_bits((float)(v - (double)poro::tc::bf16_value(h)));
                            const size_t at = base + 2 * (size_t)poro::tc::kmajor_offset16(l, m, KP);
                            std::memcpy(&tci[at], &h, 2);
                            std::memcpy(&tci[at + img], &lo, 2);
                        } else {
                            const float h = tf32((float)v), lo = tf32((float)(v - (double)h));
                            const size_t at = base + 4 * (size_t)poro::tc::kmajor_offset(l, m, KP);
                            std::memcpy(&tci[at], &h, 4);
                            std::memcpy(&tci[at + img], &lo, 4);
                        }
                    }
            }
        }
        c->mref.base = &c->dref;
        if ((e = (cudaError_t)poro::upload_residual_table(degree_N, rrow.data(), rint.data(), (int)rint.size())) !=
                cudaSuccess ||

            (e = upload((void**)&c->mref.res_inv, rinv.data(), rinv.size() * sizeof(float))) != cudaSuccess ||
            (e = upload((void**)&c->mref.res_order8, ord8.data(), ord8.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->mref.res_order4, ord4.data(), ord4.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->mref.res_order2, ord2.data(), ord2.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->mref.zinv_f32, zf.data(), zf.size() * sizeof(float))) != cudaSuccess ||
            (e = upload((void**)&c->mref.khat_tc, tci.data(), tci.size())) != cudaSuccess ||
            (e = cudaMalloc((void**)&c->mref.status, sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMemset(c->mref.status, 0, sizeof(int32_t))) != cudaSuccess) {
            free_reference(c);
            cudaStreamDestroy(c->stream);
            delete c;
            return cuda_fail(nullptr, e, "poro_create: upload (mixed)");
        }
    }
    *out = c;
    return PORO_OK;
}

poro_status poro_set_refinement(poro_ctx* c, int32_t sweeps) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_refinement: ctx is NULL");
    if (c->prec == PORO_FP64) return fail(c, PORO_EUNSUPPORTED, "poro_set_refinement: context is not mixed precision");
    if (sweeps < 0 || sweeps > 2) return fail(c, PORO_EINVAL, "poro_set_refinement: sweeps must be 0, 1 or 2");
    c->refine = sweeps;
    return PORO_OK;
}

poro_status poro_set_wait_limit(poro_ctx* c, int64_t cycles) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_wait_limit: ctx is NULL");
    if (c->prec == PORO_FP64) return fail(c, PORO_EUNSUPPORTED, "poro_set_wait_limit: context is not mixed precision");
    if (cycles < 0) return fail(c, PORO_EINVAL, "poro_set_wait_limit: cycles must be >= 0");
    c->mref.wait_limit = (long long)cycles;
    return PORO_OK;
}

poro_status poro_destroy(poro_ctx* c) {
    if (!c) return PORO_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_population(c);
    free_reference(c);
    for (cudaEvent_t ev : c->ev_in) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->ev_k) cudaEventDestroy(ev);
    if (c->s_in) cudaStreamDestroy(c->s_in);
    if (c->s_out) cudaStreamDestroy(c->s_out);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return PORO_OK;
}

poro_status poro_get_info(const poro_ctx* c, int32_t* degree_N, int32_t* precision, int64_t* n_elem) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_get_info: ctx is NULL");
    if (degree_N) *degree_N = c->N;
    if (precision) *precision = (int32_t)c->prec;
    if (n_elem) *n_elem = c->n_elem;
    return PORO_OK;
}

poro_status poro_reference_matrices(int degree_N, double* mass_diag, double* khat) {
    poro::ReferenceData R;
    std::string err;
    if (!poro::reference_data(degree_N, R, err)) return fail(nullptr, PORO_EUNSUPPORTED, err);
    if (mass_diag) std::memcpy(mass_diag, R.mass_diag.data(), sizeof(double) * R.B);
    if (khat) std::memcpy(khat, R.khat.data(), sizeof(double) * 3 * R.B * R.B);
    return PORO_OK;
}

poro_status poro_material_jacobians(const poro_material* mat, double* abc, double* e) {
    if (!mat) return fail(nullptr, PORO_EINVAL, "poro_material_jacobians: mat is NULL");
    double A[3][NQ][NQ], E[NQ][NQ];
    std::string err;
    if (!poro::material_jacobians(*mat, A, E, err)) return fail(nullptr, PORO_EINVAL, err);
    if (abc) std::memcpy(abc, A, sizeof(A));
    if (e) std::memcpy(e, E, sizeof(E));
    return PORO_OK;
}

poro_status poro_max_wave_speed(const poro_material* mat, double* speed) {
    if (!mat || !speed) return fail(nullptr, PORO_EINVAL, "poro_max_wave_speed: NULL argument");
    std::string err;
    if (!poro::max_wave_speed(*mat, *speed, err)) return fail(nullptr, PORO_EINVAL, err);
    return PORO_OK;
}

poro_status poro_cfl_dt(int degree_N, int64_t n, const double* vert, const poro_material* mat, double cfl_c,
                        double* dt) {
    if (degree_N < 1 || degree_N > poro::MAX_N) return fail(nullptr, PORO_EUNSUPPORTED, "poro_cfl_dt: degree");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt)) || !(cfl_c > 0.0))
        return fail(nullptr, PORO_EINVAL, "poro_cfl_dt: bad argument");
    for (int64_t i = 0; i < n; ++i) {
        double jinv[3][3], vol, dins, v;
        std::string err;
        if (!poro::tet_geometry(vert + 12 * i, jinv, vol, dins, err) || !poro::max_wave_speed(mat[i], v, err))
            return fail(nullptr, PORO_EINVAL, "poro_cfl_dt: element " + std::to_string(i) + ": " + err);
        dt[i] = cfl_c / (2 * degree_N + 1) * dins / v;
    }
    return PORO_OK;
}

poro_status poro_cfl_dt_system(poro_system system, int degree_N, int64_t n, const double* vert, const double* mat,
                               double cfl_c, double* dt) {
    if (system == PORO_SYSTEM_BIOT)
        return poro_cfl_dt(degree_N, n, vert, reinterpret_cast<const poro_material*>(mat), cfl_c, dt);
    if (system != PORO_SYSTEM_MAXWELL && system != PORO_SYSTEM_VISCOELASTIC)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_cfl_dt_system: unknown system");
    if (degree_N < 1 || degree_N > poro::MAX_N) return fail(nullptr, PORO_EUNSUPPORTED, "poro_cfl_dt_system: degree");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt)) || !(cfl_c > 0.0))
        return fail(nullptr, PORO_EINVAL, "poro_cfl_dt_system: bad argument");
    const int nm = system == PORO_SYSTEM_MAXWELL ? 3 : 12;
    for (int64_t i = 0; i < n; ++i) {
        double jinv[3][3], vol, dins;
        std::string err;
        const double* m = mat + nm * i;
        // fastest characteristic speed: 1 / sqrt(eps mu), or the unrelaxed P speed
        const double v = system == PORO_SYSTEM_MAXWELL ? 1.0 / std::sqrt(m[0] * m[1])
                                                       : std::sqrt((m[1] + 2.0 * m[2]) / m[0]);
        if (!poro::tet_geometry(vert + 12 * i, jinv, vol, dins, err))
            return fail(nullptr, PORO_EINVAL, "poro_cfl_dt_system: element " + std::to_string(i) + ": " + err);
        if (!(v > 0.0) || !std::isfinite(v))
            return fail(nullptr, PORO_EINVAL, "poro_cfl_dt_system: element " + std::to_string(i) + ": material");
        dt[i] = cfl_c / (2 * degree_N + 1) * dins / v;
    }
    return PORO_OK;
}

static poro_status upload_population(poro_ctx* c, int64_t n, const std::vector<double>& ec) {
    const size_t nd = (size_t)n * c->nq * c->B;
    cudaError_t e;
    if ((e = upload((void**)&c->d_econst, ec.data(), ec.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->d_q0, nd * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->d_qt, nd * c->T * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->d_iout, nd * sizeof(double) + 16)) != cudaSuccess) {
        free_population(c);
        return e == cudaErrorMemoryAllocation ? fail(c, PORO_ENOMEM, "population: out of device memory")
                                              : cuda_fail(c, e, "population");
    }
    c->n_elem = n;
    return PORO_OK;
}

poro_status poro_set_isolated(poro_ctx* c, int64_t n, const double* vert, const poro_material* mat,
                              const double* dt) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_isolated: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT)
        return fail(c, PORO_EUNSUPPORTED, "poro_set_isolated: Biot materials on a context of another system");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt))) return fail(c, PORO_EINVAL, "poro_set_isolated: bad argument");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    c->mesh_mode = false;
    std::vector<double> ec((size_t)n * c->stride);
    for (int64_t i = 0; i < n; ++i) {
        std::string err;
        if (!poro::element_constants(c->ref, vert + 12 * i, mat[i], dt[i], ec.data() + (size_t)i * c->stride, err))
            return fail(c, PORO_EINVAL, "poro_set_isolated: element " + std::to_string(i) + ": " + err);
    }
    return upload_population(c, n, ec);
}

poro_status poro_set_isolated_maxwell(poro_ctx* c, int64_t n, const double* vert, const double* mat,
                                      const double* dt) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_isolated_maxwell: ctx is NULL");
    if (c->system != PORO_SYSTEM_MAXWELL)
        return fail(c, PORO_EUNSUPPORTED, "poro_set_isolated_maxwell: context is not a damped Maxwell context");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt)))
        return fail(c, PORO_EINVAL, "poro_set_isolated_maxwell: bad argument");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    c->mesh_mode = false;
    std::vector<double> ec((size_t)n * c->stride);
    for (int64_t i = 0; i < n; ++i) {
        std::string err;
        if (!poro::maxwell_element_constants(c->ref, vert + 12 * i, mat + 3 * i, dt[i], ec.data() + (size_t)i * c->stride,
                                             err))
            return fail(c, PORO_EINVAL, "poro_set_isolated_maxwell: element " + std::to_string(i) + ": " + err);
    }
    return upload_population(c, n, ec);
}

poro_status poro_set_isolated_viscoelastic(poro_ctx* c, int64_t n, const double* vert, const double* mat,
                                           const double* dt) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_isolated_viscoelastic: ctx is NULL");
    if (c->system != PORO_SYSTEM_VISCOELASTIC)
        return fail(c, PORO_EUNSUPPORTED, "poro_set_isolated_viscoelastic: context is not a viscoelastic context");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt)))
        return fail(c, PORO_EINVAL, "poro_set_isolated_viscoelastic: bad argument");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    c->mesh_mode = false;
    std::vector<double> ec((size_t)n * c->stride);
    for (int64_t i = 0; i < n; ++i) {
        std::string err;
        if (!poro::visco_element_constants(c->ref, vert + 12 * i, mat + 12 * i, dt[i], ec.data() + (size_t)i * c->stride,
                                           err))
            return fail(c, PORO_EINVAL, "poro_set_isolated_viscoelastic: element " + std::to_string(i) + ": " + err);
    }
    return upload_population(c, n, ec);
}

poro_status poro_set_isolated_subcell(poro_ctx* c, int64_t n, const double* vert, const poro_material* mat,
                                      const double* dt) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_isolated_subcell: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT || c->prec != PORO_FP64)
        return fail(c, PORO_EUNSUPPORTED, "poro_set_isolated_subcell: built for Biot's system in FP64");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt)))
        return fail(c, PORO_EINVAL, "poro_set_isolated_subcell: bad argument");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    c->mesh_mode = false;
    std::string err;
    if (!c->sub.m3_row) {
        std::vector<int32_t> row, col;
        std::vector<double> val;
        if (!poro::subcell_mass_tensors(c->ref, row, col, val, err))
            return fail(c, PORO_EINVAL, "poro_set_isolated_subcell: " + err);
        cudaError_t e = upload((void**)&c->sub.m3_row, row.data(), row.size() * sizeof(int32_t));
        if (e == cudaSuccess) e = upload((void**)&c->sub.m3_col, col.data(), col.size() * sizeof(int32_t));
        if (e == cudaSuccess) e = upload((void**)&c->sub.m3_val, val.data(), val.size() * sizeof(double));
        if (e != cudaSuccess) {
            dfree(c->sub.m3_row);
            dfree(c->sub.m3_col);
            dfree(c->sub.m3_val);
            return cuda_fail(c, e, "poro_set_isolated_subcell: tensors");
        }
    }
    double P[4][4];
    if (!poro::subcell_projection(P, err)) return fail(c, PORO_EINVAL, "poro_set_isolated_subcell: " + err);
    const int vs = poro::subcell_var_stride();
    std::vector<double> ec((size_t)n * c->stride), ev((size_t)n * vs);
    for (int64_t i = 0; i < n; ++i)
        if (!poro::subcell_element_constants(c->ref, P, vert + 12 * i, mat + 4 * i, dt[i], ec.data() + (size_t)i * c->stride,
                                             ev.data() + (size_t)i * vs, err))
            return fail(c, PORO_EINVAL, "poro_set_isolated_subcell: element " + std::to_string(i) + ": " + err);
    poro_status st = upload_population(c, n, ec);
    if (st != PORO_OK) return st;
    cudaError_t e = upload((void**)&c->d_evar, ev.data(), ev.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_iters, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_iters, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        free_population(c);
        return cuda_fail(c, e, "poro_set_isolated_subcell");
    }
    c->subcell = true;
    return PORO_OK;
}

poro_status poro_set_subcell_tolerance(poro_ctx* c, double tol, int32_t max_iter) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_subcell_tolerance: ctx is NULL");
    if (!(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1 || max_iter > 100000)
        return fail(c, PORO_EINVAL, "poro_set_subcell_tolerance: need tol >= 0 and 1 <= max_iter <= 100000");
    c->sub_tol = tol;
    c->sub_max_iter = max_iter;
    return PORO_OK;
}

poro_status poro_get_subcell_iterations(poro_ctx* c, int64_t first, int64_t count, int32_t* out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_get_subcell_iterations: ctx is NULL");
    if (!c->subcell) return fail(c, PORO_ESTATE, "poro_get_subcell_iterations: no sub-cell population loaded");
    if (first < 0 || count < 0 || first + count > c->n_elem || (count > 0 && !out))
        return fail(c, PORO_EINVAL, "poro_get_subcell_iterations: bad range");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(out, c->d_iters + first, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "poro_get_subcell_iterations");
    return PORO_OK;
}

poro_status poro_get_system(const poro_ctx* c, int32_t* system, int32_t* n_quantities) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_get_system: ctx is NULL");
    if (system) *system = c->system;
    if (n_quantities) *n_quantities = c->nq;
    return PORO_OK;
}

poro_status poro_set_dofs(poro_ctx* c, const double* Q) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_dofs: ctx is NULL");
    if (!c->d_econst) return fail(c, PORO_ESTATE, "poro_set_dofs: no element population loaded");
    if (c->n_elem > 0 && !Q) return fail(c, PORO_EINVAL, "poro_set_dofs: Q is NULL");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(c->d_q0, Q, (size_t)c->n_elem * c->nq * c->B * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "poro_set_dofs");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "poro_set_dofs");
    c->have_dofs = true;
    return PORO_OK;
}

static poro_status dispatch_predict(poro_ctx* c, int64_t first, int64_t count, const double* q0, double* qt,
                                    double* iout, poro_solver solver, cudaStream_t st) {
    const double* ec = c->d_econst + first * c->stride;
    int rc = 0;
    if (solver == PORO_SOLVE_LU) {
        if (c->system != PORO_SYSTEM_BIOT || c->subcell)
            return fail(c, PORO_EUNSUPPORTED,
                        "predict (LU): the dense-LU comparator is built for Biot's system with constant material");
        if (count > 0 && (first < c->lu_first || first + count > c->lu_first + c->lu_count))
            return fail(c, PORO_ESTATE, "predict (LU): elements not factored; call poro_lu_factor first");
        rc = poro::launch_lu_solve(c->lref, count, c->lu, first - c->lu_first, q0, ec, qt, iout, st);
        if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "predict (LU): kernel launch");
        return PORO_OK;
    }
    if (solver != PORO_SOLVE_BLOCK) return fail(c, PORO_EINVAL, "predict: unknown solver");
    if (c->subcell) {
        rc = poro::launch_stp_subcell(c->dref, c->sub, count, q0, ec, c->d_evar + first * poro::subcell_var_stride(),
                                      qt, iout, c->d_iters + first, c->sub_tol, c->sub_max_iter, st);
    } else if (c->system == PORO_SYSTEM_MAXWELL) {
        rc = poro::launch_stp_fp64_maxwell(c->dref, nullptr, count, q0, ec, qt, iout, st);
    } else if (c->system == PORO_SYSTEM_VISCOELASTIC) {
        rc = poro::launch_stp_fp64_visco(c->dref, nullptr, count, q0, ec, qt, iout, st);
    } else if (c->prec == PORO_FP64) {
        rc = poro::launch_stp_fp64(c->dref, nullptr, count, q0, ec, qt, iout, st, c->variant);
    } else {
        rc = poro::launch_stp_mixed(c->mref, c->refine, nullptr, count, q0, ec, qt, iout, st, c->variant);
    }
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "predict: kernel launch");
    return PORO_OK;
}

poro_status poro_predict(poro_ctx* c, int32_t cluster, poro_solver solver) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_predict: ctx is NULL");
    if (cluster != -1) return fail(c, PORO_EINVAL, "poro_predict: isolated population has no clusters");
    if (!c->have_dofs) return fail(c, PORO_ESTATE, "poro_predict: DOFs not set");
    cudaSetDevice(c->device);
    poro_status s = dispatch_predict(c, 0, c->n_elem, c->d_q0, c->d_qt, c->d_iout, solver, c->stream);
    if (s == PORO_OK) c->have_pred = true;
    return s;
}

poro_status poro_predict_dev(poro_ctx* c, int64_t first, int64_t count, const double* q0, double* qt, double* iout,
                             poro_solver solver, void* stream) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_predict_dev: ctx is NULL");
    if (!c->d_econst) return fail(c, PORO_ESTATE, "poro_predict_dev: no element population loaded");
    if (first < 0 || count < 0 || first + count > c->n_elem)
        return fail(c, PORO_EINVAL, "poro_predict_dev: element range outside the population");
    if (count > 0 && !q0) return fail(c, PORO_EINVAL, "poro_predict_dev: Q0 is NULL");
    if (((uintptr_t)q0 | (uintptr_t)qt | (uintptr_t)iout) & 15)
        return fail(c, PORO_EINVAL, "poro_predict_dev: buffers must be 16-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    return dispatch_predict(c, first, count, q0, qt, iout, solver, st);
}

static poro_status device_status(poro_ctx* c, const char* who);

poro_status poro_predict_host(poro_ctx* c, const double* q0_host, double* I_out, int64_t chunk_elems,
                              poro_solver solver) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_predict_host: ctx is NULL");
    if (!c->d_econst) return fail(c, PORO_ESTATE, "poro_predict_host: no element population loaded");
    if (c->n_elem > 0 && (!q0_host || !I_out)) return fail(c, PORO_EINVAL, "poro_predict_host: NULL buffer");
    if (chunk_elems < 0) return fail(c, PORO_EINVAL, "poro_predict_host: negative chunk size");
    const int64_t n = c->n_elem;
    if (n == 0) return PORO_OK;
    cudaSetDevice(c->device);
    cudaError_t e = cudaSuccess;
    if (!c->s_in && (e = cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(c, e, "poro_predict_host");
    if (!c->s_out && (e = cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(c, e, "poro_predict_host");
    // chunk boundaries.  Only the first chunk's upload and the last chunk's
    // download are not hidden under kernels, so the automatic schedule takes
    // about 16 chunks of at least 4096 elements (measured on GB300 at N = 6,
    // 200k elements: 16 chunks leave 6.8 ms of the 3.5 GB of copies exposed, 8
    // chunks 10 ms, 4 chunks 17 ms) and ramps the first three up from 1/8 and
    // the last three down to 1/8 of that size (measured against 16 equal
    // chunks: the same within the run-to-run spread of about 1.5 ms).
    // chunk_elems > 0: equal chunks.
    std::vector<int64_t> bounds{0};
    {
        const int64_t chunk = chunk_elems > 0 ? std::min(chunk_elems, n)
                                              : std::min(n, std::max<int64_t>(4096, ((n + 15) / 16 + 255) / 256 * 256));
        int64_t ramp[3] = {chunk / 8, chunk / 4, chunk / 2}, ramp_sum = 0;
        for (int64_t& r : ramp) ramp_sum += (r = std::max<int64_t>(256, r / 256 * 256));
        const bool ramped = chunk_elems <= 0 && n - 2 * ramp_sum >= 2 * chunk;
        if (ramped)
            for (int64_t r : ramp) bounds.push_back(bounds.back() + r);
        const int64_t mid_end = ramped ? n - ramp_sum : n;
        const int64_t mid = mid_end - bounds.back();
        const int64_t k = std::max<int64_t>(1, (mid + chunk - 1) / chunk);
        const int64_t start = bounds.back();
        for (int64_t i = 1; i <= k; ++i) bounds.push_back(start + (chunk_elems > 0 ? std::min(mid, i * chunk) : mid * i / k));
        if (ramped)
            for (int i = 2; i >= 0; --i) bounds.push_back(bounds.back() + ramp[i]);
    }
    const int64_t nchunks = (int64_t)bounds.size() - 1;
    if (nchunks > 4096) return fail(c, PORO_EINVAL, "poro_predict_host: more than 4096 chunks");
    while ((int64_t)c->ev_in.size() < nchunks) {
        cudaEvent_t a = nullptr, b = nullptr;
        if ((e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "poro_predict_host");
        c->ev_in.push_back(a);
        c->ev_k.push_back(b);
    }
    // nothing queued earlier on the context stream may still use the buffers
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "poro_predict_host");
    const size_t per = (size_t)c->nq * c->B;
    for (int64_t i = 0; i < nchunks; ++i) {
        const int64_t first = bounds[i], cnt = bounds[i + 1] - bounds[i];
        if ((e = cudaMemcpyAsync(c->d_q0 + first * per, q0_host + first * per, cnt * per * sizeof(double),
                                 cudaMemcpyHostToDevice, c->s_in)) != cudaSuccess ||
            (e = cudaEventRecord(c->ev_in[i], c->s_in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(c->stream, c->ev_in[i], 0)) != cudaSuccess)
            return cuda_fail(c, e, "poro_predict_host: copy in");
        poro_status st = dispatch_predict(c, first, cnt, c->d_q0 + first * per, c->d_qt + first * per * c->T,
                                          c->d_iout + first * per, solver, c->stream);
        if (st != PORO_OK) {
            cudaStreamSynchronize(c->s_in);
            cudaStreamSynchronize(c->stream);
            return st;
        }
        if ((e = cudaEventRecord(c->ev_k[i], c->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(c->s_out, c->ev_k[i], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(I_out + first * per, c->d_iout + first * per, cnt * per * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->s_out)) != cudaSuccess)
            return cuda_fail(c, e, "poro_predict_host: copy out");
    }
    if ((e = cudaStreamSynchronize(c->s_out)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess || (e = cudaStreamSynchronize(c->s_in)) != cudaSuccess)
        return cuda_fail(c, e, "poro_predict_host");
    c->have_dofs = true;
    c->have_pred = true;
    return device_status(c, "poro_predict_host");
}

poro_status poro_lu_bytes(int degree_N, int64_t count, size_t* bytes) {
    if (degree_N < 1 || degree_N > poro::MAX_N) return fail(nullptr, PORO_EUNSUPPORTED, "poro_lu_bytes: degree");
    if (count < 0 || !bytes) return fail(nullptr, PORO_EINVAL, "poro_lu_bytes: bad argument");
    *bytes = poro::lu_scratch_bytes(degree_N, count);
    return PORO_OK;
}

poro_status poro_lu_factor(poro_ctx* c, int64_t first, int64_t count) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_lu_factor: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT || c->subcell)
        return fail(c, PORO_EUNSUPPORTED, "poro_lu_factor: the dense-LU comparator is built for Biot's system with constant material");
    if (!c->d_econst) return fail(c, PORO_ESTATE, "poro_lu_factor: no element population loaded");
    if (first < 0 || count < 0 || first + count > c->n_elem || count > 65535)
        return fail(c, PORO_EINVAL, "poro_lu_factor: element range outside the population (or > 65535)");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_lu(c);
    const size_t s = (size_t)NQ * c->B * c->T;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&c->lu.A, (size_t)count * s * s * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->lu.piv, (size_t)count * s * sizeof(int32_t) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->lu.perm, (size_t)count * s * sizeof(int32_t) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->lu.R, (size_t)count * s * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->lu.C, (size_t)count * s * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->lu.bad, sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->lu.x, (size_t)count * s * sizeof(double) + 16)) != cudaSuccess) {
        free_lu(c);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(c, PORO_ENOMEM, "poro_lu_factor: factors do not fit in HBM")
                                              : cuda_fail(c, e, "poro_lu_factor");
    }
    int rc = poro::launch_lu_factor(c->lref, count, c->d_econst + first * c->stride, c->lu, c->stream);
    if (rc != 0) {
        free_lu(c);
        return cuda_fail(c, (cudaError_t)rc, "poro_lu_factor: kernel launch");
    }
    int32_t bad = 0;
    e = cudaMemcpyAsync(&bad, c->lu.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_lu(c);
        return cuda_fail(c, e, "poro_lu_factor");
    }
    if (bad) {
        free_lu(c);
        return fail(c, PORO_ENUMERIC, "poro_lu_factor: zero pivot (singular predictor system)");
    }
    c->lu_first = first;
    c->lu_count = count;
    return PORO_OK;
}

poro_status poro_lu_release(poro_ctx* c) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_lu_release: ctx is NULL");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_lu(c);
    return PORO_OK;
}

// A kernel whose bounded wait gave up (tensor-core completion of the mixed
// predictor) leaves a flag in device memory; the next synchronising call
// reports it once.  Call only after the context's stream is idle.
static poro_status device_status(poro_ctx* c, const char* who) {
    if (!c->mref.status) return PORO_OK;
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->mref.status, sizeof st, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    if (st == 0) return PORO_OK;
    e = cudaMemsetAsync(c->mref.status, 0, sizeof st, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    return fail(c, PORO_ETIMEOUT, std::string(who) + ": a bounded tensor-core wait in the mixed predictor gave up");
}

poro_status poro_sync(poro_ctx* c, int32_t timeout_ms) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_sync: ctx is NULL");
    cudaSetDevice(c->device);
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return device_status(c, "poro_sync");
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "poro_sync");
        if (timeout_ms >= 0) {
            auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(c, PORO_ETIMEOUT, "poro_sync: timed out");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

static poro_status copy_out(poro_ctx* c, const double* src, int64_t first, int64_t count, size_t per, double* out,
                            const char* who) {
    if (!c) return fail(nullptr, PORO_EINVAL, std::string(who) + ": ctx is NULL");
    if (!c->have_pred) return fail(c, PORO_ESTATE, std::string(who) + ": no predictor computed");
    if (first < 0 || count < 0 || first + count > c->n_elem || (count > 0 && !out))
        return fail(c, PORO_EINVAL, std::string(who) + ": bad range or NULL output");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(out, src + first * per, count * per * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    return device_status(c, who);
}

poro_status poro_get_predictor(poro_ctx* c, int64_t first, int64_t count, double* out) {
    return copy_out(c, c ? c->d_qt : nullptr, first, count, c ? (size_t)c->nq * c->B * c->T : 0, out,
                    "poro_get_predictor");
}

poro_status poro_get_integrated(poro_ctx* c, int64_t first, int64_t count, double* out) {
    return copy_out(c, c ? c->d_iout : nullptr, first, count, c ? (size_t)c->nq * c->B : 0, out,
                    "poro_get_integrated");
}

poro_status poro_flop_count(const poro_ctx* c, int32_t refine_sweeps, double* f) {
    if (!c || !f) return fail(nullptr, PORO_EINVAL, "poro_flop_count: NULL argument");
    const double B = c->B, T = c->T, nq = c->nq;
    const bool mx = c->system == PORO_SYSTEM_MAXWELL, ve = c->system == PORO_SYSTEM_VISCOELASTIC;
    const double nnz = mx ? poro::maxwell::STAR_NNZ : ve ? poro::visco::STAR_NNZ : poro::STAR_NNZ;
    // couplings of E*'s strictly upper part per mode (Biot 3, viscoelastic 3 x 12)
    const double npair = mx ? 0 : ve ? 12 * poro::visco::NMECH : 3;
    // S3: nq B rows of T x T time solves + the couplings per mode
    const double s3 = 2.0 * nq * B * T * T + 2.0 * npair * B * T;
    // S4a: star products (Biot 54, Maxwell 12, viscoelastic 51 entries) of all modes of degree >= 1, 3 directions
    const double s4a = 2.0 * 3 * nnz * (B - 1) * T;
    // S4b: structural non-zeros of the Khat blocks, each applied to nq T columns
    const double s4b = 2.0 * (double)c->ref.khat_block_nnz * nq * T;
    // S1 (scaling of Q0) and S5 (time integration)
    const double s15 = nq * B * T + nq * B;
    const double alg3 = s3 + s4a + s4b + s15;
    f[0] = alg3;
    f[1] = alg3 * (1 + refine_sweeps);
    // residual per sweep: diagonal time blocks, E* diagonal and coupling,
    // star products of all modes and the Khat products, in double-binary32
    f[2] = (2.0 * NQ * B * T * T + 2.0 * 6 * B * T + 2.0 * 3 * poro::STAR_NNZ * B * T + s4b) * refine_sweeps;
    return PORO_OK;
}

// ------------------------------------------------------------ mesh mode
poro_status poro_set_mesh(poro_ctx* c, int64_t n_vert, const double* xyz, int64_t n_elem, const int64_t* tet,
                          const int64_t* nb, const int32_t* face_tag) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_mesh: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT) return fail(c, PORO_EUNSUPPORTED, "poro_set_mesh: meshes and time stepping are built for Biot's system");
    if (n_vert <= 0 || n_elem <= 0 || !xyz || !tet || !nb || !face_tag)
        return fail(c, PORO_EINVAL, "poro_set_mesh: empty mesh or NULL array");
    for (int64_t i = 0; i < 4 * n_elem; ++i) {
        if (tet[i] < 0 || tet[i] >= n_vert) return fail(c, PORO_EINVAL, "poro_set_mesh: vertex index out of range");
        if (nb[i] < -1 || nb[i] >= n_elem) return fail(c, PORO_EINVAL, "poro_set_mesh: neighbour index out of range");
        if (nb[i] < 0 && face_tag[i] != PORO_FACE_FREE_SURFACE && face_tag[i] != PORO_FACE_ABSORBING)
            return fail(c, PORO_EINVAL, "poro_set_mesh: boundary face needs a free-surface or absorbing tag");
    }
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    c->h_xyz.assign(xyz, xyz + 3 * n_vert);
    c->h_tet.assign(tet, tet + 4 * n_elem);
    c->h_nb.assign(nb, nb + 4 * n_elem);
    c->h_tag.assign(face_tag, face_tag + 4 * n_elem);
    c->h_mat.clear();
    c->mesh_mode = true;
    c->have_mat = false;
    c->rec_elem.clear();
    c->rec_phi.clear();
    c->seis_q.clear();
    c->seis_t.clear();
    c->t = 0.0;
    c->tick = 0;
    return PORO_OK;
}

poro_status poro_set_materials(poro_ctx* c, const poro_material* mat) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_materials: ctx is NULL");
    if (!c->mesh_mode) return fail(c, PORO_ESTATE, "poro_set_materials: no mesh");
    if (!mat) return fail(c, PORO_EINVAL, "poro_set_materials: NULL");
    const int64_t ne = (int64_t)c->h_tet.size() / 4;
    for (int64_t i = 0; i < ne; ++i) {
        double v;
        std::string err;
        if (!poro::max_wave_speed(mat[i], v, err))
            return fail(c, PORO_EINVAL, "poro_set_materials: element " + std::to_string(i) + ": " + err);
    }
    c->h_mat.assign(mat, mat + ne);
    c->have_mat = true;
    return PORO_OK;
}

namespace {
void elem_vertices(const poro_ctx* c, int64_t e, double v[12]) {
    for (int k = 0; k < 4; ++k)
        for (int d = 0; d < 3; ++d) v[3 * k + d] = c->h_xyz[3 * c->h_tet[4 * e + k] + d];
}

// element containing x: the lowest id whose barycentric coordinates are all >= -1e-12
bool locate_point(const poro_ctx* c, const double x[3], int64_t& elem, double xi[3]) {
    const int64_t ne = (int64_t)c->h_tet.size() / 4;
    for (int64_t e = 0; e < ne; ++e) {
        double v[12], jinv[3][3], vol, dins;
        std::string err;
        elem_vertices(c, e, v);
        if (!poro::tet_geometry(v, jinv, vol, dins, err)) continue;
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = x[d] - v[d];
        for (int j = 0; j < 3; ++j) xi[j] = jinv[j][0] * r[0] + jinv[j][1] * r[1] + jinv[j][2] * r[2];
        const double b0 = 1.0 - xi[0] - xi[1] - xi[2];
        if (b0 >= -1e-12 && xi[0] >= -1e-12 && xi[1] >= -1e-12 && xi[2] >= -1e-12) {
            elem = e;
            return true;
        }
    }
    return false;
}
}  // namespace

poro_status poro_set_clusters(poro_ctx* c, double cfl_c, int32_t max_clusters, double* dt_min_out,
                              int32_t* cluster_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_clusters: ctx is NULL");
    if (!c->mesh_mode || !c->have_mat) return fail(c, PORO_ESTATE, "poro_set_clusters: mesh and materials first");
    if (!(cfl_c > 0.0) || max_clusters < 1) return fail(c, PORO_EINVAL, "poro_set_clusters: bad argument");
    if (max_clusters > 16) return fail(c, PORO_EINVAL, "poro_set_clusters: at most 16 clusters");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    const int64_t ne = (int64_t)c->h_tet.size() / 4;
    const int N = c->N, B = c->B;
    std::vector<double> detJ(ne), dte(ne);
    double dtmin = 1e300;
    for (int64_t e = 0; e < ne; ++e) {
        double v[12], jinv[3][3], vol, dins, sp;
        std::string err;
        elem_vertices(c, e, v);
        if (!poro::tet_geometry(v, jinv, vol, dins, err) || !poro::max_wave_speed(c->h_mat[e], sp, err))
            return fail(c, PORO_EINVAL, "poro_set_clusters: element " + std::to_string(e) + ": " + err);
        detJ[e] = 6.0 * vol;
        dte[e] = cfl_c / (2 * N + 1) * dins / sp;
        dtmin = std::min(dtmin, dte[e]);
    }
    // rate-2 clusters: c_e = min(C - 1, floor(log2(dt_e / dt_min))), dt_c = 2^c dt_min
    const int C = max_clusters;
    c->h_cl.assign(ne, 0);
    for (int64_t e = 0; e < ne; ++e) {
        int ce = (int)std::floor(std::log2(dte[e] / dtmin) + 1e-12);
        c->h_cl[e] = std::max(0, std::min(C - 1, ce));
    }
    std::vector<double> ec((size_t)ne * c->stride);
    for (int64_t e = 0; e < ne; ++e) {
        double v[12];
        std::string err;
        elem_vertices(c, e, v);
        const double dt_e = std::ldexp(dtmin, c->h_cl[e]);
        if (!poro::element_constants(c->ref, v, c->h_mat[e], dt_e, ec.data() + (size_t)e * c->stride, err))
            return fail(c, PORO_EINVAL, "poro_set_clusters: element " + std::to_string(e) + ": " + err);
    }
    poro_status st = upload_population(c, ne, ec);
    if (st != PORO_OK) return st;
    cudaMemsetAsync(c->d_q0, 0, (size_t)ne * NQ * B * sizeof(double), c->stream);
    // faces: neighbour face, vertex permutation, normal, area, flux solvers
    std::vector<int32_t> nb(4 * ne), tab(4 * ne);
    std::vector<double> fc(4 * ne), fF((size_t)ne * 4 * 2 * NQ * NQ);
    // per element (independent): run over host threads, each with its own
    // cache of flux solvers keyed by (materials, normal, kind)
    auto face_setup = [&](int64_t e, std::map<std::string, std::vector<double>>& cache, std::string& ferr) -> bool {
        double v[12];
        elem_vertices(c, e, v);
        for (int f = 0; f < 4; ++f) {
            int fv[3], n_ = 0;
            for (int k = 0; k < 4; ++k)
                if (k != f) fv[n_++] = k;
            const double* p0 = v + 3 * fv[0];
            const double* p1 = v + 3 * fv[1];
            const double* p2 = v + 3 * fv[2];
            double a[3], b[3], nr[3];
            for (int d = 0; d < 3; ++d) {
                a[d] = p1[d] - p0[d];
                b[d] = p2[d] - p0[d];
            }
            nr[0] = a[1] * b[2] - a[2] * b[1];
            nr[1] = a[2] * b[0] - a[0] * b[2];
            nr[2] = a[0] * b[1] - a[1] * b[0];
            const double len = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
            double dotv = 0;
            for (int d = 0; d < 3; ++d) {
                nr[d] /= len;
                dotv += nr[d] * (v[3 * f + d] - p0[d]);
            }
            if (dotv > 0)
                for (int d = 0; d < 3; ++d) nr[d] = -nr[d];
            fc[4 * e + f] = len / detJ[e];  // 2 |S_f| / |J| with |S_f| = len / 2
            const int64_t r = c->h_nb[4 * e + f];
            nb[4 * e + f] = (int32_t)r;
            tab[4 * e + f] = -1;
            int kind = r >= 0 ? PORO_FACE_INTERIOR : c->h_tag[4 * e + f];
            if (r >= 0) {
                // neighbour face whose vertices equal ours up to one translation
                double w[12];
                elem_vertices(c, r, w);
                double scale = 0;
                for (int k = 0; k < 12; ++k) scale = std::max(scale, std::fabs(v[k]));
                const double tol = 1e-9 * (1.0 + scale);
                for (int h = 0; h < 4 && tab[4 * e + f] < 0; ++h) {
                    int hv[3], m_ = 0;
                    for (int k = 0; k < 4; ++k)
                        if (k != h) hv[m_++] = k;
                    double sh[3];
                    for (int d = 0; d < 3; ++d)
                        sh[d] = (w[3 * hv[0] + d] + w[3 * hv[1] + d] + w[3 * hv[2] + d] - p0[d] - p1[d] - p2[d]) / 3.0;
                    int perm[3];
                    bool ok = true;
                    const double* ps[3] = {p0, p1, p2};
                    for (int i = 0; i < 3 && ok; ++i) {
                        perm[i] = -1;
                        for (int j = 0; j < 3; ++j) {
                            double dd = 0;
                            for (int d = 0; d < 3; ++d) dd = std::max(dd, std::fabs(w[3 * hv[j] + d] - ps[i][d] - sh[d]));
                            if (dd < tol) perm[i] = j;
                        }
                        ok = perm[i] >= 0;
                    }
                    if (ok && perm[0] != perm[1] && perm[1] != perm[2] && perm[0] != perm[2])
                        tab[4 * e + f] = f * 24 + h * 6 + poro::face_permutation_index(perm);
                }
                if (tab[4 * e + f] < 0) {
                    ferr = "non-conforming face at element " + std::to_string(e);
                    return false;
                }
            }
            std::string key(reinterpret_cast<const char*>(&c->h_mat[e]), sizeof(poro_material));
            if (r >= 0) key.append(reinterpret_cast<const char*>(&c->h_mat[r]), sizeof(poro_material));
            key.append(reinterpret_cast<const char*>(nr), sizeof(nr));
            key.append(reinterpret_cast<const char*>(&kind), sizeof(kind));
            auto itc = cache.find(key);
            double* dst = fF.data() + ((size_t)(4 * e + f) * 2) * NQ * NQ;
            if (itc == cache.end()) {
                std::vector<double> F(2 * NQ * NQ);
                std::string err;
                if (!poro::flux_solver(c->h_mat[e], r >= 0 ? &c->h_mat[r] : nullptr, nr, kind, F.data(),
                                       F.data() + NQ * NQ, err)) {
                    ferr = "flux at element " + std::to_string(e) + ": " + err;
                    return false;
                }
                itc = cache.emplace(key, std::move(F)).first;
            }
            std::memcpy(dst, itc->second.data(), sizeof(double) * 2 * NQ * NQ);
        }
        return true;
    };
    {
        const int nthreads = (int)std::max<int64_t>(1, std::min<int64_t>(
            std::min<unsigned>(32u, std::max(1u, std::thread::hardware_concurrency())), ne / 256 + 1));
        std::vector<std::string> errs(nthreads);
        std::vector<int64_t> bad_at(nthreads, -1);
        std::vector<std::thread> pool;
        for (int t = 0; t < nthreads; ++t)
            pool.emplace_back([&, t] {
                std::map<std::string, std::vector<double>> cache;
                for (int64_t e = t; e < ne; e += nthreads)
                    if (!face_setup(e, cache, errs[t])) {
                        bad_at[t] = e;
                        return;
                    }
            });
        for (auto& th : pool) th.join();
        int64_t first_bad = -1;
        std::string msg;
        for (int t = 0; t < nthreads; ++t)
            if (bad_at[t] >= 0 && (first_bad < 0 || bad_at[t] < first_bad)) {
                first_bad = bad_at[t];
                msg = errs[t];
            }
        if (first_bad >= 0) {
            free_population(c);
            return fail(c, msg.rfind("flux", 0) == 0 ? PORO_ENUMERIC : PORO_EINVAL, "poro_set_clusters: " + msg);
        }
    }
    // volume CSR: Kv^j_kl = M_ll Khat^j_lk / M_kk
    std::vector<int32_t> vrow, vcol;
    std::vector<double> vval, minv(B);
    for (int j = 0; j < 3; ++j) {
        for (int k = 0; k < B; ++k) {
            vrow.push_back((int32_t)vcol.size());
            for (int l = 0; l < B; ++l) {
                const double kh = c->ref.khat[((size_t)j * B + l) * B + k];
                if (kh != 0.0) {
                    vcol.push_back(l);
                    vval.push_back(c->ref.mass_diag[l] * kh / c->ref.mass_diag[k]);
                }
            }
        }
        vrow.push_back((int32_t)vcol.size());
    }
    // absolute row offsets per direction: rows of direction j start at j*(B+1)
    for (int k = 0; k < B; ++k) minv[k] = 1.0 / c->ref.mass_diag[k];
    // face traces: Floc^f = Pf^T Pf, Fnb^{f,h,s} = Pf^T Pnb
    std::vector<double> Pf, Pnb;
    poro::face_traces(N, Pf, Pnb);
    // the mixed-precision form corrects in double-binary32: (hi, lo) copies
    const bool dw = c->prec != PORO_FP64;
    auto split = [](const std::vector<double>& x) {
        std::vector<float> o(2 * x.size());
        for (size_t i = 0; i < x.size(); ++i) {
            const float h = (float)x[i];
            o[2 * i] = h;
            o[2 * i + 1] = (float)(x[i] - (double)h);
        }
        return o;
    };
    cudaError_t er = cudaSuccess;
    if (dw) {
        const std::vector<float> f2 = split(fF), l2 = split(Pf), n2 = split(Pnb), v2 = split(vval);
        if ((er = upload((void**)&c->d_fF2, f2.data(), f2.size() * sizeof(float))) != cudaSuccess ||
            (er = upload((void**)&c->d_Pf2, l2.data(), l2.size() * sizeof(float))) != cudaSuccess ||
            (er = upload((void**)&c->d_Pnb2, n2.data(), n2.size() * sizeof(float))) != cudaSuccess ||
            (er = upload((void**)&c->d_vval2, v2.data(), v2.size() * sizeof(float))) != cudaSuccess) {
            free_population(c);
            return er == cudaErrorMemoryAllocation ? fail(c, PORO_ENOMEM, "poro_set_clusters: out of device memory")
                                                   : cuda_fail(c, er, "poro_set_clusters");
        }
    }
    if ((er = upload((void**)&c->d_nb, nb.data(), nb.size() * sizeof(int32_t))) != cudaSuccess ||
        (er = upload((void**)&c->d_tab, tab.data(), tab.size() * sizeof(int32_t))) != cudaSuccess ||
        (er = upload((void**)&c->d_fc, fc.data(), fc.size() * sizeof(double))) != cudaSuccess ||
        (!dw && (er = upload((void**)&c->d_fF, fF.data(), fF.size() * sizeof(double))) != cudaSuccess) ||
        (er = upload((void**)&c->d_vrow, vrow.data(), vrow.size() * sizeof(int32_t))) != cudaSuccess ||
        (er = upload((void**)&c->d_vcol, vcol.data(), vcol.size() * sizeof(int32_t))) != cudaSuccess ||
        (er = upload((void**)&c->d_vval, vval.data(), vval.size() * sizeof(double))) != cudaSuccess ||
        (er = upload((void**)&c->d_minv, minv.data(), minv.size() * sizeof(double))) != cudaSuccess ||
        (er = upload((void**)&c->d_Pf, Pf.data(), Pf.size() * sizeof(double))) != cudaSuccess ||
        (er = upload((void**)&c->d_Pnb, Pnb.data(), Pnb.size() * sizeof(double))) != cudaSuccess) {
        free_population(c);
        return er == cudaErrorMemoryAllocation ? fail(c, PORO_ENOMEM, "poro_set_clusters: out of device memory")
                                               : cuda_fail(c, er, "poro_set_clusters");
    }
    poro::CorrectorData& d = c->cd;
    d.N = N;
    d.econst = c->d_econst;
    d.iout = c->d_iout;
    d.q = c->d_q0;
    d.nb = c->d_nb;
    d.tab = c->d_tab;
    d.fc = c->d_fc;
    d.fF = c->d_fF;
    d.Pf = c->d_Pf;
    d.Pnb = c->d_Pnb;
    d.vrow = c->d_vrow;
    d.vcol = c->d_vcol;
    d.vval = c->d_vval;
    d.minv = c->d_minv;
    d.dw = dw;
    d.fF2 = c->d_fF2;
    d.Pf2 = c->d_Pf2;
    d.Pnb2 = c->d_Pnb2;
    d.vval2 = c->d_vval2;
    // clusters: element lists, buffer slots of (element, larger neighbour level)
    c->C = C;
    c->cl_elems.assign(C, std::vector<int32_t>());
    for (int64_t e = 0; e < ne; ++e) c->cl_elems[c->h_cl[e]].push_back((int32_t)e);
    std::vector<int32_t> slot((size_t)ne * C, -1);
    int32_t nslot = 0;
    c->cl_has_slot.assign(C, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < 4; ++f) {
            const int64_t r = c->h_nb[4 * e + f];
            if (r >= 0 && c->h_cl[r] > c->h_cl[e] && slot[e * C + c->h_cl[r]] < 0) {
                slot[e * C + c->h_cl[r]] = nslot++;
                c->cl_has_slot[c->h_cl[e]] = 1;
            }
        }
    for (int k = 0; k < C; ++k) {
        int32_t* d = nullptr;
        if (!c->cl_elems[k].empty() &&
            (er = upload((void**)&d, c->cl_elems[k].data(), c->cl_elems[k].size() * sizeof(int32_t))) != cudaSuccess) {
            free_population(c);
            return cuda_fail(c, er, "poro_set_clusters");
        }
        c->d_cl_elems.push_back(d);
    }
    if (C > 1) {
        if ((er = upload((void**)&c->d_cl, c->h_cl.data(), ne * sizeof(int32_t))) != cudaSuccess ||
            (er = upload((void**)&c->d_slot, slot.data(), slot.size() * sizeof(int32_t))) != cudaSuccess ||
            (er = cudaMalloc((void**)&c->d_buf, (size_t)std::max(nslot, 1) * NQ * B * sizeof(double))) != cudaSuccess) {
            free_population(c);
            return er == cudaErrorMemoryAllocation ? fail(c, PORO_ENOMEM, "poro_set_clusters: out of device memory")
                                                   : cuda_fail(c, er, "poro_set_clusters");
        }
    }
    d.C = C;
    d.cl = c->d_cl;
    d.slot = c->d_slot;
    d.buf = c->d_buf;
    d.qt = c->d_qt;
    c->dt = dtmin;
    c->t = 0.0;
    c->tick = 0;
    c->have_dofs = true;
    c->ready = true;
    c->seis_q.assign(c->rec_elem.size(), std::vector<double>());
    c->seis_t.assign(c->rec_elem.size(), std::vector<double>());
    if (dt_min_out) *dt_min_out = dtmin;
    if (cluster_out)
        for (int64_t e = 0; e < ne; ++e) cluster_out[e] = c->h_cl[e];
    er = cudaStreamSynchronize(c->stream);
    if (er != cudaSuccess) return cuda_fail(c, er, "poro_set_clusters");
    return PORO_OK;
}

poro_status poro_add_point_source(poro_ctx* c, const double xyz[3], const double w[13], double f0, double t0,
                                  double amplitude) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_add_point_source: ctx is NULL");
    if (!c->ready) return fail(c, PORO_ESTATE, "poro_add_point_source: call poro_set_clusters first");
    if (!xyz || !w || !(f0 > 0.0)) return fail(c, PORO_EINVAL, "poro_add_point_source: bad argument");
    int64_t e;
    double xi[3];
    if (!locate_point(c, xyz, e, xi)) return fail(c, PORO_EINVAL, "poro_add_point_source: point outside the mesh");
    double v[12], jinv[3][3], vol, dins;
    std::string err;
    elem_vertices(c, e, v);
    poro::tet_geometry(v, jinv, vol, dins, err);
    std::vector<double> phi(c->B), coef((size_t)NQ * c->B);
    poro::basis_at(c->N, xi, phi.data());
    for (int p = 0; p < NQ; ++p)
        for (int k = 0; k < c->B; ++k)
            coef[p * c->B + k] = amplitude * w[p] * phi[k] / (6.0 * vol * c->ref.mass_diag[k]);
    poro_ctx::Source s{e, nullptr, f0, t0};
    cudaError_t er = upload((void**)&s.d_coef, coef.data(), coef.size() * sizeof(double));
    if (er != cudaSuccess) return cuda_fail(c, er, "poro_add_point_source");
    c->sources.push_back(s);
    return PORO_OK;
}

poro_status poro_add_receiver(poro_ctx* c, const double xyz[3], int32_t* id_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_add_receiver: ctx is NULL");
    if (!c->mesh_mode) return fail(c, PORO_ESTATE, "poro_add_receiver: no mesh");
    if (!xyz) return fail(c, PORO_EINVAL, "poro_add_receiver: NULL");
    int64_t e;
    double xi[3];
    if (!locate_point(c, xyz, e, xi)) return fail(c, PORO_EINVAL, "poro_add_receiver: point outside the mesh");
    std::vector<double> phi(c->B);
    poro::basis_at(c->N, xi, phi.data());
    c->rec_elem.push_back(e);
    c->rec_phi.insert(c->rec_phi.end(), phi.begin(), phi.end());
    c->seis_q.emplace_back();
    c->seis_t.emplace_back();
    if (id_out) *id_out = (int32_t)c->rec_elem.size() - 1;
    return PORO_OK;
}

// Enqueue one cycle (2^(C-1) ticks) on the context stream: no host
// synchronisation and no allocation, so it can be captured in a CUDA graph.
// Ticks inside the kernels are relative to the cycle (only their residues
// modulo 2^c matter); the absolute tick for the sources is read from
// d_tick, which the cycle advances at its end.
// One tick k of the cycle for context c on stream st: predictors of the
// clusters that start a step at k, LTS buffers, correctors of the clusters
// whose step ends at k + 1, point sources and receivers.  `what` selects the
// parts (TICK_*): a batched group runs the predictors and correctors of all
// its runs as single launches and the rest per run.
// (prof, nullable: an event pair recorded around each cluster's launches,
// for poro_cluster_times)
struct ClusterEvent {
    int cl;
    cudaEvent_t a, b;
};
static int mark(std::vector<ClusterEvent>* prof, int cl, bool begin, cudaStream_t st) {
    if (!prof) return 0;
    if (begin) {
        ClusterEvent ev{cl, nullptr, nullptr};
        cudaError_t e = cudaEventCreate(&ev.a);
        if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
        if (e == cudaSuccess) e = cudaEventRecord(ev.a, st);
        prof->push_back(ev);
        return (int)e;
    }
    return (int)cudaEventRecord(prof->back().b, st);
}

enum : unsigned { TICK_PREDICT = 1, TICK_BUFFERS = 2, TICK_CORRECT = 4, TICK_SOURCES = 8, TICK_ALL = 15 };

static int enqueue_tick(poro_ctx* c, int64_t k, unsigned what, const double* d_rp, double* d_seis, int64_t cap,
                        int32_t* d_cnt, cudaStream_t st, std::vector<ClusterEvent>* prof = nullptr) {
    const bool predict = (what & TICK_PREDICT) != 0;
    const int C = c->C;
    const int nrec = (int)c->rec_elem.size();
    const bool want_qt = C > 1;
    int rc = 0;
    for (int cl = 0; cl < C && rc == 0; ++cl) {
        if (k % ((int64_t)1 << cl) || c->cl_elems[cl].empty()) continue;
        rc = mark(prof, cl, true, st);
        const int32_t* el = C > 1 ? c->d_cl_elems[cl] : nullptr;
        const int64_t cnt = (int64_t)c->cl_elems[cl].size();
        if (predict && c->prec == PORO_FP64)
            rc = poro::launch_stp_fp64(c->dref, el, cnt, c->d_q0, c->d_econst, want_qt ? c->d_qt : nullptr,
                                       c->d_iout, st, c->variant);
        else if (predict)
            rc = poro::launch_stp_mixed(c->mref, c->refine, el, cnt, c->d_q0, c->d_econst,
                                        want_qt ? c->d_qt : nullptr, c->d_iout, st, c->variant);
        // (a cluster whose elements buffer for no larger neighbour has nothing to add)
        if (rc == 0 && C > 1 && (what & TICK_BUFFERS) && c->cl_has_slot[cl])
            rc = poro::launch_lts_buffers(c->N, C, el, cnt, c->d_slot, c->d_iout, c->d_buf, k, st);
        if (rc == 0) rc = mark(prof, cl, false, st);
    }
    {
        for (int cl = 0; cl < C && rc == 0; ++cl) {
            const int64_t len = (int64_t)1 << cl;
            if ((k + 1) % len || c->cl_elems[cl].empty()) continue;
            rc = mark(prof, cl, true, st);
            poro::CorrectorData d = c->cd;
            d.tick = k;
            if (what & TICK_CORRECT)
                rc = poro::launch_corrector(d, C > 1 ? c->d_cl_elems[cl] : nullptr, (int64_t)c->cl_elems[cl].size(),
                                            st);
            if (!(what & TICK_SOURCES)) {
                if (rc == 0) rc = mark(prof, cl, false, st);
                continue;
            }
            for (auto& src : c->sources)
                if (rc == 0 && c->h_cl[src.elem] == cl)
                    rc = poro::launch_point_source_tick(c->N, c->d_q0, src.elem, src.d_coef, src.f0, src.t0, c->dt, len,
                                                        k, c->d_tick, st);
            for (int r = 0; r < nrec && rc == 0; ++r)
                if (c->h_cl[c->rec_elem[r]] == cl)
                    rc = poro::launch_receiver_count(c->N, c->d_q0, c->rec_elem[r], d_rp + (size_t)r * c->B,
                                                     d_seis + (size_t)r * cap * NQ, d_cnt + r, st);
            if (rc == 0) rc = mark(prof, cl, false, st);
        }
    }
    return rc;
}

static int enqueue_cycle(poro_ctx* c, const double* d_rp, double* d_seis, int64_t cap, int32_t* d_cnt) {
    const int64_t cycle = (int64_t)1 << (c->C - 1);
    int rc = 0;
    for (int64_t k = 0; k < cycle && rc == 0; ++k) rc = enqueue_tick(c, k, TICK_ALL, d_rp, d_seis, cap, d_cnt, c->stream);
    if (rc == 0) rc = poro::launch_tick_advance(c->d_tick, cycle, c->stream);
    return rc;
}

// Before `ticks` ticks of c on stream st: the device tick counter and the
// receiver staging buffers (kept across calls, grown only when a call needs
// more samples).
static poro_status prepare_advance(poro_ctx* c, int64_t ticks, cudaStream_t st, const char* who) {
    const int nrec = (int)c->rec_elem.size();
    cudaError_t er = cudaSuccess;
    if (!c->d_tick && (er = cudaMalloc((void**)&c->d_tick, sizeof(int64_t))) != cudaSuccess) return cuda_fail(c, er, who);
    if ((er = cudaMemcpyAsync(c->d_tick, &c->tick, sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, er, who);
    if (nrec > 0) {
        if (c->rp_n != (size_t)nrec) {
            dfree(c->d_rp);
            dfree(c->d_cnt);
            c->rp_n = 0;
            if ((er = upload((void**)&c->d_rp, c->rec_phi.data(), c->rec_phi.size() * sizeof(double))) != cudaSuccess ||
                (er = cudaMalloc((void**)&c->d_cnt, nrec * sizeof(int32_t))) != cudaSuccess)
                return cuda_fail(c, er, who);
            c->rp_n = nrec;
            dfree(c->d_seis);
            c->seis_cap = 0;
        }
        if (c->seis_cap < ticks) {
            dfree(c->d_seis);
            c->seis_cap = 0;
            if ((er = cudaMalloc((void**)&c->d_seis, (size_t)nrec * ticks * NQ * sizeof(double))) != cudaSuccess)
                return cuda_fail(c, er, who);
            c->seis_cap = ticks;
        }
        if ((er = cudaMemsetAsync(c->d_cnt, 0, nrec * sizeof(int32_t), st)) != cudaSuccess) return cuda_fail(c, er, who);
    }
    return PORO_OK;
}

// Receiver samples of the advance to the host staging buffer (asynchronous on st).
static cudaError_t stage_seismograms(poro_ctx* c, cudaStream_t st) {
    const int nrec = (int)c->rec_elem.size();
    if (nrec == 0) return cudaSuccess;
    c->h_seis.resize((size_t)nrec * c->seis_cap * NQ);
    return cudaMemcpyAsync(c->h_seis.data(), c->d_seis, c->h_seis.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
}

// After the stream of an advance of `ticks` ticks finished: append the staged
// receiver samples and move the clock.
static void finish_advance(poro_ctx* c, int64_t ticks) {
    const int nrec = (int)c->rec_elem.size();
    const std::vector<double>& h = c->h_seis;
    const int64_t cap = c->seis_cap;
    for (int r = 0; r < nrec; ++r) {
        const int cl = c->h_cl[c->rec_elem[r]];
        const int64_t len = (int64_t)1 << cl, ns = ticks / len;
        c->seis_q[r].insert(c->seis_q[r].end(), h.begin() + (size_t)r * cap * NQ,
                            h.begin() + ((size_t)r * cap + ns) * NQ);
        for (int64_t j = 1; j <= ns; ++j) c->seis_t[r].push_back((double)(c->tick + j * len) * c->dt);
    }
    c->tick += ticks;
    c->t = (double)c->tick * c->dt;
    c->have_pred = true;
}

poro_status poro_advance(poro_ctx* c, double t_end) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_advance: ctx is NULL");
    if (!c->ready) return fail(c, PORO_ESTATE, "poro_advance: call poro_set_clusters first");
    cudaSetDevice(c->device);
    const int C = c->C;
    const int64_t cycle = (int64_t)1 << (C - 1);            // ticks per step of the largest cluster
    const double dt_max = std::ldexp(c->dt, C - 1);
    const int64_t n_cycles = (int64_t)std::floor((t_end - c->t) / dt_max + 1e-9);
    if (n_cycles <= 0) return PORO_OK;
    const int64_t ticks = n_cycles * cycle;
    if (poro_status st = prepare_advance(c, ticks, c->stream, "poro_advance")) return st;
    double* d_rp = c->d_rp;
    double* d_seis = c->d_seis;
    int32_t* d_cnt = c->d_cnt;
    const int64_t cap = c->seis_cap;
    cudaError_t er = cudaSuccess;
    // the first cycle runs directly (it also sets the kernels' attributes);
    // the others replay a CUDA graph of one cycle
    int rc = enqueue_cycle(c, d_rp, d_seis, cap, d_cnt);
    if (rc == 0 && n_cycles > 1) {
        if (c->use_graphs) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            er = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (er == cudaSuccess) {
                rc = enqueue_cycle(c, d_rp, d_seis, cap, d_cnt);
                cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
                if (rc == 0 && e2 != cudaSuccess) rc = (int)e2;
            } else {
                rc = (int)er;
            }
            if (rc == 0) rc = (int)cudaGraphInstantiate(&exec, graph, 0);
            for (int64_t k = 1; k < n_cycles && rc == 0; ++k) rc = (int)cudaGraphLaunch(exec, c->stream);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        } else {
            for (int64_t k = 1; k < n_cycles && rc == 0; ++k) rc = enqueue_cycle(c, d_rp, d_seis, cap, d_cnt);
        }
    }
    if (rc == 0) er = stage_seismograms(c, c->stream);
    if (rc == 0 && er == cudaSuccess) er = cudaStreamSynchronize(c->stream);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "poro_advance: kernel launch / graph");
    if (er != cudaSuccess) return cuda_fail(c, er, "poro_advance");
    if (poro_status st = device_status(c, "poro_advance")) return st;
    finish_advance(c, ticks);
    return PORO_OK;
}

// ------------------------------------------------------ batched groups of runs
// Several simulations of one degree, precision, refinement, CTA variant and
// cluster count advance together: every tick's predictors of all runs' due
// clusters are one launch (items = (run, element) pairs), then each run's LTS
// buffers, correctors, sources and receivers; a cycle is captured once as a
// CUDA graph and replayed.  Results are those of each run advanced alone:
// every element's predictor is computed by one CTA with the same code.
}  // extern "C"

namespace poro {

struct RunGroup {
    std::vector<poro_ctx*> runs;
    int device = 0, C = 1;
    int64_t cycle = 1;
    cudaStream_t stream = nullptr;
    RunPtrs* d_runs = nullptr;
    int32_t* d_items = nullptr;      // elements of all runs' due clusters, tick residue by tick residue
    int32_t* d_item_run = nullptr;
    std::vector<int64_t> k_off, k_cnt;
    // correctors: per tick residue k the elements of all runs' clusters whose
    // step ends at k + 1, and each run's corrector data with tick k
    // ([cycle][runs] tables)
    CorrectorData* d_cdata = nullptr;
    int32_t* d_citems = nullptr;
    int32_t* d_citem_run = nullptr;
    std::vector<int64_t> ck_off, ck_cnt;
    // per tick residue k the point sources and the receivers of all runs
    // due at k (built for the runs' current receiver buffers)
    TickItem* d_src = nullptr;
    TickItem* d_rec = nullptr;
    int64_t** d_ticks = nullptr;     // the runs' tick counters
    std::vector<int64_t> src_off, src_cnt, rec_off, rec_cnt;
    int64_t pending = 0;             // ticks enqueued since the last group_finish
    // captured cycle, valid while every run's receiver buffers stay the same
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> exec_key;
};

static int enqueue_group_cycle(RunGroup* g) {
    poro_ctx* lead = g->runs[0];
    int rc = 0;
    for (int64_t k = 0; k < g->cycle && rc == 0; ++k) {
        const int64_t cnt = g->k_cnt[k];
        if (cnt > 0) {
            const int32_t* el = g->d_items + g->k_off[k];
            const int32_t* ir = g->d_item_run + g->k_off[k];
            if (lead->prec == PORO_FP64)
                rc = launch_stp_fp64(lead->dref, el, cnt, nullptr, nullptr, nullptr, nullptr, g->stream, lead->variant,
                                     g->d_runs, ir);
            else
                rc = launch_stp_mixed(lead->mref, lead->refine, el, cnt, nullptr, nullptr, nullptr, nullptr, g->stream,
                                      lead->variant, g->d_runs, ir);
        }
        for (poro_ctx* c : g->runs)
            if (rc == 0) rc = enqueue_tick(c, k, TICK_BUFFERS, c->d_rp, c->d_seis, c->seis_cap, c->d_cnt, g->stream);
        const int64_t cc = g->ck_cnt[k];
        if (rc == 0 && cc > 0)
            rc = launch_corrector(lead->cd, g->d_citems + g->ck_off[k], cc, g->stream,
                                  g->d_cdata + k * (int64_t)g->runs.size(), g->d_citem_run + g->ck_off[k]);
        // all runs' sources of the tick, then all their receivers (one launch each)
        if (rc == 0) rc = launch_tick_sources(lead->N, g->d_src + g->src_off[k], g->src_cnt[k], g->stream);
        if (rc == 0) rc = launch_tick_receivers(lead->N, g->d_rec + g->rec_off[k], g->rec_cnt[k], g->stream);
    }
    if (rc == 0) rc = launch_ticks_advance(g->d_ticks, (int)g->runs.size(), g->cycle, g->stream);
    return rc;
}

void group_destroy(RunGroup* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    dfree(g->d_runs);
    dfree(g->d_items);
    dfree(g->d_item_run);
    dfree(g->d_cdata);
    dfree(g->d_citems);
    dfree(g->d_citem_run);
    dfree(g->d_src);
    dfree(g->d_rec);
    dfree(g->d_ticks);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

RunGroup* group_create(poro_ctx* const* runs, int n, std::string& err) {
    if (n <= 0 || !runs) {
        err = "group_create: no runs";
        return nullptr;
    }
    poro_ctx* a = runs[0];
    for (int i = 0; i < n; ++i) {
        poro_ctx* c = runs[i];
        if (!c || !c->ready) {
            err = "group_create: a run has no mesh set-up";
            return nullptr;
        }
        if (c->device != a->device || c->N != a->N || c->prec != a->prec || c->C != a->C || c->variant != a->variant ||
            (c->prec != PORO_FP64 && (c->refine != a->refine || c->mref.wait_limit != a->mref.wait_limit))) {
            err = "group_create: runs differ in device, degree, precision, refinement, variant or clusters";
            return nullptr;
        }
        if (c->tick % ((int64_t)1 << (c->C - 1))) {
            err = "group_create: a run is not at the end of a cycle";
            return nullptr;
        }
    }
    RunGroup* g = new RunGroup();
    g->runs.assign(runs, runs + n);
    g->device = a->device;
    g->C = a->C;
    g->cycle = (int64_t)1 << (a->C - 1);
    cudaSetDevice(g->device);
    std::vector<RunPtrs> rp(n);
    for (int i = 0; i < n; ++i) {
        poro_ctx* c = runs[i];
        rp[i] = RunPtrs{c->d_q0, c->d_econst, g->C > 1 ? c->d_qt : nullptr, c->d_iout};
    }
    std::vector<int32_t> items, item_run;
    for (int64_t k = 0; k < g->cycle; ++k) {
        g->k_off.push_back((int64_t)items.size());
        for (int i = 0; i < n; ++i)
            for (int cl = 0; cl < g->C; ++cl) {
                if (k % ((int64_t)1 << cl)) continue;
                const std::vector<int32_t>& el = runs[i]->cl_elems[cl];
                items.insert(items.end(), el.begin(), el.end());
                item_run.insert(item_run.end(), el.size(), (int32_t)i);
            }
        g->k_cnt.push_back((int64_t)items.size() - g->k_off.back());
    }
    std::vector<int32_t> citems, citem_run;
    std::vector<CorrectorData> cdata;
    for (int64_t k = 0; k < g->cycle; ++k) {
        g->ck_off.push_back((int64_t)citems.size());
        for (int i = 0; i < n; ++i) {
            CorrectorData d = runs[i]->cd;
            d.tick = k;
            cdata.push_back(d);
            for (int cl = 0; cl < g->C; ++cl) {
                if ((k + 1) % ((int64_t)1 << cl)) continue;
                const std::vector<int32_t>& el = runs[i]->cl_elems[cl];
                citems.insert(citems.end(), el.begin(), el.end());
                citem_run.insert(citem_run.end(), el.size(), (int32_t)i);
            }
        }
        g->ck_cnt.push_back((int64_t)citems.size() - g->ck_off.back());
    }
    cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = upload((void**)&g->d_runs, rp.data(), rp.size() * sizeof(RunPtrs));
    if (e == cudaSuccess) e = upload((void**)&g->d_items, items.data(), items.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = upload((void**)&g->d_item_run, item_run.data(), item_run.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = upload((void**)&g->d_cdata, cdata.data(), cdata.size() * sizeof(CorrectorData));
    if (e == cudaSuccess) e = upload((void**)&g->d_citems, citems.data(), citems.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = upload((void**)&g->d_citem_run, citem_run.data(), citem_run.size() * sizeof(int32_t));
    if (e != cudaSuccess) {
        err = std::string("group_create: ") + cudaGetErrorString(e);
        group_destroy(g);
        return nullptr;
    }
    return g;
}

// Enqueue n_cycles cycles of every run of the group (asynchronous on the
// group's stream); group_finish completes them.
// the source and receiver items of every tick residue, for the runs'
// current receiver buffers (synchronous upload; the group's stream is idle)
static int group_tick_items(RunGroup* g) {
    std::vector<TickItem> src, rec;
    g->src_off.clear();
    g->src_cnt.clear();
    g->rec_off.clear();
    g->rec_cnt.clear();
    for (int64_t k = 0; k < g->cycle; ++k) {
        g->src_off.push_back((int64_t)src.size());
        g->rec_off.push_back((int64_t)rec.size());
        for (poro_ctx* c : g->runs) {
            for (int cl = 0; cl < g->C; ++cl) {
                const int64_t len = (int64_t)1 << cl;
                if ((k + 1) % len || c->cl_elems[cl].empty()) continue;
                for (auto& sr : c->sources)
                    if (c->h_cl[sr.elem] == cl) {
                        TickItem it;
                        it.q = c->d_q0;
                        it.vec = sr.d_coef;
                        it.tick = c->d_tick;
                        it.elem = sr.elem;
                        it.len = len;
                        it.k_rel = k;
                        it.f0 = sr.f0;
                        it.tc = sr.t0;
                        it.dt = c->dt;
                        src.push_back(it);
                    }
                for (int r = 0; r < (int)c->rec_elem.size(); ++r)
                    if (c->h_cl[c->rec_elem[r]] == cl) {
                        TickItem it;
                        it.q = c->d_q0;
                        it.vec = c->d_rp + (size_t)r * c->B;
                        it.out = c->d_seis + (size_t)r * c->seis_cap * NQ;
                        it.counter = c->d_cnt + r;
                        it.elem = c->rec_elem[r];
                        rec.push_back(it);
                    }
            }
        }
        g->src_cnt.push_back((int64_t)src.size() - g->src_off.back());
        g->rec_cnt.push_back((int64_t)rec.size() - g->rec_off.back());
    }
    std::vector<int64_t*> ticks;
    for (poro_ctx* c : g->runs) ticks.push_back(c->d_tick);
    dfree(g->d_src);
    dfree(g->d_rec);
    dfree(g->d_ticks);
    cudaError_t e = upload((void**)&g->d_src, src.data(), src.size() * sizeof(TickItem));
    if (e == cudaSuccess) e = upload((void**)&g->d_rec, rec.data(), rec.size() * sizeof(TickItem));
    if (e == cudaSuccess) e = upload((void**)&g->d_ticks, ticks.data(), ticks.size() * sizeof(int64_t*));
    return (int)e;
}

int group_enqueue(RunGroup* g, int64_t n_cycles, std::string& err) {
    if (n_cycles <= 0) return 0;
    cudaSetDevice(g->device);
    const int64_t ticks = n_cycles * g->cycle;
    for (poro_ctx* c : g->runs)
        if (prepare_advance(c, ticks, g->stream, "group_enqueue") != PORO_OK) {
            err = c->err;
            return -1;
        }
    std::vector<const void*> key;
    for (poro_ctx* c : g->runs) {
        key.push_back(c->d_seis);
        key.push_back((const void*)(intptr_t)c->seis_cap);
    }
    int rc = 0;
    int64_t done = 0;
    if (!g->exec || key != g->exec_key) {
        // first cycle directly (sets the kernels' attributes), then capture
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        rc = group_tick_items(g);
        if (rc == 0) rc = enqueue_group_cycle(g);
        done = 1;
        if (rc == 0 && n_cycles > 1) {
            cudaGraph_t graph = nullptr;
            cudaError_t er = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
            if (er == cudaSuccess) {
                rc = enqueue_group_cycle(g);
                cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
                if (rc == 0 && e2 != cudaSuccess) rc = (int)e2;
            } else {
                rc = (int)er;
            }
            if (rc == 0) rc = (int)cudaGraphInstantiate(&g->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (rc == 0) g->exec_key = key;
        }
    }
    for (int64_t k = done; k < n_cycles && rc == 0; ++k) rc = (int)cudaGraphLaunch(g->exec, g->stream);
    for (poro_ctx* c : g->runs)
        if (rc == 0) rc = (int)stage_seismograms(c, g->stream);
    if (rc != 0) {
        err = std::string("group_enqueue: ") + cudaGetErrorString((cudaError_t)rc);
        return rc;
    }
    g->pending += ticks;
    return 0;
}

// Wait for the enqueued cycles and complete every run's bookkeeping.  A
// bounded wait of the batched predictor that gave up fails the whole group
// (PORO_ETIMEOUT).
poro_status group_finish(RunGroup* g, std::string& err) {
    cudaSetDevice(g->device);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        err = std::string("group_finish: ") + cudaGetErrorString(e);
        return PORO_ECUDA;
    }
    const int64_t ticks = g->pending;
    g->pending = 0;
    poro_ctx* lead = g->runs[0];
    if (poro_status st = device_status(lead, "group_finish")) {
        err = lead->err;
        return st;
    }
    for (poro_ctx* c : g->runs) finish_advance(c, ticks);
    return PORO_OK;
}

}  // namespace poro

extern "C" {

poro_status poro_cluster_times(poro_ctx* c, double t_end, double* ms_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_cluster_times: ctx is NULL");
    if (!c->ready) return fail(c, PORO_ESTATE, "poro_cluster_times: call poro_set_clusters first");
    if (!ms_out) return fail(c, PORO_EINVAL, "poro_cluster_times: ms_out is NULL");
    cudaSetDevice(c->device);
    const int C = c->C;
    for (int cl = 0; cl < C; ++cl) ms_out[cl] = 0.0;
    const int64_t cycle = (int64_t)1 << (C - 1);
    const int64_t n_cycles = (int64_t)std::floor((t_end - c->t) / std::ldexp(c->dt, C - 1) + 1e-9);
    if (n_cycles <= 0) return PORO_OK;
    const int64_t ticks = n_cycles * cycle;
    if (poro_status st = prepare_advance(c, ticks, c->stream, "poro_cluster_times")) return st;
    std::vector<ClusterEvent> prof;
    int rc = 0;
    for (int64_t n = 0; n < n_cycles && rc == 0; ++n) {
        for (int64_t k = 0; k < cycle && rc == 0; ++k)
            rc = enqueue_tick(c, k, TICK_ALL, c->d_rp, c->d_seis, c->seis_cap, c->d_cnt, c->stream, &prof);
        if (rc == 0) rc = poro::launch_tick_advance(c->d_tick, cycle, c->stream);
    }
    cudaError_t er = cudaSuccess;
    if (rc == 0) er = stage_seismograms(c, c->stream);
    if (rc == 0 && er == cudaSuccess) er = cudaStreamSynchronize(c->stream);
    for (ClusterEvent& ev : prof) {
        float ms = 0.f;
        if (rc == 0 && er == cudaSuccess && ev.a && ev.b && cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess)
            ms_out[ev.cl] += ms;
        if (ev.a) cudaEventDestroy(ev.a);
        if (ev.b) cudaEventDestroy(ev.b);
    }
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "poro_cluster_times: kernel launch");
    if (er != cudaSuccess) return cuda_fail(c, er, "poro_cluster_times");
    if (poro_status st = device_status(c, "poro_cluster_times")) return st;
    finish_advance(c, ticks);
    return PORO_OK;
}

poro_status poro_set_graphs(poro_ctx* c, int32_t on) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_graphs: ctx is NULL");
    c->use_graphs = on != 0;
    return PORO_OK;
}

poro_status poro_correct(poro_ctx* c, int32_t cluster) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_correct: ctx is NULL");
    if (!c->ready || !c->have_pred) return fail(c, PORO_ESTATE, "poro_correct: mesh set-up and a predictor first");
    if (cluster != -1 && cluster != 0) return fail(c, PORO_EINVAL, "poro_correct: no such cluster");
    cudaSetDevice(c->device);
    int rc = poro::launch_corrector(c->cd, nullptr, c->n_elem, c->stream);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "poro_correct");
    return PORO_OK;
}

poro_status poro_get_dofs(poro_ctx* c, double* Q_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_get_dofs: ctx is NULL");
    if (!c->d_q0 || !c->have_dofs) return fail(c, PORO_ESTATE, "poro_get_dofs: no DOFs");
    if (!Q_out) return fail(c, PORO_EINVAL, "poro_get_dofs: NULL");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(Q_out, c->d_q0, (size_t)c->n_elem * NQ * c->B * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "poro_get_dofs");
    return device_status(c, "poro_get_dofs");
}

poro_status poro_get_seismogram(poro_ctx* c, int32_t rec, int64_t cap, double* t_out, double* q_out, int64_t* n_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_get_seismogram: ctx is NULL");
    if (rec < 0 || rec >= (int32_t)c->rec_elem.size()) return fail(c, PORO_EINVAL, "poro_get_seismogram: no such receiver");
    const int64_t n = (int64_t)c->seis_t[rec].size();
    if (n_out) *n_out = n;
    const int64_t m = std::min(n, cap);
    if (m > 0 && (!t_out || !q_out)) return fail(c, PORO_EINVAL, "poro_get_seismogram: NULL output");
    for (int64_t k = 0; k < m; ++k) {
        t_out[k] = c->seis_t[rec][k];
        for (int p = 0; p < NQ; ++p) q_out[k * NQ + p] = c->seis_q[rec][k * NQ + p];
    }
    return PORO_OK;
}

poro_status poro_get_time(const poro_ctx* c, double* t, double* dt) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_get_time: ctx is NULL");
    if (t) *t = c->t;
    if (dt) *dt = c->dt;
    return PORO_OK;
}

poro_status poro_flux_matrices(const poro_material* mL, const poro_material* mR, const double n[3], int32_t kind,
                               double* Fm, double* Fp) {
    if (!mL || !n || !Fm || !Fp) return fail(nullptr, PORO_EINVAL, "poro_flux_matrices: NULL argument");
    if (kind == PORO_FACE_INTERIOR && !mR) return fail(nullptr, PORO_EINVAL, "poro_flux_matrices: interior needs mR");
    std::string err;
    if (!poro::flux_solver(*mL, mR, n, kind, Fm, Fp, err)) return fail(nullptr, PORO_EINVAL, err);
    return PORO_OK;
}

poro_status poro_autotune(poro_ctx* c, int64_t sample, int32_t* variant_out, double* ms_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_autotune: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT || c->subcell)
        return fail(c, PORO_EUNSUPPORTED, "poro_autotune: the autotuner is built for Biot's constant-material predictor");
    if (!c->d_econst || c->n_elem <= 0) return fail(c, PORO_ESTATE, "poro_autotune: no element population loaded");
    cudaSetDevice(c->device);
    const int64_t n = std::max<int64_t>(1, std::min(sample > 0 ? sample : c->n_elem, c->n_elem));
    double best = 1e300;
    int bestv = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved = c->variant;
    for (int v = 0; v < 2; ++v) {
        c->variant = v;
        poro_status s = PORO_OK;
        for (int w = 0; w < 2 && s == PORO_OK; ++w)
            s = dispatch_predict(c, 0, n, c->d_q0, c->d_qt, c->d_iout, PORO_SOLVE_BLOCK, c->stream);
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && s == PORO_OK; ++r)
            s = dispatch_predict(c, 0, n, c->d_q0, c->d_qt, c->d_iout, PORO_SOLVE_BLOCK, c->stream);
        cudaEventRecord(e1, c->stream);
        cudaError_t er = cudaEventSynchronize(e1);
        if (s != PORO_OK || er != cudaSuccess) {
            c->variant = saved;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return s != PORO_OK ? s : cuda_fail(c, er, "poro_autotune");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) ms_out[v] = ms / 3.0;
        if (ms < best) {
            best = ms;
            bestv = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->variant = bestv;
    if (variant_out) *variant_out = bestv;
    return PORO_OK;
}

// tile choices: CTA-size variant x operand layout caps (A buffers, Khat slots)
static const int kTileCaps[6][2] = {{3, 3}, {2, 3}, {1, 3}, {2, 2}, {1, 2}, {1, 1}};

static bool tile_choice_valid(const poro_ctx* c, int choice) {
    if (choice < 0 || choice >= PORO_TILE_CHOICES) return false;
    const int cta = choice / 6, lay = choice % 6;
    if (c->prec == PORO_FP64) return lay == 0;       // the FP64 kernel has no tensor-core tiles
    if (lay != 0 && c->refine != 1) return false;    // capped layouts: one refinement sweep only
    if (c->prec == PORO_BF16X3_REFINE) return cta == 0;  // bf16 sweeps: default CTA size only
    return true;
}

static void apply_tile_choice(poro_ctx* c, int choice) {
    c->variant = choice / 6;
    c->mref.cap_a = kTileCaps[choice % 6][0];
    c->mref.cap_b = kTileCaps[choice % 6][1];
}

poro_status poro_set_tiles(poro_ctx* c, int32_t choice) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_tiles: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT) return fail(c, PORO_EUNSUPPORTED, "poro_set_tiles: Biot contexts only");
    if (!tile_choice_valid(c, choice)) return fail(c, PORO_EINVAL, "poro_set_tiles: choice not available here");
    apply_tile_choice(c, choice);
    return PORO_OK;
}

poro_status poro_autotune_tiles(poro_ctx* c, int64_t sample, int32_t* choice_out, double* ms_out) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_autotune_tiles: ctx is NULL");
    if (c->system != PORO_SYSTEM_BIOT || c->subcell)
        return fail(c, PORO_EUNSUPPORTED, "poro_autotune_tiles: Biot constant-material contexts only");
    if (!c->d_econst || c->n_elem <= 0) return fail(c, PORO_ESTATE, "poro_autotune_tiles: no element population loaded");
    cudaSetDevice(c->device);
    const int64_t n = std::max<int64_t>(1, std::min(sample > 0 ? sample : c->n_elem, c->n_elem));
    const int saved_v = c->variant, saved_a = c->mref.cap_a, saved_b = c->mref.cap_b;
    auto restore = [&] {
        c->variant = saved_v;
        c->mref.cap_a = saved_a;
        c->mref.cap_b = saved_b;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, cudaErrorMemoryAllocation, "poro_autotune_tiles: events");
    }
    double best = 1e300;
    int bestc = 0;
    poro_status st = PORO_OK;
    for (int choice = 0; choice < PORO_TILE_CHOICES && st == PORO_OK; ++choice) {
        if (ms_out) ms_out[choice] = -1.0;
        if (!tile_choice_valid(c, choice)) continue;
        apply_tile_choice(c, choice);
        for (int w = 0; w < 2 && st == PORO_OK; ++w)
            st = dispatch_predict(c, 0, n, c->d_q0, c->d_qt, c->d_iout, PORO_SOLVE_BLOCK, c->stream);
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && st == PORO_OK; ++r)
            st = dispatch_predict(c, 0, n, c->d_q0, c->d_qt, c->d_iout, PORO_SOLVE_BLOCK, c->stream);
        cudaEventRecord(e1, c->stream);
        const cudaError_t er = cudaEventSynchronize(e1);
        if (st == PORO_OK && er != cudaSuccess) st = cuda_fail(c, er, "poro_autotune_tiles");
        if (st == PORO_OK) st = device_status(c, "poro_autotune_tiles");
        float ms = 0.f;
        if (st == PORO_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (st == PORO_OK && ms_out) ms_out[choice] = ms / 3.0;
        if (st == PORO_OK && ms < best) {
            best = ms;
            bestc = choice;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    restore();
    if (st != PORO_OK) return st;
    apply_tile_choice(c, bestc);
    if (choice_out) *choice_out = bestc;
    return PORO_OK;
}

poro_status poro_set_variant(poro_ctx* c, int32_t variant) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_variant: ctx is NULL");
    if (variant < 0 || variant > 1) return fail(c, PORO_EINVAL, "poro_set_variant: variant must be 0 or 1");
    c->variant = variant;
    return PORO_OK;
}

}  // extern "C"
