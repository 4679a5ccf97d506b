// C ABI of libporoader (declared in include/poroader.h).  Argument checks,
// context state, device memory and the dispatch to the kernels.  No compute
// on the host beyond the per-element set-up of constants.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "poro_internal.h"

using poro::NQ;

struct poro_ctx {
    int device = 0;
    int N = 0, B = 0, T = 0;
    poro_precision prec = PORO_FP64;
    cudaStream_t stream = nullptr;
    poro::ReferenceData ref;
    poro::DeviceReference dref;
    poro::MixedReference mref;
    poro::LUReference lref;
    poro::LUScratch lu;
    int64_t lu_first = 0, lu_count = 0;
    int refine = 1;
    int64_t n_elem = 0;
    int stride = 0;
    double* d_econst = nullptr;
    double* d_q0 = nullptr;
    double* d_qt = nullptr;
    double* d_iout = nullptr;
    bool have_dofs = false, have_pred = false;
    std::string err;
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

void free_population(poro_ctx* c) {
    free_lu(c);
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
    c->lu_first = c->lu_count = 0;
}

void free_reference(poro_ctx* c) {
    dfree(c->lref.z);
    dfree(c->lref.krow);
    dfree(c->lref.kcol);
    dfree(c->lref.kval);
    dfree(c->mref.khat_val_f32);
    dfree(c->mref.res_row);
    dfree(c->mref.res_col);
    dfree(c->mref.res_val);
    dfree(c->mref.zinv_f32);
    dfree(c->dref.khat_val);
    dfree(c->dref.khat_col);
    dfree(c->dref.khat_row);
    dfree(c->dref.zinv);
}

}  // namespace

namespace poro {
bool ctx_view(const poro_ctx* c, CtxView& v) {
    if (!c || !c->d_econst) return false;
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

poro_status poro_create(int device, int degree_N, poro_precision precision, poro_ctx** out) {
    if (!out) return fail(nullptr, PORO_EINVAL, "poro_create: out is NULL");
    *out = nullptr;
    if (degree_N < 1 || degree_N > poro::MAX_N)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_create: degree N must be in 1..6");
    if (precision != PORO_FP64 && precision != PORO_FP32_REFINE)
        return fail(nullptr, PORO_EUNSUPPORTED, "poro_create: precision not built");
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
    std::string err;
    if (!poro::reference_data(degree_N, c->ref, err)) {
        delete c;
        return fail(nullptr, PORO_EINVAL, "poro_create: " + err);
    }
    c->B = c->ref.B;
    c->T = c->ref.T;
    c->stride = poro::elem_const_stride(degree_N);
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
    if ((e = upload((void**)&c->dref.khat_val, val.data(), val.size() * sizeof(double))) != cudaSuccess ||
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
    if (precision == PORO_FP32_REFINE) {
        // binary32 copies for the sweeps and the (hi, lo) full-row CSR of the residual
        const int B = c->B, T = c->T;
        std::vector<float> vf(val.begin(), val.end()), zf(c->ref.zinv.begin(), c->ref.zinv.end());
        std::vector<int32_t> rrow, rcol;
        std::vector<float> rval;
        for (int j = 0; j < 3; ++j) {
            rrow.push_back((int32_t)rcol.size());
            for (int l = 0; l < B; ++l) {
                for (int m = 0; m < B; ++m) {
                    const double v = c->ref.khat[((size_t)j * B + l) * B + m];
                    if (v != 0.0) {
                        const float h = (float)v;
                        rcol.push_back(m);
                        rval.push_back(h);
                        rval.push_back((float)(v - (double)h));
                    }
                }
                rrow.push_back((int32_t)rcol.size());
            }
        }
        (void)T;
        c->mref.base = &c->dref;
        if ((e = upload((void**)&c->mref.khat_val_f32, vf.data(), vf.size() * sizeof(float))) != cudaSuccess ||
            (e = upload((void**)&c->mref.res_row, rrow.data(), rrow.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->mref.res_col, rcol.data(), rcol.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload((void**)&c->mref.res_val, rval.data(), rval.size() * sizeof(float))) != cudaSuccess ||
            (e = upload((void**)&c->mref.zinv_f32, zf.data(), zf.size() * sizeof(float))) != cudaSuccess) {
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
    if (c->prec != PORO_FP32_REFINE) return fail(c, PORO_EUNSUPPORTED, "poro_set_refinement: context is not mixed precision");
    if (sweeps < 0 || sweeps > 2) return fail(c, PORO_EINVAL, "poro_set_refinement: sweeps must be 0, 1 or 2");
    c->refine = sweeps;
    return PORO_OK;
}

poro_status poro_destroy(poro_ctx* c) {
    if (!c) return PORO_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_population(c);
    free_reference(c);
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

poro_status poro_set_isolated(poro_ctx* c, int64_t n, const double* vert, const poro_material* mat,
                              const double* dt) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_isolated: ctx is NULL");
    if (n < 0 || (n > 0 && (!vert || !mat || !dt))) return fail(c, PORO_EINVAL, "poro_set_isolated: bad argument");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_population(c);
    std::vector<double> ec((size_t)n * c->stride);
    for (int64_t i = 0; i < n; ++i) {
        std::string err;
        if (!poro::element_constants(c->ref, vert + 12 * i, mat[i], dt[i], ec.data() + (size_t)i * c->stride, err))
            return fail(c, PORO_EINVAL, "poro_set_isolated: element " + std::to_string(i) + ": " + err);
    }
    const size_t nd = (size_t)n * NQ * c->B;
    cudaError_t e;
    if ((e = upload((void**)&c->d_econst, ec.data(), ec.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->d_q0, nd * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->d_qt, nd * c->T * sizeof(double) + 16)) != cudaSuccess ||
        (e = cudaMalloc((void**)&c->d_iout, nd * sizeof(double) + 16)) != cudaSuccess) {
        free_population(c);
        return e == cudaErrorMemoryAllocation ? fail(c, PORO_ENOMEM, "poro_set_isolated: out of device memory")
                                              : cuda_fail(c, e, "poro_set_isolated");
    }
    c->n_elem = n;
    return PORO_OK;
}

poro_status poro_set_dofs(poro_ctx* c, const double* Q) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_set_dofs: ctx is NULL");
    if (!c->d_econst) return fail(c, PORO_ESTATE, "poro_set_dofs: no element population loaded");
    if (c->n_elem > 0 && !Q) return fail(c, PORO_EINVAL, "poro_set_dofs: Q is NULL");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(c->d_q0, Q, (size_t)c->n_elem * NQ * c->B * sizeof(double),
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
        if (count > 0 && (first < c->lu_first || first + count > c->lu_first + c->lu_count))
            return fail(c, PORO_ESTATE, "predict (LU): elements not factored; call poro_lu_factor first");
        rc = poro::launch_lu_solve(c->lref, count, c->lu, first - c->lu_first, q0, ec, qt, iout, st);
        if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "predict (LU): kernel launch");
        return PORO_OK;
    }
    if (solver != PORO_SOLVE_BLOCK) return fail(c, PORO_EINVAL, "predict: unknown solver");
    if (c->prec == PORO_FP64) {
        rc = poro::launch_stp_fp64(c->dref, count, q0, ec, qt, iout, st);
    } else {
        rc = poro::launch_stp_mixed(c->mref, c->refine, count, q0, ec, qt, iout, st);
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

poro_status poro_lu_bytes(int degree_N, int64_t count, size_t* bytes) {
    if (degree_N < 1 || degree_N > poro::MAX_N) return fail(nullptr, PORO_EUNSUPPORTED, "poro_lu_bytes: degree");
    if (count < 0 || !bytes) return fail(nullptr, PORO_EINVAL, "poro_lu_bytes: bad argument");
    *bytes = poro::lu_scratch_bytes(degree_N, count);
    return PORO_OK;
}

poro_status poro_lu_factor(poro_ctx* c, int64_t first, int64_t count) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_lu_factor: ctx is NULL");
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
        (e = cudaMalloc((void**)&c->lu.bad, sizeof(int32_t))) != cudaSuccess) {
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

poro_status poro_sync(poro_ctx* c, int32_t timeout_ms) {
    if (!c) return fail(nullptr, PORO_EINVAL, "poro_sync: ctx is NULL");
    cudaSetDevice(c->device);
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return PORO_OK;
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
    return PORO_OK;
}

poro_status poro_get_predictor(poro_ctx* c, int64_t first, int64_t count, double* out) {
    return copy_out(c, c ? c->d_qt : nullptr, first, count, c ? (size_t)NQ * c->B * c->T : 0, out,
                    "poro_get_predictor");
}

poro_status poro_get_integrated(poro_ctx* c, int64_t first, int64_t count, double* out) {
    return copy_out(c, c ? c->d_iout : nullptr, first, count, c ? (size_t)NQ * c->B : 0, out,
                    "poro_get_integrated");
}

poro_status poro_flop_count(const poro_ctx* c, int32_t refine_sweeps, double* f) {
    if (!c || !f) return fail(nullptr, PORO_EINVAL, "poro_flop_count: NULL argument");
    const double B = c->B, T = c->T;
    // S3: 13 B rows of T x T time solves + the 3 G couplings per mode
    const double s3 = 2.0 * NQ * B * T * T + 2.0 * 3 * B * T;
    // S4a: 54-entry star products of all modes of degree >= 1, 3 directions
    const double s4a = 2.0 * 3 * poro::STAR_NNZ * (B - 1) * T;
    // S4b: structural non-zeros of the Khat blocks, each applied to 13 T columns
    const double s4b = 2.0 * (double)c->ref.khat_block_nnz * NQ * T;
    // S1 (scaling of Q0) and S5 (time integration)
    const double s15 = NQ * B * T + NQ * B;
    const double alg3 = s3 + s4a + s4b + s15;
    f[0] = alg3;
    f[1] = alg3 * (1 + refine_sweeps);
    // residual per sweep: diagonal time blocks, E* diagonal and coupling,
    // star products of all modes and the Khat products, in double-binary32
    f[2] = (2.0 * NQ * B * T * T + 2.0 * 6 * B * T + 2.0 * 3 * poro::STAR_NNZ * B * T + s4b) * refine_sweeps;
    return PORO_OK;
}

}  // extern "C"
