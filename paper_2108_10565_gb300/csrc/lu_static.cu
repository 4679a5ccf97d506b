// Allocation-free form of the dense-LU predictor (poro_lu_predict_static).
//
// Some callers cannot call cudaMalloc: code that runs on a fixed device-memory
// budget handed out by an outer framework's allocator, or loops that must not
// take the implicit device synchronisation that cudaMalloc / cudaFree may
// perform.  poro_lu_factor allocates its factor buffer on every call, so such
// callers cannot use it.  This entry point runs the same assembly,
// equilibration, factorisation and triangular-solve kernels, but keeps the
// factors in a file-scope device array of fixed size that is part of the
// loaded library: every GPU that loads libporoader holds these 64 MiB until
// the process exits.  The call itself allocates nothing.
//
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made for that device.  The address is cached for the life of the
// process: a cudaDeviceReset (or any teardown of the device's primary
// context) reloads the module, possibly elsewhere, so the library must not be
// used across a reset of a device it has run on.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "poro_internal.h"

namespace poro {
namespace {

constexpr size_t kStaticLuBytes = size_t(64) << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_lu_static[kStaticLuBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_dev_ptr[kMaxDevices] = {};

// device address of g_lu_static on `device` (which must be current)
cudaError_t static_scratch(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_dev_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_lu_static);
        if (e != cudaSuccess) return e;
        g_dev_ptr[device] = p;
    }
    *out = g_dev_ptr[device];
    return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace poro

extern "C" poro_status poro_lu_predict_static(poro_ctx* ctx, int64_t first, int64_t count, const double* q0,
                                              double* qt, double* iout, void* stream) {
    using namespace poro;
    CtxView v;
    if (!ctx) {
        ctx_set_error(nullptr, "poro_lu_predict_static: ctx is NULL");
        return PORO_EINVAL;
    }
    if (!ctx_view(ctx, v)) {
        ctx_set_error(ctx, "poro_lu_predict_static: no element population loaded");
        return PORO_ESTATE;
    }
    if (first < 0 || count < 0 || first + count > v.n_elem) {
        ctx_set_error(ctx, "poro_lu_predict_static: element range outside the population");
        return PORO_EINVAL;
    }
    if (count > 0 && !q0) {
        ctx_set_error(ctx, "poro_lu_predict_static: Q0 is NULL");
        return PORO_EINVAL;
    }
    if (((uintptr_t)q0 | (uintptr_t)qt | (uintptr_t)iout) & 15) {
        ctx_set_error(ctx, "poro_lu_predict_static: buffers must be 16-byte aligned");
        return PORO_EINVAL;
    }
    const size_t s = (size_t)NQ * n_modes(v.N) * (v.N + 1);
    const size_t bA = align256((size_t)count * s * s * sizeof(double));
    const size_t bI = align256((size_t)count * s * sizeof(int32_t));
    const size_t bD = align256((size_t)count * s * sizeof(double));
    const size_t need = bA + 2 * bI + 2 * bD + 256;
    if (need > kStaticLuBytes) {
        ctx_set_error(ctx, "poro_lu_predict_static: " + std::to_string(count) + " elements of degree " +
                               std::to_string(v.N) + " need " + std::to_string(need) +
                               " bytes of factors; the static buffer holds " + std::to_string(kStaticLuBytes) +
                               " bytes (use poro_lu_factor for larger batches)");
        return PORO_EINVAL;
    }
    if (count == 0) return PORO_OK;
    // a launch error reported below must be this call's, not one left over by
    // an earlier unrelated call; and the caller's current device is restored
    (void)cudaGetLastError();
    int caller_device = -1;
    cudaError_t e = cudaGetDevice(&caller_device);
    if (e == cudaSuccess) e = cudaSetDevice(v.device);
    void* base = nullptr;
    if (e == cudaSuccess) e = static_scratch(v.device, &base);
    if (e != cudaSuccess) {
        if (caller_device >= 0) cudaSetDevice(caller_device);
        ctx_set_error(ctx, std::string("poro_lu_predict_static: ") + cudaGetErrorString(e));
        return PORO_ECUDA;
    }
    unsigned char* p = static_cast<unsigned char*>(base);
    LUScratch w;
    w.A = reinterpret_cast<double*>(p);
    w.piv = reinterpret_cast<int32_t*>(p + bA);
    w.perm = reinterpret_cast<int32_t*>(p + bA + bI);
    w.R = reinterpret_cast<double*>(p + bA + 2 * bI);
    w.C = reinterpret_cast<double*>(p + bA + 2 * bI + bD);
    w.bad = reinterpret_cast<int32_t*>(p + bA + 2 * bI + 2 * bD);
    void* st = stream ? stream : v.stream;
    // launch_lu_factor zeroes the factor area and the zero-pivot flag first
    int rc = launch_lu_factor(*v.lref, count, v.econst + first * v.stride, w, st);
    if (rc == 0) rc = launch_lu_solve(*v.lref, count, w, 0, q0, v.econst + first * v.stride, qt, iout, st);
    cudaSetDevice(caller_device);
    if (rc != 0) {
        ctx_set_error(ctx, std::string("poro_lu_predict_static: ") + cudaGetErrorString((cudaError_t)rc));
        return PORO_ECUDA;
    }
    return PORO_OK;
}
