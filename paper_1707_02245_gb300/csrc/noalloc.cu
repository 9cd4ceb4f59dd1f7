// pat_adjoint_noalloc: K^T y for callers that must not allocate device memory during
// the call.  Its scratch (one max word and the fixed-point K^T image) lives in a
// file-scope device array that every GPU loading this library holds until exit.
#include <mutex>

#include "pat_internal.cuh"

namespace pat {

constexpr int kNoAllocMaxN = 1024;                       // largest image side served
constexpr size_t kNoAllocHeadInts = 64;                  // 256 bytes: the max word
constexpr size_t kNoAllocInts = kNoAllocHeadInts + (size_t)kNoAllocMaxN * kNoAllocMaxN;

// 4 MiB + 256 B per device.  Host code must not use this name as an address: it is a
// host-side stand-in for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocInts];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mtx;
static int* g_noalloc_ptr[kMaxDevices];   // device address of the scratch, per device

// Looks the scratch address up once per device, with that device current.
static int noalloc_scratch(int device, int** out) {
    if (device < 0 || device >= kMaxDevices) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mtx);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "pat_adjoint_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[device] = (int*)p;
    }
    *out = g_noalloc_ptr[device];
    return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" int pat_adjoint_noalloc(const pat_geometry* g, const float* y_dev, float* u_dev, void* stream) {
    if (!g || !y_dev || !u_dev) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_noalloc: NULL argument");
    const int N = g->desc.n;
    if (N > kNoAllocMaxN)
        return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_noalloc: image side exceeds the 1024 the static scratch holds");
    int device = 0;
    PAT_CUDA(cudaGetDevice(&device));
    if (device != g->device)
        return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_noalloc: the geometry belongs to another device");
    {
        std::lock_guard<std::mutex> lock(g->mtx);
        if (!g->pc.ready)
            return fail(PAT_ERR_INVALID_ARG,
                        "pat_adjoint_noalloc: geometry not prepared; call pat_steps, pat_adjoint or "
                        "pat_reconstruct on it once while allocation is allowed");
    }
    int* scratch = nullptr;
    int rc = noalloc_scratch(device, &scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the scratch keeps the previous call's contents: clear the part this call uses
    PAT_CUDA(cudaMemsetAsync(scratch, 0, (kNoAllocHeadInts + (size_t)N * N) * sizeof(int), st));
    return launch_adjoint_into(g, y_dev, (unsigned*)scratch, scratch + kNoAllocHeadInts, u_dev, st);
}
