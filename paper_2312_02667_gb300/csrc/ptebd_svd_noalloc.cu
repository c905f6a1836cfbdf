// Allocation-free variant of ptebd_svd_batched.
//
// Some callers cannot allocate device memory at all: code that runs while a
// host framework owns every device allocation (plugins handed only their input
// and output buffers), or code that must not call cudaMalloc / cudaFree because
// those calls synchronise the device or are forbidden in its context.  This
// entry point runs the same batched Jacobi SVD as ptebd_svd_batched but keeps
// its scratch (the working copy of the matrices, column norms, dims, counters,
// error word) in one file-scope device array of fixed size, so the caller
// passes only the inputs and the outputs.
//
// The array is a static __device__ object: every GPU that loads the library
// holds PTEBD_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code
// cannot use the array's name as a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture.
// All calls share the array and it keeps the previous call's contents: the
// counters and error word are cleared on every call, everything else is
// overwritten before it is read.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include <mutex>

#include "ptebd_internal.h"

namespace ptebd {
size_t svd_workspace_bytes(int precision, int batch, int rows);
int svd_batched_impl(int32_t precision, int32_t batch, int32_t rows, int32_t cols, const void* a, int32_t lda,
                     double* sigma, void* u, int32_t ldu, void* workspace, size_t workspace_bytes, void* stream,
                     int32_t check);
}  // namespace ptebd

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PTEBD_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PTEBD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PTEBD_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PTEBD_OK;
}

}  // namespace

extern "C" int ptebd_svd_batched_noalloc(int32_t precision, int32_t batch, int32_t rows, int32_t cols,
                                         const void* a, int32_t lda, double* sigma, void* u, int32_t ldu,
                                         void* stream, int32_t check) {
    size_t need = 0;
    int rc = ptebd_svd_workspace_bytes(precision, batch, rows, cols, &need);
    if (rc) return rc;
    if (need > (size_t)PTEBD_NOALLOC_SCRATCH_BYTES) return PTEBD_ERR_MEMORY;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    return ptebd::svd_batched_impl(precision, batch, rows, cols, a, lda, sigma, u, ldu, scratch,
                                   (size_t)PTEBD_NOALLOC_SCRATCH_BYTES, stream, check);
}
