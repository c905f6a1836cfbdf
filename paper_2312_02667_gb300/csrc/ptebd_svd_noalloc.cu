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
// The array is a static __device__ object of this file's module.  The module
// is loaded on a device, and the array reserved there, on first use (the CUDA
// runtime loads modules lazily by default): the first call on each device may
// therefore fail with PTEBD_ERR_CUDA when the device is out of memory, and it
// should come before any stream capture.  From then on the device holds
// PTEBD_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Host code cannot use the array's name as a device address, so every call
// looks the address up with cudaGetSymbolAddress on the current device (cheap
// once the module is loaded; no cached pointer can outlive a context that the
// caller tore down and re-created) and checks that the stream belongs to that
// device.
// All calls share the array and it keeps the previous call's contents: the
// counters and error word are cleared on every call, everything else is
// overwritten before it is read.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include "ptebd_internal.h"

namespace ptebd {
size_t svd_workspace_bytes(int precision, int batch, int rows);
int svd_batched_impl(int32_t precision, int32_t batch, int32_t rows, int32_t cols, const void* a, int32_t lda,
                     double* sigma, void* u, int32_t ldu, void* workspace, size_t workspace_bytes, void* stream,
                     int32_t check);
}  // namespace ptebd

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PTEBD_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device, which must be
// the device of `stream`.
int scratch_address(void* stream, void** out) {
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PTEBD_ERR_CUDA;
    if (cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &sdev) != cudaSuccess) return PTEBD_ERR_CUDA;
    if (sdev != dev) return PTEBD_ERR_INVALID;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PTEBD_ERR_CUDA;
    *out = p;
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
    rc = scratch_address(stream, &scratch);
    if (rc) return rc;
    return ptebd::svd_batched_impl(precision, batch, rows, cols, a, lda, sigma, u, ldu, scratch,
                                   (size_t)PTEBD_NOALLOC_SCRATCH_BYTES, stream, check);
}
