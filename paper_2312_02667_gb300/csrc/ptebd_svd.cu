// Batched SVD entry point: the layer's one-sided Jacobi SVD (the SVD step of
// the TEBD procedure, Sec. II C of arXiv:2312.02667) on caller matrices.
//   k_svd_load  : copy each input matrix into the workspace (the SVD rotates in place)
//   k_jacobi    : the layer's kernel (ptebd_jacobi.cu)
//   k_svd_store : sort the FP64 column norms, write the singular values in
//                 descending order and, when asked, the left singular vectors.
#include <algorithm>
#include <cstdio>

#include "ptebd_internal.h"

namespace ptebd {

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ldw_for(int rows) {
    int q = 1;
    while (32 * q < rows) q <<= 1;
    return 32 * q;
}

struct SvdWs {
    void* w; double* norms; int32_t* dims; int32_t* sweeps; unsigned long long* work; uint32_t* err;
    size_t bytes;
};

SvdWs svd_ws(char* base, int precision, int batch, int rows) {
    SvdWs v{};
    const size_t ldw = (size_t)ldw_for(rows), b = (size_t)batch;
    const size_t elem = precision == PTEBD_FP64 ? sizeof(double2) : sizeof(float2);
    size_t o = 0;
    v.w = base + o; o = align256(o + b * ldw * ldw * elem);
    v.norms = reinterpret_cast<double*>(base + o); o = align256(o + b * ldw * sizeof(double));
    v.dims = reinterpret_cast<int32_t*>(base + o); o = align256(o + b * kDims * sizeof(int32_t));
    v.sweeps = reinterpret_cast<int32_t*>(base + o); o = align256(o + b * sizeof(int32_t));
    v.work = reinterpret_cast<unsigned long long*>(base + o); o = align256(o + kWork * sizeof(unsigned long long));
    v.err = reinterpret_cast<uint32_t*>(base + o); o = align256(o + sizeof(uint32_t));
    v.bytes = o;
    return v;
}

// grid (ceil(rows*cols/256), batch)
template <typename R>
__global__ void __launch_bounds__(256) k_svd_load(const cx_t<R>* a, int lda, int rows, int cols, cx_t<R>* w,
                                                  int ldw, int32_t* dims) {
    const int j = blockIdx.y;
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e == 0) {
        int32_t* d = dims + j * kDims;
        d[D_CL] = 0; d[D_CM] = 0; d[D_CR] = 0; d[D_TALL] = 1; d[D_BOND] = 0; d[D_K] = 0;
        d[D_ROWS] = rows; d[D_COLS] = cols;
    }
    if (e >= (size_t)rows * cols) return;
    const int r = (int)(e % rows), c = (int)(e / rows);
    w[(size_t)j * ldw * ldw + (size_t)c * ldw + r] = a[(size_t)j * lda * cols + (size_t)c * lda + r];
}

// grid (batch), 512 threads
template <typename R>
__global__ void __launch_bounds__(512) k_svd_store(const cx_t<R>* w, int ldw, const double* norms, int rows,
                                                   int cols, double* sigma, cx_t<R>* u, int ldu) {
    using C = cx_t<R>;
    constexpr int NS = 512;
    __shared__ double key[NS];
    __shared__ int idx[NS];
    const int j = blockIdx.x, t = threadIdx.x;
    key[t] = t < cols ? norms[(size_t)j * ldw + t] : -1.0;
    idx[t] = t;
    __syncthreads();
    for (int size = 2; size <= NS; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int p = t ^ stride;
            if (p > t) {
                const bool desc = (t & size) == 0;
                const double kt = key[t], kp = key[p];
                const int it = idx[t], ip = idx[p];
                const bool t_first = (kt > kp) || (kt == kp && it < ip);
                if (desc ? !t_first : t_first) { key[t] = kp; key[p] = kt; idx[t] = ip; idx[p] = it; }
            }
            __syncthreads();
        }
    }
    if (t < cols) sigma[(size_t)j * cols + t] = key[t];
    if (u == nullptr) return;
    const C* W = w + (size_t)j * ldw * ldw;
    C* U = u + (size_t)j * ldu * cols;
    for (int c = 0; c < cols; ++c) {
        const double s = key[c];
        const R inv = s > 0.0 ? (R)(1.0 / s) : (R)0;
        const C* src = W + (size_t)idx[c] * ldw;
        for (int r = t; r < rows; r += NS) {
            C v = src[r];
            v.x *= inv; v.y *= inv;
            U[(size_t)c * ldu + r] = v;
        }
    }
}

template <typename R>
int run_svd(int batch, int rows, int cols, const void* a, int lda, double* sigma, void* u, int ldu, char* wsbase,
            cudaStream_t s, bool check) {
    using C = cx_t<R>;
    const int precision = std::is_same<R, double>::value ? PTEBD_FP64 : PTEBD_MIXED;
    SvdWs ws = svd_ws(wsbase, precision, batch, rows);
    const int ldw = ldw_for(rows);
    if (jacobi_prepare<R>() != cudaSuccess) return PTEBD_ERR_CUDA;
    if (cudaMemsetAsync(ws.work, 0, kWork * sizeof(unsigned long long), s) != cudaSuccess) return PTEBD_ERR_CUDA;
    if (cudaMemsetAsync(ws.err, 0, sizeof(uint32_t), s) != cudaSuccess) return PTEBD_ERR_CUDA;
    dim3 g1((unsigned)(((size_t)rows * cols + 255) / 256), batch);
    k_svd_load<R><<<g1, 256, 0, s>>>(static_cast<const C*>(a), lda, rows, cols, static_cast<C*>(ws.w), ldw,
                                      ws.dims);
    if (cudaGetLastError() != cudaSuccess) return PTEBD_ERR_CUDA;
    LayerArgs<R> la{};
    la.w = static_cast<C*>(ws.w);
    la.norms = ws.norms;
    la.dims = ws.dims;
    la.slot_sweeps = ws.sweeps;
    la.work = ws.work;
    la.err = ws.err;
    la.count = batch;
    la.ldw = ldw;
    la.chip = ldw / 2;
    la.max_sweeps = 40;
    la.pass = 0;
    if (launch_jacobi<R>(la, s) != cudaSuccess) return PTEBD_ERR_CUDA;
    k_svd_store<R><<<batch, 512, 0, s>>>(static_cast<const C*>(ws.w), ldw, ws.norms, rows, cols, sigma,
                                          static_cast<C*>(u), ldu);
    if (cudaGetLastError() != cudaSuccess) return PTEBD_ERR_CUDA;
    if (!check) return PTEBD_OK;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, ws.err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PTEBD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PTEBD_ERR_CUDA;
    if (err & DERR_TIMEOUT) return PTEBD_ERR_TIMEOUT;
    if (err & DERR_NONFINITE) return PTEBD_ERR_NUMERIC;
    if (err & DERR_NOT_CONVERGED) return PTEBD_ERR_NOT_CONVERGED;
    return PTEBD_OK;
}

int check_svd_args(int32_t precision, int32_t batch, int32_t rows, int32_t cols) {
    if (precision != PTEBD_FP64 && precision != PTEBD_MIXED) return PTEBD_ERR_INVALID;
    if (batch < 1 || rows < 1 || cols < 1 || cols > rows) return PTEBD_ERR_INVALID;
    if (rows > 2 * PTEBD_CHI_LIMIT) return PTEBD_ERR_UNSUPPORTED;
    if (rows % 2) return PTEBD_ERR_INVALID;  // TMA copies move whole 16-byte units of a column
    return PTEBD_OK;
}

}  // namespace

size_t svd_workspace_bytes(int precision, int batch, int rows) {
    return svd_ws(nullptr, precision, batch, rows).bytes;
}

int svd_batched_impl(int32_t precision, int32_t batch, int32_t rows, int32_t cols, const void* a, int32_t lda,
                     double* sigma, void* u, int32_t ldu, void* workspace, size_t workspace_bytes, void* stream,
                     int32_t check) {
    int rc = check_svd_args(precision, batch, rows, cols);
    if (rc) return rc;
    if (!a || !sigma || !workspace || lda < rows || (u && ldu < rows)) return PTEBD_ERR_INVALID;
    if ((uintptr_t)workspace & 255) return PTEBD_ERR_MEMORY;
    if (workspace_bytes < svd_workspace_bytes(precision, batch, rows)) return PTEBD_ERR_MEMORY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    return precision == PTEBD_FP64
               ? run_svd<double>(batch, rows, cols, a, lda, sigma, u, ldu, ws, s, check != 0)
               : run_svd<float>(batch, rows, cols, a, lda, sigma, u, ldu, ws, s, check != 0);
}

}  // namespace ptebd

extern "C" {

int ptebd_svd_workspace_bytes(int32_t precision, int32_t batch, int32_t rows, int32_t cols, size_t* bytes) {
    int rc = ptebd::check_svd_args(precision, batch, rows, cols);
    if (rc) return rc;
    if (!bytes) return PTEBD_ERR_INVALID;
    *bytes = ptebd::svd_workspace_bytes(precision, batch, rows);
    return PTEBD_OK;
}

int ptebd_svd_batched(int32_t precision, int32_t batch, int32_t rows, int32_t cols, const void* a, int32_t lda,
                      double* sigma, void* u, int32_t ldu, void* workspace, size_t workspace_bytes, void* stream,
                      int32_t check) {
    return ptebd::svd_batched_impl(precision, batch, rows, cols, a, lda, sigma, u, ldu, workspace, workspace_bytes,
                                   stream, check);
}

}  // extern "C"
