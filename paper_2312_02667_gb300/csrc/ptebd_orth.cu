// Orthonormal basis of the columns of X = Lambda_{b-1} Gamma_b Lambda_b for the
// trivial simple update (tSU, Sec. III D) of PtSU.
//
// The tSU SVD goes through theta = X Y (rank <= chi_b): an orthonormal basis Q
// of range(X) gives M = Q^dag theta with the singular values of theta, and its
// one-sided Jacobi (pass 2) gives V S of theta.  Any orthonormal basis of
// range(X) will do, so Q is built here by block classical Gram-Schmidt applied
// twice (BCGS2: the second pass restores orthogonality to working precision
// for cond(X) well below 1/u), blocks of NB columns, modified Gram-Schmidt
// inside a block.  Columns are taken in their stored order, that is by
// decreasing Lambda_b.  A column whose residual in the first pass falls below
// 32 u of its original length is numerically dependent on the ones before it
// and is dropped (set to zero, norm 0): its direction adds nothing to theta's
// row space.  norms[c] is 1 for a kept column and 0 for a dropped one, which
// is what the projection kernel divides by.
//
// One CTA per bond, one warp per column of a block.  The block being
// finished sits in shared memory; every later column is projected on it by
// one warp on its own (all NB coefficients from the column as it stands, then
// one update), so the warps need no hand-off between them.
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "ptebd_internal.h"

namespace ptebd {
namespace {

template <typename R> struct OrthNB;
template <> struct OrthNB<float> { static constexpr int v = 16; };
template <> struct OrthNB<double> { static constexpr int v = 8; };

template <typename R> struct OrthU;
template <> struct OrthU<float> { static constexpr double u = 5.9604644775390625e-08; };
template <> struct OrthU<double> { static constexpr double u = 1.1102230246251565e-16; };

template <typename R>
__device__ __forceinline__ R osum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Column entries of a lane: entry q is row 32 q + lane.
template <typename C, int RPL>
__device__ __forceinline__ void gload(C (&v)[RPL], const C* col, int lane, int rows, bool valid) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int r = 32 * q + lane;
        v[q] = (valid && r < rows) ? col[r] : cmake<C>(0, 0);
    }
}
template <typename C, int RPL>
__device__ __forceinline__ void gstore(const C (&v)[RPL], C* col, int lane, int rows) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int r = 32 * q + lane;
        if (r < rows) col[r] = v[q];
    }
}

template <typename R, int RPL>
__device__ __forceinline__ R norm2(const cx_t<R> (&v)[RPL]) {
    R s0 = 0, s1 = 0;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        s0 = fma(v[q].x, v[q].x, s0);
        s1 = fma(v[q].y, v[q].y, s1);
    }
    return osum(s0 + s1);
}

// c = q^dag v (q read from shared memory)
template <typename R, int RPL>
__device__ __forceinline__ cx_t<R> cdot(const cx_t<R>* q, const cx_t<R> (&v)[RPL], int lane) {
    R r0 = 0, r1 = 0, i0 = 0, i1 = 0;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        const cx_t<R> x = q[32 * k + lane];
        if (k & 1) {
            r1 = fma(x.x, v[k].x, r1); r1 = fma(x.y, v[k].y, r1);
            i1 = fma(x.x, v[k].y, i1); i1 = fma(-x.y, v[k].x, i1);
        } else {
            r0 = fma(x.x, v[k].x, r0); r0 = fma(x.y, v[k].y, r0);
            i0 = fma(x.x, v[k].y, i0); i0 = fma(-x.y, v[k].x, i0);
        }
    }
    return cmake<cx_t<R>>(osum(r0 + r1), osum(i0 + i1));
}

// v -= q c
template <typename R, int RPL>
__device__ __forceinline__ void caxpy_sub(cx_t<R> (&v)[RPL], const cx_t<R>* q, cx_t<R> c, int lane) {
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        const cx_t<R> x = q[32 * k + lane];
        v[k].x = fma(-x.x, c.x, v[k].x); v[k].x = fma(x.y, c.y, v[k].x);
        v[k].y = fma(-x.x, c.y, v[k].y); v[k].y = fma(-x.y, c.x, v[k].y);
    }
}

template <typename R, int NB, int RPL>
__device__ void orth_body(const LayerArgs<R>& A, cx_t<R>* W, int rows, int cols, int j, unsigned char* smem) {
    using C = cx_t<R>;
    const int ldw = A.ldw;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    C* QI = reinterpret_cast<C*>(smem);                 // [NB][ldw]: the block being finished
    C* wcoef = QI + (size_t)NB * ldw;                        // [NB][NB]: each warp's coefficients
    R* onorm = reinterpret_cast<R*>(wcoef + NB * NB);         // [2 PTEBD_CHI_LIMIT]: original |col|^2
    const int nblk = (cols + NB - 1) / NB;
    const R keep2 = (R)((32.0 * OrthU<R>::u) * (32.0 * OrthU<R>::u));

    for (int c = warp; c < cols; c += NB) {
        C v[RPL];
        gload<C, RPL>(v, W + (size_t)c * ldw, lane, rows, true);
        const R n2 = norm2<R, RPL>(v);
        if (lane == 0) onorm[c] = n2;
    }
    __syncthreads();

    for (int pass = 0; pass < 2; ++pass) {
        for (int I = 0; I < nblk; ++I) {
            const int c0 = I * NB;
            const int mycol = c0 + warp;
            const bool mine = mycol < cols;
            C a[RPL];
            gload<C, RPL>(a, W + (size_t)mycol * ldw, lane, rows, mine);
            // modified Gram-Schmidt inside the block
            for (int k = 0; k < NB; ++k) {
                if (warp == k) {
                    if (mine) {
                        const R n2 = norm2<R, RPL>(a);
                        const bool keep = pass == 0 ? (n2 > keep2 * onorm[mycol]) : (n2 > (R)0.25);
                        const R f = keep ? (R)1 / sqrt(n2) : (R)0;
#pragma unroll
                        for (int q = 0; q < RPL; ++q) { a[q].x *= f; a[q].y *= f; }
                    }
#pragma unroll
                    for (int q = 0; q < RPL; ++q) QI[(size_t)k * ldw + 32 * q + lane] = a[q];
                }
                __syncthreads();
                if (warp > k && mine) caxpy_sub<R, RPL>(a, QI + (size_t)k * ldw, cdot<R, RPL>(QI + (size_t)k * ldw, a, lane), lane);
            }
            if (mine) gstore<C, RPL>(a, W + (size_t)mycol * ldw, lane, rows);
            // every later column against the finished block (classical Gram-Schmidt:
            // all coefficients from the column as it stands, then one update)
            C* coef = wcoef + warp * NB;
            for (int c = c0 + NB + warp; c < cols; c += NB) {
                C v[RPL];
                gload<C, RPL>(v, W + (size_t)c * ldw, lane, rows, true);
#pragma unroll 1
                for (int i = 0; i < NB; ++i) {
                    const C ci = cdot<R, RPL>(QI + (size_t)i * ldw, v, lane);
                    if (lane == 0) coef[i] = ci;
                }
                __syncwarp();
#pragma unroll 1
                for (int i = 0; i < NB; ++i) caxpy_sub<R, RPL>(v, QI + (size_t)i * ldw, coef[i], lane);
                __syncwarp();
                gstore<C, RPL>(v, W + (size_t)c * ldw, lane, rows);
            }
            __syncthreads();  // QI is reused by the next block; the columns are in global memory
        }
    }
    // norms for the projection: 1 for a kept column, 0 for a dropped one
    double* nrm = A.norms + (size_t)j * ldw;
    for (int c = warp; c < cols; c += NB) {
        C v[RPL];
        gload<C, RPL>(v, W + (size_t)c * ldw, lane, rows, true);
        const R n2 = norm2<R, RPL>(v);
        if (lane == 0) {
            if (!isfinite((double)n2)) atomicOr(A.err, DERR_NONFINITE);
            nrm[c] = n2 > (R)0.25 ? 1.0 : 0.0;
        }
    }
}

// Pass 1 of the tSU SVD on X (2 chi_{b-1} x chi_b, from k_xform in w).
template <typename R, int NB>
__global__ void __launch_bounds__(NB * 32, 1) k_orth(LayerArgs<R> A) {
    using C = cx_t<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int j = blockIdx.x;
    const int32_t* d = A.dims + j * kDims;
    if (A.refine == 1 && d[D_REFINE] != 1) return;  // the FP64 resolution runs only undecided bonds
    const int rows = 2 * d[D_CL];
    const int cols = d[D_CM];
    C* W = A.w + (size_t)j * A.ldw * A.ldw;
    const int qa = (rows + 31) / 32;
    if (qa <= 1) orth_body<R, NB, 1>(A, W, rows, cols, j, smem);
    else if (qa <= 2) orth_body<R, NB, 2>(A, W, rows, cols, j, smem);
    else if (qa <= 4) orth_body<R, NB, 4>(A, W, rows, cols, j, smem);
    else if (qa <= 8) orth_body<R, NB, 8>(A, W, rows, cols, j, smem);
    else orth_body<R, NB, 16>(A, W, rows, cols, j, smem);
}

size_t orth_smem_bytes(int precision, int ldw) {
    const bool f64 = precision == PTEBD_FP64;
    const int nb = f64 ? OrthNB<double>::v : OrthNB<float>::v;
    const size_t elem = f64 ? sizeof(double2) : sizeof(float2);
    const size_t real = f64 ? sizeof(double) : sizeof(float);
    return (size_t)nb * ldw * elem + (size_t)nb * nb * elem + (size_t)2 * PTEBD_CHI_LIMIT * real;
}

}  // namespace

template <typename R> cudaError_t orth_prepare() {
    constexpr int NB = OrthNB<R>::v;
    const int prec = std::is_same<R, double>::value ? PTEBD_FP64 : PTEBD_MIXED;
    return cudaFuncSetAttribute(k_orth<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)orth_smem_bytes(prec, 2 * PTEBD_CHI_LIMIT));
}

template <typename R> cudaError_t launch_orth(const LayerArgs<R>& a, cudaStream_t s) {
    constexpr int NB = OrthNB<R>::v;
    const int prec = std::is_same<R, double>::value ? PTEBD_FP64 : PTEBD_MIXED;
    k_orth<R, NB><<<a.count, NB * 32, orth_smem_bytes(prec, a.ldw), s>>>(a);
    return cudaGetLastError();
}

template cudaError_t orth_prepare<float>();
template cudaError_t orth_prepare<double>();
template cudaError_t launch_orth<float>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_orth<double>(const LayerArgs<double>&, cudaStream_t);

}  // namespace ptebd
