// Full contractions of an MPS (norm, overlap, expectation values) by
// left-to-right transfer matrices E <- sum_s M_a[s]^dag E M_b[s], M = Gamma Lambda
// (the MPS decomposition of Sec. II A-B of arXiv:2312.02667), with every
// product accumulated in FP64.  Building blocks:
//   k_zgemm       : C = alpha * rowscale o (op(A) * (B o colscale)) + beta * C,
//                   column-major, complex64/complex128 inputs, complex128 output;
//   k_scale_max   : divide E by its largest modulus and add the log to an
//                   accumulator, so that long chains neither under- nor overflow;
//   k_fill_identity.
#include <cmath>

#include "ptebd_internal.h"

namespace ptebd {

namespace {

__device__ __forceinline__ double2 ld2(const float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 ld2(const double2 v) { return v; }

// grid (ceil(m/32), ceil(n/32)), 256 threads, 2x2 outputs per thread.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_zgemm(int m, int n, int k, double2 alpha, const TA* __restrict__ A,
                                               int lda, int opA, const TB* __restrict__ B, int ldb,
                                               const double* __restrict__ colscale, double2 beta,
                                               double2* __restrict__ Cm, int ldc, const double* __restrict__ rowscale) {
    __shared__ double2 as[16][33];  // [kk][i]
    __shared__ double2 bs[16][33];  // [kk][j]
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double2 acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[i][q] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < k; k0 += 16) {
        for (int e = threadIdx.x; e < 512; e += 256) {
            int kk, ii;
            if (opA) { kk = e & 15; ii = e >> 4; } else { ii = e & 31; kk = e >> 5; }
            const int gi = i0 + ii, gk = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (gi < m && gk < k) {
                if (opA) { v = ld2(A[(size_t)gi * lda + gk]); v.y = -v.y; }
                else v = ld2(A[(size_t)gk * lda + gi]);
            }
            as[kk][ii] = v;
        }
        for (int e = threadIdx.x; e < 512; e += 256) {
            const int kk = e & 15, jj = e >> 4;
            const int gj = j0 + jj, gk = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (gj < n && gk < k) {
                v = ld2(B[(size_t)gj * ldb + gk]);
                if (colscale) { v.x *= colscale[gj]; v.y *= colscale[gj]; }
            }
            bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const double2 x = as[kk][tx + 16 * i];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const double2 y = bs[kk][ty + 16 * q];
                    acc[i][q].x = fma(x.x, y.x, acc[i][q].x); acc[i][q].x = fma(-x.y, y.y, acc[i][q].x);
                    acc[i][q].y = fma(x.x, y.y, acc[i][q].y); acc[i][q].y = fma(x.y, y.x, acc[i][q].y);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gi = i0 + tx + 16 * i, gj = j0 + ty + 16 * q;
            if (gi >= m || gj >= n) continue;
            double2 p = acc[i][q];
            if (rowscale) { p.x *= rowscale[gi]; p.y *= rowscale[gi]; }
            double2 r = make_double2(alpha.x * p.x - alpha.y * p.y, alpha.x * p.y + alpha.y * p.x);
            double2* c = Cm + (size_t)gj * ldc + gi;
            if (beta.x != 0.0 || beta.y != 0.0) {
                const double2 o = *c;
                r.x += beta.x * o.x - beta.y * o.y;
                r.y += beta.x * o.y + beta.y * o.x;
            }
            *c = r;
        }
}

__global__ void __launch_bounds__(256) k_scale_max(double2* E, int rows, int cols, int ld, double* log_acc) {
    __shared__ double red[256];
    double mx = 0.0;
    for (int e = threadIdx.x; e < rows * cols; e += 256) {
        const double2 v = E[(size_t)(e / rows) * ld + (e % rows)];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    const double m = red[0];
    if (!(m > 0.0) || !isfinite(m)) return;  // a zero or broken chain stays as it is
    const double inv = 1.0 / m;
    for (int e = threadIdx.x; e < rows * cols; e += 256) {
        double2* p = E + (size_t)(e / rows) * ld + (e % rows);
        p->x *= inv; p->y *= inv;
    }
    if (threadIdx.x == 0) *log_acc += log(m);
}

__global__ void k_fill_identity(double2* E, int rows, int cols, int ld) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
        const int r = e % rows, c = e / rows;
        E[(size_t)c * ld + r] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
}

// One sampling step at `site` (sites are drawn from the right end), one CTA per
// sample: t_x = M_site[x] v (x = 0, 1; M = Gamma diag(Lambda_site)),
// w_x = t_x^dag L t_x with L the left environment of the site, sigma = 0 when
// u < w_0 / (w_0 + w_1); v <- t_sigma / |t_sigma|.
// v_in: samples x chip (chir valid entries; nullptr = the unit vector (1) of the
// right boundary), v_out: samples x chip (chil valid).
template <typename TG>
__global__ void __launch_bounds__(256) k_sample_site(const TG* __restrict__ gamma_s, const double* __restrict__ lam,
                                                     int chil, int chir, int chip, const double2* __restrict__ L,
                                                     const double2* __restrict__ v_in, double2* __restrict__ v_out,
                                                     const double* __restrict__ uniforms, int site, int n_sites,
                                                     int32_t* __restrict__ bits) {
    __shared__ double2 vs[512];
    __shared__ double2 ts[2][512];
    __shared__ double red[3][256];
    __shared__ int choice;
    const int k = blockIdx.x, t = threadIdx.x;
    const size_t slice = (size_t)chip * chip;
    for (int b = t; b < chir; b += 256) {
        double2 x = v_in ? v_in[(size_t)k * chip + b] : make_double2(b == 0 ? 1.0 : 0.0, 0.0);
        x.x *= lam[b]; x.y *= lam[b];
        vs[b] = x;
    }
    __syncthreads();
    for (int a = t; a < chil; a += 256) {
        double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
        for (int b = 0; b < chir; ++b) {
            const double2 g0 = ld2(gamma_s[(size_t)b * chip + a]);
            const double2 g1 = ld2(gamma_s[slice + (size_t)b * chip + a]);
            const double2 x = vs[b];
            s0.x += g0.x * x.x - g0.y * x.y; s0.y += g0.x * x.y + g0.y * x.x;
            s1.x += g1.x * x.x - g1.y * x.y; s1.y += g1.x * x.y + g1.y * x.x;
        }
        ts[0][a] = s0;
        ts[1][a] = s1;
    }
    __syncthreads();
    // w_x = sum_a conj(t_x[a]) (L t_x)[a]; |t_x|^2 alongside
    double w0 = 0.0, w1 = 0.0;
    for (int a = t; a < chil; a += 256) {
        double2 u0 = make_double2(0, 0), u1 = make_double2(0, 0);
        for (int c = 0; c < chil; ++c) {
            const double2 l = L[(size_t)c * chip + a];
            const double2 x0 = ts[0][c], x1 = ts[1][c];
            u0.x += l.x * x0.x - l.y * x0.y; u0.y += l.x * x0.y + l.y * x0.x;
            u1.x += l.x * x1.x - l.y * x1.y; u1.y += l.x * x1.y + l.y * x1.x;
        }
        w0 += ts[0][a].x * u0.x + ts[0][a].y * u0.y;
        w1 += ts[1][a].x * u1.x + ts[1][a].y * u1.y;
    }
    red[0][t] = w0;
    red[1][t] = w1;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (t < st) { red[0][t] += red[0][t + st]; red[1][t] += red[1][t + st]; }
        __syncthreads();
    }
    if (t == 0) {
        const double p0 = red[0][0] / (red[0][0] + red[1][0]);
        choice = uniforms[(size_t)k * n_sites + site] < p0 ? 0 : 1;
        bits[(size_t)k * n_sites + site] = choice;
    }
    __syncthreads();
    const int x = choice;
    double nn = 0.0;
    for (int a = t; a < chil; a += 256) nn += ts[x][a].x * ts[x][a].x + ts[x][a].y * ts[x][a].y;
    red[2][t] = nn;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (t < st) red[2][t] += red[2][t + st];
        __syncthreads();
    }
    const double inv = red[2][0] > 0.0 ? 1.0 / sqrt(red[2][0]) : 0.0;
    for (int a = t; a < chil; a += 256) {
        double2 y = ts[x][a];
        y.x *= inv; y.y *= inv;
        v_out[(size_t)k * chip + a] = y;
    }
}

}  // namespace

template <typename TG>
cudaError_t launch_sample_site(const TG* gamma_s, const double* lam, int chil, int chir, int chip, const double2* L,
                               const double2* v_in, double2* v_out, const double* uniforms, int site, int n_sites,
                               int32_t* bits, int n_samples, cudaStream_t s) {
    k_sample_site<TG><<<n_samples, 256, 0, s>>>(gamma_s, lam, chil, chir, chip, L, v_in, v_out, uniforms, site,
                                                n_sites, bits);
    return cudaGetLastError();
}
template cudaError_t launch_sample_site<float2>(const float2*, const double*, int, int, int, const double2*,
                                                const double2*, double2*, const double*, int, int, int32_t*, int,
                                                cudaStream_t);
template cudaError_t launch_sample_site<double2>(const double2*, const double*, int, int, int, const double2*,
                                                 const double2*, double2*, const double*, int, int, int32_t*, int,
                                                 cudaStream_t);

template <typename TA, typename TB>
cudaError_t launch_zgemm(int m, int n, int k, double2 alpha, const TA* A, int lda, int opA, const TB* B, int ldb,
                         const double* colscale_b, double2 beta, double2* Cm, int ldc, const double* rowscale_c,
                         cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((m + 31) / 32, (n + 31) / 32);
    k_zgemm<TA, TB><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, opA, B, ldb, colscale_b, beta, Cm, ldc,
                                         rowscale_c);
    return cudaGetLastError();
}

cudaError_t launch_scale_max(double2* E, int rows, int cols, int ld, double* log_acc, cudaStream_t s) {
    k_scale_max<<<1, 256, 0, s>>>(E, rows, cols, ld, log_acc);
    return cudaGetLastError();
}

cudaError_t launch_fill_identity(double2* E, int rows, int cols, int ld, cudaStream_t s) {
    k_fill_identity<<<64, 256, 0, s>>>(E, rows, cols, ld);
    return cudaGetLastError();
}

#define PTEBD_ZGEMM(TA, TB)                                                                                  \
    template cudaError_t launch_zgemm<TA, TB>(int, int, int, double2, const TA*, int, int, const TB*, int, \
                                              const double*, double2, double2*, int, const double*, cudaStream_t);
PTEBD_ZGEMM(double2, double2)
PTEBD_ZGEMM(double2, float2)
PTEBD_ZGEMM(float2, double2)
PTEBD_ZGEMM(float2, float2)
#undef PTEBD_ZGEMM

}  // namespace ptebd
