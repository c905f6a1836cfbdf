// Kernels of one pTEBD gate layer apart from the SVD (arXiv:2312.02667):
//   k_theta    : two-site tensor theta = Lambda_{b-1} Gamma_b Lambda_b Gamma_{b+1} Lambda_{b+1}
//                and theta' = U theta (Sec. II C), batched over the bonds of a layer;
//   k_truncate : sort the singular values, keep chi' of them (projector P_b, Sec. III B),
//                eps_b, nu_b = (1 - eps_b)^(-1/2), Lambda_b <- nu_b S_kept / |S| (the
//                Schmidt spectrum of the normalised two-site wavefunction, Sec. II B,
//                III C; two other readings selectable), in FP64;
//   k_gamma_*  : Gamma_b <- Lambda_{b-1}^{-1} U and Gamma_{b+1} <- V^dagger Lambda_{b+1}^{-1}
//                (Sec. II C), one factor straight from the rotated columns, the other
//                through one complex GEMM with the kept theta';
//   k_reduce   : deterministic per-layer sums of eps_b and ln nu_b.
#include <cmath>
#include <type_traits>

#include "ptebd_internal.h"

namespace ptebd {

template <typename C> __device__ __forceinline__ C cz() { C c; c.x = 0; c.y = 0; return c; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// acc += x * y
template <typename C> __device__ __forceinline__ void cfma(C& acc, C x, C y) {
    acc.x = fma(x.x, y.x, acc.x); acc.x = fma(-x.y, y.y, acc.x);
    acc.y = fma(x.x, y.y, acc.y); acc.y = fma(x.y, y.x, acc.y);
}
// 1 / (a b) in the kernel's precision: FP32 arithmetic on the rounded factors
// for the complex64 path (the FP64 pipe is a small fraction of the FP32 one and
// these scalings run once per element), FP64 for the complex128 path.
template <typename R> __device__ __forceinline__ R inv_prod(double a, double b) { return (R)(1.0 / (a * b)); }
template <> __device__ __forceinline__ float inv_prod<float>(double a, double b) {
    return __frcp_rn((float)a * (float)b);
}

// acc += conj(x) * y
template <typename C> __device__ __forceinline__ void cfma_cj(C& acc, C x, C y) {
    acc.x = fma(x.x, y.x, acc.x); acc.x = fma(x.y, y.y, acc.x);
    acc.y = fma(x.x, y.y, acc.y); acc.y = fma(-x.y, y.x, acc.y);
}

// ---------------------------------------------------------------- theta --
// grid (ceil(chip/32), ceil(chip/32), count), 256 threads.  Each block computes
// the 32x32 (alpha, gamma) tile of all four theta_{st} = X_s Y_t with
// X_s = diag(Lambda_{b-1}) Gamma_b^s diag(Lambda_b), Y_t = Gamma_{b+1}^t diag(Lambda_{b+1}),
// mixes them with the gate and writes theta' (tall: rows (s,alpha), cols (t,gamma))
// or its adjoint (wide) into w and w0.
// G: the complex type of the Gamma store, read as is and widened to C (the FP64
// resolution of a complex64 state forms theta' in FP64 from complex64 Gamma).
// In the resolution pass (a.refine == 1) only bonds marked undecided run, and
// their dims (written by the first pass, unchanged since) are left alone; with
// a.refine == 2 (an FP64 pass over every bond: the FP64 regauge of a complex64
// state) every bond runs and is marked.
template <typename R, typename G>
__global__ void __launch_bounds__(256) k_theta(LayerArgs<R> a) {
    using C = cx_t<R>;
    const int j = blockIdx.z;
    if (a.refine == 1 && a.dims[j * kDims + D_REFINE] != 1) return;
    const int b = a.bonds[j];
    const int chip = a.chip;
    // device-side argument check: a bond or dimension out of range (a corrupted
    // list or state) is latched as DERR_BADARG and the bond is skipped: zero
    // rows and columns make the SVD, truncation and Gamma kernels do nothing
    if (b < 0 || b > a.n_sites - 2 || a.chi[b] < 1 || a.chi[b] > chip || a.chi[b + 1] < 1 ||
        a.chi[b + 1] > chip || a.chi[b + 2] < 1 || a.chi[b + 2] > chip) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && a.refine != 1) {
            int32_t* d = a.dims + j * kDims;
            for (int q = 0; q < kDims; ++q) d[q] = 0;
            d[D_TALL] = 1;
            atomicOr(a.err, DERR_BADARG);
        }
        return;
    }
    const int cl = a.chi[b], cm = a.chi[b + 1], cr = a.chi[b + 2];
    // tSU (mode 1) always stores theta^dag: its SVD goes through the factors
    const bool tall = a.mode == 0 && cl >= cr;
    // The FP64 resolution of a gated bond runs its SVD on B = M^dag U32 (k_precond),
    // whose rotated columns are M's right singular vectors: the Gamma kernels then
    // take the bond in the other orientation, so w0 gets M^dag (the layout the other
    // orientation stores) and the dims are switched to it: rows = cols = n, the
    // columns of M.  w is left to k_precond.
    const bool precond = a.refine == 1 && a.mode == 0 && a.w32 != nullptr;
    const bool wtall = precond ? !tall : tall;
    if (precond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        int32_t* d = a.dims + j * kDims;
        const int n = tall ? 2 * cr : 2 * cl;
        d[D_TALL] = tall ? 0 : 1;
        d[D_ROWS] = n;
        d[D_COLS] = n;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && a.refine != 1) {
        int32_t* d = a.dims + j * kDims;
        d[D_CL] = cl; d[D_CM] = cm; d[D_CR] = cr; d[D_TALL] = tall ? 1 : 0; d[D_BOND] = b;
        d[D_K] = 0;
        d[D_REFINE] = a.refine == 2 ? 1 : 0;
        d[D_COND] = 0;
        if (a.mode == 0) { d[D_ROWS] = tall ? 2 * cl : 2 * cr; d[D_COLS] = tall ? 2 * cr : 2 * cl; }
        else { d[D_ROWS] = 2 * cr; d[D_COLS] = cm; }
        atomicAdd(&a.work[1], 32ull * (unsigned long long)cl * (unsigned long long)cm * (unsigned long long)cr);
    }
    const int a0 = blockIdx.x * 32, g0 = blockIdx.y * 32;
    if (a0 >= cl || g0 >= cr) return;

    __shared__ C xs[2][16][33];
    __shared__ C ys[2][16][33];
    __shared__ C ug[16];
    // the Lambdas of this tile in the kernel's precision (staged once)
    __shared__ R sL[32], sR[32], sM[PTEBD_CHI_LIMIT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t slice = (size_t)chip * chip;
    const G* G0 = static_cast<const G*>(a.gamma) + (size_t)b * 2 * slice;
    const G* G1 = static_cast<const G*>(a.gamma) + (size_t)(b + 1) * 2 * slice;
    {
        const double* lL = a.lam + (size_t)b * chip;
        const double* lM = a.lam + (size_t)(b + 1) * chip;
        const double* lR = a.lam + (size_t)(b + 2) * chip;
        const int t = threadIdx.x;
        if (t < 32) sL[t] = (a0 + t < cl) ? (R)lL[a0 + t] : (R)0;
        else if (t < 64) sR[t - 32] = (g0 + t - 32 < cr) ? (R)lR[g0 + t - 32] : (R)0;
        for (int q = t; q < cm; q += 256) sM[q] = (R)lM[q];
        __syncthreads();
    }

    C acc[2][2][2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int q = 0; q < 2; ++q) acc[s][t][i][q] = cz<C>();

    for (int k0 = 0; k0 < cm; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int s = e >> 9, rem = e & 511, kk = rem >> 5, al = rem & 31;
            const int alpha = a0 + al, beta = k0 + kk;
            C v = cz<C>();
            if (alpha < cl && beta < cm)
                v = cscale(cconv<C>(G0[s * slice + (size_t)beta * chip + alpha]), sL[al] * sM[beta]);
            xs[s][kk][al] = v;
        }
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int t = e >> 9, rem = e & 511, gg = rem >> 4, kk = rem & 15;
            const int gamma = g0 + gg, beta = k0 + kk;
            C v = cz<C>();
            if (gamma < cr && beta < cm)
                v = cscale(cconv<C>(G1[t * slice + (size_t)gamma * chip + beta]), sR[gg]);
            ys[t][kk][gg] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            C x[2][2], y[2][2];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < 2; ++i) x[s][i] = xs[s][kk][tx + 16 * i];
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int q = 0; q < 2; ++q) y[t][q] = ys[t][kk][ty + 16 * q];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int t = 0; t < 2; ++t)
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int q = 0; q < 2; ++q) cfma(acc[s][t][i][q], x[s][i], y[t][q]);
        }
        __syncthreads();
    }

    if (a.gates != nullptr) {
        if (threadIdx.x < 16) {
            const double* gp = a.gates + (size_t)j * 32 + 2 * threadIdx.x;
            ug[threadIdx.x] = cmake<C>(gp[0], gp[1]);
        }
        __syncthreads();
    }
    const size_t ldw = a.ldw;
    C* W = a.w + (size_t)j * ldw * ldw;
    C* W0 = a.w0 + (size_t)j * ldw * ldw;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int alpha = a0 + tx + 16 * i;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gamma = g0 + ty + 16 * q;
            if (alpha >= cl || gamma >= cr) continue;
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int tp = 0; tp < 2; ++tp) {
                    C v;
                    if (a.gates != nullptr) {
                        v = cz<C>();
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int t = 0; t < 2; ++t)
                                cfma(v, ug[(2 * sp + tp) * 4 + 2 * s + t], acc[s][t][i][q]);
                    } else {
                        v = acc[sp][tp][i][q];
                    }
                    const size_t r = (size_t)sp * cl + alpha, c = (size_t)tp * cr + gamma;
                    if (wtall) {
                        if (!precond) W[c * ldw + r] = v;
                        W0[c * ldw + r] = v;
                    } else {
                        const C vc = cconj(v);
                        if (a.mode == 0 && !precond) W[r * ldw + c] = vc;
                        W0[r * ldw + c] = vc;
                    }
                }
        }
    }
}

// ------------------------------------------------------------- truncate --
// Operator Schmidt rank of a two-site gate, U = sum_k A_k (x) B_k with A_k on the
// left site and B_k on the right: the rank of the rearranged matrix
// R[(s', s), (t', t)] = U[(2 s' + t'), (2 s + t)].  theta' is a sum of rank(R)
// terms (A_k (x) 1) theta (B_k (x) 1)^T of rank <= chi_b each, so
// rank(theta') <= rank(R) chi_b.  One thread: a one-sided Jacobi on the four
// columns of R in FP64 (gates are given in FP64), rank = #{s_k > 1e-12 s_1}.
__device__ int op_schmidt_rank(const double* g) {
    double re[4][4], im[4][4];  // [column (t', t)][row (s', s)]
    for (int sp = 0; sp < 2; ++sp)
        for (int s0 = 0; s0 < 2; ++s0)
            for (int tp = 0; tp < 2; ++tp)
                for (int t0 = 0; t0 < 2; ++t0) {
                    const int e = (2 * sp + tp) * 4 + (2 * s0 + t0);
                    re[2 * tp + t0][2 * sp + s0] = g[2 * e];
                    im[2 * tp + t0][2 * sp + s0] = g[2 * e + 1];
                }
    for (int sweep = 0; sweep < 30; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                double al = 0, be = 0, gr = 0, gi = 0;  // |c_p|^2, |c_q|^2, c_p^H c_q
                for (int r = 0; r < 4; ++r) {
                    al += re[p][r] * re[p][r] + im[p][r] * im[p][r];
                    be += re[q][r] * re[q][r] + im[q][r] * im[q][r];
                    gr += re[p][r] * re[q][r] + im[p][r] * im[q][r];
                    gi += re[p][r] * im[q][r] - im[p][r] * re[q][r];
                }
                const double g2 = gr * gr + gi * gi;
                if (!(g2 > 1e-30 * al * be)) continue;
                rotated = true;
                const double gm = sqrt(g2), er = gr / gm, ei = gi / gm;
                const double zeta = (be - al) / (2.0 * gm);
                double t = 1.0 / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                if (zeta < 0) t = -t;
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                // c_p' = c c_p - sn conj(e) c_q,  c_q' = c c_q + sn e c_p
                for (int r = 0; r < 4; ++r) {
                    const double pr = re[p][r], pi = im[p][r], qr = re[q][r], qi = im[q][r];
                    re[p][r] = c * pr - sn * (er * qr + ei * qi);
                    im[p][r] = c * pi - sn * (er * qi - ei * qr);
                    re[q][r] = c * qr + sn * (er * pr - ei * pi);
                    im[q][r] = c * qi + sn * (er * pi + ei * pr);
                }
            }
        if (!rotated) break;
    }
    double nrm[4], mx = 0;
    for (int p = 0; p < 4; ++p) {
        double s2 = 0;
        for (int r = 0; r < 4; ++r) s2 += re[p][r] * re[p][r] + im[p][r] * im[p][r];
        nrm[p] = sqrt(s2);
        mx = fmax(mx, nrm[p]);
    }
    int rank = 0;
    for (int p = 0; p < 4; ++p) rank += nrm[p] > 1e-12 * mx ? 1 : 0;
    return rank;
}

// grid (count), 512 threads.  norms[] holds the FP64 column norms of the
// rotated matrix (= the singular values, unsorted).
// With a.resolve > a.thr_rel (the complex64 pass of a state with FP64
// resolution), singular values <= resolve * sigma_1 are not trusted: the kept
// count is decided only if it is the same whether they are taken as real or as
// zero, that is k_hi = min(chi_max, r_max, #{S > resolve S_1}) equals
// k_lo = min(chi_max, r_max, #{S > thr S_1}), with r_max = min(cols,
// rank(gate) chi_b) the structural bound on rank(theta').  An undecided bond is
// marked (dims D_REFINE = 1) and left alone: the FP64 pass recomputes it.
template <typename R>
__global__ void __launch_bounds__(512) k_truncate(LayerArgs<R> a) {
    constexpr int NS = 512;
    __shared__ double key[NS];
    __shared__ int idx[NS];
    __shared__ double red[NS];
    __shared__ int kept_sh, kept_hi_sh, rmax_sh;
    const int j = blockIdx.x, t = threadIdx.x;
    int32_t* d = a.dims + j * kDims;
    if (a.refine == 1 && d[D_REFINE] != 1) return;
    const int ncols = d[D_COLS];
    const int b = d[D_BOND];
    const double* nrm = a.norms + (size_t)j * a.ldw;
    key[t] = (t < ncols) ? nrm[t] : -1.0;
    idx[t] = t;
    __syncthreads();
    // bitonic sort, descending by value, ascending index on ties
    for (int size = 2; size <= NS; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int p = t ^ stride;
            if (p > t) {
                const bool desc = (t & size) == 0;
                const double kt = key[t], kp = key[p];
                const int it = idx[t], ip = idx[p];
                const bool t_first = (kt > kp) || (kt == kp && it < ip);
                if (desc ? !t_first : t_first) {
                    key[t] = kp; key[p] = kt; idx[t] = ip; idx[p] = it;
                }
            }
            __syncthreads();
        }
    }
    const double smax = key[0];
    if (!(smax > 0.0) || !isfinite(smax)) {
        if (t == 0) {
            atomicOr(a.err, isfinite(smax) ? DERR_ZERO_THETA : DERR_NONFINITE);
            d[D_K] = 0;
        }
        return;
    }
    const double thr = a.thr_rel * smax;
    const bool resolving = !a.refine && a.resolve > a.thr_rel;
    const double thr_hi = resolving ? a.resolve * smax : thr;
    // numbers above the thresholds (the keys are sorted)
    if (t == 0) {
        kept_sh = 0;
        kept_hi_sh = 0;
    }
    __syncthreads();
    if (t < ncols && key[t] > thr && (t + 1 == ncols || !(key[t + 1] > thr))) kept_sh = t + 1;
    if (t < ncols && key[t] > thr_hi && (t + 1 == ncols || !(key[t + 1] > thr_hi))) kept_hi_sh = t + 1;
    __syncthreads();
    int k = max(1, min(a.chi_max, kept_sh));
    if (resolving) {
        int k_lo = min(a.chi_max, kept_sh);
        int k_hi = min(a.chi_max, kept_hi_sh);
        if (k_hi < k_lo && a.gates != nullptr) {
            // undecided on the counts alone: the structural bound on rank(theta')
            // may still decide it (taken only now, it is a few hundred cycles of one thread)
            if (t == 0) rmax_sh = min(ncols, op_schmidt_rank(a.gates + (size_t)j * 32) * d[D_CM]);
            __syncthreads();
            k_lo = min(k_lo, rmax_sh);
            k_hi = min(k_hi, rmax_sh);
        }
        if (k_hi < k_lo) {
            if (t == 0) {
                d[D_REFINE] = 1;
                d[D_K] = 0;  // the Gamma kernels of this pass skip the bond
                a.slot_eps[j] = 0.0;
                a.slot_lognu[j] = 0.0;
                // in a CUDA graph the FP64 pass is an IF node: switch it on, once per launch
                if (a.cond && atomicExch(&a.dims[D_COND], 1) == 0) cudaGraphSetConditional(a.cond, 1);
            }
            return;
        }
        k = max(1, k_hi);
    }
    // FP64 weights: total and dropped, fixed-order tree sums
    const double w = (t < ncols) ? key[t] * key[t] : 0.0;
    red[t] = w;
    __syncthreads();
    for (int s = NS / 2; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    const double total = red[0];
    __syncthreads();
    red[t] = (t >= k) ? w : 0.0;
    __syncthreads();
    for (int s = NS / 2; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    const double dropped = red[0];
    double eps = (a.eps_mode == PTEBD_EPS_ABSOLUTE) ? dropped : dropped / total;
    double nu = 1.0;
    if (a.stabilise) {
        if (eps < 1.0) {
            nu = 1.0 / sqrt(1.0 - eps);
        } else if (t == 0) {
            atomicOr(a.err, DERR_EPS);
        }
    }
    // Lambda_b <- nu S_kept, or nu S_kept / |S| (the Schmidt reading; tSU keeps S)
    const double lam_scale = (a.stabilise && a.eps_mode == PTEBD_EPS_SCHMIDT) ? nu / sqrt(total) : nu;
    double* lam_b = a.lam + (size_t)(b + 1) * a.chip;
    for (int q = t; q < a.chip; q += NS) lam_b[q] = (q < k) ? lam_scale * key[q] : 0.0;
    if (t < k) {
        a.sig[(size_t)j * a.ldw + t] = key[t];
        a.perm[(size_t)j * a.ldw + t] = idx[t];
    }
    if (t == 0) {
        d[D_K] = k;
        a.chi[b + 1] = k;
        a.slot_eps[j] = eps;
        a.slot_lognu[j] = log(nu);
        if (a.stabilise) {
            a.bond_eps[b] = eps;
            a.bond_nu[b] = nu;
            a.bond_rank[b] = ncols;
        }
        a.bond_sweeps[b] = a.slot_sweeps[j];
    }
}

// ----------------------------------------------------------- Gamma, direct --
// The factor whose singular vectors are the rotated columns themselves:
// tall (w = theta' = U S): Gamma_b[s](alpha, beta) = w[(s,alpha), perm beta] / (S_beta Lambda_{b-1,alpha})
// wide (w = theta'^dag = V S): Gamma_{b+1}[t](beta, gamma) = conj(w[(t,gamma), perm beta]) / (S_beta Lambda_{b+1,gamma})
// grid (ceil(chip*chip/256), 2, count), 256 threads; writes the whole padded slice.
template <typename R, typename G>
__global__ void __launch_bounds__(256) k_gamma_direct(LayerArgs<R> a) {
    using C = cx_t<R>;
    const int j = blockIdx.z, sg = blockIdx.y;
    const int32_t* d = a.dims + j * kDims;
    if (a.refine == 1 && d[D_REFINE] != 1) return;
    const int k = d[D_K];
    if (k == 0) return;  // error latched by k_truncate
    const int cl = d[D_CL], cr = d[D_CR], b = d[D_BOND];
    const bool tall = d[D_TALL] != 0;
    const int chip = a.chip;
    const size_t slice = (size_t)chip * chip;
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= slice) return;
    const int row = (int)(e % chip), col = (int)(e / chip);
    const size_t ldw = a.ldw;
    const C* W = a.w + (size_t)j * ldw * ldw;
    const double* sig = a.sig + (size_t)j * ldw;
    const int32_t* perm = a.perm + (size_t)j * ldw;
    C v = cz<C>();
    if (tall) {
        // row = alpha, col = beta
        if (col < k && row < cl) {
            const double* lL = a.lam + (size_t)b * chip;
            v = cscale(W[(size_t)perm[col] * ldw + (size_t)sg * cl + row], inv_prod<R>(sig[col], lL[row]));
        }
        static_cast<G*>(a.gamma)[(size_t)b * 2 * slice + sg * slice + e] = cconv<G>(v);
    } else {
        // row = beta, col = gamma
        if (row < k && col < cr) {
            const double* lR = a.lam + (size_t)(b + 2) * chip;
            v = cscale(cconj(W[(size_t)perm[row] * ldw + (size_t)sg * cr + col]), inv_prod<R>(sig[row], lR[col]));
        }
        static_cast<G*>(a.gamma)[(size_t)(b + 1) * 2 * slice + sg * slice + e] = cconv<G>(v);
    }
}

// ------------------------------------------------------------ Gamma, GEMM --
// The other factor through Z[i, j] = sum_r conj(P[r, i]) Q[r, j], the rotated
// columns (U S or V S) divided by S as they are loaded (so that no product of
// the size of S^2 is formed):
// tall: P = w (columns perm beta) / S, Q = w0 = theta', Z = S V^dag:
//       Gamma_{b+1}[t](beta, gamma) = Z[beta, (t,gamma)] / (S_beta Lambda_{b+1,gamma})
// wide: P = w0 = theta'^dag, Q = w (columns perm beta) / S, Z = U S:
//       Gamma_b[s](alpha, beta) = Z[(s,alpha), beta] / (S_beta Lambda_{b-1,alpha})
// grid (ceil(chip/32), ceil(chip/32), 2 count), 256 threads, 2x2 outputs per thread.
template <typename R, typename G>
__global__ void __launch_bounds__(256) k_gamma_gemm(LayerArgs<R> a) {
    using C = cx_t<R>;
    const int j = blockIdx.z >> 1, sg = blockIdx.z & 1;
    const int32_t* d = a.dims + j * kDims;
    if (a.refine == 1 && d[D_REFINE] != 1) return;
    const int k = d[D_K];
    if (k == 0) return;
    const int cl = d[D_CL], cr = d[D_CR], b = d[D_BOND], rows = d[D_ROWS];
    const bool tall = d[D_TALL] != 0;
    const int chip = a.chip;
    const size_t slice = (size_t)chip * chip, ldw = a.ldw;
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int rlim = tall ? k : cl;   // valid target rows
    const int clim = tall ? cr : k;   // valid target cols
    G* Gm = static_cast<G*>(a.gamma) + (size_t)(tall ? b + 1 : b) * 2 * slice + sg * slice;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (r0 >= rlim || c0 >= clim) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int row = r0 + tx + 16 * i, col = c0 + ty + 16 * q;
                if (row < chip && col < chip) Gm[(size_t)col * chip + row] = cz<G>();
            }
        return;
    }
    const C* W = a.w + (size_t)j * ldw * ldw;
    const C* W0 = a.w0 + (size_t)j * ldw * ldw;
    const C* P = tall ? W : W0;
    const C* Q = tall ? W0 : W;
    const int32_t* perm = a.perm + (size_t)j * ldw;
    const double* sig = a.sig + (size_t)j * ldw;
    __shared__ int pcol[32], qcol[32];
    __shared__ R pscl[32], qscl[32];
    __shared__ C ps[16][33], qs[16][33];
    if (threadIdx.x < 32) {
        const int row = r0 + threadIdx.x;
        int pc = -1;
        R sc = 1;
        if (row < rlim) {
            pc = tall ? perm[row] : sg * cl + row;
            if (tall) sc = (R)(1.0 / sig[row]);
        }
        pcol[threadIdx.x] = pc;
        pscl[threadIdx.x] = sc;
    } else if (threadIdx.x < 64) {
        const int col = c0 + threadIdx.x - 32;
        int qc = -1;
        R sc = 1;
        if (col < clim) {
            qc = tall ? sg * cr + col : perm[col];
            if (!tall) sc = (R)(1.0 / sig[col]);
        }
        qcol[threadIdx.x - 32] = qc;
        qscl[threadIdx.x - 32] = sc;
    }
    __syncthreads();
    C acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[i][q] = cz<C>();
    for (int k0 = 0; k0 < rows; k0 += 16) {
        for (int e = threadIdx.x; e < 512; e += 256) {
            const int kk = e & 15, cc = e >> 4;
            const int r = k0 + kk;
            const int pc = pcol[cc], qc = qcol[cc];
            ps[kk][cc] = (pc >= 0 && r < rows) ? cscale(P[(size_t)pc * ldw + r], pscl[cc]) : cz<C>();
            qs[kk][cc] = (qc >= 0 && r < rows) ? cscale(Q[(size_t)qc * ldw + r], qscl[cc]) : cz<C>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            const C p0 = ps[kk][tx], p1 = ps[kk][tx + 16];
            const C q0 = qs[kk][ty], q1 = qs[kk][ty + 16];
            cfma_cj(acc[0][0], p0, q0); cfma_cj(acc[0][1], p0, q1);
            cfma_cj(acc[1][0], p1, q0); cfma_cj(acc[1][1], p1, q1);
        }
        __syncthreads();
    }
    const double* lnb = a.lam + (size_t)(tall ? b + 2 : b) * chip;  // Lambda_{b+1} or Lambda_{b-1}
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int row = r0 + tx + 16 * i, col = c0 + ty + 16 * q;
            if (row >= chip || col >= chip) continue;
            C v = cz<C>();
            if (row < rlim && col < clim) {
                const double sb = tall ? sig[row] : sig[col];
                const double ln = tall ? lnb[col] : lnb[row];
                v = cscale(acc[i][q], inv_prod<R>(sb, ln));
            }
            Gm[(size_t)col * chip + row] = cconv<G>(v);
        }
}

// -------------------------------------------- FP64 resolution, gated bond --
// B = M^dag U32 for a gated bond left undecided by the complex64 truncation:
// M (m x n) is the matrix the complex64 Jacobi ran on, held in w0 as M^dag
// (k_theta's preconditioned store), and U32 = the complex64 pass's rotated
// columns w32 divided by their norms (a zero column stays zero).  The FP64 SVD
// then runs on B (n x n, into w): B = V S U^dag U32, and with U32 unitary up to
// the complex64 Jacobi's orthogonality (a few 1e-6) this is M's right singular
// vectors times S up to a multiplicative perturbation of that size, which moves
// every singular value by that relative amount at most, the smallest included,
// and leaves an exact zero of S exactly zero.  Its columns start nearly
// orthogonal except inside the complex64 noise, so the FP64 sweeps converge in
// fewer steps than from M.  The dims were switched by k_theta: D_TALL is the
// other orientation, D_ROWS = D_COLS = n; m = 2 chi_{b-1} (originally tall) or
// 2 chi_{b+1}.
// grid (ceil(2 chip / 32), ceil(2 chip / 32), count), 256 threads, 2x2 outputs a thread.
__global__ void __launch_bounds__(256) k_precond(LayerArgs<double> a) {
    const int j = blockIdx.z;
    const int32_t* d = a.dims + j * kDims;
    if (d[D_REFINE] != 1) return;
    const int n = d[D_ROWS];
    const int m = d[D_TALL] ? 2 * d[D_CR] : 2 * d[D_CL];
    const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    if (i0 >= n || c0 >= n) return;
    const size_t ldw = a.ldw;
    const double2* Mh = a.w0 + (size_t)j * ldw * ldw;  // M^dag: n x m, column-major
    const float2* U = a.w32 + (size_t)j * ldw * ldw;    // U32 S32: m x n
    const double* nrm = a.norms + (size_t)j * ldw;
    double2* B = a.w + (size_t)j * ldw * ldw;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    __shared__ double2 ps[16][33], qs[16][33];
    __shared__ double qscl[32];
    if (threadIdx.x < 32) {
        const int c = c0 + threadIdx.x;
        const double s = c < n ? nrm[c] : 0.0;
        qscl[threadIdx.x] = s > 0.0 ? 1.0 / s : 0.0;
    }
    __syncthreads();
    double2 acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[i][q] = make_double2(0.0, 0.0);
    for (int r0 = 0; r0 < m; r0 += 16) {
        for (int e = threadIdx.x; e < 512; e += 256) {
            const int ii = e & 31, kk = e >> 5;  // M^dag(i0 + ii, r0 + kk): contiguous in ii
            const int r = r0 + kk;
            ps[kk][ii] = (i0 + ii < n && r < m) ? Mh[(size_t)r * ldw + i0 + ii] : make_double2(0.0, 0.0);
            const int kq = e & 15, cc = e >> 4;  // U32(r0 + kq, c0 + cc): contiguous in kq
            const int rq = r0 + kq;
            double2 u = make_double2(0.0, 0.0);
            if (c0 + cc < n && rq < m) {
                const float2 v = U[(size_t)(c0 + cc) * ldw + rq];
                u = make_double2((double)v.x * qscl[cc], (double)v.y * qscl[cc]);
            }
            qs[kq][cc] = u;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            const double2 p0 = ps[kk][tx], p1 = ps[kk][tx + 16];
            const double2 q0 = qs[kk][ty], q1 = qs[kk][ty + 16];
            cfma(acc[0][0], p0, q0); cfma(acc[0][1], p0, q1);
            cfma(acc[1][0], p1, q0); cfma(acc[1][1], p1, q1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int row = i0 + tx + 16 * i, col = c0 + ty + 16 * q;
            if (row < n && col < n) B[(size_t)col * ldw + row] = acc[i][q];
        }
}

// ------------------------------------------------------- tSU factors ----
// For tSU the two-site tensor is theta = X Y with X = diag(Lambda_{b-1}) Gamma_b diag(Lambda_b)
// (2 chi_{b-1} x chi_b, rows (s, alpha)), so rank(theta) <= chi_b.  Its SVD is taken
// in two tall, narrow steps: X's columns are orthogonalised (X J = U_X Sigma_X; the
// graded column norms Lambda_b make this converge fast), then M^dag = theta^dag U_X
// (2 chi_{b+1} x chi_b) is orthogonalised: its rotated columns are V S of theta,
// because theta = U_X M exactly.
// k_xform writes X into w; grid (ceil(2 chip * chip / 256), count).
template <typename R, typename G>
__global__ void __launch_bounds__(256) k_xform(LayerArgs<R> a) {
    using C = cx_t<R>;
    const int j = blockIdx.y;
    const int32_t* d = a.dims + j * kDims;
    if (a.refine == 1 && d[D_REFINE] != 1) return;
    const int cl = d[D_CL], cm = d[D_CM], b = d[D_BOND];
    const int chip = a.chip;
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    const int rows = 2 * cl;
    const int r = (int)(e % (2 * chip)), beta = (int)(e / (2 * chip));
    if (beta >= cm || r >= rows) return;
    const int s = r / cl, alpha = r - s * cl;
    const size_t slice = (size_t)chip * chip;
    const C g = cconv<C>(static_cast<const G*>(a.gamma)[(size_t)b * 2 * slice + s * slice + (size_t)beta * chip + alpha]);
    const R sc = (R)a.lam[(size_t)b * chip + alpha] * (R)a.lam[(size_t)(b + 1) * chip + beta];
    a.w[(size_t)j * a.ldw * a.ldw + (size_t)beta * a.ldw + r] = cscale(g, sc);
}

// w1 = w0 (w diag(1 / sigma_X)) with w0 = theta^dag (2 chi_{b+1} x 2 chi_{b-1}) and
// w = U_X Sigma_X (2 chi_{b-1} x chi_b): w1 = theta^dag U_X = M^dag (the columns of
// w are divided by sigma_X as they are loaded; a zero sigma_X gives a zero column).
// grid (ceil(2 chip / 32), ceil(chip / 32), count), 256 threads.
template <typename R>
__global__ void __launch_bounds__(256) k_proj(LayerArgs<R> a) {
    using C = cx_t<R>;
    const int j = blockIdx.z;
    const int32_t* d = a.dims + j * kDims;
    if (a.refine == 1 && d[D_REFINE] != 1) return;
    const int cl = d[D_CL], cm = d[D_CM], cr = d[D_CR];
    const int rows = 2 * cr, kdim = 2 * cl;
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    if (r0 >= rows || c0 >= cm) return;
    const size_t ldw = a.ldw;
    const C* A = a.w0 + (size_t)j * ldw * ldw;  // rows x kdim
    const C* B = a.w + (size_t)j * ldw * ldw;   // kdim x cm
    C* out = a.w1 + (size_t)j * ldw * ldw;
    const double* sig = a.norms + (size_t)j * ldw;
    __shared__ C as[16][33], bs[16][33];
    __shared__ R bscl[32];
    if (threadIdx.x < 32) {
        const int gc = c0 + threadIdx.x;
        const double sg = gc < cm ? sig[gc] : 0.0;
        bscl[threadIdx.x] = sg > 0.0 ? (R)(1.0 / sg) : (R)0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    C acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[i][q] = cz<C>();
    for (int k0 = 0; k0 < kdim; k0 += 16) {
        for (int e = threadIdx.x; e < 512; e += 256) {
            const int rr = e & 31, kk = e >> 5;
            const int gr = r0 + rr, gk = k0 + kk;
            as[kk][rr] = (gr < rows && gk < kdim) ? A[(size_t)gk * ldw + gr] : cz<C>();
            const int kb = e & 15, cc = e >> 4;
            const int gc = c0 + cc, gkb = k0 + kb;
            bs[kb][cc] = (gc < cm && gkb < kdim) ? cscale(B[(size_t)gc * ldw + gkb], bscl[cc]) : cz<C>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            const C x0 = as[kk][tx], x1 = as[kk][tx + 16];
            const C y0 = bs[kk][ty], y1 = bs[kk][ty + 16];
            cfma(acc[0][0], x0, y0); cfma(acc[0][1], x0, y1);
            cfma(acc[1][0], x1, y0); cfma(acc[1][1], x1, y1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gr = r0 + tx + 16 * i, gc = c0 + ty + 16 * q;
            if (gr >= rows || gc >= cm) continue;
            out[(size_t)gc * ldw + gr] = acc[i][q];
        }
}

// ------------------------------------------------------------ reductions --
__global__ void __launch_bounds__(256) k_reduce_layer(const double* slot_eps, const double* slot_lognu,
                                                      int count, int gated, double* totals) {
    __shared__ double se[256], sl[256];
    const int t = threadIdx.x;
    double e = 0.0, l = 0.0;
    for (int i = t; i < count; i += 256) { e += slot_eps[i]; l += slot_lognu[i]; }
    se[t] = e; sl[t] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) { se[t] += se[t + s]; sl[t] += sl[t + s]; }
        __syncthreads();
    }
    if (t == 0) {
        if (gated) { totals[0] += se[0]; totals[1] += sl[0]; }
        else { totals[2] += se[0]; }
    }
}

// The per-chunk sums of a layer run on concurrent streams, added in chunk order.
__global__ void k_add_partials(const double* partials, int k, double* totals) {
    if (threadIdx.x != 0) return;
    double e = 0.0, l = 0.0, u = 0.0;
    for (int c = 0; c < k; ++c) { e += partials[4 * c]; l += partials[4 * c + 1]; u += partials[4 * c + 2]; }
    totals[0] += e;
    totals[1] += l;
    totals[2] += u;
}

// -------------------------------------------------------------- launchers --
template <typename R, typename G> cudaError_t launch_theta(const LayerArgs<R>& a, cudaStream_t s) {
    // tensor_cores 1: gated stages; 2: the tSU steps as well.  On a tSU step the
    // accumulation's residual shrinkage (about 2e-7 per product) is not
    // renormalised away, and over the bonds of a PtSU step it moves the norm of
    // the state: 5.4e-4 at N = 1024, chi = 256.
    if constexpr (std::is_same<R, float>::value)
        if (a.tensor_cores && (a.mode == 0 || a.tensor_cores == 2) && a.chip >= 64 && a.refine == 0)
            return launch_theta_tc(a, s);
    const int tiles = (a.chip + 31) / 32;
    dim3 grid(tiles, tiles, a.count);
    k_theta<R, G><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename R> cudaError_t launch_truncate(const LayerArgs<R>& a, cudaStream_t s) {
    k_truncate<R><<<a.count, 512, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename R, typename G> cudaError_t launch_gamma(const LayerArgs<R>& a, cudaStream_t s) {
    const size_t slice = (size_t)a.chip * a.chip;
    dim3 g1((unsigned)((slice + 255) / 256), 2, a.count);
    k_gamma_direct<R, G><<<g1, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if constexpr (std::is_same<R, float>::value)
        if (a.tensor_cores && (a.mode == 0 || a.tensor_cores == 2) && a.chip >= 64 && a.refine == 0)
            return launch_gamma_gemm_tc(a, s);
    const int tiles = (a.chip + 31) / 32;
    dim3 g2(tiles, tiles, 2 * a.count);
    k_gamma_gemm<R, G><<<g2, 256, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename R, typename G> cudaError_t launch_xform(const LayerArgs<R>& a, cudaStream_t s) {
    const size_t n = (size_t)2 * a.chip * a.chip;
    dim3 grid((unsigned)((n + 255) / 256), a.count);
    k_xform<R, G><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename R> cudaError_t launch_proj(const LayerArgs<R>& a, cudaStream_t s) {
    if constexpr (std::is_same<R, float>::value)
        if (a.tensor_cores == 2 && a.chip >= 64 && a.refine == 0) return launch_proj_tc(a, s);
    dim3 grid((2 * a.chip + 31) / 32, (a.chip + 31) / 32, a.count);
    k_proj<R><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_precond(const LayerArgs<double>& a, cudaStream_t s) {
    const int tiles = (2 * a.chip + 31) / 32;
    dim3 grid(tiles, tiles, a.count);
    k_precond<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_reduce_layer(const double* slot_eps, const double* slot_lognu, int count,
                                int gated, double* totals, cudaStream_t s) {
    k_reduce_layer<<<1, 256, 0, s>>>(slot_eps, slot_lognu, count, gated, totals);
    return cudaGetLastError();
}

cudaError_t launch_add_partials(const double* partials, int k, double* totals, cudaStream_t s) {
    k_add_partials<<<1, 32, 0, s>>>(partials, k, totals);
    return cudaGetLastError();
}

template cudaError_t launch_theta<float, float2>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_theta<double, double2>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_theta<double, float2>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_truncate<float>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_truncate<double>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_gamma<float, float2>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_gamma<double, double2>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_gamma<double, float2>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_xform<float, float2>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_xform<double, double2>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_xform<double, float2>(const LayerArgs<double>&, cudaStream_t);
template cudaError_t launch_proj<float>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_proj<double>(const LayerArgs<double>&, cudaStream_t);

}  // namespace ptebd
