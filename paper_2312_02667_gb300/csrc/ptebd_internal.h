// Internal declarations of libptebd: device memory layout, kernel arguments and
// the launchers each translation unit provides.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/ptebd.h"

namespace ptebd {

// ---------------------------------------------------------------- complex --
template <typename R> struct Cx;
template <> struct Cx<float>  { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <typename R> using cx_t = typename Cx<R>::T;

template <typename C> __host__ __device__ __forceinline__ C cmake(double re, double im) {
    C c; c.x = (decltype(c.x))re; c.y = (decltype(c.y))im; return c;
}
// complex conversion between storage and arithmetic types (exact from float2 to
// double2, rounded to nearest the other way)
template <typename T, typename F> __host__ __device__ __forceinline__ T cconv(F v) {
    T c; c.x = (decltype(c.x))v.x; c.y = (decltype(c.y))v.y; return c;
}

// --------------------------------------------------------- device errors --
// Bits of the latched device error word.
enum : uint32_t {
    DERR_NONFINITE = 1u,     // a non-finite singular value / norm
    DERR_ZERO_THETA = 2u,    // theta' is zero: nothing to keep
    DERR_EPS = 4u,           // eps_b >= 1 in absolute mode: nu undefined
    DERR_NOT_CONVERGED = 8u, // a Jacobi SVD hit its sweep limit
    DERR_TIMEOUT = 16u,      // a bounded wait on an mbarrier ran out
    DERR_BADARG = 32u,       // a bond or bond dimension out of range reached a kernel (skipped)
    DERR_DRAIN = 64u,        // after a wait ran out, a CTA's own bulk copies did not finish either: the CTA
                             // returned with copies into its shared memory possibly still in flight
};

// ------------------------------------------------------------- layout ----
// All device memory comes from two caller buffers.
//
// State buffer:
//   gamma  : N sites x 2 (sigma) x chip x chip complex (float2 or double2),
//            each (site, sigma) slice column-major: element (alpha, beta) at
//            beta * chip + alpha; entries outside chi_{s-1} x chi_s are zero
//   lam    : (N+1) x chip doubles, Lambda_b at (b+1)*chip; rows 0 and N are
//            the boundary vectors (1, 0, ...)
//   chi    : N+1 int32, chi_b at index b+1 (chi[0] = chi[N] = 1)
//   bond_* : per-bond metrics (N-1 each)
//   totals : [0] eps_total (gate updates), [1] sum ln nu, [2] eps of tSU steps,
//            [3] layers applied; then 4 uint64 work counters
//   err    : latched error word
//   gates  : ceil((N-1)/2) x 32 doubles, staging of host gates
//   bonds  : 3 lists of ceil((N-1)/2) int32: even bonds, odd bonds, user list
//   contraction scratch: 8 chip x chip complex128 matrices
// Workspace (per slot = one bond of a chunk):
//   w, w0, w1 : ldw x ldw complex each (ldw = 2 chip); w is rotated by the SVD,
//            w0 keeps theta' (or its adjoint) for the second factor, w1 holds
//            the second matrix of the tSU factorisation
//   norms, sig : ldw doubles; perm : ldw int32; dims : kDims int32
//   (PTEBD_MIXED with FP64 resolution) r, r0 : ldw x ldw complex128 each, the
//            FP64 recomputation of a gated bond whose truncation the complex64
//            spectrum leaves undecided
struct Layout {
    int n_sites = 0, chi_max = 0, chip = 0, ldw = 0, precision = 0, max_bonds = 0;
    size_t elem = 0;  // bytes of one complex element of gamma / w
    // state offsets (bytes)
    size_t off_gamma = 0, off_lam = 0, off_chi = 0, off_bond_eps = 0, off_bond_nu = 0,
           off_bond_rank = 0, off_bond_sweeps = 0, off_totals = 0, off_err = 0,
           off_gates = 0, off_bonds = 0, off_scratch = 0, off_partials = 0, state_bytes = 0;
    // per-slot workspace (bytes); slot_r: one complex128 matrix of the FP64
    // resolution (0 when the config does not use it)
    size_t slot_w = 0, slot_small = 0, slot_r = 0, slot_bytes = 0;
    bool resolve64 = false;  // PTEBD_MIXED bonds undecided in complex64 are recomputed in FP64
    double resolve = 0.0;    // the relative level below which complex64 singular values are not trusted
};

Layout make_layout(const ptebd_config& cfg);

// Device views handed to kernels.
template <typename R>
struct LayerArgs {
    using C = cx_t<R>;
    void* gamma;  // Gamma store: complex of the state's precision (float2 or double2), which may
                  // differ from R in the FP64 resolution of a complex64 state
    double* lam; int32_t* chi;
    C* w; C* w0; C* w1; double* norms; double* sig; int32_t* perm; int32_t* dims;
    double* slot_eps; double* slot_lognu; int32_t* slot_sweeps;
    const int32_t* bonds; const double* gates;  // gates == nullptr: tSU
    int count, chip, ldw, n_sites, chi_max;
    double thr_rel;   // relative truncation threshold: the cutoff, or max(cutoff, resolve) when the
                      // complex64 spectrum decides a bond without the FP64 resolution
    double resolve;   // > thr_rel: bonds whose kept count depends on singular values <= resolve * sigma_1
                      // are left undecided (dims D_REFINE = 1) for the FP64 resolution; 0: off
    unsigned long long cond;  // in a stream capture: the conditional handle of the IF node that holds the FP64
                              // resolution pass; the complex64 truncation sets it when it leaves a bond undecided
    int refine;       // 1: this launch is the FP64 resolution pass (only bonds with D_REFINE = 1 run);
                      // 2: an FP64 pass over every bond of a complex64 state (FP64 regauge)
    const float2* w32;  // the FP64 resolution of a gated bond: the complex64 pass's rotated columns
                        // U32 S32 of the same slots (with their FP64 norms still in `norms`); the
                        // FP64 SVD then runs on B = M^dag U32 (launch_precond) instead of on M
    int eps_mode, stabilise, max_sweeps;
    int wait_test;    // test of the bounded waits: one hand-off wait per CTA targets a count nothing
                      // reaches, with a short limit, so the CTA aborts and latches DERR_TIMEOUT
    int nw;           // Jacobi block width requested (0: the default; 8 or 16 for complex64)
    int pairs;        // complex64, width 16: I columns per warp (1: 16 warps; 2: 8 warps, two pairs a round)
    int tensor_cores; // complex64 on the tensor cores (tcgen05, 3xTF32) when chip >= 64: 1 theta' and
                      // the Gamma GEMM of gated stages, 2 the tSU steps as well
    int polish;       // complex64 Jacobi: one last sweep at the tighter threshold (see Eps::polish)
    int mode;         // 0: gated bond; 1: tSU through the rank-chi_b factorisation
    int pass;         // Jacobi: 0 = rows/cols from dims, 1 = the X factor (2 chi_{b-1} x chi_b)
    double* bond_eps; double* bond_nu; int32_t* bond_rank; int32_t* bond_sweeps;
    double* totals; uint32_t* err;
    unsigned long long* work;  // [0] Jacobi pair-row visits, [1] theta flops, [2] rotations,
                               // [3] sweeps summed, [4] SVDs; [5..7] the same for tSU;
                               // [8] bonds recomputed in FP64, [9] their Jacobi visits
};

// dims[] entries of a slot (kDims int32 per slot)
// D_COND (first slot of a launch only): set once the launch has asked for its FP64 pass
enum { D_CL = 0, D_CM = 1, D_CR = 2, D_TALL = 3, D_BOND = 4, D_K = 5, D_ROWS = 6, D_COLS = 7,
       D_REFINE = 8, D_COND = 9 };
constexpr int kDims = 16;
constexpr int kWork = 16;  // work counters

// ------------------------------------------------------------ launchers --
// G: the complex type of the Gamma store (cx_t<R> except in the FP64 resolution)
template <typename R, typename G = cx_t<R>> cudaError_t launch_theta(const LayerArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_jacobi(const LayerArgs<R>& a, cudaStream_t s);
// theta' of a complex64 state on the tensor cores (ptebd_theta_tc.cu)
cudaError_t launch_theta_tc(const LayerArgs<float>& a, cudaStream_t s);
cudaError_t launch_gamma_gemm_tc(const LayerArgs<float>& a, cudaStream_t s);  // the GEMM factor of the Gamma rebuild
cudaError_t launch_proj_tc(const LayerArgs<float>& a, cudaStream_t s);        // M^dag of the tSU factorisation
cudaError_t theta_tc_prepare();  // raises the smem limits of both tensor-core kernels
template <typename R> cudaError_t launch_truncate(const LayerArgs<R>& a, cudaStream_t s);
template <typename R, typename G = cx_t<R>> cudaError_t launch_gamma(const LayerArgs<R>& a, cudaStream_t s);
template <typename R, typename G = cx_t<R>> cudaError_t launch_xform(const LayerArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_proj(const LayerArgs<R>& a, cudaStream_t s);
// the FP64 resolution of gated bonds: B = M^dag U32 into w (k_precond)
cudaError_t launch_precond(const LayerArgs<double>& a, cudaStream_t s);
// pass 1 of the tSU SVD: an orthonormal basis of the columns of X (ptebd_orth.cu)
template <typename R> cudaError_t launch_orth(const LayerArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t orth_prepare();   // raises its dynamic smem limit
cudaError_t launch_reduce_layer(const double* slot_eps, const double* slot_lognu, int count,
                                int gated, double* totals, cudaStream_t s);
// totals[0..2] += sum over c < k of partials[4 c + 0..2], in the order of c
cudaError_t launch_add_partials(const double* partials, int k, double* totals, cudaStream_t s);

// A layer may run as up to kMaxChunks bond chunks on concurrent streams.
constexpr int kMaxChunks = 16;
template <typename R> cudaError_t jacobi_prepare();   // raises the dynamic smem limit
int jacobi_block_width(int precision, int requested);  // the NW a launch with a.nw = requested uses
size_t jacobi_smem_bytes(int precision, int ldw, int nw);

// Transfer-matrix contraction.  C = rowscale o (op(A) B) o colscale * alpha + beta C,
// all column-major; A and B are complex of type TA/TB, C is complex128.
// opA: 0 = N, 1 = conjugate transpose.
template <typename TA, typename TB>
cudaError_t launch_zgemm(int m, int n, int k, double2 alpha,
                         const TA* A, int lda, int opA, const TB* B, int ldb,
                         const double* colscale_b, double2 beta, double2* Cm, int ldc,
                         const double* rowscale_c, cudaStream_t s);
template <typename TG>
cudaError_t launch_sample_site(const TG* gamma_s, const double* lam, int chil, int chir, int chip, const double2* L,
                               const double2* v_in, double2* v_out, const double* uniforms, int site, int n_sites,
                               int32_t* bits, int n_samples, cudaStream_t s);
cudaError_t launch_scale_max(double2* E, int rows, int cols, int ld, double* log_acc, cudaStream_t s);
cudaError_t launch_fill_identity(double2* E, int rows, int cols, int ld, cudaStream_t s);

}  // namespace ptebd
