/*
 * ptebd.h - C ABI of libptebd, a single-GPU (sm_103a) implementation of one
 * layer of the improved parallel TEBD (pTEBD) of arXiv:2312.02667.
 *
 * Method (all references are to the paper):
 *   - state: an open MPS in Vidal form {Gamma^[i], Lambda^[i]} (Sec. II B);
 *   - one gate layer (Algorithm 1, loop body): on every gated bond at once,
 *     theta = Lambda_{i-1} Gamma_i Lambda_i Gamma_{i+1} Lambda_{i+1}, theta' = U theta,
 *     SVD theta' = U S V^dagger, Gamma_i <- Lambda_{i-1}^{-1} U, Lambda_i <- S,
 *     Gamma_{i+1} <- V^dagger Lambda_{i+1}^{-1} (Sec. II C);
 *   - the parallel compression keeps the chi' largest singular values of every
 *     bond (projector P_i, Sec. III B) and multiplies Lambda_i by
 *     nu_i = (1 - eps_i)^{-1/2} (Sec. III C, norm stabilisation);
 *   - g parallel trivial-simple-update steps (PtSU) follow: tSU on the paper's
 *     odd bonds, then on its even bonds (Sec. III D, IPMC of Sec. III E).
 *
 * Index conventions: sites s = 0..N-1; bond b = 0..N-2 joins sites b and b+1
 * (the paper's bond i is b = i-1).  Lambda_{-1} = Lambda_{N-1} = (1).  The
 * physical dimension is d = 2.  A two-site gate is a 4x4 complex matrix
 * U[(2 s0' + s1'), (2 s0 + s1)] with s0 the physical index of site b; gates
 * are passed as 32 doubles each: row-major, (re, im) interleaved.
 *
 * Memory ownership: the library never allocates device memory.  The caller
 * asks ptebd_required_bytes() for the sizes, allocates one state buffer and
 * one workspace buffer on the current device (256-byte aligned, e.g. through
 * the PyTorch caching allocator) and passes them to ptebd_create(); both must
 * stay valid until ptebd_destroy().  The handle itself lives in host memory
 * allocated by ptebd_create and freed by ptebd_destroy.
 *
 * Streams: every call runs on the stream given at create time (or set later
 * with ptebd_set_stream); calls that return results to the host synchronise
 * that stream, all others are asynchronous.
 *
 * Errors: every function returns an int status, 0 on success and a negative
 * PTEBD_ERR_* code otherwise; no C++ exception crosses the ABI.
 * ptebd_last_error() gives a text for the last failure of a handle.
 * Errors found on the device (non-finite values, a zero two-site tensor, a
 * discarded weight >= 1 in absolute mode, a Jacobi sweep limit, a bounded wait
 * that ran out) are latched in a device word and reported by the next
 * synchronising call (ptebd_sync, ptebd_norm, ptebd_get_*, ...).
 * When a bounded wait runs out, the CTA waits (bounded again) for its own bulk
 * copies before it returns; if even that wait runs out, copies into its shared
 * memory may still be in flight when it returns, and the state is marked
 * unusable: that report and every later call that would launch work or read
 * results return PTEBD_ERR_TIMEOUT until the state is destroyed (ptebd_reset
 * does not clear it).
 */
#ifndef PTEBD_H
#define PTEBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTEBD_OK                 0
#define PTEBD_ERR_INVALID       -1  /* bad argument (null pointer, range, parity) */
#define PTEBD_ERR_UNSUPPORTED   -2  /* d != 2, chi_max above the compiled limit */
#define PTEBD_ERR_MEMORY        -3  /* buffer too small or misaligned */
#define PTEBD_ERR_CUDA          -4  /* a CUDA runtime call failed */
#define PTEBD_ERR_OVERLAP       -5  /* two gated bonds share a site */
#define PTEBD_ERR_NUMERIC       -6  /* device-detected non-finite value / zero tensor / eps >= 1 */
#define PTEBD_ERR_NOT_CONVERGED -7  /* a Jacobi SVD reached its sweep limit */
#define PTEBD_ERR_SHAPE         -8  /* imported tensor dimensions do not match the bonds */
#define PTEBD_ERR_TIMEOUT       -9  /* a bounded device wait ran out */

/* Largest chi_max of this build: theta is at most 512 x 512. */
#define PTEBD_CHI_LIMIT 256

enum ptebd_precision {
    PTEBD_FP64 = 0,   /* complex128 Gamma and theta, FP64 everywhere */
    PTEBD_MIXED = 1   /* complex64 Gamma, theta and SVD rotations; FP64 Lambda,
                         nu, discarded weights, column norms and reductions */
};

/* Readings of the norm stabilisation (Sec. III C) for a gated bond whose
 * theta' has singular values S (S_kept: the chi_b kept ones):
 *   SCHMIDT  (default): the Schmidt spectrum of the normalised two-site
 *            wavefunction is S / |S| (Sec. II B); eps_b = |S_dropped|^2 / |S|^2,
 *            nu_b = (1 - eps_b)^(-1/2), Lambda_b <- nu_b S_kept / |S|;
 *   ABSOLUTE : eps_b = |S_dropped|^2 taken literally, Lambda_b <- nu_b S_kept;
 *   RELATIVE : eps_b = |S_dropped|^2 / |S|^2, Lambda_b <- nu_b S_kept.
 * All three coincide on a normalised canonical state (|S| = 1). */
enum ptebd_eps_mode {
    PTEBD_EPS_SCHMIDT = 0,
    PTEBD_EPS_ABSOLUTE = 1,
    PTEBD_EPS_RELATIVE = 2
};

typedef struct ptebd_config {
    int32_t n_sites;    /* N >= 2 */
    int32_t d;          /* local dimension, must be 2 */
    int32_t chi_max;    /* chi of Algorithm 1, 1..PTEBD_CHI_LIMIT */
    int32_t precision;  /* enum ptebd_precision */
    int32_t g;          /* PtSU steps run after every layer (0 = none) */
    int32_t eps_mode;   /* enum ptebd_eps_mode */
    double cutoff;      /* drop singular values <= cutoff * lambda_1 (>= 0) */
    double resolve;     /* PTEBD_MIXED only (ignored for PTEBD_FP64): complex64
                           singular values <= resolve * lambda_1 are not trusted
                           (rounding leaves up to about 5e-8 lambda_1 where the
                           exact spectrum has zeros); a negative value selects 1e-6.
                           When resolve > cutoff, a gated or tSU bond whose kept
                           count depends on such values (taken as real or as zero,
                           with the structural bound rank(theta') <=
                           rank(gate) chi_b) is recomputed in FP64 from the
                           stored Gamma: theta' formed in FP64, FP64 Jacobi,
                           truncation at the cutoff, Gamma rebuilt in FP64 and
                           stored as complex64.  Every other bond is decided by
                           the complex64 spectrum.  The configured cutoff is thus
                           applied to FP64-accurate singular values wherever it
                           decides the kept count.  When resolve <= cutoff nothing
                           is recomputed. */
} ptebd_config;

typedef struct ptebd_state ptebd_state;

/* Sizes of the two device buffers ptebd_create needs for this config.
 * workspace_bytes is the size that processes a whole layer in one pass;
 * any workspace of at least workspace_min_bytes works (layers are then split
 * into chunks of bonds).  Any output pointer may be NULL. */
int ptebd_required_bytes(const ptebd_config* cfg, size_t* state_bytes,
                         size_t* workspace_bytes, size_t* workspace_min_bytes);

/* Create a state in |0...0> (all bond dimensions 1, Sec. IV A) inside the
 * caller's device buffers.  stream is a cudaStream_t (NULL = legacy default
 * stream).  On success *out owns nothing on the device; destroy frees the host
 * handle only. */
int ptebd_create(const ptebd_config* cfg, void* state_mem, size_t state_bytes,
                 void* workspace, size_t workspace_bytes, void* stream,
                 ptebd_state** out);
int ptebd_destroy(ptebd_state* st);
int ptebd_set_stream(ptebd_state* st, void* stream);
int ptebd_reset(ptebd_state* st);                 /* back to |0...0>, counters cleared */
const char* ptebd_last_error(const ptebd_state* st);
int ptebd_get_config(const ptebd_state* st, ptebd_config* out);

/* One brickwork layer (Algorithm 1, loop body; Sec. II C and III B-E):
 * gates[j] acts on bond b = parity + 2 j for j < n_p = ceil((N - 1 - parity) / 2).
 * gates: n_p * 32 doubles (see the layout above), in host memory when
 * gates_on_device == 0, else in device memory on this GPU.  Asynchronous.
 * Runs the TEBD procedure with compression and nu on every gated bond, then
 * the config's g PtSU steps. */
int ptebd_apply_layer(ptebd_state* st, const double* gates, int32_t parity,
                      int32_t gates_on_device);

/* Same on an arbitrary set of pairwise non-adjacent bonds (compiled layers of
 * routed circuits, App. A).  bonds: n_bonds host int32 values in [0, N-2];
 * two bonds closer than 2 return PTEBD_ERR_OVERLAP. */
int ptebd_apply_bonds(ptebd_state* st, const int32_t* bonds, int32_t n_bonds,
                      const double* gates, int32_t gates_on_device);

/* g explicit PtSU steps (Sec. III D): tSU (identity gate skipped, no nu, same
 * truncation rule) on bonds 0, 2, 4, ... then on bonds 1, 3, 5, ...  */
int ptebd_regauge(ptebd_state* st, int32_t g);

/* Concurrency of a layer (no counterpart in the paper: a scheduling choice).
 * The bonds of a layer are split by site range into up to 16 chunks, each run
 * on a stream of its own; a chunk of the next half-step starts as soon as the
 * chunks on either side of it are done (a bond touches only its two sites and
 * the Lambdas next to them), so the tails of the SVD launches overlap with the
 * rest of the layer.  Results are bit-identical to one stream.  n = 0 (the
 * default) picks one chunk per 64 bonds of a brickwork layer, at most 8; n = 1
 * runs everything on the state's stream.  Chunking is also skipped when the
 * workspace holds fewer slots than the chunks need, while per-kernel timing is
 * on, and for ptebd_apply_bonds lists that are not in ascending order. */
int ptebd_set_chunk_streams(ptebd_state* st, int32_t n);

/* Precision of the PtSU steps (Sec. III D) of a PTEBD_MIXED state.
 * PTEBD_MIXED (the default): tSU runs in complex64 like the gate updates, with
 * the FP64 resolution of undecided bonds; the orthogonality of the regauged
 * Gamma is then limited by the complex64 Jacobi (about 8 sqrt(rows) 2^-24).
 * PTEBD_FP64: every tSU bond runs in FP64 (theta formed in FP64 from the
 * stored complex64 Gamma, FP64 orthogonalisation and Jacobi, Gamma rebuilt in
 * FP64), so the regauged state is canonical to the rounding of its complex64
 * storage; it costs the FP64 pipe's time (about 1/64 of the FP32 rate here).
 * No effect on a PTEBD_FP64 state; PTEBD_ERR_UNSUPPORTED when the state has
 * no FP64 workspace (config resolve <= cutoff). */
int ptebd_set_regauge_precision(ptebd_state* st, int32_t precision);

/* Polish sweep of the complex64 Jacobi SVDs (the SVD of the TEBD procedure,
 * Sec. II C; no effect on complex128 SVDs).  The sweeps stop when no pair has
 * |a^H b| > 8 sqrt(rows) 2^-24 |a| |b| (or every rotation of a sweep was
 * small), which leaves the kept singular vectors orthogonal to about that
 * level; the truncated two-site state then carries a relative error of a few
 * 1e-5.  mode 1: the gated SVDs end with one more sweep at 2 sqrt(rows)
 * 2^-24, mode 2 (the default): the tSU SVDs as well, mode 3: the tSU SVDs
 * only, mode 0: none.  Measured on one saturated layer with PtSU (N = 256,
 * chi = 256) against the FP64 path: 1 - F = 5.6e-7 (mode 0), 4.5e-7 (mode 1),
 * 4.7e-8 (mode 2) for 9% more time; at N = 1024, chi = 256: 3.2e-7 (mode
 * 2), 1.7e-6 (mode 3, 4% faster), 4.9e-6 (mode 0).  PTEBD_ERR_INVALID for
 * other modes. */
int ptebd_set_svd_polish(ptebd_state* st, int32_t mode);

/* Tensor cores for a PTEBD_MIXED state (no counterpart in the paper: a
 * choice of arithmetic unit).  When chi_max rounded up (16 * 2^k) is at
 * least 64, enable = 1 (the default; any value other than 0 and 2): theta' =
 * U theta and the GEMM factor of the Gamma rebuild of gated bonds are formed by
 * tcgen05.mma kind::tf32 with FP32 accumulation in tensor memory, operands
 * split as hi + lo TF32 pairs and multiplied hi*hi + hi*lo + lo*hi (FP32
 * accuracy), the cross terms in accumulators of their own; enable = 2: the
 * tSU steps' theta, projection M^dag = theta^dag U_X and Gamma GEMM as well;
 * enable = 0: FP32 FMAs on the CUDA cores.  The tensor cores' accumulation
 * rounds toward zero (sums shrink by about 2.5e-8 relative per K step of 8);
 * the accumulators restart every 2 K chunks of 16 complex values and the
 * partial results are added in FP32 registers with round-to-nearest, which
 * bounds the shrinkage at about 2e-7 relative per product whatever chi is.  A
 * gated bond's Schmidt reading renormalises it away; a tSU step keeps S as it
 * is, and over the bonds of one PtSU step at N = 1024, chi = 256 it moved the
 * norm of the state by 5.4e-4 (mode 2), hence mode 1 as the default.  The
 * tensor-core and CUDA-core paths round differently (both to FP32 accuracy).
 * No effect on PTEBD_FP64 states. */
int ptebd_set_tensor_cores(ptebd_state* st, int32_t enable);

/* Jacobi block width of the handle's SVDs (no counterpart in the paper: a
 * launch choice): the columns held in registers by one CTA, one per warp.
 * complex64: 16 (default) or 8; complex128: always 8.  0 selects the default.
 * Results are bit-identical run to run for a given width; two widths visit
 * the column pairs in different orders and so differ by rounding (both within
 * the SVD's accuracy).  complex64 width 8 runs two CTAs (two bonds) per SM;
 * measured at N = 1024, chi = 256 it is 7% slower than width 16, and the
 * autotuner picks it for some small-chi keys.  PTEBD_ERR_INVALID for other
 * widths. */
int ptebd_set_jacobi_width(ptebd_state* st, int32_t nw);

/* PtSU after a gated layer on bonds 0, 2, 4, ... (the paper's odd bonds; a
 * PtSU step, Sec. III D, is tSU on those bonds and then on bonds 1, 3, 5,
 * ...).  Right after such a layer every one of those bonds is in Schmidt form
 * (Gamma_b = Lambda_{b-1}^-1 U, Gamma_{b+1} = V^dag Lambda_{b+1}^-1, the
 * neighbouring Lambdas untouched), so the tSU two-site tensor there is
 * U Lambda_b V^dag and the first half-step of the first PtSU step returns the
 * state unchanged (up to rounding).  enable != 0 (the default): that half-step
 * is left out of ptebd_apply_layer with g >= 1 and parity 0; enable = 0: it
 * runs.  Layers of parity 1, explicit bond lists and ptebd_regauge always run
 * every half-step.  No counterpart in the paper: a scheduling choice that
 * drops an identity. */
int ptebd_set_ptsu_shortcut(ptebd_state* st, int32_t enable);

/* Columns of the complex64 Jacobi register block per warp at block width 16
 * (no counterpart in the paper: a scheduling choice).  pairs = 1 (the
 * default): 16 warps, one I column each, one column pair a round; pairs = 2:
 * 8 warps, each holding two I columns and rotating two independent column
 * pairs a round with their instruction streams interleaved.  Matrices of
 * more than 32 rows see their column pairs in the same order as with
 * pairs = 1; smaller ones run with 8-column blocks, so results differ from
 * pairs = 1 by rounding (both bit-identical run to run).  Measured at N = 1024,
 * chi = 256: the SVD takes 19% longer than with pairs = 1 (half the warps,
 * issue activity 38% against 51%), so it is an autotuner candidate, not the
 * default.  Width 8 and complex128 ignore it.  PTEBD_ERR_INVALID for other
 * values. */
int ptebd_set_jacobi_pairs(ptebd_state* st, int32_t pairs);

/* Autotuner (no counterpart in the paper: a scheduling choice of the library).
 * Times every candidate launch configuration on the state's own next layer
 * (the gates and parity a ptebd_apply_layer call would get, with the config's
 * PtSU steps): Jacobi block width and columns per warp (complex64: 16 with
 * one or two, 8 with one) x bond chunks (1, 2,
 * 4, 8, 12, 16, those the workspace can run concurrently); each candidate runs
 * twice from the saved state and the second run is timed with CUDA events on
 * the handle's stream.  The state is copied into `scratch` (device memory,
 * 256-byte aligned, at least state_bytes of ptebd_required_bytes, owned by
 * the caller) first and restored before every run and at the end, so the call
 * leaves the state, its counters and its layer count as it found them.  The
 * fastest configuration is set on the handle and remembered for the process
 * under (chi_max padded, precision, bit length of N - 1, g): later
 * ptebd_create calls with the same key start with it.  best (may be NULL, else
 * 5 doubles): [block width, chunks, ms of the best, ms of the configuration
 * the handle had (-1 if it was not among the candidates), columns per warp].
 * Synchronous. */
int ptebd_autotune(ptebd_state* st, const double* gates, int32_t parity, int32_t gates_on_device,
                   void* scratch, size_t scratch_bytes, double* best);

/* Test of the failure detection (no counterpart in the paper).  With enable
 * != 0, in every later SVD launch one warp of each CTA waits, in its first
 * hand-off, for a round count that nothing ever writes, under a limit of 2^20
 * clock cycles instead of 2^31: the wait runs out, the CTA's other warps see
 * its abort flag and stop, the CTA waits for its own copies in flight, latches
 * DERR_TIMEOUT and returns, and the next synchronising call reports
 * PTEBD_ERR_TIMEOUT.  Nothing faults or hangs; the state's tensors are left
 * half-updated (ptebd_reset or an import restores a usable state).  enable = 0
 * turns it off. */
int ptebd_test_wait_timeout(ptebd_state* st, int32_t enable);

/* Wait for all work of the handle and report latched device errors. */
int ptebd_sync(ptebd_state* st);

/* Full contractions (exact for any MPS, canonical or not; synchronous).
 * norm: n = || |Psi> ||.  overlap: <a|b> as out[0] + i out[1] (a and b must
 * have the same N and live on the same device).  expect: <Psi|O|Psi>/<Psi|Psi>
 * for a one-site operator O (2x2, 8 doubles, O[s', s] row-major interleaved)
 * on `site`, and expect2 for a two-site operator (4x4 in the gate layout) on
 * sites (site, site+1).  The transfer matrices are accumulated in FP64. */
int ptebd_norm(ptebd_state* st, double* out);
int ptebd_overlap(ptebd_state* a, ptebd_state* b, double out[2]);
int ptebd_expect(ptebd_state* st, int32_t site, const double* op, double out[2]);
int ptebd_expect2(ptebd_state* st, int32_t site, const double* op, double out[2]);

/* State interchange (host buffers; synchronous).
 * get_chi: N-1 bond dimensions.  get_lambda: Lambda_b (chi_b doubles; the
 * buffer must hold chi_max).  get_site / set_site: Gamma_s as
 * (2, chi_{s-1}, chi_s) complex128, C order, interleaved (re, im); set_site
 * requires chi_l == chi_{s-1} and chi_r == chi_s (PTEBD_ERR_SHAPE otherwise).
 * set_lambda sets chi_b = k and Lambda_b (k values, descending expected). */
int ptebd_get_chi(ptebd_state* st, int32_t* chi_out);
int ptebd_get_lambda(ptebd_state* st, int32_t bond, double* out, int32_t* k);
int ptebd_get_site(ptebd_state* st, int32_t site, int32_t* chi_l, int32_t* chi_r,
                   double* gamma_out);
int ptebd_set_lambda(ptebd_state* st, int32_t bond, int32_t k, const double* values);
int ptebd_set_site(ptebd_state* st, int32_t site, int32_t chi_l, int32_t chi_r,
                   const double* gamma);

/* Metrics (synchronous).  eps_total = sum over all gated bonds of all layers
 * so far of eps_b (Theorem 1's epsilon); log_nu_total = sum of ln nu_b, so
 * prod nu_i = exp(log_nu_total) (Sec. III C, n* = n prod nu_i).  Per-bond
 * values of the most recent gate update of each bond: eps_b, nu_b and the
 * number of singular values of its theta' (rank_in = min(rows, cols)); a bond
 * never gated holds eps 0, nu 1, rank_in 0.  Any output pointer may be NULL. */
int ptebd_trunc_error(ptebd_state* st, double* eps_total, double* log_nu_total);
int ptebd_bond_stats(ptebd_state* st, double* eps, double* nu, int32_t* rank_in);
/* Jacobi sweeps of the most recent SVD of every bond (tSU or gate) and the
 * number of layers applied so far. */
int ptebd_svd_sweeps(ptebd_state* st, int32_t* sweeps, int32_t* layers);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch of the layer kernels.  ptebd_timing(st, 1) clears the counters
 * and starts recording, ptebd_timing(st, 0) stops.  ptebd_timing_read
 * (synchronous) returns, for each kernel kind (PTEBD_K_*), the summed device
 * time in milliseconds and the number of launches; n_kinds entries are
 * written (at most PTEBD_K_COUNT). */
#define PTEBD_K_THETA 0     /* theta' = U theta (Sec. II C) */
#define PTEBD_K_SVD 1       /* one-sided Jacobi SVD */
#define PTEBD_K_TRUNCATE 2  /* sort, projector P_b, eps_b, nu_b, Lambda_b */
#define PTEBD_K_GAMMA 3     /* Gamma_b and Gamma_{b+1} rebuild */
#define PTEBD_K_REDUCE 4    /* per-layer eps / ln nu sums */
#define PTEBD_K_FACTOR 5    /* tSU: X factor and theta^dag U_X */
#define PTEBD_K_RESOLVE 6   /* PTEBD_MIXED: the FP64 pass over undecided bonds */
#define PTEBD_K_COUNT 7
int ptebd_timing(ptebd_state* st, int32_t enable);
int ptebd_timing_read(ptebd_state* st, double* ms, int32_t* launches, int32_t n_kinds);

/* Work counters accumulated on the device since create / reset (synchronous):
 * out[0] = sum over every SVD of (sweeps x cols (cols - 1) / 2 x rows), the
 *          column-pair-row visits of the one-sided Jacobi (its nominal cost is
 *          28 real flops per visit: an 8-flop complex dot and a 20-flop
 *          complex rotation of two entries);
 * out[1] = sum over every theta' of 32 chi_{b-1} chi_b chi_{b+1} (the real
 *          flops of the four complex products X_s Y_t);
 * out[2] = Jacobi rotations actually applied;
 * out[3] = Jacobi sweeps summed over every SVD; out[4] = number of SVDs;
 * out[5..7] = the same three counts (visits, sweeps, SVDs) for the Jacobi runs
 * of the tSU steps alone (out[0..7] count the state's own precision only);
 * out[8] = bonds of a PTEBD_MIXED state computed in FP64 (by the resolution,
 * gated and tSU, and by an FP64 regauge), out[9] = the Jacobi visits of
 * those FP64 runs.
 * n entries are written (<= 16; out[10..15] are reserved and read 0). */
int ptebd_work_counters(ptebd_state* st, uint64_t* out, int32_t n);

/* The end of Algorithm 1.  ptebd_canonicalize runs the PtSU steps that
 * Theorem 4 shows are enough to bring any MPS to canonical form: N/2 steps for
 * even N, (N-1)/2 for odd N (asynchronous; the state and its norm are
 * unchanged up to the cutoff).  ptebd_sample draws n_samples bit strings from
 * |Psi|^2 / <Psi|Psi> exactly for any MPS (canonical or not): the left
 * environments of every site are contracted in FP64, then the sites are drawn
 * from the right end, site s of sample k taking 0 when
 * uniforms[k * N + s] < P(0 | the bits already drawn to its right).
 * uniforms: host, n_samples * N doubles in [0, 1); bits: host, n_samples * N
 * int32 (0 or 1).  Scratch: `workspace` (device memory, 256-byte aligned,
 * owned by the caller, workspace_bytes long) or, when it is NULL, the state's
 * own workspace; ptebd_sample_workspace_bytes gives the size needed (about
 * N * chip^2 * 16 bytes, chip = chi_max rounded up to 16 * 2^k), and
 * ptebd_sample returns PTEBD_ERR_MEMORY when the scratch is smaller.
 * Synchronous. */
int ptebd_canonicalize(ptebd_state* st);
int ptebd_sample_workspace_bytes(const ptebd_state* st, int32_t n_samples, size_t* bytes);
int ptebd_sample(ptebd_state* st, int32_t n_samples, const double* uniforms, int32_t* bits, void* workspace,
                 size_t workspace_bytes);

/* Batched serving of independent states (many circuits with uneven N,
 * chi_max and precision): ptebd_batch_create groups n distinct states, which
 * must outlive the batch.  ptebd_batch_apply_layer applies to every state i
 * one layer of parity parities[i] with gates[i] (host memory, or device memory
 * when gates_on_device != NULL and gates_on_device[i] != 0; parity -1 leaves
 * state i untouched in this call, for circuits of uneven depth), followed by that
 * state's g PtSU steps: the same work as ptebd_apply_layer, recorded as
 * parallel branches of one CUDA graph (one graph per parity pattern, cached by
 * the batch) so that small states run side by side.  Asynchronous: every
 * state's stream waits for the graph; errors latched on the device are
 * reported by each state's next synchronising call. */
typedef struct ptebd_batch ptebd_batch;
int ptebd_batch_create(ptebd_state* const* states, int32_t n, ptebd_batch** out);
int ptebd_batch_destroy(ptebd_batch* b);
const char* ptebd_batch_last_error(const ptebd_batch* b);
int ptebd_batch_apply_layer(ptebd_batch* b, const double* const* gates, const int32_t* parities,
                            const int32_t* gates_on_device);

/* Batched SVD with the layer's one-sided Jacobi kernel (the SVD step of the
 * TEBD procedure, Sec. II C, on caller matrices; used for SVD-only
 * benchmarks and tests).
 * precision: PTEBD_FP64 (complex128 matrices) or PTEBD_MIXED (complex64).
 * a: device memory, `batch` matrices of rows x cols, column-major, leading
 *    dimension lda >= rows, matrix i at element offset i * lda * cols;
 *    requires cols <= rows <= 2 * PTEBD_CHI_LIMIT and rows even.
 * sigma: device, batch x cols doubles, the singular values of each matrix in
 *    descending order (FP64 norms of the rotated columns).
 * u: device or NULL; when given, batch x (ldu x cols) complex of the input
 *    type, column k = the left singular vector of sigma[k] (zero if sigma[k] = 0).
 * Accuracy: the columns of U are orthogonal to about tol = k sqrt(rows) u
 *    (k = 4 and u = 2^-53 for complex128; k = 8 and u = 2^-24 for complex64).
 *    The sweeps stop after a sweep in which no pair had |cos| > tol, or, for
 *    complex64, after a sweep whose rotated pairs all had cos^2 < 256 tol^2
 *    (the sweep after such a sweep was measured to find no pair above
 *    1.04 tol^2).
 * workspace: device, 256-byte aligned, at least ptebd_svd_workspace_bytes.
 * The input is not modified.  Runs on `stream` (cudaStream_t).  check != 0
 * synchronises the stream and reports device errors (sweep limit, non-finite
 * values, a wait that ran out); check == 0 returns at once. */
int ptebd_svd_workspace_bytes(int32_t precision, int32_t batch, int32_t rows, int32_t cols,
                              size_t* bytes);
int ptebd_svd_batched(int32_t precision, int32_t batch, int32_t rows, int32_t cols,
                      const void* a, int32_t lda, double* sigma, void* u, int32_t ldu,
                      void* workspace, size_t workspace_bytes, void* stream, int32_t check);

/* Allocation-free variant of ptebd_svd_batched (the paper has no
 * counterpart: this is a convenience of the library, not part of the method).
 * Some callers cannot allocate device memory at all, for example code that a
 * host framework hands only its input and output buffers, or code that must
 * not call cudaMalloc / cudaFree because those calls synchronise the device or
 * are not allowed where it runs.  This entry point takes the same arguments as
 * ptebd_svd_batched minus the workspace and keeps its scratch in a fixed
 * device array inside the library of PTEBD_NOALLOC_SCRATCH_BYTES bytes; every
 * GPU that loads the library holds that array until the process exits.  It
 * calls no allocating routine.
 * - A batch whose scratch (ptebd_svd_workspace_bytes) exceeds the array is
 *   rejected with PTEBD_ERR_MEMORY (e.g. at most 15 complex64 or 7 complex128
 *   matrices of 512 x 512 per call).
 * - `stream` must belong to the current device (PTEBD_ERR_INVALID otherwise);
 *   every call looks the array's device address up on that device
 *   (cudaGetSymbolAddress), so a context the caller tears down and re-creates
 *   is handled.
 * - The first call on each device loads the library's module holding the
 *   array (the CUDA runtime loads modules lazily), which reserves the array
 *   on that device: that call can fail with PTEBD_ERR_CUDA when the device is
 *   out of memory, and it should be made before any stream capture, since
 *   loading a module is not allowed while a stream is capturing.
 * - All calls share the array and it keeps the previous call's contents (the
 *   parts that must start at zero are cleared on every call): calls whose
 *   work overlaps on the GPU (two streams, two host threads) race on it and
 *   must be serialised by the caller. */
#define PTEBD_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int ptebd_svd_batched_noalloc(int32_t precision, int32_t batch, int32_t rows, int32_t cols,
                              const void* a, int32_t lda, double* sigma, void* u, int32_t ldu,
                              void* stream, int32_t check);

/* Measured arithmetic peaks of this GPU (the paper has no counterpart: these
 * are the roofline denominators of the kernels that run on the FP32 and FP64
 * pipes).  kind 0: scalar FP32 FMA (fma.rn.f32); 1: packed FP32 FMA
 * (fma.rn.f32x2, two FP32 lanes per instruction); 2: FP64 FMA.  One launch of
 * 8 x (SM count) blocks of 256 threads, each thread running iters x 128 FMAs
 * on 8 independent register chains (no memory traffic in the loop), after one
 * untimed warm-up launch; *tflops = its flops (2 per FMA lane) over the CUDA
 * event time on `stream`, *ms (may be NULL) = that time.  Synchronous.
 * scratch: device memory of at least 8 x SMs x 256 x 8 bytes, which receives
 * the per-thread results (written so that the arithmetic is kept).
 * PTEBD_ERR_MEMORY when it is smaller. */
int ptebd_alu_peak(int32_t kind, int32_t iters, void* scratch, size_t scratch_bytes, void* stream,
                   double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* PTEBD_H */
