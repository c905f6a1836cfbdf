// Two-site tensor theta' = U (Lambda_{b-1} Gamma_b Lambda_b Gamma_{b+1} Lambda_{b+1})
// (the TEBD procedure, Sec. II C of arXiv:2312.02667) on the 5th-generation
// tensor cores, for complex64 states: tcgen05.mma kind::tf32 with FP32
// accumulators in tensor memory, FP32 accuracy kept by the 3xTF32 split.
//
// theta, as a (2 chi_{b-1}) x (2 chi_{b+1}) matrix with rows (s, alpha) and
// columns (t, gamma), is one product X Y: X = [X_0; X_1] with
// X_s = diag(Lambda_{b-1}) Gamma_b^s diag(Lambda_b), and Y = [Y_0, Y_1] with
// Y_t = Gamma_{b+1}^t diag(Lambda_{b+1}); the inner dimension is chi_b.  A CTA
// computes the 64 x 64 (alpha, gamma) tile of all four theta_{st} as one
// 128 x 128 (rows s * 64 + alpha, columns t * 64 + gamma) block, so that the
// gate mix theta'_{s't'} = sum_{st} U[s't', st] theta_{st} is its epilogue.
//
// Complex arithmetic on the real tensor cores: with the real and imaginary
// parts of X interleaved along K (the complex64 storage order), the real part
// of theta is X' B_re^T and the imaginary part X' B_im^T, where row n of
// B_re holds (Re Y, -Im Y) and row n of B_im holds (Im Y, Re Y) pairwise.
//
// 3xTF32: every operand value v is split into hi = v rounded to TF32 and
// lo = v - hi (exact in FP32); a product is accumulated as
// hi*hi + hi*lo + lo*hi, leaving out lo*lo (about 2^-22 relative) - FP32
// accuracy, which the mixed path needs (a single TF32 product changes
// theta by 1e-3 relative).  The hi*hi products go to one FP32 accumulator and
// the two cross terms to a second one, added in the epilogue: the tensor
// cores' FP32 accumulation does not round to nearest (measured on GB300 it
// shrinks every sum by about 2.5e-8 relative per MMA, always in the same
// direction), and a separate accumulator of the small cross terms keeps that
// shrinkage of the large hi*hi sum from being applied again to every term.
// Four accumulators of 128 x 128 FP32 (real, imaginary, and their
// corrections): all 512 columns of tensor memory.
//
// Operands are staged by all threads into shared memory in the K-major,
// 128-byte-swizzled layout that the MMA descriptors describe (rows of 32 FP32
// values = 128 bytes, groups of 8 rows = 1024 bytes), scaled by the Lambdas
// and split on the way (a TMA copy could not do either); two stages of 96 KB,
// each holding a K chunk of 16 complex values: while the tensor cores work on
// one, the threads fill the other.  One thread issues the MMAs and commits
// them to the stage's mbarrier; every wait on an mbarrier is bounded.
#include <cstdint>

#include "ptebd_internal.h"

namespace ptebd {
namespace {

// ------------------------------------------------------------------ PTX --
__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void tc_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// about 2^31 SM cycles (~1 s) at most
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long start = clock64();
    while (!tc_mbar_try_wait(bar, parity))
        if (clock64() - start > (1ll << 31)) return false;
    return true;
}

// tensor memory: allocation by one whole warp; the address is written to smem
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem_tc() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile with the 128-byte
// swizzle: start address >> 4 (bits 0-13), leading byte offset 16 >> 4 (unused
// by swizzled K-major layouts), stride byte offset 1024 >> 4 between groups of
// 8 rows (bits 32-45), descriptor version 1 (bits 46-47), base offset 0 (tile
// bases are 1024-aligned), swizzle mode 2 = 128B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::tf32: dense, D = F32 (bits 4-5 = 1), A and
// B = TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A[smem] B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// the mbarrier gets one arrival when every MMA issued so far by this thread is complete
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// v = hi + lo with hi = v rounded to TF32 (10 explicit mantissa bits) and lo
// the exact remainder
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    hi = __uint_as_float(h);
    lo = v - hi;
}

// byte offset of FP32 element (row, k), k < 32, in a [rows x 32] K-major tile
// with the 128-byte swizzle (16-byte chunk index XOR row mod 8)
__device__ __forceinline__ uint32_t sw128(int row, int k) {
    const uint32_t lin = (uint32_t)row * 128u + (uint32_t)k * 4u;
    return lin ^ (((lin >> 7) & 7u) << 4);
}

// ----------------------------------------------------------------- kernel --
constexpr int kTcThreads = 256;
constexpr uint32_t kTile = 128u * 128u;  // bytes of one [128 rows x 32 FP32] operand tile
constexpr uint32_t kStage = 6u * kTile;  // A hi/lo, B_re hi/lo, B_im hi/lo
constexpr int kThPitch = 129;            // floats between columns of the epilogue staging
constexpr uint32_t kIdesc = idesc_tf32(128, 128);
// After the two stages: 64 bytes of mbarriers and TMEM address, then the small
// arrays of a kernel (theta: Lambdas and gate; Gamma: column maps and scales).
constexpr size_t kThetaExtra = 64 + (64 + 64 + PTEBD_CHI_LIMIT) * sizeof(float) + 16 * sizeof(float2);
constexpr size_t kGammaExtra = 64 + 2 * 128 * sizeof(int) + 2 * 128 * sizeof(float);
constexpr size_t kTcExtra = kThetaExtra > kGammaExtra ? kThetaExtra : kGammaExtra;
// the stages, the small arrays and 1 KB of slack for aligning the base to 1024
constexpr size_t kTcSmem = 2 * (size_t)kStage + kTcExtra + 1024;
static_assert(kTcSmem <= 227 * 1024, "tensor-core kernels exceed the shared memory of a CTA");
static_assert(2 * 128 * kThPitch * sizeof(float) <= 2 * (size_t)kStage, "epilogue staging exceeds the stages");

// The operand stores of one K chunk: element (row, kk) of A, as hi and lo
// TF32 parts (tiles 0, 1); row n of B_re and B_im (tiles 2, 3 and 4, 5), each
// given as the FP32 pair it holds at K indices 2 kk and 2 kk + 1.
__device__ __forceinline__ void put_a(unsigned char* S, int r, int kk, float2 v) {
    float hx, lx, hy, ly;
    split_tf32(v.x, hx, lx);
    split_tf32(v.y, hy, ly);
    const uint32_t o = sw128(r, 2 * kk);
    *reinterpret_cast<float2*>(S + o) = make_float2(hx, hy);
    *reinterpret_cast<float2*>(S + kTile + o) = make_float2(lx, ly);
}
__device__ __forceinline__ void put_b(unsigned char* S, int n, int kk, float2 bre, float2 bim) {
    float h0, l0, h1, l1, h2, l2, h3, l3;
    split_tf32(bre.x, h0, l0);
    split_tf32(bre.y, h1, l1);
    split_tf32(bim.x, h2, l2);
    split_tf32(bim.y, h3, l3);
    const uint32_t o = sw128(n, 2 * kk);
    *reinterpret_cast<float2*>(S + 2 * kTile + o) = make_float2(h0, h1);
    *reinterpret_cast<float2*>(S + 3 * kTile + o) = make_float2(l0, l1);
    *reinterpret_cast<float2*>(S + 4 * kTile + o) = make_float2(h2, h3);
    *reinterpret_cast<float2*>(S + 5 * kTile + o) = make_float2(l2, l3);
}

// Barriers and tensor memory of a CTA (512 columns: the four accumulators).
__device__ __forceinline__ uint32_t tc_begin(uint64_t* bar, uint32_t* tmem_slot) {
    if (threadIdx.x == 0) {
        tc_mbar_init(&bar[0], 1);
        tc_mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *tmem_slot;
}
__device__ __forceinline__ void tc_end(uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 512);
}

// The MMA pipeline of one CTA over nk K chunks of 16 complex values, two
// stages.  Each thread owns 8 elements of A and 8 of B per chunk:
// fetch(kc, ra, rb) reads chunk kc from global memory into registers and
// put(S, ra, rb) stores them into stage S through put_a / put_b.  The fetch
// of chunk kc + 1 is issued before the MMAs of chunk kc and before the wait
// for the stage it will fill, so its memory latency overlaps the tensor-core
// work.  One thread issues the chunk's 24 MMAs (3xTF32 for the real and the
// imaginary part, 4 K steps of 8 FP32 values: hi*hi into the accumulators at
// columns 0 and 128, the cross terms into the corrections at 256 and 384) and
// commits them to the stage's mbarrier, which the threads wait on before they
// refill that stage.
//
// The accumulators start afresh every kFlush chunks: at the end of such a group
// the threads wait for its MMAs and add main + correction into FP32 sums held
// in registers (round to nearest).  The tensor cores' accumulation rounds
// toward zero (about 2.5e-8 relative per K step, always shrinking), so a sum
// over the whole K dimension would shrink by that much per step (1.6e-6 at
// K = 256 complex); over a group of 8 K steps it is 2e-7, and adding the groups
// in registers adds no bias.  sum[c] of a thread: TMEM lane (row) 32 (warp & 3)
// + lane, column c of the real (warps 0-3) or imaginary (warps 4-7) result.
// Returns false when a wait ran out (the sums cannot be trusted then).
constexpr int kFlush = 2;
template <typename Fetch, typename Put>
__device__ bool tc_pipeline(unsigned char* sm, uint64_t* bar, uint32_t tmem, int nk, float (&sum)[128], Fetch&& fetch,
                            Put&& put) {
    const uint32_t d_re = tmem, d_im = tmem + 128, c_re = tmem + 256, c_im = tmem + 384;
    const int warp = threadIdx.x >> 5, kind = warp >> 2;
    const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kind * 128);
#pragma unroll
    for (int c = 0; c < 128; ++c) sum[c] = 0.f;
    float2 ra[8], rb[8];
    if (nk > 0) fetch(0, ra, rb);
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc & 1;
        unsigned char* S = sm + st * kStage;
        // (a flush already waited for chunk kc - 2 when it ended a group: the
        // phase is complete and the wait returns at once)
        if (kc >= 2 && !tc_mbar_wait(&bar[st], (uint32_t)((kc - 2) >> 1) & 1u)) ok = false;
        if (!__syncthreads_and(ok)) { ok = false; break; }
        put(S, ra, rb);
        if (kc + 1 < nk) fetch(kc + 1, ra, rb);  // in flight during the MMAs below
        fence_async_smem_tc();  // the tensor cores read the stores through the async proxy
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t base = su32(S);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t off = 32u * ks;
                const uint64_t ah = sdesc_sw128(base + off), al = sdesc_sw128(base + kTile + off);
                const uint64_t rh = sdesc_sw128(base + 2 * kTile + off), rl = sdesc_sw128(base + 3 * kTile + off);
                const uint64_t ih = sdesc_sw128(base + 4 * kTile + off), il = sdesc_sw128(base + 5 * kTile + off);
                const uint32_t acc = (kc % kFlush != 0 || ks > 0) ? 1u : 0u;
                mma_tf32(d_re, ah, rh, kIdesc, acc);
                mma_tf32(c_re, ah, rl, kIdesc, acc);
                mma_tf32(c_re, al, rh, kIdesc, 1u);
                mma_tf32(d_im, ah, ih, kIdesc, acc);
                mma_tf32(c_im, ah, il, kIdesc, acc);
                mma_tf32(c_im, al, ih, kIdesc, 1u);
            }
            mma_commit(&bar[st]);
        }
        if (kc % kFlush == kFlush - 1 || kc == nk - 1) {
            if (!tc_mbar_wait(&bar[st], (uint32_t)(kc >> 1) & 1u)) ok = false;
            if (!__syncthreads_and(ok)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int cb = 0; cb < 8; ++cb) {
                float v[16], c[16];
                tmem_ld16(lanes + (uint32_t)(16 * cb), v);
                tmem_ld16(lanes + 256u + (uint32_t)(16 * cb), c);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[16 * cb + i] += v[i] + c[i];
            }
            tc_fence_before();
            __syncthreads();  // the next group's first MMAs overwrite the accumulators
        }
    }
    return ok;
}

// The sums of tc_pipeline into shared memory: re[c * kThPitch + r] and
// im[c * kThPitch + r] for the 128 x 128 tile (rows r = TMEM lanes).
__device__ __forceinline__ void stage_sums(const float (&sum)[128], float* re, float* im) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane;
    float* dst = (warp >> 2) ? im : re;
#pragma unroll
    for (int c = 0; c < 128; ++c) dst[c * kThPitch + row] = sum[c];
}

// grid (chip / 64, chip / 64, count), 256 threads, kTcSmem bytes of dynamic smem.
// Same outputs as k_theta<float, float2>: dims of the slot (block (0, 0)), the
// work counter, theta' (or its adjoint) in w and w0 (w only for a gated bond).
__global__ void __launch_bounds__(kTcThreads, 1) k_theta_tc(LayerArgs<float> a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kStage);  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    float* sL = reinterpret_cast<float*>(sm + 2 * kStage + 64);
    float* sR = sL + 64;
    float* sM = sR + 64;
    float2* ug = reinterpret_cast<float2*>(sM + PTEBD_CHI_LIMIT);

    const int j = blockIdx.z;
    const int b = a.bonds[j];
    const int chip = a.chip;
    const int tid = threadIdx.x;
    if (b < 0 || b > a.n_sites - 2 || a.chi[b] < 1 || a.chi[b] > chip || a.chi[b + 1] < 1 ||
        a.chi[b + 1] > chip || a.chi[b + 2] < 1 || a.chi[b + 2] > chip) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
            int32_t* d = a.dims + j * kDims;
            for (int q = 0; q < kDims; ++q) d[q] = 0;
            d[D_TALL] = 1;
            atomicOr(a.err, DERR_BADARG);
        }
        return;
    }
    const int cl = a.chi[b], cm = a.chi[b + 1], cr = a.chi[b + 2];
    const bool tall = a.mode == 0 && cl >= cr;
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        int32_t* d = a.dims + j * kDims;
        d[D_CL] = cl; d[D_CM] = cm; d[D_CR] = cr; d[D_TALL] = tall ? 1 : 0; d[D_BOND] = b;
        d[D_K] = 0;
        d[D_REFINE] = 0;
        d[D_COND] = 0;
        if (a.mode == 0) { d[D_ROWS] = tall ? 2 * cl : 2 * cr; d[D_COLS] = tall ? 2 * cr : 2 * cl; }
        else { d[D_ROWS] = 2 * cr; d[D_COLS] = cm; }
        atomicAdd(&a.work[1], 32ull * (unsigned long long)cl * (unsigned long long)cm * (unsigned long long)cr);
    }
    const int a0 = blockIdx.x * 64, g0 = blockIdx.y * 64;
    if (a0 >= cl || g0 >= cr) return;  // uniform over the CTA, before any allocation

    const size_t slice = (size_t)chip * chip;
    const float2* G0 = static_cast<const float2*>(a.gamma) + (size_t)b * 2 * slice;
    const float2* G1 = static_cast<const float2*>(a.gamma) + (size_t)(b + 1) * 2 * slice;
    {
        const double* lL = a.lam + (size_t)b * chip;
        const double* lM = a.lam + (size_t)(b + 1) * chip;
        const double* lR = a.lam + (size_t)(b + 2) * chip;
        if (tid < 64) sL[tid] = (a0 + tid < cl) ? (float)lL[a0 + tid] : 0.f;
        else if (tid < 128) sR[tid - 64] = (g0 + tid - 64 < cr) ? (float)lR[g0 + tid - 64] : 0.f;
        for (int q = tid; q < cm; q += kTcThreads) sM[q] = (float)lM[q];
        if (a.gates != nullptr && tid >= 128 && tid < 144) {
            const double* gp = a.gates + (size_t)j * 32 + 2 * (tid - 128);
            ug[tid - 128] = make_float2((float)gp[0], (float)gp[1]);
        }
    }
    const uint32_t tmem = tc_begin(bar, tmem_slot);
    const int nk = (cm + 15) / 16;  // K chunks of 16 complex values
    float sum[128];
    // element i of a thread: A (r = e & 127, kk = e >> 7), B (kk = e & 15, n = e >> 4), e = tid + 256 i;
    // fetch loads and scales (A: X_s = Lambda_{b-1} Gamma_b^s Lambda_b; B: Y_t = Gamma_{b+1}^t Lambda_{b+1}),
    // put splits and stores (B_re rows (Re y, -Im y), B_im rows (Im y, Re y))
    const bool ok = tc_pipeline(
        sm, bar, tmem, nk, sum,
        [&](int kc, float2 (&ra)[8], float2 (&rb)[8]) {
            float2 ga[8], gb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + kTcThreads * i;
                const int r = e & 127, kk = e >> 7;
                const int s = r >> 6, al = r & 63, k = kc * 16 + kk;
                ga[i] = (a0 + al < cl && k < cm) ? G0[s * slice + (size_t)k * chip + a0 + al] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + kTcThreads * i;
                const int kk = e & 15, n = e >> 4;
                const int t = n >> 6, gl = n & 63, k = kc * 16 + kk;
                gb[i] = (g0 + gl < cr && k < cm) ? G1[t * slice + (size_t)(g0 + gl) * chip + k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + kTcThreads * i;
                const int r = e & 127, kk = e >> 7, k = kc * 16 + kk;
                const float f = k < cm ? sL[r & 63] * sM[k] : 0.f;
                ra[i] = make_float2(ga[i].x * f, ga[i].y * f);
                const int gl = (e >> 4) & 63;
                rb[i] = make_float2(gb[i].x * sR[gl], gb[i].y * sR[gl]);
            }
        },
        [&](unsigned char* S, const float2 (&ra)[8], const float2 (&rb)[8]) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + kTcThreads * i;
                put_a(S, e & 127, e >> 7, ra[i]);
                put_b(S, e >> 4, e & 15, make_float2(rb[i].x, -rb[i].y), make_float2(rb[i].y, rb[i].x));
            }
        });
    if (!ok) {
        // an MMA never completed: its accumulators may still be written, so the
        // state cannot be trusted any more (DERR_DRAIN); release the tensor memory
        if (tid == 0) atomicOr(a.err, DERR_TIMEOUT | DERR_DRAIN);
        tc_end(tmem);
        return;
    }
    // ---- epilogue: the sums -> shared memory (column-major, pitch 129)
    float* th_re = reinterpret_cast<float*>(sm);
    float* th_im = th_re + 128 * kThPitch;
    stage_sums(sum, th_re, th_im);
    tc_end(tmem);
    // ---- gate mix and stores: theta_{st}(alpha, gamma) at column t * 64 + gamma, row s * 64 + alpha
    const size_t ldw = a.ldw;
    float2* W = a.w + (size_t)j * ldw * ldw;
    float2* W0 = a.w0 + (size_t)j * ldw * ldw;
    const bool gated = a.gates != nullptr;
    auto theta_at = [&](int s, int t, int al, int gl) {
        const int o = (t * 64 + gl) * kThPitch + s * 64 + al;
        return make_float2(th_re[o], th_im[o]);
    };
    auto out_at = [&](int sp, int tp, int al, int gl) {
        if (!gated) return theta_at(sp, tp, al, gl);
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const float2 u = ug[(2 * sp + tp) * 4 + 2 * s + t], x = theta_at(s, t, al, gl);
                v.x = fmaf(u.x, x.x, v.x); v.x = fmaf(-u.y, x.y, v.x);
                v.y = fmaf(u.x, x.y, v.y); v.y = fmaf(u.y, x.x, v.y);
            }
        return v;
    };
    if (tall) {
        const int al = tid & 63;
        for (int gl = tid >> 6; gl < 64; gl += 4) {
            if (a0 + al >= cl || g0 + gl >= cr) continue;
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int tp = 0; tp < 2; ++tp) {
                    const float2 v = out_at(sp, tp, al, gl);
                    const size_t r = (size_t)sp * cl + a0 + al, c = (size_t)tp * cr + g0 + gl;
                    W[c * ldw + r] = v;
                    W0[c * ldw + r] = v;
                }
        }
    } else {
        const int gl = tid & 63;
        for (int al = tid >> 6; al < 64; al += 4) {
            if (a0 + al >= cl || g0 + gl >= cr) continue;
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int tp = 0; tp < 2; ++tp) {
                    float2 v = out_at(sp, tp, al, gl);
                    v.y = -v.y;
                    const size_t r = (size_t)sp * cl + a0 + al, c = (size_t)tp * cr + g0 + gl;
                    if (a.mode == 0) W[r * ldw + c] = v;
                    W0[r * ldw + c] = v;
                }
        }
    }
}

// ------------------------------------------------------------ Gamma, GEMM --
// The second factor of the Gamma rebuild (Sec. II C) on the tensor cores, the
// same product as k_gamma_gemm: Z[i, c] = sum_r conj(P[r, i]) Q[r, c] over the
// rows r of theta' (or its adjoint), with the rotated columns divided by S as
// they are loaded (tall: P = U S / S, Q = theta', Z = S V^dag; wide: P =
// theta'^dag, Q = V S / S, Z = U S), then Gamma = Z / (S Lambda).  conj(A) B is
// formed with B_re rows holding (Re b, Im b) and B_im rows (Im b, -Re b).  A
// CTA computes a 128 x 128 tile of the chip x chip slice sigma = blockIdx.z & 1
// and writes every element of it inside the slice (zero outside the kept
// block), straight from tensor memory: TMEM lane = target row, which is
// contiguous in the column-major slice.
// grid (ceil(chip / 128), ceil(chip / 128), 2 count), 256 threads, kTcSmem bytes.
__global__ void __launch_bounds__(kTcThreads, 1) k_gamma_tc(LayerArgs<float> a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kStage);  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    int* pcol = reinterpret_cast<int*>(sm + 2 * kStage + 64);  // [128]
    int* qcol = pcol + 128;                                      // [128]
    float* pscl = reinterpret_cast<float*>(qcol + 128);         // [128]
    float* qscl = pscl + 128;                                    // [128]

    const int j = blockIdx.z >> 1, sg = blockIdx.z & 1;
    const int32_t* d = a.dims + j * kDims;
    const int k = d[D_K];
    if (k == 0) return;  // error latched by k_truncate, or left to the FP64 resolution
    const int cl = d[D_CL], cr = d[D_CR], b = d[D_BOND], rows = d[D_ROWS];
    const bool tall = d[D_TALL] != 0;
    const int chip = a.chip;
    const size_t slice = (size_t)chip * chip, ldw = a.ldw;
    const int r0 = blockIdx.x * 128, c0 = blockIdx.y * 128;
    const int rlim = tall ? k : cl;  // valid target rows
    const int clim = tall ? cr : k;  // valid target cols
    float2* Gm = static_cast<float2*>(a.gamma) + (size_t)(tall ? b + 1 : b) * 2 * slice + sg * slice;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (r0 >= rlim || c0 >= clim) {
        for (int e = tid; e < 128 * 128; e += kTcThreads) {
            const int row = r0 + (e & 127), col = c0 + (e >> 7);
            if (row < chip && col < chip) Gm[(size_t)col * chip + row] = make_float2(0.f, 0.f);
        }
        return;
    }
    const float2* W = a.w + (size_t)j * ldw * ldw;
    const float2* W0 = a.w0 + (size_t)j * ldw * ldw;
    const float2* P = tall ? W : W0;
    const float2* Q = tall ? W0 : W;
    const int32_t* perm = a.perm + (size_t)j * ldw;
    const double* sig = a.sig + (size_t)j * ldw;
    if (tid < 128) {
        const int row = r0 + tid;
        int pc = -1;
        float sc = 1.f;
        if (row < rlim) {
            pc = tall ? perm[row] : sg * cl + row;
            if (tall) sc = (float)(1.0 / sig[row]);
        }
        pcol[tid] = pc;
        pscl[tid] = sc;
    } else {
        const int col = c0 + tid - 128;
        int qc = -1;
        float sc = 1.f;
        if (col < clim) {
            qc = tall ? sg * cr + col : perm[col];
            if (!tall) sc = (float)(1.0 / sig[col]);
        }
        qcol[tid - 128] = qc;
        qscl[tid - 128] = sc;
    }
    const uint32_t tmem = tc_begin(bar, tmem_slot);  // its barrier also publishes pcol .. qscl
    const int nk = (rows + 15) / 16;
    float sum[128];
    // element i of a thread: e = tid + 256 i, kk = e & 15 (K = row r of P and Q), row e >> 4 of A and of B
    const bool ok = tc_pipeline(
        sm, bar, tmem, nk, sum,
        [&](int kc, float2 (&ra)[8], float2 (&rb)[8]) {
            float2 pa[8], qb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + kTcThreads * i;
                const int kk = e & 15, c = e >> 4, r = kc * 16 + kk;
                pa[i] = (pcol[c] >= 0 && r < rows) ? P[(size_t)pcol[c] * ldw + r] : make_float2(0.f, 0.f);
                qb[i] = (qcol[c] >= 0 && r < rows) ? Q[(size_t)qcol[c] * ldw + r] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = (tid + kTcThreads * i) >> 4;
                ra[i] = make_float2(pa[i].x * pscl[c], pa[i].y * pscl[c]);
                rb[i] = make_float2(qb[i].x * qscl[c], qb[i].y * qscl[c]);
            }
        },
        [&](unsigned char* S, const float2 (&ra)[8], const float2 (&rb)[8]) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {  // conj(A) B: B_re rows (Re b, Im b), B_im rows (Im b, -Re b)
                const int e = tid + kTcThreads * i;
                put_a(S, e >> 4, e & 15, ra[i]);
                put_b(S, e >> 4, e & 15, make_float2(rb[i].x, rb[i].y), make_float2(rb[i].y, -rb[i].x));
            }
        });
    if (!ok) {
        if (tid == 0) atomicOr(a.err, DERR_TIMEOUT | DERR_DRAIN);
        tc_end(tmem);
        return;
    }
    const double* lnb = a.lam + (size_t)(tall ? b + 2 : b) * chip;  // Lambda_{b+1} or Lambda_{b-1}
    float* zr = reinterpret_cast<float*>(sm);
    float* zi = zr + 128 * kThPitch;
    stage_sums(sum, zr, zi);
    __syncthreads();
    {
        const int q = warp & 3, half = warp >> 2;
        const int row = r0 + 32 * q + lane;
#pragma unroll 1
        for (int cc = 0; cc < 64; cc += 16) {
            const int cl0 = half * 64 + cc;
            float vre[16], vim[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                vre[i] = zr[(cl0 + i) * kThPitch + 32 * q + lane];
                vim[i] = zi[(cl0 + i) * kThPitch + 32 * q + lane];
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = c0 + cl0 + i;
                if (row >= chip || col >= chip) continue;
                float2 v = make_float2(0.f, 0.f);
                if (row < rlim && col < clim) {
                    const double sb = tall ? sig[row] : sig[col];
                    const double ln = tall ? lnb[col] : lnb[row];
                    const float f = __frcp_rn((float)sb * (float)ln);
                    v = make_float2(vre[i] * f, vim[i] * f);
                }
                Gm[(size_t)col * chip + row] = v;
            }
        }
    }
    tc_end(tmem);
}

// ---------------------------------------------------------- tSU projection --
// M^dag = theta^dag U_X (the second tSU matrix, Sec. III D), the product of
// k_proj on the tensor cores: out[r, c] = sum_k A[r, k] B[k, c] / sigma_X[c]
// with A = theta^dag (rows 2 chi_{b+1}, K = 2 chi_{b-1}) in w0 and B = U_X
// Sigma_X (K x chi_b) in w; a zero sigma_X gives a zero column.  A CTA computes
// a 128 x 128 tile of out (w1).
// grid (ceil(2 chip / 128), ceil(chip / 128), count), 256 threads, kTcSmem bytes.
__global__ void __launch_bounds__(kTcThreads, 1) k_proj_tc(LayerArgs<float> a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kStage);  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    float* bscl = reinterpret_cast<float*>(sm + 2 * kStage + 64);  // [128]

    const int j = blockIdx.z;
    const int32_t* d = a.dims + j * kDims;
    const int cl = d[D_CL], cm = d[D_CM], cr = d[D_CR];
    const int rows = 2 * cr, kdim = 2 * cl;
    const int r0 = blockIdx.x * 128, c0 = blockIdx.y * 128;
    if (r0 >= rows || c0 >= cm) return;  // uniform over the CTA, before any allocation
    const size_t ldw = a.ldw;
    const float2* A = a.w0 + (size_t)j * ldw * ldw;
    const float2* B = a.w + (size_t)j * ldw * ldw;
    float2* out = a.w1 + (size_t)j * ldw * ldw;
    const double* sig = a.norms + (size_t)j * ldw;
    const int tid = threadIdx.x;
    if (tid < 128) {
        const int gc = c0 + tid;
        const double sg = gc < cm ? sig[gc] : 0.0;
        bscl[tid] = sg > 0.0 ? (float)(1.0 / sg) : 0.f;
    }
    const uint32_t tmem = tc_begin(bar, tmem_slot);  // its barrier also publishes bscl
    const int nk = (kdim + 15) / 16;
    float sum[128];
    // element i of a thread: A (row e & 127 = output row, kk = e >> 7), B (kk = e & 15, row e >> 4), e = tid + 256 i
    const bool ok = tc_pipeline(
        sm, bar, tmem, nk, sum,
        [&](int kc, float2 (&ra)[8], float2 (&rb)[8]) {
            float2 xb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = tid + kTcThreads * i;
                const int gr = r0 + (e & 127), gk = kc * 16 + (e >> 7);
                ra[i] = (gr < rows && gk < kdim) ? A[(size_t)gk * ldw + gr] : make_float2(0.f, 0.f);
                const int gc = c0 + (e >> 4), gk2 = kc * 16 + (e & 15);
                xb[i] = (gc < cm && gk2 < kdim) ? B[(size_t)gc * ldw + gk2] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = (tid + kTcThreads * i) >> 4;
                rb[i] = make_float2(xb[i].x * bscl[c], xb[i].y * bscl[c]);
            }
        },
        [&](unsigned char* S, const float2 (&ra)[8], const float2 (&rb)[8]) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {  // A B: B_re rows (Re b, -Im b), B_im rows (Im b, Re b)
                const int e = tid + kTcThreads * i;
                put_a(S, e & 127, e >> 7, ra[i]);
                put_b(S, e >> 4, e & 15, make_float2(rb[i].x, -rb[i].y), make_float2(rb[i].y, rb[i].x));
            }
        });
    if (!ok) {
        if (tid == 0) atomicOr(a.err, DERR_TIMEOUT | DERR_DRAIN);
        tc_end(tmem);
        return;
    }
    float* zr = reinterpret_cast<float*>(sm);
    float* zi = zr + 128 * kThPitch;
    stage_sums(sum, zr, zi);
    __syncthreads();
    {
        // column by column: 256 threads write rows r0 .. r0 + 127 of two columns at a time
        const int r = tid & 127;
        const int gr = r0 + r;
#pragma unroll 1
        for (int cc = tid >> 7; cc < 128; cc += 2) {
            const int gc = c0 + cc;
            if (gr < rows && gc < cm) out[(size_t)gc * ldw + gr] = make_float2(zr[cc * kThPitch + r], zi[cc * kThPitch + r]);
        }
    }
    tc_end(tmem);
}

}  // namespace

cudaError_t theta_tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_theta_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gamma_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_proj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    return e;
}

cudaError_t launch_proj_tc(const LayerArgs<float>& a, cudaStream_t s) {
    dim3 grid((2 * a.chip + 127) / 128, (a.chip + 127) / 128, a.count);
    k_proj_tc<<<grid, kTcThreads, kTcSmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gamma_gemm_tc(const LayerArgs<float>& a, cudaStream_t s) {
    const int tiles = (a.chip + 127) / 128;
    dim3 grid(tiles, tiles, 2 * a.count);
    k_gamma_tc<<<grid, kTcThreads, kTcSmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_theta_tc(const LayerArgs<float>& a, cudaStream_t s) {
    const int tiles = (a.chip + 63) / 64;
    dim3 grid(tiles, tiles, a.count);
    k_theta_tc<<<grid, kTcThreads, kTcSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ptebd
