// Batched one-sided (Hestenes) Jacobi SVD of the two-site tensors of a layer
// (the SVD step of the TEBD procedure, Sec. II C of arXiv:2312.02667).
//
// One CTA per bond.  The matrix w (rows x cols, column-major, rows >= cols)
// stays in global memory / L2; the CTA sweeps over blocks of NW columns:
//   * block I is held in registers, one column per warp (which rows a lane
//     holds: PairRows below; complex64 columns are kept pair-split while the
//     sweeps run and turned back into plain complex columns at the end);
//   * the intra-block pairs of I are rotated in shared memory (round-robin);
//   * every later block J is streamed through a double-buffered shared-memory
//     stage by TMA bulk copies (cp.async.bulk, completion on an mbarrier),
//     rotated against I in NW rounds (warp w meets column (w + r) mod NW of J,
//     handed on from warp w + 1 once its rotated rows are in the stage), and
//     written back by a TMA bulk store.
// Each sweep therefore meets every column pair once (block row-cyclic order).
// A pair (a, b) with |a^H b| > tol ||a|| ||b|| is rotated by the 2x2 unitary that
// diagonalises its Gram matrix; the sweeps stop when none was rotated (or, on
// the complex64 path, when every rotation of a sweep was a small one: Eps).  The
// squared column norms are recomputed at the start of every sweep and then
// tracked through the rotations (a' and b' norms follow from the 2x2 problem),
// so a pair costs one complex dot product; a norm that drops a lot is
// recomputed from the rotated column.  On exit the columns are U S
// (orthogonal, unsorted); their FP64 norms are the singular values.
//
// Every wait on an mbarrier is bounded by a clock budget; a wait that runs out
// latches DERR_TIMEOUT, drains the CTA's own copies and returns.
#include <cmath>
#include <type_traits>

#include "ptebd_internal.h"

namespace ptebd {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void counter_release_add(int* p) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], 1;" ::"r"(smem_u32(p)) : "memory");
}
__device__ __forceinline__ int counter_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
// Bounded spin until *p >= target (or the CTA has aborted).  The clock and the
// abort flag are looked at every 32 polls only, to keep the spin cheap in issue slots.
__device__ __forceinline__ bool counter_wait_bounded(const int* p, int target, const volatile int* abort_flag,
                                                     long long limit = 1ll << 31) {
    if (counter_acquire(p) >= target) return true;
    const long long start = clock64();
    for (unsigned it = 1;; ++it) {
        __nanosleep(32);
        if (counter_acquire(p) >= target) return true;
        if ((it & 31u) == 0u) {
            if (clock64() - start > limit) return false;
            if (*abort_flag) return false;
        }
    }
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait: about 2^31 SM cycles (~1 s) before giving up, or at once when
// another warp of the CTA has already given up (abort flag set).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  const volatile int* abort_flag = nullptr) {
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > (1ll << 31)) return false;
        if (abort_flag && *abort_flag) return false;
    }
    return true;
}

// Unit roundoff and the rotation threshold factor: a pair is rotated when
// |a^H b| > k sqrt(rows) u ||a|| ||b||.  Rounding alone leaves |a^H b| of about
// sqrt(rows) u ||a|| ||b|| after a rotation, so the factor must sit well above 1
// or rounding keeps re-triggering rotations (more sweeps, and every extra
// rotation adds rounding error to the columns).
// early: the sweeps also stop after a sweep in which every rotated pair had
// cos^2 = |a^H b|^2 / (|a|^2 |b|^2) below early * tol^2 (0 = only after a sweep
// without rotations).  On the complex64 path the sweep after such a sweep was
// measured never to meet a pair above 1.04 tol^2 (gated and tSU matrices of
// saturated layers, Ginibre and graded spectra: thousands of SVDs), and to
// spend itself on 0 to 2 rotations of pairs barely above tol, so it is skipped;
// the columns are left orthogonal to about tol instead of below tol.
template <typename R> struct Eps;
// range_e: matrices whose largest entry is not in [2^-range_e, 2^range_e) are
// rescaled before the sweeps (see the range guard in jacobi_body).
// polish: the factor of a last sweep's tighter threshold (A.polish), run once
// after the stopping rule has fired: it rotates every pair with
// |a^H b| > polish sqrt(rows) u |a| |b|, which leaves the columns orthogonal to
// near the rounding of their storage (the truncated state depends on it).
template <> struct Eps<float> {
    static constexpr double u = 5.9604644775390625e-08;  // 2^-24
    static constexpr double k = 8.0;
    static constexpr int range_e = 24;
    static constexpr double early = 256.0;
    static constexpr double polish = 2.0;
};
template <> struct Eps<double> {
    static constexpr double u = 1.1102230246251565e-16;  // 2^-53
    static constexpr double k = 4.0;
    static constexpr int range_e = 240;
    static constexpr double early = 0.0;
    static constexpr double polish = 0.0;
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The binary exponent of a non-negative value, offset so that 0 (no entry) stays
// below every real exponent: a shared atomicMax over it gives the exponent of the
// largest entry of a matrix.
constexpr int kExpOffset = 2048;
template <typename R> __device__ __forceinline__ int exp_key(R v) {
    return v > (R)0 ? ilogb((double)v) + kExpOffset : 0;
}

// Parameters of the rotation that diagonalises [[al, g e], [g conj(e), be]]
// (al = |a|^2, be = |b|^2, g e = a^H b): t = tan of the angle, cm1 = cos - 1,
// (sr, si) = sin * e.  Applied as a' = a + cm1 a - s conj(e) b, b' = b + cm1 b + s e a:
// writing cos as 1 + (cos - 1) with cos - 1 in closed form keeps the rotation norm
// preserving when t^2 is below the unit roundoff (cos itself would round to 1 while
// sin = t does not, and every such rotation would scale the pair by sqrt(1 + t^2)).
template <typename R> struct RotParams { R cm1, sr, si, tg; };
// Packed FP32 pairs (fma.rn.f32x2 and friends, sm_100 and later): two lanes of
// FP32 arithmetic per instruction on a register pair (lo, hi).
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}


__device__ __forceinline__ RotParams<float> rot_params(float al, float be, float gr, float gi, float g2) {
    // t = 2 |g| sign(d) / (|d| + sqrt(d^2 + 4 |g|^2)), d = be - al: the smaller
    // root of t^2 + (d / |g|) t - 1 = 0, formed without the quotient d / |g| (so
    // with no overflow when |g| << |d|, and one reciprocal square root less on
    // the chain).  MUFU reciprocal square roots; cos is refined by one Newton step
    // so that cos^2 (1 + t^2) = 1 to rounding (the sign of the residual is not biased).
    const float ig = rsqrtf(g2);
    const float g = g2 * ig;
    const float d = be - al;
    const float h = fmaf(d, d, 4.0f * g2);
    const float root = h * rsqrtf(h);
    float t = __fdividef(2.0f * g, fabsf(d) + root);
    if (d < 0.0f) t = -t;
    const float q = fmaf(t, t, 1.0f);
    float c = rsqrtf(q);
    c = c * fmaf(-0.5f * q * c, c, 1.5f);
    RotParams<float> p;
    p.cm1 = __fdividef(-(t * t) * (c * c), 1.0f + c);
    const float s = t * c;
    p.sr = s * gr * ig;
    p.si = s * gi * ig;
    p.tg = t * g;
    return p;
}

__device__ __forceinline__ RotParams<double> rot_params(double al, double be, double gr, double gi, double g2) {
    const double g = sqrt(g2);
    const double ig = 1.0 / g;
    const double zeta = (be - al) * (0.5 * ig);
    const double az = fabs(zeta);
    const double root = az < 1e150 ? sqrt(1.0 + zeta * zeta) : az;
    double t = 1.0 / (az + root);
    if (zeta < 0.0) t = -t;
    const double r1 = sqrt(1.0 + t * t);
    RotParams<double> p;
    p.cm1 = -(t * t) / (r1 * (1.0 + r1));
    const double s = t / r1;
    p.sr = s * gr * ig;
    p.si = s * gi * ig;
    p.tg = t * g;
    return p;
}


// complex64 rotation of a pair of columns in the pair-split layout (PairRows):
// the operations of the scalar form, applied to two rows per instruction.  With
// SA / SB the rotated rows of a / b also go to the shared-memory slot as / bs as
// soon as they are formed, so that the stores are under way before the rotation
// ends (a warp hands a column on only once its stores are complete).
template <int RPL, bool SA, bool SB>
__device__ __forceinline__ void rotate_split(float2 (&a)[RPL], float2 (&b)[RPL], const RotParams<float>& p,
                                             float2* as, float2* bs) {
    const int lane = threadIdx.x & 31;
    const unsigned long long cm = pk2(p.cm1, p.cm1);
    const unsigned long long sr = pk2(p.sr, p.sr), msr = pk2(-p.sr, -p.sr);
    const unsigned long long si = pk2(p.si, p.si), msi = pk2(-p.si, -p.si);
#pragma unroll
    for (int h = 0; h < RPL / 2; ++h) {
        const unsigned long long ax = pk2(a[2 * h].x, a[2 * h].y), ay = pk2(a[2 * h + 1].x, a[2 * h + 1].y);
        const unsigned long long bx = pk2(b[2 * h].x, b[2 * h].y), by = pk2(b[2 * h + 1].x, b[2 * h + 1].y);
        const unsigned long long t1 = fma2(msi, by, mul2(msr, bx));  // -(sr br + si bi)
        const unsigned long long t2 = fma2(si, bx, mul2(msr, by));   // -(sr bi - si br)
        const unsigned long long t3 = fma2(msi, ay, mul2(sr, ax));   // sr ar - si ai
        const unsigned long long t4 = fma2(si, ax, mul2(sr, ay));    // sr ai + si ar
        a[2 * h] = upk2(add2(ax, fma2(cm, ax, t1)));
        a[2 * h + 1] = upk2(add2(ay, fma2(cm, ay, t2)));
        b[2 * h] = upk2(add2(bx, fma2(cm, bx, t3)));
        b[2 * h + 1] = upk2(add2(by, fma2(cm, by, t4)));
        if constexpr (SB)
            *reinterpret_cast<float4*>(bs + 64 * h + 2 * lane) =
                make_float4(b[2 * h].x, b[2 * h].y, b[2 * h + 1].x, b[2 * h + 1].y);
        if constexpr (SA)
            *reinterpret_cast<float4*>(as + 64 * h + 2 * lane) =
                make_float4(a[2 * h].x, a[2 * h].y, a[2 * h + 1].x, a[2 * h + 1].y);
    }
}
// a^H b in the pair-split layout, scalar FMAs with one partial sum per row of
// the pair (packed FP32 instructions measured slower here than in the rotation)
template <int RPL>
__device__ __forceinline__ void dot_split(const float2 (&a)[RPL], const float2 (&b)[RPL], float& gr, float& gi) {
    float gr0 = 0, gr1 = 0, gi0 = 0, gi1 = 0;
#pragma unroll
    for (int h = 0; h < RPL / 2; ++h) {
        const float2 ar = a[2 * h], ai = a[2 * h + 1], br = b[2 * h], bi = b[2 * h + 1];
        gr0 = fmaf(ar.x, br.x, gr0); gr0 = fmaf(ai.x, bi.x, gr0);
        gi0 = fmaf(ar.x, bi.x, gi0); gi0 = fmaf(-ai.x, br.x, gi0);
        gr1 = fmaf(ar.y, br.y, gr1); gr1 = fmaf(ai.y, bi.y, gr1);
        gi1 = fmaf(ar.y, bi.y, gi1); gi1 = fmaf(-ai.y, br.y, gi1);
    }
    gr = gr0 + gr1;
    gi = gi0 + gi1;
}

// Rows of a column held by a lane, RPL entries per lane.  complex64 with RPL >= 2
// (rows even): the column is kept in a pair-split layout while the sweeps run,
// every two rows r, r + 1 (r even) stored as (Re r, Re r+1, Im r, Im r+1), so that
// one 16-byte access moves the pair and the packed FP32 instructions find the real
// parts and the imaginary parts of the pair in one register pair each.  Lane
// `lane` holds the pairs r = 64 h + 2 lane, h = 0 .. RPL/2 - 1: entry 2 h is
// (Re r, Re r+1), entry 2 h + 1 is (Im r, Im r+1).  Otherwise entry q is row
// 32 q + lane as a complex number.
template <typename C, int RPL> struct PairRows {
    static constexpr bool on = std::is_same<C, float2>::value && RPL >= 2;
};

template <typename R, int RPL>
__device__ __forceinline__ R col_norm2(const cx_t<R> (&a)[RPL]) {
    R s0 = 0, s1 = 0;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        s0 = fma(a[q].x, a[q].x, s0);
        s1 = fma(a[q].y, a[q].y, s1);
    }
    return warp_sum(s0 + s1);
}

template <typename C, int RPL>
__device__ __forceinline__ void slot_store(const C (&v)[RPL], C* col, int lane);

// Rotate the column pair (a, b) held by one warp (RPL entries per lane) if it is
// not yet orthogonal to within tol; al and be are their tracked squared norms and
// are updated.  Returns true if it rotated; then, with SA / SB, the rotated a / b
// have been written to the shared-memory slot as / bs as well, and big is set
// if the pair's cos^2 was at least big2.
template <typename R, int RPL, bool SA, bool SB>
__device__ __forceinline__ bool pair_rotate(cx_t<R> (&a)[RPL], cx_t<R> (&b)[RPL], R& al, R& be, R tol2,
                                            R big2, bool& big, cx_t<R>* as, cx_t<R>* bs) {
    constexpr bool split = PairRows<cx_t<R>, RPL>::on;
    R gr, gi;  // a^H b
    if constexpr (split) {
        dot_split<RPL>(a, b, gr, gi);
    } else {
        R gr0 = 0, gr1 = 0, gi0 = 0, gi1 = 0;  // two partial sums each
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            if (q & 1) {
                gr1 = fma(a[q].x, b[q].x, gr1); gr1 = fma(a[q].y, b[q].y, gr1);
                gi1 = fma(a[q].x, b[q].y, gi1); gi1 = fma(-a[q].y, b[q].x, gi1);
            } else {
                gr0 = fma(a[q].x, b[q].x, gr0); gr0 = fma(a[q].y, b[q].y, gr0);
                gi0 = fma(a[q].x, b[q].y, gi0); gi0 = fma(-a[q].y, b[q].x, gi0);
            }
        }
        gr = gr0 + gr1;
        gi = gi0 + gi1;
    }
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    // al, be >= 0 (a tracked norm that shrinks a lot is recomputed from its
    // column), so a zero column (g = 0) or a non-finite value fails this test
    // and is left alone
    const R g2 = gr * gr + gi * gi;
    if (!(g2 > (tol2 * al) * be)) return false;
    big = big || (g2 > (big2 * al) * be);
    const RotParams<R> p = rot_params(al, be, gr, gi, g2);
    if constexpr (split) {
        rotate_split<RPL, SA, SB>(a, b, p, as, bs);
    } else {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const R ar = a[q].x, ai = a[q].y, br = b[q].x, bi = b[q].y;
        a[q].x = ar + (p.cm1 * ar - (p.sr * br + p.si * bi));
        a[q].y = ai + (p.cm1 * ai - (p.sr * bi - p.si * br));
        b[q].x = br + (p.cm1 * br + (p.sr * ar - p.si * ai));
        b[q].y = bi + (p.cm1 * bi + (p.sr * ai + p.si * ar));
    }
    if constexpr (SB) slot_store<cx_t<R>, RPL>(b, bs, threadIdx.x & 31);
    if constexpr (SA) slot_store<cx_t<R>, RPL>(a, as, threadIdx.x & 31);
    }
    // norms from the 2x2 problem; the one that shrinks is recomputed when it
    // lost most of its size (cancellation in the update)
    R al2 = al - p.tg, be2 = be + p.tg;
    if (!(al2 > (R)0.125 * al)) al2 = col_norm2<R, RPL>(a);
    if (!(be2 > (R)0.125 * be)) be2 = col_norm2<R, RPL>(b);
    al = al2;
    be = be2;
    return true;
}

// Two independent column pairs (a0, b0) and (a1, b1) of one warp, complex64 in
// the pair-split layout: the test and rotation of pair_rotate for each, with the
// two instruction streams interleaved (dot products, shuffle reductions,
// rotation parameters, rotations), so that the latency of one pair's chain is
// covered by the other's work.  v0 / v1: the pair exists.  The rotated b0 / b1
// go to the shared-memory slots bs0 / bs1; r0 / r1 report which pairs rotated.
template <int RPL>
__device__ __forceinline__ void pair_rotate2(float2 (&a0)[RPL], float2 (&b0)[RPL], float& al0, float& be0, bool v0,
                                             float2 (&a1)[RPL], float2 (&b1)[RPL], float& al1, float& be1, bool v1,
                                             float tol2, float big2, bool& big, float2* bs0, float2* bs1, bool& r0,
                                             bool& r1) {
    float gr0, gi0, gr1, gi1;
    dot_split<RPL>(a0, b0, gr0, gi0);
    dot_split<RPL>(a1, b1, gr1, gi1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float x0 = __shfl_xor_sync(0xffffffffu, gr0, o), y0 = __shfl_xor_sync(0xffffffffu, gi0, o);
        const float x1 = __shfl_xor_sync(0xffffffffu, gr1, o), y1 = __shfl_xor_sync(0xffffffffu, gi1, o);
        gr0 += x0; gi0 += y0; gr1 += x1; gi1 += y1;
    }
    const float g20 = gr0 * gr0 + gi0 * gi0, g21 = gr1 * gr1 + gi1 * gi1;
    r0 = v0 && (g20 > (tol2 * al0) * be0);
    r1 = v1 && (g21 > (tol2 * al1) * be1);
    if (!(r0 || r1)) return;
    big = big || (r0 && g20 > (big2 * al0) * be0) || (r1 && g21 > (big2 * al1) * be1);
    // a pair that does not rotate gets harmless parameters (never applied)
    const RotParams<float> p0 = r0 ? rot_params(al0, be0, gr0, gi0, g20) : RotParams<float>{0.f, 0.f, 0.f, 0.f};
    const RotParams<float> p1 = r1 ? rot_params(al1, be1, gr1, gi1, g21) : RotParams<float>{0.f, 0.f, 0.f, 0.f};
    if (r0 && r1) {
        rotate_split<RPL, false, true>(a0, b0, p0, nullptr, bs0);
        rotate_split<RPL, false, true>(a1, b1, p1, nullptr, bs1);
    } else if (r0) {
        rotate_split<RPL, false, true>(a0, b0, p0, nullptr, bs0);
    } else {
        rotate_split<RPL, false, true>(a1, b1, p1, nullptr, bs1);
    }
    if (r0) {
        float al2 = al0 - p0.tg, be2 = be0 + p0.tg;
        if (!(al2 > 0.125f * al0)) al2 = col_norm2<float, RPL>(a0);
        if (!(be2 > 0.125f * be0)) be2 = col_norm2<float, RPL>(b0);
        al0 = al2;
        be0 = be2;
    }
    if (r1) {
        float al2 = al1 - p1.tg, be2 = be1 + p1.tg;
        if (!(al2 > 0.125f * al1)) al2 = col_norm2<float, RPL>(a1);
        if (!(be2 > 0.125f * be1)) be2 = col_norm2<float, RPL>(b1);
        al1 = al2;
        be1 = be2;
    }
}

template <typename C, int RPL>
__device__ __forceinline__ int lane_row(int lane, int q) {
    return PairRows<C, RPL>::on ? 64 * (q >> 1) + 2 * lane + (q & 1) : 32 * q + lane;
}
// v[q] = col[row(q)] for rows < rows (else 0); col 16-byte aligned
template <typename C, int RPL>
__device__ __forceinline__ void col_load(C (&v)[RPL], const C* col, int lane, int rows, bool valid) {
    if constexpr (PairRows<C, RPL>::on) {
#pragma unroll
        for (int h = 0; h < RPL / 2; ++h) {
            const int r = 64 * h + 2 * lane;  // rows is even: a pair is valid as a whole
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid && r < rows) t = *reinterpret_cast<const float4*>(col + r);
            v[2 * h] = make_float2(t.x, t.y);
            v[2 * h + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = 32 * q + lane;
            v[q] = (valid && r < rows) ? col[r] : cmake<C>(0, 0);
        }
    }
}
template <typename C, int RPL>
__device__ __forceinline__ void col_store(const C (&v)[RPL], C* col, int lane, int rows) {
    if constexpr (PairRows<C, RPL>::on) {
#pragma unroll
        for (int h = 0; h < RPL / 2; ++h) {
            const int r = 64 * h + 2 * lane;
            if (r < rows) *reinterpret_cast<float4*>(col + r) = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
        }
    } else {
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = 32 * q + lane;
            if (r < rows) col[r] = v[q];
        }
    }
}
// the same for a shared-memory column slot padded with zeros to mpad rows:
// every row is read and written (rows beyond `rows` stay zero)
template <typename C, int RPL>
__device__ __forceinline__ void slot_load(C (&v)[RPL], const C* col, int lane) {
    if constexpr (PairRows<C, RPL>::on) {
#pragma unroll
        for (int h = 0; h < RPL / 2; ++h) {
            const float4 t = *reinterpret_cast<const float4*>(col + 64 * h + 2 * lane);
            v[2 * h] = make_float2(t.x, t.y);
            v[2 * h + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < RPL; ++q) v[q] = col[32 * q + lane];
    }
}
template <typename C, int RPL>
__device__ __forceinline__ void slot_store(const C (&v)[RPL], C* col, int lane) {
    if constexpr (PairRows<C, RPL>::on) {
#pragma unroll
        for (int h = 0; h < RPL / 2; ++h)
            *reinterpret_cast<float4*>(col + 64 * h + 2 * lane) =
                make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
    } else {
#pragma unroll
        for (int q = 0; q < RPL; ++q) col[32 * q + lane] = v[q];
    }
}

// Columns are visited in order of decreasing norm, re-sorted at the start of
// every sweep (de Rijk's ordering idea): it lowers the number of sweeps.
constexpr int kSortN = 512;
constexpr int kShInts = 8;  // shared ints ahead of the slot round counters

// CPW: columns of the register block per warp.  1: NW warps, one I column
// each; 2 (complex64, RPL >= 2 only): NW / 2 warps, each holding I columns
// 2w and 2w + 1 and meeting two J columns per round (pair_rotate2).
template <typename R, int NW, int RPL, int CPW = 1>
__device__ void jacobi_body(const LayerArgs<R>& A, cx_t<R>* W, int rows, int cols, int j, unsigned char* smem) {
    using C = cx_t<R>;
    static_assert(CPW == 1 || (CPW == 2 && std::is_same<R, float>::value && RPL >= 2), "two columns per warp: complex64, pair-split layout");
    constexpr int NWARPS = NW / CPW;
    const int ldw = A.ldw;
    const int mpad = ldw;  // rows per column slot in shared memory
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    C* bufJ0 = reinterpret_cast<C*>(smem);
    C* bufJ1 = bufJ0 + NW * mpad;
    C* bufI = bufJ1 + NW * mpad;
    uint64_t* bar = reinterpret_cast<uint64_t*>(bufI + NW * mpad);  // [2]: TMA loads of the J stages
    R* jn2 = reinterpret_cast<R*>(bar + 2);        // [2][NW]: tracked |col|^2 of the J stage slots
    R* in2 = jn2 + 2 * NW;                          // [NW]: |col|^2 of the I block (intra phase)
    // [0] rotations, [1] abort, [2] max exponent, [3..4] a load into the stage not yet
    // waited for by thread 0, [5..6] the barrier phase that load completes, [7] a
    // rotation in this sweep had cos^2 >= early tol^2
    int* sh = reinterpret_cast<int*>(in2 + NW);
    int* slot_done = sh + kShInts;  // [2][NW]: rounds completed on each column slot of each stage
    int* cperm = slot_done + 2 * NW;                                   // [kSortN]: sweep order -> column
    float* skey = reinterpret_cast<float*>(cperm + kSortN);            // [kSortN]: sort keys
    C* bufJ[2] = {bufJ0, bufJ1};
    int jblocks[2] = {0, 0};  // J blocks processed so far on each stage
    // squared column norms between blocks (FP64), a table in shared memory
    double* nrm2 = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(skey + kSortN) + 7) & ~uintptr_t(7));
    // complex128 only: per column, bit 0 = rotated in the previous sweep, bit 1 =
    // rotated in this one.  A pair whose two columns have neither bit set met in
    // the previous sweep as the same two vectors and was found orthogonal then, so
    // its dot product is skipped (on the FP64 pipe a dot product costs as much as
    // a third of a rotation; late sweeps are mostly such checks).
    constexpr bool kSkip = std::is_same<R, double>::value;
    unsigned char* rflag = reinterpret_cast<unsigned char*>(nrm2 + kSortN);
    if constexpr (kSkip)
        for (int c = tid; c < kSortN; c += blockDim.x) rflag[c] = 1;  // sweep 0 checks every pair

    const R tol = (R)(Eps<R>::k * sqrt((double)rows) * Eps<R>::u);
    R tol2 = tol * tol;
    const R big2 = (R)Eps<R>::early * tol2;
    const bool polish = A.polish && Eps<R>::polish > 0.0;
    bool polishing = false;  // the last sweep, with the tighter threshold
    bool big_w = false;  // this warp rotated a pair with cos^2 >= big2 in the sweep
    const int nb = (cols + NW - 1) / NW;
    const uint32_t col_bytes = (uint32_t)(rows * sizeof(C));
    uint32_t phase[2] = {0u, 0u};
    int cur = 0;
    int sweep = 0;
    long long rot_total = 0;
    int rot_w = 0;  // rotations of this warp in the sweep
    bool converged = false;

    auto issue_load = [&](int J, int buf) {
        // one thread: expect the bytes, then one bulk copy per real column
        const int c0 = J * NW;
        const int nreal = min(NW, cols - c0);
        mbar_expect_tx(&bar[buf], (uint32_t)nreal * col_bytes);
        for (int c = 0; c < nreal; ++c) {
            const int gc = cperm[c0 + c];
            bulk_g2s(bufJ[buf] + (size_t)c * mpad, W + (size_t)gc * ldw, col_bytes, &bar[buf]);
            jn2[buf * NW + c] = (R)nrm2[gc];  // the tracked norm the column enters the stage with
        }
        sh[3 + buf] = 1;
        sh[5 + buf] = (int)phase[buf];
    };
    auto abort_drain = [&]() {
        // Called by all threads after a wait ran out: wait (bounded) once more
        // for the loads still in flight, drain our bulk stores, latch the error.
        // If a load still has not landed, the CTA has to return with it in flight
        // (nothing can cancel a bulk copy, and waiting on would hang the GPU):
        // DERR_DRAIN marks the state unusable until it is re-created.
        if (tid == 0) {
            bool drained = true;
            for (int b = 0; b < 2; ++b)
                if (sh[3 + b] && !mbar_wait_bounded(&bar[b], (uint32_t)sh[5 + b])) drained = false;
            bulk_wait_all();
            atomicOr(A.err, drained ? DERR_TIMEOUT : (DERR_TIMEOUT | DERR_DRAIN));
        }
        __syncthreads();
    };

    // exact squared column norms (each warp its columns c = warp mod NW); with
    // want_max, the exponent of the largest |entry| is gathered in sh[2] as well.
    // A squared norm is the sum of the squares of all the column's floats, so it
    // does not depend on the layout.  With to_split (PairRows only) the columns are
    // rewritten in the pair-split layout on the way.
    auto norm_pass = [&](bool want_max, bool to_split) {
        R mx = 0;
        for (int c = warp; c < cols; c += NWARPS) {
            R s0 = 0, s1 = 0;
            if constexpr (PairRows<C, RPL>::on) {
                float4* col = reinterpret_cast<float4*>(W + (size_t)c * ldw);
                for (int g = lane; g < rows / 2; g += 32) {
                    float4 v = col[g];
                    s0 = fma(v.x, v.x, s0); s1 = fma(v.y, v.y, s1);
                    s0 = fma(v.z, v.z, s0); s1 = fma(v.w, v.w, s1);
                    if (want_max) mx = fmax(mx, fmax(fmax(fabs(v.x), fabs(v.y)), fmax(fabs(v.z), fabs(v.w))));
                    if (to_split) col[g] = make_float4(v.x, v.z, v.y, v.w);
                }
            } else {
                for (int r = lane; r < rows; r += 32) {
                    const C v = W[(size_t)c * ldw + r];
                    s0 = fma(v.x, v.x, s0);
                    s1 = fma(v.y, v.y, s1);
                    if (want_max) mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
                }
            }
            const R s2 = warp_sum(s0 + s1);
            if (lane == 0) nrm2[c] = (double)s2;
        }
        if (want_max) {
            mx = warp_max(mx);
            if (lane == 0) atomicMax(&sh[2], exp_key<R>(mx));
        }
        if (to_split) fence_async_global();  // the sweeps read W through TMA as well
    };
    // Range guard.  Squared norms and |a^H b|^2 are formed in R: with entries of
    // 2^range_e and more they can overflow (and with tiny entries underflow), which
    // turns a rotation into a plain scaling of the pair.  Such a matrix is scaled by
    // 2^-e, exactly, so that its largest entry lies in [1, 2), and scaled back after
    // the sweeps: a power-of-two scaling commutes with every rounding of the sweeps,
    // so the result equals that of an unbounded exponent range.
    int scale_e = 0;

    for (sweep = 0; sweep < A.max_sweeps; ++sweep) {
        if constexpr (kSkip)
            if (sweep > 0)
                for (int c = tid; c < kSortN; c += blockDim.x) rflag[c] = (unsigned char)(rflag[c] >> 1);
        if (tid == 0) { sh[0] = 0; sh[7] = 0; bulk_wait_all(); fence_async_global(); }
        __syncthreads();
        norm_pass(sweep == 0, sweep == 0 && PairRows<C, RPL>::on);
        __syncthreads();
        if (sweep == 0) {
            const int ex = sh[2] - kExpOffset;  // 2^ex <= max |entry| < 2^(ex + 1)
            if (sh[2] > 0 && (ex >= Eps<R>::range_e || ex < -Eps<R>::range_e)) {
                scale_e = ex;
                const R f = ldexp((R)1, -scale_e);
                for (int c = warp; c < cols; c += NWARPS)
                    for (int r = lane; r < rows; r += 32) {
                        C v = W[(size_t)c * ldw + r];
                        v.x *= f; v.y *= f;
                        W[(size_t)c * ldw + r] = v;
                    }
                fence_async_global();  // the sweeps read W through TMA as well
                __syncwarp();
                norm_pass(false, false);
                __syncthreads();
            }
        }
        // sweep order: columns by decreasing norm (bitonic sort, ties by index)
        for (int e = tid; e < kSortN; e += blockDim.x) {
            skey[e] = e < cols ? (float)nrm2[e] : -1.0f;
            cperm[e] = e;
        }
        __syncthreads();
        for (int size = 2; size <= kSortN; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int e = tid; e < kSortN; e += blockDim.x) {
                    const int pe = e ^ stride;
                    if (pe > e) {
                        const bool desc = (e & size) == 0;
                        const float ke = skey[e], kp = skey[pe];
                        const int ie = cperm[e], ip = cperm[pe];
                        const bool e_first = (ke > kp) || (ke == kp && ie < ip);
                        if (desc ? !e_first : e_first) {
                            skey[e] = kp; skey[pe] = ke; cperm[e] = ip; cperm[pe] = ie;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int I = 0; I < nb; ++I) {
            // the polish sweep leaves pairs of two columns beyond chi_max (in the sweep
            // order, by decreasing norm) alone: they are dropped together, a rotation
            // between them changes no kept column and keeps their summed weight
            if (polishing && A.chi_max > 0 && I * NW >= A.chi_max) break;
            // all earlier bulk stores must have landed before plain loads of block I
            if (tid == 0) { bulk_wait_all(); fence_async_global(); }
            __syncthreads();
            // this warp's columns CPW warp + k of block I
            bool mine[CPW];
            int my_col[CPW];  // physical columns
            C a[CPW][RPL];
            R al[CPW];
#pragma unroll
            for (int k = 0; k < CPW; ++k) {
                const int ic = CPW * warp + k;
                mine[k] = I * NW + ic < cols;
                my_col[k] = mine[k] ? cperm[I * NW + ic] : 0;
                col_load<C, RPL>(a[k], W + (size_t)my_col[k] * ldw, lane, rows, mine[k]);
                // ---- intra-block pairs of I (round-robin), in shared memory
                slot_store<C, RPL>(a[k], bufI + (size_t)ic * mpad, lane);
                if (lane == 0) in2[ic] = mine[k] ? (R)nrm2[my_col[k]] : (R)0;
            }
            __syncthreads();
            for (int r = 0; r < NW - 1; ++r) {
                if (warp < NW / 2) {
                    auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (NW - 1)); };
                    const int p = player(warp), q2 = player(NW - 1 - warp);
                    const bool skip = kSkip && I * NW + p < cols && I * NW + q2 < cols &&
                                      !(rflag[cperm[I * NW + p]] | rflag[cperm[I * NW + q2]]);
                    if (I * NW + p < cols && I * NW + q2 < cols && !skip) {
                        C x[RPL], y[RPL];
                        slot_load<C, RPL>(x, bufI + (size_t)p * mpad, lane);
                        slot_load<C, RPL>(y, bufI + (size_t)q2 * mpad, lane);
                        R nx = in2[p], ny = in2[q2];
                        if (pair_rotate<R, RPL, true, true>(x, y, nx, ny, tol2, big2, big_w, bufI + (size_t)p * mpad,
                                                            bufI + (size_t)q2 * mpad)) {
                            __syncwarp();
                            if (lane == 0) {
                                in2[p] = nx;
                                in2[q2] = ny;
                                if constexpr (kSkip) {
                                    rflag[cperm[I * NW + p]] |= 2;
                                    rflag[cperm[I * NW + q2]] |= 2;
                                }
                            }
                            ++rot_w;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < CPW; ++k) {
                slot_load<C, RPL>(a[k], bufI + (size_t)(CPW * warp + k) * mpad, lane);
                al[k] = in2[CPW * warp + k];
            }

            // ---- cross pairs with every later block J, streamed by TMA
            if (I + 1 < nb) {
                if (tid == 0) issue_load(I + 1, cur);
                for (int J = I + 1; J < nb; ++J) {
                    const int nxt = cur ^ 1;
                    if (J + 1 < nb && tid == 0) {
                        bulk_wait_read_all();  // the store that last read bufJ[nxt] is done reading
                        issue_load(J + 1, nxt);
                    }
                    // Round r: warp w meets column (w + r) mod NW of the stage.  A column
                    // passes from warp w+1 (round r-1) to warp w (round r) through the
                    // slot's round counter (release / acquire), so a warp only waits for
                    // its one predecessor; the counters only grow, so a waiter can never
                    // mistake an older round for the one it needs.  The column's tracked
                    // squared norm travels with it (the CTA's norm table at round 0, then the
                    // stage's slot, and back to the table after the last round).
                    bool ok = mbar_wait_bounded(&bar[cur], phase[cur], &sh[1]);
                    if (tid == 0 && ok) sh[3 + cur] = 0;
                    C* buf = bufJ[cur];
                    int* done = slot_done + cur * NW;
                    R* sn2 = jn2 + cur * NW;
                    const int base = jblocks[cur] * NW;
                    const bool test_wait = A.wait_test && warp == 0 && sweep == 0 && I == 0 && J == 1;
                    for (int r = 0; r < NW && ok; ++r) {
                      if constexpr (CPW == 1) {
                        const int jc = (warp + r) & (NW - 1);
                        const int lcol = J * NW + jc;
                        if (r > 0) {
                            const bool t = test_wait && r == 1;
                            ok = counter_wait_bounded(&done[jc], t ? 0x7fffffff : base + r, &sh[1],
                                                      t ? (1ll << 20) : (1ll << 31));
                        }
                        if (!ok) break;
                        if (lcol < cols) {
                            R be = sn2[jc];
                            const bool skip = kSkip && mine[0] && !(rflag[my_col[0]] | rflag[cperm[lcol]]);
                            if (mine[0] && !skip) {
                                C y[RPL];
                                slot_load<C, RPL>(y, buf + (size_t)jc * mpad, lane);
                                // the rotated J column goes back to its slot inside the rotation
                                if (pair_rotate<R, RPL, false, true>(a[0], y, al[0], be, tol2, big2, big_w, nullptr,
                                                                     buf + (size_t)jc * mpad)) {
                                    sn2[jc] = be;  // every lane: the same value
                                    ++rot_w;
                                    if constexpr (kSkip)
                                        if (lane == 0) {
                                            rflag[my_col[0]] |= 2;
                                            rflag[cperm[lcol]] |= 2;
                                        }
                                }
                            }
                            if (r == NW - 1) nrm2[cperm[lcol]] = (double)be;
                        }
                        __syncwarp();
                        if (lane == 0) counter_release_add(&done[jc]);
                      } else {
                        // I column 2w meets jc0, which this warp's column 2w + 1 met in
                        // round r - 1 (no wait); I column 2w + 1 meets jc1, which
                        // column 2w + 2 (warp w + 1) met in round r - 1
                        const int jc0 = (2 * warp + r) & (NW - 1), jc1 = (2 * warp + 1 + r) & (NW - 1);
                        const int lc0 = J * NW + jc0, lc1 = J * NW + jc1;
                        if (r > 0) {
                            const bool t = test_wait && r == 1;
                            ok = counter_wait_bounded(&done[jc1], t ? 0x7fffffff : base + r, &sh[1],
                                                      t ? (1ll << 20) : (1ll << 31));
                        }
                        if (!ok) break;
                        R be0 = lc0 < cols ? sn2[jc0] : (R)0, be1 = lc1 < cols ? sn2[jc1] : (R)0;
                        C y0[RPL], y1[RPL];
                        slot_load<C, RPL>(y0, buf + (size_t)jc0 * mpad, lane);
                        slot_load<C, RPL>(y1, buf + (size_t)jc1 * mpad, lane);
                        bool r0, r1;
                        pair_rotate2<RPL>(a[0], y0, al[0], be0, mine[0] && lc0 < cols, a[CPW - 1], y1, al[CPW - 1], be1,
                                          mine[CPW - 1] && lc1 < cols, tol2, big2, big_w, buf + (size_t)jc0 * mpad,
                                          buf + (size_t)jc1 * mpad, r0, r1);
                        if (r0) { sn2[jc0] = be0; ++rot_w; }
                        if (r1) { sn2[jc1] = be1; ++rot_w; }
                        if (r == NW - 1) {
                            if (lc0 < cols) nrm2[cperm[lc0]] = (double)be0;
                            if (lc1 < cols) nrm2[cperm[lc1]] = (double)be1;
                        }
                        __syncwarp();
                        if (lane == 0) {
                            counter_release_add(&done[jc0]);
                            counter_release_add(&done[jc1]);
                        }
                      }
                    }
                    if (!ok) atomicOr(&sh[1], 1);
                    phase[cur] ^= 1u;
                    ++jblocks[cur];
                    // write block J back
                    fence_async_smem();
                    __syncthreads();
                    if (sh[1]) {
                        abort_drain();
                        return;
                    }
                    if (tid == 0) {
                        const int c0 = J * NW;
                        const int nreal = min(NW, cols - c0);
                        for (int c = 0; c < nreal; ++c)
                            bulk_s2g(W + (size_t)cperm[c0 + c] * ldw, buf + (size_t)c * mpad, col_bytes);
                        bulk_commit();
                    }
                    cur = nxt;
                }
            }
            // write block I back
#pragma unroll
            for (int k = 0; k < CPW; ++k)
                if (mine[k]) {
                    col_store<C, RPL>(a[k], W + (size_t)my_col[k] * ldw, lane, rows);
                    if (lane == 0) nrm2[my_col[k]] = (double)al[k];
                }
            fence_async_global();
            __syncthreads();
        }
        if (lane == 0 && rot_w) atomicAdd(&sh[0], rot_w);
        if (lane == 0 && big_w) sh[7] = 1;
        rot_w = 0;
        big_w = false;
        __syncthreads();
        const int rot = sh[0];
        const bool small = Eps<R>::early > 0.0 && sh[7] == 0;
        rot_total += rot;
        __syncthreads();
        if (polishing) { converged = true; ++sweep; break; }
        if (rot == 0 || small) {
            if (polish) {
                polishing = true;
                const R pt = (R)(Eps<R>::polish * sqrt((double)rows) * Eps<R>::u);
                tol2 = pt * pt;
                continue;
            }
            converged = true;
            ++sweep;
            break;
        }
    }
    if (tid == 0) { bulk_wait_all(); fence_async_global(); }
    __syncthreads();
    if (!converged && tid == 0) atomicOr(A.err, DERR_NOT_CONVERGED);
    if (tid == 0 && A.refine) {  // the FP64 resolution of a complex64 state, counted apart
        A.slot_sweeps[j] = sweep;
        atomicAdd(&A.work[8], 1ull);
        atomicAdd(&A.work[9], (unsigned long long)sweep * (unsigned long long)(cols * (cols - 1) / 2) *
                                  (unsigned long long)rows);
    } else if (tid == 0) {
        A.slot_sweeps[j] = sweep;
        atomicAdd(&A.work[0], (unsigned long long)sweep * (unsigned long long)(cols * (cols - 1) / 2) *
                                  (unsigned long long)rows);
        atomicAdd(&A.work[2], (unsigned long long)rot_total);
        atomicAdd(&A.work[3], (unsigned long long)sweep);
        atomicAdd(&A.work[4], 1ull);
        if (A.mode == 1) {  // tSU factors, counted apart as well
            atomicAdd(&A.work[5], (unsigned long long)sweep * (unsigned long long)(cols * (cols - 1) / 2) *
                                      (unsigned long long)rows);
            atomicAdd(&A.work[6], (unsigned long long)sweep);
            atomicAdd(&A.work[7], 1ull);
        }
    }
    // FP64 column norms = singular values; the range guard's scaling is undone and
    // the pair-split layout turned back into plain complex columns
    double* nrm = A.norms + (size_t)j * ldw;
    const R unscale = ldexp((R)1, scale_e);
    for (int c = warp; c < cols; c += NWARPS) {
        double acc = 0.0;
        if constexpr (PairRows<C, RPL>::on) {
            float4* col = reinterpret_cast<float4*>(W + (size_t)c * ldw);
            for (int g = lane; g < rows / 2; g += 32) {
                float4 v = col[g];
                acc = fma((double)v.x, (double)v.x, acc);
                acc = fma((double)v.z, (double)v.z, acc);
                acc = fma((double)v.y, (double)v.y, acc);
                acc = fma((double)v.w, (double)v.w, acc);
                if (scale_e != 0) { v.x *= unscale; v.y *= unscale; v.z *= unscale; v.w *= unscale; }
                col[g] = make_float4(v.x, v.z, v.y, v.w);
            }
        } else {
            for (int r = lane; r < rows; r += 32) {
                C v = W[(size_t)c * ldw + r];
                acc = fma((double)v.x, (double)v.x, acc);
                acc = fma((double)v.y, (double)v.y, acc);
                if (scale_e != 0) {
                    v.x *= unscale; v.y *= unscale;
                    W[(size_t)c * ldw + r] = v;
                }
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const double s = ldexp(sqrt(acc), scale_e);
            if (!isfinite(s)) atomicOr(A.err, DERR_NONFINITE);
            nrm[c] = s;
        }
    }
}

// CTAs per SM the register allocation is held to: the complex64 kernel with
// 8-column blocks (106 KB of shared memory at 512 rows) runs two CTAs per SM,
// 16 warps as with one 16-column CTA, on two independent bonds.
template <typename R, int NW> struct JacobiMinBlocks { static constexpr int v = 1; };
template <> struct JacobiMinBlocks<float, 8> { static constexpr int v = 2; };

template <typename R, int NW>
__global__ void __launch_bounds__(NW * 32, JacobiMinBlocks<R, NW>::v) k_jacobi(LayerArgs<R> A) {
    using C = cx_t<R>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int j = blockIdx.x;
    const int32_t* d = A.dims + j * kDims;
    if (A.refine == 1 && d[D_REFINE] != 1) return;  // the FP64 resolution runs only undecided bonds
    const int rows = A.pass == 1 ? 2 * d[D_CL] : d[D_ROWS];
    const int cols = A.pass == 1 ? d[D_CM] : d[D_COLS];
    C* W = A.w + (size_t)j * A.ldw * A.ldw;
    // zero the three column stages (rows beyond `rows` must read as zero)
    const size_t stage_elems = (size_t)3 * NW * A.ldw;
    C* z = reinterpret_cast<C*>(smem);
    for (size_t e = threadIdx.x; e < stage_elems; e += blockDim.x) z[e] = cmake<C>(0, 0);
    uint64_t* bar = reinterpret_cast<uint64_t*>(z + stage_elems);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        int* sh = reinterpret_cast<int*>(reinterpret_cast<R*>(bar + 2) + 3 * NW);
        for (int i = 0; i < kShInts + 2 * NW; ++i) sh[i] = 0;  // counters, flags, slot round counters
    }
    fence_async_smem();
    __syncthreads();
    const int qa = (rows + 31) / 32;
    if (qa <= 1) jacobi_body<R, NW, 1>(A, W, rows, cols, j, smem);
    else if (qa <= 2) jacobi_body<R, NW, 2>(A, W, rows, cols, j, smem);
    else if (qa <= 4) jacobi_body<R, NW, 4>(A, W, rows, cols, j, smem);
    else if (qa <= 8) jacobi_body<R, NW, 8>(A, W, rows, cols, j, smem);
    else jacobi_body<R, NW, 16>(A, W, rows, cols, j, smem);
}

// Block width (columns of the register block = warps of the CTA).  complex64:
// 16 by default, 8 selectable (a.nw); complex128: 8 (16 columns of complex128
// stages would not fit in shared memory).
// Two columns per warp (jacobi_body with CPW = 2): NW / 2 warps.  Matrices of at
// most 32 rows (one entry per lane, no pair-split layout) take jacobi_body with
// NW / 2 columns, one per warp, instead; the prologue sets up the shared-memory
// layout of the body it calls.
template <int NW>
__global__ void __launch_bounds__(NW * 16, 1) k_jacobi2(LayerArgs<float> A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int j = blockIdx.x;
    const int32_t* d = A.dims + j * kDims;
    if (A.refine == 1 && d[D_REFINE] != 1) return;
    const int rows = A.pass == 1 ? 2 * d[D_CL] : d[D_ROWS];
    const int cols = A.pass == 1 ? d[D_CM] : d[D_COLS];
    float2* W = A.w + (size_t)j * A.ldw * A.ldw;
    const int qa = (rows + 31) / 32;
    const int nwl = qa <= 1 ? NW / 2 : NW;  // columns per block of the body called
    const size_t stage_elems = (size_t)3 * nwl * A.ldw;
    float2* z = reinterpret_cast<float2*>(smem);
    for (size_t e = threadIdx.x; e < stage_elems; e += blockDim.x) z[e] = make_float2(0.f, 0.f);
    uint64_t* bar = reinterpret_cast<uint64_t*>(z + stage_elems);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        int* sh = reinterpret_cast<int*>(reinterpret_cast<float*>(bar + 2) + 3 * nwl);
        for (int i = 0; i < kShInts + 2 * nwl; ++i) sh[i] = 0;
    }
    fence_async_smem();
    __syncthreads();
    if (qa <= 1) jacobi_body<float, NW / 2, 1, 1>(A, W, rows, cols, j, smem);
    else if (qa <= 2) jacobi_body<float, NW, 2, 2>(A, W, rows, cols, j, smem);
    else if (qa <= 4) jacobi_body<float, NW, 4, 2>(A, W, rows, cols, j, smem);
    else if (qa <= 8) jacobi_body<float, NW, 8, 2>(A, W, rows, cols, j, smem);
    else jacobi_body<float, NW, 16, 2>(A, W, rows, cols, j, smem);
}

template <typename R> struct JacobiNW;
template <> struct JacobiNW<float> { static constexpr int v = 16; };
template <> struct JacobiNW<double> { static constexpr int v = 8; };

}  // namespace

int jacobi_block_width(int precision, int requested) {
    if (precision == PTEBD_FP64) return JacobiNW<double>::v;
    return requested == 8 ? 8 : JacobiNW<float>::v;
}

size_t jacobi_smem_bytes(int precision, int ldw, int nw) {
    const size_t elem = precision == PTEBD_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t real = precision == PTEBD_FP64 ? sizeof(double) : sizeof(float);
    return (size_t)3 * nw * ldw * elem + 2 * sizeof(uint64_t) + 3 * nw * real + (kShInts + 2 * nw) * sizeof(int) +
           (size_t)kSortN * (sizeof(int) + sizeof(float)) + 8 + (size_t)kSortN * sizeof(double) + kSortN;
}

template <typename R> cudaError_t jacobi_prepare() {
    const int prec = std::is_same<R, double>::value ? PTEBD_FP64 : PTEBD_MIXED;
    constexpr int NW = JacobiNW<R>::v;
    cudaError_t e = cudaFuncSetAttribute(k_jacobi<R, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)jacobi_smem_bytes(prec, 2 * PTEBD_CHI_LIMIT, NW));
    if constexpr (std::is_same<R, float>::value) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_jacobi<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)jacobi_smem_bytes(prec, 2 * PTEBD_CHI_LIMIT, 8));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_jacobi2<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)jacobi_smem_bytes(prec, 2 * PTEBD_CHI_LIMIT, 16));
    }
    return e;
}

template <typename R> cudaError_t launch_jacobi(const LayerArgs<R>& a, cudaStream_t s) {
    const int prec = std::is_same<R, double>::value ? PTEBD_FP64 : PTEBD_MIXED;
    const int nw = jacobi_block_width(prec, a.nw);
    const size_t smem = jacobi_smem_bytes(prec, a.ldw, nw);
    if constexpr (std::is_same<R, double>::value) {
        k_jacobi<R, 8><<<a.count, 8 * 32, smem, s>>>(a);  // complex128: 8-column blocks only
    } else {
        if (nw == 16 && a.pairs == 2)  // two columns per warp: 8 warps
            k_jacobi2<16><<<a.count, 16 * 16, smem, s>>>(a);
        else if (nw == 8)
            k_jacobi<R, 8><<<a.count, 8 * 32, smem, s>>>(a);
        else
            k_jacobi<R, 16><<<a.count, 16 * 32, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t jacobi_prepare<float>();
template cudaError_t jacobi_prepare<double>();
template cudaError_t launch_jacobi<float>(const LayerArgs<float>&, cudaStream_t);
template cudaError_t launch_jacobi<double>(const LayerArgs<double>&, cudaStream_t);

}  // namespace ptebd
