// C ABI of libptebd (declared in include/ptebd.h): state layout in the caller's
// device buffers, the layer driver of Algorithm 1 (arXiv:2312.02667) and the
// host side of the contractions.  All device work is issued on the handle's
// stream; the library never allocates device memory.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ptebd_internal.h"

using namespace ptebd;

struct ptebd_state {
    ptebd_config cfg;
    Layout L;
    char* mem = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int slots = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int layers = 0;
    std::string last_error;
    // per-kernel CUDA-event timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_kind;  // kind of each recorded (start, stop) pair
    // concurrent bond chunks of a layer: one stream and one event per chunk, and
    // the fork event (all owned; created on first use)
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> chunk_ev;
    cudaEvent_t fork_ev = nullptr;
    int chunk_streams = 0;  // requested number of chunks (0: chosen from N)
    int wait_test = 0;      // see ptebd_test_wait_timeout
    bool regauge64 = false; // PTEBD_MIXED: tSU stages run in FP64 (ptebd_set_regauge_precision)
    int jacobi_nw = 0;      // Jacobi block width (0: default; see ptebd_set_jacobi_width)
    int jacobi_pairs = 1;   // I columns per warp at width 16 (ptebd_set_jacobi_pairs)
    int ptsu_shortcut = 1;  // leave out the identity half-step after a layer on bonds 0, 2, 4, ... (see run_layer)
    int tensor_cores = 1;   // complex64 theta' on the tensor cores (ptebd_set_tensor_cores)
    int polish = 2;         // complex64 Jacobi polish sweep: 0 none, 1 gated SVDs, 2 gated and tSU, 3 tSU
    cudaStream_t body_stream = nullptr;  // captures the bodies of the FP64 pass's IF nodes (owned)
    // set once a device error says that a CTA returned with its own bulk copies still in
    // flight (DERR_DRAIN): the state and its workspace can no longer be trusted, and
    // every later call that launches work on it fails until it is destroyed
    bool poisoned = false;
    ~ptebd_state() {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        for (cudaEvent_t e : chunk_ev) cudaEventDestroy(e);
        if (fork_ev) cudaEventDestroy(fork_ev);
        for (cudaStream_t x : aux) cudaStreamDestroy(x);
        if (body_stream) cudaStreamDestroy(body_stream);
    }
};

namespace ptebd {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Complex64 singular values at or below 1e-6 sigma_1 are not trusted by default:
// where the exact spectrum has zeros, the rounding of theta' and of the
// rotations leaves values of up to about 5e-8 sigma_1 (measured on Trotter,
// CZ and SWAP-routed circuits), while real values above 1e-6 sigma_1 come out
// with relative errors below 1e-2 (graded spectra keep their relative accuracy).
constexpr double kResolveDefault = 1e-6;

static int chip_for(int chi_max) {
    int c = 16;
    while (c < chi_max) c <<= 1;
    return c;
}

// PTEBD_MIXED: the relative level below which complex64 singular values are not
// trusted (the config's `resolve`, negative = the default).
double resolve_level(const ptebd_config& c) {
    if (c.precision != PTEBD_MIXED) return 0.0;
    return c.resolve < 0.0 ? kResolveDefault : c.resolve;
}

Layout make_layout(const ptebd_config& cfg) {
    Layout L;
    L.n_sites = cfg.n_sites;
    L.chi_max = cfg.chi_max;
    L.chip = chip_for(cfg.chi_max);
    L.ldw = 2 * L.chip;
    L.precision = cfg.precision;
    L.max_bonds = cfg.n_sites / 2;  // ceil((N-1)/2)
    L.elem = cfg.precision == PTEBD_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t N = (size_t)cfg.n_sites, chip = (size_t)L.chip, nb = (size_t)L.max_bonds;
    size_t o = 0;
    L.off_gamma = o; o = align256(o + N * 2 * chip * chip * L.elem);
    L.off_lam = o; o = align256(o + (N + 1) * chip * sizeof(double));
    L.off_chi = o; o = align256(o + (N + 1) * sizeof(int32_t));
    L.off_bond_eps = o; o = align256(o + N * sizeof(double));
    L.off_bond_nu = o; o = align256(o + N * sizeof(double));
    L.off_bond_rank = o; o = align256(o + N * sizeof(int32_t));
    L.off_bond_sweeps = o; o = align256(o + N * sizeof(int32_t));
    L.off_totals = o; o = align256(o + 8 * sizeof(double) + kWork * sizeof(unsigned long long));
    L.off_err = o; o = align256(o + sizeof(uint32_t));
    L.off_gates = o; o = align256(o + nb * 32 * sizeof(double));
    L.off_bonds = o; o = align256(o + 3 * nb * sizeof(int32_t));
    L.off_scratch = o; o = align256(o + 8 * chip * chip * sizeof(double2) + 8 * sizeof(double));
    L.off_partials = o; o = align256(o + (size_t)kMaxChunks * 4 * sizeof(double));
    L.state_bytes = o;
    const size_t ldw = (size_t)L.ldw;
    L.slot_w = align256(ldw * ldw * L.elem);
    L.slot_small = 2 * ldw * sizeof(double) + ldw * sizeof(int32_t) + kDims * sizeof(int32_t) +
                   2 * sizeof(double) + sizeof(int32_t);
    L.resolve = resolve_level(cfg);
    L.resolve64 = cfg.precision == PTEBD_MIXED && L.resolve > cfg.cutoff;
    L.slot_r = L.resolve64 ? align256(ldw * ldw * sizeof(double2)) : 0;
    L.slot_bytes = 3 * L.slot_w + 2 * L.slot_r + L.slot_small;
    return L;
}

}  // namespace ptebd

namespace {

// Workspace regions for `slots` slots.
struct WsView {
    void* w; void* w0; void* w1; double* norms; double* sig; int32_t* perm; int32_t* dims;
    double* slot_eps; double* slot_lognu; int32_t* slot_sweeps;
    double2* r; double2* r0;  // FP64 resolution matrices (null when the config has none)
    size_t bytes;
};

WsView ws_view(const Layout& L, char* base, int slots) {
    WsView v{};
    const size_t ldw = (size_t)L.ldw, s = (size_t)slots;
    size_t o = 0;
    v.w = base + o; o = align256(o + s * L.slot_w);
    v.w0 = base + o; o = align256(o + s * L.slot_w);
    v.w1 = base + o; o = align256(o + s * L.slot_w);
    v.norms = reinterpret_cast<double*>(base + o); o = align256(o + s * ldw * sizeof(double));
    v.sig = reinterpret_cast<double*>(base + o); o = align256(o + s * ldw * sizeof(double));
    v.perm = reinterpret_cast<int32_t*>(base + o); o = align256(o + s * ldw * sizeof(int32_t));
    v.dims = reinterpret_cast<int32_t*>(base + o); o = align256(o + s * kDims * sizeof(int32_t));
    v.slot_eps = reinterpret_cast<double*>(base + o); o = align256(o + s * sizeof(double));
    v.slot_lognu = reinterpret_cast<double*>(base + o); o = align256(o + s * sizeof(double));
    v.slot_sweeps = reinterpret_cast<int32_t*>(base + o); o = align256(o + s * sizeof(int32_t));
    v.r = v.r0 = nullptr;
    if (L.slot_r) {
        v.r = reinterpret_cast<double2*>(base + o); o = align256(o + s * L.slot_r);
        v.r0 = reinterpret_cast<double2*>(base + o); o = align256(o + s * L.slot_r);
    }
    v.bytes = o;
    return v;
}

size_t ws_bytes_for(const Layout& L, int slots) { return ws_view(L, nullptr, slots).bytes; }

int set_err(ptebd_state* st, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int set_err(ptebd_state* st, int code, const char* fmt, ...) {
    if (st) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        st->last_error = buf;
    }
    return code;
}

#define CUDA_TRY(st, call)                                                                              \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return set_err((st), PTEBD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

int validate_config(const ptebd_config* c, std::string* why) {
    if (!c) { *why = "null config"; return PTEBD_ERR_INVALID; }
    if (c->d != 2) { *why = "only d = 2 is supported"; return PTEBD_ERR_UNSUPPORTED; }
    if (c->n_sites < 2) { *why = "n_sites must be >= 2"; return PTEBD_ERR_INVALID; }
    if (c->chi_max < 1) { *why = "chi_max must be >= 1"; return PTEBD_ERR_INVALID; }
    if (c->chi_max > PTEBD_CHI_LIMIT) { *why = "chi_max above PTEBD_CHI_LIMIT"; return PTEBD_ERR_UNSUPPORTED; }
    if (c->precision != PTEBD_FP64 && c->precision != PTEBD_MIXED) { *why = "bad precision"; return PTEBD_ERR_INVALID; }
    if (c->eps_mode != PTEBD_EPS_SCHMIDT && c->eps_mode != PTEBD_EPS_ABSOLUTE && c->eps_mode != PTEBD_EPS_RELATIVE) {
        *why = "bad eps_mode";
        return PTEBD_ERR_INVALID;
    }
    if (c->g < 0) { *why = "g must be >= 0"; return PTEBD_ERR_INVALID; }
    if (!(c->cutoff >= 0.0) || !std::isfinite(c->cutoff)) { *why = "cutoff must be finite and >= 0"; return PTEBD_ERR_INVALID; }
    if (std::isnan(c->resolve) || std::isinf(c->resolve)) { *why = "resolve must be finite"; return PTEBD_ERR_INVALID; }
    return PTEBD_OK;
}

template <typename T> T* at(char* base, size_t off) { return reinterpret_cast<T*>(base + off); }

__global__ void k_init_state(char* mem, Layout L) {
    const size_t N = (size_t)L.n_sites, chip = (size_t)L.chip, slice = chip * chip;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    double* lam = reinterpret_cast<double*>(mem + L.off_lam);
    int32_t* chi = reinterpret_cast<int32_t*>(mem + L.off_chi);
    double* nu = reinterpret_cast<double*>(mem + L.off_bond_nu);
    int32_t* bonds = reinterpret_cast<int32_t*>(mem + L.off_bonds);
    for (size_t s = tid; s < N; s += stride) {
        // |0>: Gamma_s[0](0,0) = 1
        if (L.precision == PTEBD_FP64)
            reinterpret_cast<double2*>(mem + L.off_gamma)[s * 2 * slice] = make_double2(1.0, 0.0);
        else
            reinterpret_cast<float2*>(mem + L.off_gamma)[s * 2 * slice] = make_float2(1.f, 0.f);
        nu[s] = 1.0;
    }
    for (size_t r = tid; r <= N; r += stride) { lam[r * chip] = 1.0; chi[r] = 1; }
    const size_t nb = (size_t)L.max_bonds;
    for (size_t i = tid; i < nb; i += stride) {
        bonds[i] = (int32_t)(2 * i);                                   // even bonds
        bonds[nb + i] = (2 * i + 1 <= N - 2) ? (int32_t)(2 * i + 1) : -1;  // odd bonds
    }
}

int n_parity_bonds(int n_sites, int parity) { return parity == 0 ? n_sites / 2 : (n_sites - 1) / 2; }

cudaEvent_t next_event(ptebd_state* st) {
    if (st->ev_used == st->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        st->ev_pool.push_back(e);
    }
    return st->ev_pool[st->ev_used++];
}

// Launch `f` and, when timing is on, bracket it with events of kind `kind`.
template <typename F>
cudaError_t timed(ptebd_state* st, int kind, F&& f) {
    if (!st->timing) return f();
    cudaEvent_t a = next_event(st), b = next_event(st);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, st->stream);
    if (e != cudaSuccess) return e;
    e = f();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(b, st->stream);
    st->ev_kind.push_back(kind);
    return e;
}

// Chunks of a layer.  Bonds are split by site range into k chunks of `width`
// consecutive bond indices; a stage (the gated bonds, or one half-step of PtSU)
// has at most `cap` bonds in a chunk (its bonds never share a site).  A bond
// reads and writes only the tensors of its own two sites and the Lambdas of
// its neighbours, so a chunk of one stage depends only on chunks c-1, c, c+1
// of the stage before.
struct ChunkPlan { int k = 1, width = 0, cap = 0; };

ChunkPlan chunk_plan(const Layout& L, int requested) {
    ChunkPlan p;
    int k = requested > 0 ? requested : std::min(8, L.max_bonds / 32);
    k = std::max(1, std::min(k, std::min(kMaxChunks, std::max(1, (L.n_sites - 1) / 2))));
    p.k = k;
    p.width = (L.n_sites - 1 + k - 1) / k;
    p.cap = (p.width + 1) / 2;
    return p;
}

int slots_wanted(const Layout& L) {
    const ChunkPlan p = chunk_plan(L, 0);
    return std::max(L.max_bonds, p.k * p.cap);
}

// One stage of a layer: bonds d_list[0..nb) (ascending when h_list or parity
// says so), gates for a gated stage.
struct Stage {
    const int32_t* d_list;
    const int32_t* h_list;  // host copy of an explicit list, or nullptr for a parity list
    int parity;             // parity of the list when h_list == nullptr
    int nb;
    const double* d_gates;
    bool gated;
};

// Positions [off, off + cnt) of the stage's bonds inside [lo, hi).
void segment(const Stage& g, int lo, int hi, int* off, int* cnt) {
    int a, b;
    if (g.h_list) {
        a = (int)(std::lower_bound(g.h_list, g.h_list + g.nb, lo) - g.h_list);
        b = (int)(std::lower_bound(g.h_list, g.h_list + g.nb, hi) - g.h_list);
    } else {
        a = std::min(g.nb, std::max(0, (lo - g.parity + 1) / 2));
        b = std::min(g.nb, std::max(0, (hi - g.parity + 1) / 2));
    }
    *off = a;
    *cnt = std::max(0, b - a);
}

template <typename R>
LayerArgs<R> stage_args(ptebd_state* st, bool gated) {
    const Layout& L = st->L;
    char* m = st->mem;
    WsView ws = ws_view(L, st->ws, st->slots);
    LayerArgs<R> a{};
    a.gamma = m + L.off_gamma;
    a.lam = at<double>(m, L.off_lam);
    a.chi = at<int32_t>(m, L.off_chi);
    a.w = reinterpret_cast<cx_t<R>*>(ws.w);
    a.w0 = reinterpret_cast<cx_t<R>*>(ws.w0);
    a.w1 = reinterpret_cast<cx_t<R>*>(ws.w1);
    a.mode = gated ? 0 : 1;
    a.pass = 0;
    a.norms = ws.norms; a.sig = ws.sig; a.perm = ws.perm; a.dims = ws.dims;
    a.slot_eps = ws.slot_eps; a.slot_lognu = ws.slot_lognu; a.slot_sweeps = ws.slot_sweeps;
    a.chip = L.chip; a.ldw = L.ldw; a.n_sites = L.n_sites; a.chi_max = L.chi_max;
    a.thr_rel = st->cfg.cutoff;
    a.resolve = L.resolve64 ? L.resolve : 0.0;
    a.refine = 0;
    a.eps_mode = st->cfg.eps_mode;
    a.stabilise = gated ? 1 : 0;
    a.max_sweeps = 40;
    a.nw = st->jacobi_nw;
    a.pairs = st->jacobi_pairs;
    a.tensor_cores = st->tensor_cores;
    a.polish = (gated && (st->polish == 1 || st->polish == 2)) || (!gated && st->polish >= 2) ? 1 : 0;
    a.wait_test = st->wait_test;
    a.bond_eps = at<double>(m, L.off_bond_eps);
    a.bond_nu = at<double>(m, L.off_bond_nu);
    a.bond_rank = at<int32_t>(m, L.off_bond_rank);
    a.bond_sweeps = at<int32_t>(m, L.off_bond_sweeps);
    a.totals = at<double>(m, L.off_totals);
    a.err = at<uint32_t>(m, L.off_err);
    a.work = reinterpret_cast<unsigned long long*>(at<double>(m, L.off_totals) + 8);
    return a;
}

// The workspace slots [base, base + count) of `a`.
template <typename R>
void at_slots(LayerArgs<R>& a, const Layout& L, int base) {
    const size_t ldw = (size_t)L.ldw, b = (size_t)base;
    const size_t per_w = L.slot_w / sizeof(cx_t<R>);
    a.w += b * per_w; a.w0 += b * per_w; a.w1 += b * per_w;
    a.norms += b * ldw; a.sig += b * ldw; a.perm += b * ldw; a.dims += b * kDims;
    a.slot_eps += b; a.slot_lognu += b; a.slot_sweeps += b;
}

// Arguments of the FP64 resolution pass over the same slots (and bonds, gates,
// counts) as the complex64 pass `c`: FP64 matrices in the r / r0 regions (slot j
// at j ldw^2 complex128 elements, as the kernels index them), the small per-slot
// arrays shared with the complex64 pass (dead for an undecided bond, untouched
// for the others), the cutoff alone as threshold.  For tSU the X factor takes
// the first chip columns of r and M^dag the last chip columns.
LayerArgs<double> refine_args(ptebd_state* st, const LayerArgs<float>& c, int base) {
    const Layout& L = st->L;
    WsView ws = ws_view(L, st->ws, st->slots);
    LayerArgs<double> a{};
    a.gamma = c.gamma; a.lam = c.lam; a.chi = c.chi;
    const size_t per = (size_t)L.ldw * L.ldw, b = (size_t)base;
    a.w = ws.r + b * per;
    a.w0 = ws.r0 + b * per;
    a.w1 = a.w + (size_t)L.chip * L.ldw;
    a.norms = c.norms; a.sig = c.sig; a.perm = c.perm; a.dims = c.dims;
    a.slot_eps = c.slot_eps; a.slot_lognu = c.slot_lognu; a.slot_sweeps = c.slot_sweeps;
    a.bonds = c.bonds; a.gates = c.gates;
    a.count = c.count; a.chip = c.chip; a.ldw = c.ldw; a.n_sites = c.n_sites; a.chi_max = c.chi_max;
    a.thr_rel = st->cfg.cutoff;
    a.resolve = 0.0;
    a.refine = 1;
    a.eps_mode = c.eps_mode; a.stabilise = c.stabilise; a.max_sweeps = c.max_sweeps; a.wait_test = 0; a.nw = 0;
    a.mode = c.mode; a.pass = 0;
    a.bond_eps = c.bond_eps; a.bond_nu = c.bond_nu; a.bond_rank = c.bond_rank; a.bond_sweeps = c.bond_sweeps;
    a.totals = c.totals; a.err = c.err; a.work = c.work;
    a.w32 = c.w;  // a gated bond's FP64 SVD starts from the complex64 one (k_precond)
    return a;
}

// The kernels of one stage on a.count bonds (slots and bonds already set), on
// stream s, Gamma stored as G; `wrap(kind, launch)` brackets each launch.  With
// a.refine every kernel runs only the bonds the complex64 pass left undecided.
template <typename R, typename G, typename W>
int launch_pass(ptebd_state* st, LayerArgs<R> a, bool gated, cudaStream_t s, W&& wrap) {
    const int kt = a.refine ? PTEBD_K_RESOLVE : PTEBD_K_THETA, ks = a.refine ? PTEBD_K_RESOLVE : PTEBD_K_SVD,
              kc = a.refine ? PTEBD_K_RESOLVE : PTEBD_K_TRUNCATE, kg = a.refine ? PTEBD_K_RESOLVE : PTEBD_K_GAMMA,
              kf = a.refine ? PTEBD_K_RESOLVE : PTEBD_K_FACTOR;
    if (gated) {
        CUDA_TRY(st, wrap(kt, [&] { return launch_theta<R, G>(a, s); }));
        if constexpr (std::is_same<R, double>::value)
            if (a.refine == 1 && a.w32) CUDA_TRY(st, wrap(kt, [&] { return launch_precond(a, s); }));
        CUDA_TRY(st, wrap(ks, [&] { return launch_jacobi<R>(a, s); }));
        CUDA_TRY(st, wrap(kc, [&] { return launch_truncate<R>(a, s); }));
        CUDA_TRY(st, wrap(kg, [&] { return launch_gamma<R, G>(a, s); }));
    } else {
        // tSU: SVD of theta = X Y through its rank-chi_b factors
        LayerArgs<R> x = a;
        x.pass = 1;
        LayerArgs<R> y = a;
        y.w = a.w1;
        CUDA_TRY(st, wrap(kt, [&] { return launch_theta<R, G>(a, s); }));
        CUDA_TRY(st, wrap(kf, [&] { return launch_xform<R, G>(x, s); }));
        CUDA_TRY(st, wrap(kf, [&] { return launch_orth<R>(x, s); }));
        CUDA_TRY(st, wrap(kf, [&] { return launch_proj<R>(x, s); }));
        CUDA_TRY(st, wrap(ks, [&] { return launch_jacobi<R>(y, s); }));
        CUDA_TRY(st, wrap(kc, [&] { return launch_truncate<R>(y, s); }));
        CUDA_TRY(st, wrap(kg, [&] { return launch_gamma<R, G>(y, s); }));
    }
    return PTEBD_OK;
}

// The kernel chain of one stage on a.count bonds starting at workspace slot
// `base` (a already points there), on stream s; for a complex64 state with FP64
// resolution the FP64 pass over the undecided bonds follows, then the sums.
template <typename R, typename W>
int launch_chain(ptebd_state* st, LayerArgs<R> a, int base, bool gated, cudaStream_t s, W&& wrap) {
    int rc = PTEBD_OK;
    bool done = false;
    if constexpr (std::is_same<R, float>::value) {
        if (!gated && st->regauge64) {  // the whole tSU stage in FP64
            LayerArgs<double> f = refine_args(st, a, base);
            f.refine = 2;
            rc = launch_pass<double, float2>(st, f, gated, s, wrap);
            if (rc) return rc;
            done = true;
        }
    }
    if (!done) {
        // The FP64 resolution pass runs only for bonds the complex64 truncation
        // leaves undecided, which it usually leaves none.  Launched directly, its
        // CTAs return at once; inside a stream capture (the batch graphs) it
        // becomes an IF node that the truncation switches on, so that a graph of
        // many small states launches no idle kernels (they would wait for whole
        // SMs behind the other states' Jacobi CTAs).
        bool as_if = false;
        if constexpr (std::is_same<R, float>::value) {
            if (st->L.resolve64) {
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                CUDA_TRY(st, cudaStreamIsCapturing(s, &cs));
                if (cs == cudaStreamCaptureStatusActive) {
                    cudaGraph_t g = nullptr;
                    CUDA_TRY(st, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
                    cudaGraphConditionalHandle h = 0;
                    CUDA_TRY(st, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
                    a.cond = h;
                    as_if = true;
                }
            }
        }
        rc = launch_pass<R, cx_t<R>>(st, a, gated, s, wrap);
        if (rc) return rc;
        if constexpr (std::is_same<R, float>::value) {
            if (st->L.resolve64 && !as_if) {
                rc = launch_pass<double, float2>(st, refine_args(st, a, base), gated, s, wrap);
                if (rc) return rc;
            } else if (as_if) {
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                cudaGraph_t g = nullptr;
                const cudaGraphNode_t* deps = nullptr;
                const cudaGraphEdgeData* edges = nullptr;
                size_t nd = 0;
                CUDA_TRY(st, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd));
                cudaGraphNodeParams p{};
                p.type = cudaGraphNodeTypeConditional;
                p.conditional.handle = a.cond;
                p.conditional.type = cudaGraphCondTypeIf;
                p.conditional.size = 1;
                cudaGraphNode_t node = nullptr;
                CUDA_TRY(st, cudaGraphAddNode(&node, g, deps, edges, nd, &p));
                cudaGraph_t body = p.conditional.phGraph_out[0];
                CUDA_TRY(st, cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
                CUDA_TRY(st, cudaStreamBeginCaptureToGraph(st->body_stream, body, nullptr, nullptr, 0,
                                                           cudaStreamCaptureModeRelaxed));
                LayerArgs<double> f = refine_args(st, a, base);
                f.cond = 0;
                rc = launch_pass<double, float2>(st, f, gated, st->body_stream, wrap);
                cudaGraph_t out = nullptr;
                const cudaError_t e = cudaStreamEndCapture(st->body_stream, &out);
                if (rc) return rc;
                if (e != cudaSuccess)
                    return set_err(st, PTEBD_ERR_CUDA, "capturing the FP64 pass failed: %s", cudaGetErrorString(e));
            }
        }
    }
    CUDA_TRY(st, wrap(PTEBD_K_REDUCE, [&] {
                 return launch_reduce_layer(a.slot_eps, a.slot_lognu, a.count, gated ? 1 : 0, a.totals, s);
             }));
    return PTEBD_OK;
}

// One stage on the state's stream, in pieces of at most `slots` bonds.
template <typename R>
int run_stage_serial(ptebd_state* st, const Stage& g) {
    auto wrap = [&](int kind, auto&& f) { return timed(st, kind, f); };
    for (int c0 = 0; c0 < g.nb; c0 += st->slots) {
        LayerArgs<R> a = stage_args<R>(st, g.gated);
        a.count = std::min(st->slots, g.nb - c0);
        a.bonds = g.d_list + c0;
        a.gates = g.gated ? g.d_gates + (size_t)c0 * 32 : nullptr;
        int rc = launch_chain<R>(st, a, 0, g.gated, st->stream, wrap);
        if (rc) return rc;
    }
    return PTEBD_OK;
}

int ensure_chunk_streams(ptebd_state* st, int k) {
    while ((int)st->aux.size() < k) {
        cudaStream_t x;
        CUDA_TRY(st, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        st->aux.push_back(x);
        cudaEvent_t e;
        CUDA_TRY(st, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        st->chunk_ev.push_back(e);
    }
    if (!st->fork_ev) CUDA_TRY(st, cudaEventCreateWithFlags(&st->fork_ev, cudaEventDisableTiming));
    return PTEBD_OK;
}

// All stages of a call, each split into chunks on concurrent streams.  The
// state's stream forks into the chunk streams and joins them again at the end;
// chunk c of a stage waits for the events of chunks c-1 and c+1 of the stages
// before (its own earlier work is ahead of it on its stream).  Every bond runs
// the same kernels on the same data as on one stream, so the state is
// bit-identical; the per-chunk eps and ln nu sums go to per-chunk partials that
// one kernel adds in chunk order.
template <typename R>
int run_stages_chunked(ptebd_state* st, const std::vector<Stage>& stages, const ChunkPlan& p) {
    int rc = ensure_chunk_streams(st, p.k);
    if (rc) return rc;
    const Layout& L = st->L;
    double* part = at<double>(st->mem, L.off_partials);
    CUDA_TRY(st, cudaMemsetAsync(part, 0, (size_t)kMaxChunks * 4 * sizeof(double), st->stream));
    CUDA_TRY(st, cudaEventRecord(st->fork_ev, st->stream));
    for (int c = 0; c < p.k; ++c) CUDA_TRY(st, cudaStreamWaitEvent(st->aux[c], st->fork_ev, 0));
    auto wrap = [](int, auto&& f) { return f(); };
    bool recorded[kMaxChunks] = {};
    for (const Stage& g : stages) {
        int off[kMaxChunks], cnt[kMaxChunks];
        for (int c = 0; c < p.k; ++c) segment(g, c * p.width, (c + 1) * p.width, &off[c], &cnt[c]);
        // first every wait on the neighbours' previous work, then the launches
        for (int c = 0; c < p.k; ++c) {
            if (!cnt[c]) continue;
            for (int nb : {c - 1, c + 1})
                if (nb >= 0 && nb < p.k && recorded[nb])
                    CUDA_TRY(st, cudaStreamWaitEvent(st->aux[c], st->chunk_ev[nb], 0));
        }
        for (int c = 0; c < p.k; ++c) {
            if (!cnt[c]) continue;
            if (cnt[c] > p.cap) return set_err(st, PTEBD_ERR_INVALID, "chunk %d holds %d bonds", c, cnt[c]);
            LayerArgs<R> a = stage_args<R>(st, g.gated);
            at_slots(a, L, c * p.cap);
            a.count = cnt[c];
            a.bonds = g.d_list + off[c];
            a.gates = g.gated ? g.d_gates + (size_t)off[c] * 32 : nullptr;
            a.totals = part + 4 * c;
            rc = launch_chain<R>(st, a, c * p.cap, g.gated, st->aux[c], wrap);
            if (rc) return rc;
            CUDA_TRY(st, cudaEventRecord(st->chunk_ev[c], st->aux[c]));
            recorded[c] = true;
        }
    }
    for (int c = 0; c < p.k; ++c)
        if (recorded[c]) CUDA_TRY(st, cudaStreamWaitEvent(st->stream, st->chunk_ev[c], 0));
    CUDA_TRY(st, launch_add_partials(part, p.k, at<double>(st->mem, L.off_totals), st->stream));
    return PTEBD_OK;
}

// NVTX range around a host-side call (visible in timeline profilers; a no-op
// without one attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// A gated stage (or none) followed by g PtSU steps.
int refuse_poisoned(ptebd_state* st) {
    return set_err(st, PTEBD_ERR_TIMEOUT, "the state is unusable after an earlier device wait ran out with copies "
                                          "in flight: destroy and re-create it");
}

int run_layer(ptebd_state* st, const Stage* gated_stage, int g) {
    if (st->poisoned) return refuse_poisoned(st);
    NvtxRange range(gated_stage ? (g ? "ptebd layer + PtSU" : "ptebd layer") : "ptebd PtSU");
    const Layout& L = st->L;
    const int32_t* lists = at<int32_t>(st->mem, L.off_bonds);
    std::vector<Stage> stages;
    if (gated_stage && gated_stage->nb > 0) stages.push_back(*gated_stage);
    // A PtSU step is tSU on bonds 0, 2, 4, ... (the paper's odd bonds) then on
    // bonds 1, 3, 5, ....  Right after a gated layer on every bond of parity 0,
    // each of those bonds is in Schmidt form: Gamma_b = Lambda_{b-1}^-1 U and
    // Gamma_{b+1} = V^dag Lambda_{b+1}^-1 with Lambda_b the kept values, and the
    // neighbouring Lambdas are untouched by the layer, so the tSU two-site tensor
    // is U Lambda_b V^dag: its SVD returns the same U, Lambda_b, V (all kept
    // values lie above the cutoff), and the first half-step of the first PtSU
    // step leaves the state as it is.  It is left out (ptebd_set_ptsu_shortcut).
    const bool identity_half = st->ptsu_shortcut && gated_stage && gated_stage->nb > 0 &&
                               gated_stage->h_list == nullptr && gated_stage->parity == 0 &&
                               gated_stage->nb == n_parity_bonds(L.n_sites, 0);
    for (int step = 0; step < g; ++step) {
        if (!(step == 0 && identity_half))
            stages.push_back(Stage{lists, nullptr, 0, n_parity_bonds(L.n_sites, 0), nullptr, false});
        stages.push_back(Stage{lists + L.max_bonds, nullptr, 1, n_parity_bonds(L.n_sites, 1), nullptr, false});
    }
    if (stages.empty()) return PTEBD_OK;
    const ChunkPlan p = chunk_plan(L, st->chunk_streams);
    bool chunked = p.k > 1 && !st->timing && st->slots >= p.k * p.cap;
    for (const Stage& x : stages)
        if (x.h_list && !std::is_sorted(x.h_list, x.h_list + x.nb)) chunked = false;
    const bool f64 = st->cfg.precision == PTEBD_FP64;
    if (chunked) return f64 ? run_stages_chunked<double>(st, stages, p) : run_stages_chunked<float>(st, stages, p);
    for (const Stage& x : stages) {
        int rc = f64 ? run_stage_serial<double>(st, x) : run_stage_serial<float>(st, x);
        if (rc) return rc;
    }
    return PTEBD_OK;
}

int regauge_steps(ptebd_state* st, int g) { return run_layer(st, nullptr, g); }

const double* stage_gates(ptebd_state* st, const double* gates, int n, int on_device, int* rc) {
    *rc = PTEBD_OK;
    if (on_device) return gates;
    double* dst = at<double>(st->mem, st->L.off_gates);
    cudaError_t e = cudaMemcpyAsync(dst, gates, (size_t)n * 32 * sizeof(double), cudaMemcpyHostToDevice, st->stream);
    if (e != cudaSuccess) *rc = set_err(st, PTEBD_ERR_CUDA, "gate upload failed: %s", cudaGetErrorString(e));
    return dst;
}

int check_device_errors(ptebd_state* st) {
    uint32_t err = 0;
    uint32_t* d_err = at<uint32_t>(st->mem, st->L.off_err);
    CUDA_TRY(st, cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    if (!err) return PTEBD_OK;
    CUDA_TRY(st, cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    if (err & DERR_DRAIN) {
        st->poisoned = true;
        return set_err(st, PTEBD_ERR_TIMEOUT,
                       "a bounded device wait ran out and a CTA returned with bulk copies in flight (0x%x): "
                       "destroy and re-create the state",
                       err);
    }
    if (err & DERR_BADARG)
        return set_err(st, PTEBD_ERR_INVALID, "a bond or bond dimension out of range reached the device (0x%x)", err);
    if (err & DERR_TIMEOUT) return set_err(st, PTEBD_ERR_TIMEOUT, "a bounded device wait ran out (0x%x)", err);
    if (err & DERR_NONFINITE) return set_err(st, PTEBD_ERR_NUMERIC, "non-finite singular value (0x%x)", err);
    if (err & DERR_ZERO_THETA) return set_err(st, PTEBD_ERR_NUMERIC, "zero two-site tensor (0x%x)", err);
    if (err & DERR_EPS) return set_err(st, PTEBD_ERR_NUMERIC, "discarded weight >= 1, nu undefined (0x%x)", err);
    if (err & DERR_NOT_CONVERGED) return set_err(st, PTEBD_ERR_NOT_CONVERGED, "Jacobi sweep limit reached (0x%x)", err);
    return set_err(st, PTEBD_ERR_NUMERIC, "device error 0x%x", err);
}

int sync_and_check(ptebd_state* st) {
    if (st->poisoned) return refuse_poisoned(st);
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    return check_device_errors(st);
}

std::vector<int32_t> host_chi(ptebd_state* st, int* rc) {
    std::vector<int32_t> chi((size_t)st->L.n_sites + 1);
    *rc = PTEBD_OK;
    cudaError_t e = cudaMemcpyAsync(chi.data(), at<int32_t>(st->mem, st->L.off_chi), chi.size() * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) *rc = set_err(st, PTEBD_ERR_CUDA, "reading bond dimensions failed: %s", cudaGetErrorString(e));
    return chi;
}

// ------------------------------------------------------------ contraction --
struct Chain {
    ptebd_state* st;       // owns the scratch and the stream
    double2* mat[8];
    double* logacc;
};

Chain chain_of(ptebd_state* st) {
    Chain c;
    c.st = st;
    const size_t chip = (size_t)st->L.chip;
    double2* base = at<double2>(st->mem, st->L.off_scratch);
    for (int i = 0; i < 8; ++i) c.mat[i] = base + (size_t)i * chip * chip;
    c.logacc = reinterpret_cast<double*>(base + 8 * chip * chip);
    return c;
}

template <typename TB>
const TB* gamma_ptr(ptebd_state* st, int site, int sigma) {
    const size_t chip = (size_t)st->L.chip;
    return reinterpret_cast<const TB*>(st->mem + st->L.off_gamma) + ((size_t)site * 2 + sigma) * chip * chip;
}
const double* lam_ptr(ptebd_state* st, int bond) {  // bond in -1..N-1
    return at<double>(st->mem, st->L.off_lam) + (size_t)(bond + 1) * st->L.chip;
}

// Generic GEMM dispatch on the precisions of the two operands.
int gemm(ptebd_state* owner, int m, int n, int k, double2 alpha, const void* A, bool a64, int lda, int opA,
         const void* B, bool b64, int ldb, const double* colscale, double2 beta, double2* Cm, int ldc,
         const double* rowscale) {
    cudaError_t e;
    cudaStream_t s = owner->stream;
    if (a64 && b64)
        e = launch_zgemm<double2, double2>(m, n, k, alpha, (const double2*)A, lda, opA, (const double2*)B, ldb,
                                           colscale, beta, Cm, ldc, rowscale, s);
    else if (a64)
        e = launch_zgemm<double2, float2>(m, n, k, alpha, (const double2*)A, lda, opA, (const float2*)B, ldb,
                                          colscale, beta, Cm, ldc, rowscale, s);
    else if (b64)
        e = launch_zgemm<float2, double2>(m, n, k, alpha, (const float2*)A, lda, opA, (const double2*)B, ldb,
                                          colscale, beta, Cm, ldc, rowscale, s);
    else
        e = launch_zgemm<float2, float2>(m, n, k, alpha, (const float2*)A, lda, opA, (const float2*)B, ldb,
                                         colscale, beta, Cm, ldc, rowscale, s);
    if (e != cudaSuccess) return set_err(owner, PTEBD_ERR_CUDA, "gemm launch failed: %s", cudaGetErrorString(e));
    return PTEBD_OK;
}

const void* gptr(ptebd_state* st, int site, int sigma) {
    return st->cfg.precision == PTEBD_FP64 ? (const void*)gamma_ptr<double2>(st, site, sigma)
                                           : (const void*)gamma_ptr<float2>(st, site, sigma);
}
bool is64(ptebd_state* st) { return st->cfg.precision == PTEBD_FP64; }

const double2 ONE = {1.0, 0.0};
const double2 ZERO = {0.0, 0.0};

// <a| O |b> with O = identity everywhere except a one-site op on `site1` or a
// two-site op on (site2, site2+1) (both -1 for none).  op is row-major complex.
int contract(ptebd_state* a, ptebd_state* b, int site1, int site2, const double* op, double out[2]) {
    ptebd_state* own = a;
    Chain ch = chain_of(own);
    int rc;
    std::vector<int32_t> ca = host_chi(a, &rc);
    if (rc) return rc;
    std::vector<int32_t> cb = host_chi(b, &rc);
    if (rc) return rc;
    const int N = a->L.n_sites, lda_a = a->L.chip, lda_b = b->L.chip, ldc = own->L.chip;
    double2* E = ch.mat[0];
    double2* En = ch.mat[1];
    CUDA_TRY(own, cudaMemsetAsync(ch.logacc, 0, sizeof(double), own->stream));
    CUDA_TRY(own, launch_fill_identity(E, 1, 1, ldc, own->stream));
    auto opc = [&](int r, int c, int dim) { return make_double2(op[2 * (r * dim + c)], op[2 * (r * dim + c) + 1]); };
    int s = 0;
    while (s < N) {
        const int al = ca[s], ar = ca[s + 1], bl = cb[s], br = cb[s + 1];
        const double* lamA = lam_ptr(a, s);
        const double* lamB = lam_ptr(b, s);
        if (s == site1) {
            // T_x = sum_y O[x,y] E M_b[y];  E' = sum_x M_a[x]^dag T_x
            for (int x = 0; x < 2; ++x)
                for (int y = 0; y < 2; ++y)
                    if ((rc = gemm(own, al, br, bl, opc(x, y, 2), E, true, ldc, 0, gptr(b, s, y), is64(b), lda_b, lamB,
                                   y == 0 ? ZERO : ONE, ch.mat[2 + x], ldc, nullptr)))
                        return rc;
            for (int x = 0; x < 2; ++x)
                if ((rc = gemm(own, ar, br, al, ONE, gptr(a, s, x), is64(a), lda_a, 1, ch.mat[2 + x], true, ldc,
                               nullptr, x == 0 ? ZERO : ONE, En, ldc, lamA)))
                    return rc;
            s += 1;
        } else if (s == site2) {
            const int bm = cb[s + 2], am = ca[s + 2];
            const double* lamB2 = lam_ptr(b, s + 1);
            const double* lamA2 = lam_ptr(a, s + 1);
            // R_y = E M_b,s[y]  (al x br)
            for (int y = 0; y < 2; ++y)
                if ((rc = gemm(own, al, br, bl, ONE, E, true, ldc, 0, gptr(b, s, y), is64(b), lda_b, lamB, ZERO,
                               ch.mat[2 + y], ldc, nullptr)))
                    return rc;
            // X_xz = sum_{y,w} O[(x z), (y w)] R_y M_b,s+1[w]   (al x bm)
            for (int x = 0; x < 2; ++x)
                for (int z = 0; z < 2; ++z) {
                    double2* X = ch.mat[4 + 2 * x + z];
                    bool first = true;
                    for (int y = 0; y < 2; ++y)
                        for (int w = 0; w < 2; ++w) {
                            if ((rc = gemm(own, al, bm, br, opc(2 * x + z, 2 * y + w, 4), ch.mat[2 + y], true, ldc, 0,
                                           gptr(b, s + 1, w), is64(b), lda_b, lamB2, first ? ZERO : ONE, X, ldc,
                                           nullptr)))
                                return rc;
                            first = false;
                        }
                }
            // E' = sum_{x,z} M_a,s+1[z]^dag (M_a,s[x]^dag X_xz)
            bool firstE = true;
            for (int x = 0; x < 2; ++x)
                for (int z = 0; z < 2; ++z) {
                    double2* Y = ch.mat[2];
                    if ((rc = gemm(own, ar, bm, al, ONE, gptr(a, s, x), is64(a), lda_a, 1, ch.mat[4 + 2 * x + z], true,
                                   ldc, nullptr, ZERO, Y, ldc, lamA)))
                        return rc;
                    if ((rc = gemm(own, am, bm, ar, ONE, gptr(a, s + 1, z), is64(a), lda_a, 1, Y, true, ldc, nullptr,
                                   firstE ? ZERO : ONE, En, ldc, lamA2)))
                        return rc;
                    firstE = false;
                }
            s += 2;
        } else {
            for (int x = 0; x < 2; ++x) {
                if ((rc = gemm(own, al, br, bl, ONE, E, true, ldc, 0, gptr(b, s, x), is64(b), lda_b, lamB, ZERO,
                               ch.mat[2], ldc, nullptr)))
                    return rc;
                if ((rc = gemm(own, ar, br, al, ONE, gptr(a, s, x), is64(a), lda_a, 1, ch.mat[2], true, ldc, nullptr,
                               x == 0 ? ZERO : ONE, En, ldc, lamA)))
                    return rc;
            }
            s += 1;
        }
        const int rows = ca[s], cols = cb[s];
        CUDA_TRY(own, launch_scale_max(En, rows, cols, ldc, ch.logacc, own->stream));
        std::swap(E, En);
    }
    double2 e00;
    double lg;
    CUDA_TRY(own, cudaMemcpyAsync(&e00, E, sizeof e00, cudaMemcpyDeviceToHost, own->stream));
    CUDA_TRY(own, cudaMemcpyAsync(&lg, ch.logacc, sizeof lg, cudaMemcpyDeviceToHost, own->stream));
    CUDA_TRY(own, cudaStreamSynchronize(own->stream));
    const double sc = std::exp(lg);
    out[0] = e00.x * sc;
    out[1] = e00.y * sc;
    return PTEBD_OK;
}

// Left environments E_0..E_{N-1} of `st` (E_0 = (1); E_{s+1} = sum_x M_s[x]^dag E_s M_s[x]),
// each rescaled by its largest modulus, written to env[s] (chip x chip complex128).
int left_envs(ptebd_state* st, const std::vector<int32_t>& chi, double2* env, double* logacc) {
    const int N = st->L.n_sites, ld = st->L.chip;
    const size_t slice = (size_t)ld * ld;
    Chain ch = chain_of(st);
    CUDA_TRY(st, launch_fill_identity(env, 1, 1, ld, st->stream));
    int rc;
    for (int s = 0; s + 1 < N; ++s) {
        const int al = chi[s], ar = chi[s + 1];
        double2* E = env + (size_t)s * slice;
        double2* En = env + (size_t)(s + 1) * slice;
        const double* lam = lam_ptr(st, s);
        for (int x = 0; x < 2; ++x) {
            if ((rc = gemm(st, al, ar, al, ONE, E, true, ld, 0, gptr(st, s, x), is64(st), ld, lam, ZERO, ch.mat[2],
                           ld, nullptr)))
                return rc;
            if ((rc = gemm(st, ar, ar, al, ONE, gptr(st, s, x), is64(st), ld, 1, ch.mat[2], true, ld, nullptr,
                           x == 0 ? ZERO : ONE, En, ld, lam)))
                return rc;
        }
        CUDA_TRY(st, launch_scale_max(En, ar, ar, ld, logacc, st->stream));
    }
    return PTEBD_OK;
}

// Launch sequence of one gate layer on `st` (gates already staged in the
// state's own device buffer), on whatever stream st->stream currently is.
int layer_launches(ptebd_state* st, int parity) {
    const int nb = n_parity_bonds(st->L.n_sites, parity);
    const int32_t* lists = at<int32_t>(st->mem, st->L.off_bonds);
    const double* dg = at<double>(st->mem, st->L.off_gates);
    const Stage gs{lists + (parity ? st->L.max_bonds : 0), nullptr, parity, nb, dg, true};
    return run_layer(st, &gs, st->cfg.g);
}

}  // namespace

// A set of independent states whose layers are launched together: one CUDA
// graph per parity pattern, each state a parallel branch on its own stream.
struct ptebd_batch {
    std::vector<ptebd_state*> states;
    cudaStream_t capture = nullptr;            // capture stream (owned)
    std::vector<cudaStream_t> branch;          // one per state (owned)
    std::vector<cudaEvent_t> ev;               // fork / join events (owned)
    std::vector<std::pair<std::vector<int32_t>, cudaGraphExec_t>> cache;
    std::string last_error;
    ~ptebd_batch() {
        for (auto& c : cache) cudaGraphExecDestroy(c.second);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaStream_t s : branch) cudaStreamDestroy(s);
        if (capture) cudaStreamDestroy(capture);
    }
};

// Launch configurations chosen by ptebd_autotune, remembered for the process
// and applied by ptebd_create to states of the same shape.
struct TuneKey {
    int chip, precision, n_sites, g;
    bool operator<(const TuneKey& o) const {
        return std::tie(chip, precision, n_sites, g) < std::tie(o.chip, o.precision, o.n_sites, o.g);
    }
};
struct TuneChoice { int nw, chunks, pairs; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tuned;

// N enters by its bucket (the bit length of N - 1): states of similar length
// split into the same chunks and share a choice.
TuneKey tune_key(const ptebd_state* st) {
    int bucket = 0;
    for (int v = st->cfg.n_sites - 1; v > 0; v >>= 1) ++bucket;
    return TuneKey{st->L.chip, st->cfg.precision, bucket, st->cfg.g};
}

// =================================================================== ABI ==
extern "C" {

int ptebd_required_bytes(const ptebd_config* cfg, size_t* state_bytes, size_t* workspace_bytes,
                         size_t* workspace_min_bytes) {
    std::string why;
    int rc = validate_config(cfg, &why);
    if (rc) return rc;
    Layout L = make_layout(*cfg);
    if (state_bytes) *state_bytes = L.state_bytes;
    if (workspace_bytes) *workspace_bytes = ws_bytes_for(L, slots_wanted(L));
    if (workspace_min_bytes) *workspace_min_bytes = ws_bytes_for(L, 1);
    return PTEBD_OK;
}

int ptebd_create(const ptebd_config* cfg, void* state_mem, size_t state_bytes, void* workspace,
                 size_t workspace_bytes, void* stream, ptebd_state** out) {
    if (!out) return PTEBD_ERR_INVALID;
    *out = nullptr;
    std::string why;
    int rc = validate_config(cfg, &why);
    if (rc) return rc;
    Layout L = make_layout(*cfg);
    if (!state_mem || !workspace) return PTEBD_ERR_INVALID;
    if (((uintptr_t)state_mem & 255) || ((uintptr_t)workspace & 255)) return PTEBD_ERR_MEMORY;
    if (state_bytes < L.state_bytes) return PTEBD_ERR_MEMORY;
    int slots = 0;
    const int most = slots_wanted(L);
    while (slots < most && ws_bytes_for(L, slots + 1) <= workspace_bytes) ++slots;
    if (slots < 1) return PTEBD_ERR_MEMORY;
    ptebd_state* st = new (std::nothrow) ptebd_state();
    if (!st) return PTEBD_ERR_MEMORY;
    st->cfg = *cfg;
    st->L = L;
    st->mem = static_cast<char*>(state_mem);
    st->ws = static_cast<char*>(workspace);
    st->ws_bytes = workspace_bytes;
    st->slots = slots;
    st->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&st->device);
    cudaError_t e = cfg->precision == PTEBD_FP64 ? jacobi_prepare<double>() : jacobi_prepare<float>();
    if (e == cudaSuccess) e = cfg->precision == PTEBD_FP64 ? orth_prepare<double>() : orth_prepare<float>();
    if (e == cudaSuccess && cfg->precision == PTEBD_MIXED) e = theta_tc_prepare();
    if (e == cudaSuccess && L.resolve64) e = jacobi_prepare<double>();
    if (e == cudaSuccess && L.resolve64) e = orth_prepare<double>();
    if (e != cudaSuccess) {
        delete st;
        return PTEBD_ERR_CUDA;
    }
    if (L.resolve64 && cudaStreamCreateWithFlags(&st->body_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete st;
        return PTEBD_ERR_CUDA;
    }
    rc = ptebd_reset(st);
    if (!rc) rc = ensure_chunk_streams(st, chunk_plan(L, 0).k);  // created here, never during a capture
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(tune_key(st));
        if (it != g_tuned.end()) {
            st->jacobi_nw = it->second.nw;
            st->jacobi_pairs = it->second.pairs;
            st->chunk_streams = it->second.chunks;
        }
    }
    if (!rc) rc = ensure_chunk_streams(st, chunk_plan(L, st->chunk_streams).k);
    if (rc) {
        delete st;
        return rc;
    }
    *out = st;
    return PTEBD_OK;
}

int ptebd_set_svd_polish(ptebd_state* st, int32_t mode) {
    if (!st || mode < 0 || mode > 3) return set_err(st, PTEBD_ERR_INVALID, "polish mode must be 0, 1, 2 or 3");
    st->polish = mode;
    return PTEBD_OK;
}

int ptebd_set_tensor_cores(ptebd_state* st, int32_t enable) {
    if (!st) return PTEBD_ERR_INVALID;
    st->tensor_cores = enable == 2 ? 2 : (enable ? 1 : 0);
    return PTEBD_OK;
}

int ptebd_set_jacobi_width(ptebd_state* st, int32_t nw) {
    if (!st) return PTEBD_ERR_INVALID;
    if (nw != 0 && nw != 8 && nw != 16) return set_err(st, PTEBD_ERR_INVALID, "Jacobi block width must be 0, 8 or 16");
    st->jacobi_nw = nw;
    return PTEBD_OK;
}

int ptebd_set_ptsu_shortcut(ptebd_state* st, int32_t enable) {
    if (!st) return PTEBD_ERR_INVALID;
    st->ptsu_shortcut = enable ? 1 : 0;
    return PTEBD_OK;
}

int ptebd_set_jacobi_pairs(ptebd_state* st, int32_t pairs) {
    if (!st) return PTEBD_ERR_INVALID;
    if (pairs != 1 && pairs != 2) return set_err(st, PTEBD_ERR_INVALID, "Jacobi columns per warp must be 1 or 2");
    st->jacobi_pairs = pairs;
    return PTEBD_OK;
}

int ptebd_autotune(ptebd_state* st, const double* gates, int32_t parity, int32_t gates_on_device, void* scratch,
                   size_t scratch_bytes, double* best) {
    if (!st) return PTEBD_ERR_INVALID;
    if (parity != 0 && parity != 1) return set_err(st, PTEBD_ERR_INVALID, "parity must be 0 or 1");
    if (!scratch || scratch_bytes < st->L.state_bytes || ((uintptr_t)scratch & 255))
        return set_err(st, PTEBD_ERR_MEMORY, "autotune needs a 256-byte aligned scratch of state_bytes (%zu)",
                       st->L.state_bytes);
    if (st->poisoned) return refuse_poisoned(st);
    const int nb = n_parity_bonds(st->L.n_sites, parity);
    if (nb > 0 && !gates) return set_err(st, PTEBD_ERR_INVALID, "null gates");
    int rc = sync_and_check(st);
    if (rc) return rc;
    // candidates: (block width, columns per warp) x chunk counts the workspace can run concurrently
    std::vector<std::pair<int, int>> widths = {{0, 1}};
    if (st->cfg.precision == PTEBD_MIXED) widths = {{16, 1}, {16, 2}, {8, 1}};
    std::vector<int> chunks;
    for (int k : {1, 2, 4, 8, 12, 16}) {
        const ChunkPlan p = chunk_plan(st->L, k);
        if (p.k == k && (k == 1 || st->slots >= p.k * p.cap)) chunks.push_back(k);
    }
    const int saved_nw = st->jacobi_nw, saved_chunks = st->chunk_streams, saved_pairs = st->jacobi_pairs;
    const bool saved_timing = st->timing;
    st->timing = false;
    CUDA_TRY(st, cudaMemcpyAsync(scratch, st->mem, st->L.state_bytes, cudaMemcpyDeviceToDevice, st->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(st, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_err(st, PTEBD_ERR_CUDA, "event creation failed");
    }
    double best_ms = 1e300, default_ms = -1.0;
    int best_nw = saved_nw, best_chunks = saved_chunks, best_pairs = saved_pairs;
    const int def_nw = jacobi_block_width(st->cfg.precision, saved_nw);
    const int def_pairs = def_nw == 16 ? saved_pairs : 1;
    const int def_k = chunk_plan(st->L, saved_chunks).k;
    for (const auto& wp : widths) {
        const int nw = wp.first, pairs = wp.second;
        for (int k : chunks) {
            st->jacobi_nw = nw;
            st->jacobi_pairs = pairs;
            st->chunk_streams = k;
            if ((rc = ensure_chunk_streams(st, chunk_plan(st->L, k).k))) break;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && !rc; ++rep) {  // the second run is timed
                if (cudaMemcpyAsync(st->mem, scratch, st->L.state_bytes, cudaMemcpyDeviceToDevice, st->stream) !=
                    cudaSuccess) {
                    rc = set_err(st, PTEBD_ERR_CUDA, "state restore failed");
                    break;
                }
                const double* dg = stage_gates(st, gates, nb, gates_on_device, &rc);
                if (rc) break;
                const int32_t* lists = at<int32_t>(st->mem, st->L.off_bonds);
                const Stage gs{lists + (parity ? st->L.max_bonds : 0), nullptr, parity, nb, dg, true};
                if (cudaEventRecord(e0, st->stream) != cudaSuccess) rc = PTEBD_ERR_CUDA;
                if (!rc) rc = run_layer(st, &gs, st->cfg.g);
                if (!rc && cudaEventRecord(e1, st->stream) != cudaSuccess) rc = PTEBD_ERR_CUDA;
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = PTEBD_ERR_CUDA;
                if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PTEBD_ERR_CUDA;
                if (!rc) rc = check_device_errors(st);
            }
            if (rc) break;
            if (jacobi_block_width(st->cfg.precision, nw) == def_nw && pairs == def_pairs && k == def_k) default_ms = ms;
            if (ms < best_ms) { best_ms = ms; best_nw = nw; best_chunks = k; best_pairs = pairs; }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the state as it was, whatever happened above
    const cudaError_t er = cudaMemcpyAsync(st->mem, scratch, st->L.state_bytes, cudaMemcpyDeviceToDevice, st->stream);
    const cudaError_t es = cudaStreamSynchronize(st->stream);
    st->timing = saved_timing;
    if (rc) {
        st->jacobi_nw = saved_nw;
        st->jacobi_pairs = saved_pairs;
        st->chunk_streams = saved_chunks;
        ensure_chunk_streams(st, chunk_plan(st->L, saved_chunks).k);
        return rc;
    }
    if (er != cudaSuccess || es != cudaSuccess) return set_err(st, PTEBD_ERR_CUDA, "state restore failed");
    st->jacobi_nw = best_nw;
    st->jacobi_pairs = best_pairs;
    st->chunk_streams = best_chunks;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[tune_key(st)] = TuneChoice{best_nw, best_chunks, best_pairs};
    }
    if (best) {
        best[0] = jacobi_block_width(st->cfg.precision, best_nw);
        best[1] = best_chunks ? best_chunks : chunk_plan(st->L, 0).k;
        best[2] = best_ms;
        best[3] = default_ms;
        best[4] = best_pairs;
    }
    return ensure_chunk_streams(st, chunk_plan(st->L, best_chunks).k);
}

int ptebd_test_wait_timeout(ptebd_state* st, int32_t enable) {
    if (!st) return PTEBD_ERR_INVALID;
    st->wait_test = enable ? 1 : 0;
    return PTEBD_OK;
}

int ptebd_set_regauge_precision(ptebd_state* st, int32_t precision) {
    if (!st) return PTEBD_ERR_INVALID;
    if (precision != PTEBD_FP64 && precision != PTEBD_MIXED)
        return set_err(st, PTEBD_ERR_INVALID, "precision must be PTEBD_FP64 or PTEBD_MIXED");
    if (st->cfg.precision == PTEBD_FP64) return PTEBD_OK;  // already FP64 throughout
    if (precision == PTEBD_FP64 && !st->L.resolve64)
        return set_err(st, PTEBD_ERR_UNSUPPORTED,
                       "an FP64 regauge needs the FP64 workspace of the resolution (config resolve > cutoff)");
    st->regauge64 = precision == PTEBD_FP64;
    return PTEBD_OK;
}

int ptebd_set_chunk_streams(ptebd_state* st, int32_t n) {
    if (!st || n < 0 || n > kMaxChunks) return set_err(st, PTEBD_ERR_INVALID, "chunk streams must be 0..%d", kMaxChunks);
    st->chunk_streams = n;
    return ensure_chunk_streams(st, chunk_plan(st->L, n).k);
}

int ptebd_destroy(ptebd_state* st) {
    if (!st) return PTEBD_ERR_INVALID;
    delete st;
    return PTEBD_OK;
}

int ptebd_set_stream(ptebd_state* st, void* stream) {
    if (!st) return PTEBD_ERR_INVALID;
    st->stream = static_cast<cudaStream_t>(stream);
    return PTEBD_OK;
}

int ptebd_reset(ptebd_state* st) {
    if (!st) return PTEBD_ERR_INVALID;
    if (st->poisoned) return refuse_poisoned(st);
    CUDA_TRY(st, cudaMemsetAsync(st->mem, 0, st->L.state_bytes, st->stream));
    k_init_state<<<64, 256, 0, st->stream>>>(st->mem, st->L);
    CUDA_TRY(st, cudaGetLastError());
    st->layers = 0;
    return PTEBD_OK;
}

const char* ptebd_last_error(const ptebd_state* st) {
    if (!st) return "null handle";
    return st->last_error.c_str();
}

int ptebd_get_config(const ptebd_state* st, ptebd_config* out) {
    if (!st || !out) return PTEBD_ERR_INVALID;
    *out = st->cfg;
    return PTEBD_OK;
}

int ptebd_apply_layer(ptebd_state* st, const double* gates, int32_t parity, int32_t gates_on_device) {
    if (!st) return PTEBD_ERR_INVALID;
    if (parity != 0 && parity != 1) return set_err(st, PTEBD_ERR_INVALID, "parity must be 0 or 1");
    const int nb = n_parity_bonds(st->L.n_sites, parity);
    if (nb > 0 && !gates) return set_err(st, PTEBD_ERR_INVALID, "null gates");
    int rc;
    const double* dg = stage_gates(st, gates, nb, gates_on_device, &rc);
    if (rc) return rc;
    const int32_t* lists = at<int32_t>(st->mem, st->L.off_bonds);
    const Stage gs{lists + (parity ? st->L.max_bonds : 0), nullptr, parity, nb, dg, true};
    rc = run_layer(st, &gs, st->cfg.g);
    if (rc) return rc;
    ++st->layers;
    return PTEBD_OK;
}

int ptebd_apply_bonds(ptebd_state* st, const int32_t* bonds, int32_t n_bonds, const double* gates,
                      int32_t gates_on_device) {
    if (!st) return PTEBD_ERR_INVALID;
    if (n_bonds < 0 || n_bonds > st->L.max_bonds) return set_err(st, PTEBD_ERR_INVALID, "bad bond count %d", n_bonds);
    if (n_bonds == 0) { ++st->layers; return regauge_steps(st, st->cfg.g); }
    if (!bonds || !gates) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    std::vector<int32_t> sorted(bonds, bonds + n_bonds);
    std::sort(sorted.begin(), sorted.end());
    for (int i = 0; i < n_bonds; ++i) {
        if (sorted[i] < 0 || sorted[i] > st->L.n_sites - 2)
            return set_err(st, PTEBD_ERR_INVALID, "bond %d out of range", sorted[i]);
        if (i && sorted[i] - sorted[i - 1] < 2)
            return set_err(st, PTEBD_ERR_OVERLAP, "bonds %d and %d share a site", sorted[i - 1], sorted[i]);
    }
    int32_t* dl = at<int32_t>(st->mem, st->L.off_bonds) + 2 * st->L.max_bonds;
    CUDA_TRY(st, cudaMemcpyAsync(dl, bonds, (size_t)n_bonds * sizeof(int32_t), cudaMemcpyHostToDevice, st->stream));
    int rc;
    const double* dg = stage_gates(st, gates, n_bonds, gates_on_device, &rc);
    if (rc) return rc;
    const Stage gs{dl, bonds, 0, n_bonds, dg, true};
    rc = run_layer(st, &gs, st->cfg.g);
    if (rc) return rc;
    ++st->layers;
    return PTEBD_OK;
}

int ptebd_regauge(ptebd_state* st, int32_t g) {
    if (!st || g < 0) return set_err(st, PTEBD_ERR_INVALID, "bad argument");
    return regauge_steps(st, g);
}

int ptebd_sync(ptebd_state* st) {
    if (!st) return PTEBD_ERR_INVALID;
    return sync_and_check(st);
}

int ptebd_norm(ptebd_state* st, double* out) {
    if (!st || !out) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    int rc = sync_and_check(st);
    if (rc) return rc;
    double v[2];
    rc = contract(st, st, -1, -1, nullptr, v);
    if (rc) return rc;
    *out = std::sqrt(std::max(v[0], 0.0));
    return PTEBD_OK;
}

int ptebd_overlap(ptebd_state* a, ptebd_state* b, double out[2]) {
    if (!a || !b || !out) return set_err(a, PTEBD_ERR_INVALID, "null argument");
    if (a->L.n_sites != b->L.n_sites) return set_err(a, PTEBD_ERR_INVALID, "different n_sites");
    if (a->L.chip != b->L.chip) return set_err(a, PTEBD_ERR_INVALID, "overlap needs equal chi_max padding");
    int rc = sync_and_check(a);
    if (rc) return rc;
    if ((rc = sync_and_check(b))) return rc;
    return contract(a, b, -1, -1, nullptr, out);
}

int ptebd_expect(ptebd_state* st, int32_t site, const double* op, double out[2]) {
    if (!st || !op || !out) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    if (site < 0 || site >= st->L.n_sites) return set_err(st, PTEBD_ERR_INVALID, "site out of range");
    int rc = sync_and_check(st);
    if (rc) return rc;
    double num[2], den[2];
    if ((rc = contract(st, st, site, -1, op, num))) return rc;
    if ((rc = contract(st, st, -1, -1, nullptr, den))) return rc;
    out[0] = num[0] / den[0];
    out[1] = num[1] / den[0];
    return PTEBD_OK;
}

int ptebd_expect2(ptebd_state* st, int32_t site, const double* op, double out[2]) {
    if (!st || !op || !out) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    if (site < 0 || site >= st->L.n_sites - 1) return set_err(st, PTEBD_ERR_INVALID, "site out of range");
    int rc = sync_and_check(st);
    if (rc) return rc;
    double num[2], den[2];
    if ((rc = contract(st, st, -1, site, op, num))) return rc;
    if ((rc = contract(st, st, -1, -1, nullptr, den))) return rc;
    out[0] = num[0] / den[0];
    out[1] = num[1] / den[0];
    return PTEBD_OK;
}

int ptebd_get_chi(ptebd_state* st, int32_t* chi_out) {
    if (!st || !chi_out) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    int rc = sync_and_check(st);
    if (rc) return rc;
    std::vector<int32_t> chi = host_chi(st, &rc);
    if (rc) return rc;
    for (int b = 0; b < st->L.n_sites - 1; ++b) chi_out[b] = chi[b + 1];
    return PTEBD_OK;
}

int ptebd_get_lambda(ptebd_state* st, int32_t bond, double* out, int32_t* k) {
    if (!st || !out) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    if (bond < 0 || bond > st->L.n_sites - 2) return set_err(st, PTEBD_ERR_INVALID, "bond out of range");
    int rc = sync_and_check(st);
    if (rc) return rc;
    int32_t kk;
    CUDA_TRY(st, cudaMemcpyAsync(&kk, at<int32_t>(st->mem, st->L.off_chi) + bond + 1, sizeof kk, cudaMemcpyDeviceToHost,
                                 st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    CUDA_TRY(st, cudaMemcpyAsync(out, lam_ptr(st, bond), (size_t)kk * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    if (k) *k = kk;
    return PTEBD_OK;
}

int ptebd_get_site(ptebd_state* st, int32_t site, int32_t* chi_l, int32_t* chi_r, double* gamma_out) {
    if (!st) return PTEBD_ERR_INVALID;
    if (site < 0 || site >= st->L.n_sites) return set_err(st, PTEBD_ERR_INVALID, "site out of range");
    int rc = sync_and_check(st);
    if (rc) return rc;
    std::vector<int32_t> chi = host_chi(st, &rc);
    if (rc) return rc;
    const int cl = chi[site], cr = chi[site + 1];
    if (chi_l) *chi_l = cl;
    if (chi_r) *chi_r = cr;
    if (!gamma_out) return PTEBD_OK;
    const size_t chip = (size_t)st->L.chip, slice = chip * chip;
    const size_t elem = st->L.elem;
    std::vector<char> raw(2 * slice * elem);
    CUDA_TRY(st, cudaMemcpyAsync(raw.data(), st->mem + st->L.off_gamma + (size_t)site * 2 * slice * elem, raw.size(),
                                 cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < cl; ++a)
            for (int b = 0; b < cr; ++b) {
                const size_t src = s * slice + (size_t)b * chip + a;
                const size_t dst = ((size_t)s * cl + a) * cr + b;
                if (elem == sizeof(double2)) {
                    const double2 v = reinterpret_cast<const double2*>(raw.data())[src];
                    gamma_out[2 * dst] = v.x; gamma_out[2 * dst + 1] = v.y;
                } else {
                    const float2 v = reinterpret_cast<const float2*>(raw.data())[src];
                    gamma_out[2 * dst] = v.x; gamma_out[2 * dst + 1] = v.y;
                }
            }
    return PTEBD_OK;
}

int ptebd_set_lambda(ptebd_state* st, int32_t bond, int32_t k, const double* values) {
    if (!st || !values) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    if (bond < 0 || bond > st->L.n_sites - 2) return set_err(st, PTEBD_ERR_INVALID, "bond out of range");
    if (k < 1 || k > st->L.chi_max) return set_err(st, PTEBD_ERR_INVALID, "k out of range");
    std::vector<double> row((size_t)st->L.chip, 0.0);
    std::copy(values, values + k, row.begin());
    CUDA_TRY(st, cudaMemcpyAsync(const_cast<double*>(lam_ptr(st, bond)), row.data(), row.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, st->stream));
    CUDA_TRY(st, cudaMemcpyAsync(at<int32_t>(st->mem, st->L.off_chi) + bond + 1, &k, sizeof k, cudaMemcpyHostToDevice,
                                 st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    return PTEBD_OK;
}

int ptebd_set_site(ptebd_state* st, int32_t site, int32_t chi_l, int32_t chi_r, const double* gamma) {
    if (!st || !gamma) return set_err(st, PTEBD_ERR_INVALID, "null argument");
    if (site < 0 || site >= st->L.n_sites) return set_err(st, PTEBD_ERR_INVALID, "site out of range");
    int rc;
    std::vector<int32_t> chi = host_chi(st, &rc);
    if (rc) return rc;
    if (chi[site] != chi_l || chi[site + 1] != chi_r)
        return set_err(st, PTEBD_ERR_SHAPE, "site %d: got %dx%d, bonds say %dx%d", site, chi_l, chi_r, chi[site],
                       chi[site + 1]);
    const size_t chip = (size_t)st->L.chip, slice = chip * chip, elem = st->L.elem;
    std::vector<char> raw(2 * slice * elem, 0);
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < chi_l; ++a)
            for (int b = 0; b < chi_r; ++b) {
                const size_t dst = s * slice + (size_t)b * chip + a;
                const size_t src = ((size_t)s * chi_l + a) * chi_r + b;
                if (elem == sizeof(double2))
                    reinterpret_cast<double2*>(raw.data())[dst] = make_double2(gamma[2 * src], gamma[2 * src + 1]);
                else
                    reinterpret_cast<float2*>(raw.data())[dst] =
                        make_float2((float)gamma[2 * src], (float)gamma[2 * src + 1]);
            }
    CUDA_TRY(st, cudaMemcpyAsync(st->mem + st->L.off_gamma + (size_t)site * 2 * slice * elem, raw.data(), raw.size(),
                                 cudaMemcpyHostToDevice, st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    return PTEBD_OK;
}

int ptebd_trunc_error(ptebd_state* st, double* eps_total, double* log_nu_total) {
    if (!st) return PTEBD_ERR_INVALID;
    int rc = sync_and_check(st);
    if (rc) return rc;
    double t[8];
    CUDA_TRY(st, cudaMemcpyAsync(t, at<double>(st->mem, st->L.off_totals), sizeof t, cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    if (eps_total) *eps_total = t[0];
    if (log_nu_total) *log_nu_total = t[1];
    return PTEBD_OK;
}

int ptebd_bond_stats(ptebd_state* st, double* eps, double* nu, int32_t* rank_in) {
    if (!st) return PTEBD_ERR_INVALID;
    int rc = sync_and_check(st);
    if (rc) return rc;
    const size_t nb = (size_t)st->L.n_sites - 1;
    if (eps) CUDA_TRY(st, cudaMemcpyAsync(eps, at<double>(st->mem, st->L.off_bond_eps), nb * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    if (nu) CUDA_TRY(st, cudaMemcpyAsync(nu, at<double>(st->mem, st->L.off_bond_nu), nb * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    if (rank_in) CUDA_TRY(st, cudaMemcpyAsync(rank_in, at<int32_t>(st->mem, st->L.off_bond_rank), nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    return PTEBD_OK;
}

int ptebd_work_counters(ptebd_state* st, uint64_t* out, int32_t n) {
    if (!st || !out || n < 0) return PTEBD_ERR_INVALID;
    unsigned long long w[kWork];
    CUDA_TRY(st, cudaMemcpyAsync(w, at<double>(st->mem, st->L.off_totals) + 8, sizeof w, cudaMemcpyDeviceToHost,
                                 st->stream));
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    for (int i = 0; i < std::min(n, kWork); ++i) out[i] = w[i];
    return PTEBD_OK;
}

int ptebd_timing(ptebd_state* st, int32_t enable) {
    if (!st) return PTEBD_ERR_INVALID;
    if (enable) {
        CUDA_TRY(st, cudaStreamSynchronize(st->stream));
        st->ev_used = 0;
        st->ev_kind.clear();
    }
    st->timing = enable != 0;
    return PTEBD_OK;
}

int ptebd_timing_read(ptebd_state* st, double* ms, int32_t* launches, int32_t n_kinds) {
    if (!st || n_kinds < 0) return PTEBD_ERR_INVALID;
    CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    const int nk = std::min<int>(n_kinds, PTEBD_K_COUNT);
    for (int k = 0; k < nk; ++k) {
        if (ms) ms[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    for (size_t i = 0; i < st->ev_kind.size(); ++i) {
        const int k = st->ev_kind[i];
        float t = 0.f;
        CUDA_TRY(st, cudaEventElapsedTime(&t, st->ev_pool[2 * i], st->ev_pool[2 * i + 1]));
        if (k < nk) {
            if (ms) ms[k] += t;
            if (launches) launches[k] += 1;
        }
    }
    return PTEBD_OK;
}

int ptebd_batch_create(ptebd_state* const* states, int32_t n, ptebd_batch** out) {
    if (!out || !states || n < 1) return PTEBD_ERR_INVALID;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!states[i]) return PTEBD_ERR_INVALID;
        for (int k = 0; k < i; ++k)
            if (states[k] == states[i]) return PTEBD_ERR_INVALID;  // a state appears once
    }
    ptebd_batch* b = new (std::nothrow) ptebd_batch();
    if (!b) return PTEBD_ERR_MEMORY;
    b->states.assign(states, states + n);
    bool ok = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess;
    b->branch.resize(n, nullptr);
    b->ev.resize(n + 1, nullptr);
    for (int i = 0; ok && i < n; ++i) ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i <= n; ++i) ok = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        delete b;
        return PTEBD_ERR_CUDA;
    }
    *out = b;
    return PTEBD_OK;
}

int ptebd_batch_destroy(ptebd_batch* b) {
    if (!b) return PTEBD_ERR_INVALID;
    cudaStreamSynchronize(b->capture);
    delete b;
    return PTEBD_OK;
}

const char* ptebd_batch_last_error(const ptebd_batch* b) { return b ? b->last_error.c_str() : "null batch"; }

int ptebd_batch_apply_layer(ptebd_batch* b, const double* const* gates, const int32_t* parities,
                            const int32_t* gates_on_device) {
    if (!b || !parities) return PTEBD_ERR_INVALID;
    const int n = (int)b->states.size();
    std::vector<int32_t> key(parities, parities + n);
    for (int i = 0; i < n; ++i) {
        if (key[i] < -1 || key[i] > 1) { b->last_error = "parity must be -1, 0 or 1"; return PTEBD_ERR_INVALID; }
        if (key[i] >= 0 && n_parity_bonds(b->states[i]->L.n_sites, key[i]) > 0 && (!gates || !gates[i])) {
            b->last_error = "null gates";
            return PTEBD_ERR_INVALID;
        }
    }
    // 1. the branches start after all earlier work of every state; gates are
    //    staged into each state's own buffer (fixed addresses: the graph is reused)
    for (int i = 0; i < n; ++i) {
        ptebd_state* st = b->states[i];
        const int nb = key[i] >= 0 ? n_parity_bonds(st->L.n_sites, key[i]) : 0;
        if (nb > 0) {
            const cudaMemcpyKind kind = (gates_on_device && gates_on_device[i]) ? cudaMemcpyDeviceToDevice
                                                                                 : cudaMemcpyHostToDevice;
            if (cudaMemcpyAsync(at<double>(st->mem, st->L.off_gates), gates[i], (size_t)nb * 32 * sizeof(double), kind,
                                st->stream) != cudaSuccess) {
                b->last_error = "gate staging failed";
                return PTEBD_ERR_CUDA;
            }
        }
        if (cudaEventRecord(b->ev[i], st->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->capture, b->ev[i], 0) != cudaSuccess) {
            b->last_error = "event failed";
            return PTEBD_ERR_CUDA;
        }
    }
    // 2. the graph of this parity pattern (recorded once)
    cudaGraphExec_t exec = nullptr;
    for (auto& c : b->cache)
        if (c.first == key) exec = c.second;
    if (!exec) {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return PTEBD_ERR_CUDA;
        int rc = PTEBD_OK;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PTEBD_ERR_CUDA;
        if (!rc && cudaEventRecord(b->ev[n], cap) != cudaSuccess) rc = PTEBD_ERR_CUDA;
        for (int i = 0; !rc && i < n; ++i) {
            ptebd_state* st = b->states[i];
            const cudaStream_t saved = st->stream;
            const bool timing = st->timing;
            st->timing = false;
            st->stream = b->branch[i];
            if (cudaStreamWaitEvent(b->branch[i], b->ev[n], 0) != cudaSuccess) rc = PTEBD_ERR_CUDA;
            if (!rc && key[i] >= 0) rc = layer_launches(st, key[i]);
            if (!rc && cudaEventRecord(b->ev[i], b->branch[i]) != cudaSuccess) rc = PTEBD_ERR_CUDA;
            if (!rc && cudaStreamWaitEvent(cap, b->ev[i], 0) != cudaSuccess) rc = PTEBD_ERR_CUDA;
            st->stream = saved;
            st->timing = timing;
        }
        const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (!rc && ee != cudaSuccess) rc = PTEBD_ERR_CUDA;
        if (!rc && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = PTEBD_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (rc) {
            b->last_error = "recording the batch graph failed";
            return rc;
        }
        b->cache.emplace_back(key, exec);
    }
    // 3. launch; every state's stream waits for the graph
    if (cudaGraphLaunch(exec, b->capture) != cudaSuccess) {
        b->last_error = "graph launch failed";
        return PTEBD_ERR_CUDA;
    }
    if (cudaEventRecord(b->ev[n], b->capture) != cudaSuccess) return PTEBD_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        ptebd_state* st = b->states[i];
        if (cudaStreamWaitEvent(st->stream, b->ev[n], 0) != cudaSuccess) return PTEBD_ERR_CUDA;
        if (key[i] >= 0) ++st->layers;
    }
    return PTEBD_OK;
}

int ptebd_canonicalize(ptebd_state* st) {
    if (!st) return PTEBD_ERR_INVALID;
    const int n = st->L.n_sites;
    return regauge_steps(st, n % 2 == 0 ? n / 2 : (n - 1) / 2);
}

namespace {
size_t sample_ws_bytes(int n_sites, int chip, int n_samples) {
    const int batch = std::max(1, std::min(n_samples, 1024));
    // N environments, two vector buffers, uniforms and bits of one batch, one log accumulator
    return align256((size_t)n_sites * chip * chip * sizeof(double2)) +
           2 * align256((size_t)batch * chip * sizeof(double2)) + align256((size_t)batch * n_sites * sizeof(double)) +
           align256((size_t)batch * n_sites * sizeof(int32_t)) + 256;
}
}  // namespace

int ptebd_sample_workspace_bytes(const ptebd_state* st, int32_t n_samples, size_t* bytes) {
    if (!st || n_samples < 0 || !bytes) return PTEBD_ERR_INVALID;
    *bytes = sample_ws_bytes(st->L.n_sites, st->L.chip, n_samples);
    return PTEBD_OK;
}

int ptebd_sample(ptebd_state* st, int32_t n_samples, const double* uniforms, int32_t* bits, void* workspace,
                 size_t workspace_bytes) {
    if (!st || n_samples < 0 || (n_samples > 0 && (!uniforms || !bits)))
        return set_err(st, PTEBD_ERR_INVALID, "bad argument");
    if (n_samples == 0) return PTEBD_OK;
    if (workspace && ((uintptr_t)workspace & 255))
        return set_err(st, PTEBD_ERR_INVALID, "the sampling workspace must be 256-byte aligned");
    int rc = sync_and_check(st);
    if (rc) return rc;
    std::vector<int32_t> chi = host_chi(st, &rc);
    if (rc) return rc;
    const int N = st->L.n_sites;
    const size_t chip = (size_t)st->L.chip, slice = chip * chip;
    const int batch = std::min(n_samples, 1024);
    const size_t vec_bytes = (size_t)batch * chip * sizeof(double2);
    const size_t need = sample_ws_bytes(N, (int)chip, n_samples);
    char* w = workspace ? static_cast<char*>(workspace) : st->ws;
    const size_t have = workspace ? workspace_bytes : st->ws_bytes;
    if (need > have)
        return set_err(st, PTEBD_ERR_MEMORY, "sampling needs %zu workspace bytes, %zu given", need, have);
    double2* env = reinterpret_cast<double2*>(w); w += align256((size_t)N * slice * sizeof(double2));
    double2* va = reinterpret_cast<double2*>(w); w += align256(vec_bytes);
    double2* vb = reinterpret_cast<double2*>(w); w += align256(vec_bytes);
    double* du = reinterpret_cast<double*>(w); w += align256((size_t)batch * N * sizeof(double));
    int32_t* db = reinterpret_cast<int32_t*>(w); w += align256((size_t)batch * N * sizeof(int32_t));
    double* logacc = reinterpret_cast<double*>(w);
    CUDA_TRY(st, cudaMemsetAsync(logacc, 0, sizeof(double), st->stream));
    if ((rc = left_envs(st, chi, env, logacc))) return rc;
    for (int k0 = 0; k0 < n_samples; k0 += batch) {
        const int nb = std::min(batch, n_samples - k0);
        CUDA_TRY(st, cudaMemcpyAsync(du, uniforms + (size_t)k0 * N, (size_t)nb * N * sizeof(double),
                                     cudaMemcpyHostToDevice, st->stream));
        const double2* vin = nullptr;  // the right boundary: v = (1)
        double2* vout = va;
        for (int s = N - 1; s >= 0; --s) {
            const int chil = chi[s], chir = chi[s + 1];
            cudaError_t e;
            if (is64(st))
                e = launch_sample_site<double2>(gamma_ptr<double2>(st, s, 0), lam_ptr(st, s), chil, chir, (int)chip,
                                                env + (size_t)s * slice, vin, vout, du, s, N, db, nb, st->stream);
            else
                e = launch_sample_site<float2>(gamma_ptr<float2>(st, s, 0), lam_ptr(st, s), chil, chir, (int)chip,
                                               env + (size_t)s * slice, vin, vout, du, s, N, db, nb, st->stream);
            if (e != cudaSuccess) return set_err(st, PTEBD_ERR_CUDA, "sampling launch failed: %s", cudaGetErrorString(e));
            vin = vout;
            vout = (vout == va) ? vb : va;
        }
        CUDA_TRY(st, cudaMemcpyAsync(bits + (size_t)k0 * N, db, (size_t)nb * N * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st->stream));
        CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    }
    return PTEBD_OK;
}

int ptebd_svd_sweeps(ptebd_state* st, int32_t* sweeps, int32_t* layers) {
    if (!st) return PTEBD_ERR_INVALID;
    int rc = sync_and_check(st);
    if (rc) return rc;
    if (sweeps) {
        CUDA_TRY(st, cudaMemcpyAsync(sweeps, at<int32_t>(st->mem, st->L.off_bond_sweeps),
                                     (size_t)(st->L.n_sites - 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st->stream));
        CUDA_TRY(st, cudaStreamSynchronize(st->stream));
    }
    if (layers) *layers = st->layers;
    return PTEBD_OK;
}

}  // extern "C"
