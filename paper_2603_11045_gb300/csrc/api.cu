// C-ABI of libnefty: argument checks, device workspace, host<->device staging,
// the checkpoint/recompute schedule of the reverse sweep, and the launches of
// the persistent solver kernels (solver.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "nefty.h"

using namespace nefty;

struct nefty_handle {
    int device = 0;
    uint64_t budget = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int grid_max[2] = {0, 0};
    int grid_tiled = 0;
    int grid_share = 1;          // the persistent grids use 1/grid_share of the device (serving lanes)
    nefty::Batcher* batch = nullptr;   // serving: TMA-staged sweeps run in the batcher's shared launches
    int batch_launches = 0;      // launches that carried this handle's sweeps
    int batch_shared = 0;        // ... of which carried other handles' sweeps too
    nefty::Server* server = nullptr;
    std::string err;
    // fault injection of the solver launches (nefty_debug_barrier_fault)
    uint32_t fault_missing = 0;
    uint64_t fault_wait_ns = 0;
    // keep_activations field buffer: a backward-layout field workspace, then
    // the theta and band-weight copies of the evaluation it holds, then a flag
    void* keep = nullptr;
    size_t keep_bytes = 0;
    bool keep_valid = false;     // the buffer holds the evaluation of keep_dims at the copied parameters
    bool keep_bw = false;        // ... with band weights (else none)
    nefty::FieldDims keep_dims{};
    uint64_t field_reuses = 0;
};

void nefty::set_grid_share(nefty_handle* h, int share) { h->grid_share = share > 1 ? share : 1; }
uint64_t nefty::set_budget(nefty_handle* h, uint64_t bytes) {
    const uint64_t old = h->budget;
    h->budget = bytes;
    return old;
}
void nefty::set_batcher(nefty_handle* h, Batcher* b) { h->batch = b; }
void nefty::batch_counts(nefty_handle* h, int* launches, int* shared) {
    *launches = h->batch_launches;
    *shared = h->batch_shared;
}

static thread_local std::string t_err;

void nefty::set_thread_error(const char* msg) { t_err = msg; }

namespace {

// Increments the FP32 CG start extrapolates from when the problem leaves it
// at 0 (quadratic extrapolation).
constexpr int kDefaultExtrap = 3;

nefty_status fail(nefty_handle* h, nefty_status s, const std::string& msg) {
    if (h) h->err = msg;
    t_err = msg;
    return s;
}

nefty_status cuda_fail(nefty_handle* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, NEFTY_ECUDA, m);
}

#define NEFTY_CUDA(h, expr)                                       \
    do {                                                          \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Where an array lives, seen from device `dev`: host memory (staged by the
// call), memory the kernels on `dev` may read in place (device memory of
// `dev`, or managed memory), or device memory of another GPU, which the
// kernels on `dev` must never dereference.
enum PtrKind { kPtrHost, kPtrDevice, kPtrOtherDevice };
PtrKind ptr_kind(const void* p, int dev) {
    if (!p) return kPtrHost;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return kPtrHost;
    }
    if (at.type == cudaMemoryTypeManaged) return kPtrDevice;
    if (at.type == cudaMemoryTypeDevice) return at.device == dev ? kPtrDevice : kPtrOtherDevice;
    return kPtrHost;
}

// Effective problem with defaults filled in.
struct Prob {
    int nx, ny, nz, nt, bc, obs_face, prec, max_iter, ckpt_every, extrap, jacobi_k, residual;
    double dx, dy, dz, dt, robin_h, rtol, loss_scale;
    unsigned N, S;
};

nefty_status check_problem(const nefty_problem* p, Prob* out, std::string* why) {
    if (!p) { *why = "problem is NULL"; return NEFTY_EINVAL; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { *why = "nx, ny, nz must be >= 1"; return NEFTY_EINVAL; }
    const double cells = (double)p->nx * p->ny * p->nz;
    if (cells >= 2147483647.0) { *why = "nx*ny*nz must be < 2^31"; return NEFTY_EINVAL; }
    if (p->nt < 1) { *why = "nt must be >= 1"; return NEFTY_EINVAL; }
    if (!(p->dx > 0) || !(p->dy > 0) || !(p->dz > 0) || !std::isfinite(p->dx) ||
        !std::isfinite(p->dy) || !std::isfinite(p->dz)) {
        *why = "dx, dy, dz must be positive and finite";
        return NEFTY_EINVAL;
    }
    if (!(p->dt > 0) || !std::isfinite(p->dt)) { *why = "dt must be positive and finite"; return NEFTY_EINVAL; }
    if (p->bc != NEFTY_BC_NEUMANN && p->bc != NEFTY_BC_PERIODIC_XY) { *why = "unknown bc"; return NEFTY_EINVAL; }
    if (!(p->robin_h >= 0) || !std::isfinite(p->robin_h)) { *why = "robin_h must be >= 0"; return NEFTY_EINVAL; }
    if (p->obs_face != 0 && p->obs_face != 1) { *why = "obs_face must be 0 or 1"; return NEFTY_EINVAL; }
    if (p->prec != NEFTY_FP32 && p->prec != NEFTY_FP64) { *why = "unknown precision"; return NEFTY_EINVAL; }
    if (p->rtol < 0 || !std::isfinite(p->rtol)) { *why = "rtol must be >= 0"; return NEFTY_EINVAL; }
    if (p->max_iter < 0) { *why = "max_iter must be >= 0"; return NEFTY_EINVAL; }
    if (p->ckpt_every < 0) { *why = "ckpt_every must be >= 0"; return NEFTY_EINVAL; }
    if (p->loss_scale < 0 || !std::isfinite(p->loss_scale)) { *why = "loss_scale must be >= 0"; return NEFTY_EINVAL; }
    if (p->extrap < -1 || p->extrap > tiled::kRing) { *why = "extrap must be -1, 0, 1, 2, 3 or 4"; return NEFTY_EINVAL; }
    if (p->jacobi_k < 0 || p->jacobi_k > 100000) { *why = "jacobi_k must be in [0, 100000]"; return NEFTY_EINVAL; }
    if (p->residual < -1 || p->residual > 1) { *why = "residual must be -1, 0 or 1"; return NEFTY_EINVAL; }
    if (out) {
        out->nx = p->nx; out->ny = p->ny; out->nz = p->nz; out->nt = p->nt; out->bc = p->bc;
        out->obs_face = p->obs_face; out->prec = p->prec;
        out->max_iter = p->max_iter > 0 ? p->max_iter : kDefaultMaxIter;
        out->ckpt_every = p->ckpt_every;
        // increments the start extrapolates from: 0 .. kRing
        out->extrap = p->extrap == 0 ? kDefaultExtrap : (p->extrap < 0 ? 0 : p->extrap);
        // the paper's fixed Jacobi sweeps start from T^n (mu^(n+1)) exactly
        out->jacobi_k = p->jacobi_k;
        if (out->jacobi_k > 0) out->extrap = 0;
        out->residual = p->residual < 0 ? -1 : 1;
        out->dx = p->dx; out->dy = p->dy; out->dz = p->dz; out->dt = p->dt; out->robin_h = p->robin_h;
        out->rtol = p->rtol > 0 ? p->rtol : (p->prec == NEFTY_FP32 ? kDefaultRtolFp32 : kDefaultRtolFp64);
        out->loss_scale = p->loss_scale > 0 ? p->loss_scale : 1.0 / ((double)p->nt * p->nx * p->ny);
        out->S = (unsigned)p->nx * (unsigned)p->ny;
        out->N = out->S * (unsigned)p->nz;
    }
    return NEFTY_OK;
}

// Bump allocator over the handle's device workspace.  A first pass with
// base == nullptr only measures.
struct Arena {
    char* base = nullptr;
    size_t off = 0;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

void drop_keep(nefty_handle* h) {
    if (h->keep) cudaFree(h->keep);
    h->keep = nullptr;
    h->keep_bytes = 0;
    h->keep_valid = false;
}

nefty_status ensure_workspace(nefty_handle* h, size_t bytes) {
    // the kept field activations give way to a workspace that needs their room
    if (h->keep && bytes > h->ws_bytes && bytes + h->keep_bytes > h->budget) drop_keep(h);
    if (bytes > h->budget) {
        char buf[160];
        snprintf(buf, sizeof buf, "workspace of %zu bytes exceeds the memory budget of %llu bytes", bytes,
                 (unsigned long long)h->budget);
        return fail(h, NEFTY_ENOMEM, buf);
    }
    if (bytes <= h->ws_bytes) return NEFTY_OK;
    if (h->ws) {
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        char buf[160];
        snprintf(buf, sizeof buf, "cudaMalloc of %zu workspace bytes failed (%s)", bytes, cudaGetErrorName(e));
        return fail(h, NEFTY_ENOMEM, buf);
    }
    h->ws_bytes = bytes;
    return NEFTY_OK;
}

// Input arrays: used in place when on the device, staged into the workspace
// when on the host.
struct Input {
    const void* user = nullptr;
    size_t bytes = 0;
    bool stage = false;
    bool foreign = false;   // device memory of another GPU: rejected by the call
    void* dev = nullptr;
    void plan(const void* p, size_t b, int device) {
        user = p;
        bytes = b;
        const PtrKind k = ptr_kind(p, device);
        stage = p && k == kPtrHost;
        foreign = p && k == kPtrOtherDevice;
    }
    void place(Arena& a) {
        if (!user) { dev = nullptr; return; }
        if (stage) dev = a.take(bytes);
        else { a.take(0); dev = const_cast<void*>(user); }
    }
};

// Output arrays: written in place when on the device, staged and copied back
// when on the host.
struct Output {
    void* user = nullptr;
    size_t bytes = 0;
    bool stage = false;
    bool foreign = false;   // device memory of another GPU: rejected by the call
    void* dev = nullptr;
    void plan(void* p, size_t b, int device) {
        user = p;
        bytes = b;
        const PtrKind k = ptr_kind(p, device);
        stage = p && k == kPtrHost;
        foreign = p && k == kPtrOtherDevice;
    }
    void place(Arena& a) {
        if (!user) { dev = nullptr; return; }
        if (stage) dev = a.take(bytes);
        else { a.take(0); dev = user; }
    }
};

// EINVAL when any planned array is device memory of a GPU other than the
// handle's: the kernels would dereference it without peer access.
template <class... A>
nefty_status reject_foreign(nefty_handle* h, const A&... arrays) {
    const bool any = (false || ... || arrays.foreign);
    if (any) return fail(h, NEFTY_EINVAL, "an array is device memory of another GPU than the handle's");
    return NEFTY_OK;
}

int grid_for(nefty_handle* h, int prec, unsigned N) {
    if (h->grid_max[prec] == 0) h->grid_max[prec] = solver_grid_blocks(h->device, prec);
    const int gmax = std::max(1, h->grid_max[prec] / h->grid_share);
    // about four cells per thread; small grids use few CTAs so that the grid
    // barriers of the CG loop stay cheap.
    long want = ((long)N + (long)kThreads * 4 - 1) / ((long)kThreads * 4);
    if (want < 1) want = 1;
    return (int)std::min<long>(want, gmax);
}

// Whether the tiled kernels stage this problem through TMA (16-byte row
// pitch; zero-flux or periodic lateral walls); the encoder may still refuse
// (see prepare_tma).
bool tma_grid(const Prob& P) { return P.nx % 4 == 0; }

int grid_for_tiled(nefty_handle* h, const Prob& P) {
    if (h->grid_tiled == 0) h->grid_tiled = tiled_grid_blocks(h->device);
    // batched sweeps all run on the batcher's grid
    if (h->batch && tma_grid(P) && P.jacobi_k == 0) return batcher_grid(h->batch);
    const int gmax = std::max(1, h->grid_tiled / h->grid_share);
    const long tiles = (long)((P.nx + tiled::TX - 1) / tiled::TX) * ((P.ny + tiled::TY - 1) / tiled::TY);
    const long units = tiles * P.nz;
    // at least two planes per CTA, so small grids keep their barriers cheap
    long want = std::max(1L, units / 2);
    return (int)std::min<long>(std::min<long>(want, gmax), tiled::kMaxGrid);
}

template <typename Real>
OperatorView<Real> make_view(const Prob& P, Real* coef) {
    OperatorView<Real> v;
    v.nx = P.nx; v.ny = P.ny; v.nz = P.nz;
    v.px = P.bc == NEFTY_BC_PERIODIC_XY && P.nx > 1;
    v.py = P.bc == NEFTY_BC_PERIODIC_XY && P.ny > 1;
    v.N = P.N; v.S = P.S;
    v.cx = coef;
    v.cy = coef + P.N;
    v.cz = coef + 2 * (size_t)P.N;
    v.d = coef + 3 * (size_t)P.N;
    v.dinv = coef + 4 * (size_t)P.N;
    v.robin = (Real)(P.dt * P.robin_h / P.dz);
    return v;
}

// Shared state of one forward / adjoint call.
template <typename Real>
struct Call {
    nefty_handle* h;
    Prob P;
    cudaStream_t s;
    int G;
    // workspace regions
    Real* coef = nullptr;
    Real *r = nullptr, *p = nullptr, *q = nullptr;
    DevCtl* ctl = nullptr;
    double* partials = nullptr;
    double* loss_partials = nullptr;
    int* iters = nullptr;        // [3][nt]: forward, recompute, adjoint
    double* resid = nullptr;     // [3][nt]
    Real** tables = nullptr;
    Input alpha, T0, qf, qfull, obs;
    // CUDA events around every solver launch (kind 0 forward, 1 recompute, 2 adjoint)
    bool timing = false;
    struct Timed { cudaEvent_t a, b; int kind; };
    std::vector<Timed> timed;
    int launches = 0;

    ~Call() {
        for (auto& t : timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    }

    static constexpr bool kTiled = std::is_same<Real, float>::value;
    // every state slot of the call (slots of SB bytes) in one slab, so that a
    // single tensor map reaches all of them
    Real* slab = nullptr;
    unsigned slab_halves = 0;   // blocks of N values in the slab
    Real* carve_slab(Arena& a, size_t slots, size_t slot_bytes) {
        slab = (Real*)a.take(slots * slot_bytes);
        slab_halves = (unsigned)(slots * (slot_bytes / sizeof(Real)) / P.N);
        return slab;
    }
    tiled::Vecs tv{};
    tiled::TmaMaps host_maps{};        // descriptors of the TMA-staged passes (when use_tma)
    float* ring_f = nullptr;           // increment rings of the forward and adjoint sweeps ([kRing][N] each)
    float* ring_a = nullptr;
    float* ystart = nullptr;           // the next solve's start (a slot of the state slab)
    float* diag_buf = nullptr;
    int* cflag = nullptr;
    // The TMA-staged PCG carries the residual of each solve into the next
    // (cg_tiled.cu); checkpoints then keep it beside the increments.
    bool carries() const { return kTiled && tma_grid(P) && P.jacobi_k == 0 && P.residual >= 0; }

    void place_common(Arena& a, size_t ntables) {
        const size_t N = P.N;
        coef = (Real*)a.take(5 * N * sizeof(Real));
        if (kTiled) {
            // u, ws, ss of one ping-pong set and p, delta are contiguous (one copy each)
            for (int i = 0; i < 2; ++i) {
                tv.u[i] = (float*)a.take(3 * N * sizeof(float));
                tv.ws[i] = tv.u[i] + N;
                tv.ss[i] = tv.u[i] + 2 * N;
            }
            tv.p = (float*)a.take(2 * N * sizeof(float));
            tv.delta = tv.p + N;
            ring_f = (float*)a.take(tiled::kRing * N * sizeof(float));
            ring_a = (float*)a.take(tiled::kRing * N * sizeof(float));
            // the carried residual of the forward and adjoint sweeps, and the
            // diagonal of A (used by the TMA-staged PCG only: diag stays null
            // otherwise, which the kernels read as "not carried")
            tv.sig[0] = (float*)a.take(3 * N * sizeof(float));
            tv.sig[1] = tv.sig[0] + N;
            diag_buf = tv.sig[0] + 2 * N;
        } else {
            r = (Real*)a.take(N * sizeof(Real));
            p = (Real*)a.take(N * sizeof(Real));
            q = (Real*)a.take(N * sizeof(Real));
        }
        ctl = (DevCtl*)a.take(sizeof(DevCtl));
        partials = (double*)a.take(2 * kMaxRed * (size_t)G * sizeof(double));
        loss_partials = (double*)a.take((size_t)G * sizeof(double));
        iters = (int*)a.take(3 * (size_t)P.nt * sizeof(int));
        cflag = (int*)a.take(2 * ((size_t)P.nt + 1) * sizeof(int));   // forward, adjoint (FwdTiled::cflag)
        resid = (double*)a.take(3 * (size_t)P.nt * sizeof(double));
        tables = (Real**)a.take(ntables * sizeof(Real*));
        alpha.place(a); T0.place(a); qf.place(a); qfull.place(a); obs.place(a);
    }

    nefty_status upload_inputs() {
        for (Input* in : {&alpha, &T0, &qf, &qfull, &obs})
            if (in->user && in->stage)
                NEFTY_CUDA(h, cudaMemcpyAsync(in->dev, in->user, in->bytes, cudaMemcpyHostToDevice, s));
        NEFTY_CUDA(h, cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
        if (h->fault_missing || h->fault_wait_ns) {   // test hook: see nefty_debug_barrier_fault
            DevCtl init{};
            init.missing = h->fault_missing;
            init.wait_ns = h->fault_wait_ns;
            NEFTY_CUDA(h, cudaMemcpyAsync(ctl, &init, sizeof init, cudaMemcpyHostToDevice, s));
            NEFTY_CUDA(h, cudaStreamSynchronize(s));   // init lives on this stack frame
        }
        if (kTiled) {   // no increment history yet
            NEFTY_CUDA(h, cudaMemsetAsync(ring_f, 0, tiled::kRing * (size_t)P.N * sizeof(float), s));
            NEFTY_CUDA(h, cudaMemsetAsync(ring_a, 0, tiled::kRing * (size_t)P.N * sizeof(float), s));
        }
        return NEFTY_OK;
    }

    // TMA-staged passes serve grids with a 16-byte row pitch (either wall
    // setting); other grids take the plain-load pass.
    bool use_tma = false;
    nefty_status prepare_tma() {
        if constexpr (kTiled) {
            if (!tma_grid(P)) return NEFTY_OK;
            tiled::Geo g{};
            g.nx = P.nx; g.ny = P.ny; g.nz = P.nz; g.S = P.S;
            if (!tiled_encode_maps(&host_maps, g, tv, (const float*)alpha.dev, (const float*)slab, slab_halves))
                return NEFTY_OK;
            use_tma = true;
            if (carries()) tv.diag = diag_buf;
        }
        return NEFTY_OK;
    }

    // Face values of A(alpha); rejects alpha <= 0 or non-finite.
    nefty_status coefficients() {
        Real* c = coef;
        NEFTY_CUDA(h, launch_coefficients<Real>((const Real*)alpha.dev, P.nx, P.ny, P.nz, P.bc, P.dx,
                                                P.dy, P.dz, P.dt, P.robin_h, c, c + P.N, c + 2 * (size_t)P.N,
                                                c + 3 * (size_t)P.N, c + 4 * (size_t)P.N, ctl, s));
        ++launches;
        DevCtl hc;
        NEFTY_CUDA(h, cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, s));
        NEFTY_CUDA(h, cudaStreamSynchronize(s));
        if (hc.err == kDevBadAlpha) return fail(h, NEFTY_EINVAL, "alpha must be > 0 and finite in every cell");
        return NEFTY_OK;
    }

    FwdArgs<Real> fwd_args(int n0, int n1, Real* const* src, Real* const* dst, int* it, double* rs) {
        FwdArgs<Real> a{};
        a.op = make_view<Real>(P, coef);
        a.r = r; a.p = p; a.q = q;
        a.n0 = n0; a.n1 = n1;
        a.src = src; a.dst = dst;
        a.q_face = (const Real*)qf.dev;
        a.q_steps = qf.dev ? q_steps : 0;
        a.q_full = (const Real*)qfull.dev;
        a.src_scale = P.dt / P.dz;
        a.obs_off = P.obs_face ? (unsigned)(P.nz - 1) * P.S : 0u;
        a.obs = nullptr;
        a.frames = nullptr;
        a.tol2 = P.rtol * P.rtol;
        a.max_iter = P.max_iter;
        a.ctl = ctl;
        a.partials = partials;
        a.iters = it;
        a.resid = rs;
        a.loss_partials = nullptr;
        a.jacobi_k = P.jacobi_k;
        return a;
    }
    int q_steps = 0;

    nefty_status begin_timed(int kind, Timed* t) {
        t->kind = kind;
        t->a = t->b = nullptr;
        if (!timing) return NEFTY_OK;
        NEFTY_CUDA(h, cudaEventCreate(&t->a));
        NEFTY_CUDA(h, cudaEventCreate(&t->b));
        NEFTY_CUDA(h, cudaEventRecord(t->a, s));
        return NEFTY_OK;
    }
    nefty_status end_timed(Timed& t) {
        ++launches;
        if (!timing) return NEFTY_OK;
        NEFTY_CUDA(h, cudaEventRecord(t.b, s));
        timed.push_back(t);
        return NEFTY_OK;
    }
    nefty_status launch_fwd(const FwdArgs<Real>& a, int kind = 0) {
        NEFTY_CUDA(h, cudaMemsetAsync(&ctl->bar, 0, 2 * sizeof(unsigned), s));
        Timed t;
        if (nefty_status e = begin_timed(kind, &t)) return e;
        NEFTY_CUDA(h, launch_forward<Real>(a, G, s));
        return end_timed(t);
    }
    tiled::Common tiled_common(int* it, double* rs) {
        tiled::Common c{};
        c.g.nx = P.nx; c.g.ny = P.ny; c.g.nz = P.nz;
        c.g.px = P.bc == NEFTY_BC_PERIODIC_XY && P.nx > 1;
        c.g.py = P.bc == NEFTY_BC_PERIODIC_XY && P.ny > 1;
        c.g.S = P.S;
        c.g.tiles_x = (P.nx + tiled::TX - 1) / tiled::TX;
        c.g.units = (unsigned)(c.g.tiles_x * ((P.ny + tiled::TY - 1) / tiled::TY)) * (unsigned)P.nz;
        c.maps = host_maps;
        c.tma = use_tma ? 1 : 0;
        c.slab = (const float*)slab;
        c.slab_halves = slab_halves;
        c.alpha = (const float*)alpha.dev;
        c.kx = (float)(P.dt / (P.dx * P.dx));
        c.ky = (float)(P.dt / (P.dy * P.dy));
        c.kz = (float)(P.dt / (P.dz * P.dz));
        c.robin = (float)(P.dt * P.robin_h / P.dz);
        c.v = tv;
        c.ctl = ctl;
        c.partials = partials;
        const double tol2 = P.rtol * P.rtol;
        c.tol2_hi = (float)tol2;
        c.tol2_lo = (float)(tol2 - (double)c.tol2_hi);
        c.max_iter = P.max_iter;
        c.jacobi_k = P.jacobi_k;
        c.iters = it;
        c.resid = rs;
        return c;
    }
    // Batched sweeps (serving): the whole sweep goes to the batcher, whose
    // launches each run a part of it (until their device-time budget is
    // spent) beside the other running jobs' sweeps; the call's stream
    // continues after the launch that ran its last step.
    nefty_status run_batched(const tiled::BatchSweep& whole) {
        int launched = 0, shared = 0;
        std::string why;
        const nefty_status e = batcher_run(h->batch, whole, G, s, &launched, &shared, &why);
        h->batch_launches += launched;
        h->batch_shared += shared;
        launches += std::max(0, launched - 1);
        if (e != NEFTY_OK) return fail(h, e, why);
        return NEFTY_OK;
    }
    nefty_status batched_fwd(const tiled::FwdTiled& a) {
        // the parts add their frame losses into loss_partials
        if (a.loss_partials) NEFTY_CUDA(h, cudaMemsetAsync(a.loss_partials, 0, (size_t)G * sizeof(double), s));
        tiled::BatchSweep w{};
        w.adjoint = 0;
        w.f = a;
        w.f.loss_add = 1;
        return run_batched(w);
    }
    nefty_status batched_adj(const tiled::AdjTiled& a) {
        tiled::BatchSweep w{};
        w.adjoint = 1;
        w.a = a;
        return run_batched(w);
    }
    nefty_status launch_fwd_tiled(const tiled::FwdTiled& a, int kind) {
        NEFTY_CUDA(h, cudaMemsetAsync(&ctl->bar, 0, 2 * sizeof(unsigned), s));
        Timed t;
        if (nefty_status e = begin_timed(kind, &t)) return e;
        if (h->batch && use_tma && P.jacobi_k == 0) {
            if (nefty_status e = batched_fwd(a)) return e;
        } else {
            NEFTY_CUDA(h, launch_forward_tiled(a, G, s));
        }
        return end_timed(t);
    }
    nefty_status launch_adj_tiled(const tiled::AdjTiled& a) {
        NEFTY_CUDA(h, cudaMemsetAsync(&ctl->bar, 0, 2 * sizeof(unsigned), s));
        Timed t;
        if (nefty_status e = begin_timed(2, &t)) return e;
        if (h->batch && use_tma && P.jacobi_k == 0) {
            if (nefty_status e = batched_adj(a)) return e;
        } else {
            NEFTY_CUDA(h, launch_adjoint_tiled(a, G, s));
        }
        return end_timed(t);
    }
    // forward launch over steps [n0, n1) with either kernel family
    // ring_load / ring_save / hist0 / carry: the increment history and the
    // carried residual (FP32 path, see FwdTiled)
    nefty_status forward_steps(int n0, int n1, Real* const* src, Real* const* dst, int* it, double* rs,
                               Real* frames, const Real* obsp, double* lossp, int kind,
                               const Real* ring_load = nullptr, Real* const* ring_save = nullptr, int hist0 = 0,
                               int carry = 0) {
        if constexpr (kTiled) {
            tiled::FwdTiled a{};
            a.c = tiled_common(it, rs);
            a.n0 = n0; a.n1 = n1;
            a.ring = ring_f;
            a.ystart = ystart;
            a.extrap = P.extrap;
            a.hist0 = hist0;
            a.ring_load = ring_load;
            a.ring_save = ring_save;
            a.carry = carry;
            a.cflag = cflag;
            a.n_end = P.nt;
            a.src = src; a.dst = dst;
            a.q_face = (const float*)qf.dev;
            a.q_steps = qf.dev ? q_steps : 0;
            a.q_full = (const float*)qfull.dev;
            a.src_scale = (float)(P.dt / P.dz);
            a.obs_off = P.obs_face ? (unsigned)(P.nz - 1) * P.S : 0u;
            a.obs = obsp;
            a.frames = frames;
            a.loss_partials = lossp;
            return launch_fwd_tiled(a, kind);
        } else {
            FwdArgs<Real> a = fwd_args(n0, n1, src, dst, it, rs);
            a.frames = frames;
            a.obs = obsp;
            a.loss_partials = lossp;
            return launch_fwd(a, kind);
        }
    }
    nefty_status launch_adj(const AdjArgs<Real>& a) {
        NEFTY_CUDA(h, cudaMemsetAsync(&ctl->bar, 0, 2 * sizeof(unsigned), s));
        Timed t;
        if (nefty_status e = begin_timed(2, &t)) return e;
        NEFTY_CUDA(h, launch_adjoint<Real>(a, G, s));
        return end_timed(t);
    }

    // Wait for the stream, then turn the device control word into a status.
    nefty_status finish(double* loss_out, bool want_loss, nefty_stats* st, int fwd_steps,
                        int rec_steps, int adj_steps, int K, int nck) {
        NEFTY_CUDA(h, cudaStreamSynchronize(s));
        DevCtl hc;
        NEFTY_CUDA(h, cudaMemcpy(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost));
        if (hc.err == kDevTimeout)
            return fail(h, NEFTY_ETIMEOUT, "a grid barrier of the persistent solver timed out");
        if (hc.err == kDevBadState)
            return fail(h, NEFTY_ECUDA, "internal error: a solver state lies outside the state slab");
        if (want_loss && loss_out) {
            std::vector<double> lp(G);
            NEFTY_CUDA(h, cudaMemcpy(lp.data(), loss_partials, G * sizeof(double), cudaMemcpyDeviceToHost));
            double t = 0.0;
            for (int b = 0; b < G; ++b) t += lp[b];
            *loss_out = P.loss_scale * t;
        }
        if (st) {
            std::memset(st, 0, sizeof *st);
            const size_t nt = (size_t)P.nt;
            std::vector<int> it(3 * nt);
            std::vector<double> rs(3 * nt);
            NEFTY_CUDA(h, cudaMemcpy(it.data(), iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost));
            NEFTY_CUDA(h, cudaMemcpy(rs.data(), resid, rs.size() * sizeof(double), cudaMemcpyDeviceToHost));
            const int counts[3] = {fwd_steps, rec_steps, adj_steps};
            int64_t tot[3] = {0, 0, 0};
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < counts[k]; ++i) {
                    tot[k] += it[k * nt + i];
                    st->max_step_iters = std::max(st->max_step_iters, it[k * nt + i]);
                    st->max_rel_residual = std::max(st->max_rel_residual, rs[k * nt + i]);
                }
            st->fwd_iters = tot[0]; st->recompute_iters = tot[1]; st->adj_iters = tot[2];
            st->fwd_steps = fwd_steps; st->recompute_steps = rec_steps; st->adj_steps = adj_steps;
            st->not_converged = hc.notconv;
            st->ckpt_every = K;
            st->n_checkpoints = nck;
            st->workspace_bytes = h->ws_bytes;
            st->grid_blocks = G;
            st->kernel_launches = launches;
            st->tma_staged = use_tma ? 1 : 0;
            st->folded_last_iters = hc.folded;
            st->carried_solves = hc.carried;
            double ms[3] = {0.0, 0.0, 0.0};
            for (auto& t : timed) {
                float v = 0.f;
                NEFTY_CUDA(h, cudaEventElapsedTime(&v, t.a, t.b));
                ms[t.kind] += v;
            }
            st->fwd_ms = ms[0];
            st->recompute_ms = ms[1];
            st->adj_ms = ms[2];
        }
        if (hc.notconv > 0) {
            char buf[128];
            snprintf(buf, sizeof buf, "%d CG solve(s) reached max_iter = %d", hc.notconv, P.max_iter);
            return fail(h, NEFTY_ENOTCONV, buf);
        }
        return NEFTY_OK;
    }
};

// dry != NULL: only size the workspace of the call into *dry.
template <typename Real>
nefty_status run_forward(nefty_handle* h, const Prob& P, const void* alpha, const void* T0,
                         const void* q_face, int q_steps, const void* q_full, void* frames_out,
                         void* T_final, const void* obs, double* loss_out, nefty_stats* st,
                         cudaStream_t s, size_t* dry = nullptr) {
    const size_t N = P.N, S = P.S, nt = (size_t)P.nt, R = sizeof(Real);
    Call<Real> C;
    C.h = h; C.P = P; C.s = s; C.q_steps = q_steps;
    C.timing = st != nullptr;
    C.G = Call<Real>::kTiled ? grid_for_tiled(h, P) : grid_for(h, P.prec, P.N);
    if (C.G <= 0) return fail(h, NEFTY_ECUDA, "cannot size the persistent solver grid on this device");
    C.alpha.plan(alpha, N * R, h->device);
    C.T0.plan(T0, N * R, h->device);
    C.qf.plan(q_face, S * R, h->device);
    C.qfull.plan(q_full, nt * S * R, h->device);
    C.obs.plan(loss_out ? obs : nullptr, nt * S * R, h->device);
    Output fr, tf;
    fr.plan(frames_out, nt * S * R, h->device);
    tf.plan(T_final, N * R, h->device);
    if (nefty_status e = reject_foreign(h, C.alpha, C.T0, C.qf, C.qfull, C.obs, fr, tf)) return e;
    Real *work[2], *t0buf = nullptr;
    // one state = N values; the FP32 path keeps it as a compensated (hi, lo)
    // pair, so its state slots hold 2N floats
    const size_t SB = (Call<Real>::kTiled ? 2 : 1) * N * R;
    const bool own_t0 = Call<Real>::kTiled || !C.T0.user;
    auto layout = [&](Arena& a) {
        C.place_common(a, 2 * nt);
        // slots: the work pair, the start of the next solve, T^0 (when copied in)
        Real* blk = C.carve_slab(a, own_t0 ? 4 : 3, SB);
        work[0] = blk;
        work[1] = blk + SB / R;
        if (Call<Real>::kTiled) C.ystart = (float*)(blk + 2 * (SB / R));
        t0buf = own_t0 ? blk + 3 * (SB / R) : nullptr;
        fr.place(a);
        tf.place(a);
    };
    Arena probe;
    layout(probe);
    if (dry) { *dry = probe.off; return NEFTY_OK; }
    if (nefty_status e = ensure_workspace(h, probe.off)) return e;
    Arena arena;
    arena.base = (char*)h->ws;
    layout(arena);
    if (nefty_status e = C.upload_inputs()) return e;
    if (nefty_status e = C.coefficients()) return e;
    if (nefty_status e = C.prepare_tma()) return e;
    const Real* T0dev = own_t0 ? t0buf : (const Real*)C.T0.dev;
    if (own_t0) {
        NEFTY_CUDA(h, cudaMemsetAsync(t0buf, 0, SB, s));
        if (C.T0.user) NEFTY_CUDA(h, cudaMemcpyAsync(t0buf, C.T0.dev, N * R, cudaMemcpyDeviceToDevice, s));
    }
    // step n reads src[n], writes dst[n]; states alternate between two buffers
    std::vector<Real*> tab(2 * nt);
    for (size_t n = 0; n < nt; ++n) {
        tab[n] = n == 0 ? const_cast<Real*>(T0dev) : work[(n - 1) & 1];
        tab[nt + n] = work[n & 1];
    }
    NEFTY_CUDA(h, cudaMemcpyAsync(C.tables, tab.data(), tab.size() * sizeof(Real*), cudaMemcpyHostToDevice, s));
    if (nefty_status e = C.forward_steps(0, P.nt, C.tables, C.tables + nt, C.iters, C.resid, (Real*)fr.dev,
                                         (const Real*)C.obs.dev, C.loss_partials, 0))
        return e;
    if (tf.user) NEFTY_CUDA(h, cudaMemcpyAsync(tf.dev, work[(nt - 1) & 1], N * R, cudaMemcpyDeviceToDevice, s));
    for (Output* o : {&fr, &tf})
        if (o->user && o->stage)
            NEFTY_CUDA(h, cudaMemcpyAsync(o->user, o->dev, o->bytes, cudaMemcpyDeviceToHost, s));
    return C.finish(loss_out, true, st, P.nt, 0, 0, 1, 2);
}

// Storage plan of the reverse sweep.  The first gB segments of K steps,
// [0, B) with B = min(gB K, nt), keep only their first state (a checkpoint)
// in the forward sweep and are recomputed from it segment by segment; every
// state of the tail [B, nt] is kept and needs no recompute.  gB = 0 keeps
// every state.  States are counted in slots of one state each (SB bytes),
// with c extra slots per checkpoint for its increment history.
struct CkPlan {
    int K;    // segment length (1 when gB == 0)
    int gB;   // recomputed segments
};
long long plan_slots(int nt, int K, int gB, int c) {
    const long long B = std::min((long long)gB * K, (long long)nt);
    return 3 + (long long)gB * (1 + c) + (gB > 0 ? K + 2 : 0) + (B < nt ? nt - B + 1 : 0);
}
// ckpt_every = 1: every state; >= 2: every segment of that length recomputed;
// 0: every state when it fits the budget, else the (K, gB) that fits and
// recomputes the fewest steps (the tail takes whatever memory is left, so with
// plenty of memory far less than one extra forward sweep is recomputed).
CkPlan plan_checkpoints(const Prob& P, size_t fixed_bytes, uint64_t budget, size_t slot_bytes, int c) {
    const int nt = P.nt;
    if (P.ckpt_every == 1) return CkPlan{1, 0};
    if (P.ckpt_every >= 2) {
        const int K = std::min(P.ckpt_every, nt);
        return CkPlan{K, (nt + K - 1) / K};
    }
    // state slots that fit (the slab's own alignment padding is under 256 B)
    const uint64_t avail = budget > fixed_bytes + 256 ? budget - fixed_bytes - 256 : 0;
    const long long M = (long long)(avail / slot_bytes);
    if (plan_slots(nt, 1, 0, c) <= M) return CkPlan{1, 0};
    const int Ks = std::max(2, (int)std::ceil(std::sqrt((double)nt)));
    CkPlan best{Ks, (nt + Ks - 1) / Ks};   // when nothing fits: about sqrt(nt) checkpoints
    long long best_cost = -1, best_slots = 0;
    for (int K = 2; K <= nt; ++K) {
        const int gmax = (nt + K - 1) / K;
        // with a tail, slots fall by K - 1 - c per extra segment
        int g = gmax;
        if (K > 1 + c) {
            const long long need = (long long)nt + K + 6 - M;
            g = need <= 0 ? 1 : (int)std::min<long long>(gmax, (need + (K - 1 - c) - 1) / (K - 1 - c));
            g = std::max(g, 1);
        }
        while (g < gmax && plan_slots(nt, K, g, c) > M) ++g;
        const long long sl = plan_slots(nt, K, g, c);
        if (sl > M) continue;
        const long long cost = std::min((long long)g * K, (long long)nt);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && sl < best_slots)) {
            best = CkPlan{K, g};
            best_cost = cost;
            best_slots = sl;
        }
    }
    return best;
}

template <typename Real>
nefty_status run_adjoint(nefty_handle* h, const Prob& P, const void* alpha, const void* T0,
                         const void* q_face, int q_steps, const void* q_full, const void* obs,
                         double* loss_out, void* grad_alpha, void* grad_T0, nefty_stats* st,
                         cudaStream_t s, size_t* dry = nullptr) {
    const size_t N = P.N, S = P.S, nt = (size_t)P.nt, R = sizeof(Real);
    Call<Real> C;
    C.h = h; C.P = P; C.s = s; C.q_steps = q_steps;
    C.timing = st != nullptr;
    C.G = Call<Real>::kTiled ? grid_for_tiled(h, P) : grid_for(h, P.prec, P.N);
    if (C.G <= 0) return fail(h, NEFTY_ECUDA, "cannot size the persistent solver grid on this device");
    C.alpha.plan(alpha, N * R, h->device);
    C.T0.plan(T0, N * R, h->device);
    C.qf.plan(q_face, S * R, h->device);
    C.qfull.plan(q_full, nt * S * R, h->device);
    C.obs.plan(obs, nt * S * R, h->device);
    Output ga, gt;
    ga.plan(grad_alpha, N * R, h->device);
    gt.plan(grad_T0, N * R, h->device);
    if (nefty_status e = reject_foreign(h, C.alpha, C.T0, C.qf, C.qfull, C.obs, ga, gt)) return e;

    // Fixed part of the workspace (everything except stored states).
    size_t fixed = 0;
    {
        Arena a;
        C.place_common(a, 7 * nt + 4);
        a.take(N * sizeof(double));
        ga.place(a);
        gt.place(a);
        fixed = a.off;
    }
    const size_t SB = (Call<Real>::kTiled ? 2 : 1) * N * R;   // one state slot (see run_forward)
    // FP32 checkpoints also keep the increments before them (as many as the
    // start extrapolates from) and, on the TMA-staged path, the carried
    // residual, so a recomputed segment starts from the same bits as the
    // first sweep
    const int ck_hist_if = Call<Real>::kTiled ? P.extrap + (C.carries() ? 1 : 0) : 0;
    const CkPlan plan = plan_checkpoints(P, fixed, h->budget, SB, (ck_hist_if + 1) / 2);
    const int K = plan.K, gB = plan.gB;
    const int B = (int)std::min((long long)gB * K, (long long)P.nt);   // recomputed steps [0, B)
    const int ntail = B < P.nt ? P.nt - B + 1 : 0;                     // kept states T^B .. T^nt
    const int ck_hist = gB > 0 ? ck_hist_if : 0;
    const bool ck_ring = ck_hist > 0;
    const int ck_slots = (ck_hist + 1) / 2;   // state slots (2N floats) holding them
    Real* mu[2];
    double* grad = nullptr;
    std::vector<Real*> ck(gB), segbuf(gB > 0 ? K : 0), tail(ntail);
    Real* work[2] = {nullptr, nullptr};
    auto layout = [&](Arena& a) {
        C.place_common(a, 7 * nt + 4);
        grad = (double*)a.take(N * sizeof(double));
        ga.place(a);
        gt.place(a);
        // state slots: mu[2], the next start, checkpoints, recompute buffer,
        // forward work pair, kept tail
        const size_t slots = (size_t)plan_slots(P.nt, K, gB, ck_slots);
        Real* next = C.carve_slab(a, slots, SB);
        auto slot = [&]() { Real* p = next; next += SB / R; return p; };
        mu[0] = slot();
        mu[1] = slot();
        Real* ys = slot();   // the next solve's start
        if (Call<Real>::kTiled) C.ystart = (float*)ys;
        for (int i = 0; i < gB; ++i) {
            ck[i] = slot();
            for (int k = 0; k < ck_slots; ++k) slot();   // [delta^{gK-1}; delta^{gK-2}; ...] after the state
        }
        for (auto& p : segbuf) p = slot();
        if (gB > 0) {
            work[0] = slot();
            work[1] = slot();
        }
        for (auto& p : tail) p = slot();
    };
    Arena probe;
    layout(probe);
    if (dry) { *dry = probe.off; return NEFTY_OK; }
    if (nefty_status e = ensure_workspace(h, probe.off)) return e;
    Arena arena;
    arena.base = (char*)h->ws;
    layout(arena);
    if (nefty_status e = C.upload_inputs()) return e;
    if (nefty_status e = C.coefficients()) return e;
    if (nefty_status e = C.prepare_tma()) return e;
    // where the first sweep keeps T^n
    auto state_fwd = [&](int n) -> Real* {
        if (ntail > 0 && n >= B) return tail[n - B];
        if (n % K == 0 && n / K < gB) return ck[n / K];
        return work[n & 1];
    };
    NEFTY_CUDA(h, cudaMemsetAsync(state_fwd(0), 0, SB, s));
    if (C.T0.user) NEFTY_CUDA(h, cudaMemcpyAsync(state_fwd(0), C.T0.dev, N * R, cudaMemcpyDeviceToDevice, s));
    NEFTY_CUDA(h, cudaMemsetAsync(grad, 0, N * sizeof(double), s));

    // Pointer tables: forward src/dst (2 nt), recompute src/dst (2 nt), adjoint T
    // (nt + segments), ring saves of the first sweep (nt).
    std::vector<Real*> tab(7 * nt + 4, nullptr);
    Real** F_src = tab.data();
    Real** F_dst = tab.data() + nt;
    Real** R_src = tab.data() + 2 * nt;
    Real** R_dst = tab.data() + 3 * nt;
    Real** A_T = tab.data() + 4 * nt;
    Real** F_ring = tab.data() + 6 * nt + 4;
    for (int n = 0; n < P.nt; ++n) {
        F_src[n] = state_fwd(n);
        F_dst[n] = state_fwd(n + 1);
        if (ck_ring && n + 1 < B && (n + 1) % K == 0) F_ring[n] = ck[(n + 1) / K] + 2 * N;
    }
    // Reverse-sweep segments, latest first: the kept tail [B, nt], then
    // segment g = gB-1 .. 0 over [g K, min(g K + K, B)], recomputed from
    // checkpoint g into segbuf (T^{gK+j} -> segbuf[j-1]).
    struct Seg { int a0, a1; bool rec; size_t aoff; };
    std::vector<Seg> segs;
    size_t aoff = 0;
    if (ntail > 0) {
        segs.push_back(Seg{B, P.nt, false, aoff});
        for (int n = B; n <= P.nt; ++n) A_T[aoff + (n - B)] = tail[n - B];
        aoff += (size_t)ntail;
    }
    for (int g = gB - 1; g >= 0; --g) {
        const int a0 = g * K, a1 = std::min(a0 + K, B);
        segs.push_back(Seg{a0, a1, true, aoff});
        for (int n = a0; n <= a1; ++n) A_T[aoff + (n - a0)] = n == a0 ? ck[g] : segbuf[n - a0 - 1];
        aoff += (size_t)(a1 - a0 + 1);
        for (int n = a0; n < a1; ++n) {
            R_src[n] = n == a0 ? ck[g] : segbuf[n - a0 - 1];
            R_dst[n] = segbuf[n - a0];
        }
    }
    NEFTY_CUDA(h, cudaMemcpyAsync(C.tables, tab.data(), tab.size() * sizeof(Real*), cudaMemcpyHostToDevice, s));
    Real** dF_src = C.tables;
    Real** dF_dst = C.tables + nt;
    Real** dR_src = C.tables + 2 * nt;
    Real** dR_dst = C.tables + 3 * nt;
    Real** dA_T = C.tables + 4 * nt;

    Real** dF_ring = C.tables + 6 * nt + 4;
    // forward sweep with the loss
    if (nefty_status e = C.forward_steps(0, P.nt, dF_src, dF_dst, C.iters, C.resid, nullptr,
                                         (const Real*)C.obs.dev, C.loss_partials, 0, nullptr,
                                         ck_ring ? dF_ring : nullptr, 0))
        return e;

    // FP32: the adjoint sweep runs on a power-of-two multiple 2^k of the
    // adjoint problem (exact, as it is linear), with k chosen from the surface
    // misfit so that mu is of order one; its squared norms and error terms
    // then stay in the normal range of FP32 however small the misfit is.  The
    // gradient and dJ/dT0 are scaled back by 2^-k.
    double adj_scale = 1.0;
    if constexpr (Call<Real>::kTiled) {
        std::vector<double> lp(C.G);
        NEFTY_CUDA(h, cudaMemcpyAsync(lp.data(), C.loss_partials, C.G * sizeof(double), cudaMemcpyDeviceToHost, s));
        NEFTY_CUDA(h, cudaStreamSynchronize(s));
        double sq = 0.0;
        for (double v : lp) sq += v;
        const double src = 2.0 * P.loss_scale * std::sqrt(sq / ((double)P.nt * (double)P.S));
        if (src > 0.0 && std::isfinite(src))
            adj_scale = std::ldexp(1.0, std::max(-120, std::min(120, -(int)std::lround(std::log2(src)))));
    }

    // reverse sweep, one segment at a time
    NEFTY_CUDA(h, cudaMemsetAsync(mu[(P.nt + 1) & 1], 0, SB, s));
    int rec_steps = 0, adj_steps = 0;
    AdjArgs<Real> aa{};
    aa.op = make_view<Real>(P, C.coef);
    aa.r = C.r; aa.p = C.p; aa.q = C.q;
    aa.mu[0] = mu[0]; aa.mu[1] = mu[1];
    aa.alpha = (const Real*)C.alpha.dev;
    aa.wx = 2.0 * P.dt / (P.dx * P.dx);
    aa.wy = 2.0 * P.dt / (P.dy * P.dy);
    aa.wz = 2.0 * P.dt / (P.dz * P.dz);
    aa.g_scale = 2.0 * P.loss_scale;
    aa.obs_off = P.obs_face ? (unsigned)(P.nz - 1) * P.S : 0u;
    aa.obs = (const Real*)C.obs.dev;
    aa.grad = grad;
    aa.tol2 = P.rtol * P.rtol;
    aa.max_iter = P.max_iter;
    aa.jacobi_k = P.jacobi_k;
    aa.ctl = C.ctl;
    aa.partials = C.partials;
    for (const Seg& sg : segs) {
        const int a0 = sg.a0, a1 = sg.a1;
        if (sg.rec) {
            const int g = a0 / K;
            if (nefty_status e = C.forward_steps(a0, a1, dR_src + a0, dR_dst + a0, C.iters + nt + rec_steps,
                                                 C.resid + nt + rec_steps, nullptr, nullptr, nullptr, 1,
                                                 ck_ring && g > 0 ? ck[g] + 2 * N : nullptr, nullptr,
                                                 std::min(a0, tiled::kRing), ck_ring && g > 0 ? 1 : 0))
                return e;
            rec_steps += a1 - a0;
        }
        if constexpr (Call<Real>::kTiled) {
            tiled::AdjTiled ta{};
            ta.c = C.tiled_common(C.iters + 2 * nt + adj_steps, C.resid + 2 * nt + adj_steps);
            ta.n0 = a0;
            ta.n1 = a1;
            ta.ring = C.ring_a;
            ta.ystart = C.ystart;
            ta.extrap = P.extrap;
            ta.hist0 = std::min(adj_steps, tiled::kRing);
            ta.carry = adj_steps > 0 ? 1 : 0;   // the launch before left the residual of step a1
            ta.cflag = C.cflag + (P.nt + 1);
            ta.T = (float* const*)(dA_T + sg.aoff);
            ta.mu[0] = mu[0];
            ta.mu[1] = mu[1];
            ta.alpha = (const float*)C.alpha.dev;
            ta.wx = (float)aa.wx; ta.wy = (float)aa.wy; ta.wz = (float)aa.wz;
            ta.g_scale = (float)(aa.g_scale * adj_scale);
            ta.obs_off = aa.obs_off;
            ta.obs = (const float*)C.obs.dev;
            ta.grad = reinterpret_cast<float2*>(grad);   // N pairs in the N-double accumulator
            if (nefty_status e = C.launch_adj_tiled(ta)) return e;
        } else {
            aa.n0 = a0;
            aa.n1 = a1;
            aa.T = dA_T + sg.aoff;
            aa.iters = C.iters + 2 * nt + adj_steps;
            aa.resid = C.resid + 2 * nt + adj_steps;
            if (nefty_status e = C.launch_adj(aa)) return e;
        }
        adj_steps += a1 - a0;
    }
    if constexpr (Call<Real>::kTiled) {
        const float unscale = (float)(1.0 / adj_scale);
        NEFTY_CUDA(h, launch_cast_pairs(reinterpret_cast<const float2*>(grad), (float*)ga.dev, P.N, unscale, s));
        if (gt.user)   // dJ/dT0 = mu^1, a compensated pair
            NEFTY_CUDA(h, launch_cast_split_pairs((const float*)mu[1], (const float*)mu[1] + N, (float*)gt.dev, P.N,
                                                  unscale, s));
    } else {
        NEFTY_CUDA(h, launch_cast<Real>(grad, (Real*)ga.dev, P.N, s));
        if (gt.user) NEFTY_CUDA(h, cudaMemcpyAsync(gt.dev, mu[1], N * R, cudaMemcpyDeviceToDevice, s));
    }
    ++C.launches;
    for (Output* o : {&ga, &gt})
        if (o->user && o->stage)
            NEFTY_CUDA(h, cudaMemcpyAsync(o->user, o->dev, o->bytes, cudaMemcpyDeviceToHost, s));
    return C.finish(loss_out, true, st, P.nt, rec_steps, adj_steps, K, gB + (int)segbuf.size() + ntail);
}

}  // namespace

// Workspace one forward (adjoint = false) or adjoint_grad call of the problem
// would take on h, with its checkpoint stride chosen within h's budget.
nefty_status nefty::job_workspace_bytes(nefty_handle* h, const nefty_problem* p, bool adjoint, const void* alpha,
                                        const void* T0, const void* q_face, const void* q_full, const void* obs,
                                        size_t* bytes) {
    Prob P;
    std::string why;
    if (check_problem(p, &P, &why)) return fail(h, NEFTY_EINVAL, why);
    DeviceGuard guard(h->device);
    const int qs = q_face ? 1 : 0;
    if (P.prec == NEFTY_FP32)
        return adjoint ? run_adjoint<float>(h, P, alpha, T0, q_face, qs, q_full, obs, nullptr, nullptr, nullptr,
                                            nullptr, nullptr, bytes)
                       : run_forward<float>(h, P, alpha, T0, q_face, qs, q_full, nullptr, nullptr, obs, nullptr,
                                            nullptr, nullptr, bytes);
    return adjoint ? run_adjoint<double>(h, P, alpha, T0, q_face, qs, q_full, obs, nullptr, nullptr, nullptr,
                                         nullptr, nullptr, bytes)
                   : run_forward<double>(h, P, alpha, T0, q_face, qs, q_full, nullptr, nullptr, obs, nullptr,
                                         nullptr, nullptr, bytes);
}

// ===================================================================== C ABI
extern "C" {

const char* nefty_status_string(nefty_status s) {
    switch (s) {
        case NEFTY_OK: return "NEFTY_OK";
        case NEFTY_EINVAL: return "NEFTY_EINVAL";
        case NEFTY_ENOMEM: return "NEFTY_ENOMEM";
        case NEFTY_ENOTCONV: return "NEFTY_ENOTCONV";
        case NEFTY_ECUDA: return "NEFTY_ECUDA";
        case NEFTY_ETIMEOUT: return "NEFTY_ETIMEOUT";
        case NEFTY_EBUSY: return "NEFTY_EBUSY";
        case NEFTY_ECANCELLED: return "NEFTY_ECANCELLED";
        case NEFTY_ENOTFOUND: return "NEFTY_ENOTFOUND";
    }
    return "NEFTY_UNKNOWN";
}

nefty_status nefty_debug_barrier_fault(nefty_handle* h, uint32_t missing_arrivals, uint64_t wait_limit_ns) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (missing_arrivals > 1024u) return fail(h, NEFTY_EINVAL, "missing_arrivals must be <= 1024");
    if (wait_limit_ns > 60ull * 1000000000ull) return fail(h, NEFTY_EINVAL, "wait_limit_ns must be <= 60 s");
    h->fault_missing = missing_arrivals;
    h->fault_wait_ns = wait_limit_ns;
    return NEFTY_OK;
}

const char* nefty_last_error(const nefty_handle* h) {
    if (h) return h->err.c_str();
    return t_err.c_str();
}

nefty_status nefty_problem_check(const nefty_problem* p) {
    std::string why;
    nefty_status s = check_problem(p, nullptr, &why);
    if (s) t_err = why;
    return s;
}

nefty_status nefty_create(nefty_handle** out, int device, uint64_t mem_budget_bytes) {
    if (!out) return fail(nullptr, NEFTY_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(nullptr, NEFTY_ECUDA, std::string("no CUDA device: ") + cudaGetErrorName(e));
    }
    if (device < 0 || device >= count) return fail(nullptr, NEFTY_EINVAL, "device index out of range");
    DeviceGuard guard(device);
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMemGetInfo");
    nefty_handle* h = new nefty_handle();
    h->device = device;
    h->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(0.9 * (double)free_b);
    *out = h;
    return NEFTY_OK;
}

nefty_status nefty_destroy(nefty_handle* h) {
    if (!h) return NEFTY_OK;
    if (h->server) {
        server_stop(h->server);
        h->server = nullptr;
    }
    {
        DeviceGuard guard(h->device);
        if (h->ws) cudaFree(h->ws);
        drop_keep(h);
    }
    delete h;
    return NEFTY_OK;
}

nefty_status nefty_forward(nefty_handle* h, const nefty_problem* p, const void* alpha, const void* T0,
                           const void* q_face, int32_t q_steps, const void* q_full, void* frames_out,
                           void* T_final, const void* obs, double* loss_out, nefty_stats* stats,
                           void* stream) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    Prob P;
    std::string why;
    if (check_problem(p, &P, &why)) return fail(h, NEFTY_EINVAL, why);
    if (!alpha) return fail(h, NEFTY_EINVAL, "alpha is NULL");
    if (loss_out && !obs) return fail(h, NEFTY_EINVAL, "loss_out needs obs");
    if (q_steps < 0) return fail(h, NEFTY_EINVAL, "q_steps must be >= 0");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (P.prec == NEFTY_FP32)
        return run_forward<float>(h, P, alpha, T0, q_face, q_steps, q_full, frames_out, T_final, obs,
                                  loss_out, stats, s);
    return run_forward<double>(h, P, alpha, T0, q_face, q_steps, q_full, frames_out, T_final, obs,
                               loss_out, stats, s);
}

nefty_status nefty_adjoint_grad(nefty_handle* h, const nefty_problem* p, const void* alpha,
                                const void* T0, const void* q_face, int32_t q_steps,
                                const void* q_full, const void* obs, double* loss_out,
                                void* grad_alpha, void* grad_T0, nefty_stats* stats, void* stream) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    Prob P;
    std::string why;
    if (check_problem(p, &P, &why)) return fail(h, NEFTY_EINVAL, why);
    if (!alpha || !obs || !grad_alpha) return fail(h, NEFTY_EINVAL, "alpha, obs and grad_alpha are required");
    if (q_steps < 0) return fail(h, NEFTY_EINVAL, "q_steps must be >= 0");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (P.prec == NEFTY_FP32)
        return run_adjoint<float>(h, P, alpha, T0, q_face, q_steps, q_full, obs, loss_out, grad_alpha,
                                  grad_T0, stats, s);
    return run_adjoint<double>(h, P, alpha, T0, q_face, q_steps, q_full, obs, loss_out, grad_alpha,
                               grad_T0, stats, s);
}

nefty_status nefty_serve_start(nefty_handle* h, const nefty_serve_config* cfg) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (h->server) return fail(h, NEFTY_EINVAL, "a server is already attached to this handle");
    nefty_status st = NEFTY_OK;
    std::string why;
    h->server = server_start(h->device, cfg, &st, &why);
    if (!h->server) return fail(h, st, why);
    return NEFTY_OK;
}

nefty_status nefty_serve_submit(nefty_handle* h, const nefty_job* job, uint64_t* job_id) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (!job || !job_id) return fail(h, NEFTY_EINVAL, "job and job_id are required");
    if (!h->server) return fail(h, NEFTY_EBUSY, "no server attached (nefty_serve_start)");
    std::string why;
    const nefty_status st = server_submit(h->server, job, job_id, &why);
    if (st != NEFTY_OK) return fail(h, st, why);
    return NEFTY_OK;
}

nefty_status nefty_serve_poll(nefty_handle* h, uint64_t job_id, nefty_job_result* out) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (!out) return fail(h, NEFTY_EINVAL, "out is NULL");
    if (!h->server) return fail(h, NEFTY_ENOTFOUND, "no server attached");
    const nefty_status st = server_poll(h->server, job_id, out);
    if (st != NEFTY_OK) return fail(h, st, "unknown job id");
    return NEFTY_OK;
}

nefty_status nefty_serve_cancel(nefty_handle* h, uint64_t job_id) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (!h->server) return fail(h, NEFTY_ENOTFOUND, "no server attached");
    const nefty_status st = server_cancel(h->server, job_id);
    if (st != NEFTY_OK) return fail(h, st, "unknown job id");
    return NEFTY_OK;
}

nefty_status nefty_serve_stop(nefty_handle* h) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (h->server) {
        server_stop(h->server);
        h->server = nullptr;
    }
    return NEFTY_OK;
}

}  // extern "C"

namespace {

bool field_dims(const nefty_field_desc* d, FieldDims* out, std::string* why) {
    if (!d) { *why = "field descriptor is NULL"; return false; }
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) { *why = "field grid must be >= 1 in each direction"; return false; }
    const double cells = (double)d->nx * d->ny * d->nz;
    if (cells >= 2147483647.0 - 128) { *why = "field grid too large"; return false; }
    if (d->n_freq < 1 || d->n_freq > 1024) { *why = "n_freq must be in 1..1024"; return false; }
    if (d->width < 128 || d->width % 128 != 0) { *why = "width must be a positive multiple of 128"; return false; }
    if (d->depth < 1 || d->depth > 15) { *why = "depth must be in 1..15"; return false; }
    if (d->skip_layer < 0 || (d->skip_layer > 0 && d->skip_layer >= d->depth)) {
        *why = "skip_layer must be 0 (none) or a hidden layer 1..depth-1";
        return false;
    }
    if (d->precision != 0 && d->precision != 1) { *why = "precision must be 0 (BF16) or 1 (split BF16)"; return false; }
    if (d->keep_activations != 0 && d->keep_activations != 1) { *why = "keep_activations must be 0 or 1"; return false; }
    if (!(d->freq_lo > 0) || !(d->freq_hi >= d->freq_lo) || !std::isfinite(d->freq_hi)) {
        *why = "need 0 < freq_lo <= freq_hi";
        return false;
    }
    if (!(d->alpha_min > 0) || !(d->alpha_max > d->alpha_min) || !std::isfinite(d->alpha_max)) {
        *why = "need 0 < alpha_min < alpha_max";
        return false;
    }
    if (out) {
        out->nx = d->nx; out->ny = d->ny; out->nz = d->nz;
        out->M = (unsigned)cells;
        out->Mp = (out->M + 127u) / 128u * 128u;
        out->F = d->n_freq; out->W = d->width; out->depth = d->depth;
        out->skip = d->skip_layer;
        out->Dp = (6 * d->n_freq + 63) / 64 * 64;
        out->ns = d->precision == 1 ? 3 : 1;
        out->freq_lo = d->freq_lo; out->freq_hi = d->freq_hi;
        out->alpha_min = d->alpha_min; out->alpha_max = d->alpha_max;
        // split-K of the weight-gradient GEMMs: one CTA per SM (per layer, see
        // field_backward); `splits` bounds it for the partials buffer
        out->sms = 152;
        const int kblocks = (int)(out->Mp / 64);
        const int min_tiles = ((out->W + 127) / 128) * ((std::min(out->Dp, out->W) + 127) / 128);
        out->splits = std::min(std::max(1, out->sms / std::max(1, min_tiles)), kblocks);
        out->colsum_blocks = (int)std::min<unsigned>(1024u, std::max(1u, out->Mp / 256u));
    }
    return true;
}

// Descriptors that give the same activations and head.
bool same_field(const FieldDims& a, const FieldDims& b) {
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.F == b.F && a.W == b.W && a.depth == b.depth &&
           a.skip == b.skip && a.ns == b.ns && a.freq_lo == b.freq_lo && a.freq_hi == b.freq_hi &&
           a.alpha_min == b.alpha_min && a.alpha_max == b.alpha_max;
}

}  // namespace

extern "C" {

uint64_t nefty_field_param_count(const nefty_field_desc* d) {
    FieldDims fd;
    std::string why;
    if (!field_dims(d, &fd, &why)) return 0;
    return field_param_count(fd.F, fd.W, fd.depth, fd.skip);
}

static nefty_status field_call(nefty_handle* h, const nefty_field_desc* d, const float* theta,
                               const float* band_weights, const float* grad_alpha, float* out, bool backward,
                               void* stream) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    FieldDims fd;
    std::string why;
    if (!field_dims(d, &fd, &why)) return fail(h, NEFTY_EINVAL, why);
    if (!theta || !out || (backward && !grad_alpha)) return fail(h, NEFTY_EINVAL, "missing array argument");
    DeviceGuard guard(h->device);
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess && sms > 0 &&
            sms != fd.sms) {
            const int kblocks = (int)(fd.Mp / 64);
            const int min_tiles = ((fd.W + 127) / 128) * ((std::min(fd.Dp, fd.W) + 127) / 128);
            fd.sms = sms;
            fd.splits = std::min(std::max(1, sms / std::max(1, min_tiles)), kblocks);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = field_param_count(fd.F, fd.W, fd.depth, fd.skip);
    Input th, bw, ga;
    th.plan(theta, P * 4, h->device);
    bw.plan(band_weights, (size_t)fd.F * 4, h->device);
    ga.plan(backward ? grad_alpha : nullptr, (size_t)fd.M * 4, h->device);
    Output o;
    o.plan(out, (backward ? P : (size_t)fd.M) * 4, h->device);
    if (nefty_status e = reject_foreign(h, th, bw, ga, o)) return e;
    // keep_activations: the field workspace is the handle's kept buffer (the
    // backward layout, then copies of theta and the band weights, then a flag)
    const size_t bwd_bytes = field_workspace_bytes(fd, true);
    const size_t snap_th = (bwd_bytes + 255) & ~(size_t)255, snap_bw = snap_th + ((P * 4 + 255) & ~(size_t)255);
    const size_t snap_flag = snap_bw + (((size_t)fd.F * 4 + 255) & ~(size_t)255), keep_need = snap_flag + 256;
    bool keep = d->keep_activations == 1;
    char* fws = nullptr;
    auto layout = [&](Arena& a) {
        th.place(a); bw.place(a); ga.place(a); o.place(a);
        if (!keep) fws = (char*)a.take(field_workspace_bytes(fd, backward));
    };
    Arena probe;
    if (keep) {   // the staging workspace first, then the kept buffer in the room left
        layout(probe);
        if (nefty_status e = ensure_workspace(h, probe.off)) return e;
        if (h->keep_bytes < keep_need) {
            drop_keep(h);
            if (keep_need + h->ws_bytes <= h->budget && cudaMalloc(&h->keep, keep_need) == cudaSuccess)
                h->keep_bytes = keep_need;
            else {
                cudaGetLastError();
                h->keep = nullptr;
                keep = false;   // no room: run as without keep_activations
            }
        }
        probe = Arena();
    }
    layout(probe);
    if (nefty_status e = ensure_workspace(h, probe.off)) return e;
    if (keep && !h->keep) keep = false;   // the workspace took the kept buffer's room
    Arena arena;
    arena.base = (char*)h->ws;
    layout(arena);
    if (keep) fws = (char*)h->keep;
    for (Input* in : {&th, &bw, &ga})
        if (in->user && in->stage) NEFTY_CUDA(h, cudaMemcpyAsync(in->dev, in->user, in->bytes, cudaMemcpyHostToDevice, s));
    float* const kth = keep ? (float*)(fws + snap_th) : nullptr;
    float* const kbw = keep ? (float*)(fws + snap_bw) : nullptr;
    bool reuse = false;
    if (keep && backward && h->keep_valid && same_field(h->keep_dims, fd) && h->keep_bw == (bw.dev != nullptr)) {
        // the kept evaluation is reused only at bitwise-equal parameters
        int* flag = (int*)(fws + snap_flag);
        NEFTY_CUDA(h, cudaMemsetAsync(flag, 1, sizeof(int), s));
        NEFTY_CUDA(h, field_params_equal((const float*)th.dev, kth, P, flag, s));
        if (bw.dev) NEFTY_CUDA(h, field_params_equal((const float*)bw.dev, kbw, (size_t)fd.F, flag, s));
        int same = 0;
        NEFTY_CUDA(h, cudaMemcpyAsync(&same, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        NEFTY_CUDA(h, cudaStreamSynchronize(s));
        reuse = same != 0;
    }
    if (keep) h->keep_valid = false;   // until this call has finished writing the buffer
    if (backward)
        NEFTY_CUDA(h, field_backward(fd, (const float*)th.dev, (const float*)bw.dev, (const float*)ga.dev,
                                     (float*)o.dev, fws, s, reuse));
    else
        NEFTY_CUDA(h, field_eval(fd, (const float*)th.dev, (const float*)bw.dev, (float*)o.dev, fws, s, keep));
    if (keep && !reuse) {   // the buffer now holds the evaluation at these parameters
        NEFTY_CUDA(h, cudaMemcpyAsync(kth, th.dev, P * 4, cudaMemcpyDeviceToDevice, s));
        if (bw.dev) NEFTY_CUDA(h, cudaMemcpyAsync(kbw, bw.dev, (size_t)fd.F * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (o.stage) NEFTY_CUDA(h, cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, s));
    const int err = field_error(fd, fws, s, backward || keep);
    if (err < 0) return fail(h, NEFTY_ECUDA, "field: stream synchronisation failed");
    if (err > 0) return fail(h, NEFTY_ETIMEOUT, "field: a tensor-core pipeline wait timed out");
    if (keep) {
        h->keep_valid = true;
        h->keep_bw = bw.dev != nullptr;
        h->keep_dims = fd;
    }
    if (reuse) ++h->field_reuses;
    return NEFTY_OK;
}

uint64_t nefty_field_activation_reuses(const nefty_handle* h) { return h ? h->field_reuses : 0; }

nefty_status nefty_field_eval(nefty_handle* h, const nefty_field_desc* d, const float* theta,
                              const float* band_weights, float* alpha_out, void* stream) {
    return field_call(h, d, theta, band_weights, nullptr, alpha_out, false, stream);
}

nefty_status nefty_field_backward(nefty_handle* h, const nefty_field_desc* d, const float* theta,
                                  const float* band_weights, const float* grad_alpha, float* grad_theta,
                                  void* stream) {
    return field_call(h, d, theta, band_weights, grad_alpha, grad_theta, true, stream);
}

nefty_status nefty_gemm_bf16(nefty_handle* h, const void* A, int32_t lda, const void* B, int32_t ldb, int32_t M,
                             int32_t N, int32_t K, float* C, void* stream) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    if (!A || !B || !C || M < 1 || N < 1 || K < 64 || K % 64 || lda % 8 || ldb % 8 || lda < K || ldb < K)
        return fail(h, NEFTY_EINVAL, "gemm: bad arguments");
    if (ptr_kind(A, h->device) != kPtrDevice || ptr_kind(B, h->device) != kPtrDevice ||
        ptr_kind(C, h->device) != kPtrDevice)
        return fail(h, NEFTY_EINVAL, "gemm: device pointers of the handle's GPU only");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (nefty_status e = ensure_workspace(h, 256)) return e;
    int* err = (int*)h->ws;
    NEFTY_CUDA(h, cudaMemsetAsync(err, 0, sizeof(int), s));
    NEFTY_CUDA(h, umma_gemm((const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, M, N, K, 2, nullptr, nullptr,
                            nullptr, C, N, 1, err, s));
    int herr = 0;
    NEFTY_CUDA(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NEFTY_CUDA(h, cudaStreamSynchronize(s));
    if (herr) return fail(h, NEFTY_ETIMEOUT, "gemm: a tensor-core pipeline wait timed out");
    return NEFTY_OK;
}

nefty_status nefty_tv(nefty_handle* h, const nefty_problem* p, const void* alpha, double lam, double eps,
                      double* tv_out, void* grad_alpha_accum, void* stream) {
    if (!h) return fail(nullptr, NEFTY_EINVAL, "handle is NULL");
    Prob P;
    std::string why;
    if (check_problem(p, &P, &why)) return fail(h, NEFTY_EINVAL, why);
    if (!alpha) return fail(h, NEFTY_EINVAL, "alpha is NULL");
    if (!(lam >= 0) || !std::isfinite(lam) || !(eps >= 0) || !std::isfinite(eps))
        return fail(h, NEFTY_EINVAL, "lam and eps must be finite and >= 0");
    DeviceGuard guard(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t R = P.prec == NEFTY_FP32 ? 4 : 8, N = P.N;
    const int blocks = tv_blocks(P.N);
    Input a;
    a.plan(alpha, N * R, h->device);
    Output g;
    g.plan(grad_alpha_accum, N * R, h->device);
    if (nefty_status e = reject_foreign(h, a, g)) return e;
    double* partials = nullptr;
    auto layout = [&](Arena& ar) {
        partials = (double*)ar.take((size_t)blocks * sizeof(double));
        a.place(ar);
        g.place(ar);
    };
    Arena probe;
    layout(probe);
    if (nefty_status e = ensure_workspace(h, probe.off)) return e;
    Arena arena;
    arena.base = (char*)h->ws;
    layout(arena);
    if (a.stage) NEFTY_CUDA(h, cudaMemcpyAsync(a.dev, a.user, a.bytes, cudaMemcpyHostToDevice, s));
    if (g.user && g.stage) NEFTY_CUDA(h, cudaMemcpyAsync(g.dev, g.user, g.bytes, cudaMemcpyHostToDevice, s));
    if (P.prec == NEFTY_FP32)
        NEFTY_CUDA(h, launch_tv<float>((const float*)a.dev, P.nx, P.ny, P.nz, P.bc, P.dx, P.dy, P.dz, lam, eps,
                                       (float*)g.dev, partials, blocks, s));
    else
        NEFTY_CUDA(h, launch_tv<double>((const double*)a.dev, P.nx, P.ny, P.nz, P.bc, P.dx, P.dy, P.dz, lam, eps,
                                        (double*)g.dev, partials, blocks, s));
    if (g.user && g.stage) NEFTY_CUDA(h, cudaMemcpyAsync(g.user, g.dev, g.bytes, cudaMemcpyDeviceToHost, s));
    std::vector<double> part(blocks);
    NEFTY_CUDA(h, cudaMemcpyAsync(part.data(), partials, blocks * sizeof(double), cudaMemcpyDeviceToHost, s));
    NEFTY_CUDA(h, cudaStreamSynchronize(s));
    double t = 0.0;
    for (double v : part) t += v;
    if (tv_out) *tv_out = lam * P.dx * P.dy * P.dz * t;
    return NEFTY_OK;
}

}  // extern "C"
