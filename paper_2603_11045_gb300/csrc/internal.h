// Internal interface between the C-ABI layer (api.cu) and the solver kernels
// (solver.cu).  Not installed; callers use include/nefty.h.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nefty.h"

namespace nefty {

// Threads per CTA of the persistent solver kernels.
constexpr int kThreads = 512;
// Maximum number of values reduced together across the grid.
constexpr int kMaxRed = 8;
// Defaults of a problem's CG stop test (rtol = 0, max_iter = 0), shared by
// every entry point.
constexpr double kDefaultRtolFp32 = 5e-10;
constexpr double kDefaultRtolFp64 = 1e-13;
constexpr int kDefaultMaxIter = 1000;
// Device-side wait limit of a grid barrier (nanoseconds of %globaltimer).
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

// Device error word values.
enum DevError : int { kDevOk = 0, kDevTimeout = 1, kDevBadAlpha = 2, kDevBadState = 3 };

// Shared control block of one persistent launch (device memory, zeroed by the
// host before each launch except `err`, which persists over a call).
struct DevCtl {
    unsigned int bar;      // grid-barrier arrival counter
    unsigned int bar2;     // the second counter of grouped launches (they alternate; see group_tiled)
    int err;               // DevError of the call
    int notconv;           // number of solves that hit max_iter
    unsigned int missing;  // fault injection (tests): arrivals every grid barrier waits for in vain; 0 normally
    unsigned long long wait_ns;   // grid-barrier wait limit (%globaltimer ns); 0 = kBarrierTimeoutNs
    int folded;            // solves whose last CG iteration was applied by the state update
    int carried;           // solves that started from the carried residual
    int stop;              // time-budgeted launches: this step is the launch's last (set by CTA 0)
    int pad;
};

// Grid geometry and the precomputed operator of A(alpha) = I - dt L(alpha).
template <typename Real>
struct OperatorView {
    int nx, ny, nz;
    int px, py;            // lateral wrap active along x / y (periodic and extent > 1)
    unsigned N, S;         // cells, cells per z-plane
    const Real* cx;        // dt * a of the +x face of every cell (0 on a zero-flux wall)
    const Real* cy;
    const Real* cz;
    const Real* d;         // diagonal of A: 1 + sum of the six face values (+ dt*h/dz)
    const Real* dinv;      // 1 / d (Jacobi preconditioner)
    Real robin;            // dt * h / dz on the k = nz-1 cells (0 without a Robin face)
};

// Arguments of the forward persistent kernel: steps n in [n0, n1).
template <typename Real>
struct FwdArgs {
    OperatorView<Real> op;
    Real* r; Real* p; Real* q;         // CG work vectors
    int n0, n1;
    Real* const* src;                  // src[n - n0] = T^n
    Real* const* dst;                  // dst[n - n0] = T^{n+1} (written)
    const Real* q_face; int q_steps;   // flux map applied for n < q_steps
    const Real* q_full;                // per-step flux maps (overrides q_face)
    double src_scale;                  // dt / dz
    unsigned obs_off;                  // first cell of the observed plane
    const Real* obs;                   // target frames [nt][S] or null
    Real* frames;                      // Pi T^{n+1} -> frames[n] or null
    double tol2;                       // rtol^2
    int max_iter;
    DevCtl* ctl;
    double* partials;                  // [2][kMaxRed][G]
    int* iters;                        // per-step CG iterations [n1 - n0]
    double* resid;                     // per-step final ||r||/||b||
    double* loss_partials;             // [G] per-CTA sum of squared frame errors
    int jacobi_k;                      // > 0: K Jacobi sweeps per solve instead of CG
};

// Arguments of the adjoint persistent kernel: steps n = n1 down to n0 + 1.
template <typename Real>
struct AdjArgs {
    OperatorView<Real> op;
    Real* r; Real* p; Real* q;
    int n0, n1;
    Real* const* T;                    // T[n - n0] = T^n, n in [n0, n1]
    Real* mu[2];                       // mu^n lives in mu[n & 1]
    const Real* alpha;
    double wx, wy, wz;                 // 2 dt / h_d^2 (harmonic-mean derivative weights)
    double g_scale;                    // 2 * loss_scale
    unsigned obs_off;
    const Real* obs;                   // [nt][S]
    double* grad;                      // dJ/dalpha accumulator (FP64)
    double tol2;
    int max_iter;
    DevCtl* ctl;
    double* partials;
    int* iters;                        // per-step iterations, index n1 - n
    double* resid;
    int jacobi_k;                      // > 0: K Jacobi sweeps per solve instead of CG
};

// ------------------------------------------------------------ serving (serve.cu)
class Server;
class Batcher;
Server* server_start(int device, const nefty_serve_config* cfg, nefty_status* st, std::string* why);
void server_stop(Server* s);
nefty_status server_submit(Server* s, const nefty_job* job, uint64_t* id, std::string* why);
nefty_status server_poll(Server* s, uint64_t id, nefty_job_result* out);
nefty_status server_cancel(Server* s, uint64_t id);
// api.cu: the persistent grids of h use 1/share of the device; h's memory
// budget (returns the previous one); workspace of a call.
void set_grid_share(nefty_handle* h, int share);
uint64_t set_budget(nefty_handle* h, uint64_t bytes);
nefty_status job_workspace_bytes(nefty_handle* h, const nefty_problem* p, bool adjoint, const void* alpha,
                                 const void* T0, const void* q_face, const void* q_full, const void* obs,
                                 size_t* bytes);

// Message returned by nefty_last_error(NULL) on the calling thread (api.cu).
void set_thread_error(const char* msg);
inline void set_thread_error(const std::string& msg) { set_thread_error(msg.c_str()); }

// Launch helpers (solver.cu).  All are stream-ordered.
int solver_grid_blocks(int device, int prec);
template <typename Real>
cudaError_t launch_coefficients(const Real* alpha, int nx, int ny, int nz, int bc, double dx,
                                double dy, double dz, double dt, double robin_h, Real* cx,
                                Real* cy, Real* cz, Real* d, Real* dinv, DevCtl* ctl,
                                cudaStream_t s);
template <typename Real>
cudaError_t launch_forward(const FwdArgs<Real>& a, int grid, cudaStream_t s);
template <typename Real>
cudaError_t launch_adjoint(const AdjArgs<Real>& a, int grid, cudaStream_t s);
template <typename Real>
cudaError_t launch_cast(const double* in, Real* out, unsigned n, cudaStream_t s);

// Total variation (tv.cu): per-block partial sums of the un-scaled terms into
// partials[blocks]; grad_accum (or null) += lam * dx*dy*dz * dR/dalpha.
int tv_blocks(unsigned N);
template <typename Real>
cudaError_t launch_tv(const Real* alpha, int nx, int ny, int nz, int bc, double dx, double dy, double dz,
                      double lam, double eps, Real* grad_accum, double* partials, int blocks, cudaStream_t s);

// ------------------------------------------------- tiled FP32 solver (cg_tiled.cu)
namespace tiled {

// CTA of the tiled kernels: CW compute warps and one copy warp.  A tile is a
// 32 x 32 column of cells; a compute thread owns QX = 4 consecutive cells
// along x in one row, so the CW = 8 compute warps cover the 32 rows.
constexpr int TX = 32, TY = 32, QX = 4;
constexpr int CW = TY * TX / (32 * QX);          // compute warps
constexpr int NCT = CW * 32;                     // compute threads
constexpr int NT = NCT + 32;                     // + the copy warp
constexpr int kMaxGrid = 320;                    // most CTAs a tiled launch may have

struct Geo {
    int nx, ny, nz;
    int px, py;            // lateral wrap active
    unsigned S;            // nx * ny
    int tiles_x;           // ceil(nx / TX)
    unsigned units;        // (tiles_x * tiles_y) * nz  (tile, plane) work units
};

// CG vectors of the single-reduction iteration (ping-pong pairs are read with
// a halo in one pass and written in the next).
struct Vecs {
    float* u[2];           // M^{-1} r
    float* ws[2];          // M^{-1} A u      (= u[i] + N)
    float* ss[2];          // M^{-1} A p      (= u[i] + 2N)
    float* p;
    float* delta;          // increment of the current solve (= p + N)
    // Carried residual (TMA-staged PCG): the residual of each solve at a zero
    // increment, s = b - A x0, follows from the solve before it (see
    // cg_tiled.cu); sig[0] carries it through a forward sweep, sig[1] through
    // an adjoint sweep (contiguous, sig[1] = sig[0] + N).  diag: the diagonal
    // of A, written at the start of every such launch.
    float* sig[2];
    float* diag;
};

// TMA descriptors of the staged passes (tiled FP32 path).  They travel by
// value in the kernel parameters (which the kernels declare __grid_constant__),
// so every copy reads its descriptor from parameter space.
struct TmaMaps {
    CUtensorMap uws[2];    // u, ws, ss of one ping-pong set (3 x N floats, contiguous):
                           //   4D (x, y, z, 3), box 40 x 34 x 1 x 3 at (x0-4, y0-1, k, 0)
    CUtensorMap u0;        // u of set 0 alone: box 40 x 34 x 1
    CUtensorMap alpha;     // box 40 x 34 x 1 at (x0-4, y0-1, k)
    CUtensorMap pd;        // p, delta (2 x N floats, contiguous): 4D, box 32 x 32 x 1 x 2 at (x0, y0, k, 0)
    CUtensorMap states;    // the state slab as 4D (x, y, z, halves): box 40 x 34 x 1 x 2 at
                           //   (x0-4, y0-1, k, h) reads the hi and lo halves of the state at half h
    CUtensorMap dh;        // delta alone: box 40 x 34 x 1 at (x0-4, y0-1, k)
    CUtensorMap sg;        // sig[0], sig[1] (2 x N floats, contiguous): 4D, box 32 x 32 x 1 x 1 at (x0, y0, k, i)
};

struct Common {
    Geo g;
    TmaMaps maps;          // valid when tma != 0
    int tma;               // passes staged through TMA (else plain loads)
    // Every state the kernels read (T^n and mu^n as compensated pairs of N
    // floats each) lives in one slab of `slab_halves` blocks of N floats; a
    // state at slab offset o (floats) has its hi half at block o / N and its
    // lo half at block o / N + 1.
    const float* slab;
    unsigned slab_halves;
    const float* alpha;    // cell diffusivity; face values are recomputed from it
    float kx, ky, kz;      // dt / h_d^2
    float robin;           // dt h / dz on k = nz-1
    Vecs v;
    DevCtl* ctl;
    double* partials;      // [2][G][kMaxRed] (hi, lo) float pairs
    float tol2_hi, tol2_lo;   // rtol^2 as a double-float
    int bar_sel;           // grid-barrier counter: 0 = ctl->bar, 1 = ctl->bar2 (grouped launches alternate)
    int max_iter;
    int jacobi_k;          // > 0: every solve is K Jacobi sweeps from its warm start (no CG)
    int* iters;
    double* resid;
};

// Increment extrapolation (the CG start of each step): ring slot (m mod
// kRing) of a sweep holds its increment of step m (forward: T^{m+1} - T^m;
// adjoint: mu^m - mu^{m+1}).  With h usable increments the start is x0 + d,
// d = 0 (h = 0) or the next value of the polynomial of degree h - 1 through
// the newest h increments (h = 1: the newest; 2: linear; 3: quadratic; 4:
// cubic); h = min(extrap, increments available).  The end of each solve
// writes the next start y = x0 + d (compensated pairs, a slot of the state
// slab) and d (into delta).
constexpr int kRing = 4;
struct FwdTiled {
    Common c;
    int n0, n1;
    float* ring;              // [kRing][N]
    float* ystart;            // [2][N] the next solve's start y = x0 + d (a slot of the state slab)
    int extrap;               // 0 .. kRing
    int hist0;                // increments valid at launch start (steps n0-1, n0-2, ...)
    const float* ring_load;   // [delta^{n0-1}; delta^{n0-2}; ...] (extrap of them) copied in at launch start, or null
                              //   (+ the carried residual of step n0 after them when carry)
    float* const* ring_save;  // per step n (index n - n0), after T^{n+1}: [delta^n; delta^{n-1}; ...] or null
                              //   (+ the carried residual of step n + 1 after them when the sweep carries it)
    int carry;                // 1: the carried residual of step n0 is valid at launch start (in sig[0], or in
                              //   ring_load when that is given) if cflag[n0] says step n0 uses it; 0: step n0
                              //   forms its residual from the state
    int* cflag;               // [n_end] per step n: 1 if step n starts from the carried residual (written by
                              //   the step before, read by a launch that resumes at n)
    int n_end;                // steps of the whole sweep (the forcing of step n exists for n < n_end)
    unsigned long long budget_ns;   // > 0: stop after the step during which this much device time has
                                    //   passed since the launch began (at least one step)
    int* progress;            // with budget_ns: the next step to run is written here (n1 when all ran)
    float* const* src;
    float* const* dst;
    const float* q_face; int q_steps; const float* q_full;
    float src_scale;
    unsigned obs_off;
    const float* obs;
    float* frames;
    double* loss_partials;
    int loss_add;             // 1: add this launch's frame losses to loss_partials (chunks of one sweep)
};

struct AdjTiled {
    Common c;
    int n0, n1;
    float* ring;              // [kRing][N] adjoint increments
    float* ystart;            // as FwdTiled::ystart
    int extrap;
    int hist0;                // increments valid at launch start (steps n1+1, n1+2, ...)
    int carry;                // 1: the carried residual of step n1 is valid in sig[1] at launch start
    int* cflag;               // as FwdTiled::cflag, per adjoint step (index n)
    unsigned long long budget_ns;   // as FwdTiled::budget_ns
    int* progress;            // with budget_ns: the next step to run (downwards; n0 when all ran)
    float* const* T;
    float* mu[2];
    const float* alpha;
    float wx, wy, wz;      // 2 dt / h_d^2
    float g_scale;         // 2 * loss_scale
    unsigned obs_off;
    const float* obs;
    float2* grad;          // dJ/dalpha accumulator: compensated (hi, lo) pairs
};

// Several sweeps in one persistent launch (serving).  A sweep is the
// argument block of one forward or adjoint launch (its own control word and
// reduction partials); sweep j runs on CTAs off[j] .. off[j + 1] - 1 of the
// launch exactly as a launch of its own would run on that many CTAs.
constexpr int kMaxBatch = 16;
struct BatchSweep {
    int adjoint;           // 0: f is used, 1: a is used
    union {
        FwdTiled f;
        AdjTiled a;
    };
};
struct BatchArgs {
    int n;                 // sweeps in s[0, n)
    int off[kMaxBatch + 1];   // CTA ranges
    BatchSweep s[kMaxBatch];
};

}  // namespace tiled

// -------------------------------------------------- neural field (field.cu)
struct FieldDims {
    int nx, ny, nz;
    unsigned M, Mp;          // points (cells) and rows padded to a multiple of 128
    int F, W, depth;         // bands per axis, hidden width, hidden layers
    int skip;                // hidden layer whose input is [h | gamma(x)] (0 = none)
    int Dp;                  // 6F rounded up to a multiple of 64 (zero-padded feature columns)
    int ns;                  // BF16 blocks per stored value: 1 (BF16) or 3 (split BF16, see field.cu)
    double freq_lo, freq_hi, alpha_min, alpha_max;
    int sms;                 // SMs of the device (split-K sizing)
    int splits;              // largest split-K factor of the weight-gradient GEMMs
    int colsum_blocks;       // row blocks of the bias-gradient reductions
};
size_t field_param_count(int F, int W, int depth, int skip);
size_t field_workspace_bytes(const FieldDims& d, bool backward);
// keep: ws has the backward layout and the evaluation also leaves there what
// field_backward needs (activations, their transposes, the axis tables);
// reuse: field_backward takes them from ws instead of recomputing them.
cudaError_t field_eval(const FieldDims& d, const float* theta, const float* band_w, float* alpha, char* ws,
                       cudaStream_t s, bool keep = false);
cudaError_t field_backward(const FieldDims& d, const float* theta, const float* band_w, const float* g_alpha,
                           float* g_theta, char* ws, cudaStream_t s, bool reuse = false);
// *flag = 0 if the n floats at a and b differ in any bit (left as is otherwise)
cudaError_t field_params_equal(const float* a, const float* b, size_t n, int* flag, cudaStream_t s);
int field_error(const FieldDims& d, char* ws, cudaStream_t s, bool backward);
// tcgen05 BF16 GEMM (umma_gemm.cu): D = A B^T, epi 0 bias+relu->bf16, 1 mask->bf16, 2 fp32 split partials;
// the BF16 epilogues can also write D^T [N x ldt] (out_t); the mask has leading
// dimension ldm (0 = ldo).  Split BF16 outputs (so, tso > 0): each value as
// hi = bf16(v), lo = bf16(v - hi), written [hi | hi | lo] at column offsets
// 0, so, 2 so of out_bf16 and at 0, tso, 2 tso of out_t ([hi | lo | hi] when
// t_order = 1): the operand layouts of a K-concatenated split product
// [Ah | Ah | Al] [Bh | Bl | Bh]^T = Ah Bh^T + Ah Bl^T + Al Bh^T.
cudaError_t umma_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                      int epi, const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out_bf16,
                      float* out_f32, int ldo, int splits, int* err, cudaStream_t s,
                      __nv_bfloat16* out_t = nullptr, int ldt = 0, int ldm = 0, int so = 0, int tso = 0,
                      int t_order = 0, int a_blk = 0, int b_blk = 0, int t_rows = 0, float* colsum = nullptr);
// a_blk / b_blk = R > 0: A / B are K-blocked with R rows (element (r, k) at
// (k / 64) R 64 + r 64 + k % 64; R >= M for A, >= N for B; lda / ldb unused);
// t_rows > 0: out_t is written K-blocked with t_rows rows (ldt unused).
// colsum (BF16 epilogues, M and N multiples of 128): column sums of the stored
// output over each 32 rows, colsum[(row / 32) N + col] (FP32, fixed order).

int tiled_grid_blocks(int device);
// Shared memory (bytes) the tiled kernels request dynamically.
int tiled_dynamic_smem();
// Fill `maps` for the given device buffers; false if the driver refused.
bool tiled_encode_maps(tiled::TmaMaps* maps, const tiled::Geo& g, const tiled::Vecs& v, const float* alpha,
                       const float* slab, unsigned slab_halves);
cudaError_t launch_forward_tiled(const tiled::FwdTiled& a, int grid, cudaStream_t s);
cudaError_t launch_adjoint_tiled(const tiled::AdjTiled& a, int grid, cudaStream_t s);
// One grouped launch (TMA-staged sweeps only): sweep j counts its grid barriers
// on ctl->bar or ctl->bar2 (Common::bar_sel), which must be zero, and zeroes the
// other one at its end for the sweep's next launch.
cudaError_t launch_batch_tiled(const tiled::BatchArgs& b, int grid, cudaStream_t s);
// Batched serving launches (serve.cu).  A Batcher owns one stream and runs the
// sweeps handed to batcher_run from any thread in shared persistent launches
// (tiled::group_tiled) on the whole device.
// api.cu: h's TMA-staged sweeps go to b (null: h launches its own grids);
// the launches that carried h's sweeps so far, and those shared with others.
void set_batcher(nefty_handle* h, Batcher* b);
void batch_counts(nefty_handle* h, int* launches, int* shared);
int batcher_grid(Batcher* b);
// Runs the whole sweep (one forward or adjoint launch's descriptor) in
// launches of b after the work issued on s so far, each launch running the
// next part of it beside the other pending sweeps; returns once the last part
// is launched, with s ordered after that launch.  *launches / *shared:
// launches used, and those that carried other sweeps too.  grid must be
// batcher_grid(b).
nefty_status batcher_run(Batcher* b, const tiled::BatchSweep& whole, int grid, cudaStream_t s, int* launches,
                         int* shared, std::string* why);
// out[i] = (in[i].x + in[i].y) * scale (the tiled gradient accumulator to FP32);
// the split form reads a state's hi and lo halves.
cudaError_t launch_cast_pairs(const float2* in, float* out, unsigned n, float scale, cudaStream_t s);
cudaError_t launch_cast_split_pairs(const float* hi, const float* lo, float* out, unsigned n, float scale,
                                    cudaStream_t s);

}  // namespace nefty
