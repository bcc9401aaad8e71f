/*
 * nefty.h — C ABI of libnefty, the GB300 (sm_103a) hot path of NeFTY
 * (Neural Field Thermal Tomography): the differentiable 3D implicit-Euler
 * heat solve, its discrete adjoint and the diffusivity gradient.
 *
 * Discretisation (Sec. 4.2 and App. D.2 of the paper):
 *   grid of nx*ny*nz cells, layout [z][y][x] with x fastest, spacing dx,dy,dz;
 *   face conductance a_pq = 2 alpha_p alpha_q / (alpha_p + alpha_q) / h_d^2
 *   (harmonic mean, Prop. 1); L(alpha) the 7-point operator built from them;
 *   A(alpha) = I - dt L(alpha); each step solves
 *       A T^{n+1} = T^n + dt * q^n / dz * [k == 0]            (Eq. state_eq)
 *   by Jacobi-preconditioned conjugate gradients, warm-started from T^n.
 *   The surface flux q^n (a map on the z = 0 face) is spread over the k = 0
 *   cell slab; the paper's state equation has no source term (its heat enters
 *   through the initial condition), so q = 0 and T^0 != 0 reproduces it.
 * Objective (Eq. nefty_obj):  J = loss_scale * sum_{n=1..nt} ||Pi T^n - obs^n||^2
 *   with Pi the k = 0 plane (obs_face = 0) or the k = nz-1 plane (obs_face = 1).
 * Adjoint (Eq. adjoint_eq): A^T mu^n = mu^{n+1} + 2 loss_scale Pi^T (Pi T^n - obs^n),
 *   mu^{nt+1} = 0; A is symmetric so the same operator is used.
 * Gradient (Eq. grad_assembly): dJ/dalpha = dt sum_n (d(L T^n)/dalpha)^T mu^n,
 *   with d a_pq / d alpha_p = 2 alpha_q^2 / (alpha_p + alpha_q)^2 / h_d^2;
 *   dJ/dT^0 = mu^1 (App. D.3, "Sensitivity to initial conditions").
 *
 * Conventions for every call below:
 *   - Array arguments are plain pointers.  Each may point to device memory or
 *     to host memory (pageable or pinned); host arrays are copied to the
 *     device inside the call and host outputs are copied back before return.
 *   - Element type: float when prec == NEFTY_FP32, double when NEFTY_FP64.
 *   - The caller owns every array it passes.  The handle owns its workspace
 *     (operator coefficients, CG vectors, checkpoints), allocated with
 *     cudaMalloc on first use, reused by later calls, freed by nefty_destroy.
 *   - Work is issued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Every call returns after its work on `stream` has completed.
 *   - A handle serves one call at a time; calls on one handle from several
 *     threads must be serialised by the caller.
 *   - Errors: argument errors are returned before any work is issued.  A
 *     device-side failure (a grid barrier that timed out, a CUDA error) is
 *     returned by the same call.  nefty_last_error() gives a message.
 */
#ifndef NEFTY_H
#define NEFTY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NEFTY_OK = 0,
    NEFTY_EINVAL = 1,      /* bad argument: sizes, spacing, null pointer, alpha <= 0 or not finite */
    NEFTY_ENOMEM = 2,      /* workspace does not fit the handle's memory budget or the device */
    NEFTY_ENOTCONV = 3,    /* some CG solve hit max_iter; outputs are written but less accurate */
    NEFTY_ECUDA = 4,       /* a CUDA runtime error; see nefty_last_error */
    NEFTY_ETIMEOUT = 5,    /* a device-side wait exceeded its time limit; outputs are invalid */
    NEFTY_EBUSY = 6,       /* serving queue full */
    NEFTY_ECANCELLED = 7,  /* serving job cancelled */
    NEFTY_ENOTFOUND = 8    /* unknown serving job id */
} nefty_status;

typedef enum { NEFTY_FP32 = 0, NEFTY_FP64 = 1 } nefty_precision;

typedef enum {
    NEFTY_BC_NEUMANN = 0,     /* zero-flux walls on all six faces */
    NEFTY_BC_PERIODIC_XY = 1  /* paper default (App. A.5): periodic in x and y, adiabatic in z */
} nefty_bc;

/* One heat-inversion problem.  Fields set to 0 take the stated default. */
typedef struct {
    int32_t nx, ny, nz;    /* cells, each >= 1, nx*ny*nz < 2^31 */
    double dx, dy, dz;     /* cell spacing, > 0 */
    double dt;             /* time step, > 0 */
    int32_t nt;            /* implicit-Euler steps, >= 1 */
    int32_t bc;            /* nefty_bc */
    double robin_h;        /* Robin coefficient h on the k = nz-1 face (App. A.5); 0 = adiabatic */
    int32_t obs_face;      /* 0: observe k = 0 (the heated face); 1: observe k = nz-1 */
    int32_t prec;          /* nefty_precision: FP32 = float vectors and stencil, FP64 inner
                              products and residual norms; FP64 = double throughout */
    double rtol;           /* CG stop: ||b - A x||_2 <= rtol ||b||_2 (recursive residual);
                              0 = 5e-10 (FP32) or 1e-13 (FP64) */
    int32_t max_iter;      /* CG iteration cap per solve; 0 = 1000 */
    int32_t ckpt_every;    /* adjoint: 0 = automatic: every state kept if it fits the budget,
                              else checkpoints every K steps over the first B steps (recomputed
                              segment by segment) and every state of the last nt - B steps, with
                              K and B chosen to recompute the fewest steps the budget allows;
                              1 = keep every state; K >= 2 = checkpoint every K steps over the
                              whole horizon and recompute */
    double loss_scale;     /* 0 = 1/(nt*nx*ny), i.e. the surface mean-squared error */
    int32_t extrap;        /* FP32 path: each solve starts from T^n plus an extrapolation of the
                              previous steps' increments (the adjoint likewise from mu^(n+1));
                              0 = default (3), -1 = none (start at T^n), h = 1..4: the next value
                              of the polynomial of degree h-1 through the last h increments
                              (1 = the last increment, 2 = linear, 3 = quadratic, 4 = cubic).
                              The FP64 path always starts at T^n. */
    int32_t jacobi_k;      /* 0 = each solve is the converged Jacobi-PCG above; K >= 1 = the
                              paper's inner solver (App. D.2, Eq. jacobi_iter): exactly K Jacobi
                              sweeps T <- D^-1 (b - R T) per solve from the warm start T^n (the
                              adjoint from mu^(n+1)), with no stopping test and no extrapolation;
                              rtol, max_iter and extrap are then ignored.  At most 100000. */
    int32_t residual;      /* start residual of each FP32 solve on the TMA-staged kernels: 0 = default
                              (1); 1 = carried: the state update of each step forms the next step's
                              residual at a zero increment from the residual its solve ended with
                              (exact for the fixed A of a sweep), and the next solve starts with one
                              FP32 stencil pass over the predicted increment; a step after a large
                              start residual (above 1000 rtol ||b||) and every 32nd step form it from
                              the state instead; -1 = every solve forms it from the state (the
                              error-free pass).  Ignored on the other paths. */
} nefty_problem;

/* Solver statistics of one call. */
typedef struct {
    int64_t fwd_iters;          /* CG iterations summed over forward steps */
    int64_t recompute_iters;    /* CG iterations of forward steps re-run from checkpoints */
    int64_t adj_iters;          /* CG iterations summed over adjoint steps */
    int32_t fwd_steps, recompute_steps, adj_steps;
    int32_t max_step_iters;     /* largest CG iteration count of any solve */
    int32_t not_converged;      /* solves that hit max_iter */
    int32_t ckpt_every;         /* checkpoint stride used (1 = every state kept); recompute_steps
                                   is the length of the checkpointed part */
    int32_t n_checkpoints;      /* states held for the reverse sweep */
    double max_rel_residual;    /* largest final ||r||/||b|| over all solves */
    uint64_t workspace_bytes;   /* device workspace held by the handle */
    int32_t grid_blocks;        /* persistent CTAs of the solver launch */
    int32_t kernel_launches;    /* library kernels launched by the call */
    double fwd_ms;              /* device time of the forward-sweep launches (CUDA events) */
    double recompute_ms;        /* device time of the checkpoint-recompute launches */
    double adj_ms;              /* device time of the adjoint-sweep launches */
    int32_t tma_staged;         /* 1: the FP32 sweeps ran on the TMA-staged kernels (nx % 4 == 0, either
                                   wall setting); 0: plain global loads (nx % 4 != 0) or the FP64 path */
    int32_t folded_last_iters;  /* solves whose last CG iteration was applied by the state update (its
                                   residual norm known before its pass), so that its pass was left out */
    int32_t carried_solves;     /* solves that started from the carried residual (nefty_problem.residual) */
} nefty_stats;

typedef struct nefty_handle nefty_handle;

/* Create a handle on CUDA device `device`.  mem_budget_bytes caps the
 * workspace (0 = 90% of the device's free memory at creation).
 * Returns NEFTY_ECUDA when no usable device is present. */
nefty_status nefty_create(nefty_handle **out, int device, uint64_t mem_budget_bytes);

/* Free the handle and its workspace.  NULL is accepted. */
nefty_status nefty_destroy(nefty_handle *h);

/* Message of the last failed call on `h` (or of the calling thread when h is
 * NULL, e.g. after nefty_create failed).  Never NULL; owned by the library. */
const char *nefty_last_error(const nefty_handle *h);

/* Static name of a status code. */
const char *nefty_status_string(nefty_status s);

/* Fault injection for tests of the bounded device-side waits; the paper has
 * no counterpart.  Every grid barrier of the solver kernels waits at most a
 * limit of %globaltimer time (2 s by default) and then gives up: the launch
 * records the failure, ends, and the call returns NEFTY_ETIMEOUT with the
 * CUDA context intact.  With missing_arrivals > 0, every grid barrier of the
 * later solver launches of `h` (forward and adjoint sweeps, both precisions)
 * waits for that many CTAs more than the launch has, an arrival that never
 * comes, so the limit runs out on purpose; wait_limit_ns > 0 replaces the
 * 2 s limit of those launches (0 = 2 s).  (0, 0) restores normal operation.
 * Pipeline (mbarrier) waits inside a pass keep their own limit.  Limits:
 * missing_arrivals <= 1024, wait_limit_ns <= 60 s; NEFTY_EINVAL otherwise. */
nefty_status nefty_debug_barrier_fault(nefty_handle *h, uint32_t missing_arrivals, uint64_t wait_limit_ns);

/* Host-only validation of a problem (no device work): NEFTY_OK or NEFTY_EINVAL. */
nefty_status nefty_problem_check(const nefty_problem *p);

/* Forward sweep (Eq. state_eq).
 *   alpha      [nz*ny*nx]  cell diffusivity, every value > 0 and finite.
 *   T0         [nz*ny*nx]  initial temperature, or NULL for zero.
 *   q_face     [ny*nx]     surface flux on z = 0 applied for steps n < q_steps, or NULL.
 *   q_full     [nt*ny*nx]  per-step flux maps (overrides q_face), or NULL.
 *   frames_out [nt*ny*nx]  Pi T^1 .. Pi T^nt, or NULL.
 *   T_final    [nz*ny*nx]  T^nt, or NULL.
 *   obs        [nt*ny*nx]  target frames; with loss_out non-NULL the objective is written.
 *   loss_out   host double*, or NULL.
 *   stats      host nefty_stats*, or NULL. */
nefty_status nefty_forward(nefty_handle *h, const nefty_problem *p, const void *alpha,
                           const void *T0, const void *q_face, int32_t q_steps, const void *q_full,
                           void *frames_out, void *T_final, const void *obs, double *loss_out,
                           nefty_stats *stats, void *stream);

/* Forward sweep, then the reverse-time adjoint (Eq. adjoint_eq) and gradient
 * assembly (Eq. grad_assembly).  Inputs as in nefty_forward; obs is required.
 *   grad_alpha [nz*ny*nx]  dJ/dalpha, overwritten.
 *   grad_T0    [nz*ny*nx]  dJ/dT^0 = mu^1, or NULL.
 * States for the reverse sweep follow p->ckpt_every. */
nefty_status nefty_adjoint_grad(nefty_handle *h, const nefty_problem *p, const void *alpha,
                                const void *T0, const void *q_face, int32_t q_steps,
                                const void *q_full, const void *obs, double *loss_out,
                                void *grad_alpha, void *grad_T0, nefty_stats *stats, void *stream);

/* Neural diffusivity field (Sec. 4.1, App. D.1).  Cell centres x_d = 2(i+1/2)/N_d - 1
 * are encoded with n_freq log-spaced bands per axis, w_b = freq_lo (freq_hi/freq_lo)^(b/(n_freq-1)):
 * features d*2F + 2b, d*2F + 2b + 1 = band_weights[b] * (sin(w_b x_d), cos(w_b x_d)) (band
 * weights: the frequency-annealing weights of Eq. fa_schedule, NULL = 1).  Then `depth` hidden
 * ReLU layers of `width` units and a linear output f; alpha = alpha_min + (alpha_max - alpha_min)
 * * sigmoid(f) (Eq. bracket).  With skip_layer = s > 0 the encoding is re-injected at hidden
 * layer s (App. D.1): its input is [h_s, features] (width + 6 n_freq values).  Dense layers run
 * on the tensor cores with BF16 operands (or split BF16 operands, see `precision`) and FP32
 * accumulation; features, head, biases and gradients are FP32.
 * Parameter vector (FP32, packed): W_0 [width x 6 n_freq], b_0 [width], then W_l [width x in_l],
 * b_l [width] for l = 1 .. depth-1 (in_l = width + 6 n_freq for l = skip_layer, else width),
 * then w_out [width], b_out [1]; weights row-major [out][in].
 * Constraints: 1 <= n_freq <= 1024, width a multiple of 128, 1 <= depth <= 15,
 * skip_layer 0 or in 1 .. depth-1, 0 < freq_lo <= freq_hi, 0 < alpha_min < alpha_max.
 * The paper's field (App. D.4): n_freq 12 with freq_lo = pi, freq_hi = 2^11 pi (the bands
 * 2^k pi), width 512, depth 10, skip_layer 4. */
typedef struct {
    int32_t nx, ny, nz;     /* grid; the field is evaluated at every cell centre */
    int32_t n_freq;         /* bands per axis */
    int32_t width;          /* hidden width */
    int32_t depth;          /* hidden layers */
    double freq_lo, freq_hi;
    double alpha_min, alpha_max;
    int32_t skip_layer;     /* 0 = none; s = 1 .. depth-1: the encoding joins the input of layer s */
    int32_t precision;      /* 0 = BF16 operands (default); 1 = split BF16: every weight, activation
                               and back-propagated delta v is held as hi = bf16(v) plus
                               lo = bf16(v - hi) (about 16 significant bits) and every product
                               takes the three tensor-core products hi*hi + hi*lo + lo*hi into the
                               same FP32 accumulator: 3x the tensor work and activation memory */
    int32_t keep_activations; /* 0 = off (default).  1: nefty_field_eval also writes what the
                               backward needs (activations and their transposes) into a second
                               device buffer of the handle, the size of a backward's field
                               workspace, kept between calls; a following nefty_field_backward
                               with the same descriptor, bitwise-equal theta and band weights
                               (compared on the device) takes them from there instead of
                               running the forward layers again.  Any other call leaves the
                               result unchanged: the backward recomputes, bit for bit the same
                               gradient.  The buffer counts against the memory budget; when a
                               workspace needs the room it is freed (the next backward then
                               recomputes), and when it does not fit the call runs as with 0. */
} nefty_field_desc;

/* Number of FP32 parameters of the packed vector for `d` (0 if d is invalid). */
uint64_t nefty_field_param_count(const nefty_field_desc *d);

/* alpha_out [nz*ny*nx] (float) = field(theta) at every cell centre.
 * theta [param_count] FP32; band_weights [n_freq] FP32 or NULL. */
nefty_status nefty_field_eval(nefty_handle *h, const nefty_field_desc *d, const float *theta,
                              const float *band_weights, float *alpha_out, void *stream);

/* grad_theta [param_count] (overwritten) = (d alpha / d theta)^T grad_alpha, with
 * grad_alpha [nz*ny*nx] FP32 (e.g. dJ/dalpha from nefty_adjoint_grad plus the TV term). */
nefty_status nefty_field_backward(nefty_handle *h, const nefty_field_desc *d, const float *theta,
                                  const float *band_weights, const float *grad_alpha, float *grad_theta,
                                  void *stream);

/* Number of nefty_field_backward calls on h that took the activations of a
 * keep_activations evaluation instead of recomputing them (0 for NULL). */
uint64_t nefty_field_activation_reuses(const nefty_handle *h);

/* The field's tensor-core GEMM on its own: C[M x N] (FP32, row-major, ld N) =
 * A[M x K] B[N x K]^T with A, B BF16 row-major (lda, ldb in elements, multiples of 8)
 * and K a multiple of 64.  Device pointers only. */
nefty_status nefty_gemm_bf16(nefty_handle *h, const void *A, int32_t lda, const void *B, int32_t ldb, int32_t M,
                             int32_t N, int32_t K, float *C, void *stream);

/* Total-variation regulariser (Eq. tv_discrete) and its gradient:
 *   lam * R(alpha),  R = dx dy dz * sum_cells sqrt((d_x a/dx)^2 + (d_y a/dy)^2 + (d_z a/dz)^2 + eps^2)
 * with forward differences; the lateral ones wrap when p->bc is periodic and
 * vanish on the last column/row with zero-flux walls; the z difference
 * vanishes on the last slice.
 *   alpha             [nz*ny*nx] (float for FP32, double for FP64).
 *   tv_out            host double*: lam * R, or NULL.
 *   grad_alpha_accum  [nz*ny*nx]: lam * dR/dalpha is ADDED to it, or NULL.
 * lam, eps >= 0 and finite. */
nefty_status nefty_tv(nefty_handle *h, const nefty_problem *p, const void *alpha, double lam, double eps,
                      double *tv_out, void *grad_alpha_accum, void *stream);

/* Forward sweep that allocates no device memory.
 *
 * The paper has no counterpart; this entry point exists for integration.
 * nefty_forward takes its scratch from a handle that grows with cudaMalloc.
 * Some callers cannot allow that when they need a solve: a serving or
 * real-time loop that has reserved the whole device for its own buffers (so
 * no memory is left to allocate), a loop that cannot take the device-wide
 * synchronisation cudaMalloc and cudaFree may imply, or a host application or
 * plug-in framework that hands out device memory only from its own pool.
 * This call needs no handle and calls no allocator (no cudaMalloc, no
 * cudaFree, no allocating library routine): its scratch is one static device
 * array of 48 MiB that every GPU loading the library holds until the process
 * exits.
 *
 *   device      CUDA device to run on (made current for the call, then restored).
 *   p           as for nefty_forward, with the same defaults for rtol and
 *               max_iter (FP32 or FP64; the FP64 kernel family of nefty_forward
 *               runs in both precisions here).
 *   alpha, T0, q_face, frames_out, T_final, obs: as for nefty_forward, but every
 *               non-NULL array must be device memory of `device` (or managed
 *               memory): nothing is staged.
 *   loss_out    host double*, or NULL; needs obs.
 * Each solve is the converged Jacobi-PCG (p->jacobi_k must be 0).
 * Limits: the problem's scratch, 10 values per cell (40 B FP32, 80 B FP64) plus
 * about 2 MiB of fixed tables, must fit the 48 MiB array (e.g. about 1.1 M cells
 * FP32, 0.57 M cells FP64), and nt <= 65536; larger problems return NEFTY_EINVAL
 * with a message, and so do host arrays and arrays on another device.
 * Set-up: the first call on each device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress) and sizes the launch; make
 * that first call before any stream capture.  All calls on a device share the
 * array and it keeps the last call's contents (each call clears what must start
 * at zero), so calls whose work overlaps on the GPU race and must be serialised
 * by the caller.  Returns after the work on `stream` has completed. */
nefty_status nefty_forward_static(int device, const nefty_problem *p, const void *alpha, const void *T0,
                                  const void *q_face, int32_t q_steps, void *frames_out, void *T_final,
                                  const void *obs, double *loss_out, void *stream);

/* ------------------------------------------------------------------ serving
 * Continuous batching of ragged jobs (forward sweeps and short inversions on
 * grids of any size) behind a non-blocking queue.  nefty_serve_start attaches
 * a server to a handle; `lanes` worker threads (job slots), each with its own
 * CUDA stream and workspace, take queued jobs in arrival order as soon as they
 * are free.  Each lane owns mem_budget_bytes / lanes of device memory; a job's
 * checkpoint plan is chosen within that share (as for ckpt_every = 0), and a
 * job that cannot fit even then is refused at submit with NEFTY_ENOMEM.
 *
 * Batched (the default): the FP32 sweeps of all running jobs whose grids have
 * nx % 4 == 0 (either wall setting) run together in ONE persistent launch over
 * the whole device, whatever their grid sizes and step counts: each sweep runs
 * on its own range of the launch's CTAs, sized in proportion to its work per
 * step, with its own grid barriers.  A launch lasts about launch_us of device
 * time: every sweep in it runs its next time steps until that time has
 * passed, and the next launch continues each from where it stopped, so a
 * newly admitted job joins the launch that follows.  Other sweeps
 * (FP64, nx % 4 != 0, Jacobi-K) and unbatched servers (batched = -1) run each
 * lane's own persistent grid on 1 / lanes of the SMs, resident beside the
 * others.  On lanes a job's results are the same bits alone or among other
 * jobs; batched, its CTA share depends on the mix, which changes only the
 * order of its reductions (results agree to rounding).
 *
 * Job kinds:
 *   NEFTY_JOB_FORWARD    nefty_forward on the job's arrays (frames_out, loss when obs given).
 *   NEFTY_JOB_INVERSION  `iters` steps of projected gradient descent on alpha:
 *                        alpha <- max(alpha - lr * dJ/dalpha, alpha_floor), each step one
 *                        nefty_adjoint_grad; alpha is updated in place; result.loss is the
 *                        loss of the last step's alpha (before its update).
 * Arrays follow the conventions of nefty_forward (device or host memory, element type by
 * problem.prec) and must stay valid until the job is DONE, FAILED or CANCELLED.
 * The serving calls may be made from any thread; the other calls on the same
 * handle stay the caller's to serialise. */
typedef enum { NEFTY_JOB_FORWARD = 0, NEFTY_JOB_INVERSION = 1 } nefty_job_kind;
typedef enum {
    NEFTY_JOB_QUEUED = 0,
    NEFTY_JOB_RUNNING = 1,
    NEFTY_JOB_DONE = 2,
    NEFTY_JOB_FAILED = 3,
    NEFTY_JOB_CANCELLED = 4
} nefty_job_state;

typedef struct {
    nefty_problem problem;
    int32_t kind;               /* nefty_job_kind */
    int32_t iters;              /* inversion steps (>= 1 for NEFTY_JOB_INVERSION) */
    double lr;                  /* inversion step length (> 0) */
    double alpha_floor;         /* inversion lower bound on alpha (> 0) */
    void *alpha;                /* [nz*ny*nx]; updated in place by an inversion */
    const void *T0;             /* or NULL */
    const void *q_face;         /* or NULL */
    int32_t q_steps;
    const void *q_full;         /* or NULL */
    const void *obs;            /* [nt*ny*nx]; required for an inversion */
    void *frames_out;           /* forward: [nt*ny*nx] or NULL */
} nefty_job;

typedef struct {
    int32_t state;              /* nefty_job_state */
    int32_t status;             /* nefty_status of the job (NEFTY_OK while queued or running) */
    int32_t lane;               /* lane that ran it, -1 before admission */
    int32_t iters_done;         /* inversion steps completed */
    uint64_t t_submit_ns;       /* steady-clock timestamps (ns); 0 = not reached */
    uint64_t t_admit_ns;
    uint64_t t_done_ns;
    double loss;                /* see NEFTY_JOB_INVERSION; forward: the loss when obs was given */
    int32_t launches;           /* batched launches that carried the job's sweeps */
    int32_t shared_launches;    /* ... of which carried other jobs' sweeps too */
} nefty_job_result;

typedef struct {
    int32_t lanes;              /* concurrent jobs, 1..16 (0 = 2) */
    int32_t max_queue;          /* queued-job limit for NEFTY_EBUSY (0 = 4096) */
    uint64_t mem_budget_bytes;  /* device memory shared by the lanes (0 = 80% of free memory) */
    int32_t batched;            /* 0 or 1: batched launches (see above); -1: each lane its own grid */
    int32_t chunk_steps;        /* batched: at most this many time steps of a sweep per launch (0 = no
                                   cap beyond launch_us) */
    int32_t launch_us;          /* batched: device time of one launch in microseconds (0 = 20000):
                                   each sweep of a launch runs time steps until that much time has
                                   passed since the launch began (at least one step), so the sweeps
                                   of a launch end together; a job submitted meanwhile joins the
                                   next launch */
} nefty_serve_config;

/* Start serving on h's device (cfg may be NULL for the defaults).
 * NEFTY_EINVAL if a server is already attached. */
nefty_status nefty_serve_start(nefty_handle *h, const nefty_serve_config *cfg);

/* Queue a job (non-blocking); *job_id receives its id.  The job description is
 * copied; the arrays it points to are not.  NEFTY_EINVAL (bad job), NEFTY_ENOMEM
 * (cannot fit a lane's share), NEFTY_EBUSY (queue full, or no server). */
nefty_status nefty_serve_submit(nefty_handle *h, const nefty_job *job, uint64_t *job_id);

/* State of a job (non-blocking).  NEFTY_ENOTFOUND for an unknown id. */
nefty_status nefty_serve_poll(nefty_handle *h, uint64_t job_id, nefty_job_result *out);

/* Cancel a job: a queued job is dropped at once and a running inversion stops
 * after its current step (both end NEFTY_JOB_CANCELLED); a running forward
 * sweep, or a job already finished, is left as it is.  NEFTY_ENOTFOUND for an
 * unknown id. */
nefty_status nefty_serve_cancel(nefty_handle *h, uint64_t job_id);

/* Stop serving: cancels queued jobs, waits for the running ones, frees the
 * lanes.  Also done by nefty_destroy.  NEFTY_OK when no server is attached. */
nefty_status nefty_serve_stop(nefty_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* NEFTY_H */
