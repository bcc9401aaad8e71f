// Persistent Jacobi-preconditioned CG kernels for the implicit-Euler heat
// solve and its adjoint (Sec. 4.2-4.3, App. D.2-D.3 of the paper).
//
// One cooperative launch runs a whole range of time steps: each step forms
// its right-hand side, solves A x = b to ||r|| <= rtol ||b|| with CG, and
// writes its epilogue (surface frame and loss for the forward sweep; the
// face-product gradient for the adjoint sweep) without returning to the host.
// Global reductions are FP64 and deterministic: every CTA writes one partial
// per value, and after a grid barrier every CTA sums all partials in the same
// fixed order, so all CTAs take identical branch decisions and a re-run (the
// recompute of a checkpointed segment) reproduces the states bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace nefty {

// ------------------------------------------------------------------ sync
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-thread view of the grid synchronisation state.  `epoch` is only
// meaningful in thread 0; `red` (number of reductions so far) is uniform.
struct Grid {
    DevCtl* ctl;
    double* partials;
    unsigned G;
    unsigned epoch;
    unsigned red;
    unsigned missing;              // arrivals that never come (fault injection; 0 normally)
    unsigned long long wait_ns;    // barrier wait limit
};

// Grid-wide barrier.  Thread 0 of each CTA arrives with a release add on the
// monotonic counter and polls it with acquire loads.  The wait is bounded:
// after the launch's limit (DevCtl::wait_ns, by default kBarrierTimeoutNs),
// or when another CTA has flagged an error, the CTA
// records kDevTimeout and every thread returns false so the kernel can exit.
__device__ bool grid_sync(Grid& g) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        g.epoch += 1;
        const unsigned target = g.epoch * g.G + g.missing;
        __threadfence();
        red_release_add_u32(&g.ctl->bar, 1u);
        int ok = 1;
        unsigned spins = 0;
        unsigned long long t0 = 0;
        while (ld_acquire_u32(&g.ctl->bar) < target) {
            if ((++spins & 63u) == 0) {
                if (ld_relaxed_s32(&g.ctl->err) != kDevOk) { ok = 0; break; }
                const unsigned long long t = global_ns();
                if (t0 == 0) {
                    t0 = t;
                } else if (t - t0 > g.wait_ns) {
                    atomicCAS(&g.ctl->err, kDevOk, kDevTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum NV doubles over the whole grid.  On return every thread of every CTA
// holds the same totals in v[].  Returns false if the barrier failed.
template <int NV>
__device__ bool grid_sum(Grid& g, double (&v)[NV]) {
    __shared__ double s_warp[kThreads / 32][kMaxRed];
    __shared__ double s_tot[kMaxRed];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double t = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_warp[warp][i] = t;
    }
    __syncthreads();
    double* part = g.partials + (size_t)(g.red & 1u) * kMaxRed * g.G;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = lane < kThreads / 32 ? s_warp[lane][i] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) part[(size_t)i * g.G + blockIdx.x] = t;
        }
    }
    if (!grid_sync(g)) return false;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = 0.0;
            for (unsigned b = lane; b < g.G; b += 32) t += part[(size_t)i * g.G + b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) s_tot[i] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = s_tot[i];
    g.red += 1;
    return true;
}

// Sum of one double over a CTA (result valid in thread 0).
__device__ double block_sum(double v) {
    __shared__ double s[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < kThreads / 32 ? s[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// -------------------------------------------------------------- operator
// (A - I) v at cell c in flux form, sum over the faces f = (c, q) of
// (dt a_f)(v_c - v_q), plus the Robin sink on the back face (App. D.2).
// Writing A v = v + (A - I) v this way keeps the residual b - A x free of the
// cancellation between v_c and its neighbours that the d_c v_c - sum form
// suffers when v is nearly uniform (the warm-started late time steps).
template <typename Real>
__device__ __forceinline__ Real apply_AmI(const OperatorView<Real>& op, const Real* __restrict__ v,
                                          unsigned c) {
    const unsigned i = c % op.nx;
    const unsigned j = (c / op.nx) % op.ny;
    const unsigned k = c / op.S;
    const Real vc = v[c];
    Real s = Real(0);
    if (i + 1 < (unsigned)op.nx) s += op.cx[c] * (vc - v[c + 1]);
    else if (op.px) s += op.cx[c] * (vc - v[c - (op.nx - 1)]);
    if (i > 0) s += op.cx[c - 1] * (vc - v[c - 1]);
    else if (op.px) s += op.cx[c + op.nx - 1] * (vc - v[c + op.nx - 1]);
    const unsigned row = (unsigned)op.nx;
    if (j + 1 < (unsigned)op.ny) s += op.cy[c] * (vc - v[c + row]);
    else if (op.py) s += op.cy[c] * (vc - v[c - (op.ny - 1) * row]);
    if (j > 0) s += op.cy[c - row] * (vc - v[c - row]);
    else if (op.py) s += op.cy[c + (op.ny - 1) * row] * (vc - v[c + (op.ny - 1) * row]);
    if (k + 1 < (unsigned)op.nz) s += op.cz[c] * (vc - v[c + op.S]);
    if (k > 0) s += op.cz[c - op.S] * (vc - v[c - op.S]);
    if (k + 1 == (unsigned)op.nz) s += op.robin * vc;
    return s;
}

template <typename Real>
__device__ __forceinline__ Real apply_A(const OperatorView<Real>& op, const Real* __restrict__ v,
                                        unsigned c) {
    return v[c] + apply_AmI(op, v, c);
}

// ------------------------------------------------------------- CG core
// Solve A (x0 + x) = b for the increment x, given x = 0, r = b - A x0,
// p = M^{-1} r and the grid totals rz = r.z, rr = r.r, bb = b.b.
// Returns false if a barrier failed.  *iters_out / *rel_out get the iteration
// count and the final relative residual (uniform over the grid).
template <typename Real>
__device__ bool cg_iterate(Grid& g, const OperatorView<Real>& op, Real* __restrict__ x,
                           Real* __restrict__ r, Real* __restrict__ p, Real* __restrict__ q,
                           double rz, double rr, double bb, double tol2, int max_iter,
                           int* iters_out, double* rel_out) {
    const unsigned N = op.N;
    const unsigned stride = gridDim.x * kThreads;
    const unsigned c0 = blockIdx.x * kThreads + threadIdx.x;
    const double lim = tol2 * bb;
    int it = 0;
    while (rr > lim && it < max_iter) {
        // q = A p, p.q
        double pq[1] = {0.0};
        for (unsigned c = c0; c < N; c += stride) {
            const Real qc = apply_A(op, p, c);
            q[c] = qc;
            pq[0] += (double)p[c] * (double)qc;
        }
        if (!grid_sum<1>(g, pq)) return false;
        const Real a = (Real)(rz / pq[0]);
        // x += a p, r -= a q, z = M^{-1} r; r.z and r.r
        double s2[2] = {0.0, 0.0};
        for (unsigned c = c0; c < N; c += stride) {
            const Real pc = p[c];
            x[c] += a * pc;
            const Real rc = r[c] - a * q[c];
            r[c] = rc;
            const Real zc = op.dinv[c] * rc;
            s2[0] += (double)rc * (double)zc;
            s2[1] += (double)rc * (double)rc;
        }
        if (!grid_sum<2>(g, s2)) return false;
        ++it;
        rr = s2[1];
        if (rr <= lim) break;
        const Real beta = (Real)(s2[0] / rz);
        rz = s2[0];
        // p = z + beta p
        for (unsigned c = c0; c < N; c += stride) p[c] = op.dinv[c] * r[c] + beta * p[c];
        if (!grid_sync(g)) return false;
    }
    *iters_out = it;
    *rel_out = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    return true;
}

// The paper's inner solver (App. D.2, Eq. jacobi_iter) on the increment:
// with T^(0) the warm start and r0 = b - A T^(0), the sweep
// T <- D^{-1}(b - R T) is delta <- delta + D^{-1}(r0 - A delta) for
// delta = T - T^(0).  Given p = D^{-1} r0 (the first sweep from delta = 0),
// runs the other K - 1 sweeps (ping-pong p / q) and leaves delta^(K) in x.
template <typename Real>
__device__ bool jacobi_iterate(Grid& g, const OperatorView<Real>& op, Real* __restrict__ x,
                               const Real* __restrict__ r, Real* __restrict__ p, Real* __restrict__ q, int K) {
    const unsigned N = op.N;
    const unsigned stride = gridDim.x * kThreads;
    const unsigned c0 = blockIdx.x * kThreads + threadIdx.x;
    if (K <= 1) {
        for (unsigned c = c0; c < N; c += stride) x[c] = p[c];
        return true;
    }
    Real* in = p;
    Real* spare = q;
    for (int kappa = 1; kappa < K; ++kappa) {
        Real* out = kappa == K - 1 ? x : spare;
        for (unsigned c = c0; c < N; c += stride) out[c] = in[c] + op.dinv[c] * (r[c] - apply_A(op, in, c));
        if (!grid_sync(g)) return false;
        spare = in;
        in = out;
    }
    return true;
}

__device__ __forceinline__ Grid make_grid(DevCtl* ctl, double* partials) {
    Grid g;
    g.ctl = ctl;
    g.partials = partials;
    g.G = gridDim.x;
    g.epoch = 0;
    g.red = 0;
    g.missing = ctl->missing;
    g.wait_ns = ctl->wait_ns ? ctl->wait_ns : kBarrierTimeoutNs;
    return g;
}

// ---------------------------------------------------------- forward sweep
template <typename Real>
__global__ void __launch_bounds__(kThreads) forward_kernel(FwdArgs<Real> a) {
    Grid g = make_grid(a.ctl, a.partials);
    const OperatorView<Real>& op = a.op;
    const unsigned N = op.N, S = op.S;
    const unsigned stride = gridDim.x * kThreads;
    const unsigned c0 = blockIdx.x * kThreads + threadIdx.x;
    double loss = 0.0;
    for (int n = a.n0; n < a.n1; ++n) {
        const Real* __restrict__ Tn = a.src[n - a.n0];
        Real* __restrict__ x = a.dst[n - a.n0];
        const Real* qmap = a.q_full ? a.q_full + (size_t)n * S : (n < a.q_steps ? a.q_face : nullptr);
        const Real sc = (Real)a.src_scale;
        // b = T^n + dt q^n / dz on the k = 0 slab; x0 = T^n; r = b - A x0; p = M^{-1} r
        double s3[3] = {0.0, 0.0, 0.0};
        for (unsigned c = c0; c < N; c += stride) {
            const Real t = Tn[c];   // x0 = T^n (warm start)
            const Real src = (qmap && c < S) ? sc * qmap[c] : Real(0);
            const Real b = t + src;
            const Real rc = src - apply_AmI(op, Tn, c);
            const Real zc = op.dinv[c] * rc;
            x[c] = Real(0);
            a.r[c] = rc;
            a.p[c] = zc;
            s3[0] += (double)rc * (double)zc;
            s3[1] += (double)rc * (double)rc;
            s3[2] += (double)b * (double)b;
        }
        if (!grid_sum<3>(g, s3)) return;
        int it = 0;
        double rel = 0.0;
        if (a.jacobi_k > 0) {
            if (!jacobi_iterate(g, op, x, a.r, a.p, a.q, a.jacobi_k)) return;
            it = a.jacobi_k;
        } else if (!cg_iterate(g, op, x, a.r, a.p, a.q, s3[0], s3[1], s3[2], a.tol2, a.max_iter, &it, &rel)) {
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.iters[n - a.n0] = it;
            a.resid[n - a.n0] = rel;
            if (a.jacobi_k == 0 && it >= a.max_iter && rel * rel > a.tol2) atomicAdd(&a.ctl->notconv, 1);
        }
        // T^{n+1} = T^n + delta: the increment was accumulated on its own so that
        // corrections far below one ulp of T survive; one rounding per step.
        for (unsigned c = c0; c < N; c += stride) x[c] = Tn[c] + x[c];
        if (!grid_sync(g)) return;
        // surface frame and squared error of step n + 1
        if (a.frames || a.obs) {
            for (unsigned s = c0; s < S; s += stride) {
                const Real v = x[a.obs_off + s];
                if (a.frames) a.frames[(size_t)n * S + s] = v;
                if (a.obs) {
                    const double e = (double)v - (double)a.obs[(size_t)n * S + s];
                    loss += e * e;
                }
            }
        }
    }
    if (a.loss_partials) {
        const double t = block_sum(loss);
        if (threadIdx.x == 0) a.loss_partials[blockIdx.x] = t;
    }
}

// ----------------------------------------------------------- adjoint sweep
// Face-product gradient of one step (Eq. grad_assembly): for every face
// (c, q) of cell c on axis d,
//   g_c -= dt * (mu_c - mu_q)(T_c - T_q) * 2 alpha_q^2 / (alpha_c + alpha_q)^2 / h_d^2,
// accumulated in FP64 by the thread that owns c.
template <typename Real>
__device__ __forceinline__ double face_term(double w, double ac, double aq, Real dmu, Real dT) {
    const double s = ac + aq;
    return w * aq * aq / (s * s) * (double)dmu * (double)dT;
}

template <typename Real>
__device__ void accumulate_gradient(const AdjArgs<Real>& a, const Real* __restrict__ mu,
                                    const Real* __restrict__ T) {
    const OperatorView<Real>& op = a.op;
    const unsigned N = op.N, S = op.S;
    const unsigned stride = gridDim.x * kThreads;
    const unsigned row = (unsigned)op.nx;
    for (unsigned c = blockIdx.x * kThreads + threadIdx.x; c < N; c += stride) {
        const unsigned i = c % op.nx;
        const unsigned j = (c / op.nx) % op.ny;
        const unsigned k = c / S;
        const double ac = (double)a.alpha[c];
        const Real mc = mu[c], tc = T[c];
        double s = 0.0;
        unsigned qn;
        // +x / -x
        if (i + 1 < (unsigned)op.nx || op.px) {
            qn = (i + 1 < (unsigned)op.nx) ? c + 1 : c - (op.nx - 1);
            s += face_term(a.wx, ac, (double)a.alpha[qn], (Real)(mc - mu[qn]), (Real)(tc - T[qn]));
        }
        if (i > 0 || op.px) {
            qn = (i > 0) ? c - 1 : c + op.nx - 1;
            s += face_term(a.wx, ac, (double)a.alpha[qn], (Real)(mc - mu[qn]), (Real)(tc - T[qn]));
        }
        if (j + 1 < (unsigned)op.ny || op.py) {
            qn = (j + 1 < (unsigned)op.ny) ? c + row : c - (op.ny - 1) * row;
            s += face_term(a.wy, ac, (double)a.alpha[qn], (Real)(mc - mu[qn]), (Real)(tc - T[qn]));
        }
        if (j > 0 || op.py) {
            qn = (j > 0) ? c - row : c + (op.ny - 1) * row;
            s += face_term(a.wy, ac, (double)a.alpha[qn], (Real)(mc - mu[qn]), (Real)(tc - T[qn]));
        }
        if (k + 1 < (unsigned)op.nz) {
            qn = c + S;
            s += face_term(a.wz, ac, (double)a.alpha[qn], (Real)(mc - mu[qn]), (Real)(tc - T[qn]));
        }
        if (k > 0) {
            qn = c - S;
            s += face_term(a.wz, ac, (double)a.alpha[qn], (Real)(mc - mu[qn]), (Real)(tc - T[qn]));
        }
        a.grad[c] -= s;
    }
}

template <typename Real>
__global__ void __launch_bounds__(kThreads) adjoint_kernel(AdjArgs<Real> a) {
    Grid g = make_grid(a.ctl, a.partials);
    const OperatorView<Real>& op = a.op;
    const unsigned N = op.N, S = op.S;
    const unsigned stride = gridDim.x * kThreads;
    const unsigned c0 = blockIdx.x * kThreads + threadIdx.x;
    const Real gs = (Real)a.g_scale;
    for (int n = a.n1; n > a.n0; --n) {
        const Real* __restrict__ Tn = a.T[n - a.n0];
        const Real* __restrict__ mnext = a.mu[(n + 1) & 1];
        Real* __restrict__ x = a.mu[n & 1];
        const Real* ob = a.obs + (size_t)(n - 1) * S;
        // b = mu^{n+1} + 2 s Pi^T (Pi T^n - obs^n); x0 = mu^{n+1}
        double s3[3] = {0.0, 0.0, 0.0};
        for (unsigned c = c0; c < N; c += stride) {
            const Real m = mnext[c];
            const Real inj = (c >= a.obs_off && c < a.obs_off + S) ? gs * (Tn[c] - ob[c - a.obs_off]) : Real(0);
            const Real b = m + inj;
            const Real rc = inj - apply_AmI(op, mnext, c);
            const Real zc = op.dinv[c] * rc;
            x[c] = Real(0);
            a.r[c] = rc;
            a.p[c] = zc;
            s3[0] += (double)rc * (double)zc;
            s3[1] += (double)rc * (double)rc;
            s3[2] += (double)b * (double)b;
        }
        if (!grid_sum<3>(g, s3)) return;
        int it = 0;
        double rel = 0.0;
        if (a.jacobi_k > 0) {
            if (!jacobi_iterate(g, op, x, a.r, a.p, a.q, a.jacobi_k)) return;
            it = a.jacobi_k;
        } else if (!cg_iterate(g, op, x, a.r, a.p, a.q, s3[0], s3[1], s3[2], a.tol2, a.max_iter, &it, &rel)) {
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.iters[a.n1 - n] = it;
            a.resid[a.n1 - n] = rel;
            if (a.jacobi_k == 0 && it >= a.max_iter && rel * rel > a.tol2) atomicAdd(&a.ctl->notconv, 1);
        }
        // mu^n = mu^{n+1} + delta (increment accumulated on its own, as forward)
        for (unsigned c = c0; c < N; c += stride) x[c] = mnext[c] + x[c];
        if (!grid_sync(g)) return;
        // The barrier made every CTA's mu^n visible; the gradient reads mu^n and
        // T^n only, and the next step writes mu^{n-1} (the buffer of mu^{n+1}),
        // so no further barrier is needed here.
        accumulate_gradient(a, x, Tn);
    }
}

// ------------------------------------------------------------ coefficients
// dt * a of the +x, +y, +z face of every cell, the diagonal d of A and 1/d.
// alpha must be > 0 and finite; otherwise ctl->err = kDevBadAlpha.
template <typename Real>
__global__ void coeff_kernel(const Real* __restrict__ alpha, int nx, int ny, int nz, int px, int py,
                             double kx, double ky, double kz, double robin, Real* cx, Real* cy,
                             Real* cz, Real* d, Real* dinv, DevCtl* ctl) {
    const unsigned S = (unsigned)nx * ny, N = S * nz;
    const unsigned row = (unsigned)nx;
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const unsigned i = c % nx, j = (c / nx) % ny, k = c / S;
        const double ac = (double)alpha[c];
        if (!(ac > 0.0) || !isfinite(ac)) atomicCAS(&ctl->err, kDevOk, kDevBadAlpha);
        auto face = [&](unsigned q, double kk) {
            const double aq = (double)alpha[q];
            return (Real)(kk * (2.0 * ac * aq / (ac + aq)));
        };
        // Each face value is computed from the same two alphas by both cells
        // that share it, and rounded the same way, so A stays symmetric.
        Real fxp = 0, fxm = 0, fyp = 0, fym = 0, fzp = 0, fzm = 0;
        if (i + 1 < (unsigned)nx) fxp = face(c + 1, kx); else if (px) fxp = face(c - (nx - 1), kx);
        if (i > 0) fxm = face(c - 1, kx); else if (px) fxm = face(c + nx - 1, kx);
        if (j + 1 < (unsigned)ny) fyp = face(c + row, ky); else if (py) fyp = face(c - (ny - 1) * row, ky);
        if (j > 0) fym = face(c - row, ky); else if (py) fym = face(c + (ny - 1) * row, ky);
        if (k + 1 < (unsigned)nz) fzp = face(c + S, kz);
        if (k > 0) fzm = face(c - S, kz);
        const double dd = 1.0 + (double)fxp + (double)fxm + (double)fyp + (double)fym + (double)fzp +
                          (double)fzm + (k + 1 == (unsigned)nz ? robin : 0.0);
        cx[c] = fxp;
        cy[c] = fyp;
        cz[c] = fzp;
        d[c] = (Real)dd;
        dinv[c] = (Real)(1.0 / dd);
    }
}

template <typename Real>
__global__ void cast_kernel(const double* __restrict__ in, Real* __restrict__ out, unsigned n) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (Real)in[i];
}

// ------------------------------------------------------------------ launch
int solver_grid_blocks(int device, int prec) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
    int per_sm = 0;
    cudaError_t e = prec == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, forward_kernel<float>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, forward_kernel<double>, kThreads, 0);
    if (e != cudaSuccess) return 0;
    int per_sm_adj = 0;
    e = prec == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_adj, adjoint_kernel<float>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_adj, adjoint_kernel<double>, kThreads, 0);
    if (e != cudaSuccess) return 0;
    per_sm = per_sm < per_sm_adj ? per_sm : per_sm_adj;
    if (per_sm > 2) per_sm = 2;
    return per_sm * prop.multiProcessorCount;
}

template <typename Real>
cudaError_t launch_coefficients(const Real* alpha, int nx, int ny, int nz, int bc, double dx,
                                double dy, double dz, double dt, double robin_h, Real* cx,
                                Real* cy, Real* cz, Real* d, Real* dinv, DevCtl* ctl,
                                cudaStream_t s) {
    const unsigned N = (unsigned)nx * ny * nz;
    const int px = bc == 1 && nx > 1, py = bc == 1 && ny > 1;
    unsigned blocks = (N + 255) / 256;
    if (blocks > 65535u * 8u) blocks = 65535u * 8u;
    coeff_kernel<Real><<<blocks, 256, 0, s>>>(alpha, nx, ny, nz, px, py, dt / (dx * dx),
                                              dt / (dy * dy), dt / (dz * dz), dt * robin_h / dz,
                                              cx, cy, cz, d, dinv, ctl);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_forward(const FwdArgs<Real>& a, int grid, cudaStream_t s) {
    FwdArgs<Real> copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)forward_kernel<Real>, dim3(grid), dim3(kThreads),
                                       args, 0, s);
}

template <typename Real>
cudaError_t launch_adjoint(const AdjArgs<Real>& a, int grid, cudaStream_t s) {
    AdjArgs<Real> copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)adjoint_kernel<Real>, dim3(grid), dim3(kThreads),
                                       args, 0, s);
}

template <typename Real>
cudaError_t launch_cast(const double* in, Real* out, unsigned n, cudaStream_t s) {
    unsigned blocks = (n + 255) / 256;
    if (blocks > 65535u * 8u) blocks = 65535u * 8u;
    if (blocks == 0) return cudaSuccess;
    cast_kernel<Real><<<blocks, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

#define NEFTY_INSTANTIATE(R)                                                                     \
    template cudaError_t launch_coefficients<R>(const R*, int, int, int, int, double, double,    \
                                                double, double, double, R*, R*, R*, R*, R*,      \
                                                DevCtl*, cudaStream_t);                          \
    template cudaError_t launch_forward<R>(const FwdArgs<R>&, int, cudaStream_t);                \
    template cudaError_t launch_adjoint<R>(const AdjArgs<R>&, int, cudaStream_t);                \
    template cudaError_t launch_cast<R>(const double*, R*, unsigned, cudaStream_t);
NEFTY_INSTANTIATE(float)
NEFTY_INSTANTIATE(double)
#undef NEFTY_INSTANTIATE

}  // namespace nefty
