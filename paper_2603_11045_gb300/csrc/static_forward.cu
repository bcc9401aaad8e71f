// nefty_forward_static: the forward sweep for callers that cannot allocate
// device memory.
//
// nefty_forward draws its scratch from a handle that grows with cudaMalloc.
// Some callers cannot let that happen when they need a solve: a serving or
// real-time loop that has already reserved the whole device for its own
// buffers (there is nothing left to allocate), a loop that cannot take the
// device-wide synchronisation that cudaMalloc and cudaFree may imply, or a
// host application or plug-in framework that hands out device memory only
// from its own pool and forbids the library to call the CUDA allocator.
// This entry point takes every input and output from the caller and keeps all
// of its scratch (operator coefficients, CG vectors, two state buffers, the
// grid-barrier control word, reduction partials and per-step tables) in one
// file-scope device array of kStaticScratchBytes.  The array exists on every
// GPU that loads the library and is held until the process exits.
//
// The persistent PCG forward kernel and the coefficient kernel are the ones
// nefty_forward launches for FP64 problems (solver.cu); only where their scratch
// lives differs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "nefty.h"

namespace nefty {
namespace {

constexpr size_t kStaticScratchBytes = 48ull << 20;   // 48 MiB per device
constexpr int kStaticMaxSteps = 65536;
constexpr int kStaticMaxBlocks = 1024;
constexpr int kStaticMaxDevices = 64;

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_dev[kStaticMaxDevices] = {};   // device address of g_scratch per device
int g_grid[kStaticMaxDevices][2] = {};

// Step tables: step n reads src[n] and writes dst[n]; states alternate
// between the two work buffers, step 0 reads t0.
template <typename Real>
__global__ void static_tables_kernel(Real** src, Real** dst, const Real* t0, Real* w0, Real* w1, int nt) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nt; n += gridDim.x * blockDim.x) {
        src[n] = n == 0 ? const_cast<Real*>(t0) : ((n - 1) & 1 ? w1 : w0);
        dst[n] = (n & 1) ? w1 : w0;
    }
}

// True when the kernels on `dev` may read p in place: NULL, device memory of
// `dev` itself or managed memory.  Host memory and device memory of another
// GPU are refused (no staging buffer can be allocated here).
bool on_device(const void* p, int dev) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

nefty_status fail(nefty_status s, const std::string& m) {
    set_thread_error(m);
    return s;
}

// First call on a device (with that device current): resolve the device
// address of g_scratch.  In host code the symbol itself is only a host-side
// stand-in, never a device address.
nefty_status setup(int dev, void** ptr) {
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(NEFTY_EINVAL, "device index beyond the static table");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(NEFTY_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorName(e));
        g_scratch_dev[dev] = p;
        g_grid[dev][0] = solver_grid_blocks(dev, 0);
        g_grid[dev][1] = solver_grid_blocks(dev, 1);
    }
    *ptr = g_scratch_dev[dev];
    return NEFTY_OK;
}

template <typename Real>
nefty_status run(int dev, char* base, const nefty_problem& p, const void* alpha, const void* T0,
                  const void* q_face, int32_t q_steps, void* frames_out, void* T_final, const void* obs,
                  double* loss_out, cudaStream_t s) {
    const size_t N = (size_t)p.nx * p.ny * p.nz, S = (size_t)p.nx * p.ny, nt = (size_t)p.nt, R = sizeof(Real);
    int G = g_grid[dev][p.prec];
    if (G <= 0) return fail(NEFTY_ECUDA, "cannot size the persistent solver grid on this device");
    long want = ((long)N + (long)kThreads * 4 - 1) / ((long)kThreads * 4);
    if (want < 1) want = 1;
    if (want < G) G = (int)want;
    if (G > kStaticMaxBlocks) G = kStaticMaxBlocks;
    // carve the scratch: fixed part first, then 10 values per cell
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        char* q = base + off;
        off += bytes;
        return q;
    };
    DevCtl* ctl = (DevCtl*)take(sizeof(DevCtl));
    double* partials = (double*)take(2 * kMaxRed * (size_t)kStaticMaxBlocks * sizeof(double));
    double* loss_part = (double*)take((size_t)kStaticMaxBlocks * sizeof(double));
    int* iters = (int*)take((size_t)kStaticMaxSteps * sizeof(int));
    double* resid = (double*)take((size_t)kStaticMaxSteps * sizeof(double));
    Real** tab = (Real**)take(2 * (size_t)kStaticMaxSteps * sizeof(Real*));
    Real* coef = (Real*)take(5 * N * R);
    Real* r = (Real*)take(N * R);
    Real* pv = (Real*)take(N * R);
    Real* qv = (Real*)take(N * R);
    Real* w0 = (Real*)take(N * R);
    Real* w1 = (Real*)take(N * R);
    if (off > kStaticScratchBytes) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "problem needs %zu bytes of scratch; the no-allocation forward holds %zu "
                 "(10 values per cell plus fixed tables)",
                 off, kStaticScratchBytes);
        return fail(NEFTY_EINVAL, buf);
    }
#define NS_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) return fail(NEFTY_ECUDA, std::string(#expr ": ") + cudaGetErrorName(e_)); \
    } while (0)
    NS_CUDA(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
    NS_CUDA(launch_coefficients<Real>((const Real*)alpha, p.nx, p.ny, p.nz, p.bc, p.dx, p.dy, p.dz, p.dt,
                                      p.robin_h, coef, coef + N, coef + 2 * N, coef + 3 * N, coef + 4 * N, ctl, s));
    DevCtl hc;
    NS_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, s));
    NS_CUDA(cudaStreamSynchronize(s));
    if (hc.err == kDevBadAlpha) return fail(NEFTY_EINVAL, "alpha must be > 0 and finite in every cell");
    const Real* t0 = (const Real*)T0;
    if (!t0) {   // zero initial state in the buffer step 0 reads
        NS_CUDA(cudaMemsetAsync(w1, 0, N * R, s));
        t0 = w1;
    }
    static_tables_kernel<Real><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(tab, tab + nt, t0, w0, w1, (int)nt);
    NS_CUDA(cudaGetLastError());
    FwdArgs<Real> a{};
    a.op.nx = p.nx; a.op.ny = p.ny; a.op.nz = p.nz;
    a.op.px = p.bc == NEFTY_BC_PERIODIC_XY && p.nx > 1;
    a.op.py = p.bc == NEFTY_BC_PERIODIC_XY && p.ny > 1;
    a.op.N = (unsigned)N; a.op.S = (unsigned)S;
    a.op.cx = coef; a.op.cy = coef + N; a.op.cz = coef + 2 * N; a.op.d = coef + 3 * N; a.op.dinv = coef + 4 * N;
    a.op.robin = (Real)(p.dt * p.robin_h / p.dz);
    a.r = r; a.p = pv; a.q = qv;
    a.n0 = 0; a.n1 = p.nt;
    a.src = tab; a.dst = tab + nt;
    a.q_face = (const Real*)q_face;
    a.q_steps = q_face ? q_steps : 0;
    a.q_full = nullptr;
    a.src_scale = p.dt / p.dz;
    a.obs_off = p.obs_face ? (unsigned)(p.nz - 1) * (unsigned)S : 0u;
    a.obs = loss_out ? (const Real*)obs : nullptr;
    a.frames = (Real*)frames_out;
    const double rtol = p.rtol > 0 ? p.rtol : (p.prec == NEFTY_FP32 ? kDefaultRtolFp32 : kDefaultRtolFp64);
    a.tol2 = rtol * rtol;
    a.max_iter = p.max_iter > 0 ? p.max_iter : kDefaultMaxIter;
    a.ctl = ctl;
    a.partials = partials;
    a.iters = iters;
    a.resid = resid;
    a.loss_partials = loss_part;
    NS_CUDA(launch_forward<Real>(a, G, s));
    if (T_final) NS_CUDA(cudaMemcpyAsync(T_final, ((nt - 1) & 1) ? w1 : w0, N * R, cudaMemcpyDeviceToDevice, s));
    NS_CUDA(cudaStreamSynchronize(s));
    NS_CUDA(cudaMemcpy(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost));
    if (hc.err == kDevTimeout) return fail(NEFTY_ETIMEOUT, "a grid barrier of the persistent solver timed out");
    if (loss_out) {
        std::vector<double> lp(G);
        NS_CUDA(cudaMemcpy(lp.data(), loss_part, G * sizeof(double), cudaMemcpyDeviceToHost));
        double t = 0.0;
        for (int b = 0; b < G; ++b) t += lp[b];
        *loss_out = (p.loss_scale > 0 ? p.loss_scale : 1.0 / ((double)p.nt * p.nx * p.ny)) * t;
    }
    if (hc.notconv > 0) return fail(NEFTY_ENOTCONV, "a CG solve reached max_iter");
#undef NS_CUDA
    return NEFTY_OK;
}

}  // namespace
}  // namespace nefty

extern "C" nefty_status nefty_forward_static(int device, const nefty_problem* p, const void* alpha,
                                             const void* T0, const void* q_face, int32_t q_steps,
                                             void* frames_out, void* T_final, const void* obs,
                                             double* loss_out, void* stream) {
    using namespace nefty;
    if (nefty_problem_check(p) != NEFTY_OK) return NEFTY_EINVAL;   // message already set
    if (p->jacobi_k != 0) return fail(NEFTY_EINVAL, "jacobi_k is not supported by the no-allocation entry point");
    if (!alpha) return fail(NEFTY_EINVAL, "alpha is NULL");
    if (loss_out && !obs) return fail(NEFTY_EINVAL, "loss_out needs obs");
    if (q_steps < 0) return fail(NEFTY_EINVAL, "q_steps must be >= 0");
    if (p->nt > kStaticMaxSteps) return fail(NEFTY_EINVAL, "nt exceeds the no-allocation limit of 65536 steps");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        prev = -1;
    }
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return fail(NEFTY_ECUDA, "cannot make the requested device current");
    }
    nefty_status st = NEFTY_OK;
    void* base = nullptr;
    if (!on_device(alpha, device) || !on_device(T0, device) || !on_device(q_face, device) ||
        !on_device(frames_out, device) || !on_device(T_final, device) || !on_device(obs, device)) {
        st = fail(NEFTY_EINVAL,
                  "every array must be device memory of the requested device (host arrays would need staging "
                  "buffers)");
    } else if ((st = setup(device, &base)) == NEFTY_OK) {
        cudaStream_t s = (cudaStream_t)stream;
        st = p->prec == NEFTY_FP32
                 ? run<float>(device, (char*)base, *p, alpha, T0, q_face, q_steps, frames_out, T_final, obs, loss_out, s)
                 : run<double>(device, (char*)base, *p, alpha, T0, q_face, q_steps, frames_out, T_final, obs, loss_out,
                               s);
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
