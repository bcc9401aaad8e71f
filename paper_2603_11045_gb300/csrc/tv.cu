// Discrete isotropic total variation of the diffusivity field (Eq. tv_discrete)
// and its gradient.
//
//   R(alpha) = dx dy dz * sum_cells sqrt((dx_a/dx)^2 + (dy_a/dy)^2 + (dz_a/dz)^2 + eps^2)
//
// with forward differences: the lateral ones wrap when the lateral walls are
// periodic and vanish on the last column/row otherwise; the z difference
// vanishes on the last slice.  The gradient is gathered, not scattered: cell c
// takes the derivative of its own term and of the terms of its -x, -y, -z
// neighbours (the only other terms whose differences contain alpha_c), so each
// thread writes only its own cell and no atomics are needed.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace nefty {
namespace {

constexpr int kTvThreads = 256;

template <typename Real>
struct TvGeo {
    int nx, ny, nz, px, py;
    unsigned S, N;
    Real ix, iy, iz, eps2;   // 1/dx, 1/dy, 1/dz, eps^2
};

// Forward differences (scaled by 1/h) of the term of cell (i, j, k); returns
// false for a cell outside the grid.
template <typename Real>
__device__ __forceinline__ bool term_diffs(const TvGeo<Real>& g, const Real* __restrict__ a, int i, int j, int k,
                                           Real& gx, Real& gy, Real& gz) {
    if (i < 0 || j < 0 || k < 0) return false;
    const unsigned c = (unsigned)k * g.S + (unsigned)j * g.nx + i;
    const Real ac = a[c];
    gx = Real(0);
    gy = Real(0);
    gz = Real(0);
    if (i + 1 < g.nx) gx = (a[c + 1] - ac) * g.ix;
    else if (g.px) gx = (a[c + 1 - g.nx] - ac) * g.ix;
    if (j + 1 < g.ny) gy = (a[c + g.nx] - ac) * g.iy;
    else if (g.py) gy = (a[c - (unsigned)(g.ny - 1) * g.nx] - ac) * g.iy;
    if (k + 1 < g.nz) gz = (a[c + g.S] - ac) * g.iz;
    return true;
}

template <typename Real>
__global__ void __launch_bounds__(kTvThreads) tv_kernel(TvGeo<Real> g, const Real* __restrict__ a, Real lamV,
                                                        Real* grad, double* partials) {
    double acc = 0.0;
    for (unsigned c = blockIdx.x * kTvThreads + threadIdx.x; c < g.N; c += gridDim.x * kTvThreads) {
        const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.S);
        Real gx, gy, gz;
        term_diffs(g, a, i, j, k, gx, gy, gz);
        const Real t = sqrt(gx * gx + gy * gy + gz * gz + g.eps2);
        acc += (double)t;
        if (!grad) continue;
        // d t_c / d alpha_c
        Real d = -(gx * g.ix + gy * g.iy + gz * g.iz) / t;
        // terms of the -x, -y, -z neighbours, whose forward differences end at c
        const int im = i > 0 ? i - 1 : (g.px ? g.nx - 1 : -1);
        const int jm = j > 0 ? j - 1 : (g.py ? g.ny - 1 : -1);
        Real hx, hy, hz;
        if (term_diffs(g, a, im, j, k, hx, hy, hz)) d += hx * g.ix / sqrt(hx * hx + hy * hy + hz * hz + g.eps2);
        if (term_diffs(g, a, i, jm, k, hx, hy, hz)) d += hy * g.iy / sqrt(hx * hx + hy * hy + hz * hz + g.eps2);
        if (term_diffs(g, a, i, j, k - 1, hx, hy, hz)) d += hz * g.iz / sqrt(hx * hx + hy * hy + hz * hz + g.eps2);
        grad[c] += lamV * d;
    }
    __shared__ double s[kTvThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kTvThreads / 32; ++w) t += s[w];
        partials[blockIdx.x] = t;
    }
}

}  // namespace

int tv_blocks(unsigned N) {
    unsigned b = (N + kTvThreads * 4 - 1) / (kTvThreads * 4);
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

template <typename Real>
cudaError_t launch_tv(const Real* alpha, int nx, int ny, int nz, int bc, double dx, double dy, double dz,
                      double lam, double eps, Real* grad_accum, double* partials, int blocks, cudaStream_t s) {
    TvGeo<Real> g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.px = bc == 1 && nx > 1;
    g.py = bc == 1 && ny > 1;
    g.S = (unsigned)nx * ny;
    g.N = g.S * nz;
    g.ix = (Real)(1.0 / dx); g.iy = (Real)(1.0 / dy); g.iz = (Real)(1.0 / dz);
    g.eps2 = (Real)(eps * eps);
    tv_kernel<Real><<<blocks, kTvThreads, 0, s>>>(g, alpha, (Real)(lam * dx * dy * dz), grad_accum, partials);
    return cudaGetLastError();
}

template cudaError_t launch_tv<float>(const float*, int, int, int, int, double, double, double, double, double,
                                      float*, double*, int, cudaStream_t);
template cudaError_t launch_tv<double>(const double*, int, int, int, int, double, double, double, double, double,
                                       double*, double*, int, cudaStream_t);

}  // namespace nefty
