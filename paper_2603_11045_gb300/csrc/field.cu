// Neural diffusivity field (Sec. 4.1, App. D.1): Fourier features of the cell
// centres -> ReLU MLP -> bounded output, evaluated at every cell, and its
// backward pass to the parameters.  Dense layers run on tcgen05 (umma_gemm.cu)
// in BF16 with FP32 accumulation; everything else is FP32.
//
// Encoding: centre coordinates x_d = 2 (i + 1/2) / N_d - 1 in (-1, 1); F bands
// per axis with log-spaced frequencies w_b = freq_lo * (freq_hi/freq_lo)^(b/(F-1));
// band b of axis d contributes (wt_b sin(w_b x_d), wt_b cos(w_b x_d)) at feature
// indices d*2F + 2b and d*2F + 2b + 1, wt_b being the band's annealing weight
// (Eq. fa_schedule; 1 when none is given).  The encoding is separable, so it is
// tabulated per axis once and assembled per cell.
//
// Network: h_0 = gamma(x) (6F), h_{l+1} = relu(W_l h_l + b_l) for l < depth
// (width W), f = w_out . h_depth + b_out, alpha = alpha_min +
// (alpha_max - alpha_min) * sigmoid(f) (Eq. bracket).  With a skip layer s
// (App. D.1: the encoding re-injected at the middle layer), layer s reads
// [h_s | gamma(x)] (W + 6F inputs).
//
// Parameter vector theta (FP32, packed): W_0 [W x 6F], b_0 [W], then for
// l = 1 .. depth-1: W_l [W x in_l], b_l [W] (in_l = W + 6F for l = s, else W);
// then w_out [W], b_out [1].  Weights are row-major [out][in].
//
// Storage: the feature block is zero-padded to Dp = 6F rounded up to 64 columns
// (the tensor-core K step), so every GEMM has K a multiple of 64 for any F; the
// BF16 weight copies carry the matching zero columns, and the layer-s input
// buffer holds h_s and the padded features side by side.
//
// Split BF16 (ns = 3, nefty_field_desc.precision = 1): every operand value v
// is kept as hi = bf16(v) and lo = bf16(v - hi), about 16 significant bits,
// and every product X Y^T runs as ONE tensor-core GEMM over a tripled K,
// [Xh | Xh | Xl] [Yh | Yl | Yh]^T = Xh Yh^T + Xh Yl^T + Xl Yh^T (the dropped
// Xl Yl^T is below the FP32 accumulation's rounding).  A-side operands
// (activations, deltas and their transposes as A) are stored in the order
// [hi | hi | lo], B-side operands (weights, activation transposes as B) in
// the order [hi | lo | hi], each block as wide as the plain operand.  With
// ns = 1 every buffer is the plain BF16 one.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace nefty {
namespace {

constexpr int kT = 256;

// tab[i][2b + {0,1}] for cell index i along one axis.  The phase w_b x_i
// reaches thousands of radians for the paper's top band (2^11 pi), where a
// single-precision product or frequency would already be off by about 1e-3
// rad, so the n F table entries are formed in double and rounded once.
__global__ void axis_table_kernel(float* tab, int n, int F, double lo, double ratio_log, const float* band_w) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * F; e += gridDim.x * blockDim.x) {
        const int i = e / F, b = e % F;
        const double x = 2.0 * ((double)i + 0.5) / (double)n - 1.0;
        const double w = F > 1 ? lo * exp(ratio_log * (double)b / (double)(F - 1)) : lo;
        const double wt = band_w ? (double)band_w[b] : 1.0;
        tab[(size_t)i * 2 * F + 2 * b] = (float)(wt * sin(w * x));
        tab[(size_t)i * 2 * F + 2 * b + 1] = (float)(wt * cos(w * x));
    }
}

// h0[c][d*2F + j] = tab_d[index_d(c)][j], as BF16, rows padded to Mp and
// columns to Dp (zeros); rows of ns * Dp values, the split blocks [hi | hi | lo]
// at offsets 0, Dp, 2 Dp when ns = 3.  With F % 4 == 0 each thread writes 8
// features (16 bytes) of one cell per block, which never straddle two axes;
// otherwise one feature at a time.
__global__ void features_kernel(__nv_bfloat16* h0, unsigned M, unsigned Mp, int nx, int ny, int F, int Dp, int ns,
                                const float* tx, const float* ty, const float* tz) {
    const int D = 6 * F, F2 = 2 * F;
    const size_t ld = (size_t)ns * Dp;
    if ((F & 3) == 0) {
        const unsigned per = (unsigned)Dp / 8;   // 16-byte chunks per cell
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)Mp * per;
             e += (size_t)gridDim.x * blockDim.x) {
            const unsigned c = (unsigned)(e / per);
            const int f = (int)(e - (size_t)c * per) * 8;
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (c < M && f < D) {
                const unsigned cy = c / (unsigned)nx, i = c - cy * (unsigned)nx;
                const unsigned k = cy / (unsigned)ny, j = cy - k * (unsigned)ny;
                const int d = f / F2, r = f - d * F2;
                const float* row = d == 0 ? tx + (size_t)i * F2 : (d == 1 ? ty + (size_t)j * F2 : tz + (size_t)k * F2);
                const float4 p = *reinterpret_cast<const float4*>(row + r);
                const float4 q = *reinterpret_cast<const float4*>(row + r + 4);
                v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
            }
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * t], v[2 * t + 1]);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * t] - __low2float(h2), v[2 * t + 1] - __high2float(h2));
                hi[t] = *reinterpret_cast<const uint32_t*>(&h2);
                lo[t] = *reinterpret_cast<const uint32_t*>(&l2);
            }
            __nv_bfloat16* out = h0 + (size_t)c * ld + f;
            *reinterpret_cast<uint4*>(out) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            if (ns == 3) {
                *reinterpret_cast<uint4*>(out + Dp) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(out + 2 * Dp) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
        return;
    }
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)Mp * Dp;
         e += (size_t)gridDim.x * blockDim.x) {
        const unsigned c = (unsigned)(e / Dp);
        const int f = (int)(e % Dp);
        float v = 0.f;
        if (c < M && f < D) {
            const unsigned i = c % nx, j = (c / nx) % ny, k = c / ((unsigned)nx * ny);
            const int d = f / F2, r = f % F2;
            v = d == 0 ? tx[(size_t)i * F2 + r] : (d == 1 ? ty[(size_t)j * F2 + r] : tz[(size_t)k * F2 + r]);
        }
        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
        __nv_bfloat16* out = h0 + (size_t)c * ld + f;
        out[0] = hv;
        if (ns == 3) {
            out[Dp] = hv;
            out[2 * Dp] = __float2bfloat16_rn(v - __bfloat162float(hv));
        }
    }
}

// h_0^T [Dp x ns Mp] straight from the axis tables, as the B side of the
// first layer's weight-gradient product: row f holds feature f of every cell,
// the split blocks in B-side order [hi | lo | hi] at column offsets 0, Mp,
// 2 Mp (zeros for padded cells and features).  The same BF16 values as
// features_kernel writes, transposed; each thread writes 8 consecutive cells
// (16 bytes per block; Mp is a multiple of 128).
__global__ void features_t_kernel(__nv_bfloat16* hT, unsigned M, unsigned Mp, int nx, int ny, int F, int Dp, int ns,
                                  const float* tx, const float* ty, const float* tz) {
    const int D = 6 * F, F2 = 2 * F;
    const unsigned per = Mp / 8;   // 8-cell chunks per feature row
    const size_t ldt = (size_t)ns * Mp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)Dp * per;
         e += (size_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / per);
        const unsigned c0 = (unsigned)(e - (size_t)f * per) * 8;
        float v[8];
        const int d = f / F2, r = f - d * F2;
        unsigned cy = c0 / (unsigned)nx, i = c0 - cy * (unsigned)nx;
        unsigned k = cy / (unsigned)ny, j = cy - k * (unsigned)ny;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const unsigned c = c0 + t;
            float x = 0.f;
            if (c < M && f < D)
                x = d == 0 ? tx[(size_t)i * F2 + r] : (d == 1 ? ty[(size_t)j * F2 + r] : tz[(size_t)k * F2 + r]);
            v[t] = x;
            if (++i == (unsigned)nx) {
                i = 0;
                if (++j == (unsigned)ny) { j = 0; ++k; }
            }
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * t], v[2 * t + 1]);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * t] - __low2float(h2), v[2 * t + 1] - __high2float(h2));
            hi[t] = *reinterpret_cast<const uint32_t*>(&h2);
            lo[t] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        __nv_bfloat16* out = hT + (size_t)f * ldt + c0;
        *reinterpret_cast<uint4*>(out) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if (ns == 3) {
            *reinterpret_cast<uint4*>(out + Mp) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            *reinterpret_cast<uint4*>(out + 2 * (size_t)Mp) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        }
    }
}

// dst [R x Cp] = bf16(src [R x C]) with zero columns C .. Cp-1; with ns = 3
// rows of 3 Cp values, the split blocks in B-side order [hi | lo | hi].
__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, int R, int C, int Cp, int ns) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)R * Cp;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Cp), c = (int)(e % Cp);
        const float v = c < C ? src[(size_t)r * C + c] : 0.f;
        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
        __nv_bfloat16* out = dst + (size_t)r * ns * Cp + c;
        out[0] = hv;
        if (ns == 3) {
            out[Cp] = __float2bfloat16_rn(v - __bfloat162float(hv));
            out[2 * Cp] = hv;
        }
    }
}

// dst [Cp x R] = bf16(src [R x C])^T with zero rows C .. Cp-1; with ns = 3
// rows of 3 R values in B-side order [hi | lo | hi].
__global__ void transpose_f32_bf16_kernel(const float* src, __nv_bfloat16* dst, int R, int C, int Cp, int ns) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)R * Cp;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / R), r = (int)(e % R);
        const float v = c < C ? src[(size_t)r * C + c] : 0.f;
        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
        __nv_bfloat16* out = dst + (size_t)c * ns * R + r;
        out[0] = hv;
        if (ns == 3) {
            out[R] = __float2bfloat16_rn(v - __bfloat162float(hv));
            out[2 * R] = hv;
        }
    }
}

// dst[m][col0 + j] = src[m][j] for j < n, rows of lds / ldd elements (BF16);
// n, col0, lds, ldd are multiples of 8, so each thread moves 16 bytes.
__global__ void copy_cols_kernel(const __nv_bfloat16* src, int lds, __nv_bfloat16* dst, int ldd, int col0, int n,
                                 unsigned rows) {
    const unsigned per = (unsigned)n / 8;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)rows * per;
         e += (size_t)gridDim.x * blockDim.x) {
        const unsigned m = (unsigned)(e / per), j = (unsigned)(e % per) * 8;
        *reinterpret_cast<uint4*>(dst + (size_t)m * ldd + col0 + j) =
            *reinterpret_cast<const uint4*>(src + (size_t)m * lds + j);
    }
}

// dst[c][r] = src[r][c] for a BF16 [R x C] matrix (R rows = points, row
// pitch lds), into rows of pitch ldd; tiled.
__global__ void transpose_bf16_kernel(const __nv_bfloat16* src, size_t lds, __nv_bfloat16* dst, size_t ldd,
                                      unsigned R, int C) {
    __shared__ __nv_bfloat16 t[32][33];
    const unsigned r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const unsigned r = r0 + yy, c = c0 + threadIdx.x;
        t[yy][threadIdx.x] = (r < R && c < (unsigned)C) ? src[(size_t)r * lds + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const unsigned c = c0 + yy, r = r0 + threadIdx.x;
        if (c < (unsigned)C && r < R) dst[(size_t)c * ldd + r] = t[threadIdx.x][yy];
    }
}

// h[m][j] as stored: the BF16 value, or hi + lo of a split row (lo block at
// column offset lo_off, 0 = plain).
__device__ __forceinline__ float hval(const __nv_bfloat16* h, size_t ld, int lo_off, unsigned m, int j) {
    const float v = __bfloat162float(h[(size_t)m * ld + j]);
    return lo_off ? v + __bfloat162float(h[(size_t)m * ld + lo_off + j]) : v;
}

// Output head: f = w_out . h + b_out, alpha = lo + (hi - lo) sigmoid(f).
__global__ void head_kernel(const __nv_bfloat16* h, size_t ld, int lo_off, int W, const float* w_out,
                            const float* b_out, unsigned M, float a_lo, float a_hi, float* alpha) {
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned m = warp; m < M; m += nwarps) {
        float s = 0.f;
        for (int j = lane; j < W; j += 32) s += hval(h, ld, lo_off, m, j) * w_out[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const float f = s + b_out[0];
            alpha[m] = a_lo + (a_hi - a_lo) / (1.f + expf(-f));
        }
    }
}

// Backward of the head: g_f = g_alpha (hi - lo) sig (1 - sig);
// delta[m][j] = bf16(g_f w_out[j] [h[m][j] > 0]) (split: [hi | hi | lo] blocks
// of W columns, rows of ns W); gf[m] kept for dw_out, db_out.
__global__ void head_back_kernel(const __nv_bfloat16* h, size_t ld, int lo_off, int W, const float* w_out,
                                 const float* b_out, unsigned M, unsigned Mp, float a_lo, float a_hi,
                                 const float* g_alpha, float* gf, __nv_bfloat16* delta, int ns) {
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const size_t ldd = (size_t)ns * W;
    for (unsigned m = warp; m < Mp; m += nwarps) {
        float g = 0.f;
        if (m < M) {
            float s = 0.f;
            for (int j = lane; j < W; j += 32) s += hval(h, ld, lo_off, m, j) * w_out[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const float sg = 1.f / (1.f + expf(-(s + b_out[0])));
            g = g_alpha[m] * (a_hi - a_lo) * sg * (1.f - sg);
        }
        if (lane == 0) gf[m] = g;
        for (int j = lane; j < W; j += 32) {
            const float hv = __bfloat162float(h[(size_t)m * ld + j]);
            const float v = hv > 0.f ? g * w_out[j] : 0.f;
            const __nv_bfloat16 dh = __float2bfloat16_rn(v);
            delta[(size_t)m * ldd + j] = dh;
            if (ns == 3) {
                delta[(size_t)m * ldd + W + j] = dh;
                delta[(size_t)m * ldd + 2 * W + j] = __float2bfloat16_rn(v - __bfloat162float(dh));
            }
        }
    }
}

// out[j] = sum_m A[m][j] * (v ? v[m] : 1) over rows, in fixed order:
// per-block partial sums, then a second pass.  A is BF16 (rows of pitch lda;
// a split row adds its lo block at column offset lo_off) or FP32.
template <typename T>
__device__ __forceinline__ float ld(const T* p, size_t i, int lo_off);
template <>
__device__ __forceinline__ float ld<float>(const float* p, size_t i, int) { return p[i]; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, size_t i, int lo_off) {
    const float v = __bfloat162float(p[i]);
    return lo_off ? v + __bfloat162float(p[i + lo_off]) : v;
}

template <typename T>
__global__ void colsum_partial_kernel(const T* A, size_t lda, int lo_off, const float* v, unsigned M, int C,
                                      unsigned rows_per_block, double* part) {
    const unsigned r0 = blockIdx.x * rows_per_block, r1 = min(M, r0 + rows_per_block);
    if (C == 1) {   // one column: every thread takes a stride of rows, then a fixed tree over the block
        __shared__ float red[1024];
        float s = 0.f;
        for (unsigned m = r0 + threadIdx.x; m < r1; m += blockDim.x) s += ld<T>(A, (size_t)m * lda, lo_off) * (v ? v[m] : 1.f);
        red[threadIdx.x] = s;
        __syncthreads();
        for (unsigned h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x] = (double)red[0];
        return;
    }
    for (int j = threadIdx.x; j < C; j += blockDim.x) {
        float s = 0.f;   // FP32 within a block of rows, FP64 across blocks
        for (unsigned m = r0; m < r1; ++m) s += ld<T>(A, (size_t)m * lda + j, lo_off) * (v ? v[m] : 1.f);
        part[(size_t)blockIdx.x * C + j] = (double)s;
    }
}

// One warp per column: lane t sums partials t, t + 32, ..., then a fixed
// butterfly over the lanes (the same order on every run).
__global__ void colsum_final_kernel(const double* part, int nblk, int C, float* out) {
    const int lane = threadIdx.x & 31;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < C; j += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * C + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[j] = (float)s;
    }
}

// sum of split-K partials [splits][R][Cp] -> out[R][C], C <= Cp (fixed order;
// the padded columns are dropped)
__global__ void split_reduce_kernel(const float* part, int splits, int R, int Cp, int C, float* out) {
    const size_t n = (size_t)R * Cp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)R * C;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / C, c = e % C, i = r * Cp + c;
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * n + i];
        out[e] = s;
    }
}

// *flag = 0 when a and b differ in any bit (the caller sets it nonzero first)
__global__ void same_bits_kernel(const uint32_t* a, const uint32_t* b, size_t n, int* flag) {
    bool differ = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        differ |= a[e] != b[e];
    if (__any_sync(0xffffffffu, differ) && (threadIdx.x & 31) == 0) *flag = 0;
}

inline unsigned blocks_for(size_t n, unsigned t = kT) {
    size_t b = (n + t - 1) / t;
    if (b > 65535u * 16u) b = 65535u * 16u;
    return (unsigned)(b ? b : 1);
}

}  // namespace

// Inputs of layer l: in the packed parameters (in_packed) and as stored
// (in_store, the feature block padded to Dp); h_w(l) is the logical width of
// h[l], the input of layer l (l = depth: the head's input), and h_ld(l) its
// row pitch (ns blocks of h_w(l) BF16 values).
static inline int in_packed(const FieldDims& d, int l) {
    return l == 0 ? 6 * d.F : (l == d.skip ? d.W + 6 * d.F : d.W);
}
static inline int in_store(const FieldDims& d, int l) { return l == 0 ? d.Dp : (l == d.skip ? d.W + d.Dp : d.W); }
static inline int h_w(const FieldDims& d, int l) { return l < d.depth ? in_store(d, l) : d.W; }
static inline int h_ld(const FieldDims& d, int l) { return d.ns * h_w(d, l); }

size_t field_param_count(int F, int W, int depth, int skip) {
    size_t n = (size_t)W * 6 * F + W;
    for (int l = 1; l < depth; ++l) n += (size_t)W * (l == skip ? W + 6 * F : W) + W;
    return n + W + 1;
}

// Workspace of one field call (bytes) for M points.  Every BF16 operand
// buffer holds ns blocks (split BF16: 3).
size_t field_workspace_bytes(const FieldDims& d, bool backward) {
    const size_t Mp = d.Mp, W = d.W, ns = d.ns;
    size_t b = 0, wsum = 0, maxin = 0;
    for (int l = 0; l < d.depth; ++l) {
        wsum += W * (size_t)in_store(d, l);
        maxin = std::max(maxin, (size_t)in_store(d, l));
    }
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add((size_t)(d.nx + d.ny + d.nz) * 2 * d.F * 4);   // axis tables
    for (int l = 0; l <= d.depth; ++l) add(Mp * (size_t)h_ld(d, l) * 2);   // h_0 .. h_depth
    add(wsum * ns * 2);                                 // BF16 weights
    add(sizeof(int));
    if (backward) {
        add(wsum * ns * 2);                             // transposed weights
        add(Mp * W * ns * 2 * 2);                       // delta ping-pong
        add(Mp * 4);                                    // g_f
        for (int l = 1; l < d.depth; ++l) add(Mp * ns * (size_t)in_store(d, l) * 2);   // h_l^T
        add(Mp * ns * W * 2);                           // delta^T
        add(Mp * ns * (size_t)d.Dp * 2);                // h_0^T
        add((size_t)d.splits * W * maxin * 4);          // split-K partials
        add((size_t)d.colsum_blocks * W * 8);           // column-sum partials
    }
    return b;
}

// Carves the workspace identically to field_workspace_bytes.
struct FieldWs {
    float *tx, *ty, *tz;
    __nv_bfloat16* h[16];
    __nv_bfloat16* wb;      // BF16 weights, layer l at offset ns * woff[l]
    __nv_bfloat16* wt;      // BF16 transposed weights
    __nv_bfloat16* dl[2];
    float* gf;
    __nv_bfloat16* hT[16];  // h_l^T [in_store(l) x ns Mp], l = 1 .. depth-1
    __nv_bfloat16 *tA, *tB; // delta^T [W x ns Mp], h_0^T [Dp x ns Mp]
    float* split;
    double* colpart;
    int* err;
};

static FieldWs carve(char* base, const FieldDims& d, bool backward) {
    const size_t Mp = d.Mp, W = d.W, ns = d.ns;
    size_t wsum = 0, maxin = 0;
    for (int l = 0; l < d.depth; ++l) {
        wsum += W * (size_t)in_store(d, l);
        maxin = std::max(maxin, (size_t)in_store(d, l));
    }
    FieldWs w{};
    size_t off = 0;
    auto take = [&](size_t x) { char* p = base + off; off += (x + 255) & ~(size_t)255; return p; };
    char* tab = take((size_t)(d.nx + d.ny + d.nz) * 2 * d.F * 4);
    w.tx = (float*)tab;
    w.ty = w.tx + (size_t)d.nx * 2 * d.F;
    w.tz = w.ty + (size_t)d.ny * 2 * d.F;
    for (int l = 0; l <= d.depth; ++l) w.h[l] = (__nv_bfloat16*)take(Mp * (size_t)h_ld(d, l) * 2);
    w.wb = (__nv_bfloat16*)take(wsum * ns * 2);
    w.err = (int*)take(sizeof(int));
    if (backward) {
        w.wt = (__nv_bfloat16*)take(wsum * ns * 2);
        char* dd = take(Mp * W * ns * 2 * 2);
        w.dl[0] = (__nv_bfloat16*)dd;
        w.dl[1] = w.dl[0] + Mp * W * ns;
        w.gf = (float*)take(Mp * 4);
        for (int l = 1; l < d.depth; ++l) w.hT[l] = (__nv_bfloat16*)take(Mp * ns * (size_t)in_store(d, l) * 2);
        w.tA = (__nv_bfloat16*)take(Mp * ns * W * 2);
        w.tB = (__nv_bfloat16*)take(Mp * ns * (size_t)d.Dp * 2);
        w.split = (float*)take((size_t)d.splits * W * maxin * 4);
        w.colpart = (double*)take((size_t)d.colsum_blocks * W * 8);
    }
    return w;
}

// dst [C x ns R] = src [R x C]^T from a stored operand (rows of pitch lds,
// split blocks [hi | hi | lo] at column offsets 0, C, 2 C when ns = 3), each
// block transposed into its place in the requested order: A-side [hi | hi | lo]
// (b_side = false) or B-side [hi | lo | hi].
static void transpose_operand(const __nv_bfloat16* src, size_t lds, __nv_bfloat16* dst, unsigned R, int C, int ns,
                              bool b_side, cudaStream_t s) {
    const dim3 tb(32, 8), grid((R + 31) / 32, (C + 31) / 32);
    const size_t ldd = (size_t)ns * R;
    for (int b = 0; b < ns; ++b) {
        const int from = ns == 1 ? 0 : (b_side ? (b == 1 ? 2 : 0) : b);   // source block of output block b
        transpose_bf16_kernel<<<grid, tb, 0, s>>>(src + (size_t)from * C, lds, dst + (size_t)b * R, ldd, R, C);
    }
}

// with_t: the epilogues also write h_l^T (l = 1 .. depth-1) for the backward.
static cudaError_t forward_layers(const FieldDims& d, const float* theta, const float* band_w, FieldWs& w,
                                  cudaStream_t s, bool with_t) {
    const int F = d.F, W = d.W, ns = d.ns;
    const double lo = d.freq_lo, ratio_log = log(d.freq_hi / d.freq_lo);
    axis_table_kernel<<<blocks_for((size_t)d.nx * F), kT, 0, s>>>(w.tx, d.nx, F, lo, ratio_log, band_w);
    axis_table_kernel<<<blocks_for((size_t)d.ny * F), kT, 0, s>>>(w.ty, d.ny, F, lo, ratio_log, band_w);
    axis_table_kernel<<<blocks_for((size_t)d.nz * F), kT, 0, s>>>(w.tz, d.nz, F, lo, ratio_log, band_w);
    // one thread per 16-byte chunk of a cell's features (F % 4 == 0), else per feature
    const size_t fwork = (size_t)d.Mp * (F % 4 == 0 ? d.Dp / 8 : d.Dp);
    features_kernel<<<blocks_for(fwork), kT, 0, s>>>(w.h[0], d.M, d.Mp, d.nx, d.ny, F, d.Dp, ns, w.tx, w.ty, w.tz);
    if (d.skip > 0)   // the encoding beside h_s in each block of the skip layer's input
        for (int b = 0; b < ns; ++b)
            copy_cols_kernel<<<blocks_for((size_t)d.Mp * d.Dp / 8), kT, 0, s>>>(
                w.h[0] + (size_t)b * d.Dp, ns * d.Dp, w.h[d.skip], h_ld(d, d.skip), b * h_w(d, d.skip) + W, d.Dp,
                d.Mp);
    // BF16 copies of the weights, zero-padded to the stored inputs
    const float* p = theta;
    size_t woff = 0;
    for (int l = 0; l < d.depth; ++l) {
        const int in = in_packed(d, l), ins = in_store(d, l);
        to_bf16_kernel<<<blocks_for((size_t)W * ins), kT, 0, s>>>(p, w.wb + ns * woff, W, in, ins, ns);
        p += (size_t)W * in + W;
        woff += (size_t)W * ins;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    p = theta;
    woff = 0;
    for (int l = 0; l < d.depth; ++l) {
        const int in = in_packed(d, l), ins = in_store(d, l);
        const float* bias = p + (size_t)W * in;
        const bool t = with_t && l + 1 < d.depth;
        const int so = ns == 3 ? h_w(d, l + 1) : 0;
        e = umma_gemm(w.h[l], ns * ins, w.wb + ns * woff, ns * ins, (int)d.Mp, W, ns * ins, 0 /*bias+relu*/, bias,
                      nullptr, w.h[l + 1], nullptr, h_ld(d, l + 1), 1, w.err, s, t ? w.hT[l + 1] : nullptr,
                      t ? ns * (int)d.Mp : 0, 0, so, (t && ns == 3) ? (int)d.Mp : 0, 1 /*B-side transposes*/);
        if (e != cudaSuccess) return e;
        p += (size_t)W * in + W;
        woff += (size_t)W * ins;
    }
    return cudaSuccess;
}

cudaError_t field_eval(const FieldDims& d, const float* theta, const float* band_w, float* alpha, char* ws,
                       cudaStream_t s, bool keep) {
    FieldWs w = carve(ws, d, keep);
    cudaError_t e = cudaMemsetAsync(w.err, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if ((e = forward_layers(d, theta, band_w, w, s, keep)) != cudaSuccess) return e;
    const float* w_out = theta + field_param_count(d.F, d.W, d.depth, d.skip) - d.W - 1;
    head_kernel<<<blocks_for((size_t)d.M * 32), kT, 0, s>>>(w.h[d.depth], (size_t)h_ld(d, d.depth),
                                                            d.ns == 3 ? 2 * d.W : 0, d.W, w_out, w_out + d.W, d.M,
                                                            (float)d.alpha_min, (float)d.alpha_max, alpha);
    return cudaGetLastError();
}

cudaError_t field_backward(const FieldDims& d, const float* theta, const float* band_w, const float* g_alpha,
                           float* g_theta, char* ws, cudaStream_t s, bool reuse) {
    FieldWs w = carve(ws, d, true);
    const int W = d.W, ns = d.ns;
    const int lo_w = ns == 3 ? 2 * W : 0;   // column offset of the lo block of a W-wide split row
    cudaError_t e = cudaMemsetAsync(w.err, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    // reuse: ws already holds the activations, their transposes and the axis
    // tables of a keep-mode evaluation at these same parameters
    if (!reuse && (e = forward_layers(d, theta, band_w, w, s, true)) != cudaSuccess) return e;
    // parameter offsets (packed) and weight-copy offsets (stored, in units of one block)
    size_t poff[16], woff[16];
    {
        size_t p = 0, q = 0;
        for (int l = 0; l < d.depth; ++l) {
            poff[l] = p;
            woff[l] = q;
            p += (size_t)W * in_packed(d, l) + W;
            q += (size_t)W * in_store(d, l);
        }
        poff[d.depth] = p;
    }
    const float* w_out = theta + poff[d.depth];
    float* g_wout = g_theta + poff[d.depth];
    // head
    head_back_kernel<<<blocks_for((size_t)d.Mp * 32), kT, 0, s>>>(w.h[d.depth], (size_t)h_ld(d, d.depth), lo_w, W,
                                                                  w_out, w_out + W, d.M, d.Mp, (float)d.alpha_min,
                                                                  (float)d.alpha_max, g_alpha, w.gf, w.dl[0], ns);
    // dw_out[j] = sum_m gf[m] h[m][j];  db_out = sum_m gf[m]
    const unsigned rpb = (d.Mp + d.colsum_blocks - 1) / d.colsum_blocks;
    colsum_partial_kernel<__nv_bfloat16><<<d.colsum_blocks, kT, 0, s>>>(w.h[d.depth], (size_t)h_ld(d, d.depth), lo_w,
                                                                      w.gf, d.Mp, W, rpb, w.colpart);
    colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(w.colpart, d.colsum_blocks, W, g_wout);
    colsum_partial_kernel<float><<<d.colsum_blocks, kT, 0, s>>>(w.gf, 1, 0, nullptr, d.Mp, 1, rpb, w.colpart);
    colsum_final_kernel<<<1, 32, 0, s>>>(w.colpart, d.colsum_blocks, 1, g_wout + W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // transposed BF16 weights W_l^T [in_store x ns W] (B side) for the input-gradient GEMMs
    {
        const float* p = theta;
        for (int l = 0; l < d.depth; ++l) {
            const int in = in_packed(d, l), ins = in_store(d, l);
            transpose_f32_bf16_kernel<<<blocks_for((size_t)W * ins), kT, 0, s>>>(p, w.wt + ns * woff[l], W, in, ins,
                                                                                 ns);
            p += (size_t)W * in + W;
        }
    }
    // h_0^T (B side), also the encoding rows of the skip layer's h^T
    features_t_kernel<<<blocks_for((size_t)d.Dp * (d.Mp / 8)), kT, 0, s>>>(w.tB, d.M, d.Mp, d.nx, d.ny, d.F, d.Dp,
                                                                          ns, w.tx, w.ty, w.tz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (d.skip > 0 && d.skip < d.depth) {
        e = cudaMemcpyAsync(w.hT[d.skip] + (size_t)W * ns * d.Mp, w.tB, (size_t)d.Dp * ns * d.Mp * 2,
                            cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    // layers, top to bottom: delta_l = dJ/dz_{l+1} [Mp x ns W] lives in dl[cur]
    int cur = 0;
    for (int l = d.depth - 1; l >= 0; --l) {
        const int in = in_packed(d, l), ins = in_store(d, l);
        // db_l = column sums of delta
        colsum_partial_kernel<__nv_bfloat16><<<d.colsum_blocks, kT, 0, s>>>(w.dl[cur], (size_t)ns * W, lo_w, nullptr,
                                                                          d.Mp, W, rpb, w.colpart);
        colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(w.colpart, d.colsum_blocks, W,
                                                         g_theta + poff[l] + (size_t)W * in);
        // dW_l = delta^T h_l: K-major operands are the transposes [W x ns Mp] (A
        // side) and [ins x ns Mp] (B side).  delta^T comes from the previous
        // masked product's epilogue (top layer: transposed here); h_l^T from the
        // forward epilogues (l = 0: h_0^T).
        if (l == d.depth - 1) transpose_operand(w.dl[cur], (size_t)ns * W, w.tA, d.Mp, W, ns, false, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // split-K: one CTA per SM over the layer's output tiles
        const int tiles = ((W + 127) / 128) * ((ins + 127) / 128);
        const int splits = std::min(d.splits, std::max(1, d.sms / tiles));
        e = umma_gemm(w.tA, ns * (int)d.Mp, l == 0 ? w.tB : w.hT[l], ns * (int)d.Mp, W, ins, ns * (int)d.Mp,
                      2 /*f32 partials*/, nullptr, nullptr, nullptr, w.split, ins, splits, w.err, s);
        if (e != cudaSuccess) return e;
        split_reduce_kernel<<<blocks_for((size_t)W * in), kT, 0, s>>>(w.split, splits, W, ins, in,
                                                                      g_theta + poff[l]);
        // delta_{l-1} = (delta_l W_l[:, :W]) masked by h_l > 0 (the h part of the
        // skip layer's input; its encoding part needs no gradient)
        if (l > 0) {
            e = umma_gemm(w.dl[cur], ns * W, w.wt + ns * woff[l], ns * W, (int)d.Mp, W, ns * W, 1 /*mask*/, nullptr,
                          w.h[l], w.dl[cur ^ 1], nullptr, ns * W, 1, w.err, s, w.tA, ns * (int)d.Mp, h_ld(d, l),
                          ns == 3 ? W : 0, ns == 3 ? (int)d.Mp : 0, 0 /*A-side transposes*/);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    return cudaGetLastError();
}

cudaError_t field_params_equal(const float* a, const float* b, size_t n, int* flag, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    same_bits_kernel<<<blocks_for(n), kT, 0, s>>>(reinterpret_cast<const uint32_t*>(a),
                                                  reinterpret_cast<const uint32_t*>(b), n, flag);
    return cudaGetLastError();
}

int field_error(const FieldDims& d, char* ws, cudaStream_t s, bool backward) {
    FieldWs w = carve(ws, d, backward);
    int h = 0;
    if (cudaMemcpyAsync(&h, w.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return h;
}

}  // namespace nefty
