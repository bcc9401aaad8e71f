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
// tabT [2F][n] gets the same values feature-major (for h_0^T).
__global__ void axis_table_kernel(float* tab, float* tabT, int n, int F, double lo, double ratio_log,
                                  const float* band_w) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * F; e += gridDim.x * blockDim.x) {
        const int i = e / F, b = e % F;
        const double x = 2.0 * ((double)i + 0.5) / (double)n - 1.0;
        const double w = F > 1 ? lo * exp(ratio_log * (double)b / (double)(F - 1)) : lo;
        const double wt = band_w ? (double)band_w[b] : 1.0;
        const float sv = (float)(wt * sin(w * x)), cv = (float)(wt * cos(w * x));
        tab[(size_t)i * 2 * F + 2 * b] = sv;
        tab[(size_t)i * 2 * F + 2 * b + 1] = cv;
        tabT[(size_t)(2 * b) * n + i] = sv;
        tabT[(size_t)(2 * b + 1) * n + i] = cv;
    }
}

// Split of 8 FP32 values into BF16 hi words and lo = bf16(v - hi) words.
__device__ __forceinline__ void split8(const float* v, uint32_t* hi, uint32_t* lo) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * t], v[2 * t + 1]);
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * t] - __low2float(h2), v[2 * t + 1] - __high2float(h2));
        hi[t] = *reinterpret_cast<const uint32_t*>(&h2);
        lo[t] = *reinterpret_cast<const uint32_t*>(&l2);
    }
}

// h0[c][d*2F + j] = tab_d[index_d(c)][j], as BF16, rows padded to Mp and
// columns to Dp (zeros); rows of ns * Dp values, the split blocks [hi | hi | lo]
// at offsets 0, Dp, 2 Dp when ns = 3.  With F % 4 == 0 a warp writes one
// cell's row at a time, lane l its 16-byte chunks l, l + 32, ... (8 features,
// never straddling two axes; the cell's axis indices are warp-uniform);
// otherwise one feature per thread.
__global__ void features_kernel(__nv_bfloat16* h0, unsigned M, unsigned Mp, int nx, int ny, int F, int Dp, int ns,
                                const float* tx, const float* ty, const float* tz) {
    const int D = 6 * F, F2 = 2 * F;
    const size_t ld = (size_t)ns * Dp;
    if ((F & 3) == 0) {
        const int per = Dp / 8, lane = threadIdx.x & 31;   // 16-byte chunks per cell
        const unsigned warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
        for (unsigned c = warp0; c < Mp; c += nwarps) {
            const unsigned cy = c / (unsigned)nx, i = c - cy * (unsigned)nx;
            const unsigned k = cy / (unsigned)ny, j = cy - k * (unsigned)ny;
            for (int q = lane; q < per; q += 32) {
                const int f = 8 * q;
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (c < M && f < D) {
                    const int d = f / F2, r = f - d * F2;
                    const float* row = d == 0 ? tx + (size_t)i * F2 : (d == 1 ? ty + (size_t)j * F2 : tz + (size_t)k * F2);
                    const float4 p = *reinterpret_cast<const float4*>(row + r);
                    const float4 p2 = *reinterpret_cast<const float4*>(row + r + 4);
                    v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = p2.x; v[5] = p2.y; v[6] = p2.z; v[7] = p2.w;
                }
                uint32_t hi[4], lo[4];
                split8(v, hi, lo);
                __nv_bfloat16* out = h0 + (size_t)c * ld + f;
                *reinterpret_cast<uint4*>(out) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                if (ns == 3) {
                    *reinterpret_cast<uint4*>(out + Dp) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4*>(out + 2 * Dp) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
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

// h_0^T [Dp x ns Mp], K-blocked, straight from the feature-major axis tables txT [2F][nx],
// tyT [2F][ny], tzT [2F][nz], as the B side of the first layer's
// weight-gradient product: row f holds feature f of every cell, the split
// blocks in B-side order [hi | lo | hi] at column offsets 0, Mp, 2 Mp (zeros
// for padded cells and features).  The same BF16 values as features_kernel
// writes, transposed.  Row f = blockIdx.y; each thread writes 8 consecutive
// cells (16 bytes per block; Mp is a multiple of 128), reading consecutive
// table entries (x features) or one entry (y, z features) when nx % 8 == 0.
__global__ void features_t_kernel(__nv_bfloat16* hT, unsigned M, unsigned Mp, int nx, int ny, int nz, int F, int Dp,
                                  int ns, const float* tx, const float* ty, const float* tz) {
    const int D = 6 * F, F2 = 2 * F, f = blockIdx.y;
    const int d = f / F2, r = f - d * F2;
    const unsigned per = Mp / 8;   // 8-cell chunks per feature row
    __nv_bfloat16* rowT = hT + (size_t)f * 64;   // K-blocked: (k / 64) Dp 64 + f 64 + k % 64
    const bool fast = (nx & 7) == 0;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < per; q += gridDim.x * blockDim.x) {
        const unsigned c0 = q * 8;
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (f < D && c0 < M) {
            unsigned cy = c0 / (unsigned)nx, i = c0 - cy * (unsigned)nx;
            unsigned k = cy / (unsigned)ny, j = cy - k * (unsigned)ny;
            if (fast && c0 + 8 <= M) {   // the 8 cells share j and k
                if (d == 0) {
                    const float4 p = *reinterpret_cast<const float4*>(tx + (size_t)r * nx + i);
                    const float4 p2 = *reinterpret_cast<const float4*>(tx + (size_t)r * nx + i + 4);
                    v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = p2.x; v[5] = p2.y; v[6] = p2.z; v[7] = p2.w;
                } else {
                    const float x = d == 1 ? ty[(size_t)r * ny + j] : tz[(size_t)r * nz + k];
#pragma unroll
                    for (int t = 0; t < 8; ++t) v[t] = x;
                }
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (c0 + t < M)
                        v[t] = d == 0 ? tx[(size_t)r * nx + i] : (d == 1 ? ty[(size_t)r * ny + j] : tz[(size_t)r * nz + k]);
                    if (++i == (unsigned)nx) {
                        i = 0;
                        if (++j == (unsigned)ny) { j = 0; ++k; }
                    }
                }
            }
        }
        uint32_t hi[4], lo[4];
        split8(v, hi, lo);
        __nv_bfloat16* out = rowT + (size_t)(c0 >> 6) * Dp * 64 + (c0 & 63);
        *reinterpret_cast<uint4*>(out) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if (ns == 3) {   // the split blocks start Mp and 2 Mp along k: Mp Dp and 2 Mp Dp elements on
            *reinterpret_cast<uint4*>(out + (size_t)Mp * Dp) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            *reinterpret_cast<uint4*>(out + 2 * (size_t)Mp * Dp) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        }
    }
}

// dst [R x Cp] = bf16(src [R x C]) with zero columns C .. Cp-1; with ns = 3
// rows of 3 Cp values, the split blocks in B-side order [hi | lo | hi].
// K-blocked (the B operand of a layer product): element (r, k) of the [R x ns
// Cp] matrix at (k / 64) R 64 + r 64 + k % 64; Cp is a multiple of 64.
__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, int R, int C, int Cp, int ns) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)R * Cp;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Cp), c = (int)(e % Cp);
        const float v = c < C ? src[(size_t)r * C + c] : 0.f;
        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
        __nv_bfloat16* out = dst + (size_t)(c >> 6) * R * 64 + (size_t)r * 64 + (c & 63);
        out[0] = hv;
        if (ns == 3) {   // blocks at k = Cp and 2 Cp: Cp R and 2 Cp R elements on
            out[(size_t)Cp * R] = __float2bfloat16_rn(v - __bfloat162float(hv));
            out[2 * (size_t)Cp * R] = hv;
        }
    }
}

// dst [Cp x R] = bf16(src [R x C])^T with zero rows C .. Cp-1; with ns = 3
// rows of 3 R values in B-side order [hi | lo | hi].  K-blocked: element
// (c, k) of the [Cp x ns R] matrix at (k / 64) Cp 64 + c 64 + k % 64; R is a
// multiple of 64.
__global__ void transpose_f32_bf16_kernel(const float* src, __nv_bfloat16* dst, int R, int C, int Cp, int ns) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)R * Cp;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / R), r = (int)(e % R);
        const float v = c < C ? src[(size_t)r * C + c] : 0.f;
        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
        __nv_bfloat16* out = dst + (size_t)(r >> 6) * Cp * 64 + (size_t)c * 64 + (r & 63);
        out[0] = hv;
        if (ns == 3) {   // blocks at k = R and 2 R: R Cp and 2 R Cp elements on
            out[(size_t)R * Cp] = __float2bfloat16_rn(v - __bfloat162float(hv));
            out[2 * (size_t)R * Cp] = hv;
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
                                      unsigned R, int C, int rt) {
    __shared__ __nv_bfloat16 t[32][33];
    const unsigned r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const unsigned r = r0 + yy, c = c0 + threadIdx.x;
        t[yy][threadIdx.x] = (r < R && c < (unsigned)C) ? src[(size_t)r * lds + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const unsigned c = c0 + yy, r = r0 + threadIdx.x;
        if (c < (unsigned)C && r < R)
            dst[rt ? (size_t)(r >> 6) * rt * 64 + (size_t)c * 64 + (r & 63) : (size_t)c * ldd + r] = t[threadIdx.x][yy];
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

// The head's backward in one pass over h = h_depth, in tiles of kHR = 64
// rows: per row g_f (as head_back_kernel) and the top layer's delta, written
// row-major (rows of ns W, blocks [hi | hi | lo]) and transposed as the A side
// of its weight-gradient product (deltaT [W x ns Mp] K-blocked, blocks
// [hi | hi | lo] at k offsets 0, Mp, 2 Mp); and, per block of rows, the partial sums of
// dw_out[j] = sum_m g_f[m] h[m][j], db_out = sum_m g_f[m] and db_top[j] =
// sum_m delta[m][j] (the stored value: hi, + lo when split) at part
// [blk][W], [nblk][W] + blk and [nblk][W + 1] + blk * W + j, for
// colsum_final_kernel.  Warp w takes rows kRW w .. kRW w + kRW - 1 of a tile,
// lane l the 16-byte column chunks l, l + 32, ... (VC of them): a row's dot
// product is a warp reduction and its delta is written from registers; only
// the transpose goes through shared memory, as words holding two consecutive
// rows of one column (kHQ = 32 words per column, the word index XOR-swizzled
// by the column's chunk so that the writes and the column reads each cover
// the 32 banks), and leaves it 128 contiguous bytes per column.  Sums are
// FP32 per thread in row order, then over the block's warps in warp order.
constexpr int kHR = 64, kRW = kHR / (kT / 32), kHQ = kHR / 2;
__device__ __forceinline__ size_t hq_index(int col, int pair) {
    return (size_t)col * kHQ + (pair ^ ((col >> 3) & (kHQ - 1)));
}
inline int head_vc(int W) { return (W / 8 + 31) / 32; }
inline size_t head_fused_smem(int W, int ns) {
    const size_t tiles = (size_t)(ns == 3 ? 2 : 1) * W * kHQ * 4;   // hi (and lo) transposed tiles
    const size_t sums = (size_t)(kT / 32) * (2 * W + 1) * 4;         // per-warp partial sums, at the end
    return std::max(tiles, sums);
}
constexpr size_t kHeadSmemMax = 200 * 1024;   // wider heads take the unfused kernels

template <int VC, int NS>
__global__ void __launch_bounds__(kT, (VC == 1 && NS == 1) ? 2 : 1) head_back_fused_kernel(
    const __nv_bfloat16* h, size_t ld, int lo_off, int W, const float* w_out, const float* b_out, unsigned M,
    unsigned Mp, float a_lo, float a_hi, const float* g_alpha, float* gf, __nv_bfloat16* delta,
    __nv_bfloat16* deltaT, unsigned rows_per_block, double* part) {
    extern __shared__ uint32_t hsm[];
    uint32_t* thi = hsm;                          // [W][kHQ] transposed hi pairs
    uint32_t* tlo = hsm + (size_t)W * kHQ;        // [W][kHQ] transposed lo pairs (NS = 3)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kT / 32;
    const int cpr = W / 8;                        // 16-byte chunks per row
    const unsigned r0 = blockIdx.x * rows_per_block, r1 = min(Mp, r0 + rows_per_block);
    const size_t ldd = (size_t)NS * W;
    const float bo = b_out[0], span = a_hi - a_lo;
    float sw[VC][8], sd[VC][8], sb = 0.f;
#pragma unroll
    for (int v = 0; v < VC; ++v)
#pragma unroll
        for (int t = 0; t < 8; ++t) sw[v][t] = sd[v][t] = 0.f;
    // the value of column t of a raw 16-byte chunk (hi, + lo when split)
    auto val = [&](const uint4& a, const uint4& b, int t) {
        const uint32_t wa = t < 2 ? a.x : (t < 4 ? a.y : (t < 6 ? a.z : a.w));
        const float hv = __uint_as_float((t & 1) ? (wa & 0xFFFF0000u) : (wa << 16));
        if (NS == 1) return hv;
        const uint32_t wb = t < 2 ? b.x : (t < 4 ? b.y : (t < 6 ? b.z : b.w));
        return hv + __uint_as_float((t & 1) ? (wb & 0xFFFF0000u) : (wb << 16));
    };
    for (unsigned m0 = r0; m0 < r1; m0 += kHR) {   // Mp and rows_per_block are multiples of kHR
        const unsigned mw = m0 + kRW * warp;        // this warp's first row
        float ga[kRW];
#pragma unroll
        for (int i = 0; i < kRW; ++i) ga[i] = mw + i < M ? g_alpha[mw + i] : 0.f;
        uint4 ra[kRW][VC], rb[kRW][VC];             // raw hi (and lo) chunks of the warp's rows
#pragma unroll
        for (int i = 0; i < kRW; ++i)
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                const int q = lane + 32 * v;
                ra[i][v] = rb[i][v] = make_uint4(0u, 0u, 0u, 0u);
                if (q < cpr) {
                    const __nv_bfloat16* src = h + (size_t)(mw + i) * ld + 8 * q;
                    ra[i][v] = *reinterpret_cast<const uint4*>(src);
                    if (NS == 3) rb[i][v] = *reinterpret_cast<const uint4*>(src + lo_off);
                }
            }
        float g[kRW];
#pragma unroll
        for (int i = 0; i < kRW; ++i) {
            float sacc = 0.f;
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                const int q = lane + 32 * v;
                if (q < cpr)
#pragma unroll
                    for (int t = 0; t < 8; ++t) sacc += val(ra[i][v], rb[i][v], t) * w_out[8 * q + t];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            const float sg = 1.f / (1.f + expf(-(sacc + bo)));
            g[i] = mw + i < M ? ga[i] * span * sg * (1.f - sg) : 0.f;
            sb += g[i];
        }
        if (lane < kRW) {
            float gl = g[0];
#pragma unroll
            for (int i = 1; i < kRW; ++i) gl = lane == i ? g[i] : gl;
            gf[mw + lane] = gl;
        }
        __syncthreads();                            // the previous tile's transposed reads are done
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const int q = lane + 32 * v;
            if (q >= cpr) continue;
#pragma unroll
            for (int pr = 0; pr < kRW / 2; ++pr) {  // rows kRW w + 2 pr, + 1
                uint32_t hp[8], lp[8];              // one word per column: the pair's two rows
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int i = 2 * pr + e;
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float hv = val(ra[i][v], rb[i][v], t);
                        const float wj = w_out[8 * q + t];
                        const float dv = hv > 0.f ? g[i] * wj : 0.f;
                        const __nv_bfloat16 dh = __float2bfloat16_rn(dv);
                        const uint32_t hb = __bfloat16_as_ushort(dh);
                        sw[v][t] += g[i] * hv;
                        uint32_t lb = 0u;
                        if (NS == 3) {
                            const __nv_bfloat16 dl = __float2bfloat16_rn(dv - __bfloat162float(dh));
                            lb = __bfloat16_as_ushort(dl);
                            sd[v][t] += __bfloat162float(dh) + __bfloat162float(dl);
                        } else {
                            sd[v][t] += __bfloat162float(dh);
                        }
                        if (e == 0) { hp[t] = hb; lp[t] = lb; }
                        else { hp[t] |= hb << 16; lp[t] |= lb << 16; }
                        if (t & 1) { hw[t >> 1] |= hb << 16; lw[t >> 1] |= lb << 16; }
                        else { hw[t >> 1] = hb; lw[t >> 1] = lb; }
                    }
                    __nv_bfloat16* out = delta + (size_t)(mw + i) * ldd + 8 * q;
                    *reinterpret_cast<uint4*>(out) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    if (NS == 3) {
                        *reinterpret_cast<uint4*>(out + W) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(out + 2 * W) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const size_t o = hq_index(8 * q + t, (kRW / 2) * warp + pr);
                    thi[o] = hp[t];
                    if (NS == 3) tlo[o] = lp[t];
                }
            }
        }
        __syncthreads();
        // deltaT, K-blocked (element (j, k) at (k / 64) W 64 + j 64 + k % 64; the
        // tile is one 64-wide k-block): a warp writes one column's 64 rows,
        // 128 contiguous bytes per block
        for (int j = warp; j < W; j += nw) {
            const size_t o = hq_index(j, lane);
            uint32_t* dst = reinterpret_cast<uint32_t*>(deltaT + (size_t)(m0 >> 6) * W * 64 + (size_t)j * 64) + lane;
            const uint32_t wv = thi[o];
            *dst = wv;
            if (NS == 3) {
                dst[(size_t)Mp * W / 2] = wv;
                dst[(size_t)Mp * W] = tlo[o];
            }
        }
    }
    // block sums: per-warp partials through shared memory, summed in warp order
    __syncthreads();
    float* red = reinterpret_cast<float*>(hsm);   // [nw][2 W + 1]
    const int rw = 2 * W + 1;
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        const int q = lane + 32 * v;
        if (q >= cpr) continue;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            red[(size_t)warp * rw + 8 * q + t] = sw[v][t];
            red[(size_t)warp * rw + W + 8 * q + t] = sd[v][t];
        }
    }
    if (lane == 0) red[(size_t)warp * rw + 2 * W] = sb;
    __syncthreads();
    const unsigned nblk = gridDim.x;
    for (int c = threadIdx.x; c < rw; c += kT) {
        float s = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) s += red[(size_t)w2 * rw + c];
        if (c < W) part[(size_t)blockIdx.x * W + c] = (double)s;
        else if (c < 2 * W) part[(size_t)nblk * (W + 1) + (size_t)blockIdx.x * W + (c - W)] = (double)s;
        else part[(size_t)nblk * W + blockIdx.x] = (double)s;
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
    add((size_t)(d.nx + d.ny + d.nz) * 2 * d.F * 4 * 2 + 16);   // axis tables, cell-major and feature-major
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
        add((size_t)d.colsum_blocks * (2 * W + 1) * 8); // column-sum partials (the fused head: 2 W + 1 per block)
        add(Mp / 32 * W * 4);                           // per-32-row delta column sums of the masked products
    }
    return b;
}

// Carves the workspace identically to field_workspace_bytes.
struct FieldWs {
    float *tx, *ty, *tz;          // axis tables [n][2F]
    float *txT, *tyT, *tzT;       // the same, [2F][n]
    __nv_bfloat16* h[16];
    __nv_bfloat16* wb;      // BF16 weights [W x ns in_store], K-blocked, layer l at offset ns * woff[l]
    __nv_bfloat16* wt;      // BF16 transposed weights [in_store x ns W], K-blocked
    __nv_bfloat16* dl[2];
    float* gf;
    // transposes for the weight-gradient products, K-blocked: element (r, k) of
    // R rows at (k / 64) R 64 + r 64 + k % 64 (one 64-wide k-block of 128
    // rows is 16 contiguous KB, a single TMA box)
    __nv_bfloat16* hT[16];  // h_l^T [in_store(l) x ns Mp], l = 1 .. depth-1
    __nv_bfloat16 *tA, *tB; // delta^T [W x ns Mp], h_0^T [Dp x ns Mp]
    float* split;
    double* colpart;
    float* cs32;            // [Mp / 32][W] column sums of a masked product's delta over each 32 rows
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
    char* tab = take((size_t)(d.nx + d.ny + d.nz) * 2 * d.F * 4 * 2 + 16);
    w.tx = (float*)tab;
    w.ty = w.tx + (size_t)d.nx * 2 * d.F;
    w.tz = w.ty + (size_t)d.ny * 2 * d.F;
    w.txT = w.tx + ((size_t)(d.nx + d.ny + d.nz) * 2 * d.F + 3) / 4 * 4;   // 16-byte aligned
    w.tyT = w.txT + (size_t)d.nx * 2 * d.F;
    w.tzT = w.tyT + (size_t)d.ny * 2 * d.F;
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
        w.colpart = (double*)take((size_t)d.colsum_blocks * (2 * W + 1) * 8);
        w.cs32 = (float*)take(Mp / 32 * W * 4);
    }
    return w;
}

// dst [C x ns R] = src [R x C]^T from a stored operand (rows of pitch lds,
// split blocks [hi | hi | lo] at column offsets 0, C, 2 C when ns = 3), each
// block transposed into its place in the requested order: A-side [hi | hi | lo]
// (b_side = false) or B-side [hi | lo | hi].
// dst is written K-blocked (element (c, k) of C rows at (k / 64) C 64 + c 64 +
// k % 64, k = block * R + r; R is a multiple of 64), the layout the
// weight-gradient products read.
static void transpose_operand(const __nv_bfloat16* src, size_t lds, __nv_bfloat16* dst, unsigned R, int C, int ns,
                              bool b_side, cudaStream_t s) {
    const dim3 tb(32, 8), grid((R + 31) / 32, (C + 31) / 32);
    for (int b = 0; b < ns; ++b) {
        const int from = ns == 1 ? 0 : (b_side ? (b == 1 ? 2 : 0) : b);   // source block of output block b
        transpose_bf16_kernel<<<grid, tb, 0, s>>>(src + (size_t)from * C, lds, dst + (size_t)b * R * C, 0, R, C, C);
    }
}

// with_t: the epilogues also write h_l^T (l = 1 .. depth-1) for the backward.
static cudaError_t forward_layers(const FieldDims& d, const float* theta, const float* band_w, FieldWs& w,
                                  cudaStream_t s, bool with_t) {
    const int F = d.F, W = d.W, ns = d.ns;
    const double lo = d.freq_lo, ratio_log = log(d.freq_hi / d.freq_lo);
    axis_table_kernel<<<blocks_for((size_t)d.nx * F), kT, 0, s>>>(w.tx, w.txT, d.nx, F, lo, ratio_log, band_w);
    axis_table_kernel<<<blocks_for((size_t)d.ny * F), kT, 0, s>>>(w.ty, w.tyT, d.ny, F, lo, ratio_log, band_w);
    axis_table_kernel<<<blocks_for((size_t)d.nz * F), kT, 0, s>>>(w.tz, w.tzT, d.nz, F, lo, ratio_log, band_w);
    // one thread per 16-byte chunk of a cell's features (F % 4 == 0), else per feature
    const size_t fwork = F % 4 == 0 ? (size_t)d.Mp * 32 : (size_t)d.Mp * d.Dp;   // one warp per cell, else per feature
    const unsigned fblocks = F % 4 == 0 ? std::min(blocks_for(fwork), (unsigned)(16 * d.sms)) : blocks_for(fwork);
    features_kernel<<<fblocks, kT, 0, s>>>(w.h[0], d.M, d.Mp, d.nx, d.ny, F, d.Dp, ns, w.tx, w.ty, w.tz);
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
                      t ? ns * (int)d.Mp : 0, 0, so, (t && ns == 3) ? (int)d.Mp : 0, 1 /*B-side transposes*/, 0,
                      W /*K-blocked weights*/, t ? in_store(d, l + 1) : 0 /*K-blocked transposes*/);
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
    const unsigned rpb = (d.Mp + d.colsum_blocks - 1) / d.colsum_blocks;
    // head: g_f, the top delta and its transpose, dw_out, db_out and the top
    // layer's db in one pass when its row tile fits in shared memory
    const size_t hsm = head_fused_smem(W, ns);
    const int vc = head_vc(W);
    // up to 1024 columns per row (512 split) in registers; wider heads take the unfused kernels
    const bool fused = hsm <= kHeadSmemMax && (vc == 1 || vc == 2 || (vc == 4 && ns == 1));
    if (fused) {
        auto kern = ns == 1 ? (vc == 1 ? head_back_fused_kernel<1, 1>
                                       : (vc == 2 ? head_back_fused_kernel<2, 1> : head_back_fused_kernel<4, 1>))
                            : (vc == 1 ? head_back_fused_kernel<1, 3> : head_back_fused_kernel<2, 3>);
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeadSmemMax)) !=
            cudaSuccess)
            return e;
        int occ = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kT, hsm)) != cudaSuccess) return e;
        // blocks: the resident ones, at most the partial buffer's colsum_blocks
        const unsigned nblk = (unsigned)std::max(1, std::min(d.colsum_blocks, std::max(1, occ) * d.sms));
        const unsigned hrpb = ((d.Mp + nblk - 1) / nblk + kHR - 1) / kHR * kHR;
        kern<<<nblk, kT, hsm, s>>>(w.h[d.depth], (size_t)h_ld(d, d.depth), lo_w, W, w_out, w_out + W, d.M, d.Mp,
                                   (float)d.alpha_min, (float)d.alpha_max, g_alpha, w.gf, w.dl[0], w.tA, hrpb,
                                   w.colpart);
        const double* part = w.colpart;
        colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(part, (int)nblk, W, g_wout);
        colsum_final_kernel<<<1, 32, 0, s>>>(part + (size_t)nblk * W, (int)nblk, 1, g_wout + W);
        colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(
            part + (size_t)nblk * (W + 1), (int)nblk, W, g_theta + poff[d.depth - 1] + (size_t)W * in_packed(d, d.depth - 1));
    } else {
        head_back_kernel<<<blocks_for((size_t)d.Mp * 32), kT, 0, s>>>(w.h[d.depth], (size_t)h_ld(d, d.depth), lo_w, W,
                                                                      w_out, w_out + W, d.M, d.Mp, (float)d.alpha_min,
                                                                      (float)d.alpha_max, g_alpha, w.gf, w.dl[0], ns);
        // dw_out[j] = sum_m gf[m] h[m][j];  db_out = sum_m gf[m]
        colsum_partial_kernel<__nv_bfloat16><<<d.colsum_blocks, kT, 0, s>>>(
            w.h[d.depth], (size_t)h_ld(d, d.depth), lo_w, w.gf, d.Mp, W, rpb, w.colpart);
        colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(w.colpart, d.colsum_blocks, W, g_wout);
        colsum_partial_kernel<float><<<d.colsum_blocks, kT, 0, s>>>(w.gf, 1, 0, nullptr, d.Mp, 1, rpb, w.colpart);
        colsum_final_kernel<<<1, 32, 0, s>>>(w.colpart, d.colsum_blocks, 1, g_wout + W);
    }
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
    {
        const unsigned gx = std::min(blocks_for(d.Mp / 8), (unsigned)std::max(1, 8 * d.sms / std::max(1, d.Dp / 8)));
        features_t_kernel<<<dim3(gx, d.Dp), kT, 0, s>>>(w.tB, d.M, d.Mp, d.nx, d.ny, d.nz, d.F, d.Dp, ns, w.txT, w.tyT,
                                                         w.tzT);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (d.skip > 0 && d.skip < d.depth) {
        // K-blocked: per 64-wide k-block, rows W .. W + Dp of the skip layer's input
        e = cudaMemcpy2DAsync(w.hT[d.skip] + (size_t)W * 64, (size_t)(W + d.Dp) * 64 * 2, w.tB,
                              (size_t)d.Dp * 64 * 2, (size_t)d.Dp * 64 * 2, (size_t)ns * d.Mp / 64,
                              cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    // layers, top to bottom: delta_l = dJ/dz_{l+1} [Mp x ns W] lives in dl[cur]
    int cur = 0;
    for (int l = d.depth - 1; l >= 0; --l) {
        const int in = in_packed(d, l), ins = in_store(d, l);
        // db_l = column sums of delta: the top layer's in the fused head pass,
        // the others from the 32-row sums the masked product's epilogue left
        if (l == d.depth - 1 && !fused) {
            colsum_partial_kernel<__nv_bfloat16><<<d.colsum_blocks, kT, 0, s>>>(w.dl[cur], (size_t)ns * W, lo_w,
                                                                              nullptr, d.Mp, W, rpb, w.colpart);
            colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(w.colpart, d.colsum_blocks, W,
                                                                         g_theta + poff[l] + (size_t)W * in);
        } else if (l < d.depth - 1) {
            const unsigned rows = d.Mp / 32, rpb32 = (rows + d.colsum_blocks - 1) / d.colsum_blocks;
            colsum_partial_kernel<float><<<d.colsum_blocks, kT, 0, s>>>(w.cs32, W, 0, nullptr, rows, W, rpb32,
                                                                      w.colpart);
            colsum_final_kernel<<<blocks_for((size_t)W * 32), kT, 0, s>>>(w.colpart, d.colsum_blocks, W,
                                                                         g_theta + poff[l] + (size_t)W * in);
        }
        // dW_l = delta^T h_l: K-major operands are the transposes [W x ns Mp] (A
        // side) and [ins x ns Mp] (B side), both K-blocked.  delta^T comes from the previous
        // masked product's epilogue (top layer: transposed here); h_l^T from the
        // forward epilogues (l = 0: h_0^T).
        if (l == d.depth - 1 && !fused) transpose_operand(w.dl[cur], (size_t)ns * W, w.tA, d.Mp, W, ns, false, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // split-K: one CTA per SM over the layer's output tiles
        const int tiles = ((W + 127) / 128) * ((ins + 127) / 128);
        const int splits = std::min(d.splits, std::max(1, d.sms / tiles));
        e = umma_gemm(w.tA, ns * (int)d.Mp, l == 0 ? w.tB : w.hT[l], ns * (int)d.Mp, W, ins, ns * (int)d.Mp,
                      2 /*f32 partials*/, nullptr, nullptr, nullptr, w.split, ins, splits, w.err, s, nullptr, 0, 0,
                      0, 0, 0, W, ins /*K-blocked A and B*/);
        if (e != cudaSuccess) return e;
        split_reduce_kernel<<<blocks_for((size_t)W * in), kT, 0, s>>>(w.split, splits, W, ins, in,
                                                                      g_theta + poff[l]);
        // delta_{l-1} = (delta_l W_l[:, :W]) masked by h_l > 0 (the h part of the
        // skip layer's input; its encoding part needs no gradient)
        if (l > 0) {
            e = umma_gemm(w.dl[cur], ns * W, w.wt + ns * woff[l], ns * W, (int)d.Mp, W, ns * W, 1 /*mask*/, nullptr,
                          w.h[l], w.dl[cur ^ 1], nullptr, ns * W, 1, w.err, s, w.tA, ns * (int)d.Mp, h_ld(d, l),
                          ns == 3 ? W : 0, ns == 3 ? (int)d.Mp : 0, 0 /*A-side transposes*/, 0,
                          ins /*K-blocked weights*/, W /*K-blocked transposes*/, w.cs32 /*db_{l-1} partials*/);
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
