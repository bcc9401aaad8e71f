// BF16 GEMM on the 5th-generation tensor cores (tcgen05), for the neural
// field's dense layers (Sec. 4.1, App. D.1).
//
//   D[m, n] = sum_k A[m, k] * B[n, k]        A: [M x K], B: [N x K], both BF16, K contiguous
//
// One CTA computes one 128 x 128 tile of D (or one split-K slice of it).
// A and B tiles of 64 K-elements arrive by TMA (128-byte swizzle, the canonical
// K-major layout the tensor core reads) in a shared-memory ring: two stages
// when K is short (the layers' 256-384; three CTAs then share an SM and overlap
// one tile's epilogue with the others' loads and MMAs), six for the long-K
// weight-gradient products; a
// single thread issues tcgen05.mma (M = 128, N = 128, K = 16 per instruction)
// with the FP32 accumulator in tensor memory and releases each stage with
// tcgen05.commit onto that stage's "empty" mbarrier.  After the last k-block the
// four warps read their 32 accumulator lanes with tcgen05.ld and apply the
// epilogue, each thread writing 16-byte pieces of its row (and, where asked,
// the transposed output and per-warp column sums).
//
// An operand is either row-major (a 2D tensor map, box 64 x 128) or K-blocked:
// element (r, k) of R rows at (k / 64) R 64 + r 64 + k % 64, read through a 3D
// map whose box {64, 128, 1} is 16 contiguous KB and lands in shared memory
// exactly as the 2D box does.  The long-K weight-gradient products read their
// transposed operands that way; a row-major box there would fetch 128 rows a
// whole K apart.
//
// Every wait is bounded: on timeout the kernel records an error, waits
// (bounded) for its own copies and MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace nefty {
namespace umma {

constexpr int BM = 128, BN = 128, BK = 64;      // tile and k-block (64 BF16 = one 128-byte swizzle row)
constexpr int THREADS = 128;                     // 4 warps = the 128 accumulator lanes
constexpr int TILE_BYTES = BM * BK * 2;          // 16 KB per operand per stage
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int smem_bytes(int stages) { return stages * STAGE_BYTES + 1024; }   // + 1024-byte alignment slack
// short K: 2 stages, 3 CTAs per SM (3 x 128 TMEM columns, 3 x 65 KB); long K: 6 stages, 1 CTA
constexpr int ctas_per_sm(int stages) { return stages == 2 ? 3 : 1; }
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long g_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint32_t b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, unsigned bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(b), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t b, unsigned parity) {
    unsigned long long t0 = 0;
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(b), "r"(parity) : "memory");
        if (done) return true;
        if ((i & 63u) == 63u) {
            const unsigned long long t = g_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitNs) return false;
        }
    }
}
__device__ __forceinline__ void tma2(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(b) : "memory");
}
__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(b) : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout: 8-row atoms of 1024 bytes stacked along M/N (stride 1024), start
// address in 16-byte units, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major,
// N = BN, M = BM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

enum Epi : int {
    kEpiBiasReluBf16 = 0,   // out_bf16 = bf16(relu(acc + bias[n]))
    kEpiMaskBf16 = 1,       // out_bf16 = bf16(acc * (mask_bf16[m, n] > 0))
    kEpiF32 = 2,            // out_f32[split] = acc (split-K partial)
};

struct Args {
    int M, N, K;            // K is a multiple of BK; M, N may be ragged (masked)
    int k_blocks_per_split;
    int epi;
    const float* bias;      // [N]
    const __nv_bfloat16* mask;   // [M, ldm]
    __nv_bfloat16* out_bf16;     // [M, ldo]
    float* out_f32;              // [splits][M, ldo]
    int ldo;
    int ldm;                     // leading dimension of mask
    int vec;                     // ldo, ldm and every base 16-byte aligned: 16-byte epilogue stores
    __nv_bfloat16* out_t;        // BF16 epilogues: also D^T [N, ldt] (or null)
    int ldt;
    int n_tiles;                 // output tiles along N
    int* err;
    // Split BF16 outputs (0 = plain): a value v is written as hi = bf16(v) and
    // lo = bf16(v - hi).  out_bf16 gets [hi | hi | lo] at column offsets 0,
    // so, 2 so; out_t gets three blocks at column offsets 0, tso, 2 tso in the
    // order [hi | hi | lo] (t_order 0) or [hi | lo | hi] (t_order 1).
    int so, tso, t_order;
    // K-blocked operands and transposed output (0 = row-major): element
    // (r, k) of a matrix with R rows sits at (k / 64) R 64 + r 64 + k % 64,
    // so one 64-wide k-block of 128 rows is 16 contiguous KB
    int a_blk, b_blk;            // A, B in that layout (TMA through a 3D map): its row count R, 0 = row-major
    int t_rows;                  // out_t in that layout with t_rows rows
    // BF16 epilogues, whole tiles only: column sums of the stored output (hi,
    // + lo when split) over each warp's 32 rows, at colsum[(row / 32) N + col]
    float* colsum;
};

// COLSUM: the variant with the epilogue's column sums (Args::colsum)
template <int STAGES, bool COLSUM>
__global__ void __launch_bounds__(THREADS, ctas_per_sm(STAGES))
gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Args a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[STAGES], empty[STAGES], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the N tiles of one M tile are consecutive CTAs, so the A tile they share
    // is read from DRAM once and from L2 by the others
    const int m0 = (int)(blockIdx.x / (unsigned)a.n_tiles) * BM, n0 = (int)(blockIdx.x % (unsigned)a.n_tiles) * BN;
    const int kb0 = blockIdx.z * a.k_blocks_per_split;
    const int kb1 = min(a.K / BK, kb0 + a.k_blocks_per_split);
    const int nk = kb1 - kb0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(s_u32(&full[s]), 1);
            bar_init(s_u32(&empty[s]), 1);
        }
        bar_init(s_u32(&done), 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&s_tmem)),
                     "r"(BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    // ---- producer + MMA issue (one thread)
    if (threadIdx.x == 0 && nk > 0) {
        auto sa = [&](int s) { return s_u32(smem + s * STAGE_BYTES); };
        auto sb = [&](int s) { return s_u32(smem + s * STAGE_BYTES + TILE_BYTES); };
        auto load = [&](int i) {   // k-block kb0 + i into stage i % STAGES
            const int s = i % STAGES;
            bar_expect_tx(s_u32(&full[s]), STAGE_BYTES);
            if (a.a_blk) tma3(sa(s), &mapA, 0, m0, kb0 + i, s_u32(&full[s]));
            else tma2(sa(s), &mapA, (kb0 + i) * BK, m0, s_u32(&full[s]));
            if (a.b_blk) tma3(sb(s), &mapB, 0, n0, kb0 + i, s_u32(&full[s]));
            else tma2(sb(s), &mapB, (kb0 + i) * BK, n0, s_u32(&full[s]));
        };
        int issued = 0;
        for (; issued < nk && issued < STAGES; ++issued) load(issued);
        bool ok = true;
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % STAGES;
            ok = bar_wait(s_u32(&full[s]), (unsigned)(i / STAGES) & 1u);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < BK / 16; ++j)   // K = 16 per instruction: 32 bytes along the swizzled row
                mma(tmem, smem_desc(sa(s) + 32 * j), smem_desc(sb(s) + 32 * j), (i > 0 || j > 0) ? 1u : 0u);
            mma_commit(s_u32(&empty[s]));
            // refill the stage used one k-block ago once its MMAs are done
            if (i > 0 && issued < nk) {
                const int sp = (i - 1) % STAGES;
                ok = bar_wait(s_u32(&empty[sp]), (unsigned)((i - 1) / STAGES) & 1u);
                if (ok) load(issued++);
            }
        }
        if (ok) {
            mma_commit(s_u32(&done));
        } else {
            s_fail = 1;
            atomicExch(a.err, 1);
        }
    }
    __syncthreads();
    bool ok = s_fail == 0;
    if (ok && nk > 0) ok = bar_wait(s_u32(&done), 0);
    if (!ok && threadIdx.x == 0) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31; a thread
    // holds 32 consecutive columns of its row per tcgen05.ld and writes them as
    // 16-byte pieces when the chunk is whole and aligned (a.vec), else singly.
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            if (nk > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int t = 0; t < 32; ++t) v[t] = 0u;
            }
            const int cb = n0 + c0;
            if (row >= a.M || cb >= a.N) continue;
            const size_t o = (size_t)row * a.ldo + cb;
            if (a.vec && cb + 32 <= a.N) {
                if (a.epi == kEpiF32) {
                    float4* dst = reinterpret_cast<float4*>(a.out_f32 + (size_t)blockIdx.z * a.M * a.ldo + o);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                             __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                } else {
                    uint32_t mk[16];
                    float xs[32];   // the values before rounding (split outputs)
                    if (a.epi == kEpiMaskBf16) {
                        const uint4* src = reinterpret_cast<const uint4*>(a.mask + (size_t)row * a.ldm + cb);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint4 w = src[q];
                            mk[4 * q] = w.x; mk[4 * q + 1] = w.y; mk[4 * q + 2] = w.z; mk[4 * q + 3] = w.w;
                        }
                    }
                    uint32_t pk[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        float x0 = __uint_as_float(v[2 * t]), x1 = __uint_as_float(v[2 * t + 1]);
                        if (a.epi == kEpiBiasReluBf16) {
                            x0 = fmaxf(x0 + a.bias[cb + 2 * t], 0.f);
                            x1 = fmaxf(x1 + a.bias[cb + 2 * t + 1], 0.f);
                        } else {   // mask: keep where the BF16 mask value is > 0
                            const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mk[t]);
                            if (!(__low2float(m2) > 0.f)) x0 = 0.f;
                            if (!(__high2float(m2) > 0.f)) x1 = 0.f;
                        }
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(x0, x1);
                        pk[t] = *reinterpret_cast<const uint32_t*>(&b2);
                        xs[2 * t] = x0;
                        xs[2 * t + 1] = x1;
                    }
                    uint32_t pl[16];   // lo parts of a split output
                    if (a.so || a.tso) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&pk[t]);
                            const __nv_bfloat162 l2 = __floats2bfloat162_rn(xs[2 * t] - __low2float(h2),
                                                                            xs[2 * t + 1] - __high2float(h2));
                            pl[t] = *reinterpret_cast<const uint32_t*>(&l2);
                        }
                    }
                    uint4* dst = reinterpret_cast<uint4*>(a.out_bf16 + o);
#pragma unroll
                    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                    if (COLSUM) {   // every lane is here: whole tiles (checked on the host)
                        // butterfly reduce-scatter over the warp's 32 rows: after the
                        // round with offset o a lane holds o partial column sums, the
                        // upper half of its 2o when lane & o; at the end column lane
                        float cs[32];
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&pk[t]);
                            cs[2 * t] = __low2float(h2);
                            cs[2 * t + 1] = __high2float(h2);
                            if (a.so || a.tso) {
                                const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&pl[t]);
                                cs[2 * t] += __low2float(l2);
                                cs[2 * t + 1] += __high2float(l2);
                            }
                        }
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) {
                            const bool up = (lane & off) != 0;
#pragma unroll
                            for (int j = 0; j < off; ++j) {
                                const float send = up ? cs[j] : cs[j + off];
                                const float keep = up ? cs[j + off] : cs[j];
                                cs[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                            }
                        }
                        a.colsum[(size_t)(row >> 5) * a.N + cb + lane] = cs[0];
                    }
                    if (a.so) {
                        uint4* d1 = reinterpret_cast<uint4*>(a.out_bf16 + o + a.so);
                        uint4* d2 = reinterpret_cast<uint4*>(a.out_bf16 + o + 2 * (size_t)a.so);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            d1[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                            d2[q] = make_uint4(pl[4 * q], pl[4 * q + 1], pl[4 * q + 2], pl[4 * q + 3]);
                        }
                    }
                    if (a.out_t) {   // the warp's 32 rows of one column are 64 contiguous bytes of D^T
                        const int nb = a.tso ? 3 : 1;
                        for (int b = 0; b < nb; ++b) {
                            const bool lo = b == (a.t_order == 0 ? 2 : 1);
                            const uint32_t* src = lo ? pl : pk;
                            const size_t k = (size_t)b * a.tso + row, cs = a.t_rows ? 64 : (size_t)a.ldt;
                            const size_t ko = a.t_rows ? (k >> 6) * (size_t)a.t_rows * 64 + (k & 63) : k;
                            unsigned short* dt = reinterpret_cast<unsigned short*>(a.out_t) + ko + (size_t)cb * cs;
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                dt[(size_t)(2 * t) * cs] = (unsigned short)(src[t] & 0xFFFFu);
                                dt[(size_t)(2 * t + 1) * cs] = (unsigned short)(src[t] >> 16);
                            }
                        }
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int col = cb + t;
                    if (col >= a.N) continue;
                    const float acc = __uint_as_float(v[t]);
                    const size_t e = (size_t)row * a.ldo + col;
                    if (a.epi == kEpiBiasReluBf16 || a.epi == kEpiMaskBf16) {
                        const __nv_bfloat16 r = a.epi == kEpiBiasReluBf16
                                                    ? __float2bfloat16_rn(fmaxf(acc + a.bias[col], 0.f))
                                                    : __float2bfloat16_rn(
                                                          __bfloat162float(a.mask[(size_t)row * a.ldm + col]) > 0.f
                                                              ? acc : 0.f);
                        a.out_bf16[e] = r;
                        const float xv = a.epi == kEpiBiasReluBf16
                                             ? fmaxf(acc + a.bias[col], 0.f)
                                             : (__bfloat162float(a.mask[(size_t)row * a.ldm + col]) > 0.f ? acc : 0.f);
                        const __nv_bfloat16 rl = __float2bfloat16_rn(xv - __bfloat162float(r));
                        if (a.so) {
                            a.out_bf16[e + a.so] = r;
                            a.out_bf16[e + 2 * (size_t)a.so] = rl;
                        }
                        if (a.out_t) {
                            const int nb = a.tso ? 3 : 1;
                            for (int b = 0; b < nb; ++b) {
                                const bool lo = b == (a.t_order == 0 ? 2 : 1);
                                const size_t k = (size_t)b * a.tso + row;
                                const size_t o = a.t_rows ? (k >> 6) * (size_t)a.t_rows * 64 + (size_t)col * 64 + (k & 63)
                                                          : (size_t)col * a.ldt + k;
                                a.out_t[o] = lo ? rl : r;
                            }
                        }
                    } else {
                        a.out_f32[(size_t)blockIdx.z * a.M * a.ldo + e] = acc;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        // wait (bounded) for whatever this CTA still has in flight
        for (int s = 0; s < STAGES; ++s) bar_wait(s_u32(&empty[s]), 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

}  // namespace umma

// ------------------------------------------------------------------- host
namespace {
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D BF16 map over [rows x cols] (cols contiguous, pitch ld elements), box
// 64 x 128 with the 128-byte swizzle; with blk, a 3D map over the K-blocked
// layout [cols / 64][rows][64], box 64 x 128 x 1 (16 contiguous KB), which
// lands in shared memory exactly as the 2D box does.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, bool blk = false) {
    auto enc = encoder();
    if (!enc) return false;
    if (blk) {
        const cuuint64_t dims[3] = {(cuuint64_t)umma::BK, (cuuint64_t)rows, (cuuint64_t)(cols / umma::BK)};
        const cuuint64_t strides[2] = {(cuuint64_t)umma::BK * 2, (cuuint64_t)rows * umma::BK * 2};
        const cuuint32_t box[3] = {(cuuint32_t)umma::BK, (cuuint32_t)umma::BM, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)umma::BK, (cuuint32_t)umma::BM};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

// D[M x N] = A[M x K] B[N x K]^T with the chosen epilogue (and, for the BF16
// epilogues, D^T into out_t when given).  K % 64 == 0, lda/ldb in elements
// (multiples of 8).  splits > 1 only with kEpiF32.
cudaError_t umma_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                      int epi, const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out_bf16,
                      float* out_f32, int ldo, int splits, int* err, cudaStream_t s, __nv_bfloat16* out_t, int ldt,
                      int ldm, int so, int tso, int t_order, int a_blk, int b_blk, int t_rows, float* colsum) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(umma::gemm_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             umma::smem_bytes(2));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(umma::gemm_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     umma::smem_bytes(2));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(umma::gemm_kernel<6, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     umma::smem_bytes(6));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(umma::gemm_kernel<6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     umma::smem_bytes(6));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (K % umma::BK != 0 || lda % 8 != 0 || ldb % 8 != 0 || splits < 1) return cudaErrorInvalidValue;
    if (out_t && (epi == umma::kEpiF32 || (t_rows ? t_rows < N : ldt < M))) return cudaErrorInvalidValue;
    if (t_rows && ((tso ? 3 * (size_t)tso : (size_t)M) % umma::BK != 0 || (tso && tso % umma::BK != 0)))
        return cudaErrorInvalidValue;   // K-blocked D^T: whole 64-wide k-blocks
    if ((so || tso) && epi == umma::kEpiF32) return cudaErrorInvalidValue;
    if (so < 0 || so % 8 != 0 || tso < 0 || (tso && (tso < M || ldt < 2 * tso + M))) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if ((a_blk && a_blk < M) || (b_blk && b_blk < N)) return cudaErrorInvalidValue;
    if (!make_map(&ma, A, a_blk ? a_blk : M, K, lda, a_blk != 0) || !make_map(&mb, B, b_blk ? b_blk : N, K, ldb, b_blk != 0))
        return cudaErrorInvalidValue;
    umma::Args a;
    a.M = M; a.N = N; a.K = K;
    const int kb = K / umma::BK;
    a.k_blocks_per_split = (kb + splits - 1) / splits;
    a.epi = epi;
    a.bias = bias; a.mask = mask; a.out_bf16 = out_bf16; a.out_f32 = out_f32; a.ldo = ldo;
    a.ldm = ldm > 0 ? ldm : ldo;
    a.out_t = out_t;
    a.ldt = ldt;
    a.so = so;
    a.tso = out_t ? tso : 0;
    a.t_order = t_order;
    a.a_blk = a_blk;
    a.b_blk = b_blk;
    a.t_rows = out_t ? t_rows : 0;
    a.colsum = colsum;
    auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    a.vec = (epi == umma::kEpiF32 ? (ldo % 4 == 0 && al16(out_f32))
                                  : (ldo % 8 == 0 && al16(out_bf16) &&
                                     (epi != umma::kEpiMaskBf16 || (al16(mask) && a.ldm % 8 == 0))))
                ? 1 : 0;
    a.err = err;
    if (colsum && (epi == umma::kEpiF32 || M % umma::BM || N % umma::BN || !a.vec)) return cudaErrorInvalidValue;
    a.n_tiles = (N + umma::BN - 1) / umma::BN;
    const long long tiles = (long long)((M + umma::BM - 1) / umma::BM) * a.n_tiles;
    if (tiles < 1 || tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)tiles, 1, splits);
    if (colsum && a.k_blocks_per_split <= 8)
        umma::gemm_kernel<2, true><<<grid, umma::THREADS, umma::smem_bytes(2), s>>>(ma, mb, a);
    else if (colsum)
        umma::gemm_kernel<6, true><<<grid, umma::THREADS, umma::smem_bytes(6), s>>>(ma, mb, a);
    else if (a.k_blocks_per_split <= 8)
        umma::gemm_kernel<2, false><<<grid, umma::THREADS, umma::smem_bytes(2), s>>>(ma, mb, a);
    else
        umma::gemm_kernel<6, false><<<grid, umma::THREADS, umma::smem_bytes(6), s>>>(ma, mb, a);
    return cudaGetLastError();
}

}  // namespace nefty
