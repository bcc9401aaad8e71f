// FP32 persistent single-reduction PCG for the implicit-Euler heat solve and
// its adjoint, on z-marching xy-tiles (Sec. 4.2-4.3, App. D.2-D.3).
//
// Each CG iteration is ONE pass over the grid and ONE grid barrier.  The
// recurrences are the single-reduction (Chronopoulos-Gear) form of Jacobi-PCG:
// with u = M^{-1} r and w = A u, the scalars alpha_i and beta_i come from the
// two inner products (r, u) and (w, u) taken in the same reduction, and
// s = A p follows from s_i = w_i + beta_i s_{i-1}.  The kernel stores the
// preconditioned vectors u, ws = M^{-1} w and ss = M^{-1} s, so that the next
// iterate u_{i+1} = u_i - alpha_i (ws_i + beta_i ss_{i-1}) can be formed at any
// cell from that cell's own stored values; a pass needs nothing from its
// neighbours but those values.
//
// Work layout: the grid is cut into 32 x 32 columns and the (tile, plane)
// pairs are split evenly over the CTAs; each CTA marches up z through its
// share.  A CTA has eight compute warps and one copy warp.  A compute thread
// owns four consecutive cells along x (a quad) in one row of the tile.
//
// Iteration passes stage their inputs through the Tensor Memory Accelerator:
// the copy warp streams every plane (u, ws, ss and alpha with a one-cell halo;
// p and delta) into a ring of shared-memory stages guarded by full/empty
// mbarriers, and the compute warps consume the stages in order with no
// CTA-wide barrier.  A thread that needs u_{i+1} at a neighbour cell forms it
// again from the staged values with the same fused multiply-adds as the
// cell's owner, so every thread sees the same bits.  The passes that run once
// per solve (initial residual, first product, gradient) are staged the same
// way (periodic lateral walls included: the wrapped halo cells are fetched by
// the threads that read them); grids TMA cannot stage (nx % 4 != 0) read global
// memory directly.
//
// Numerics: the stencil is evaluated in flux form, A v = v + sum_f c_f (v_c - v_q)
// (+ Robin sink), and each solve accumulates its increment delta separately so
// that T^{n+1} = T^n + delta is rounded once per step.  Inner products are
// accumulated per thread as compensated FP32 pairs and summed across threads
// and CTAs in a fixed order, so repeated runs are bitwise equal.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace nefty {
namespace tiled {

constexpr int NW = NT / 32;   // warps per CTA

// The CTA's index within, and the number of CTAs of, the sweep it works on:
// cta_id() and cta_count() in a launch of one sweep; in a grouped launch
// (several sweeps, each on its own range of CTAs) the index within the range
// and the range's size.  Set by each kernel before any sweep code runs.
static __shared__ unsigned s_cta, s_ncta;
__device__ __forceinline__ unsigned cta_id() { return s_cta; }
__device__ __forceinline__ unsigned cta_count() { return s_ncta; }

// ------------------------------------------------------------------ sync
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Sync {
    DevCtl* ctl;
    unsigned* bar;      // the arrival counter in use (ctl->bar or ctl->bar2)
    double* partials;   // [2][kMaxRed][G] float2 pairs
    unsigned G;
    unsigned epoch;     // thread 0 only
    unsigned red;       // uniform
    unsigned missing;   // arrivals that never come (fault injection; 0 normally)
    unsigned long long wait_ns;   // barrier wait limit
};

// Bounded grid barrier: returns false on timeout or when another CTA has
// flagged an error.  The CTA's writes are ordered before thread 0's release
// add by the CTA barrier (release is cumulative), and the acquire load that
// sees every arrival orders the other CTAs' writes before the closing CTA
// barrier, so no separate fences are needed.
__device__ bool barrier(Sync& g) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        g.epoch += 1;
        const unsigned target = g.epoch * g.G + g.missing;
        red_release(g.bar, 1u);
        int ok = 1;
        unsigned spins = 0;
        unsigned long long t0 = 0;
        while (ld_acquire(g.bar) < target) {
            if ((++spins & 63u) == 0) {
                if (ld_relaxed(&g.ctl->err) != kDevOk) { ok = 0; break; }
                const unsigned long long t = now_ns();
                if (t0 == 0) t0 = t;
                else if (t - t0 > g.wait_ns) {
                    atomicCAS(&g.ctl->err, kDevOk, kDevTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Error-free transformation of a + b (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bv = s - a;
    e = (a - (s - bv)) + (b - bv);
}

// (hi, lo) + d as a renormalised compensated pair.
__device__ __forceinline__ void add_pair(float hi, float lo, float d, float& oh, float& ol) {
    float s, e;
    two_sum(hi, d, s, e);
    two_sum(s, lo + e, oh, ol);
}

// Per-thread compensated accumulators of NV inner products.
template <int NV>
struct Acc {
    float h[NV], l[NV];
    __device__ Acc() {
#pragma unroll
        for (int i = 0; i < NV; ++i) h[i] = l[i] = 0.f;
    }
    __device__ __forceinline__ void add(int i, float v) { add_pair(h[i], l[i], v, h[i], l[i]); }
};

// Compensated warp sum of (hi, lo) pairs, every lane gets the result: the
// high parts are summed with TwoSum and the rounding errors collected in lo,
// which is folded in only by the caller (the cascaded summation of Ogita,
// Rump and Oishi, accurate as if computed in twice the precision).  The
// dependency chain per level is one shuffle and one add.
__device__ __forceinline__ void warp_sum2(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, e;
        two_sum(hi, oh, sh, e);
        hi = sh;
        lo = lo + ol + e;
    }
}

// --------------------------------------------------------- double-float
// The CG scalars are kept as unevaluated sums hi + lo of two floats and
// updated with error-free transformations on the FP32 pipes (Dekker's
// double-length arithmetic): about 44 bits of precision at a fraction of the
// latency of GB300's FP64 units.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_norm(float a, float b) {   // Fast2Sum: needs |a| >= |b| or a == 0
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_make(float hi, float lo) {   // renormalise any pair
    float s, e;
    two_sum(hi, lo, s, e);
    return DF{s, e};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
    float sh, sl, th, tl;
    two_sum(x.hi, y.hi, sh, sl);
    two_sum(x.lo, y.lo, th, tl);
    const DF v = df_norm(sh, sl + th);
    return df_norm(v.hi, tl + v.lo);
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float ch = x.hi * y.hi;
    const float cl1 = fmaf(x.hi, y.hi, -ch);
    const float cl2 = fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, x.lo * y.lo));
    return df_norm(ch, cl1 + cl2);
}
// q1 from the hardware reciprocal (about 1 ulp): the remainder x - q1 y is
// formed exactly (TwoProd through fmaf, and x.hi - p is exact for q1 that
// close), so the quotient keeps the precision of the pair whatever q1's last
// bit; a correctly rounded division would only add latency to the chain of
// CG scalars every iteration waits on.
__device__ __forceinline__ DF df_div(DF x, DF y) {
    float ry;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(y.hi));
    const float q1 = x.hi * ry;
    const float p = q1 * y.hi;
    const float pe = fmaf(q1, y.hi, -p);
    const float r = (((x.hi - p) - pe) + x.lo) - q1 * y.lo;   // x - q1 y
    return df_norm(q1, r * ry);
}
__device__ __forceinline__ bool df_le(DF x, DF y) { return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo); }

// After the grid barrier of a grid sum: compute warp i sums value i of the
// G CTA partials (every load of the warp first, then the fixed order: the
// rows of a lane, then the warp tree), so all values take one round trip to
// L2 at once; values i < NV as compensated pairs, the others (pout) in plain
// FP32.  The totals reach thread 0 through shared memory.
template <int NV, int NP>
__device__ void sum_partials(const Sync& g, const float2* part, DF (&out)[NV], float* pout) {
    static_assert(NV + NP <= CW && NV + NP <= kMaxRed, "one compute warp per value");
    __shared__ float s_th[kMaxRed], s_tl[kMaxRed];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < NV + NP) {
        float2 v[kMaxGrid / 32];
#pragma unroll
        for (int r = 0; r < kMaxGrid / 32; ++r) {
            const unsigned b = lane + 32u * r;
            v[r] = b < g.G ? part[(size_t)b * kMaxRed + warp] : make_float2(0.f, 0.f);
        }
        float hi = 0.f, lo = 0.f;
        if (warp < NV) {
#pragma unroll
            for (int r = 0; r < kMaxGrid / 32; ++r) {
                float sh, e;
                two_sum(hi, v[r].x, sh, e);
                hi = sh;
                lo = lo + v[r].y + e;
            }
            warp_sum2(hi, lo);
        } else {
#pragma unroll
            for (int r = 0; r < kMaxGrid / 32; ++r) hi += v[r].x;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hi += __shfl_xor_sync(0xffffffffu, hi, o);
        }
        if (lane == 0) {
            s_th[warp] = hi;
            s_tl[warp] = lo;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i] = df_make(s_th[i], s_tl[i]);
#pragma unroll
        for (int i = 0; i < NP; ++i) pout[i] = s_th[NV + i];
    }
}

// Grid sum of NV compensated per-thread pairs.  The sums run on the FP32
// pipes as (hi, lo) pairs, which keeps about twice the FP32 precision: TwoSum
// trees over the warp, the CTA and the G CTA partials (fixed order, so every
// run gives the same bits).  GB300's FP64 rate is a small fraction of its FP32
// rate, so no FP64 arithmetic is done per thread.  On return thread 0 holds
// the totals as double-floats; the other threads' out[] is unspecified.
// Every pass ends here, so this is also where each thread orders its global
// stores of the pass before the TMA reads of later passes.  after_barrier()
// runs in every thread right after the grid barrier, before the partials are
// summed (the copy thread starts the next pass's copies there).  Every thread
// of the CTA takes part (sum_partials ends with a CTA barrier).
template <int NV, class Hook>
__device__ bool grid_sum(Sync& g, const Acc<NV>& in, DF (&out)[NV], Hook after_barrier) {
    __shared__ float s_h[NW][kMaxRed], s_l[NW][kMaxRed];
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float hi = in.h[i], lo = in.l[i];
        warp_sum2(hi, lo);
        if (lane == 0) { s_h[warp][i] = hi; s_l[warp][i] = lo; }
    }
    __syncthreads();
    // partials: [2][G][kMaxRed] (hi, lo) pairs
    float2* part = reinterpret_cast<float2*>(g.partials) + (size_t)(g.red & 1u) * kMaxRed * g.G;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float hi = lane < NW ? s_h[lane][i] : 0.f, lo = lane < NW ? s_l[lane][i] : 0.f;
            warp_sum2(hi, lo);
            if (lane == 0) part[(size_t)cta_id() * kMaxRed + i] = make_float2(hi, lo);
        }
    }
    if (!barrier(g)) return false;
    after_barrier();
    sum_partials<NV, 0>(g, part, out, nullptr);
    g.red += 1;
    return true;
}

// grid_sum plus NP values reduced in plain FP32 (warp trees, CTA partials
// and a fixed-order grid sum, as grid_sum but without the compensation): the
// residual-norm expansion's sums, whose use needs about 1e-5 of relative
// accuracy.  They ride in partial slots NV .. NV + NP - 1.
template <int NV, int NP, class Hook>
__device__ bool grid_sum_p(Sync& g, const Acc<NV>& in, const float (&pin)[NP], DF (&out)[NV], float (&pout)[NP],
                           Hook after_barrier) {
    static_assert(NV + NP <= kMaxRed, "reduction slots");
    __shared__ float s_h[NW][kMaxRed], s_l[NW][kMaxRed];
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float hi = in.h[i], lo = in.l[i];
        warp_sum2(hi, lo);
        if (lane == 0) { s_h[warp][i] = hi; s_l[warp][i] = lo; }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        float v = pin[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_h[warp][NV + i] = v;
    }
    __syncthreads();
    float2* part = reinterpret_cast<float2*>(g.partials) + (size_t)(g.red & 1u) * kMaxRed * g.G;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float hi = lane < NW ? s_h[lane][i] : 0.f, lo = lane < NW ? s_l[lane][i] : 0.f;
            warp_sum2(hi, lo);
            if (lane == 0) part[(size_t)cta_id() * kMaxRed + i] = make_float2(hi, lo);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            float v = lane < NW ? s_h[lane][NV + i] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) part[(size_t)cta_id() * kMaxRed + NV + i] = make_float2(v, 0.f);
        }
    }
    if (!barrier(g)) return false;
    after_barrier();
    sum_partials<NV, NP>(g, part, out, pout);
    g.red += 1;
    return true;
}

__device__ double block_sum(double v) {
    __shared__ double s[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < NW ? s[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// --------------------------------------------------------------- operator
// Hardware reciprocal (rcp.approx, about 1 ulp).  Used for the face values and
// the Jacobi diagonal: their rounding moves the solution far less than the
// FP32 CG arithmetic does, and every pass evaluates them identically.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Harmonic-mean face value dt * a_f = k * 2 a b / (a + b), k = dt / h^2, of the
// face between cells of diffusivity a and b (Prop. 1).  face(a, b) and
// face(b, a) are the same products of the same two values, so A stays exactly
// symmetric.  b = 0 (a cell beyond a zero-flux wall, as TMA fills it) gives 0.
__device__ __forceinline__ float face(float a, float b, float k) {
    return k * (2.f * a * b) * rcp_approx(a + b);
}

// Neighbours of cell c = (x, y, k) in the order +x, -x, +y, -y, +z, -z; bit f
// of m is set when neighbour f exists (inside the grid or across a periodic
// wrap).  A missing neighbour is a zero-flux wall.
struct Nb {
    unsigned q[6];
    unsigned m;
};
__device__ __forceinline__ Nb neighbours(const Geo& g, unsigned c, int x, int y, int k) {
    Nb n;
    n.m = 0;
    const unsigned wrap_y = (unsigned)(g.ny - 1) * g.nx;
    if (x + 1 < g.nx) { n.q[0] = c + 1; n.m |= 1u; } else if (g.px) { n.q[0] = c + 1 - g.nx; n.m |= 1u; }
    if (x > 0) { n.q[1] = c - 1; n.m |= 2u; } else if (g.px) { n.q[1] = c + g.nx - 1; n.m |= 2u; }
    if (y + 1 < g.ny) { n.q[2] = c + g.nx; n.m |= 4u; } else if (g.py) { n.q[2] = c - wrap_y; n.m |= 4u; }
    if (y > 0) { n.q[3] = c - g.nx; n.m |= 8u; } else if (g.py) { n.q[3] = c + wrap_y; n.m |= 8u; }
    if (k + 1 < g.nz) { n.q[4] = c + g.S; n.m |= 16u; }
    if (k > 0) { n.q[5] = c - g.S; n.m |= 32u; }
    return n;
}

// The six face values of cell c (0 where there is no neighbour).
__device__ __forceinline__ void cell_faces(const Common& C, const Nb& n, float ac, float (&cf)[6]) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const float kf = f < 2 ? C.kx : (f < 4 ? C.ky : C.kz);
        cf[f] = (n.m >> f & 1u) ? face(ac, C.alpha[n.q[f]], kf) : 0.f;
    }
}

// Diagonal of A: 1 + the face values (+x, -x, +y, -y, +z, -z, in this order)
// + the Robin sink.  Every path sums in this order.
__device__ __forceinline__ float diag(float cxp, float cxm, float cyp, float cym, float czp, float czm,
                                      float rob) {
    return 1.f + cxp + cxm + cyp + cym + czp + czm + rob;
}

// --------------------------------------------------------------- work split
// Iterate over this CTA's (tile, plane) segments.
template <class SegFn>
__device__ __forceinline__ void for_segments(const Geo& g, SegFn seg) {
    const unsigned long long U = g.units;
    unsigned u = (unsigned)(U * cta_id() / cta_count());
    const unsigned ue = (unsigned)(U * (cta_id() + 1) / cta_count());
    while (u < ue) {
        const int tile = (int)(u / g.nz);
        const int k0 = (int)(u % g.nz);
        const int k1 = (int)min((unsigned)g.nz, k0 + (ue - u));
        seg(tile, k0, k1);
        u += (unsigned)(k1 - k0);
    }
}

// Visit every own cell of this CTA's segments, plane by plane: compute thread
// t owns the quad x = x0 + 4 (t % 8) .. + 3 in row y0 + t / 8 of each tile.
// The copy warp visits nothing.
template <class CellFn>
__device__ __forceinline__ void for_cells(const Geo& g, CellFn f) {
    if (threadIdx.x >= NCT) return;
    const int qx = threadIdx.x % (TX / QX), row = threadIdx.x / (TX / QX);
    for_segments(g, [&](int tile, int k0, int k1) {
        const int xq = (tile % g.tiles_x) * TX + qx * QX, y = (tile / g.tiles_x) * TY + row;
        if (y >= g.ny || xq >= g.nx) return;
        unsigned cb = (unsigned)k0 * g.S + (unsigned)y * g.nx + xq;
        for (int k = k0; k < k1; ++k, cb += g.S) {
#pragma unroll
            for (int j = 0; j < QX; ++j)
                if (xq + j < g.nx) f(k, cb + j, xq + j, y);
        }
    });
}

// ------------------------------------------------------------ TMA staging
// A stage holds one plane of a tile in six slots of one halo box each: a
// 40 x 34 box at (x0 - 4, y0 - 1), the tile with a one-cell halo, widened on
// the left to keep the copy 16-byte aligned.  Arrays that a pass reads
// together sit in consecutive slots and arrive in one 4D copy (u, ws, ss;
// the hi and lo halves of a state; p and delta, whose own-cell 32 x 32 boxes
// share the last two slots).  Cells outside the grid arrive as zeros, which
// is exactly a zero-flux wall (their face values are zero); with periodic
// walls the wrapped cells are patched in (wrap_patch).  The path serves grids
// with nx % 4 == 0 (row pitch a
// multiple of 16 bytes).  Every stencil pass of a solve is staged this way;
// only what the slots hold differs (PassKind).
constexpr int NS = 6;                         // stages
constexpr int HB = TX + 8, HR = TY + 2;       // halo box
constexpr int SZ_H = HB * HR * 4;             // 5440
constexpr int SZ_O = TX * TY * 4;             // 4096
constexpr int al128(int b) { return (b + 127) & ~127; }
// Every copy lands on a 128-byte boundary (the TMA requirement for its
// shared-memory destination); the boxes of one 4D copy follow each other
// densely.  Slots 0-2: one copy of up to three halo boxes; slot 3: alpha;
// slots 4-5: a second pair (mu hi, lo), or the own-cell boxes p and delta.
constexpr int OFF_A = al128(3 * SZ_H);        // 16384
constexpr int OFF_B = al128(OFF_A + SZ_H);    // 21888
constexpr int OFF_P = OFF_B, OFF_D = OFF_B + SZ_O;
constexpr int STAGE_BYTES = al128(OFF_B + 2 * SZ_H);
constexpr int DYN_SMEM = NS * STAGE_BYTES + 128;   // + alignment slack
__device__ __forceinline__ constexpr int sl(int s) {
    return s < 3 ? s * SZ_H : (s == 3 ? OFF_A : OFF_B + (s - 4) * SZ_H);
}
static_assert(OFF_A % 128 == 0 && OFF_B % 128 == 0 && STAGE_BYTES % 128 == 0, "TMA destinations");
static_assert(OFF_D + SZ_O <= STAGE_BYTES && sl(5) + SZ_H <= STAGE_BYTES, "stage layout");

// What the slots of a staged pass hold.
enum PassKind : int {
    kIter,    // 0 u_i, 1 ws_i, 2 ss_{i-1}, 3 alpha, 4-5 p and delta (own boxes)
    kInit1,   // 0 start hi, 1 start lo, 3 alpha, 4-5 p and delta (own boxes; delta = d when used)
    kInit2,   // 0 u_0, 3 alpha
    kGrad,    // 0 T hi, 1 T lo, 3 alpha, 4 mu hi, 5 mu lo
    kJacobi,  // 0-2 u, ws, ss of set 0 (u0 and the two sweep buffers), 3 alpha
    kInitC    // 0 delta (= d), 3 alpha, 4 the carried residual sig[cur] (own box)
};
struct PassIn {
    int kind;
    int cur;          // kIter: ping-pong index of the inputs
    bool first;       // kIter: first iteration (ss and p are not read)
    unsigned zx, zm;  // slab half of the state read (x0, or T) and of mu
    int hu;           // kInit1: 0 = the start is x0 itself; > 0 = the start is y = x0 + d with d in delta
};
__device__ __forceinline__ unsigned pass_bytes(const PassIn& in) {
    switch (in.kind) {
        case kIter: return 4 * SZ_H + 2 * SZ_O;
        case kInit1: return 3 * SZ_H + (in.hu > 0 ? 2 * SZ_O : 0);
        case kInit2: return 2 * SZ_H;
        case kJacobi: return 4 * SZ_H;
        case kInitC: return 2 * SZ_H + SZ_O;
        default: return 5 * SZ_H;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar) : "memory");
}
// Bounded wait for the completion of the mbarrier phase of the given parity;
// false after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity) {
    unsigned long long t0 = 0;
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((i & 63u) == 63u) {
            const unsigned long long t = now_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kBarrierTimeoutNs) return false;
        }
    }
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar) : "memory");
}
// Bring a descriptor into the descriptor cache ahead of its first use.
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// The stage ring.  Planes are copied and consumed in the same order (the
// for_segments order, pass after pass), so a stage index that advances by one
// (mod NS) and one parity bit per stage describe each side.  A stage's full
// barrier completes when its copies land; its empty barrier when all CW
// compute warps are done with it.
struct Ring {
    unsigned char* base;   // NS stages, 128-byte aligned
    uint32_t full0;        // shared addresses of the NS full / NS empty mbarriers
    uint32_t empty0;
    // copy side (lane 0 of the copy warp)
    unsigned ps;           // stage of the next copy
    unsigned pph;          // bit s: parity of the next empty-wait on stage s
    unsigned fiss;         // bit s: number of copies issued into stage s, mod 2
    unsigned used;         // bit s: stage s has received a copy
    // compute side (same in every compute thread)
    unsigned cs;           // stage of the next full-wait
    unsigned cph;          // bit s: parity of the next full-wait on stage s
};

__device__ __forceinline__ unsigned ring_next(unsigned s) { return s + 1 == NS ? 0u : s + 1; }

__device__ Ring make_ring(unsigned char* dyn, unsigned long long* full, unsigned long long* empty, bool init) {
    Ring R;
    R.base = (unsigned char*)(((uintptr_t)dyn + 127) & ~(uintptr_t)127);
    R.full0 = smem_u32(full);
    R.empty0 = smem_u32(empty);
    R.ps = 0;
    R.pph = (1u << NS) - 1;   // a fresh barrier's preceding phase counts as complete
    R.fiss = 0;
    R.used = 0;
    R.cs = 0;
    R.cph = 0;
    if (init) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < NS; ++i) {
                mbar_init(R.full0 + 8u * i, 1u);
                mbar_init(R.empty0 + 8u * i, (unsigned)CW);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
    }
    return R;
}

// Planes one pass copies into this CTA's ring: every plane of every segment,
// with the plane below and above each segment.
__device__ __forceinline__ int pass_planes(const Geo& g) {
    int n = 0;
    for_segments(g, [&](int, int k0, int k1) {
        n += (k1 < g.nz ? k1 : g.nz - 1) - (k0 > 0 ? k0 - 1 : 0) + 1;
    });
    return n;
}

// Copy side of one staged pass (lane 0 of the copy warp): planes [from, to)
// of the pass, in ring order.  Returns false if a stage did not come free in
// time.
__device__ bool produce(const Common& C, Ring& R, const PassIn& in, int from, int to) {
    const Geo& g = C.g;
    const TmaMaps* M = &C.maps;
    const unsigned bytes = pass_bytes(in);
    bool ok = true;
    int idx = 0;
    for_segments(g, [&](int tile, int k0, int k1) {
        if (!ok) return;
        const int x0 = (tile % g.tiles_x) * TX, y0 = (tile / g.tiles_x) * TY;
        const int kl = k0 > 0 ? k0 - 1 : 0, kh = k1 < g.nz ? k1 : g.nz - 1;
        for (int k = kl; k <= kh; ++k, ++idx) {
            if (idx < from) continue;
            if (idx >= to) return;
            const unsigned st = R.ps;
            if (!mbar_wait(R.empty0 + 8u * st, (R.pph >> st) & 1u)) { ok = false; return; }
            R.pph ^= 1u << st;
            const uint32_t dst = smem_u32(R.base + st * STAGE_BYTES), bar = R.full0 + 8u * st;
            mbar_expect_tx(bar, bytes);
            const int xh = x0 - 4, yh = y0 - 1;
            switch (in.kind) {
                case kIter:
                    tma_load4(dst, &M->uws[in.cur], xh, yh, k, 0, bar);
                    tma_load3(dst + OFF_A, &M->alpha, xh, yh, k, bar);
                    tma_load4(dst + OFF_P, &M->pd, x0, y0, k, 0, bar);
                    break;
                case kInit1:
                    tma_load4(dst, &M->states, xh, yh, k, (int)in.zx, bar);
                    tma_load3(dst + OFF_A, &M->alpha, xh, yh, k, bar);
                    if (in.hu > 0) tma_load4(dst + OFF_P, &M->pd, x0, y0, k, 0, bar);
                    break;
                case kInit2:
                    tma_load3(dst, &M->u0, xh, yh, k, bar);
                    tma_load3(dst + OFF_A, &M->alpha, xh, yh, k, bar);
                    break;
                case kJacobi:
                    tma_load4(dst, &M->uws[0], xh, yh, k, 0, bar);
                    tma_load3(dst + OFF_A, &M->alpha, xh, yh, k, bar);
                    break;
                case kInitC:
                    tma_load3(dst, &M->dh, xh, yh, k, bar);
                    tma_load3(dst + OFF_A, &M->alpha, xh, yh, k, bar);
                    tma_load4(dst + OFF_P, &M->sg, x0, y0, k, in.cur, bar);
                    break;
                default:
                    tma_load4(dst, &M->states, xh, yh, k, (int)in.zx, bar);
                    tma_load3(dst + OFF_A, &M->alpha, xh, yh, k, bar);
                    tma_load4(dst + OFF_B, &M->states, xh, yh, k, (int)in.zm, bar);
                    break;
            }
            R.fiss ^= 1u << st;
            R.used |= 1u << st;
            R.ps = ring_next(st);
        }
    });
    return ok;
}

// After a failure: wait (again bounded) for the latest copy into every stage,
// so no copy is landing in shared memory when the kernel exits.
__device__ void drain(Ring& R) {
    for (int s = 0; s < NS; ++s)
        if (R.used >> s & 1u) mbar_wait(R.full0 + 8u * s, ((R.fiss >> s) & 1u) ^ 1u);
}

// ---- periodic lateral walls on the staged path.  The halo boxes arrive with
// zeros beyond the grid (a zero-flux wall).  With periodic walls the cells a
// thread reads across a lateral wall are fetched from the opposite edge by
// that thread itself, straight into the stage (cp.async from global, no
// registers held), right after the stage lands and one plane before it is
// worked on; cp_wait() precedes the plane's work.  Only the thread that reads
// a patched position writes it (the halo row above row 0, the one below the
// last row, the column left of x = 0 and right of x = nx - 1), and corner
// cells are never read by the 7-point stencil.
__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Global array staged in halo slot j of a pass (null if the slot holds no
// halo box for this kind of pass).
__device__ __forceinline__ const float* halo_src(const Common& C, const PassIn& in, int j) {
    const size_t N = (size_t)C.g.S * C.g.nz;
    if (j == 3) return C.alpha;
    switch (in.kind) {
        case kIter: return j < 3 ? C.v.u[in.cur] + (size_t)j * N : nullptr;
        case kJacobi: return j < 3 ? C.v.u[0] + (size_t)j * N : nullptr;
        case kInit2: return j == 0 ? C.v.u[0] : nullptr;
        case kInitC: return j == 0 ? C.v.delta : nullptr;
        case kInit1: return j < 2 ? C.slab + (size_t)(in.zx + j) * N : nullptr;
        default:   // kGrad: T (hi, lo) in slots 0-1, mu (hi, lo) in slots 4-5, slot 2 unused
            if (j < 2) return C.slab + (size_t)(in.zx + j) * N;
            if (j >= 4) return C.slab + (size_t)(in.zm + (j - 4)) * N;
            return nullptr;
    }
}

// The wrapped halo cells this thread reads on plane k (stage st), requested
// by cp.async.  (xq, y): the thread's first cell; valid: it has cells.
__device__ __forceinline__ void wrap_patch(const Common& C, const PassIn& in, const unsigned char* st, int k, int xq,
                                           int y, bool valid, int hb) {
    const Geo& g = C.g;
    if (!valid) return;
    const bool top = g.py && y == 0, bot = g.py && y == g.ny - 1;
    const bool lft = g.px && xq == 0, rgt = g.px && xq + QX == g.nx;
    if (!(top || bot || lft || rgt)) return;
    const size_t plane = (size_t)k * g.S;
    const uint32_t base = smem_u32(st);
    const int nslot = in.kind == kGrad ? 6 : 4;
    for (int j = 0; j < nslot; ++j) {
        const float* src = halo_src(C, in, j);
        if (!src) continue;
        src += plane;
        const uint32_t sb = base + (uint32_t)sl(j);
        if (top) {
            const float* q = src + (size_t)(g.ny - 1) * g.nx + xq;
            if constexpr (QX == 4) cp_async16(sb + 4u * (hb - HB), q);
            else for (int t = 0; t < QX; ++t) cp_async4(sb + 4u * (hb - HB + t), q + t);
        }
        if (bot) {
            const float* q = src + xq;
            if constexpr (QX == 4) cp_async16(sb + 4u * (hb + HB), q);
            else for (int t = 0; t < QX; ++t) cp_async4(sb + 4u * (hb + HB + t), q + t);
        }
        if (lft) cp_async4(sb + 4u * (hb - 1), src + (size_t)y * g.nx + (g.nx - 1));
        if (rgt) cp_async4(sb + 4u * (hb + QX), src + (size_t)y * g.nx);
    }
}

// Compute side of one staged pass: walk the same planes in the same order,
// waiting for each stage and handing it back once every warp is done with it.
// A compute thread owns the quad at halo-box index hb (own-box index ob).
// Body holds the thread's values of the own quad on planes k-1, k, k+1:
//   reset()            segment start;      below(st)  plane k0 - 1;
//   own(st, has_below) plane k0;           above(st)  plane k + 1;
//   top()              no plane above k;   shift()    k -> k + 1;
//   plane(k, c, valid, st, st1) the work on plane k (st1: the stage of plane
//                      k + 1, or null at the top).
// kWrap: periodic lateral walls, the wrapped halo cells are patched in (a
// separate instantiation, so the zero-flux path carries none of its code).
template <bool kWrap, class Body>
__device__ bool consume(const Common& C, const PassIn& in, Ring& R, Body& B) {
    const Geo& g = C.g;
    const int lane = threadIdx.x & 31, qx = threadIdx.x % (TX / QX), row = threadIdx.x / (TX / QX);
    const int hb = (row + 1) * HB + 4 + QX * qx;
    const int ob = row * TX + QX * qx;
    constexpr bool wrap = kWrap;
    bool ok = true;
    auto wait = [&]() -> int {
        const unsigned st = R.cs;
        const bool done = mbar_wait(R.full0 + 8u * st, (R.cph >> st) & 1u);
        R.cph ^= 1u << st;
        R.cs = ring_next(st);
        return done ? (int)st : -1;
    };
    auto release = [&](int st) {
        // generic-proxy writes into the stage (the wrap patches) before the
        // next TMA copy into it
        if constexpr (wrap) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(R.empty0 + 8u * st);
    };
    auto stage = [&](int st) -> const unsigned char* { return R.base + (unsigned)st * STAGE_BYTES; };
    for_segments(g, [&](int tile, int k0, int k1) {
        if (!ok) return;
        const int xq = (tile % g.tiles_x) * TX + QX * qx, y = (tile / g.tiles_x) * TY + row;
        const bool valid = xq < g.nx && y < g.ny;   // nx % 4 == 0: a thread's cells are all in or all out
        B.reset();
        if (k0 > 0) {
            const int s = wait();
            if (s < 0) { ok = false; return; }
            B.below(stage(s), hb);
            release(s);
        }
        int sk = wait();
        if (sk < 0) { ok = false; return; }
        if constexpr (wrap) wrap_patch(C, in, stage(sk), k0, xq, y, valid, hb);
        B.own(stage(sk), hb, k0 > 0);
        unsigned c = (unsigned)k0 * g.S + (unsigned)y * g.nx + xq;
        for (int k = k0; k < k1; ++k, c += g.S) {
            int sk1 = -1;
            if (k + 1 < g.nz) {
                sk1 = wait();
                if (sk1 < 0) { ok = false; return; }
                B.above(stage(sk1), hb);
            } else {
                B.top();
            }
            if constexpr (wrap) {   // plane k's patches land; plane k + 1's are requested behind this plane's work
                cp_wait();
                if (sk1 >= 0 && k + 1 < k1) wrap_patch(C, in, stage(sk1), k + 1, xq, y, valid, hb);
            }
            B.plane(k, c, valid, stage(sk), sk1 >= 0 ? stage(sk1) : nullptr, hb, ob);
            release(sk);
            B.shift();
            sk = sk1;
        }
        if (sk >= 0 && k1 < g.nz) release(sk);   // the plane above the segment
    });
    return ok;
}

__device__ __forceinline__ float lds1(const unsigned char* st, int off, int i) {
    return *reinterpret_cast<const float*>(st + off + 4 * i);
}
// The QX values of a thread's cells (or of the QX cells at halo-box index i):
// one 8- or 16-byte shared load, one global store.
__device__ __forceinline__ void ldq(const unsigned char* st, int off, int i, float (&v)[QX]) {
    if constexpr (QX == 4) {
        const float4 q = *reinterpret_cast<const float4*>(st + off + 4 * i);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const float2 q = *reinterpret_cast<const float2*>(st + off + 4 * i);
        v[0] = q.x; v[1] = q.y;
    }
}
__device__ __forceinline__ void stgq(float* p, const float (&v)[QX]) {
    if constexpr (QX == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
__device__ __forceinline__ void setq(float (&d)[QX], float v) {
#pragma unroll
    for (int j = 0; j < QX; ++j) d[j] = v;
}
__device__ __forceinline__ void cpyq(float (&d)[QX], const float (&s)[QX]) {
#pragma unroll
    for (int j = 0; j < QX; ++j) d[j] = s[j];
}

// Lateral face values of the own quad from the staged alpha (slot 3):
// cx[j] is the face between cells j - 1 and j of the quad (j = 0..4, cell -1
// and cell 4 being the neighbours left and right of it); cyp / cym the +y / -y
// faces of each cell.  Shared faces are evaluated once: face(a, b) and
// face(b, a) are the same number.
__device__ __forceinline__ void quad_faces(const unsigned char* st, int hb, const float (&ac)[QX], float kx, float ky,
                                           float (&cx)[QX + 1], float (&cyp)[QX], float (&cym)[QX]) {
    float aym[QX], ayp[QX];
    ldq(st, sl(3), hb - HB, aym);
    ldq(st, sl(3), hb + HB, ayp);
    cx[0] = face(ac[0], lds1(st, sl(3), hb - 1), kx);
#pragma unroll
    for (int j = 1; j < QX; ++j) cx[j] = face(ac[j - 1], ac[j], kx);
    cx[QX] = face(ac[QX - 1], lds1(st, sl(3), hb + QX), kx);
#pragma unroll
    for (int j = 0; j < QX; ++j) {
        cyp[j] = face(ac[j], ayp[j], ky);
        cym[j] = face(ac[j], aym[j], ky);
    }
}

// CG step scalars of one iteration pass.
struct Step {
    float a, bt;
    bool first;
    // s_i = ws_i + beta ss_{i-1} and u_{i+1} = u_i - alpha s_i at one cell; every
    // thread that needs u_{i+1} at a cell evaluates exactly these two FMAs.
    __device__ __forceinline__ float sdir(float w, float s) const { return first ? w : fmaf(bt, s, w); }
    __device__ __forceinline__ float next(float u, float sn) const { return fmaf(-a, sn, u); }
};

// u_{i+1} (f), s_i (sn) and u_i (u) at the quad at halo-box index h of a stage.
__device__ __forceinline__ void fieldq(const unsigned char* st, int h, const Step& S, float (&f)[QX], float (&sn)[QX],
                                       float (&u)[QX]) {
    float w[QX], s[QX] = {};
    ldq(st, sl(0), h, u);
    ldq(st, sl(1), h, w);
    if (!S.first) ldq(st, sl(2), h, s);
#pragma unroll
    for (int j = 0; j < QX; ++j) {
        sn[j] = S.sdir(w[j], s[j]);
        f[j] = S.next(u[j], sn[j]);
    }
}
__device__ __forceinline__ void fieldq(const unsigned char* st, int h, const Step& S, float (&f)[QX]) {
    float sn[QX], u[QX];
    fieldq(st, h, S, f, sn, u);
}
__device__ __forceinline__ float field1(const unsigned char* st, int h, const Step& S) {
    const float sv = S.first ? 0.f : lds1(st, sl(2), h);
    return S.next(lds1(st, sl(0), h), S.sdir(lds1(st, sl(1), h), sv));
}

// ---- one CG iteration: u_{i+1}, ws_{i+1} = M^{-1} A u_{i+1}, ss_i, p_i, delta
// kPred: also the five sums that give the next iteration's residual norm
// before its pass (see solve()): with r = D u_{i+1}, e = D ws_{i+1} = A u_{i+1}
// and t = D s_i, q = (r.e, r.t, e.e, e.t, t.t), per thread in plain FP32 (the
// expansion they feed is accurate well past what its use needs).
template <bool kPred = false>
struct IterBody {
    const Common& C;
    const Step& S;
    int cur;
    Acc<3>& acc;
    float* q = nullptr;                      // kPred: [5] per-thread sums
    float fm[QX], am[QX];                    // plane k-1: u_{i+1}, alpha
    float fc[QX], sc[QX], uc[QX], ac[QX];      // plane k: u_{i+1}, s_i, u_i, alpha
    float fp[QX], sp[QX], up[QX], ap[QX];      // plane k+1
    float czm[QX], czp[QX];                  // -z / +z faces of the own cells
    __device__ IterBody(const Common& c, const Step& s, int cu, Acc<3>& a, float* q5 = nullptr)
        : C(c), S(s), cur(cu), acc(a), q(q5) {}
    __device__ __forceinline__ void reset() { setq(fm, 0.f); setq(am, 0.f); setq(czm, 0.f); }
    __device__ __forceinline__ void below(const unsigned char* st, int hb) {
        fieldq(st, hb, S, fm);
        ldq(st, sl(3), hb, am);
    }
    __device__ __forceinline__ void own(const unsigned char* st, int hb, bool has_below) {
        fieldq(st, hb, S, fc, sc, uc);
        ldq(st, sl(3), hb, ac);
        if (has_below) {
#pragma unroll
            for (int j = 0; j < QX; ++j) czm[j] = face(ac[j], am[j], C.kz);
        }
    }
    __device__ __forceinline__ void above(const unsigned char* st, int hb) {
        fieldq(st, hb, S, fp, sp, up);
        ldq(st, sl(3), hb, ap);
#pragma unroll
        for (int j = 0; j < QX; ++j) czp[j] = face(ac[j], ap[j], C.kz);
    }
    __device__ __forceinline__ void top() {
        cpyq(fp, fc);
        setq(sp, 0.f); setq(up, 0.f); setq(ap, 0.f); setq(czp, 0.f);
    }
    __device__ __forceinline__ void plane(int k, unsigned c, bool valid, const unsigned char* st,
                                          const unsigned char*, int hb, int ob) {
        const Geo& g = C.g;
        float fym[QX], fyp[QX], cx[QX + 1], cyp[QX], cym[QX];
        fieldq(st, hb - HB, S, fym);
        fieldq(st, hb + HB, S, fyp);
        const float fxl = field1(st, hb - 1, S), fxr = field1(st, hb + QX, S);
        quad_faces(st, hb, ac, C.kx, C.ky, cx, cyp, cym);
        float pp[QX] = {}, dd[QX];
        if (!S.first) ldq(st, OFF_P, ob, pp);
        ldq(st, OFF_D, ob, dd);
        const float rob = k + 1 == g.nz ? C.robin : 0.f;
        float wn[QX], pn[QX], dl[QX], s0 = 0.f, s1 = 0.f, s2 = 0.f;
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            const float f = fc[j];
            const float fxm = j > 0 ? fc[j - 1] : fxl, fxp = j < QX - 1 ? fc[j + 1] : fxr;
            const float fzmv = k > 0 ? fm[j] : f;
            const float cxp = cx[j + 1], cxm = cx[j];
            const float d = diag(cxp, cxm, cyp[j], cym[j], czp[j], czm[j], rob);
            const float Au = f + cxp * (f - fxp) + cxm * (f - fxm) + cyp[j] * (f - fyp[j]) + cym[j] * (f - fym[j]) +
                             czp[j] * (f - fp[j]) + czm[j] * (f - fzmv) + rob * f;
            wn[j] = rcp_approx(d) * Au;
            pn[j] = S.first ? uc[j] : fmaf(S.bt, pp[j], uc[j]);
            dl[j] = fmaf(S.a, pn[j], dd[j]);
            const float r = d * f;
            s0 += r * f;
            s1 += Au * f;
            s2 += r * r;
            if constexpr (kPred) {   // e = D ws_{i+1} = A u_{i+1}
                const float e = Au, t = d * sc[j];
                q0 = fmaf(r, e, q0);
                q1 = fmaf(r, t, q1);
                q2 = fmaf(e, e, q2);
                q3 = fmaf(e, t, q3);
                q4 = fmaf(t, t, q4);
            }
        }
        if (valid) {
            stgq(C.v.p + c, pn);
            stgq(C.v.delta + c, dl);
            stgq(C.v.u[cur ^ 1] + c, fc);
            stgq(C.v.ws[cur ^ 1] + c, wn);
            stgq(C.v.ss[cur ^ 1] + c, sc);
            acc.add(0, s0);
            acc.add(1, s1);
            acc.add(2, s2);
            if constexpr (kPred) {
                q[0] += q0; q[1] += q1; q[2] += q2; q[3] += q3; q[4] += q4;
            }
        }
    }
    __device__ __forceinline__ void shift() {
        cpyq(fm, fc); cpyq(czm, czp);
        cpyq(fc, fp); cpyq(sc, sp); cpyq(uc, up); cpyq(ac, ap);
    }
};

// The flux term cf ((hc + lc) - (hq + lq)) of a face as pr + pe: the high
// difference by TwoSum, the product by TwoProd through fmaf; pr is its
// rounded value.  The same face seen from the other cell gives exactly
// (-pr, -pe) (TwoSum's error is unique, and negation is exact), so a face
// between two cells of one thread is formed once.
struct FaceTerm {
    float pr, pe;
};
__device__ __forceinline__ FaceTerm face_term(float cf, float hc, float lc, float hq, float lq) {
    float dh, dhe;
    two_sum(hc, -hq, dh, dhe);
    const float dl = (lc - lq) + dhe;
    const float pr = cf * dh;
    return FaceTerm{pr, fmaf(cf, dh, -pr) + cf * dl};
}
__device__ __forceinline__ FaceTerm neg(FaceTerm f) { return FaceTerm{-f.pr, -f.pe}; }
// sh + sl += pr + pe, error-free up to the final rounding (a zero face adds nothing).
__device__ __forceinline__ void add_term(FaceTerm f, float& sh, float& sl) {
    float t, te;
    two_sum(sh, f.pr, t, te);
    sh = t;
    sl += te + f.pe;
}
// sh + sl += cf ((hc + lc) - (hq + lq)) for a face of one cell.
__device__ __forceinline__ void exact_term(float cf, float hc, float lc, float hq, float lq, float& sh, float& sl) {
    if (cf == 0.f) return;
    add_term(face_term(cf, hc, lc, hq, lq), sh, sl);
}
// sh + sl += rob (hc + lc), the Robin sink, the same way.
__device__ __forceinline__ void exact_sink(float rob, float hc, float lc, float& sh, float& sl) {
    if (rob == 0.f) return;
    const float pr = rob * hc;
    const float pe = fmaf(rob, hc, -pr) + rob * lc;
    float t, te;
    two_sum(sh, pr, t, te);
    sh = t;
    sl += te + pe;
}

// ---- init 1: the residual of the start y = x0 + d (d = 0 or the predicted
// increment, see add_state), r0 = e - d - (A - I) y, formed error-free up to
// its final rounding: (A - I) y from the compensated pairs y through TwoProd /
// TwoSum, then d by TwoSum, so r0 is accurate relative to itself however small
// it is against x0 or d.  u0 = M^{-1} r0; delta = d (already there when d != 0).
template <class RhsFn>
struct Init1Body {
    const Common& C;
    RhsFn& rhs;
    Acc<3>& acc;
    int hu;                            // 0: y = x0, d = 0
    float hm[QX], lm[QX], am[QX];         // plane k-1: y as (hi, lo), alpha
    float hc[QX], lc[QX], ac[QX];
    float hp[QX], lp[QX], ap[QX];
    float czm[QX], czp[QX];
    FaceTerm zdn[QX];                   // the -z face terms of plane k (the +z ones of plane k-1, negated)
    __device__ Init1Body(const Common& c, RhsFn& r, Acc<3>& a, int hu_) : C(c), rhs(r), acc(a), hu(hu_) {}
    __device__ __forceinline__ void reset() {
        setq(hm, 0.f); setq(lm, 0.f); setq(am, 0.f); setq(czm, 0.f);
#pragma unroll
        for (int j = 0; j < QX; ++j) zdn[j] = FaceTerm{0.f, 0.f};
    }
    __device__ __forceinline__ void below(const unsigned char* st, int hb) {
        ldq(st, sl(0), hb, hm);
        ldq(st, sl(1), hb, lm);
        ldq(st, sl(3), hb, am);
    }
    __device__ __forceinline__ void own(const unsigned char* st, int hb, bool has_below) {
        ldq(st, sl(0), hb, hc);
        ldq(st, sl(1), hb, lc);
        ldq(st, sl(3), hb, ac);
        if (has_below) {
#pragma unroll
            for (int j = 0; j < QX; ++j) {
                czm[j] = face(ac[j], am[j], C.kz);
                zdn[j] = face_term(czm[j], hc[j], lc[j], hm[j], lm[j]);
            }
        }
    }
    __device__ __forceinline__ void above(const unsigned char* st, int hb) {
        ldq(st, sl(0), hb, hp);
        ldq(st, sl(1), hb, lp);
        ldq(st, sl(3), hb, ap);
#pragma unroll
        for (int j = 0; j < QX; ++j) czp[j] = face(ac[j], ap[j], C.kz);
    }
    __device__ __forceinline__ void top() { setq(hp, 0.f); setq(lp, 0.f); setq(ap, 0.f); setq(czp, 0.f); }
    __device__ __forceinline__ void plane(int k, unsigned c, bool valid, const unsigned char* st,
                                          const unsigned char*, int hb, int ob) {
        if (!valid) return;
        const Geo& g = C.g;
        float hym[QX], lym[QX], hyp[QX], lyp[QX], cx[QX + 1], cyp[QX], cym[QX], d[QX] = {};
        ldq(st, sl(0), hb - HB, hym);
        ldq(st, sl(1), hb - HB, lym);
        ldq(st, sl(0), hb + HB, hyp);
        ldq(st, sl(1), hb + HB, lyp);
        if (hu > 0) ldq(st, OFF_D, ob, d);
        const float hxl = lds1(st, sl(0), hb - 1), lxl = lds1(st, sl(1), hb - 1);
        const float hxr = lds1(st, sl(0), hb + QX), lxr = lds1(st, sl(1), hb + QX);
        quad_faces(st, hb, ac, C.kx, C.ky, cx, cyp, cym);
        const float rob = k + 1 == g.nz ? C.robin : 0.f;
        // x faces: X[f] between cells f - 1 and f seen from the left (f = 1..3),
        // X[0] / X[QX] the outer faces seen from cells 0 / 3
        FaceTerm X[QX + 1];
        X[0] = face_term(cx[0], hc[0], lc[0], hxl, lxl);
#pragma unroll
        for (int f = 1; f < QX; ++f) X[f] = face_term(cx[f], hc[f - 1], lc[f - 1], hc[f], lc[f]);
        X[QX] = face_term(cx[QX], hc[QX - 1], lc[QX - 1], hxr, lxr);
        float u[QX], s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            float sh = 0.f, sx = 0.f;
            const FaceTerm zup = face_term(czp[j], hc[j], lc[j], hp[j], lp[j]);
            add_term(X[j + 1], sh, sx);
            add_term(j > 0 ? neg(X[j]) : X[0], sh, sx);
            exact_term(cyp[j], hc[j], lc[j], hyp[j], lyp[j], sh, sx);
            exact_term(cym[j], hc[j], lc[j], hym[j], lym[j], sh, sx);
            add_term(zup, sh, sx);
            add_term(zdn[j], sh, sx);
            zdn[j] = neg(zup);   // the -z term of the cell above
            exact_sink(rob, hc[j], lc[j], sh, sx);
            if (hu > 0) {   // + d
                float t, te;
                two_sum(sh, d[j], t, te);
                sh = t;
                sx += te;
            }
            const float e = rhs(c + j, k);
            const float r = (e - sh) - sx;
            u[j] = rcp_approx(diag(cx[j + 1], cx[j], cyp[j], cym[j], czp[j], czm[j], rob)) * r;
            const float b = ((hc[j] - d[j]) + lc[j]) + e;   // x0 + e, for ||b||
            s0 += b * b;
            s1 += r * u[j];
            s2 += r * r;
        }
        acc.add(0, s0);
        acc.add(1, s1);
        acc.add(2, s2);
        stgq(C.v.u[0] + c, u);
        if (hu == 0) stgq(C.v.delta + c, d);
    }
    __device__ __forceinline__ void shift() {
        cpyq(hm, hc); cpyq(lm, lc); cpyq(czm, czp);
        cpyq(hc, hp); cpyq(lc, lp); cpyq(ac, ap);
    }
};

// ---- init 2: ws0 = M^{-1} A u0 ; (A u0, u0); with q (the first
// iteration's residual-norm expansion, see IterBody): r = D u0, e = D ws0,
// q = (r.e, e.e) per thread
struct Init2Body {
    const Common& C;
    Acc<1>& acc;
    float* q;
    float um[QX], am[QX], uc[QX], ac[QX], up[QX], ap[QX], czm[QX], czp[QX];
    __device__ Init2Body(const Common& c, Acc<1>& a, float* q2 = nullptr) : C(c), acc(a), q(q2) {}
    __device__ __forceinline__ void reset() { setq(um, 0.f); setq(am, 0.f); setq(czm, 0.f); }
    __device__ __forceinline__ void below(const unsigned char* st, int hb) {
        ldq(st, sl(0), hb, um);
        ldq(st, sl(3), hb, am);
    }
    __device__ __forceinline__ void own(const unsigned char* st, int hb, bool has_below) {
        ldq(st, sl(0), hb, uc);
        ldq(st, sl(3), hb, ac);
        if (has_below) {
#pragma unroll
            for (int j = 0; j < QX; ++j) czm[j] = face(ac[j], am[j], C.kz);
        }
    }
    __device__ __forceinline__ void above(const unsigned char* st, int hb) {
        ldq(st, sl(0), hb, up);
        ldq(st, sl(3), hb, ap);
#pragma unroll
        for (int j = 0; j < QX; ++j) czp[j] = face(ac[j], ap[j], C.kz);
    }
    __device__ __forceinline__ void top() { setq(up, 0.f); setq(ap, 0.f); setq(czp, 0.f); }
    __device__ __forceinline__ void plane(int k, unsigned c, bool valid, const unsigned char* st,
                                          const unsigned char*, int hb, int) {
        if (!valid) return;
        float uym[QX], uyp[QX], cx[QX + 1], cyp[QX], cym[QX], w[QX], qe = 0.f, qq = 0.f;
        ldq(st, sl(0), hb - HB, uym);
        ldq(st, sl(0), hb + HB, uyp);
        const float uxl = lds1(st, sl(0), hb - 1), uxr = lds1(st, sl(0), hb + QX);
        quad_faces(st, hb, ac, C.kx, C.ky, cx, cyp, cym);
        const float rob = k + 1 == C.g.nz ? C.robin : 0.f;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            const float f = uc[j];
            const float fxm = j > 0 ? uc[j - 1] : uxl, fxp = j < QX - 1 ? uc[j + 1] : uxr;
            const float cxp = cx[j + 1], cxm = cx[j];
            const float Au = f + cxp * (f - fxp) + cxm * (f - fxm) + cyp[j] * (f - uyp[j]) + cym[j] * (f - uym[j]) +
                             czp[j] * (f - up[j]) + czm[j] * (f - um[j]) + rob * f;
            const float d = diag(cxp, cxm, cyp[j], cym[j], czp[j], czm[j], rob);
            w[j] = rcp_approx(d) * Au;
            acc.add(0, Au * f);
            const float r = d * f;   // and e = D ws0 = A u0
            qe = fmaf(r, Au, qe);
            qq = fmaf(Au, Au, qq);
        }
        if (q) {
            q[0] += qe;
            q[1] += qq;
        }
        stgq(C.v.ws[0] + c, w);
    }
    __device__ __forceinline__ void shift() {
        cpyq(um, uc); cpyq(czm, czp);
        cpyq(uc, up); cpyq(ac, ap);
    }
};

// ---- init 1 from the carried residual: r0 = s - A d = g - (A - I) d with
// g = s - d (carried from the solve before, see add_state) and d the
// predicted increment (in delta, staged with its halo); (A - I) d in plain
// FP32.  g and (A - I) d are small against d when the prediction is good and
// the field smooth, and the rounding of r0 is relative to them, not to d.
// u0 = M^{-1} r0; the sums (r0, u0), (r0, r0) join the carried ||b||^2 of
// the state update.
struct InitCBody {
    const Common& C;
    Acc<3>& acc;
    float dm[QX], am[QX], dc[QX], ac[QX], dp[QX], ap[QX], czm[QX], czp[QX];
    __device__ InitCBody(const Common& c, Acc<3>& a) : C(c), acc(a) {}
    __device__ __forceinline__ void reset() { setq(dm, 0.f); setq(am, 0.f); setq(czm, 0.f); }
    __device__ __forceinline__ void below(const unsigned char* st, int hb) {
        ldq(st, sl(0), hb, dm);
        ldq(st, sl(3), hb, am);
    }
    __device__ __forceinline__ void own(const unsigned char* st, int hb, bool has_below) {
        ldq(st, sl(0), hb, dc);
        ldq(st, sl(3), hb, ac);
        if (has_below) {
#pragma unroll
            for (int j = 0; j < QX; ++j) czm[j] = face(ac[j], am[j], C.kz);
        }
    }
    __device__ __forceinline__ void above(const unsigned char* st, int hb) {
        ldq(st, sl(0), hb, dp);
        ldq(st, sl(3), hb, ap);
#pragma unroll
        for (int j = 0; j < QX; ++j) czp[j] = face(ac[j], ap[j], C.kz);
    }
    __device__ __forceinline__ void top() { setq(dp, 0.f); setq(ap, 0.f); setq(czp, 0.f); }
    __device__ __forceinline__ void plane(int k, unsigned c, bool valid, const unsigned char* st,
                                          const unsigned char*, int hb, int ob) {
        if (!valid) return;
        float dym[QX], dyp[QX], sv[QX], cx[QX + 1], cyp[QX], cym[QX], u[QX], s1 = 0.f, s2 = 0.f;
        ldq(st, sl(0), hb - HB, dym);
        ldq(st, sl(0), hb + HB, dyp);
        ldq(st, OFF_P, ob, sv);
        const float dxl = lds1(st, sl(0), hb - 1), dxr = lds1(st, sl(0), hb + QX);
        quad_faces(st, hb, ac, C.kx, C.ky, cx, cyp, cym);
        const float rob = k + 1 == C.g.nz ? C.robin : 0.f;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            const float f = dc[j];
            const float fxm = j > 0 ? dc[j - 1] : dxl, fxp = j < QX - 1 ? dc[j + 1] : dxr;
            const float cxp = cx[j + 1], cxm = cx[j];
            const float Ld = cxp * (f - fxp) + cxm * (f - fxm) + cyp[j] * (f - dyp[j]) + cym[j] * (f - dym[j]) +
                             czp[j] * (f - dp[j]) + czm[j] * (f - dm[j]) + rob * f;   // (A - I) d
            const float r = sv[j] - Ld;
            u[j] = rcp_approx(diag(cxp, cxm, cyp[j], cym[j], czp[j], czm[j], rob)) * r;
            s1 += r * u[j];
            s2 += r * r;
        }
        acc.add(1, s1);
        acc.add(2, s2);
        stgq(C.v.u[0] + c, u);
    }
    __device__ __forceinline__ void shift() {
        cpyq(dm, dc); cpyq(czm, czp);
        cpyq(dc, dp); cpyq(ac, ap);
    }
};

// ---- one sweep of the paper's Jacobi inner solver (App. D.2, Eq. jacobi_iter)
// on the increment delta = T - T^(0): the sweep T <- D^{-1}(b - R T) reads
// delta' = u0 + D^{-1} sum_f c_f delta_q with u0 = D^{-1} r0 (slot 0) and
// delta in slot `src` (0 for the first sweep, when delta = u0; else 1 or 2).
struct JacobiBody {
    const Common& C;
    int src;
    float* out;
    float dm[QX], am[QX], dc[QX], ac[QX], dp[QX], ap[QX], czm[QX], czp[QX];
    __device__ JacobiBody(const Common& c, int s, float* o) : C(c), src(s), out(o) {}
    __device__ __forceinline__ void reset() { setq(dm, 0.f); setq(am, 0.f); setq(czm, 0.f); }
    __device__ __forceinline__ void below(const unsigned char* st, int hb) {
        ldq(st, sl(src), hb, dm);
        ldq(st, sl(3), hb, am);
    }
    __device__ __forceinline__ void own(const unsigned char* st, int hb, bool has_below) {
        ldq(st, sl(src), hb, dc);
        ldq(st, sl(3), hb, ac);
        if (has_below) {
#pragma unroll
            for (int j = 0; j < QX; ++j) czm[j] = face(ac[j], am[j], C.kz);
        }
    }
    __device__ __forceinline__ void above(const unsigned char* st, int hb) {
        ldq(st, sl(src), hb, dp);
        ldq(st, sl(3), hb, ap);
#pragma unroll
        for (int j = 0; j < QX; ++j) czp[j] = face(ac[j], ap[j], C.kz);
    }
    __device__ __forceinline__ void top() { setq(dp, 0.f); setq(ap, 0.f); setq(czp, 0.f); }
    __device__ __forceinline__ void plane(int k, unsigned c, bool valid, const unsigned char* st,
                                          const unsigned char*, int hb, int) {
        if (!valid) return;
        float dym[QX], dyp[QX], u0[QX], cx[QX + 1], cyp[QX], cym[QX], o[QX];
        ldq(st, sl(src), hb - HB, dym);
        ldq(st, sl(src), hb + HB, dyp);
        ldq(st, sl(0), hb, u0);
        const float dxl = lds1(st, sl(src), hb - 1), dxr = lds1(st, sl(src), hb + QX);
        quad_faces(st, hb, ac, C.kx, C.ky, cx, cyp, cym);
        const float rob = k + 1 == C.g.nz ? C.robin : 0.f;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            const float sum = cx[j + 1] * (j < QX - 1 ? dc[j + 1] : dxr) + cx[j] * (j > 0 ? dc[j - 1] : dxl) +
                              cyp[j] * dyp[j] + cym[j] * dym[j] + czp[j] * dp[j] + czm[j] * dm[j];
            o[j] = fmaf(rcp_approx(diag(cx[j + 1], cx[j], cyp[j], cym[j], czp[j], czm[j], rob)), sum, u0[j]);
        }
        stgq(out + c, o);
    }
    __device__ __forceinline__ void shift() {
        cpyq(dm, dc); cpyq(czm, czp);
        cpyq(dc, dp); cpyq(ac, ap);
    }
};

// ---- gradient of one step (Eq. grad_assembly) at the own cells:
// g_c -= sum_f w_f h^2 (mu_c - mu_q)(T_c - T_q), h = alpha_q / (alpha_c + alpha_q),
// with T and mu as compensated pairs.  A face between two cells of the same
// thread (inside the quad along x, and along z between consecutive planes)
// is evaluated once for both: P = w (mu_c - mu_q)(T_c - T_q) is symmetric,
// and the two cells take P (alpha_q / s)^2 and P (alpha_c / s)^2 with
// s = alpha_c + alpha_q.  A cell beyond a zero-flux wall stages alpha_q = 0,
// so h = 0 and it adds nothing.  Plane values are read from the stages when
// needed (the stage of plane k + 1 is held while plane k is worked on); only
// the -z terms of the next plane are carried in registers, and the plane's
// accumulator is loaded before its terms are formed.
struct GradBody {
    float2* grad;          // dJ/dalpha accumulator, compensated (hi, lo) pairs
    float wx, wy, wz;
    int nz;
    unsigned S;            // cells per plane
    float bth[QX], btl[QX], bmh[QX], bml[QX], bac[QX];   // plane k0 - 1 (segment start only)
    float zdn[QX], zdn1[QX];                          // -z terms of plane k and of plane k + 1
    __device__ __forceinline__ static float term(float a0, float mc, float mcl, float tc, float tcl, float aq,
                                                 float mq, float mql, float tq, float tql, float w) {
        const float h = aq * rcp_approx(a0 + aq);
        const float dm = (mc - mq) + (mcl - mql);
        const float dT = (tc - tq) + (tcl - tql);
        return w * h * h * dm * dT;
    }
    // the face (c, q) for both cells: to_c as term(c, q), to_q as term(q, c)
    __device__ __forceinline__ static void pair(float ac, float mc, float mcl, float tc, float tcl, float aq, float mq,
                                                float mql, float tq, float tql, float w, float& to_c, float& to_q) {
        const float inv = rcp_approx(ac + aq);
        const float hc = aq * inv, hq = ac * inv;
        const float dm = (mc - mq) + (mcl - mql);
        const float dT = (tc - tq) + (tcl - tql);
        const float P = w * dm * dT;
        to_c = hc * hc * P;
        to_q = hq * hq * P;
    }
    __device__ __forceinline__ static void load(const unsigned char* st, int hb, float (&t)[QX], float (&tlo)[QX],
                                                float (&m)[QX], float (&mlo)[QX], float (&a)[QX]) {
        ldq(st, sl(0), hb, t);
        ldq(st, sl(1), hb, tlo);
        ldq(st, sl(4), hb, m);
        ldq(st, sl(5), hb, mlo);
        ldq(st, sl(3), hb, a);
    }
    __device__ __forceinline__ void reset() {}
    __device__ __forceinline__ void below(const unsigned char* st, int hb) { load(st, hb, bth, btl, bmh, bml, bac); }
    __device__ __forceinline__ void own(const unsigned char* st, int hb, bool has_below) {
        if (!has_below) return;
        float th[QX], tl[QX], mh[QX], ml[QX], ac[QX];
        load(st, hb, th, tl, mh, ml, ac);
#pragma unroll
        for (int j = 0; j < QX; ++j)
            zdn[j] = term(ac[j], mh[j], ml[j], th[j], tl[j], bac[j], bmh[j], bml[j], bth[j], btl[j], wz);
    }
    __device__ __forceinline__ void above(const unsigned char*, int) {}
    __device__ __forceinline__ void top() {}
    __device__ __forceinline__ void plane(int k, unsigned c, bool valid, const unsigned char* st,
                                          const unsigned char* st1, int hb, int) {
        if (!valid) return;
        float4 gv[QX / 2];   // the cells' accumulator pairs, two per 16-byte load
#pragma unroll
        for (int q = 0; q < QX / 2; ++q) gv[q] = *reinterpret_cast<const float4*>(grad + c + 2 * q);
        float th[QX], tl[QX], mh[QX], ml[QX], ac[QX];
        load(st, hb, th, tl, mh, ml, ac);
        float s[QX] = {};
        {   // x: the three faces inside the quad once for both cells, then the two outer faces
#pragma unroll
            for (int j = 0; j < QX - 1; ++j) {
                float a2b, b2a;
                pair(ac[j], mh[j], ml[j], th[j], tl[j], ac[j + 1], mh[j + 1], ml[j + 1], th[j + 1], tl[j + 1], wx,
                     a2b, b2a);
                s[j] += a2b;
                s[j + 1] += b2a;
            }
            const int hr = hb + QX, hl = hb - 1;
            s[QX - 1] += term(ac[QX - 1], mh[QX - 1], ml[QX - 1], th[QX - 1], tl[QX - 1], lds1(st, sl(3), hr), lds1(st, sl(4), hr),
                         lds1(st, sl(5), hr), lds1(st, sl(0), hr), lds1(st, sl(1), hr), wx);
            s[0] += term(ac[0], mh[0], ml[0], th[0], tl[0], lds1(st, sl(3), hl), lds1(st, sl(4), hl),
                         lds1(st, sl(5), hl), lds1(st, sl(0), hl), lds1(st, sl(1), hl), wx);
        }
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {   // +y, then -y
            float t[QX], tlo[QX], m[QX], mlo[QX], a[QX];
            load(st, sd == 0 ? hb + HB : hb - HB, t, tlo, m, mlo, a);
#pragma unroll
            for (int j = 0; j < QX; ++j) s[j] += term(ac[j], mh[j], ml[j], th[j], tl[j], a[j], m[j], mlo[j], t[j], tlo[j], wy);
        }
        if (st1) {   // +z, and the -z terms of plane k + 1
            float t[QX], tlo[QX], m[QX], mlo[QX], a[QX];
            load(st1, hb, t, tlo, m, mlo, a);
#pragma unroll
            for (int j = 0; j < QX; ++j) {
                float up;
                pair(ac[j], mh[j], ml[j], th[j], tl[j], a[j], m[j], mlo[j], t[j], tlo[j], wz, up, zdn1[j]);
                s[j] += up;
            }
        }
        float gh[QX], gl[QX];
#pragma unroll
        for (int q = 0; q < QX / 2; ++q) {
            gh[2 * q] = gv[q].x; gl[2 * q] = gv[q].y;
            gh[2 * q + 1] = gv[q].z; gl[2 * q + 1] = gv[q].w;
        }
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            if (k > 0) s[j] += zdn[j];
            add_pair(gh[j], gl[j], -s[j], gh[j], gl[j]);
        }
#pragma unroll
        for (int q = 0; q < QX / 2; ++q)
            *reinterpret_cast<float4*>(grad + c + 2 * q) = make_float4(gh[2 * q], gl[2 * q], gh[2 * q + 1], gl[2 * q + 1]);
    }
    __device__ __forceinline__ void shift() { cpyq(zdn, zdn1); }
};

// Compute threads: wait for the next n stages and hand them back unread
// (copies started for a pass that is not run).
__device__ bool discard(Ring& R, int n) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        const unsigned st = R.cs;
        ok = mbar_wait(R.full0 + 8u * st, (R.cph >> st) & 1u) && ok;
        R.cph ^= 1u << st;
        R.cs = ring_next(st);
        __syncwarp();
        if (lane == 0) mbar_arrive(R.empty0 + 8u * st);
    }
    return ok;
}

// One staged pass: the copy thread streams the planes (from `from` on: the
// first ones may have been started early, see Pipe), the compute threads run
// Body over them.  Returns false (CTA-uniform, with the error recorded and
// every copy landed) if a wait timed out anywhere in the CTA, or if `pre_ok`
// (the early copies) is false in any thread.
template <bool kWrap, class Body>
__device__ bool staged(const Common& C, Ring& R, const PassIn& in, Body& B, int from = 0, bool pre_ok = true) {
    bool ok = pre_ok;
    if (threadIdx.x < NCT) ok = consume<kWrap>(C, in, R, B) && ok;
    else if (threadIdx.x == NCT) ok = produce(C, R, in, from, 1 << 30) && ok;
    if (__syncthreads_or(ok ? 0 : 1)) {
        if (threadIdx.x == NCT) drain(R);
        if (threadIdx.x == 0) atomicCAS(&C.ctl->err, kDevOk, kDevTimeout);
        return false;
    }
    return true;
}

// Early copies.  Right after a grid barrier every stage of the ring is free,
// so the copy thread can start the first stages of the pass that most likely
// comes next; their latency then hides behind the reduction that follows the
// barrier.  The pass takes over with staged(..., pipe.n, pipe.ok); if it does
// not run, pipe_cancel() lets the compute threads discard the stages.
struct Pipe {
    int n;       // planes of the next pass already issued (same in every thread)
    bool ok;     // copy thread: the early issue succeeded
};
__device__ __forceinline__ Pipe pipe_none() { return Pipe{0, true}; }
constexpr int NPRE = 5;   // stages started early (5 against 3: -0.8 ms per inversion step, measured)
__device__ __forceinline__ Pipe pipe_start(const Common& C, Ring& R, const PassIn& in) {
    Pipe p{min(NPRE, pass_planes(C.g)), true};
    if (threadIdx.x == NCT) p.ok = produce(C, R, in, 0, p.n);
    return p;
}
__device__ bool pipe_cancel(const Common& C, Ring& R, const Pipe& p) {
    bool ok = p.ok;
    if (threadIdx.x < NCT) ok = discard(R, p.n) && ok;
    if (__syncthreads_or(ok ? 0 : 1)) {
        if (threadIdx.x == NCT) drain(R);
        if (threadIdx.x == 0) atomicCAS(&C.ctl->err, kDevOk, kDevTimeout);
        return false;
    }
    return true;
}

// Slab half of a state (see Common::slab); false (with the error recorded)
// if the pointer is not a state of the slab.  Uniform over the grid.
__device__ __forceinline__ bool slab_half(const Common& C, const float* p, unsigned* h) {
    const long long off = (long long)(p - C.slab);
    const long long N = (long long)C.g.S * C.g.nz;
    if (off < 0 || off % N != 0 || off / N + 2 > (long long)C.slab_halves) {
        if (threadIdx.x == 0) atomicCAS(&C.ctl->err, kDevOk, kDevBadState);
        return false;
    }
    *h = (unsigned)(off / N);
    return true;
}

// One iteration pass with plain global loads (grids TMA cannot stage).
__device__ void plain_pass(const Common& C, int cur, const Step& S, Acc<3>& acc) {
    const Geo& g = C.g;
    const float* __restrict__ ui = C.v.u[cur];
    const float* __restrict__ wi = C.v.ws[cur];
    const float* __restrict__ si = C.v.ss[cur];
    float* __restrict__ uo = C.v.u[cur ^ 1];
    float* __restrict__ wo = C.v.ws[cur ^ 1];
    float* __restrict__ so = C.v.ss[cur ^ 1];
    auto fld = [&](unsigned q) { return S.next(ui[q], S.sdir(wi[q], S.first ? 0.f : si[q])); };
    for_cells(g, [&](int k, unsigned c, int x, int y) {
        const Nb n = neighbours(g, c, x, y, k);
        const float ac = C.alpha[c];
        float cf[6];
        cell_faces(C, n, ac, cf);
        const float rob = k + 1 == g.nz ? C.robin : 0.f;
        const float d = diag(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5], rob);
        const float uold = ui[c];
        const float sn = S.sdir(wi[c], S.first ? 0.f : si[c]);
        const float f = S.next(uold, sn);
        float fq[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) fq[i] = (n.m >> i & 1u) ? fld(n.q[i]) : 0.f;
        const float Au = f + cf[0] * (f - fq[0]) + cf[1] * (f - fq[1]) + cf[2] * (f - fq[2]) +
                         cf[3] * (f - fq[3]) + cf[4] * (f - fq[4]) + cf[5] * (f - fq[5]) + rob * f;
        const float pn = S.first ? uold : fmaf(S.bt, C.v.p[c], uold);
        C.v.p[c] = pn;
        C.v.delta[c] = fmaf(S.a, pn, C.v.delta[c]);
        uo[c] = f;
        wo[c] = rcp_approx(d) * Au;
        so[c] = sn;
        const float r = d * f;
        acc.add(0, r * f);
        acc.add(1, Au * f);
        acc.add(2, r * r);
    });
}

// --------------------------------------------------------------- solve
// One linear solve A (x0 + delta) = x0 + e, where e (the forcing of this
// step) is given per own cell by Rhs(c, k) and the state x0 = x0hi + x0lo is
// a compensated pair (read-only).  The initial residual r0 = e - (A - I) x0 is
// formed with error-free products and sums (TwoProd through fmaf, TwoSum), so
// it is accurate relative to itself however small it is against x0; the CG
// then runs in FP32 on the increment.  On return delta holds the increment.
// `pre`: early copies of the first pass (TMA path; see Pipe).  In thread 0:
// *it_out iterations, *rel_out ||r|| / ||b||, *conv_out whether the stop test
// passed.  Returns false if a barrier or a stage wait failed.
// Start of one solve: y = x0 + d as compensated pairs (hi at y, lo at y + N);
// hu == 0: y is the state x0 itself and d = 0; hu > 0: d is in delta (both
// written by the previous step's add_state, or by prepare_start).
struct Start {
    const float* y;
    int hu;
};

// The last CG iteration of a solve, when its pass is left out: its whole
// effect on the state is delta += a p with p = u (the first iteration) or
// p = u + b p_prev, u = u[cur] and p_prev = p, which the state update applies
// with the same arithmetic as an iteration pass (see solve()).  Without it
// (apply == 0), cur is the set whose u holds the solve's last M^{-1} r.
struct Final {
    int apply;
    float a, b;
    int first, cur;
};

// The start of a solve from the carried residual (on != 0): the residual at
// a zero increment is in sig[sig], and (bh, bl) is this thread's part of
// ||b||^2, summed by the state update that carried it.
struct Carry {
    int on, sig;
    float bh, bl;
};
// When the next solve may start from the carried residual.  Carrying never
// recomputes the residual from the state, so rounding made while it is
// carried stays in it: the recursive residual of a solve drifts from the
// true one by FP32 rounding relative to the residuals the solve went
// through, about ||r0|| (measured: a surface pulse left a fixed error of
// 1e-5 of its start residuals in every later carried step).  The next step
// therefore forms its residual from the state (the error-free pass) when
// this step started with ||r0|| > kCarryBound tol ||b|| (a transient: fewer
// than one step in ten on the inversion workloads), and on every step that
// is a multiple of kCarryRefresh, which bounds what the smaller roundings
// add up to.
constexpr float kCarryBound = 1000.f;
constexpr int kCarryRefresh = 32;

// ||D u_next||^2 for u_next = u - A (w + (B/A) t') expanded in the sums of the
// pass that made u, w and t': rho = (r, r), q = (r.e, r.t, e.e, e.t, t.t) with
// r = D u, e = D w, t = D t'; A = alpha, B = alpha beta:
// rho - 2A q0 - 2B q1 + A^2 q2 + 2AB q3 + B^2 q4.  Single precision: the terms
// are about rho and the result one to four decades smaller, and the sums
// carry about 1e-6 of relative error, so the expansion is good to about 1e-4
// of itself, which is what a stop decision needs.
__device__ __forceinline__ float next_rho(float rho, float A, float B, float q0, float q1, float q2, float q3,
                                          float q4) {
    float v = fmaf(-2.f * A, q0, rho);
    v = fmaf(-2.f * B, q1, v);
    v = fmaf(A * A, q2, v);
    v = fmaf(2.f * A * B, q3, v);
    return fmaf(B * B, q4, v);
}

// kPred (the staged kernels): the residual norm of the next iteration is
// known before its pass (next_rho, from five more sums of the pass before);
// when it passes the stop test, that iteration's pass (whose product A u and
// stores would be discarded) is left out and its update returned in *fin
// for the state update.  The stop test then sees the expanded norm, equal to
// the pass's own sum up to rounding.
template <int kMode, class RhsFn>
__device__ bool solve(const Common& C, Sync& sy, Ring& ring, const Pipe& pre, const Start& st0, RhsFn rhs,
                      int* it_out, float* rel_out, bool* conv_out, Final* fin, const Carry& cy = Carry{0, 0, 0.f, 0.f},
                      bool* big = nullptr) {
    constexpr bool kTma = kMode > 0, kWrap = kMode == 2, kPred = kTma;
    const Geo& g = C.g;
    Pipe pp = pipe_none();
    *fin = Final{0, 0.f, 0.f, 0, 0};
    // ---- init 1: r0 = e - d - (A - I) y, u0 = M^{-1} r0 ; bb, (r0,u0), (r0,r0)
    Acc<3> acc3;
    if constexpr (kTma) {
        if (cy.on) {   // r0 = s - A d from the carried residual
            const PassIn in{kInitC, cy.sig, false, 0u, 0u, 0};
            acc3.h[0] = cy.bh;
            acc3.l[0] = cy.bl;
            InitCBody B(C, acc3);
            if (!staged<kWrap>(C, ring, in, B, pre.n, pre.ok)) return false;
        } else {
            PassIn in{kInit1, 0, false, 0u, 0u, st0.hu};
            if (!slab_half(C, st0.y, &in.zx)) return false;
            Init1Body<RhsFn> B(C, rhs, acc3, st0.hu);
            if (!staged<kWrap>(C, ring, in, B, pre.n, pre.ok)) return false;
        }
    } else {
        const unsigned N = g.S * (unsigned)g.nz;
        const float* __restrict__ yh = st0.y;
        const float* __restrict__ yl = st0.y + N;
        for_cells(g, [&](int k, unsigned c, int x, int y) {
            const Nb n = neighbours(g, c, x, y, k);
            const float ac = C.alpha[c];
            float cf[6];
            cell_faces(C, n, ac, cf);
            const float rob = k + 1 == g.nz ? C.robin : 0.f;
            const float fc = yh[c], lc = yl[c];
            const float d = st0.hu > 0 ? C.v.delta[c] : 0.f;
            float sh = 0.f, sx = 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i)
                if (n.m >> i & 1u) exact_term(cf[i], fc, lc, yh[n.q[i]], yl[n.q[i]], sh, sx);
            exact_sink(rob, fc, lc, sh, sx);
            {
                float t, te;
                two_sum(sh, d, t, te);
                sh = t;
                sx += te;
            }
            const float e = rhs(c, k);
            const float r = (e - sh) - sx;
            const float u = rcp_approx(diag(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5], rob)) * r;
            C.v.u[0][c] = u;
            C.v.delta[c] = d;
            const float b = ((fc - d) + lc) + e;
            acc3.add(0, b * b);
            acc3.add(1, r * u);
            acc3.add(2, r * r);
        });
    }
    // CG scalars live in thread 0 (double-floats); the FP32 step lengths and
    // the stop decision reach the other threads through shared memory.  The
    // sums of the initial residual join the one of the first product: a grid
    // barrier between the two passes (u0 complete, its stores ordered before
    // the copies of the next pass), one reduction after both.
    __shared__ float s_a, s_b;
    __shared__ int s_go, s_fin, s_big;
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (!barrier(sy)) return false;
    // ---- init 2: ws0 = M^{-1} A u0 ; (A u0, u0)
    Acc<1> acc1;
    float q2[2] = {0.f, 0.f};
    if constexpr (kTma) {
        const PassIn in{kInit2, 0, false, 0u, 0u};
        Init2Body B(C, acc1, q2);
        if (!staged<kWrap>(C, ring, in, B)) return false;
    } else {
        const float* __restrict__ u0 = C.v.u[0];
        for_cells(g, [&](int k, unsigned c, int x, int y) {
            const Nb n = neighbours(g, c, x, y, k);
            const float ac = C.alpha[c];
            float cf[6];
            cell_faces(C, n, ac, cf);
            const float rob = k + 1 == g.nz ? C.robin : 0.f;
            const float f = u0[c];
            float fq[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) fq[i] = (n.m >> i & 1u) ? u0[n.q[i]] : 0.f;
            const float Au = f + cf[0] * (f - fq[0]) + cf[1] * (f - fq[1]) + cf[2] * (f - fq[2]) +
                             cf[3] * (f - fq[3]) + cf[4] * (f - fq[4]) + cf[5] * (f - fq[5]) + rob * f;
            C.v.ws[0][c] = rcp_approx(diag(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5], rob)) * Au;
            acc1.add(0, Au * f);
        });
    }
    // bb, (r0, u0), (r0, r0), (A u0, u0) [+ the expansion's (r.e, e.e) of init 2]
    Acc<4> acc4;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        acc4.h[i] = acc3.h[i];
        acc4.l[i] = acc3.l[i];
    }
    acc4.h[3] = acc1.h[0];
    acc4.l[3] = acc1.l[0];
    DF t4[4];
    float e4[2] = {0.f, 0.f};
    auto early = [&] {
        if constexpr (kTma) pp = pipe_start(C, ring, PassIn{kIter, 0, true, 0u, 0u});
    };
    if constexpr (kPred) {
        if (!grid_sum_p<4, 2>(sy, acc4, q2, t4, e4, early)) return false;
    } else {
        if (!grid_sum<4>(sy, acc4, t4, early)) return false;
    }
    const DF bb = t4[0], lim = df_mul(DF{C.tol2_hi, C.tol2_lo}, bb);
    DF gam = t4[1], rho = t4[2];
    int it = 0;
    if (threadIdx.x == 0) {
        s_go = (!df_le(rho, lim) && C.max_iter > 0) ? 1 : 0;
        s_big = rho.hi > kCarryBound * kCarryBound * lim.hi ? 1 : 0;   // a transient (see kCarryBound)
    }
    __syncthreads();
    if (big) *big = s_big != 0;
    if (!s_go) {
        if constexpr (kTma) {
            if (!pipe_cancel(C, ring, pp)) return false;
        }
    } else {
        DF alpha{0.f, 0.f};
        if (threadIdx.x == 0) {
            alpha = df_div(gam, t4[3]);
            s_a = alpha.hi;
            s_b = 0.f;
            s_fin = 0;
            if constexpr (kPred) {   // the first iteration's residual norm, before its pass
                const float pr = next_rho(rho.hi, alpha.hi, 0.f, e4[0], 0.f, e4[1], 0.f, 0.f);
                if (pr <= lim.hi) {
                    rho = DF{pr, 0.f};
                    s_fin = 1;
                }
            }
        }
        __syncthreads();
        int cur = 0;
        if (s_fin) {   // the first iteration is the last: its update goes to the state update
            if constexpr (kTma) {
                if (!pipe_cancel(C, ring, pp)) return false;
            }
            *fin = Final{1, s_a, 0.f, 1, cur};
            it = 1;
        } else {
            // ---- iterations: one pass, one reduction each
            while (true) {
                Step S;
                S.a = s_a;
                S.bt = s_b;
                S.first = it == 0;
                // (r,u), (Au,u), (r,r) [+ the expansion's five sums of the next norm]
                Acc<3> acc;
                float q5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                if constexpr (kTma) {
                    const PassIn in{kIter, cur, S.first, 0u, 0u};
                    IterBody<kPred> B(C, S, cur, acc, q5);
                    if (!staged<kWrap>(C, ring, in, B, pp.n, pp.ok)) return false;
                } else {
                    plain_pass(C, cur, S, acc);
                }
                DF t[3];
                float e5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                auto early = [&] {
                    if constexpr (kTma) pp = pipe_start(C, ring, PassIn{kIter, cur ^ 1, false, 0u, 0u});
                };
                if constexpr (kPred) {
                    if (!grid_sum_p<3, 5>(sy, acc, q5, t, e5, early)) return false;
                } else {
                    if (!grid_sum<3>(sy, acc, t, early)) return false;
                }
                ++it;
                cur ^= 1;
                if (threadIdx.x == 0) {
                    rho = t[2];
                    bool go = !(df_le(rho, lim) || it >= C.max_iter);
                    s_fin = 0;
                    if (go) {
                        // beta = gam' / gam ; alpha = gam' / ((w, u) - beta gam' / alpha)
                        const DF gam_new = t[0];
                        const DF beta = df_div(gam_new, gam);
                        alpha = df_div(gam_new, df_add(t[1], df_neg(df_div(df_mul(beta, gam_new), alpha))));
                        gam = gam_new;
                        s_a = alpha.hi;
                        s_b = beta.hi;
                        if constexpr (kPred) {   // the next iteration's residual norm, before its pass
                            const float pr = next_rho(rho.hi, alpha.hi, alpha.hi * beta.hi, e5[0], e5[1], e5[2],
                                                      e5[3], e5[4]);
                            if (pr <= lim.hi) {
                                rho = DF{pr, 0.f};
                                s_fin = 1;
                                go = false;
                            }
                        }
                    }
                    s_go = go ? 1 : 0;
                }
                __syncthreads();
                if (!s_go) {
                    if constexpr (kTma) {
                        if (!pipe_cancel(C, ring, pp)) return false;
                    }
                    if (s_fin) {   // the next iteration is the last: its update goes to the state update
                        *fin = Final{1, s_a, s_b, 0, cur};
                        ++it;
                    } else {
                        fin->cur = cur;
                    }
                    break;
                }
            }
        }
    }
    *it_out = it;
    *rel_out = bb.hi > 0.f ? sqrtf(rho.hi / bb.hi) : 0.f;
    *conv_out = df_le(rho, lim);
    return true;
}

// One solve by the paper's inner solver (App. D.2): exactly K Jacobi sweeps
// from the warm start x0 (st0.hu must be 0), on the increment as in solve():
// the initial-residual pass gives u0 = D^{-1} r0, which is the first sweep;
// sweeps 2..K alternate between the ws and ss buffers of set 0, the last one
// writes delta.  No reduction, one grid barrier per sweep.
template <int kMode, class RhsFn>
__device__ bool solve_jacobi(const Common& C, Sync& sy, Ring& ring, const Pipe& pre, const Start& st0, RhsFn rhs,
                             int K) {
    constexpr bool kTma = kMode > 0, kWrap = kMode == 2;
    const Geo& g = C.g;
    Acc<3> acc3;   // the pass's sums are not needed here
    if constexpr (kTma) {
        PassIn in{kInit1, 0, false, 0u, 0u, 0};
        if (!slab_half(C, st0.y, &in.zx)) return false;
        Init1Body<RhsFn> B(C, rhs, acc3, 0);
        if (!staged<kWrap>(C, ring, in, B, pre.n, pre.ok)) return false;
    } else {
        const unsigned N = g.S * (unsigned)g.nz;
        const float* __restrict__ yh = st0.y;
        const float* __restrict__ yl = st0.y + N;
        for_cells(g, [&](int k, unsigned c, int x, int y) {
            const Nb n = neighbours(g, c, x, y, k);
            const float ac = C.alpha[c];
            float cf[6];
            cell_faces(C, n, ac, cf);
            const float rob = k + 1 == g.nz ? C.robin : 0.f;
            const float fc = yh[c], lc = yl[c];
            float sh = 0.f, sx = 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i)
                if (n.m >> i & 1u) exact_term(cf[i], fc, lc, yh[n.q[i]], yl[n.q[i]], sh, sx);
            exact_sink(rob, fc, lc, sh, sx);
            const float r = (rhs(c, k) - sh) - sx;
            C.v.u[0][c] = rcp_approx(diag(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5], rob)) * r;
        });
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (!barrier(sy)) return false;
    const unsigned N = g.S * (unsigned)g.nz;
    if (K <= 1) {   // delta = u0
        const unsigned stride = cta_count() * NT;
        for (unsigned c = cta_id() * NT + threadIdx.x; c < N; c += stride) C.v.delta[c] = C.v.u[0][c];
        return barrier(sy);
    }
    int src = 0;   // slot (and buffer of set 0) holding the current delta
    for (int kappa = 1; kappa < K; ++kappa) {
        const int dst = src == 1 ? 2 : 1;
        float* out = kappa == K - 1 ? C.v.delta : (dst == 1 ? C.v.ws[0] : C.v.ss[0]);
        if constexpr (kTma) {
            JacobiBody B(C, src, out);
            if (!staged<kWrap>(C, ring, PassIn{kJacobi, 0, false, 0u, 0u}, B)) return false;
        } else {
            const float* __restrict__ in = src == 0 ? C.v.u[0] : (src == 1 ? C.v.ws[0] : C.v.ss[0]);
            const float* __restrict__ u0 = C.v.u[0];
            for_cells(g, [&](int k, unsigned c, int x, int y) {
                const Nb n = neighbours(g, c, x, y, k);
                const float ac = C.alpha[c];
                float cf[6];
                cell_faces(C, n, ac, cf);
                const float rob = k + 1 == g.nz ? C.robin : 0.f;
                float sum = 0.f;
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    if (n.m >> i & 1u) sum += cf[i] * in[n.q[i]];
                out[c] = fmaf(rcp_approx(diag(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5], rob)), sum, u0[c]);
            });
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!barrier(sy)) return false;
        src = dst;
    }
    return true;
}

__device__ __forceinline__ void prefetch_maps(const TmaMaps& M) {
    tma_prefetch_desc(&M.uws[0]);
    tma_prefetch_desc(&M.uws[1]);
    tma_prefetch_desc(&M.u0);
    tma_prefetch_desc(&M.alpha);
    tma_prefetch_desc(&M.pd);
    tma_prefetch_desc(&M.states);
    tma_prefetch_desc(&M.dh);
    tma_prefetch_desc(&M.sg);
}

__device__ __forceinline__ Sync make_sync(DevCtl* ctl, double* partials, int bar_sel = 0) {
    Sync s;
    s.ctl = ctl;
    s.bar = bar_sel ? &ctl->bar2 : &ctl->bar;
    s.partials = partials;
    s.G = cta_count();
    s.epoch = 0;
    s.red = 0;
    s.missing = ctl->missing;
    s.wait_ns = ctl->wait_ns ? ctl->wait_ns : kBarrierTimeoutNs;
    return s;
}

// The increment ring of a sweep: slot(m) holds the increment of step m
// (kRing slots, m mod kRing).
struct IncRing {
    float* base;
    unsigned N;
    __device__ __forceinline__ float* slot(int m) const { return base + (size_t)(m & (kRing - 1)) * N; }
};
// The three increments before the one of step m, in the order they were
// made: steps m - 1, m - 2, m - 3 of a forward sweep (dir = -1), m + 1, m + 2,
// m + 3 of an adjoint sweep (dir = +1).
struct Older {
    const float* r[3];
};
__device__ __forceinline__ Older older(const IncRing& R, int m, int dir) {
    return Older{{R.slot(m + dir), R.slot(m + 2 * dir), R.slot(m + 3 * dir)}};
}

// The start increment of the next solve from the newest h increments (dn the
// newest, d1, d2, d3 the ones before): the next value of the polynomial of
// degree h - 1 through them, i.e. dn, 2dn - d1, 3dn - 3d1 + d2 or
// 4dn - 6d1 + 4d2 - d3 (backward-difference extrapolation).
__device__ __forceinline__ float predict(int h, float dn, float d1, float d2, float d3) {
    switch (h) {
        case 1: return dn;
        case 2: return fmaf(2.f, dn, -d1);
        case 3: return fmaf(3.f, dn - d1, d2);
        default: return fmaf(4.f, dn + d2, fmaf(-6.f, d1, -d3));
    }
}
__device__ __forceinline__ float4 ld_older(const float* p, unsigned i, bool use) {
    return use ? reinterpret_cast<const float4*>(p)[i] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The carried residual (TMA-staged PCG).  With s^m = b^m - A x0^m, the
// residual of step m's system at a zero increment, and r^m = s^m - A delta^m
// the residual the solve ends with (r^m = D u, u the CG's last M^{-1} r),
// the next step's system (x0 <- x0 + delta, b = x0 + e) gives exactly
//   s^{next} = r^m + delta^m + (e^{next} - e^m)
// (A is the same for every step of a sweep).  The state update forms, at
// each cell, g = s^{next} - d^{next} = (r^m + (e^{next} - e^m)) + (delta^m -
// d^{next}) with d^{next} the next predicted increment, so the next solve
// needs no error-free pass over the state: its start residual is
// r0 = g - (A - I) d (InitCBody).  Both parts of g are small (a residual and
// the error of the prediction, formed from two close numbers), so their
// rounding is far below that of delta itself; the rounding of r^m (FP32,
// relative to the residuals of the solve) stays in s, well below the solve's
// tolerance, which is relative to ||b||.
// Forcing e of a step at a cell: the source plane of the sweep holds it, every
// other cell has none.
struct CarryOut {
    float* sig;            // g = s^{next} - d^{next} (written)
    const float* diag;     // D
    const float* u;        // u of the solve's last set
    const float* ws;       // ws and ss of that set (a folded last iteration only)
    const float* ss;
};

// End of a solve, by every thread of the grid (quads when N % 4 == 0):
//   y = x + delta as compensated pairs (hi in [0, N), lo in [N, 2N)), the new state;
//   rd = delta, the ring slot of this step's increment;
//   when the next solve predicts (hu_next > 0): d = predict(delta and the
//   hu_next - 1 increments before it), delta = d and ys = y + d (the next
//   start, as pairs).
// Ends with the proxy fence that orders these stores before later TMA reads.
// fin (when fin.apply): the solve's last iteration, whose pass was left out,
// is applied first: delta += a p with p = u[fin.cur] (+ b p_prev), the same
// fused multiply-adds as an iteration pass.
// co (quads only): the next solve starts from the carried residual instead:
// co->sig = g (ecur, enext: the forcing of this step and the next at a cell;
// d with hu_next increments, which must be the count the next step uses
// even when another launch runs it), delta = d (0 when it does not
// predict), no ys; (bh, bl) = this thread's part of ||y + e^{next}||^2, the
// next solve's ||b||^2, summed quad by quad in the order of the quads
// (prepare_carried sums the same way).
template <class EFn>
__device__ void add_state(const float* __restrict__ x, float* __restrict__ delta, float* __restrict__ y,
                          unsigned N, float* __restrict__ rd, const Older& old, int hu_next,
                          float* __restrict__ ys, bool stream_y, const Final& fin, const Vecs* vv,
                          const CarryOut* co, EFn ecur, EFn enext, float& bh, float& bl) {
    const unsigned stride = cta_count() * NT, t0 = cta_id() * NT + threadIdx.x;
    const bool fa = fin.apply && vv;
    const float* __restrict__ fu = fa ? vv->u[fin.cur] : nullptr;
    const float* __restrict__ fp = fa ? vv->p : nullptr;
    auto last = [&](float dv, float uv, float pv) {   // delta + a (u or u + b p)
        return fmaf(fin.a, fin.first ? uv : fmaf(fin.b, pv, uv), dv);
    };
    bh = bl = 0.f;
    if ((N & 3u) == 0) {
        // One quad per thread and loop step, every load of the quad issued
        // before its stores (batches of two quads cost the adjoint kernel
        // 110 more bytes of spills and were slower).  x (the old state) is not read again soon, so it
        // streams past L2 (evict-first), and so does the new state y when
        // stream_y (a forward state, read again only a step later); delta,
        // the ring and the next start stay there for the passes that follow.
        constexpr int B = 1;
        const unsigned N4 = N >> 2;
        const float4* __restrict__ xh = reinterpret_cast<const float4*>(x);
        const float4* __restrict__ xl = reinterpret_cast<const float4*>(x + N);
        float4* __restrict__ d4 = reinterpret_cast<float4*>(delta);
        float4* __restrict__ yh = reinterpret_cast<float4*>(y);
        float4* __restrict__ yl = reinterpret_cast<float4*>(y + N);
        float4* __restrict__ r4 = reinterpret_cast<float4*>(rd);
        const float4* __restrict__ o1p = reinterpret_cast<const float4*>(old.r[0]);
        const float4* __restrict__ o2p = reinterpret_cast<const float4*>(old.r[1]);
        const float4* __restrict__ o3p = reinterpret_cast<const float4*>(old.r[2]);
        float4* __restrict__ sh4 = reinterpret_cast<float4*>(ys);
        float4* __restrict__ sl4 = reinterpret_cast<float4*>(ys + N);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4* __restrict__ fu4 = reinterpret_cast<const float4*>(co ? co->u : fu);
        const float4* __restrict__ fp4 = reinterpret_cast<const float4*>(fp);
        const float4* __restrict__ cw4 = reinterpret_cast<const float4*>(co && fa ? co->ws : nullptr);
        const float4* __restrict__ cs4 = reinterpret_cast<const float4*>(co && fa ? co->ss : nullptr);
        const float4* __restrict__ dg4 = reinterpret_cast<const float4*>(co ? co->diag : nullptr);
        float4* __restrict__ sg4 = reinterpret_cast<float4*>(co ? co->sig : nullptr);
        Acc<1> bb;
        for (unsigned i0 = t0; i0 < N4; i0 += B * stride) {
            float4 h[B], l[B], e[B], o1[B], o2[B], o3[B], uf[B], dg[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const unsigned i = i0 + u * stride;
                const bool in = i < N4;
                h[u] = in ? __ldcs(xh + i) : z4;
                l[u] = in ? __ldcs(xl + i) : z4;
                e[u] = in ? d4[i] : z4;
                o1[u] = in && hu_next > 1 ? o1p[i] : z4;
                o2[u] = in && hu_next > 2 ? o2p[i] : z4;
                o3[u] = in && hu_next > 3 ? o3p[i] : z4;
                uf[u] = in && (fa || co) ? fu4[i] : z4;
                dg[u] = in && co ? dg4[i] : z4;
                if (fa && in) {
                    const float4 uu = uf[u], pq = fin.first ? z4 : fp4[i];
                    e[u] = make_float4(last(e[u].x, uu.x, pq.x), last(e[u].y, uu.y, pq.y), last(e[u].z, uu.z, pq.z),
                                       last(e[u].w, uu.w, pq.w));
                    if (co) {   // the last u: u - a (ws + b ss), as an iteration pass forms it
                        const float4 w = cw4[i], sv = fin.first ? z4 : cs4[i];
                        const Step S{fin.a, fin.b, fin.first != 0};
                        uf[u] = make_float4(S.next(uu.x, S.sdir(w.x, sv.x)), S.next(uu.y, S.sdir(w.y, sv.y)),
                                            S.next(uu.z, S.sdir(w.z, sv.z)), S.next(uu.w, S.sdir(w.w, sv.w)));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const unsigned i = i0 + u * stride;
                if (i >= N4) break;
                float4 oh, ol;
                add_pair(h[u].x, l[u].x, e[u].x, oh.x, ol.x);
                add_pair(h[u].y, l[u].y, e[u].y, oh.y, ol.y);
                add_pair(h[u].z, l[u].z, e[u].z, oh.z, ol.z);
                add_pair(h[u].w, l[u].w, e[u].w, oh.w, ol.w);
                if (stream_y) {
                    __stcs(yh + i, oh);
                    __stcs(yl + i, ol);
                } else {
                    yh[i] = oh;
                    yl[i] = ol;
                }
                r4[i] = e[u];
                float4 dn = z4;
                if (hu_next > 0)
                    dn = make_float4(predict(hu_next, e[u].x, o1[u].x, o2[u].x, o3[u].x),
                                     predict(hu_next, e[u].y, o1[u].y, o2[u].y, o3[u].y),
                                     predict(hu_next, e[u].z, o1[u].z, o2[u].z, o3[u].z),
                                     predict(hu_next, e[u].w, o1[u].w, o2[u].w, o3[u].w));
                if (co) {
                    // g = (r + (e^{next} - e)) + (delta - d^{next})
                    const unsigned c = 4u * i;
                    const float en[4] = {enext(c), enext(c + 1), enext(c + 2), enext(c + 3)};
                    const float ec[4] = {ecur(c), ecur(c + 1), ecur(c + 2), ecur(c + 3)};
                    const float dgv[4] = {dg[u].x, dg[u].y, dg[u].z, dg[u].w};
                    const float ufv[4] = {uf[u].x, uf[u].y, uf[u].z, uf[u].w};
                    const float ev[4] = {e[u].x, e[u].y, e[u].z, e[u].w};
                    const float dnv[4] = {dn.x, dn.y, dn.z, dn.w};
                    const float ohv[4] = {oh.x, oh.y, oh.z, oh.w}, olv[4] = {ol.x, ol.y, ol.z, ol.w};
                    float sv[4], q = 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        sv[j] = (dgv[j] * ufv[j] + (en[j] - ec[j])) + (ev[j] - dnv[j]);
                        const float b = (ohv[j] + olv[j]) + en[j];
                        q += b * b;
                    }
                    bb.add(0, q);
                    sg4[i] = make_float4(sv[0], sv[1], sv[2], sv[3]);
                    d4[i] = dn;
                } else if (hu_next > 0) {
                    float4 sh, sl;
                    add_pair(oh.x, ol.x, dn.x, sh.x, sl.x);
                    add_pair(oh.y, ol.y, dn.y, sh.y, sl.y);
                    add_pair(oh.z, ol.z, dn.z, sh.z, sl.z);
                    add_pair(oh.w, ol.w, dn.w, sh.w, sl.w);
                    d4[i] = dn;
                    sh4[i] = sh;
                    sl4[i] = sl;
                }
            }
        }
        bh = bb.h[0];
        bl = bb.l[0];
    } else {   // plain-load path only (the staged path needs nx % 4 == 0)
        for (unsigned c = t0; c < N; c += stride) {
            const float e = fa ? last(delta[c], fu[c], fin.first ? 0.f : fp[c]) : delta[c];
            float oh, ol;
            add_pair(x[c], x[N + c], e, oh, ol);
            y[c] = oh;
            y[N + c] = ol;
            rd[c] = e;
            if (hu_next > 0) {
                const float dn = predict(hu_next, e, hu_next > 1 ? old.r[0][c] : 0.f,
                                         hu_next > 2 ? old.r[1][c] : 0.f, hu_next > 3 ? old.r[2][c] : 0.f);
                delta[c] = dn;
                add_pair(oh, ol, dn, ys[c], ys[N + c]);
            }
        }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// The start of a launch's first solve from the carried residual (the
// previous step ran in another launch): delta = d = predict(rn and the
// hu - 1 increments before it) or 0, and (bh, bl) = this thread's part of
// ||x + e||^2, with the loop and arithmetic of add_state's carried path, so a
// launch resumed here starts from the same bits as one that ran through.
template <class EFn>
__device__ void prepare_carried(const float* __restrict__ x, const float* __restrict__ rn, const Older& old, int hu,
                                float* __restrict__ delta, unsigned N, EFn ecur, float& bh, float& bl) {
    const unsigned stride = cta_count() * NT, t0 = cta_id() * NT + threadIdx.x;
    const unsigned N4 = N >> 2;
    const float4* __restrict__ xh = reinterpret_cast<const float4*>(x);
    const float4* __restrict__ xl = reinterpret_cast<const float4*>(x + N);
    const float4* __restrict__ r4 = reinterpret_cast<const float4*>(rn);
    const float4* __restrict__ o1p = reinterpret_cast<const float4*>(old.r[0]);
    const float4* __restrict__ o2p = reinterpret_cast<const float4*>(old.r[1]);
    const float4* __restrict__ o3p = reinterpret_cast<const float4*>(old.r[2]);
    float4* __restrict__ d4 = reinterpret_cast<float4*>(delta);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    Acc<1> bb;
    for (unsigned i = t0; i < N4; i += stride) {
        float4 dn = z4;
        if (hu > 0) {
            const float4 e = r4[i], o1 = hu > 1 ? o1p[i] : z4, o2 = hu > 2 ? o2p[i] : z4, o3 = hu > 3 ? o3p[i] : z4;
            dn = make_float4(predict(hu, e.x, o1.x, o2.x, o3.x), predict(hu, e.y, o1.y, o2.y, o3.y),
                             predict(hu, e.z, o1.z, o2.z, o3.z), predict(hu, e.w, o1.w, o2.w, o3.w));
        }
        d4[i] = dn;
        const float4 h = xh[i], l = xl[i];
        const unsigned c = 4u * i;
        const float hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float b = (hv[j] + lv[j]) + ecur(c + j);
            q += b * b;
        }
        bb.add(0, q);
    }
    bh = bb.h[0];
    bl = bb.l[0];
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// The diagonal of A at every cell (plain loads, every thread of the grid),
// for the carried residual: the same face values and sum as the passes.
__device__ void write_diag(const Common& C) {
    const Geo& g = C.g;
    const unsigned stride = cta_count() * NT, t0 = cta_id() * NT + threadIdx.x, N = g.S * (unsigned)g.nz;
    for (unsigned c = t0; c < N; c += stride) {
        const int k = (int)(c / g.S), y = (int)((c % g.S) / (unsigned)g.nx), x = (int)(c % (unsigned)g.nx);
        const Nb n = neighbours(g, c, x, y, k);
        float cf[6];
        cell_faces(C, n, C.alpha[c], cf);
        C.v.diag[c] = diag(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5], k + 1 == g.nz ? C.robin : 0.f);
    }
}

// The start of a launch's first solve when it predicts (the previous step ran
// in another launch): d = predict(rn and the hu - 1 increments before it),
// delta = d, ys = x + d as pairs; every thread of the grid, then the proxy
// fence.  The same arithmetic as add_state, so a launch resumed from a
// checkpoint starts from the same bits.
__device__ void prepare_start(const float* __restrict__ x, const float* __restrict__ rn, const Older& old, int hu,
                              float* __restrict__ delta, float* __restrict__ ys, unsigned N) {
    const unsigned stride = cta_count() * NT, t0 = cta_id() * NT + threadIdx.x;
    for (unsigned c = t0; c < N; c += stride) {
        const float dn = predict(hu, rn[c], hu > 1 ? old.r[0][c] : 0.f, hu > 2 ? old.r[1][c] : 0.f,
                                 hu > 3 ? old.r[2][c] : 0.f);
        delta[c] = dn;
        add_pair(x[c], x[N + c], dn, ys[c], ys[N + c]);
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// A checkpoint's increment history: dst[i N, (i + 1) N) = the increment of
// step m - i (forward; m + i adjoint is not needed), i < h; every thread of
// the grid.  load_hist is the inverse at a launch start.
// sig (or null): the carried residual of step m + 1, kept after the increments.
__device__ void save_hist(float* __restrict__ dst, const IncRing& R, int m, int h, const float* sig) {
    const unsigned stride = cta_count() * NT, t0 = cta_id() * NT + threadIdx.x, N = R.N;
    for (int k = 0; k < h; ++k) {
        const float* src = R.slot(m - k);
        for (unsigned i = t0; i < N; i += stride) dst[(size_t)k * N + i] = src[i];
    }
    if (sig)
        for (unsigned i = t0; i < N; i += stride) dst[(size_t)h * N + i] = sig[i];
}
__device__ void load_hist(const float* __restrict__ src, const IncRing& R, int m, int h, float* sig) {
    const unsigned stride = cta_count() * NT, t0 = cta_id() * NT + threadIdx.x, N = R.N;
    for (int k = 0; k < h; ++k) {
        float* dst = R.slot(m - k);
        for (unsigned i = t0; i < N; i += stride) dst[i] = src[(size_t)k * N + i];
    }
    if (sig)
        for (unsigned i = t0; i < N; i += stride) sig[i] = src[(size_t)h * N + i];
}

// Forcing of a forward step at a cell: the surface flux of the step on plane 0.
struct FwdForce {
    const float* q;        // the step's flux map, or null
    float sc;
    unsigned S;
    __device__ __forceinline__ float operator()(unsigned c) const { return (q && c < S) ? sc * q[c] : 0.f; }
};
__device__ __forceinline__ FwdForce fwd_force(const FwdTiled& a, int n) {
    const unsigned S = a.c.g.S;
    const float* q = a.q_full ? a.q_full + (size_t)n * S : (n < a.q_steps ? a.q_face : nullptr);
    return FwdForce{q, a.src_scale, S};
}
// Forcing of an adjoint step n at a cell: the surface misfit of T^n.
struct AdjForce {
    const float* T;        // T^n (pair), or null
    const float* ob;       // its target frame
    unsigned o0, S, N;
    float gs;
    __device__ __forceinline__ float operator()(unsigned c) const {
        return (T && c - o0 < S) ? gs * ((T[c] - ob[c - o0]) + T[N + c]) : 0.f;
    }
};
__device__ __forceinline__ AdjForce adj_force(const AdjTiled& a, int n) {
    const unsigned S = a.c.g.S, N = S * (unsigned)a.c.g.nz;
    return AdjForce{a.T[n - a.n0], a.obs + (size_t)(n - 1) * S, a.obs_off, S, N, a.g_scale};
}

// ------------------------------------------------------------- forward
// kTma: iterations and stencil passes staged through TMA (a.c.tma set);
// otherwise plain global loads.
template <int kMode, bool kJac>
__device__ __forceinline__ void forward_sweep(const FwdTiled& a) {
    constexpr bool kTma = kMode > 0;
    extern __shared__ unsigned char dyn_smem[];
    __shared__ __align__(8) unsigned long long s_full[NS], s_empty[NS];
    Ring ring = make_ring(dyn_smem, s_full, s_empty, kTma);
    if (kTma && threadIdx.x == NCT) prefetch_maps(a.c.maps);

    Sync sy = make_sync(a.c.ctl, a.c.partials, a.c.bar_sel);
    const Geo& g = a.c.g;
    const unsigned N = g.S * (unsigned)g.nz, S = g.S;
    const unsigned stride = cta_count() * NT;
    const unsigned c0 = cta_id() * NT + threadIdx.x;
    double loss = 0.0;
    Pipe pre = pipe_none();
    const unsigned long long t_start = a.budget_ns ? now_ns() : 0ull;   // used by CTA 0 only
    int n_next = a.n1;   // the next step to run after this launch
    // the carried residual (TMA-staged PCG, when the workspace has it)
    const bool carry_on = kTma && !kJac && a.c.v.diag != nullptr;
    if (carry_on) write_diag(a.c);
    // increments used by the start of step n (ring slot m holds delta^m)
    auto hu_at = [&](int n) { return min(a.extrap, min(a.hist0 + (n - a.n0), kRing)); };
    const IncRing ring_d{a.ring, N};
    // increments of steps n0-1, n0-2, ... from a checkpoint (recompute
    // launches), copied by the same threads that read them in prepare_start
    const bool carried0 = carry_on && a.carry && a.n0 > 0 && a.cflag && a.cflag[a.n0];
    if (a.ring_load) {
        load_hist(a.ring_load, ring_d, a.n0 - 1, a.extrap, carried0 ? a.c.v.sig[0] : nullptr);
        // prepare_carried reads them by quads, other threads than the copy's
        if (carried0 && !barrier(sy)) return;
    }
    float bh = 0.f, bl = 0.f;   // this thread's part of the next solve's ||b||^2 (carried)
    bool carried = false;
    if (carried0) {
        prepare_carried(a.src[0], ring_d.slot(a.n0 - 1), older(ring_d, a.n0 - 1, -1), hu_at(a.n0), a.c.v.delta, N,
                        fwd_force(a, a.n0), bh, bl);
        if (!barrier(sy)) return;
        carried = true;
    } else if (hu_at(a.n0) > 0) {
        prepare_start(a.src[0], ring_d.slot(a.n0 - 1), older(ring_d, a.n0 - 1, -1), hu_at(a.n0), a.c.v.delta,
                      a.ystart, N);
        if (!barrier(sy)) return;
    }
    for (int n = a.n0; n < a.n1; ++n) {
        // states are compensated pairs: hi in [0, N), lo in [N, 2N)
        const float* __restrict__ Tn = a.src[n - a.n0];
        float* __restrict__ Tn1 = a.dst[n - a.n0];
        const float* qmap = a.q_full ? a.q_full + (size_t)n * S : (n < a.q_steps ? a.q_face : nullptr);
        const float sc = a.src_scale;
        int it = 0;
        float rel = 0.f;
        bool conv = true;
        Final fin{0, 0.f, 0.f, 0, 0};
        bool big = true;
        const int hu = hu_at(n);
        auto rhs = [=](unsigned c, int k) { return (qmap && k == 0) ? sc * qmap[c] : 0.f; };
        bool ok;
        if constexpr (kJac) {   // the paper's inner solver: K sweeps from T^n
            ok = solve_jacobi<kMode>(a.c, sy, ring, pre, Start{Tn, 0}, rhs, a.c.jacobi_k);
            it = a.c.jacobi_k;
        } else {
            ok = solve<kMode>(a.c, sy, ring, pre, Start{hu > 0 ? a.ystart : Tn, hu}, rhs, &it, &rel, &conv, &fin,
                              Carry{carried ? 1 : 0, 0, bh, bl}, &big);
        }
        if (!ok) return;
        if (cta_id() == 0 && threadIdx.x == 0) {
            a.c.iters[n - a.n0] = it;
            a.c.resid[n - a.n0] = rel;
            if (!conv) atomicAdd(&a.c.ctl->notconv, 1);
            if (fin.apply) atomicAdd(&a.c.ctl->folded, 1);
            if (carried) atomicAdd(&a.c.ctl->carried, 1);
        }
        // T^{n+1} = T^n + delta as a compensated pair, delta^n into the ring, and
        // the start of step n+1 when it predicts (carried: the residual of step
        // n+1, also at the end of a launch that another one continues; the
        // choice is kept per step for launches that resume there)
        carried = carry_on && n + 1 < a.n_end && !big && (n + 1) % kCarryRefresh != 0;
        if (carry_on && cta_id() == 0 && threadIdx.x == 0 && n + 1 < a.n_end) a.cflag[n + 1] = carried ? 1 : 0;
        const int hu1 = n + 1 < (carried ? a.n_end : a.n1) ? hu_at(n + 1) : 0;
        const CarryOut co{a.c.v.sig[0], a.c.v.diag, a.c.v.u[fin.cur], a.c.v.ws[fin.cur], a.c.v.ss[fin.cur]};
        add_state(Tn, a.c.v.delta, Tn1, N, ring_d.slot(n), older(ring_d, n, -1), hu1, a.ystart, true, fin, &a.c.v,
                  carried ? &co : nullptr, fwd_force(a, n), fwd_force(a, carried ? n + 1 : n), bh, bl);
        if (a.budget_ns && cta_id() == 0 && threadIdx.x == 0)   // the launch's last step? (read after the barrier)
            *(volatile int*)&a.c.ctl->stop = (n + 1 < a.n1 && now_ns() - t_start >= a.budget_ns) ? 1 : 0;
        if (!barrier(sy)) return;
        const bool stop = a.budget_ns && *(volatile int*)&a.c.ctl->stop != 0;
        if (a.ring_save && a.ring_save[n - a.n0])   // a checkpoint keeps [delta^n; delta^{n-1}; ...] (+ s^{n+1})
            save_hist(a.ring_save[n - a.n0], ring_d, n, a.extrap, carried ? a.c.v.sig[0] : nullptr);
        pre = pipe_none();
        if constexpr (kTma) {   // the next step's first pass, behind the frame below
            if (n + 1 < a.n1 && !stop) {
                if (carried) {
                    pre = pipe_start(a.c, ring, PassIn{kInitC, 0, false, 0u, 0u, 0});
                } else {
                    PassIn in{kInit1, 0, false, 0u, 0u, hu1};
                    if (!slab_half(a.c, hu1 > 0 ? a.ystart : a.src[n + 1 - a.n0], &in.zx)) return;
                    pre = pipe_start(a.c, ring, in);
                }
            }
        }
        if (a.frames || a.obs) {
            for (unsigned s = c0; s < S; s += stride) {
                const float v = Tn1[a.obs_off + s];
                if (a.frames) a.frames[(size_t)n * S + s] = v;
                if (a.obs) {
                    const double e = ((double)v - (double)a.obs[(size_t)n * S + s]) + (double)Tn1[N + a.obs_off + s];
                    loss += e * e;
                }
            }
        }
        if (stop) {   // the budget of this launch is spent; a later one continues at n + 1
            n_next = n + 1;
            break;
        }
    }
    if (a.progress && cta_id() == 0 && threadIdx.x == 0) *a.progress = n_next;
    if (a.loss_partials) {
        const double t = block_sum(loss);
        if (threadIdx.x == 0) {
            if (a.loss_add) a.loss_partials[cta_id()] += t;   // chunks of one sweep add up
            else a.loss_partials[cta_id()] = t;
        }
    }
}

// ------------------------------------------------------------- adjoint
template <int kMode, bool kJac>
__device__ __forceinline__ void adjoint_sweep(const AdjTiled& a) {
    constexpr bool kTma = kMode > 0;
    extern __shared__ unsigned char dyn_smem[];
    __shared__ __align__(8) unsigned long long s_full[NS], s_empty[NS];
    Ring ring = make_ring(dyn_smem, s_full, s_empty, kTma);
    if (kTma && threadIdx.x == NCT) prefetch_maps(a.c.maps);

    Sync sy = make_sync(a.c.ctl, a.c.partials, a.c.bar_sel);
    const Geo& g = a.c.g;
    const unsigned N = g.S * (unsigned)g.nz, S = g.S;
    const float gs = a.g_scale;
    const unsigned stride = cta_count() * NT;
    const unsigned c0 = cta_id() * NT + threadIdx.x;
    (void)stride;
    (void)c0;
    // the carried residual (TMA-staged PCG, when the workspace has it)
    const bool carry_on = kTma && !kJac && a.c.v.diag != nullptr;
    if (carry_on) write_diag(a.c);
    // increments used by the start of step n (ring slot m holds mu^m - mu^{m+1})
    auto hu_at = [&](int n) { return min(a.extrap, min(a.hist0 + (a.n1 - n), kRing)); };
    const IncRing ring_d{a.ring, N};
    float bh = 0.f, bl = 0.f;   // this thread's part of the next solve's ||b||^2 (carried)
    bool carried = false;
    const unsigned long long t_start = a.budget_ns ? now_ns() : 0ull;   // used by CTA 0 only
    int n_next = a.n0;   // the next step to run after this launch (downwards)
    if (carry_on && a.carry && a.cflag && a.cflag[a.n1]) {
        prepare_carried(a.mu[(a.n1 + 1) & 1], ring_d.slot(a.n1 + 1), older(ring_d, a.n1 + 1, 1), hu_at(a.n1),
                        a.c.v.delta, N, adj_force(a, a.n1), bh, bl);
        if (!barrier(sy)) return;
        carried = true;
    } else if (hu_at(a.n1) > 0) {
        prepare_start(a.mu[(a.n1 + 1) & 1], ring_d.slot(a.n1 + 1), older(ring_d, a.n1 + 1, 1), hu_at(a.n1),
                      a.c.v.delta, a.ystart, N);
        if (!barrier(sy)) return;
    }
    for (int n = a.n1; n > a.n0; --n) {
        const float* __restrict__ Tn = a.T[n - a.n0];
        const float* __restrict__ mnext = a.mu[(n + 1) & 1];
        float* __restrict__ mu = a.mu[n & 1];
        const float* ob = a.obs + (size_t)(n - 1) * S;
        int it = 0;
        float rel = 0.f;
        bool conv = true;
        Final fin{0, 0.f, 0.f, 0, 0};
        bool big = true;
        const int hu = hu_at(n);
        const unsigned o0 = a.obs_off;
        auto rhs = [=](unsigned c, int) {
            return (c - o0 < S) ? gs * ((Tn[c] - ob[c - o0]) + Tn[N + c]) : 0.f;
        };
        bool ok;
        if constexpr (kJac) {   // the paper's inner solver: K sweeps from mu^{n+1}
            ok = solve_jacobi<kMode>(a.c, sy, ring, pipe_none(), Start{mnext, 0}, rhs, a.c.jacobi_k);
            it = a.c.jacobi_k;
        } else {
            ok = solve<kMode>(a.c, sy, ring, pipe_none(), Start{hu > 0 ? a.ystart : mnext, hu}, rhs, &it, &rel,
                              &conv, &fin, Carry{carried ? 1 : 0, 1, bh, bl}, &big);
        }
        if (!ok) return;
        if (cta_id() == 0 && threadIdx.x == 0) {
            a.c.iters[a.n1 - n] = it;
            a.c.resid[a.n1 - n] = rel;
            if (!conv) atomicAdd(&a.c.ctl->notconv, 1);
            if (fin.apply) atomicAdd(&a.c.ctl->folded, 1);
            if (carried) atomicAdd(&a.c.ctl->carried, 1);
        }
        // mu^n = mu^{n+1} + delta; carried: the residual of step n - 1 (the
        // last adjoint step is n = 1), also at the end of a launch that
        // another one continues
        carried = carry_on && n - 1 >= 1 && !big && (n - 1) % kCarryRefresh != 0;
        if (carry_on && cta_id() == 0 && threadIdx.x == 0 && n - 1 >= 1) a.cflag[n - 1] = carried ? 1 : 0;
        const CarryOut co{a.c.v.sig[1], a.c.v.diag, a.c.v.u[fin.cur], a.c.v.ws[fin.cur], a.c.v.ss[fin.cur]};
        add_state(mnext, a.c.v.delta, mu, N, ring_d.slot(n), older(ring_d, n, 1),
                  (carried || n - 1 > a.n0) ? hu_at(n - 1) : 0,
                  a.ystart, false, fin, &a.c.v, carried ? &co : nullptr, adj_force(a, n),
                  adj_force(a, carried ? n - 1 : n), bh, bl);
        if (a.budget_ns && cta_id() == 0 && threadIdx.x == 0)   // the launch's last step? (read after the barrier)
            *(volatile int*)&a.c.ctl->stop = (n - 1 > a.n0 && now_ns() - t_start >= a.budget_ns) ? 1 : 0;
        if (!barrier(sy)) return;
        const bool stop = a.budget_ns && *(volatile int*)&a.c.ctl->stop != 0;
        // gradient of step n with mu^n and T^n (the next step writes only the
        // other mu buffer and the CG vectors, so no barrier is needed after it)
        if constexpr (kTma) {
            PassIn in{kGrad, 0, false, 0u, 0u};
            if (!slab_half(a.c, Tn, &in.zx) || !slab_half(a.c, mu, &in.zm)) return;
            GradBody B;
            B.grad = a.grad;
            B.wx = a.wx; B.wy = a.wy; B.wz = a.wz;
            B.nz = g.nz;
            B.S = g.S;
            if (!staged<kMode == 2>(a.c, ring, in, B)) return;
        } else {
            for_cells(g, [&](int k, unsigned c, int x, int y) {
                const Nb nb = neighbours(g, c, x, y, k);
                const float ac = a.alpha[c], mc = mu[c], tc = Tn[c], mcl = mu[N + c], tcl = Tn[N + c];
                float s = 0.f;
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    if (!(nb.m >> f & 1u)) continue;
                    const unsigned q = nb.q[f];
                    const float w = f < 2 ? a.wx : (f < 4 ? a.wy : a.wz);
                    const float aq = a.alpha[q];
                    const float h = aq * rcp_approx(ac + aq);
                    const float dm = (mc - mu[q]) + (mcl - mu[N + q]);
                    const float dT = (tc - Tn[q]) + (tcl - Tn[N + q]);
                    s += w * h * h * dm * dT;
                }
                const float2 gv = a.grad[c];
                float gh, gl;
                add_pair(gv.x, gv.y, -s, gh, gl);
                a.grad[c] = make_float2(gh, gl);
            });
        }
        if (stop) {   // the budget of this launch is spent; a later one continues at n - 1
            n_next = n - 1;
            break;
        }
    }
    if (a.progress && cta_id() == 0 && threadIdx.x == 0) *a.progress = n_next;
}

// Launches of one sweep on the whole grid.
template <int kMode, bool kJac>
__global__ void __launch_bounds__(NT, 1) forward_tiled(const __grid_constant__ FwdTiled a) {
    if (threadIdx.x == 0) {
        s_cta = blockIdx.x;
        s_ncta = gridDim.x;
    }
    __syncthreads();
    forward_sweep<kMode, kJac>(a);
}
template <int kMode, bool kJac>
__global__ void __launch_bounds__(NT, 1) adjoint_tiled(const __grid_constant__ AdjTiled a) {
    if (threadIdx.x == 0) {
        s_cta = blockIdx.x;
        s_ncta = gridDim.x;
    }
    __syncthreads();
    adjoint_sweep<kMode, kJac>(a);
}

// ------------------------------------------------------------- grouped sweeps
// Serving runs the sweeps of several jobs (forward or adjoint, ragged grids)
// in one persistent launch: each sweep gets its own range of CTAs
// (B.off[j] .. B.off[j + 1] - 1, sized by the host in proportion to its work)
// and runs there exactly what a launch of its own would run, with its own
// grid barriers and reductions, so the sweeps proceed independently inside
// the launch.
static_assert(sizeof(BatchArgs) <= 32764, "kernel parameter space");

__global__ void __launch_bounds__(NT, 1) group_tiled(const __grid_constant__ BatchArgs B) {
    int j = -1;
    for (int i = 0; i < B.n; ++i)
        if ((int)blockIdx.x >= B.off[i] && (int)blockIdx.x < B.off[i + 1]) j = i;
    if (j < 0) return;   // beyond the sweeps' ranges
    if (threadIdx.x == 0) {
        s_cta = blockIdx.x - (unsigned)B.off[j];
        s_ncta = (unsigned)(B.off[j + 1] - B.off[j]);
    }
    __syncthreads();
    const BatchSweep& w = B.s[j];
    if (w.adjoint) {
        if (w.a.c.g.px || w.a.c.g.py) adjoint_sweep<2, false>(w.a);
        else adjoint_sweep<1, false>(w.a);
    } else {
        if (w.f.c.g.px || w.f.c.g.py) forward_sweep<2, false>(w.f);
        else forward_sweep<1, false>(w.f);
    }
    // the counter this launch did not use is idle until the sweep's next
    // launch, which counts on it: zero it now (no CTA of this launch reads it)
    if (s_cta == 0 && threadIdx.x == 0) {
        const Common& c = w.adjoint ? w.a.c : w.f.c;
        *(c.bar_sel ? &c.ctl->bar : &c.ctl->bar2) = 0u;
    }
}

}  // namespace tiled

// ------------------------------------------------------------------ host
// The TMA kernels take the stage ring in dynamic shared memory; the
// plain-load kernels need none (and keep that memory as L1 cache).
// Kernel variant of a launch: mode 0 = plain loads, 1 = TMA-staged, 2 =
// TMA-staged with periodic lateral walls; the Jacobi-K sweeps are their own
// instantiations, so the PCG kernels carry none of their code.
static int tiled_mode(const tiled::Common& c) { return c.tma ? ((c.g.px || c.g.py) ? 2 : 1) : 0; }

template <bool kJac>
static const void* forward_fn(int mode) {
    return mode == 0 ? (const void*)tiled::forward_tiled<0, kJac>
                     : (mode == 1 ? (const void*)tiled::forward_tiled<1, kJac> : (const void*)tiled::forward_tiled<2, kJac>);
}
template <bool kJac>
static const void* adjoint_fn(int mode) {
    return mode == 0 ? (const void*)tiled::adjoint_tiled<0, kJac>
                     : (mode == 1 ? (const void*)tiled::adjoint_tiled<1, kJac> : (const void*)tiled::adjoint_tiled<2, kJac>);
}

cudaError_t launch_forward_tiled(const tiled::FwdTiled& a, int grid, cudaStream_t s) {
    tiled::FwdTiled copy = a;
    void* args[] = {&copy};
    const int mode = tiled_mode(a.c);
    const void* fn = a.c.jacobi_k > 0 ? forward_fn<true>(mode) : forward_fn<false>(mode);
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(tiled::NT), args, mode ? tiled::DYN_SMEM : 0, s);
}

cudaError_t launch_adjoint_tiled(const tiled::AdjTiled& a, int grid, cudaStream_t s) {
    tiled::AdjTiled copy = a;
    void* args[] = {&copy};
    const int mode = tiled_mode(a.c);
    const void* fn = a.c.jacobi_k > 0 ? adjoint_fn<true>(mode) : adjoint_fn<false>(mode);
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(tiled::NT), args, mode ? tiled::DYN_SMEM : 0, s);
}

cudaError_t launch_batch_tiled(const tiled::BatchArgs& b, int grid, cudaStream_t s) {
    tiled::BatchArgs copy = b;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)tiled::group_tiled, dim3(grid), dim3(tiled::NT), args,
                                       tiled::DYN_SMEM, s);
}

int tiled_dynamic_smem() { return tiled::DYN_SMEM; }

namespace tiled {
__global__ void cast_pairs(const float2* __restrict__ in, float* __restrict__ out, unsigned n, float scale) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (in[i].x + in[i].y) * scale;
}
__global__ void cast_split_pairs(const float* __restrict__ hi, const float* __restrict__ lo, float* __restrict__ out,
                                 unsigned n, float scale) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (hi[i] + lo[i]) * scale;
}
}  // namespace tiled

cudaError_t launch_cast_pairs(const float2* in, float* out, unsigned n, float scale, cudaStream_t s) {
    const unsigned blocks = std::min(4096u, (n + 255u) / 256u);
    tiled::cast_pairs<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(in, out, n, scale);
    return cudaGetLastError();
}
cudaError_t launch_cast_split_pairs(const float* hi, const float* lo, float* out, unsigned n, float scale,
                                    cudaStream_t s) {
    const unsigned blocks = std::min(4096u, (n + 255u) / 256u);
    tiled::cast_split_pairs<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(hi, lo, out, n, scale);
    return cudaGetLastError();
}

// CTAs of the tiled kernels: as many as fit on the device at once (a
// cooperative launch), at most two per SM; every kernel variant gets the same.
int tiled_grid_blocks(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
    std::vector<const void*> tma_fns = {(const void*)tiled::group_tiled}, plain_fns;
    for (int mode = 0; mode < 3; ++mode)
        for (const void* f : {forward_fn<false>(mode), forward_fn<true>(mode), adjoint_fn<false>(mode),
                              adjoint_fn<true>(mode)})
            (mode ? tma_fns : plain_fns).push_back(f);
    for (const void* f : tma_fns)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, tiled::DYN_SMEM) != cudaSuccess)
            return 0;
    int per = 2;
    for (const void* f : tma_fns) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, tiled::NT, tiled::DYN_SMEM) != cudaSuccess) return 0;
        per = std::min(per, b);
    }
    for (const void* f : plain_fns) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, tiled::NT, 0) != cudaSuccess) return 0;
        per = std::min(per, b);
    }
    return per * prop.multiProcessorCount;
}

// Tensor maps of the staged passes (see TmaMaps).  The encoder comes from the
// driver through the runtime's entry-point query, so no libcuda link is needed.
bool tiled_encode_maps(tiled::TmaMaps* M, const tiled::Geo& g, const tiled::Vecs& v, const float* alpha,
                       const float* slab, unsigned slab_halves) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    if (g.nx % 4 != 0) return false;
    const cuuint64_t N = (cuuint64_t)g.S * g.nz;
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.S * 4, N * 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    // rank 3 (x, y, z) or, with nw > 0, rank 4 (x, y, z, w): w counts
    // consecutive blocks of N floats
    auto make = [&](CUtensorMap* m, const float* base, unsigned bx, unsigned by, unsigned nw, unsigned bw) {
        const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, nw};
        const cuuint32_t box[4] = {bx, by, 1, bw};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nw ? 4 : 3, (void*)base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    using tiled::HB;
    using tiled::HR;
    bool ok = true;
    for (int i = 0; i < 2; ++i) ok = ok && make(&M->uws[i], v.u[i], HB, HR, 3, 3);
    ok = ok && make(&M->u0, v.u[0], HB, HR, 0, 1) && make(&M->alpha, alpha, HB, HR, 0, 1) &&
         make(&M->pd, v.p, tiled::TX, tiled::TY, 2, 2) && make(&M->states, slab, HB, HR, slab_halves, 2) &&
         make(&M->dh, v.delta, HB, HR, 0, 1) && make(&M->sg, v.sig[0], tiled::TX, tiled::TY, 2, 1);
    return ok;
}

}  // namespace nefty
