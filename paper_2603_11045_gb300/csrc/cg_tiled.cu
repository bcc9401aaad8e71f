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
// cell from its own values; the only neighbour data a pass needs is u_{i+1}
// itself, staged plane by plane in shared memory.
//
// Work layout: the grid is cut into 32 x 32 columns (one warp per row of 32
// cells along x) and the (tile, plane) pairs are split evenly over the CTAs;
// each CTA marches up z through its planes, keeping the field of planes k-1 and
// k+1 for its own column in registers and plane k with a one-cell halo ring in a
// triple-buffered shared tile.
//
// Numerics: the stencil is evaluated in flux form, A v = v + sum_f c_f (v_c - v_q)
// (+ Robin sink), and each solve accumulates its increment delta separately so
// that T^{n+1} = T^n + delta is rounded once per step.  Inner products are
// summed per thread in FP32 over the thread's cells of one pass and then in FP64
// across threads and CTAs in a fixed order, so repeated runs are bitwise equal.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace nefty {
namespace tiled {

constexpr int BX = TX + 2, BY = TY + 2;         // shared tile with halo
constexpr int RING = 2 * BX + 2 * TY;           // halo cells per plane

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
    double* partials;   // [2][kMaxRed][G]
    unsigned G;
    unsigned epoch;     // thread 0 only
    unsigned red;       // uniform
};

// Bounded grid barrier (see solver.cu): returns false on timeout or when
// another CTA has flagged an error.
__device__ bool barrier(Sync& g) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        g.epoch += 1;
        const unsigned target = g.epoch * g.G;
        __threadfence();
        red_release(&g.ctl->bar, 1u);
        int ok = 1;
        unsigned spins = 0;
        unsigned long long t0 = 0;
        while (ld_acquire(&g.ctl->bar) < target) {
            if ((++spins & 63u) == 0) {
                if (ld_relaxed(&g.ctl->err) != kDevOk) { ok = 0; break; }
                const unsigned long long t = now_ns();
                if (t0 == 0) t0 = t;
                else if (t - t0 > kBarrierTimeoutNs) {
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

// Compensated warp sum of (hi, lo) pairs; lane 0 holds the result.
__device__ __forceinline__ void warp_sum2(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, e;
        two_sum(hi, oh, sh, e);
        lo = lo + ol + e;
        two_sum(sh, lo, hi, lo);
    }
}

// Grid sum of NV values given per thread in FP32.  The sums run on the FP32
// pipes as compensated (hi, lo) pairs, which keeps about twice the FP32
// precision: per thread over its cells, then TwoSum trees over the warp, the
// CTA and the G CTA partials (fixed order, so every run gives the same bits).
// GB300's FP64 rate is a small fraction of its FP32 rate, so no FP64 arithmetic
// is done per thread.  On return thread 0 holds the totals as doubles
// (hi + lo); the other threads' out[] is unspecified.
template <int NV>
__device__ bool grid_sum(Sync& g, const float (&in)[NV], double (&out)[NV]) {
    __shared__ float s_h[NT / 32][kMaxRed], s_l[NT / 32][kMaxRed];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float hi = in[i], lo = 0.f;
        warp_sum2(hi, lo);
        if (lane == 0) { s_h[warp][i] = hi; s_l[warp][i] = lo; }
    }
    __syncthreads();
    float2* part = reinterpret_cast<float2*>(g.partials) + (size_t)(g.red & 1u) * kMaxRed * g.G;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float hi = lane < NT / 32 ? s_h[lane][i] : 0.f, lo = lane < NT / 32 ? s_l[lane][i] : 0.f;
            warp_sum2(hi, lo);
            if (lane == 0) part[(size_t)i * g.G + blockIdx.x] = make_float2(hi, lo);
        }
    }
    if (!barrier(g)) return false;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float hi = 0.f, lo = 0.f;
            for (unsigned b = lane; b < g.G; b += 32) {
                const float2 v = part[(size_t)i * g.G + b];
                float sh, e;
                two_sum(hi, v.x, sh, e);
                lo = lo + v.y + e;
                two_sum(sh, lo, hi, lo);
            }
            warp_sum2(hi, lo);
            out[i] = (double)hi + (double)lo;
        }
    }
    g.red += 1;
    return true;
}

__device__ double block_sum(double v) {
    __shared__ double s[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < NT / 32 ? s[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// --------------------------------------------------------------- geometry
// Map a lateral coordinate through the boundary condition: wrapped when
// periodic, -1 when outside a zero-flux wall.
__device__ __forceinline__ int map_x(const Geo& g, int x) {
    if (x < 0) return g.px ? x + g.nx : -1;
    if (x >= g.nx) { x = g.px ? x - g.nx : -1; return x < g.nx ? x : -1; }
    return x;
}
__device__ __forceinline__ int map_y(const Geo& g, int y) {
    if (y < 0) return g.py ? y + g.ny : -1;
    if (y >= g.ny) { y = g.py ? y - g.ny : -1; return y < g.ny ? y : -1; }
    return y;
}

// The halo ring's RING cells are spread over the high lanes of all warps
// (slot r -> warp r % 16, lane 31 - r / 16), keeping thread 0 free to issue
// copies and every warp's share of the ring equal.  Returns -1 for no slot.
__device__ __forceinline__ int ring_slot() {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (31 - lane) * (NT / 32) + warp;
    return r < RING ? r : -1;
}

// Halo-ring slot t in [0, RING) -> (row, col) in the BY x BX shared tile.
__device__ __forceinline__ void ring_pos(int t, int& hy, int& hx) {
    if (t < BX) { hy = 0; hx = t; }
    else if (t < 2 * BX) { hy = BY - 1; hx = t - BX; }
    else if (t < 2 * BX + TY) { hy = t - 2 * BX + 1; hx = 0; }
    else { hy = t - 2 * BX - TY + 1; hx = BX - 1; }
}

// Hardware reciprocal (rcp.approx, about 1 ulp).  Used for the face values and
// the Jacobi diagonal: their rounding moves the solution far less than the
// FP32 CG arithmetic does, and every pass evaluates them identically.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Harmonic-mean face value dt * a_f = k * 2 a b / (a + b), k = dt / h^2, of the
// face between cells of diffusivity a and b (Prop. 1).  Both cells that share a
// face evaluate the same products on the same two values, so A stays exactly
// symmetric.  b = 0 (a cell beyond a zero-flux wall, as TMA fills it) gives 0.
__device__ __forceinline__ float face(float a, float b, float k) {
    return k * (2.f * a * b) * rcp_approx(a + b);
}

// Face values +x, -x, +y, -y of the own cell c = (x, y, k), from alpha.
struct Faces { float xp, xm, yp, ym; };
__device__ __forceinline__ Faces lateral_faces(const Geo& g, const float* __restrict__ al, unsigned c, int x,
                                               int y, float ac, float kx, float ky) {
    Faces f;
    const unsigned wrap_y = (unsigned)(g.ny - 1) * g.nx;
    f.xp = x + 1 < g.nx ? face(ac, al[c + 1], kx) : (g.px ? face(ac, al[c + 1 - g.nx], kx) : 0.f);
    f.xm = x > 0 ? face(ac, al[c - 1], kx) : (g.px ? face(ac, al[c + g.nx - 1], kx) : 0.f);
    f.yp = y + 1 < g.ny ? face(ac, al[c + g.nx], ky) : (g.py ? face(ac, al[c - wrap_y], ky) : 0.f);
    f.ym = y > 0 ? face(ac, al[c - g.nx], ky) : (g.py ? face(ac, al[c + wrap_y], ky) : 0.f);
    return f;
}

// --------------------------------------------------------------- marching
// Generic z-march over the planes [k0, k1) of one tile.  FieldFn(cell, own)
// returns the stencil field at a global cell; BodyFn(k, c, x, y, valid,
// fc, fxm, fxp, fym, fyp, fzm, fzp) consumes it at the own cell.  Cells outside
// a zero-flux wall give 0 (their face value is 0, so they never contribute).
template <class FieldFn, class BodyFn>
__device__ __forceinline__ void march(const Geo& g, int tile, int k0, int k1, float (*sm)[BY][BX],
                                      FieldFn field, BodyFn body) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x0 = (tile % g.tiles_x) * TX, y0 = (tile / g.tiles_x) * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < g.nx && y < g.ny;
    // where this thread's box slot maps (own slot; invalid threads may map
    // to a wrapped cell that a valid neighbour needs)
    const int mx = map_x(g, x), my = map_y(g, y);
    const bool own_mapped = mx >= 0 && my >= 0;
    const unsigned own_col = own_mapped ? (unsigned)my * g.nx + mx : 0u;
    // ring slot (first RING threads)
    int rhy = 0, rhx = 0;
    unsigned ring_col = 0;
    bool ring_mapped = false;
    const int rslot = ring_slot();
    if (rslot >= 0) {
        ring_pos(rslot, rhy, rhx);
        const int gx = map_x(g, x0 - 1 + rhx), gy = map_y(g, y0 - 1 + rhy);
        ring_mapped = gx >= 0 && gy >= 0;
        ring_col = ring_mapped ? (unsigned)gy * g.nx + gx : 0u;
    }
    auto fill = [&](int k) -> float {   // plane k into sm[k % 3]; returns own value
        float* buf = &sm[k % 3][0][0];
        const float v = own_mapped ? field(own_col + (unsigned)k * g.S, valid) : 0.f;
        buf[(ty + 1) * BX + tx + 1] = v;
        if (rslot >= 0) buf[rhy * BX + rhx] = ring_mapped ? field(ring_col + (unsigned)k * g.S, false) : 0.f;
        return v;
    };
    float fzm = 0.f;
    if (k0 > 0 && own_mapped) fzm = field(own_col + (unsigned)(k0 - 1) * g.S, valid);
    float fc = fill(k0);
    for (int k = k0; k < k1; ++k) {
        float fzp = fc;
        if (k + 1 < g.nz) fzp = fill(k + 1);
        __syncthreads();
        const float* buf = &sm[k % 3][0][0];
        const int b = (ty + 1) * BX + tx + 1;
        const float fxm = buf[b - 1], fxp = buf[b + 1], fym = buf[b - BX], fyp = buf[b + BX];
        body(k, own_col + (unsigned)k * g.S, x, y, valid, fc, fxm, fxp, fym, fyp, k > 0 ? fzm : fc, fzp);
        fzm = fc;
        fc = fzp;
    }
    __syncthreads();
}

// Iterate over this CTA's (tile, plane) segments.
template <class SegFn>
__device__ __forceinline__ void for_segments(const Geo& g, SegFn seg) {
    const unsigned long long U = g.units;
    unsigned u = (unsigned)(U * blockIdx.x / gridDim.x);
    const unsigned ue = (unsigned)(U * (blockIdx.x + 1) / gridDim.x);
    while (u < ue) {
        const int tile = (int)(u / g.nz);
        const int k0 = (int)(u % g.nz);
        const int k1 = (int)min((unsigned)g.nz, k0 + (ue - u));
        seg(tile, k0, k1);
        u += (unsigned)(k1 - k0);
    }
}


// ------------------------------------------------------------ TMA staging
// The CG iteration pass can take its inputs through the Tensor Memory
// Accelerator: for every plane a single thread issues bulk tensor copies of
// the six arrays the pass reads (u, ws, ss and alpha with a one-cell halo; p
// and delta) into one stage of a six-stage shared-memory ring, completing on
// that stage's mbarrier.  Copies run four planes ahead of the plane being
// computed.  Cells outside the grid
// arrive as zeros, which is exactly a zero-flux wall (their face values are
// zero), so this path serves grids with zero-flux lateral walls and nx % 4 == 0
// (row pitch a multiple of 16 bytes).
constexpr int NS = 6;                         // stages
constexpr int HB = TX + 8, HR = TY + 2;       // halo box: x0-4 .. x0+35, y0-1 .. y0+TY
constexpr int SZ_H = HB * HR * 4;             // 5440
constexpr int SZ_O = TX * TY * 4;             // 4096
constexpr int al128(int b) { return (b + 127) & ~127; }
constexpr int OFF_U = 0;
constexpr int OFF_W = OFF_U + al128(SZ_H);
constexpr int OFF_S = OFF_W + al128(SZ_H);
constexpr int OFF_A = OFF_S + al128(SZ_H);
constexpr int OFF_P = OFF_A + al128(SZ_H);
constexpr int OFF_D = OFF_P + al128(SZ_O);
constexpr int STAGE_BYTES = al128(OFF_D + SZ_O);
constexpr unsigned TX_BYTES = 4 * SZ_H + 2 * SZ_O;
constexpr int DYN_SMEM = NS * STAGE_BYTES + 128;   // + alignment slack

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
// Bounded wait on an mbarrier phase; false after about one second.
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

// Ring bookkeeping without division: copies are issued and waited in the same
// order, so a stage index that advances by one (mod NS) and one parity bit per
// stage describe both sides.
struct TmaRing {
    unsigned char* base;   // NS stages, 128-byte aligned
    uint32_t bar0;         // shared address of NS mbarriers (8 bytes each)
    unsigned issue_s;      // stage of the next copy (thread 0)
    unsigned wait_s;       // stage of the next wait (uniform)
    unsigned wait_ph;      // bit s: parity of the next wait on stage s (uniform)
    unsigned in_flight;    // copies issued and not yet waited (thread 0)
};

__device__ __forceinline__ unsigned ring_next(unsigned s) { return s + 1 == NS ? 0u : s + 1; }

__device__ __forceinline__ void issue_plane(TmaRing& R, const TmaMaps* M, int cur, int x0, int y0, int k) {
    const unsigned st = R.issue_s;
    const uint32_t dst = smem_u32(R.base + st * STAGE_BYTES);
    const uint32_t bar = R.bar0 + 8u * st;
    mbar_expect_tx(bar, TX_BYTES);
    tma_load3(dst + OFF_U, &M->u[cur], x0 - 4, y0 - 1, k, bar);
    tma_load3(dst + OFF_W, &M->ws[cur], x0 - 4, y0 - 1, k, bar);
    tma_load3(dst + OFF_S, &M->ss[cur], x0 - 4, y0 - 1, k, bar);
    tma_load3(dst + OFF_A, &M->alpha, x0 - 4, y0 - 1, k, bar);
    tma_load3(dst + OFF_P, &M->p, x0, y0, k, bar);
    tma_load3(dst + OFF_D, &M->delta, x0, y0, k, bar);
    R.issue_s = ring_next(st);
    R.in_flight += 1;
}

// Wait for the next stage in order; returns its index, or -1 on timeout.
__device__ __forceinline__ int wait_next(TmaRing& R) {
    const unsigned st = R.wait_s;
    const bool ok = mbar_wait(R.bar0 + 8u * st, (R.wait_ph >> st) & 1u);
    R.wait_ph ^= 1u << st;
    R.wait_s = ring_next(st);
    return ok ? (int)st : -1;
}

// After a timed-out wait: wait (again bounded) for the copies this CTA still
// has in flight, so none is landing in shared memory when the kernel exits.
__device__ void drain(TmaRing& R) {
    while (R.in_flight > 0) {
        wait_next(R);
        R.in_flight -= 1;
    }
}

// One single-reduction CG iteration over this CTA's segments, inputs staged by
// TMA.  Same arithmetic as the plain-load pass in solve().
__device__ bool iter_pass_tma(const Common& C, TmaRing& R, float (*fr)[BY][BX], int cur, float a, float bt,
                              bool first, float (&acc)[3]) {
    const Geo& g = C.g;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float* __restrict__ uo = C.v.u[cur ^ 1];
    float* __restrict__ wo = C.v.ws[cur ^ 1];
    float* __restrict__ so = C.v.ss[cur ^ 1];
    // per-thread offsets that do not change with the plane
    const int hb = (ty + 1) * HB + tx + 4;      // own cell in a halo box
    const int ob = ty * TX + tx;                 // own cell in an own-cell box
    const int fb = (ty + 1) * BX + tx + 1;       // own cell in the field tile
    const int rslot = ring_slot();
    int rhb = 0, rfb = 0;
    if (rslot >= 0) {
        int hy, hx;
        ring_pos(rslot, hy, hx);
        rhb = hy * HB + hx + 3;
        rfb = hy * BX + hx;
    }
    bool ok = true;
    if (threadIdx.x == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
    for_segments(g, [&](int tile, int k0, int k1) {
        if (!ok) return;
        const int x0 = (tile % g.tiles_x) * TX, y0 = (tile / g.tiles_x) * TY;
        const int x = x0 + tx, y = y0 + ty;
        const bool valid = x < g.nx && y < g.ny;
        const int kl = k0 > 0 ? k0 - 1 : 0;
        const int kh = k1 < g.nz ? k1 : g.nz - 1;
        int next = kl;   // next plane to copy (thread 0)
        if (threadIdx.x == 0)
            while (next <= kh && next < kl + NS) issue_plane(R, C.maps, cur, x0, y0, next++);
        auto stage_ptr = [&](int s) -> const unsigned char* { return R.base + (unsigned)s * STAGE_BYTES; };
        // u_{i+1} = u_i - a (ws_i + b ss_{i-1}) at the own cell and the ring cell
        // of one staged plane, into field buffer fbuf; returns the own value
        auto fill = [&](const unsigned char* st, float* fbuf) -> float {
            const float* U = (const float*)(st + OFF_U);
            const float* W = (const float*)(st + OFF_W);
            const float* Sv = (const float*)(st + OFF_S);
            const float vo = U[hb] - a * (first ? W[hb] : W[hb] + bt * Sv[hb]);
            fbuf[fb] = vo;
            if (rslot >= 0) fbuf[rfb] = U[rhb] - a * (first ? W[rhb] : W[rhb] + bt * Sv[rhb]);
            return vo;
        };
        // A failed (timed-out) wait aborts the whole CTA together: the decision
        // is taken with __syncthreads_or so no thread is left at a barrier.
        auto abort_uniform = [&](bool mine_ok) -> bool {
            if (!__syncthreads_or(mine_ok ? 0 : 1)) return false;
            if (threadIdx.x == 0) drain(R);
            ok = false;
            return true;
        };
        auto waited = [&]() { if (threadIdx.x == 0) R.in_flight -= 1; };
        float czm = 0.f, fzm = 0.f;
        int sm1 = -1;
        bool w_ok = true;
        if (k0 > 0) {
            sm1 = wait_next(R);
            waited();
            w_ok = sm1 >= 0;
            if (w_ok) {
                const unsigned char* st = stage_ptr(sm1);
                const float* U = (const float*)(st + OFF_U);
                const float* W = (const float*)(st + OFF_W);
                const float* Sv = (const float*)(st + OFF_S);
                fzm = U[hb] - a * (first ? W[hb] : W[hb] + bt * Sv[hb]);
            }
        }
        int sk = -1;
        if (w_ok) {
            sk = wait_next(R);
            waited();
            w_ok = sk >= 0;
        }
        int fk = 0;   // field buffer of plane k (rotates 0, 1, 2)
        float fc = 0.f;
        if (w_ok) {
            if (k0 > 0) czm = face(((const float*)(stage_ptr(sk) + OFF_A))[hb], ((const float*)(stage_ptr(sm1) + OFF_A))[hb], C.kz);
            fc = fill(stage_ptr(sk), &fr[fk][0][0]);
        }
        if (abort_uniform(w_ok)) return;
        unsigned c = (unsigned)k0 * g.S + (unsigned)y * g.nx + x;
        for (int k = k0; k < k1; ++k, c += g.S) {
            const int fk1 = fk == 2 ? 0 : fk + 1;
            float fzp = fc;
            int sk1 = -1;
            w_ok = true;
            if (k + 1 < g.nz) {
                sk1 = wait_next(R);
                waited();
                w_ok = sk1 >= 0;
                if (w_ok) fzp = fill(stage_ptr(sk1), &fr[fk1][0][0]);
            }
            if (abort_uniform(w_ok)) return;
            // plane k-1 is no longer read by anyone: refill its stage
            if (threadIdx.x == 0)
                while (next <= kh && next <= k - 1 + NS) issue_plane(R, C.maps, cur, x0, y0, next++);
            if (valid) {
                const unsigned char* st = stage_ptr(sk);
                const float* buf = &fr[fk][0][0];
                const float fxm = buf[fb - 1], fxp = buf[fb + 1], fym = buf[fb - BX], fyp = buf[fb + BX];
                const float fzmv = k > 0 ? fzm : fc;
                const float* As = (const float*)(st + OFF_A);
                const float ac = As[hb];
                const float cxp = face(ac, As[hb + 1], C.kx), cxm = face(ac, As[hb - 1], C.kx);
                const float cyp = face(ac, As[hb + HB], C.ky), cym = face(ac, As[hb - HB], C.ky);
                const float czp = sk1 >= 0 ? face(ac, ((const float*)(stage_ptr(sk1) + OFF_A))[hb], C.kz) : 0.f;
                const float rob = k + 1 == g.nz ? C.robin : 0.f;
                const float d = 1.f + cxp + cxm + cyp + cym + czp + czm + rob;
                const float Au = fc + cxp * (fc - fxp) + cxm * (fc - fxm) + cyp * (fc - fyp) + cym * (fc - fym) +
                                 czp * (fc - fzp) + czm * (fc - fzmv) + rob * fc;
                const float wn = rcp_approx(d) * Au;
                const float uold = ((const float*)(st + OFF_U))[hb];
                const float wold = ((const float*)(st + OFF_W))[hb];
                const float sn = first ? wold : wold + bt * ((const float*)(st + OFF_S))[hb];
                const float pn = first ? uold : uold + bt * ((const float*)(st + OFF_P))[ob];
                const float dl = ((const float*)(st + OFF_D))[ob] + a * pn;
                C.v.p[c] = pn;
                C.v.delta[c] = dl;
                uo[c] = fc;
                wo[c] = wn;
                so[c] = sn;
                const float r = d * fc;
                acc[0] += r * fc;
                acc[1] += Au * fc;
                acc[2] += r * r;
                czm = czp;
            }
            fzm = fc;
            fc = fzp;
            sk = sk1;
            fk = fk1;
        }
        __syncthreads();
    });
    return ok;
}

// Diagonal of A at the own cell from its six face values.
__device__ __forceinline__ float diag(const Faces& f, float czp, float czm, float rob) {
    return 1.f + f.xp + f.xm + f.yp + f.ym + czp + czm + rob;
}

// --------------------------------------------------------------- solve
// One linear solve A (x0 + delta) = x0 + e, where e (the forcing of this
// step) is given per own cell by Rhs(c, k) and the state x0 = x0hi + x0lo is
// a compensated pair (read-only).  The initial residual r0 = e - (A - I) x0 is
// formed with error-free products and sums (TwoProd through fmaf, TwoSum), so
// it is accurate relative to itself however small it is against x0; the CG
// then runs in FP32 on the increment.  On return delta holds the increment.
// Returns false if a barrier failed.
template <class RhsFn>
__device__ bool solve(const Common& C, Sync& sy, float (*sm)[BY][BX], TmaRing* ring,
                      const float* __restrict__ x0, const float* __restrict__ x0lo, RhsFn rhs, int* it_out,
                      double* rel_out) {
    const Geo& g = C.g;
    // ---- init 1: r0 = e - (A - I) x0, u0 = M^{-1} r0 ; bb, (r0,u0), (r0,r0)
    float acc3[3] = {0.f, 0.f, 0.f};
    const unsigned wrap_y = (unsigned)(g.ny - 1) * g.nx;
    for_segments(g, [&](int tile, int k0, int k1) {
        float czm = 0.f;
        march(g, tile, k0, k1, sm,
              [&](unsigned q, bool) { return x0[q]; },
              [&](int k, unsigned c, int x, int y, bool valid, float fc, float fxm, float fxp, float fym,
                  float fyp, float fzm, float fzp) {
                  if (!valid) return;
                  const float ac = C.alpha[c];
                  if (k == k0 && k > 0) czm = face(ac, C.alpha[c - g.S], C.kz);
                  const Faces f = lateral_faces(g, C.alpha, c, x, y, ac, C.kx, C.ky);
                  const float czp = k + 1 < g.nz ? face(ac, C.alpha[c + g.S], C.kz) : 0.f;
                  const float rob = k + 1 == g.nz ? C.robin : 0.f;
                  const float lc = x0lo[c];
                  float sh = 0.f, sl = 0.f;
                  // sh + sl += cf * ((fc + lc) - (hq + lq)), error-free up to the final rounding
                  auto term = [&](float cf, float hq, unsigned q) {
                      if (cf == 0.f) return;
                      float dh, dhe;
                      two_sum(fc, -hq, dh, dhe);
                      const float dl = (lc - x0lo[q]) + dhe;
                      const float pr = cf * dh;
                      const float pe = fmaf(cf, dh, -pr) + cf * dl;
                      float t, te;
                      two_sum(sh, pr, t, te);
                      sh = t;
                      sl += te + pe;
                  };
                  term(f.xp, fxp, x + 1 < g.nx ? c + 1 : c + 1 - g.nx);
                  term(f.xm, fxm, x > 0 ? c - 1 : c + g.nx - 1);
                  term(f.yp, fyp, y + 1 < g.ny ? c + g.nx : c - wrap_y);
                  term(f.ym, fym, y > 0 ? c - g.nx : c + wrap_y);
                  term(czp, fzp, c + g.S);
                  term(czm, fzm, c - g.S);
                  if (rob != 0.f) {
                      const float pr = rob * fc;
                      const float pe = fmaf(rob, fc, -pr) + rob * lc;
                      float t, te;
                      two_sum(sh, pr, t, te);
                      sh = t;
                      sl += te + pe;
                  }
                  const float e = rhs(c, k);
                  const float r = (e - sh) - sl;
                  const float dinv = rcp_approx(diag(f, czp, czm, rob));
                  const float u = dinv * r;
                  C.v.u[0][c] = u;
                  C.v.delta[c] = 0.f;
                  const float b = (fc + lc) + e;
                  acc3[0] += b * b;
                  acc3[1] += r * u;
                  acc3[2] += r * r;
                  czm = czp;
              });
    });
    // CG scalars live in thread 0 (FP64); the FP32 step lengths and the stop
    // decision reach the other threads through shared memory.
    __shared__ float s_a, s_b;
    __shared__ int s_go;
    double t3[3] = {0.0, 0.0, 0.0};
    if (!grid_sum<3>(sy, acc3, t3)) return false;
    const double bb = t3[0], lim = C.tol2 * bb;
    double gam = t3[1], rho = t3[2];
    int it = 0;
    if (threadIdx.x == 0) s_go = (rho > lim && C.max_iter > 0) ? 1 : 0;
    __syncthreads();
    if (s_go) {
        // ---- init 2: ws0 = M^{-1} A u0 ; (A u0, u0)
        float acc1[1] = {0.f};
        for_segments(g, [&](int tile, int k0, int k1) {
            float czm = 0.f;
            const float* u0 = C.v.u[0];
            march(g, tile, k0, k1, sm,
                  [&](unsigned q, bool) { return u0[q]; },
                  [&](int k, unsigned c, int x, int y, bool valid, float fc, float fxm, float fxp, float fym,
                      float fyp, float fzm, float fzp) {
                      if (!valid) return;
                      const float ac = C.alpha[c];
                      if (k == k0 && k > 0) czm = face(ac, C.alpha[c - g.S], C.kz);
                      const Faces f = lateral_faces(g, C.alpha, c, x, y, ac, C.kx, C.ky);
                      const float czp = k + 1 < g.nz ? face(ac, C.alpha[c + g.S], C.kz) : 0.f;
                      const float rob = k + 1 == g.nz ? C.robin : 0.f;
                      const float Au = fc + f.xp * (fc - fxp) + f.xm * (fc - fxm) + f.yp * (fc - fyp) +
                                       f.ym * (fc - fym) + czp * (fc - fzp) + czm * (fc - fzm) + rob * fc;
                      const float dinv = rcp_approx(diag(f, czp, czm, rob));
                      C.v.ws[0][c] = dinv * Au;
                      acc1[0] += Au * fc;
                      czm = czp;
                  });
        });
        double t1[1] = {0.0};
        if (!grid_sum<1>(sy, acc1, t1)) return false;
        double alpha = 0.0, beta = 0.0;
        if (threadIdx.x == 0) {
            alpha = gam / t1[0];
            s_a = (float)alpha;
            s_b = 0.f;
        }
        __syncthreads();
        int cur = 0;
        // ---- iterations: one pass, one reduction each
        while (true) {
            const float a = s_a, bt = s_b;
            const bool first = it == 0;
            const float* __restrict__ ui = C.v.u[cur];
            const float* __restrict__ wi = C.v.ws[cur];
            const float* __restrict__ si = C.v.ss[cur];
            float* __restrict__ uo = C.v.u[cur ^ 1];
            float* __restrict__ wo = C.v.ws[cur ^ 1];
            float* __restrict__ so = C.v.ss[cur ^ 1];
            float acc[3] = {0.f, 0.f, 0.f};
            if (C.maps) {
                if (!iter_pass_tma(C, *ring, sm, cur, a, bt, first, acc)) {
                    if (threadIdx.x == 0) atomicCAS(&C.ctl->err, kDevOk, kDevTimeout);
                    return false;
                }
            } else
            for_segments(g, [&](int tile, int k0, int k1) {
                float czm = 0.f;
                march(g, tile, k0, k1, sm,
                      [&](unsigned q, bool) {
                          const float sn = first ? wi[q] : wi[q] + bt * si[q];
                          return ui[q] - a * sn;
                      },
                      [&](int k, unsigned c, int x, int y, bool valid, float fc, float fxm, float fxp,
                          float fym, float fyp, float fzm, float fzp) {
                          if (!valid) return;
                          const float ac = C.alpha[c];
                          if (k == k0 && k > 0) czm = face(ac, C.alpha[c - g.S], C.kz);
                          const Faces f = lateral_faces(g, C.alpha, c, x, y, ac, C.kx, C.ky);
                          const float czp = k + 1 < g.nz ? face(ac, C.alpha[c + g.S], C.kz) : 0.f;
                          const float rob = k + 1 == g.nz ? C.robin : 0.f;
                          const float d = diag(f, czp, czm, rob);
                          const float Au = fc + f.xp * (fc - fxp) + f.xm * (fc - fxm) + f.yp * (fc - fyp) +
                                           f.ym * (fc - fym) + czp * (fc - fzp) + czm * (fc - fzm) + rob * fc;
                          const float wn = rcp_approx(d) * Au;
                          const float uold = ui[c];
                          const float sn = first ? wi[c] : wi[c] + bt * si[c];
                          const float pn = first ? uold : uold + bt * C.v.p[c];
                          C.v.p[c] = pn;
                          C.v.delta[c] += a * pn;
                          uo[c] = fc;
                          wo[c] = wn;
                          so[c] = sn;
                          const float r = d * fc;
                          acc[0] += r * fc;
                          acc[1] += Au * fc;
                          acc[2] += r * r;
                          czm = czp;
                      });
            });
            double t[3] = {0.0, 0.0, 0.0};
            if (!grid_sum<3>(sy, acc, t)) return false;
            ++it;
            cur ^= 1;
            if (threadIdx.x == 0) {
                rho = t[2];
                const bool go = !(rho <= lim || it >= C.max_iter);
                if (go) {
                    const double gam_new = t[0];
                    beta = gam_new / gam;
                    alpha = gam_new / (t[1] - beta * gam_new / alpha);
                    gam = gam_new;
                    s_a = (float)alpha;
                    s_b = (float)beta;
                }
                s_go = go ? 1 : 0;
            }
            __syncthreads();
            if (!s_go) break;
        }
    }
    *it_out = it;
    *rel_out = bb > 0.0 ? sqrt(rho / bb) : 0.0;
    return true;
}

__device__ __forceinline__ Sync make_sync(DevCtl* ctl, double* partials) {
    Sync s;
    s.ctl = ctl;
    s.partials = partials;
    s.G = gridDim.x;
    s.epoch = 0;
    s.red = 0;
    return s;
}

// ------------------------------------------------------------- forward
__global__ void __launch_bounds__(NT, 1) forward_tiled(FwdTiled a) {
    __shared__ float sm[3][BY][BX];
    extern __shared__ unsigned char dyn_smem[];
    __shared__ __align__(8) unsigned long long s_bars[NS];
    TmaRing ring;
    ring.base = (unsigned char*)(((uintptr_t)dyn_smem + 127) & ~(uintptr_t)127);
    ring.bar0 = smem_u32(&s_bars[0]);
    ring.issue_s = 0;
    ring.wait_s = 0;
    ring.wait_ph = 0;
    ring.in_flight = 0;
    if (a.c.maps) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < NS; ++i) mbar_init(ring.bar0 + 8u * i, 1u);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
    }

    Sync sy = make_sync(a.c.ctl, a.c.partials);
    const Geo& g = a.c.g;
    const unsigned N = g.S * (unsigned)g.nz, S = g.S;
    const unsigned stride = gridDim.x * NT;
    const unsigned c0 = blockIdx.x * NT + threadIdx.x;
    double loss = 0.0;
    for (int n = a.n0; n < a.n1; ++n) {
        // states are compensated pairs: hi in [0, N), lo in [N, 2N)
        const float* __restrict__ Tn = a.src[n - a.n0];
        float* __restrict__ Tn1 = a.dst[n - a.n0];
        const float* qmap = a.q_full ? a.q_full + (size_t)n * S : (n < a.q_steps ? a.q_face : nullptr);
        const float sc = a.src_scale;
        int it = 0;
        double rel = 0.0;
        bool ok = solve(a.c, sy, sm, &ring, Tn, Tn + N,
                        [&](unsigned c, int k) { return (qmap && k == 0) ? sc * qmap[c] : 0.f; }, &it, &rel);
        if (!ok) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.c.iters[n - a.n0] = it;
            a.c.resid[n - a.n0] = rel;
            if (it >= a.c.max_iter && rel * rel > a.c.tol2) atomicAdd(&a.c.ctl->notconv, 1);
        }
        // T^{n+1} = T^n + delta, kept as a compensated pair
        for (unsigned c = c0; c < N; c += stride) add_pair(Tn[c], Tn[N + c], a.c.v.delta[c], Tn1[c], Tn1[N + c]);
        if (!barrier(sy)) return;
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
    }
    if (a.loss_partials) {
        const double t = block_sum(loss);
        if (threadIdx.x == 0) a.loss_partials[blockIdx.x] = t;
    }
}

// ------------------------------------------------------------- adjoint
// Face-product gradient of step n at the own cells (Eq. grad_assembly):
// g_c -= sum_f (2 dt / h_f^2) alpha_q^2 / (alpha_c + alpha_q)^2 (mu_c - mu_q)(T_c - T_q).
__global__ void __launch_bounds__(NT, 1) adjoint_tiled(AdjTiled a) {
    __shared__ float sm[3][BY][BX];
    extern __shared__ unsigned char dyn_smem[];
    __shared__ __align__(8) unsigned long long s_bars[NS];
    TmaRing ring;
    ring.base = (unsigned char*)(((uintptr_t)dyn_smem + 127) & ~(uintptr_t)127);
    ring.bar0 = smem_u32(&s_bars[0]);
    ring.issue_s = 0;
    ring.wait_s = 0;
    ring.wait_ph = 0;
    ring.in_flight = 0;
    if (a.c.maps) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < NS; ++i) mbar_init(ring.bar0 + 8u * i, 1u);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
    }

    Sync sy = make_sync(a.c.ctl, a.c.partials);
    const Geo& g = a.c.g;
    const unsigned N = g.S * (unsigned)g.nz, S = g.S;
    const unsigned stride = gridDim.x * NT;
    const unsigned c0 = blockIdx.x * NT + threadIdx.x;
    const float gs = a.g_scale;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int n = a.n1; n > a.n0; --n) {
        const float* __restrict__ Tn = a.T[n - a.n0];
        const float* __restrict__ mnext = a.mu[(n + 1) & 1];
        float* __restrict__ mu = a.mu[n & 1];
        const float* ob = a.obs + (size_t)(n - 1) * S;
        int it = 0;
        double rel = 0.0;
        bool ok = solve(a.c, sy, sm, &ring, mnext, mnext + N,
                        [&](unsigned c, int) {
                            return (c >= a.obs_off && c < a.obs_off + S)
                                       ? gs * ((Tn[c] - ob[c - a.obs_off]) + Tn[N + c]) : 0.f;
                        },
                        &it, &rel);
        if (!ok) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.c.iters[a.n1 - n] = it;
            a.c.resid[a.n1 - n] = rel;
            if (it >= a.c.max_iter && rel * rel > a.c.tol2) atomicAdd(&a.c.ctl->notconv, 1);
        }
        for (unsigned c = c0; c < N; c += stride) add_pair(mnext[c], mnext[N + c], a.c.v.delta[c], mu[c], mu[N + c]);
        if (!barrier(sy)) return;
        // gradient of step n with mu^n and T^n (the next step writes only the
        // other mu buffer and the CG vectors, so no barrier is needed after it)
        for_segments(g, [&](int tile, int k0, int k1) {
            const int x = (tile % g.tiles_x) * TX + tx, y = (tile / g.tiles_x) * TY + ty;
            if (x >= g.nx || y >= g.ny) return;
            for (int k = k0; k < k1; ++k) {
                const unsigned c = (unsigned)k * S + (unsigned)y * g.nx + x;
                const float ac = a.alpha[c], mc = mu[c], tc = Tn[c], mcl = mu[N + c], tcl = Tn[N + c];
                float s = 0.f;
                auto term = [&](unsigned q, float w) {
                    const float aq = a.alpha[q];
                    const float h = aq / (ac + aq);
                    const float dm = (mc - mu[q]) + (mcl - mu[N + q]);
                    const float dT = (tc - Tn[q]) + (tcl - Tn[N + q]);
                    s += w * h * h * dm * dT;
                };
                if (x + 1 < g.nx) term(c + 1, a.wx); else if (g.px) term(c + 1 - g.nx, a.wx);
                if (x > 0) term(c - 1, a.wx); else if (g.px) term(c + g.nx - 1, a.wx);
                if (y + 1 < g.ny) term(c + g.nx, a.wy);
                else if (g.py) term(c - (unsigned)(g.ny - 1) * g.nx, a.wy);
                if (y > 0) term(c - g.nx, a.wy);
                else if (g.py) term(c + (unsigned)(g.ny - 1) * g.nx, a.wy);
                if (k + 1 < g.nz) term(c + S, a.wz);
                if (k > 0) term(c - S, a.wz);
                a.grad[c] -= (double)s;
            }
        });
    }
}

}  // namespace tiled

// ------------------------------------------------------------------ host
cudaError_t launch_forward_tiled(const tiled::FwdTiled& a, int grid, cudaStream_t s) {
    tiled::FwdTiled copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)tiled::forward_tiled, dim3(grid), dim3(tiled::NT), args,
                                       tiled::DYN_SMEM, s);
}

cudaError_t launch_adjoint_tiled(const tiled::AdjTiled& a, int grid, cudaStream_t s) {
    tiled::AdjTiled copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)tiled::adjoint_tiled, dim3(grid), dim3(tiled::NT), args,
                                       tiled::DYN_SMEM, s);
}

int tiled_dynamic_smem() { return tiled::DYN_SMEM; }

int tiled_grid_blocks(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(tiled::forward_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, tiled::DYN_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tiled::adjoint_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, tiled::DYN_SMEM) !=
            cudaSuccess)
        return 0;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, tiled::forward_tiled, tiled::NT, tiled::DYN_SMEM) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tiled::adjoint_tiled, tiled::NT, tiled::DYN_SMEM) !=
        cudaSuccess)
        return 0;
    int per = a < b ? a : b;
    if (per > 2) per = 2;
    return per * prop.multiProcessorCount;
}

// Tensor maps of one iteration pass (see TmaMaps).  The encoder comes from the
// driver through the runtime's entry-point query, so no libcuda link is needed.
bool tiled_encode_maps(tiled::TmaMaps* M, const tiled::Geo& g, float* const u[2], float* const ws[2],
                       float* const ss[2], float* p, float* delta, const float* alpha) {
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
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.S * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    auto make = [&](CUtensorMap* m, const float* base, unsigned bx, unsigned by) {
        const cuuint32_t box[3] = {bx, by, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    bool ok = true;
    for (int i = 0; i < 2; ++i) {
        ok = ok && make(&M->u[i], u[i], tiled::HB, tiled::HR);
        ok = ok && make(&M->ws[i], ws[i], tiled::HB, tiled::HR);
        ok = ok && make(&M->ss[i], ss[i], tiled::HB, tiled::HR);
    }
    ok = ok && make(&M->alpha, alpha, tiled::HB, tiled::HR) && make(&M->p, p, tiled::TX, tiled::TY) &&
         make(&M->delta, delta, tiled::TX, tiled::TY);
    return ok;
}

}  // namespace nefty
