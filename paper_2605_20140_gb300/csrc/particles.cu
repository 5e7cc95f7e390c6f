// Particle side of the SIPF-W step on sm_103a: Philox noise, the
// Euler-Maruyama push with trilinear gather (paper Eq. u_hat_update, Alg. 2,
// Eq. g2ph), the particle-to-grid deposit (Alg. 1), the per-step binning of
// particles by tile, and FP64 diagnostics.
//
// Storage (two buffers, ping-pong): structure of arrays with positions in
// grid units s = (x - x_min)/h (float32), the log-mass relative to a fixed
// reference, dl = log a - logref (float64), and persistent ids (uint32).
// Particles are bucketed by tile (8^3 cells); bucket t of a buffer occupies
// [bstart[t], bstart[t] + cap[t]) and holds min(cnt[t], cap[t]) particles in
// unspecified order; arrivals beyond the capacity go to an overflow region
// of N slots, so no particle is ever dropped.
//
// One step is one persistent kernel over "items" (<= 1024 particles of one
// bucket, or of the overflow region): for each particle it deposits a R_h of
// X^(n-1) into a 9^3 shared-memory node block of the tile (integer fixed
// point: float32 contributions scaled by 2^S below 2^21 and rounded to
// integers, summed exactly, so the density does not depend on particle order
// and needs no float atomics), gathers grad v and w at X^(n-1), draws the Philox normals,
// pushes, updates the log-mass, and writes the particle into its new tile's
// bucket straight from registers: the lanes of a warp bound for the same
// tile reserve consecutive slots with one global atomic.  A one-block plan
// kernel then builds the next step's items and the next bucket layout from
// the counts.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sipf_internal.cuh"

namespace sipf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// (2 (b >> 9) + 1) 2^-24, in (0, 1): the float 1 + (b >> 9) 2^-23 minus
// 1 - 2^-24; the difference has at most 24 significant bits, so it is exact.
__device__ __forceinline__ float unit_open(uint32_t b) {
    return __fsub_rn(__uint_as_float(0x3F800000u | (b >> 9)), __uint_as_float(0x3F7FFFFFu));
}

// ------------------------------------------------------------------ short math
// Box-Muller needs -2 ln u, a square root and cos/sin(2 pi u) of uniforms
// u in (0, 1) with at most 24 significant bits, and the mass update needs
// ln(1 + x) for |x| <= tau.  Their arguments lie in these known ranges, so
// branch-free forms from textbook series suffice (the logarithm from the
// atanh series, sine and cosine from their Taylor series on an eighth of a
// turn); each is within a few float32 ulp, checked against the FP64
// oracle's normals and masses.

// float(e) for |e| < 2^22: the low mantissa bits of 1.5 2^23 + e.
__device__ __forceinline__ float small_int_to_float(int e) {
    return __fsub_rn(__int_as_float(0x4B400000 + e), 12582912.0f);
}

// -2 ln u for u in (0, 1): u = m 2^e with m in [sqrt(1/2), sqrt(2)) (the
// exponent taken from the bits of u / sqrt(1/2)), ln m = 2 atanh(s) with
// s = (m - 1)/(m + 1), |s| <= 0.1716, summed to s^9 (remainder < 3e-9
// relative).
__device__ __forceinline__ float neg2_log_unit(float u) {
    const int e = static_cast<int>(__float_as_uint(u) - 0x3F3504F3u) >> 23;
    const float m = __int_as_float(__float_as_int(u) - (e << 23));
    const float f = __fsub_rn(m, 1.0f);
    const float s = __fdividef(f, __fadd_rn(2.0f, f));
    const float z = __fmul_rn(s, s);
    // -2 ln m = s (-4 - z (4/3 + z (4/5 + z (4/7 + z 4/9))))
    float p = __fmaf_rn(z, -4.0f / 9.0f, -4.0f / 7.0f);
    p = __fmaf_rn(z, p, -4.0f / 5.0f);
    p = __fmaf_rn(z, p, -4.0f / 3.0f);
    p = __fmaf_rn(z, p, -4.0f);
    return __fmaf_rn(small_int_to_float(e), -1.3862943611198906f, __fmul_rn(s, p));
}

// sqrt(x) for 0 < x < 2^126: x times the hardware reciprocal square root.
__device__ __forceinline__ float sqrt_pos(float x) { return __fmul_rn(x, rsqrtf(x)); }

// cos 2 pi u and sin 2 pi u for u in (0, 1) with at most 24 significant
// bits.  a = min(u, 1 - u) and b = min(a, 1/2 - a) are exact, and with
// theta = 2 pi b in [0, pi/2]: cos 2 pi u = cos theta, negated for a > 1/4,
// and sin 2 pi u = sin theta, negated for u > 1/2.  cos theta and
// sin theta / b come from their Taylor series to theta^12 and theta^13,
// evaluated in b^2 (remainders below 7e-9).
struct QuarterTurn {
    float b, p;          // b in [0, 1/4], p = b^2
    bool neg_cos;        // a > 1/4
};
__device__ __forceinline__ QuarterTurn quarter_turn(float u) {
    const float a = fminf(u, __fsub_rn(1.0f, u));
    QuarterTurn q;
    q.b = fminf(a, __fsub_rn(0.5f, a));
    q.p = __fmul_rn(q.b, q.b);
    q.neg_cos = a > 0.25f;
    return q;
}
__device__ __forceinline__ float cos_series(float p) {
    float c = __fmaf_rn(p, 7.903536371318465f, -26.426256783374388f);
    c = __fmaf_rn(p, c, 60.24464137187664f);
    c = __fmaf_rn(p, c, -85.45681720669371f);
    c = __fmaf_rn(p, c, 64.93939402266828f);
    c = __fmaf_rn(p, c, -19.739208802178716f);
    return __fmaf_rn(p, c, 1.0f);
}
__device__ __forceinline__ float sin_series(float b, float p) {
    float c = __fmaf_rn(p, 3.8199525848482803f, -15.094642576822984f);
    c = __fmaf_rn(p, c, 42.058693944897634f);
    c = __fmaf_rn(p, c, -76.70585975306136f);
    c = __fmaf_rn(p, c, 81.60524927607504f);
    c = __fmaf_rn(p, c, -41.341702240399755f);
    c = __fmaf_rn(p, c, 6.283185307179586f);
    return __fmul_rn(b, c);
}
__device__ __forceinline__ float cos_2pi(float u) {
    const QuarterTurn q = quarter_turn(u);
    const float c = cos_series(q.p);
    return q.neg_cos ? -c : c;
}
__device__ __forceinline__ float2 cis_2pi(float u) {
    const QuarterTurn q = quarter_turn(u);
    const float c = cos_series(q.p), sn = sin_series(q.b, q.p);
    return make_float2(q.neg_cos ? -c : c, u > 0.5f ? -sn : sn);
}

// Box-Muller on the four words of one Philox block: three standard normals,
// z0, z1 from (u0, u1) and z2 from (u2, u3).
__device__ __forceinline__ float3 box_muller(const uint4 b) {
    const float r01 = sqrt_pos(neg2_log_unit(unit_open(b.x)));
    const float r23 = sqrt_pos(neg2_log_unit(unit_open(b.z)));
    const float2 e1 = cis_2pi(unit_open(b.y));
    const float c3 = cos_2pi(unit_open(b.w));
    return make_float3(__fmul_rn(r01, e1.x), __fmul_rn(r01, e1.y), __fmul_rn(r23, c3));
}

// 2^x (hardware approximation, relative error about 2^-22).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ln(1 + x) = 2 atanh(s) with s = x/(2 + x), for |x| <= 1/16 (|s| <= 0.0323),
// summed to s^7 (remainder below 1e-12 relative).
__device__ __forceinline__ float log1p_from_s(float s) {
    const float z = __fmul_rn(s, s);
    return __fmul_rn(s, __fmaf_rn(z, __fmaf_rn(z, __fmaf_rn(z, 2.0f / 7.0f, 2.0f / 5.0f),
                                                2.0f / 3.0f),
                                  2.0f));
}

// Three standard normals of particle `id` in step n: Box-Muller on the four
// Philox words of counter (n, 0, id, 0).
__device__ __forceinline__ float3 brownian(uint32_t id, uint32_t n, uint32_t k0, uint32_t k1,
                                           uint4* raw = nullptr) {
    const uint4 b = philox4x32_10(make_uint4(n, 0u, id, 0u), k0, k1);
    if (raw) *raw = b;
    return box_muller(b);
}

// ------------------------------------------------------------------ cells
struct Cell {
    int cx, cy, cz;      // cell of the particle
    float fx, fy, fz;    // fractional position in the cell
};

// Positions are in [0, H): every position a buffer holds went through the
// periodic wrap (non-finite values become 0).  For 0 <= s < 2^23, 2^23 + s
// rounded toward zero is 2^23 + floor(s): its low mantissa bits are the cell
// and subtracting 2^23 gives floor(s) as a float, both exact (no conversion
// instructions).  The paths that index global memory by the cell clamp it
// (clamp_cell); the tile paths check the cell against the tile.
__device__ __forceinline__ void split_cell(float s, int H, int& cell, float& frac) {
    const float t = __fadd_rz(s, 8388608.0f);
    cell = static_cast<int>(__float_as_uint(t) - 0x4B000000u);
    frac = __fsub_rn(s, __fsub_rn(t, 8388608.0f));
}

__device__ __forceinline__ int clamp_cell(int c, int H) { return min(max(c, 0), H - 1); }

// The cell with its indices clamped to [0, H) (for kernels that index
// per-cell or per-tile arrays by it).
__device__ __forceinline__ Cell locate_clamped(float x, float y, float z, int H);

__device__ __forceinline__ Cell locate(float x, float y, float z, int H) {
    Cell c;
    split_cell(x, H, c.cx, c.fx);
    split_cell(y, H, c.cy, c.fy);
    split_cell(z, H, c.cz, c.fz);
    return c;
}

__device__ __forceinline__ Cell locate_clamped(float x, float y, float z, int H) {
    Cell c = locate(x, y, z, H);
    c.cx = clamp_cell(c.cx, H);
    c.cy = clamp_cell(c.cy, H);
    c.cz = clamp_cell(c.cz, H);
    return c;
}

// i mod H for -H <= i < 2H.
__device__ __forceinline__ int wrap_index(int i, int H) { return i < 0 ? i + H : (i >= H ? i - H : i); }

__device__ __forceinline__ int tile_of(int cx, int cy, int cz, int T) {
    return ((cz >> 3) * T + (cy >> 3)) * T + (cx >> 3);
}

__device__ __forceinline__ uint32_t cell_key(int cx, int cy, int cz, int T) {
    return (static_cast<uint32_t>(tile_of(cx, cy, cz, T)) << 9) |
           static_cast<uint32_t>(((cz & 7) << 6) | ((cy & 7) << 3) | (cx & 7));
}

// The eight trilinear weights R_h(X - node) h^3 of a particle's cell corners
// (Alg. 1, 2), corner k at offset (k & 1, (k >> 1) & 1, k >> 2): products of
// (1 - f, f) along each axis.  The deposit and the gather share them.
__device__ __forceinline__ void corner_weights(const Cell& c, float (&W)[8]) {
    const float wx0 = __fsub_rn(1.0f, c.fx), wy0 = __fsub_rn(1.0f, c.fy);
    const float wz0 = __fsub_rn(1.0f, c.fz);
    const float xy[4] = {__fmul_rn(wx0, wy0), __fmul_rn(c.fx, wy0), __fmul_rn(wx0, c.fy),
                         __fmul_rn(c.fx, c.fy)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        W[k] = __fmul_rn(xy[k], wz0);
        W[4 + k] = __fmul_rn(xy[k], c.fz);
    }
}

// sum_k W[k] a[k] per component (K_h = h^3 R_h, Alg. 2).
__device__ __forceinline__ float4 interpolate8(const float4 (&a)[8], const float (&W)[8]) {
    float4 r = make_float4(__fmul_rn(W[0], a[0].x), __fmul_rn(W[0], a[0].y),
                           __fmul_rn(W[0], a[0].z), __fmul_rn(W[0], a[0].w));
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        r.x = __fmaf_rn(W[k], a[k].x, r.x);
        r.y = __fmaf_rn(W[k], a[k].y, r.y);
        r.z = __fmaf_rn(W[k], a[k].z, r.z);
        r.w = __fmaf_rn(W[k], a[k].w, r.w);
    }
    return r;
}

// Interpolation of the float4 field (dv/dx, dv/dy, dv/dz, w) from global
// memory (periodic; the cell is clamped).
__device__ __forceinline__ float4 gather4(const float4* __restrict__ G, const Cell& c, int H,
                                          const float (&W)[8]) {
    const int cx = clamp_cell(c.cx, H), cy = clamp_cell(c.cy, H), cz = clamp_cell(c.cz, H);
    const int x1 = cx + 1 < H ? cx + 1 : 0;
    const int y1 = cy + 1 < H ? cy + 1 : 0;
    const int z1 = cz + 1 < H ? cz + 1 : 0;
    float4 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int nx = (k & 1) ? x1 : cx, ny = ((k >> 1) & 1) ? y1 : cy, nz = (k >> 2) ? z1 : cz;
        a[k] = __ldg(G + (nz * H + ny) * H + nx);
    }
    return interpolate8(a, W);
}

// The same from a tile's 9^3 node block in shared memory (node (lx, ly, lz)
// at (lz * 9 + ly) * 9 + lx).
__device__ __forceinline__ float4 gather4_block(const float4* B, int base, const float (&W)[8]) {
    float4 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = B[base + (k & 1) + ((k >> 1) & 1) * 9 + (k >> 2) * 81];
    return interpolate8(a, W);
}

// Periodic wrap into [0, H); a result that rounds to H becomes 0.
__device__ __forceinline__ float wrap(float s, float Hf, int* bad) {
    if (s >= 0.0f && s < Hf) return s;
    if (!isfinite(s)) {
        *bad = 1;
        return 0.0f;
    }
    float r = __fsub_rn(s, __fmul_rn(Hf, floorf(__fdiv_rn(s, Hf))));
    if (r < 0.0f) r = __fadd_rn(r, Hf);
    if (!(r < Hf)) r = 0.0f;
    return r;
}

struct Buf {
    float* sx;
    float* sy;
    float* sz;
    double* dl;
    uint32_t* id;
};

struct Layout {
    const int* bstart;
    const int* cap;
    int* cnt;
    int* ovf;
    int ovf_base;
    int ovf_cap;
};

// ------------------------------------------------------------------ the step kernel
constexpr int kNT = 256;                  // threads of the step kernel
constexpr int kPT = 4;                    // particles per thread and item
constexpr int kItem = kNT * kPT;          // particles per item
constexpr int kBlock = 9 * 9 * 9;         // nodes of a tile's gather block
constexpr int kSparsePerTile = 256;       // below this mean tile occupancy, skip idle warps

// Deposit node block of a tile for assignment order ORDER: local node
// coordinates [-DO, 8 + DO] per axis (trilinear: the cells' corners 0..8;
// R^(4): one more node on each side for the star arms).  MIN_BLOCKS: blocks
// per SM the register budget is set for (48 and 60 registers per thread).
template <int ORDER> struct DepBlock {
    static constexpr int DO = ORDER == 4 ? 1 : 0;
    static constexpr int B = 9 + 2 * DO;
    static constexpr int N = B * B * B;
    static constexpr int MIN_BLOCKS = ORDER == 4 ? 4 : 5;
    static __device__ __forceinline__ int idx(int lx, int ly, int lz) {
        return ((lz + DO) * B + (ly + DO)) * B + (lx + DO);
    }
};

// round(v) for |v| < 2^22, ties to even (as __float2int_rn): the low mantissa
// bits of 1.5 2^23 + v.
__device__ __forceinline__ int round_signed_small(float v) {
    return __float_as_int(__fadd_rn(v, 12582912.0f)) - 0x4B400000;
}

// Wrap of a pushed position, all three axes at once: positions normally stay
// in [0, H), so the full periodic reduction runs only when one leaves it.
__device__ __forceinline__ void wrap3(float& x, float& y, float& z, float Hf, int* bad) {
    // [0, H) as bit patterns: non-negative floats order like their bits, and
    // negative values, infinities and NaNs compare above H (-0 goes to wrap,
    // which keeps it)
    const uint32_t hb = __float_as_uint(Hf);
    if (!(__float_as_uint(x) < hb && __float_as_uint(y) < hb && __float_as_uint(z) < hb)) {
        x = wrap(x, Hf, bad);
        y = wrap(y, Hf, bad);
        z = wrap(z, Hf, bad);
    }
}

// Tile of a position in [0, H) (the cell split without the fraction).
__device__ __forceinline__ int tile_at(float x, float y, float z, int T) {
    const int cx = static_cast<int>(__float_as_uint(__fadd_rz(x, 8388608.0f)) - 0x4B000000u);
    const int cy = static_cast<int>(__float_as_uint(__fadd_rz(y, 8388608.0f)) - 0x4B000000u);
    const int cz = static_cast<int>(__float_as_uint(__fadd_rz(z, 8388608.0f)) - 0x4B000000u);
    return ((cz >> 3) * T + (cy >> 3)) * T + (cx >> 3);
}

// Asks the copy engine to bring the 16-byte-aligned interior of elements
// [beg, end) of a particle array into L2 (a bulk prefetch: no registers, no
// completion to wait for).  The range lies inside the array.
__device__ __forceinline__ void prefetch_l2(const void* base, size_t elem, int beg, int end) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(base);
    const uintptr_t lo = (a + static_cast<size_t>(beg) * elem + 15) & ~static_cast<uintptr_t>(15);
    const uintptr_t hi = (a + static_cast<size_t>(end) * elem) & ~static_cast<uintptr_t>(15);
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo),
                     "r"(static_cast<uint32_t>(hi - lo))
                     : "memory");
}

// Mask of the lanes below this one.
__device__ __forceinline__ unsigned lanes_below() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// A slot in the overflow region, or -1 (with the status bit) when it is full.
__device__ __forceinline__ int overflow_slot(const Layout& L, int* status) {
    const int o = atomicAdd(L.ovf, 1);
    if (o < L.ovf_cap) return L.ovf_base + o;
    atomicOr(status, kStatusSlot);
    return -1;
}

// What one run's particle step reads: the single-run kernel builds it from
// its launch arguments, the ensemble kernel from its run table.
struct StepView {
    int H;
    float drift, noise, tau;
    uint32_t k0, k1;
    int push;
    const StepScalars* sc;
    const float4* G;
    Buf src, dst;
    Layout L;
    const Item* items;
    unsigned long long* acc;
    int* status;
    int do_deposit, do_move;
};

// Philox round keys: from the launch arguments (precomputed), or advanced by
// the Weyl constants from the key (the ensemble kernel, whose runs have
// keys of their own).
struct KeysGiven {
    const uint32_t (&rk)[20];
    __device__ __forceinline__ uint4 operator()(uint4 c) const { return philox4x32_10(c, rk); }
};
struct KeysScheduled {
    const StepView& v;
    __device__ __forceinline__ uint4 operator()(uint4 c) const {
        return philox4x32_10(c, v.k0, v.k1);
    }
};

// Shared memory of the step kernels.
template <int ORDER> struct StepShared {
    int dep[DepBlock<ORDER>::N];          // node sums of the items since the last flush
    long long dep64[DepBlock<ORDER>::N];  // node sums of the tile's items so far
    float4 gblk[kBlock];                  // (dv/dx, dv/dy, dv/dz, w) on the tile's 9^3 nodes
    int tslot[2];                         // capacity and first slot of the item tile's bucket
};

// Items [i_lo, i_hi) of one run: deposit of X^(n-1), gather, noise, push,
// mass update and binning of every particle.  dep and dep64 are zero on entry
// and on exit.
template <int ORDER, bool SKIP, class Keys>
__device__ __forceinline__ void step_items(const StepView& v, const Keys& keys, int i_lo, int i_hi,
                                           StepShared<ORDER>& sh) {
    using DB = DepBlock<ORDER>;
    // Item sums in 32 bits: the trilinear contributions are non-negative and
    // below 2^19.5 (the deposit scale's bound), so kFlushItems items (4096
    // particles) sum below 2^32 unsigned; R^(4)'s signed sums are moved to
    // the 64-bit tile sums after every item.
    constexpr int kFlushItems = ORDER == 2 ? 4 : 1;
    int* dep = sh.dep;
    long long* dep64 = sh.dep64;
    float4* gblk = sh.gblk;
    int* tslot = sh.tslot;
    const int H = v.H, T = H >> 3;
    const float Hf = __int2float_rn(H);
    const uint32_t step_n = v.sc->n;               // Philox counter word 0 of this step
    const float dscale = v.sc->deposit_scale;      // 2^S of the fixed-point deposit
    const float dshift = static_cast<float>(v.sc->deposit_shift);
    // a contribution's mass in deposit units, a 2^S = 2^(dl log2 e + S), is
    // below 2^19.5 by the choice of S; the clamp keeps a corrupt log-mass
    // (NaN) inside the bound the item sums rely on
    constexpr float kMaxLog2Unit = 19.49f;
    const Buf& src = v.src;
    const Buf& dst = v.dst;
    const Layout& L = v.L;
    unsigned long long* acc = v.acc;
    const float4* G = v.G;
    int* status = v.status;
    const int do_deposit = v.do_deposit, do_move = v.do_move;
    int cur = -1, cx0 = 0, cy0 = 0, cz0 = 0;   // tile held in dep64 / gblk, its first cell
    int pending = 0;                           // items summed in dep since its last flush
    for (int item_idx = i_lo; item_idx <= i_hi; ++item_idx) {
        const Item it = item_idx < i_hi ? v.items[item_idx] : Item{-1, 0, 0, 0, 0, 0, 0, 0};
        const int tile = it.tile;
        if (threadIdx.x < 5 && item_idx + 1 < i_hi) {
            // the next item's particles are read in about one item's time: have
            // them in L2 by then (one array per thread)
            const Item nx = v.items[item_idx + 1];
            const int k = threadIdx.x;
            const void* arr = k == 0 ? static_cast<const void*>(src.sx)
                            : k == 1 ? static_cast<const void*>(src.sy)
                            : k == 2 ? static_cast<const void*>(src.sz)
                            : k == 3 ? static_cast<const void*>(src.dl)
                                     : static_cast<const void*>(src.id);
            prefetch_l2(arr, k == 3 ? sizeof(double) : sizeof(float), nx.beg, nx.end);
        }
        const bool change = tile != cur || tile < 0;
        // every thread moves its own nodes (j = threadIdx.x + k kNT) from dep
        // to dep64 and from dep64 to the grid, so no barrier is needed between
        // the two; the barrier that ended the last item ordered them after
        // its atomics
        if (do_deposit && pending > 0 && (change || pending == kFlushItems)) {
            for (int j = threadIdx.x; j < DB::N; j += kNT) {
                const int d = dep[j];
                if (d) {
                    dep64[j] += ORDER == 2 ? static_cast<long long>(static_cast<unsigned>(d))
                                           : static_cast<long long>(d);
                    dep[j] = 0;
                }
            }
            pending = 0;
        }
        if (change) {
            if (cur >= 0 && do_deposit) {
                // flush the finished tile's node block into the grid accumulator
                // (two's complement sums)
                for (int j = threadIdx.x; j < DB::N; j += kNT) {
                    const long long d = dep64[j];
                    if (d) {
                        const int lx = j % DB::B - DB::DO, ly = (j / DB::B) % DB::B - DB::DO;
                        const int lz = j / (DB::B * DB::B) - DB::DO;
                        const int nx = wrap_index(cx0 + lx, H), ny = wrap_index(cy0 + ly, H);
                        const int nz = wrap_index(cz0 + lz, H);
                        atomicAdd(acc + (nz * H + ny) * H + nx, static_cast<unsigned long long>(d));
                        dep64[j] = 0;
                    }
                }
            }
            if (item_idx == i_hi) break;
            cur = tile;
            cx0 = it.tx * 8;
            cy0 = it.ty * 8;
            cz0 = it.tz * 8;
            if (do_move && v.push && tile >= 0) {
                // the tile's node block of the gather array (periodic), 9 float4 per row
                for (int q = threadIdx.x; q < kBlock; q += kNT) {
                    const int lx = q % 9, ly = (q / 9) % 9, lz = q / 81;
                    const int nx = cx0 + lx < H ? cx0 + lx : cx0 + lx - H;
                    const int ny = cy0 + ly < H ? cy0 + ly : cy0 + ly - H;
                    const int nz = cz0 + lz < H ? cz0 + lz : cz0 + lz - H;
                    gblk[q] = __ldg(G + (nz * H + ny) * H + nx);
                }
            }
        }
        const int tx0 = cx0, ty0 = cy0, tz0 = cz0;
        // the destination bucket of the particles that stay in this tile (the
        // common case: a step moves a particle by a fraction of a cell)
        const bool binned = tile >= 0;
        if (do_move && binned && threadIdx.x == 0) {
            tslot[0] = __ldg(L.cap + tile);
            tslot[1] = __ldg(L.bstart + tile);
        }
        __syncthreads();
        int bad = 0;
        // SKIP: only the iterations with an element for this warp (short items,
        // common in small runs, leave whole warps idle; the count is
        // warp-uniform, so the warp-wide votes below see whole warps).  Dense
        // runs take all kPT iterations, which keeps a register free.
        int jn = kPT;
        if constexpr (SKIP) {
            const int wfirst = it.beg + static_cast<int>(threadIdx.x & ~31u);
            jn = it.end > wfirst ? min(kPT, (it.end - wfirst + kNT - 1) / kNT) : 0;
        }
        for (int j = 0; j < jn; ++j) {
            const int e = j * kNT + threadIdx.x;     // element of the item, coalesced
            const int i = it.beg + e;
            const bool valid = i < it.end;
            float px = 0.f, py = 0.f, pz = 0.f;
            double pl = 0.0;
            uint32_t pid = 0u;
            if (valid) {
                // read and written once per step: evict first, so that the
                // gather blocks and deposit sums keep their place in L2
                px = __ldcs(src.sx + i);
                py = __ldcs(src.sy + i);
                pz = __ldcs(src.sz + i);
                pl = __ldcs(src.dl + i);
                pid = __ldcs(src.id + i);
            }
            const Cell c = locate(px, py, pz, H);
            const int lx = c.cx - tx0, ly = c.cy - ty0, lz = c.cz - tz0;
            const bool in_tile = binned && ((lx | ly | lz) & ~7) == 0;
            if (binned && valid && !in_tile) bad |= 2;   // bucket does not match position

            float W[8];
            corner_weights(c, W);
            if (do_deposit && valid) {
                // a_p R_h(X_p, node) h^3 in units of exp(logref) 2^-S as integers
                if constexpr (ORDER == 2) {
                    const float ea = exp2_approx(
                        fminf(__fmaf_rn(__double2float_rn(pl), 1.4426950408889634f, dshift),
                              kMaxLog2Unit));
                    // round(ea W[k]) in one rounding: ea W[k] < 2^22, so the
                    // fused 2^23 + ea W[k] has unit spacing
                    uint32_t q[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        q[k] = __float_as_uint(__fmaf_rn(ea, W[k], 8388608.0f)) - 0x4B000000u;
                    if (in_tile) {
                        // particles of a bucket are in random cells of the tile, so lanes
                        // rarely collide: one shared 32-bit atomic per corner
                        unsigned* depu = reinterpret_cast<unsigned*>(dep) + DB::idx(lx, ly, lz);
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            atomicAdd(depu + (k & 1) + ((k >> 1) & 1) * 9 + (k >> 2) * 81, q[k]);
                    } else {
                        const int cx = clamp_cell(c.cx, H), cy = clamp_cell(c.cy, H);
                        const int cz = clamp_cell(c.cz, H);
                        const int x1 = cx + 1 < H ? cx + 1 : 0;
                        const int y1 = cy + 1 < H ? cy + 1 : 0;
                        const int z1 = cz + 1 < H ? cz + 1 : 0;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int nx = (k & 1) ? x1 : cx, ny = ((k >> 1) & 1) ? y1 : cy;
                            const int nz = (k >> 2) ? z1 : cz;
                            if (q[k])
                                atomicAdd(acc + (nz * H + ny) * H + nx,
                                          static_cast<unsigned long long>(q[k]));
                        }
                    }
                } else {
                    // R^(4): the 8 corners carry the trilinear weight times
                    // g = 1 + sum_j f_j (1 - f_j) / 2; along axis j the nodes c_j - 1 and
                    // c_j + 2 carry -f (1 - f)(2 - f) / 6 and -f (1 - f)(1 + f) / 6 times
                    // the bilinear weight of the other two axes (cases of R_h^(4))
                    const float ea = fminf(__fmul_rn(expf(__double2float_rn(pl)), dscale), 741455.0f);
                    const float fx = c.fx, fy = c.fy, fz = c.fz;
                    const float wx0 = __fsub_rn(1.0f, fx), wy0 = __fsub_rn(1.0f, fy);
                    const float wz0 = __fsub_rn(1.0f, fz);
                    const float bx = __fmul_rn(fx, wx0), by = __fmul_rn(fy, wy0), bz = __fmul_rn(fz, wz0);
                    const float g = __fadd_rn(1.0f, __fmul_rn(0.5f, __fadd_rn(__fadd_rn(bx, by), bz)));
                    const float sx[2] = {__fmul_rn(__fmul_rn(bx, __fsub_rn(2.0f, fx)), -1.0f / 6.0f),
                                         __fmul_rn(__fmul_rn(bx, __fadd_rn(1.0f, fx)), -1.0f / 6.0f)};
                    const float sy[2] = {__fmul_rn(__fmul_rn(by, __fsub_rn(2.0f, fy)), -1.0f / 6.0f),
                                         __fmul_rn(__fmul_rn(by, __fadd_rn(1.0f, fy)), -1.0f / 6.0f)};
                    const float sz[2] = {__fmul_rn(__fmul_rn(bz, __fsub_rn(2.0f, fz)), -1.0f / 6.0f),
                                         __fmul_rn(__fmul_rn(bz, __fadd_rn(1.0f, fz)), -1.0f / 6.0f)};
                    const float wx[2] = {wx0, fx}, wy[2] = {wy0, fy}, wz[2] = {wz0, fz};
                    const float eg = __fmul_rn(ea, g);
                    auto emit = [&](int ox, int oy, int oz, float value) {
                        const int q = round_signed_small(value);
                        if (!q) return;
                        if (in_tile) {
                            atomicAdd(dep + DB::idx(lx + ox, ly + oy, lz + oz), q);
                        } else {
                            const int nx = wrap_index(clamp_cell(c.cx, H) + ox, H);
                            const int ny = wrap_index(clamp_cell(c.cy, H) + oy, H);
                            const int nz = wrap_index(clamp_cell(c.cz, H) + oz, H);
                            atomicAdd(acc + (nz * H + ny) * H + nx,
                                      static_cast<unsigned long long>(static_cast<long long>(q)));
                        }
                    };
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
                        emit(dx, dy, dz, __fmul_rn(eg, __fmul_rn(__fmul_rn(wx[dx], wy[dy]), wz[dz])));
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int side = k & 1, u = (k >> 1) & 1, w2 = k >> 2;
                        const int o = side ? 2 : -1;
                        emit(o, u, w2, __fmul_rn(ea, __fmul_rn(sx[side], __fmul_rn(wy[u], wz[w2]))));
                        emit(u, o, w2, __fmul_rn(ea, __fmul_rn(sy[side], __fmul_rn(wx[u], wz[w2]))));
                        emit(u, w2, o, __fmul_rn(ea, __fmul_rn(sz[side], __fmul_rn(wx[u], wy[w2]))));
                    }
                }
            }

            if (do_move) {
                if (v.push && valid) {
                    const float4 g = in_tile ? gather4_block(gblk, (lz * 9 + ly) * 9 + lx, W)
                                             : gather4(G, c, H, W);
                    // mass factor 1 + x, x = tau (rho(w_H) - 1), rho(w) = 2w/(1+w)
                    // (Eq. u_hat_update); ln(1 + x) = 2 atanh(x/(2 + x)) and
                    // x/(2 + x) = n/(2(1 + w) + n) with n = tau (w - 1)
                    float inc;
                    if (v.tau <= 0.0625f) {
                        const float n = __fmaf_rn(v.tau, g.w, -v.tau);
                        inc = log1p_from_s(__fdividef(n, __fadd_rn(__fmaf_rn(2.0f, g.w, 2.0f), n)));
                    } else {
                        const float rho = __fdividef(__fmul_rn(2.0f, g.w), __fadd_rn(1.0f, g.w));
                        inc = log1pf(__fmul_rn(v.tau, __fsub_rn(rho, 1.0f)));
                    }
                    pl = pl + static_cast<double>(inc);
                    // Euler-Maruyama push in grid units
                    const float3 nz = box_muller(keys(make_uint4(step_n, 0u, pid, 0u)));
                    px = __fmaf_rn(v.noise, nz.x, __fmaf_rn(v.drift, g.x, px));
                    py = __fmaf_rn(v.noise, nz.y, __fmaf_rn(v.drift, g.y, py));
                    pz = __fmaf_rn(v.noise, nz.z, __fmaf_rn(v.drift, g.z, pz));
                    wrap3(px, py, pz, Hf, &bad);
                }
                const int nt = valid ? tile_at(px, py, pz, T) : -1;
                int dest = -1;
                if (binned) {
                    // the lanes that stay in the item's tile take consecutive slots
                    // reserved by one atomic; the few that leave it reserve their own
                    const bool stay = nt == tile;
                    const unsigned sm = __ballot_sync(kFull, stay);
                    int base = 0;
                    if (sm) {
                        // the lowest staying lane reserves for all of them
                        if (stay && !(sm & lanes_below())) base = atomicAdd(L.cnt + tile, __popc(sm));
                        base = __shfl_sync(kFull, base, __ffs(sm) - 1);
                    }
                    if (stay) {
                        const int slot = base + __popc(sm & lanes_below());
                        dest = slot < tslot[0] ? tslot[1] + slot : overflow_slot(L, status);
                    } else if (nt >= 0) {
                        const int slot = atomicAdd(L.cnt + nt, 1);
                        dest = slot < __ldg(L.cap + nt) ? __ldg(L.bstart + nt) + slot
                                                        : overflow_slot(L, status);
                    }
                } else {
                    // unbinned input or the overflow region: particles of one warp go to
                    // many tiles; the lanes bound for one tile share one atomic
                    const unsigned peers = __match_any_sync(kFull, nt);
                    int base = 0;
                    if (nt >= 0 && !(peers & lanes_below())) base = atomicAdd(L.cnt + nt, __popc(peers));
                    base = __shfl_sync(kFull, base, __ffs(peers) - 1);
                    if (nt >= 0) {
                        const int slot = base + __popc(peers & lanes_below());
                        dest = slot < __ldg(L.cap + nt) ? __ldg(L.bstart + nt) + slot
                                                        : overflow_slot(L, status);
                    }
                }
                if (dest >= 0) {
                    __stcs(dst.sx + dest, px);
                    __stcs(dst.sy + dest, py);
                    __stcs(dst.sz + dest, pz);
                    __stcs(dst.dl + dest, pl);
                    __stcs(dst.id + dest, pid);
                }
            }
        }
        if (bad & 1) atomicOr(status, kStatusNonfinite);
        if (bad & 2) atomicOr(status, kStatusSlot);
        if (do_deposit && binned) ++pending;
        __syncthreads();
    }
}

template <int ORDER, bool SKIP>
__global__ void __launch_bounds__(kNT, DepBlock<ORDER>::MIN_BLOCKS)
    k_step(PushArgs a, const StepScalars* __restrict__ sc, const float4* __restrict__ G, Buf src,
           Buf dst, Layout L, const Item* __restrict__ items, const int* __restrict__ n_items,
           unsigned long long* __restrict__ acc, int do_deposit, int do_move,
           int* __restrict__ status) {
    __shared__ StepShared<ORDER> sh;
    pdl_trigger();
    for (int i = threadIdx.x; i < DepBlock<ORDER>::N; i += kNT) {
        sh.dep[i] = 0;
        sh.dep64[i] = 0;
    }
    pdl_wait();   // the gather array of the spectral passes before
    // block b takes a contiguous run of items; consecutive items of one tile
    // share the node block of the gather array and the deposit sums, which
    // go to the grid accumulator once, when the tile changes
    const int total = *n_items;
    const int i_lo = static_cast<int>(static_cast<long long>(blockIdx.x) * total / gridDim.x);
    const int i_hi = static_cast<int>(static_cast<long long>(blockIdx.x + 1) * total / gridDim.x);
    const StepView v{a.H, a.drift, a.noise, a.tau, a.k0, a.k1, a.push, sc, G, src, dst, L,
                     items, acc, status, do_deposit, do_move};
    step_items<ORDER, SKIP>(v, KeysGiven{a.rk}, i_lo, i_hi, sh);
}

// ------------------------------------------------------------------ planning
// Block-wide exclusive scan (one value per thread) of kPlanNT threads.
constexpr int kPlanNT = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) smem[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < (blockDim.x >> 5)) ? smem[lane] : 0;
        int si = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(kFull, si, off);
            if (lane >= off) si += t;
        }
        smem[lane] = si - s;
        if (lane == 31) smem[32] = si;
    }
    __syncthreads();
    const int r = smem[warp] + incl - v;
    *total = smem[32];
    __syncthreads();
    return r;
}

// From the counts of buffer `b` (just written): the items that read it next
// (tile buckets split into kItem chunks, then the overflow region) with
// their offsets in the compacted particle order; and, when next_cnt is not
// null, the bucket layout of the other buffer for the next step (capacity
// count + count/slack_div + slack_add, rounded up to a multiple of 4; the
// context's buffers hold at least slack_div = 8, slack_add = 32) with its
// counters reset; with next_sc, the next step's scalars from those of this
// step.
__device__ __forceinline__ void plan_body(
    int ntiles, int T, const int* __restrict__ cnt, const int* __restrict__ cap,
    const int* __restrict__ bstart, const int* __restrict__ ovf, int ovf_base, Item* items,
    int* n_items, int* next_bstart, int* next_cap, int* next_cnt, int* next_ovf,
    int* __restrict__ status, const StepScalars* __restrict__ cur_sc,
    StepScalars* __restrict__ next_sc, double dt, double log2_maxrel, double exp_logref,
    double h3, int slack_div, int slack_add) {
    __shared__ int smem[33];
    const int per = (ntiles + kPlanNT - 1) / kPlanNT;
    const int t0 = threadIdx.x * per;
    int my_items = 0, my_fill = 0, my_cap = 0;
    for (int k = 0; k < per; ++k) {
        const int t = t0 + k;
        if (t >= ntiles) break;
        const int c = cnt[t];
        const int f = min(c, cap[t]);
        my_items += (f + kItem - 1) / kItem;
        my_fill += f;
        if (next_cnt) my_cap += ((c + c / slack_div + slack_add) + 3) & ~3;
    }
    int tot_items, tot_fill, tot_cap;
    int item0 = block_exclusive_scan(my_items, smem, &tot_items);
    int out0 = block_exclusive_scan(my_fill, smem, &tot_fill);
    int cap0 = next_cnt ? block_exclusive_scan(my_cap, smem, &tot_cap) : 0;
    for (int k = 0; k < per; ++k) {
        const int t = t0 + k;
        if (t >= ntiles) break;
        const int c = cnt[t];
        const int f = min(c, cap[t]);
        for (int q = 0; q * kItem < f; ++q) {
            Item it;
            it.tile = t;
            it.beg = bstart[t] + q * kItem;
            it.end = bstart[t] + min((q + 1) * kItem, f);
            it.out = out0 + q * kItem;
            it.tx = t % T;
            it.ty = (t / T) % T;
            it.tz = t / (T * T);
            it.pad = 0;
            items[item0++] = it;
        }
        out0 += f;
        if (next_cnt) {
            const int cp = ((c + c / slack_div + slack_add) + 3) & ~3;
            next_bstart[t] = cap0;
            next_cap[t] = cp;
            next_cnt[t] = 0;
            cap0 += cp;
        }
    }
    if (threadIdx.x == 0) {
        const int no = *ovf;
        int n = tot_items;
        for (int q = 0; q * kItem < no; ++q) {
            Item it;
            it.tile = -1;
            it.beg = ovf_base + q * kItem;
            it.end = ovf_base + min((q + 1) * kItem, no);
            it.out = tot_fill + q * kItem;
            it.tx = it.ty = it.tz = it.pad = 0;
            items[n++] = it;
        }
        *n_items = n;
        if (next_ovf) *next_ovf = 0;
        if (tot_fill + no < 0) atomicOr(status, kStatusTotal);
        // scalars of the next step: n + 1 at time t_n = t_{n-1} + dt
        if (next_sc)
            fill_step_scalars(next_sc, cur_sc->n + 1u, cur_sc->time + dt, log2_maxrel, exp_logref,
                              h3);
    }
}

__global__ void __launch_bounds__(kPlanNT)
    k_plan(int ntiles, int T, const int* __restrict__ cnt, const int* __restrict__ cap,
           const int* __restrict__ bstart, const int* __restrict__ ovf, int ovf_base, Item* items,
           int* n_items, int* next_bstart, int* next_cap, int* next_cnt, int* next_ovf,
           int* __restrict__ status, const StepScalars* __restrict__ cur_sc,
           StepScalars* __restrict__ next_sc, double dt, double log2_maxrel, double exp_logref,
           double h3, int slack_div, int slack_add) {
    plan_body(ntiles, T, cnt, cap, bstart, ovf, ovf_base, items, n_items, next_bstart, next_cap,
              next_cnt, next_ovf, status, cur_sc, next_sc, dt, log2_maxrel, exp_logref, h3,
              slack_div, slack_add);
}

// The plan of every run of an ensemble after a batched step from buffer
// `parity` (block r plans run r: items of the written buffer parity ^ 1,
// layout of buffer parity, scalars of the next step).
__global__ void __launch_bounds__(kPlanNT) k_plan_multi(const RunDesc* __restrict__ runs,
                                                        int parity) {
    const RunDesc& d = runs[blockIdx.x];
    const int b = parity ^ 1, o = parity;
    plan_body(d.ntiles, d.H / 8, d.cnt[b], d.cap[b], d.bstart[b], d.ovf[b], d.ovf_base, d.items,
              d.n_items, d.bstart[o], d.cap[o], d.cnt[o], d.ovf[o], d.status, d.dsc + o,
              d.dsc + b, d.dt, d.log2_maxrel, d.exp_logref, d.h3, d.slack_div, d.slack_add);
}

// One persistent launch over the items of all runs of an ensemble (all
// reading buffer `parity`): the runs' item lists are concatenated, each
// block takes a contiguous range and steps it run segment by run segment,
// with the segment's run read from the table into shared memory (its
// values are read from there where the single-run kernel has launch
// arguments).  Trilinear assignment only.
__global__ void __launch_bounds__(kNT, DepBlock<2>::MIN_BLOCKS)
    k_step_multi(const RunDesc* __restrict__ runs, int nruns, int parity) {
    __shared__ StepShared<2> sh;
    __shared__ int prefix[kMaxRuns + 1];
    __shared__ int scan_tmp[33];
    __shared__ StepView view;
    for (int i = threadIdx.x; i < DepBlock<2>::N; i += kNT) {
        sh.dep[i] = 0;
        sh.dep64[i] = 0;
    }
    const int cnt = threadIdx.x < nruns ? *runs[threadIdx.x].n_items : 0;
    int total;
    const int ex = block_exclusive_scan(cnt, scan_tmp, &total);
    if (threadIdx.x < nruns) prefix[threadIdx.x] = ex;
    if (threadIdx.x == 0) prefix[nruns] = total;
    __syncthreads();
    const int i_lo = static_cast<int>(static_cast<long long>(blockIdx.x) * total / gridDim.x);
    const int i_hi = static_cast<int>(static_cast<long long>(blockIdx.x + 1) * total / gridDim.x);
    const int b = parity, o = parity ^ 1;
    for (int r = 0; r < nruns; ++r) {
        const int lo = max(i_lo, prefix[r]) - prefix[r];
        const int hi = min(i_hi, prefix[r + 1]) - prefix[r];
        if (lo >= hi) continue;
        if (threadIdx.x == 0) {
            const RunDesc& d = runs[r];
            view = StepView{d.H, d.drift, d.noise, d.tau, d.k0, d.k1, 1, d.dsc + b,
                            reinterpret_cast<const float4*>(d.G),
                            Buf{d.sx[b], d.sy[b], d.sz[b], d.dl[b], d.id[b]},
                            Buf{d.sx[o], d.sy[o], d.sz[o], d.dl[o], d.id[o]},
                            Layout{d.bstart[o], d.cap[o], d.cnt[o], d.ovf[o], d.ovf_base, d.ovf_cap},
                            d.items, d.acc, d.status, 1, 1};
        }
        __syncthreads();
        step_items<2, true>(view, KeysScheduled{view}, lo, hi, sh);
        __syncthreads();
    }
}

// Particles per tile of an unbinned input array (positions already wrapped).
__global__ void k_tile_count(const float* __restrict__ sx, const float* __restrict__ sy,
                             const float* __restrict__ sz, int N, int H, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int t = -1;
    if (i < N) {
        const Cell c = locate_clamped(sx[i], sy[i], sz[i], H);
        t = tile_of(c.cx, c.cy, c.cz, H >> 3);
    }
    const unsigned peers = __match_any_sync(kFull, t);
    if (t >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + t, __popc(peers));
}

// Whole input as overflow-style items (tile -1) for the initial binning.
__global__ void k_plan_flat(int N, Item* items, int* n_items) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int nq = (N + kItem - 1) / kItem;
    if (q < nq) {
        Item it;
        it.tile = -1;
        it.beg = q * kItem;
        it.end = min((q + 1) * kItem, N);
        it.out = q * kItem;
        it.tx = it.ty = it.tz = it.pad = 0;
        items[q] = it;
    }
    if (q == 0) *n_items = nq;
}

// Compacted copy of the live particles (items in order) into `out`.
__global__ void k_compact(const Item* __restrict__ items, const int* __restrict__ n_items,
                          Buf src, Buf out) {
    const int q = blockIdx.x;
    if (q >= *n_items) return;
    const Item it = items[q];
    for (int i = it.beg + threadIdx.x; i < it.end; i += blockDim.x) {
        const int o = it.out + (i - it.beg);
        out.sx[o] = src.sx[i];
        out.sy[o] = src.sy[i];
        out.sz[o] = src.sz[i];
        out.dl[o] = src.dl[i];
        out.id[o] = src.id[i];
    }
}

// ------------------------------------------------------------------ per-cell histogram
__global__ void k_cell_count(const float* __restrict__ sx, const float* __restrict__ sy,
                             const float* __restrict__ sz, int N, int H, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t key = 0xffffffffu;
    if (i < N) {
        const Cell c = locate_clamped(sx[i], sy[i], sz[i], H);
        key = cell_key(c.cx, c.cy, c.cz, H >> 3);
    }
    const unsigned peers = __match_any_sync(kFull, key);
    if (i < N && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
}

constexpr int kScanNT = 1024;
constexpr int kScanIPT = 8;
constexpr int kScanTile = kScanNT * kScanIPT;

__global__ void __launch_bounds__(kScanNT) k_scan_tiles(const int* __restrict__ count, int n,
                                                        int* __restrict__ tile_sum) {
    __shared__ int smem[33];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanIPT;
    int s = 0;
    if (base < n) {
        const int4 a = *reinterpret_cast<const int4*>(count + base);
        const int4 b = *reinterpret_cast<const int4*>(count + base + 4);
        s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
    }
    int total;
    block_exclusive_scan(s, smem, &total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanNT) k_scan_tile_sums(int* __restrict__ tile_sum, int ntiles,
                                                            int* __restrict__ cell_start, int n) {
    __shared__ int smem[33];
    int carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += kScanNT) {
        const int j = b0 + threadIdx.x;
        const int v = j < ntiles ? tile_sum[j] : 0;
        int total;
        const int ex = block_exclusive_scan(v, smem, &total);
        if (j < ntiles) tile_sum[j] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) cell_start[n] = carry;
}

__global__ void __launch_bounds__(kScanNT) k_scan_apply(const int* __restrict__ count, int n,
                                                        const int* __restrict__ tile_off,
                                                        int* __restrict__ cell_start) {
    __shared__ int smem[33];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanIPT;
    int v[kScanIPT] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (base < n) {
        const int4 a = *reinterpret_cast<const int4*>(count + base);
        const int4 b = *reinterpret_cast<const int4*>(count + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) s += v[k];
    int total;
    int run = block_exclusive_scan(s, smem, &total) + tile_off[blockIdx.x];
    if (base < n) {
        int o[kScanIPT];
#pragma unroll
        for (int k = 0; k < kScanIPT; ++k) {
            o[k] = run;
            run += v[k];
        }
        *reinterpret_cast<int4*>(cell_start + base) = make_int4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<int4*>(cell_start + base + 4) = make_int4(o[4], o[5], o[6], o[7]);
    }
}

// ------------------------------------------------------------------ canonical order
// The particles of a buffer sorted by (cell key, id): a counting sort by key
// (slots of a cell's run taken in arrival order), then each particle's rank
// among the ids of its run, which places it at its canonical position.  Ties
// in id (possible only for caller-given duplicate ids) are broken by slot,
// so the result is always a permutation.
__global__ void k_canon_scatter(const float* __restrict__ sx, const float* __restrict__ sy,
                                const float* __restrict__ sz, const uint32_t* __restrict__ id,
                                int N, int H, const int* __restrict__ cell_start,
                                int* __restrict__ fill, uint32_t* __restrict__ keys_tmp,
                                uint32_t* __restrict__ ids_tmp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Cell c = locate_clamped(sx[i], sy[i], sz[i], H);
    const uint32_t key = cell_key(c.cx, c.cy, c.cz, H >> 3);
    const int slot = cell_start[key] + atomicAdd(fill + key, 1);
    keys_tmp[slot] = key;
    ids_tmp[slot] = id[i];
}

__global__ void k_canon_rank(const uint32_t* __restrict__ keys_tmp,
                             const uint32_t* __restrict__ ids_tmp, int N,
                             const int* __restrict__ cell_start, uint32_t* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const uint32_t key = keys_tmp[j];
    const int b = cell_start[key], e = cell_start[key + 1];
    const uint32_t me = ids_tmp[j];
    int rank = 0;
    for (int t = b; t < e; ++t) {
        const uint32_t o = ids_tmp[t];
        rank += (o < me) || (o == me && t < j);
    }
    out[b + rank] = me;
}

// ------------------------------------------------------------------ misc
// Physical coordinates (three arrays) -> grid units wrapped into [0, H).
__global__ void k_wrap_positions(const float* __restrict__ x, const float* __restrict__ y,
                                 const float* __restrict__ z, int N, float o0, float o1, float o2,
                                 float h, int H, float* sx, float* sy, float* sz,
                                 int* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float Hf = __int2float_rn(H);
    int bad = 0;
    sx[i] = wrap(__fdiv_rn(__fsub_rn(x[i], o0), h), Hf, &bad);
    sy[i] = wrap(__fdiv_rn(__fsub_rn(y[i], o1), h), Hf, &bad);
    sz[i] = wrap(__fdiv_rn(__fsub_rn(z[i], o2), h), Hf, &bad);
    if (bad) atomicOr(status, kStatusNonfinite);
}

__global__ void k_rel_log_mass(const double* __restrict__ mass, int N, double logref, double* dl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dl[i] = log(mass[i]) - logref;
}

__global__ void k_iota(uint32_t* id, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) id[i] = static_cast<uint32_t>(i);
}

// Grid units -> physical coordinates, in place (each array on its own).
__global__ void k_export_inplace(float* __restrict__ s, int N, float o, float h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) s[i] = __fmaf_rn(s[i], h, o);
}

__global__ void k_export_mass(const double* __restrict__ dl, int N, double logref, double* out,
                              int as_log) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = as_log ? dl[i] + logref : exp(dl[i] + logref);
}

// u_bar = acc * scale; the accumulator is cleared for the next deposit.
__global__ void k_acc_to_float(unsigned long long* __restrict__ acc, int n, float scale,
                               float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long q = acc[i];
    acc[i] = 0ull;
    // two's complement: signed high half, unsigned low half
    const float f = fmaf(__int2float_rn(static_cast<int>(static_cast<unsigned>(q >> 32))),
                         4294967296.0f, __uint2float_rn(static_cast<unsigned>(q)));
    out[i] = f * scale;
}

// One component of the interleaved (dv/dx, dv/dy, dv/dz, w) array.
__global__ void k_component(const float4* __restrict__ G, int n, int comp, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 g = G[i];
    out[i] = comp == 0 ? g.x : comp == 1 ? g.y : g.z;
}

// Diagnostics: deterministic two-level reduction (fixed grid, fixed trees).
// The particle mass is summed exactly, as 128-bit fixed point: each
// a_p / exp(logref) times 2^K (K chosen on the host so that a term stays
// below 2^62) rounded to an integer, so the total does not depend on the
// order in which the particles are stored.
constexpr int kDiagBlocks = 304;
constexpr int kDiagNT = 256;

__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }

__global__ void __launch_bounds__(kDiagNT)
    k_diag_partials(const double* __restrict__ dl, double logref, const float* __restrict__ sx,
                    const float* __restrict__ sy, const float* __restrict__ sz, int N,
                    const float* __restrict__ v, const float* __restrict__ m,
                    const float* __restrict__ w, const unsigned long long* __restrict__ acc,
                    int ncell, int K, double* __restrict__ part_d, long long* __restrict__ part_l) {
    double mv = INFINITY, mm = INFINITY, mw = INFINITY, nf = 0.0;
    unsigned __int128 mass = 0;
    long long as = 0, amin = LLONG_MAX;
    const int stride = kDiagBlocks * kDiagNT;
    for (int i = blockIdx.x * kDiagNT + threadIdx.x; i < N; i += stride) {
        mass += __double2ull_rn(scalbn(exp(dl[i]), K));
        if (!isfinite(sx[i]) || !isfinite(sy[i]) || !isfinite(sz[i])) nf += 1.0;
    }
    for (int i = blockIdx.x * kDiagNT + threadIdx.x; i < ncell; i += stride) {
        const float a = v[i], b = m[i], c = w[i];
        mv = dmin(mv, a);
        mm = dmin(mm, b);
        mw = dmin(mw, c);
        nf += (!isfinite(a)) + (!isfinite(b)) + (!isfinite(c));
        const long long q = static_cast<long long>(acc[i]);
        as += q;
        amin = q < amin ? q : amin;
    }
    __shared__ double sd[5][kDiagNT];
    __shared__ long long sl[2][kDiagNT];
    __shared__ unsigned __int128 sq[kDiagNT];
    sq[threadIdx.x] = mass;
    sd[0][threadIdx.x] = 0.0;
    sd[1][threadIdx.x] = mv;
    sd[2][threadIdx.x] = mm;
    sd[3][threadIdx.x] = mw;
    sd[4][threadIdx.x] = nf;
    sl[0][threadIdx.x] = as;
    sl[1][threadIdx.x] = amin;
    __syncthreads();
    for (int s = kDiagNT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int j = threadIdx.x + s;
            sq[threadIdx.x] += sq[j];
            sd[1][threadIdx.x] = dmin(sd[1][threadIdx.x], sd[1][j]);
            sd[2][threadIdx.x] = dmin(sd[2][threadIdx.x], sd[2][j]);
            sd[3][threadIdx.x] = dmin(sd[3][threadIdx.x], sd[3][j]);
            sd[4][threadIdx.x] += sd[4][j];
            sl[0][threadIdx.x] += sl[0][j];
            sl[1][threadIdx.x] = sl[1][j] < sl[1][threadIdx.x] ? sl[1][j] : sl[1][threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) part_d[blockIdx.x * 5 + k] = sd[k][0];
        part_l[blockIdx.x * 4] = sl[0][0];
        part_l[blockIdx.x * 4 + 1] = sl[1][0];
        part_l[blockIdx.x * 4 + 2] = static_cast<long long>(static_cast<uint64_t>(sq[0]));
        part_l[blockIdx.x * 4 + 3] = static_cast<long long>(static_cast<uint64_t>(sq[0] >> 64));
    }
}

// One block: each thread folds a strided share of the partials, then a
// shared-memory tree.  Every quantity is exact (integer sums, 128-bit mass
// sum, minima, counts held exactly in doubles), so the result does not
// depend on the order of the combination.
constexpr int kDiagFinalNT = 256;

__global__ void __launch_bounds__(kDiagFinalNT)
    k_diag_final(const double* __restrict__ part_d, const long long* __restrict__ part_l,
                 double acc_to_u, int K, double logref, double* __restrict__ out) {
    double mv = INFINITY, mm = INFINITY, mw = INFINITY, nf = 0;
    unsigned __int128 mass = 0;
    long long as = 0, amin = LLONG_MAX;
    for (int b = threadIdx.x; b < kDiagBlocks; b += kDiagFinalNT) {
        mv = dmin(mv, part_d[b * 5 + 1]);
        mm = dmin(mm, part_d[b * 5 + 2]);
        mw = dmin(mw, part_d[b * 5 + 3]);
        nf += part_d[b * 5 + 4];
        as += part_l[b * 4];
        amin = part_l[b * 4 + 1] < amin ? part_l[b * 4 + 1] : amin;
        mass += (static_cast<unsigned __int128>(static_cast<uint64_t>(part_l[b * 4 + 3])) << 64) |
                static_cast<uint64_t>(part_l[b * 4 + 2]);
    }
    __shared__ double sd[4][kDiagFinalNT];
    __shared__ long long sl[2][kDiagFinalNT];
    __shared__ unsigned __int128 sq[kDiagFinalNT];
    const int t = threadIdx.x;
    sd[0][t] = mv;
    sd[1][t] = mm;
    sd[2][t] = mw;
    sd[3][t] = nf;
    sl[0][t] = as;
    sl[1][t] = amin;
    sq[t] = mass;
    __syncthreads();
    for (int s = kDiagFinalNT / 2; s > 0; s >>= 1) {
        if (t < s) {
            sd[0][t] = dmin(sd[0][t], sd[0][t + s]);
            sd[1][t] = dmin(sd[1][t], sd[1][t + s]);
            sd[2][t] = dmin(sd[2][t], sd[2][t + s]);
            sd[3][t] += sd[3][t + s];
            sl[0][t] += sl[0][t + s];
            sl[1][t] = sl[1][t + s] < sl[1][t] ? sl[1][t + s] : sl[1][t];
            sq[t] += sq[t + s];
        }
        __syncthreads();
    }
    if (t != 0) return;
    const unsigned __int128 total = sq[0];
    const double mass_d = static_cast<double>(static_cast<uint64_t>(total >> 64)) * 18446744073709551616.0 +
                          static_cast<double>(static_cast<uint64_t>(total));
    out[0] = scalbn(mass_d, -K) * exp(logref);
    out[1] = static_cast<double>(sl[0][0]) * acc_to_u;   // sum of u_bar (times h^3 on the host)
    out[2] = static_cast<double>(sl[1][0]) * acc_to_u;
    out[3] = sd[0][0];
    out[4] = sd[1][0];
    out[5] = sd[2][0];
    out[6] = sd[3][0];
}

__global__ void k_normals(const uint32_t* __restrict__ ids, int64_t N, uint32_t n, uint32_t k0,
                          uint32_t k1, float* __restrict__ z, uint32_t* __restrict__ bits) {
    // 64-bit offsets: 4 N exceeds the int range for N above 2^29
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint4 raw;
    const float3 r = brownian(ids[i], n, k0, k1, &raw);
    z[i] = r.x;
    z[N + i] = r.y;
    z[2 * N + i] = r.z;
    if (bits) {
        bits[i] = raw.x;
        bits[N + i] = raw.y;
        bits[2 * N + i] = raw.z;
        bits[3 * N + i] = raw.w;
    }
}

inline int blocks_for(int64_t n, int nt) { return static_cast<int>((n + nt - 1) / nt); }

inline Buf buf_of(sipf_ctx* c, int b) {
    return Buf{c->sx[b], c->sy[b], c->sz[b], c->dl[b], c->id[b]};
}

inline Layout layout_of(sipf_ctx* c, int b) {
    return Layout{c->bstart[b], c->cap[b], c->cnt[b], c->ovf[b], c->ovf_base,
                  static_cast<int>(c->N)};
}

}  // namespace

// ---------------------------------------------------------------- launchers
int step_grid(sipf_ctx* c) {
    int dev = c->device, nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (c->p.p2g_order == 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<4, false>, kNT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<2, false>, kNT, 0);
    // a tuning may ask for fewer blocks per SM than the occupancy limit
    if (c->step_bps > 0 && c->step_bps < per_sm) per_sm = c->step_bps;
    int g = nsm * (per_sm > 0 ? per_sm : 1);
    // no more blocks than items can exist: a small run leaves the rest of the
    // GPU to the runs beside it
    if (g > c->max_items) g = c->max_items;
    return g > 0 ? g : 1;
}

cudaError_t launch_step_kernel(sipf_ctx* c, const PushArgs& a, int do_deposit, int do_move) {
    const int b = c->cur;
    // runs with fewer than kSparsePerTile particles per tile on average have
    // many short items: they take the form that skips idle warps
    const bool sparse = c->N < static_cast<int64_t>(kSparsePerTile) * c->ntiles;
    auto kernel = c->p.p2g_order == 4 ? (sparse ? k_step<4, true> : k_step<4, false>)
                                      : (sparse ? k_step<2, true> : k_step<2, false>);
    return launch_pdl(kernel, dim3(c->step_blocks), dim3(kNT), 0, c->stream, a,
                      static_cast<const StepScalars*>(c->dsc + b),
                      static_cast<const float4*>(reinterpret_cast<float4*>(c->G)), buf_of(c, b),
                      buf_of(c, b ^ 1), layout_of(c, b ^ 1), static_cast<const Item*>(c->items),
                      static_cast<const int*>(c->n_items),
                      reinterpret_cast<unsigned long long*>(c->acc), do_deposit, do_move,
                      c->status);
}

// Items of buffer `b` and, with next_layout, the layout of b ^ 1.
cudaError_t launch_plan(sipf_ctx* c, int b, int next_layout, cudaStream_t s, double dt) {
    const int o = b ^ 1;
    k_plan<<<1, kPlanNT, 0, s>>>(
        c->ntiles, c->H / 8, c->cnt[b], c->cap[b], c->bstart[b], c->ovf[b], c->ovf_base, c->items,
        c->n_items, next_layout ? c->bstart[o] : nullptr,
        next_layout ? c->cap[o] : nullptr, next_layout ? c->cnt[o] : nullptr,
        next_layout ? c->ovf[o] : nullptr, c->status,
        // b is the buffer the step just wrote: its slot is the next step's, o's the current one
        c->dsc + o, dt > 0.0 ? c->dsc + b : nullptr, dt, c->log2_maxrel, c->exp_logref, c->h3,
        c->slack_div, c->slack_add);
    return cudaGetLastError();
}

cudaError_t launch_step_multi(const RunDesc* runs, int n, int parity, cudaStream_t s) {
    if (n < 1 || n > kMaxRuns) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_multi, kNT, 0);
    k_step_multi<<<nsm * (per_sm > 0 ? per_sm : 1), kNT, 0, s>>>(runs, n, parity);
    return cudaGetLastError();
}

cudaError_t launch_plan_multi(const RunDesc* runs, int n, int parity, cudaStream_t s) {
    if (n < 1) return cudaErrorInvalidValue;
    k_plan_multi<<<n, kPlanNT, 0, s>>>(runs, parity);
    return cudaGetLastError();
}

RunDesc run_desc(const sipf_ctx* c, double dt) {
    RunDesc d{};
    d.H = c->H;
    d.ntiles = c->ntiles;
    d.ovf_base = c->ovf_base;
    d.ovf_cap = static_cast<int>(c->N);
    d.drift = static_cast<float>(c->p.chi * dt / c->h);
    d.noise = static_cast<float>(sqrt(2.0 * c->p.Du * dt) / c->h);
    d.tau = static_cast<float>(dt);
    d.k0 = static_cast<uint32_t>(c->p.seed);
    d.k1 = static_cast<uint32_t>(c->p.seed >> 32);
    for (int b = 0; b < 2; ++b) {
        d.sx[b] = c->sx[b];
        d.sy[b] = c->sy[b];
        d.sz[b] = c->sz[b];
        d.dl[b] = c->dl[b];
        d.id[b] = c->id[b];
        d.bstart[b] = c->bstart[b];
        d.cap[b] = c->cap[b];
        d.cnt[b] = c->cnt[b];
        d.ovf[b] = c->ovf[b];
    }
    d.items = c->items;
    d.n_items = c->n_items;
    d.acc = reinterpret_cast<unsigned long long*>(c->acc);
    d.G = c->G;
    d.status = c->status;
    d.dsc = c->dsc;
    d.dt = dt;
    d.log2_maxrel = c->log2_maxrel;
    d.exp_logref = c->exp_logref;
    d.h3 = c->h3;
    d.slack_div = c->slack_div;
    d.slack_add = c->slack_add;
    return d;
}

cudaError_t launch_tile_count(sipf_ctx* c, int b, int* cnt) {
    const int N = static_cast<int>(c->N);
    k_tile_count<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->sx[b], c->sy[b], c->sz[b], N, c->H,
                                                             cnt);
    return cudaGetLastError();
}

cudaError_t launch_plan_flat(sipf_ctx* c) {
    const int nq = (static_cast<int>(c->N) + kItem - 1) / kItem;
    k_plan_flat<<<blocks_for(nq, 256), 256, 0, c->stream>>>(static_cast<int>(c->N), c->items,
                                                             c->n_items);
    return cudaGetLastError();
}

cudaError_t launch_compact(sipf_ctx* c, int b, int out) {
    k_compact<<<c->max_items, 256, 0, c->stream>>>(c->items, c->n_items, buf_of(c, b),
                                                   buf_of(c, out));
    return cudaGetLastError();
}

cudaError_t launch_cell_histogram(sipf_ctx* c, int b, int* count, int* tmp, int* cell_start) {
    const int N = static_cast<int>(c->N);
    const int n = c->H * c->H * c->H;
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync(count, 0, static_cast<size_t>(n) * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    k_cell_count<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->sx[b], c->sy[b], c->sz[b], N, c->H,
                                                             count);
    k_scan_tiles<<<ntiles, kScanNT, 0, c->stream>>>(count, n, tmp);
    k_scan_tile_sums<<<1, kScanNT, 0, c->stream>>>(tmp, ntiles, cell_start, n);
    k_scan_apply<<<ntiles, kScanNT, 0, c->stream>>>(count, n, tmp, cell_start);
    return cudaGetLastError();
}

cudaError_t launch_canonical_order(sipf_ctx* c, int b) {
    const int N = static_cast<int>(c->N);
    const int n = c->H * c->H * c->H;
    cudaError_t e = launch_cell_histogram(c, b, c->count, c->scan_tmp, c->cell_start);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->count, 0, static_cast<size_t>(n) * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    // the buffer's log-mass array (8 N bytes) holds the keys and ids of the
    // counting sort; the ranked ids go to the buffer's id array
    uint32_t* keys_tmp = reinterpret_cast<uint32_t*>(c->dl[b]);
    uint32_t* ids_tmp = keys_tmp + N;
    k_canon_scatter<<<blocks_for(N, 256), 256, 0, c->stream>>>(
        c->sx[b], c->sy[b], c->sz[b], c->id[b], N, c->H, c->cell_start, c->count, keys_tmp,
        ids_tmp);
    k_canon_rank<<<blocks_for(N, 256), 256, 0, c->stream>>>(keys_tmp, ids_tmp, N, c->cell_start,
                                                            c->id[b]);
    return cudaGetLastError();
}

cudaError_t launch_wrap_positions(sipf_ctx* c, const float* x, const float* y, const float* z,
                                  int buf) {
    const int N = static_cast<int>(c->N);
    k_wrap_positions<<<blocks_for(N, 256), 256, 0, c->stream>>>(
        x, y, z, N, static_cast<float>(c->origin[0]), static_cast<float>(c->origin[1]),
        static_cast<float>(c->origin[2]), static_cast<float>(c->h), c->H, c->sx[buf], c->sy[buf],
        c->sz[buf], c->status);
    return cudaGetLastError();
}

cudaError_t launch_rel_log_mass(sipf_ctx* c, const double* mass, int buf) {
    const int N = static_cast<int>(c->N);
    k_rel_log_mass<<<blocks_for(N, 256), 256, 0, c->stream>>>(mass, N, c->logref, c->dl[buf]);
    return cudaGetLastError();
}

cudaError_t launch_iota(sipf_ctx* c, int buf) {
    const int N = static_cast<int>(c->N);
    k_iota<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->id[buf], N);
    return cudaGetLastError();
}

cudaError_t launch_export_positions_inplace(sipf_ctx* c, int b) {
    const int N = static_cast<int>(c->N);
    float* arr[3] = {c->sx[b], c->sy[b], c->sz[b]};
    for (int d = 0; d < 3; ++d)
        k_export_inplace<<<blocks_for(N, 256), 256, 0, c->stream>>>(
            arr[d], N, static_cast<float>(c->origin[d]), static_cast<float>(c->h));
    return cudaGetLastError();
}

cudaError_t launch_export_mass(sipf_ctx* c, int b, double* out, int as_log) {
    const int N = static_cast<int>(c->N);
    k_export_mass<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->dl[b], N, c->logref, out, as_log);
    return cudaGetLastError();
}

cudaError_t launch_acc_to_float(sipf_ctx* c, float* dst, float scale) {
    const int n = c->H * c->H * c->H;
    k_acc_to_float<<<blocks_for(n, 256), 256, 0, c->stream>>>(
        reinterpret_cast<unsigned long long*>(c->acc), n, scale, dst);
    return cudaGetLastError();
}

cudaError_t launch_component(sipf_ctx* c, int comp, float* dst) {
    const int n = c->H * c->H * c->H;
    k_component<<<blocks_for(n, 256), 256, 0, c->stream>>>(reinterpret_cast<const float4*>(c->G), n,
                                                            comp, dst);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(sipf_ctx* c, int b, double acc_to_u) {
    // a_p / exp(logref) <= maxrel e^time (growth factor of a step < e^tau)
    const double bound = log2(c->maxrel) + c->time * 1.4426950408889634 + 1.0;
    int K = 61 - static_cast<int>(ceil(bound));
    K = K < -900 ? -900 : (K > 900 ? 900 : K);
    k_diag_partials<<<kDiagBlocks, kDiagNT, 0, c->stream>>>(
        c->dl[b], c->logref, c->sx[b], c->sy[b], c->sz[b], static_cast<int>(c->N), c->v, c->m,
        c->w, reinterpret_cast<const unsigned long long*>(c->acc), c->H * c->H * c->H, K,
        c->diag_tmp, c->diag_ll);
    k_diag_final<<<1, kDiagFinalNT, 0, c->stream>>>(c->diag_tmp, c->diag_ll, acc_to_u, K, c->logref,
                                          c->diag_out);
    return cudaGetLastError();
}

cudaError_t launch_normals(const uint32_t* ids, int64_t N, uint32_t n, uint64_t seed, float* z,
                           uint32_t* bits, cudaStream_t s) {
    k_normals<<<blocks_for(N, 256), 256, 0, s>>>(ids, N, n,
                                                 static_cast<uint32_t>(seed),
                                                 static_cast<uint32_t>(seed >> 32), z, bits);
    return cudaGetLastError();
}

size_t diag_scratch_doubles() { return static_cast<size_t>(kDiagBlocks) * 5; }
size_t diag_scratch_ll() { return static_cast<size_t>(kDiagBlocks) * 4; }
int scan_tiles(int n) { return (n + kScanTile - 1) / kScanTile; }
int item_size() { return kItem; }

}  // namespace sipf
