// Particle side of the SIPF-W step on sm_103a: Philox noise, the
// Euler-Maruyama push with trilinear gather (paper Eq. u_hat_update, Alg. 2,
// Eq. g2ph), the per-step counting sort of particles by cell, the
// particle-to-grid deposit (Alg. 1) and FP64 diagnostics.
//
// Storage: structure of arrays, positions in grid units s = (x - x_min)/h
// (float32), log-masses (float64), persistent ids (uint32).  The store is
// bucketed by cell key; each step is two passes over it:
//   count   : recompute X^n from X^(n-1) and count particles per new cell;
//   scatter : recompute X^n (bit-identical: same device function, explicit
//             rounding intrinsics), update the log-mass, deposit u_bar^(n-1)
//             from X^(n-1), and write each particle into its new cell's run.
// Deposit values are summed as 64-bit fixed-point integers (a float32
// contribution times 2^S, exact for all but sub-2^-S parts), so the grid
// density does not depend on the order of particles within a cell and is
// bit-reproducible without float atomics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sipf_internal.cuh"

namespace sipf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNT = 256;

// ------------------------------------------------------------------ Philox
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with key mixing; the key advances by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// (2 (b >> 9) + 1) 2^-24: exact in float32, in (0, 1).
__device__ __forceinline__ float unit_open(uint32_t b) {
    return __uint2float_rn(((b >> 9) << 1) | 1u) * 5.9604644775390625e-8f;
}

// Three standard normals of particle `id` in step n: Box-Muller on the four
// Philox words of counter (n, 0, id, 0).
__device__ __forceinline__ float3 brownian(uint32_t id, uint32_t n, uint32_t k0, uint32_t k1,
                                           uint4* raw = nullptr) {
    const uint4 b = philox4x32_10(make_uint4(n, 0u, id, 0u), k0, k1);
    if (raw) *raw = b;
    const float u0 = unit_open(b.x), u1 = unit_open(b.y);
    const float u2 = unit_open(b.z), u3 = unit_open(b.w);
    const float r01 = sqrtf(-2.0f * logf(u0));
    const float r23 = sqrtf(-2.0f * logf(u2));
    float s1, c1;
    sincospif(2.0f * u1, &s1, &c1);
    const float c3 = cospif(2.0f * u3);
    return make_float3(r01 * c1, r01 * s1, r23 * c3);
}

// ------------------------------------------------------------------ cells
struct Cell {
    int base;            // flat node index of the cell's lower corner (z*H + y)*H + x
    int dx, dy, dz;      // offsets to the +1 neighbours (periodic)
    float fx, fy, fz;    // fractional position in the cell
    uint32_t key;        // tile-major cell key
};

__device__ __forceinline__ Cell locate(float x, float y, float z, int H) {
    Cell c;
    int cx = min(static_cast<int>(x), H - 1);
    int cy = min(static_cast<int>(y), H - 1);
    int cz = min(static_cast<int>(z), H - 1);
    c.fx = __fsub_rn(x, __int2float_rn(cx));
    c.fy = __fsub_rn(y, __int2float_rn(cy));
    c.fz = __fsub_rn(z, __int2float_rn(cz));
    c.base = (cz * H + cy) * H + cx;
    c.dx = (cx + 1 < H) ? 1 : 1 - H;
    c.dy = (cy + 1 < H) ? H : H - H * H;
    c.dz = (cz + 1 < H) ? H * H : H * H - H * H * H;
    const int T = H >> 3;
    const uint32_t tile = ((cz >> 3) * T + (cy >> 3)) * T + (cx >> 3);
    c.key = (tile << 9) | ((cz & 7) << 6) | ((cy & 7) << 3) | (cx & 7);
    return c;
}

__device__ __forceinline__ uint32_t key_of(float x, float y, float z, int H) {
    return locate(x, y, z, H).key;
}

// Trilinear interpolation (K_h = h^3 R_h, Alg. 2) with a fixed evaluation
// order: along x, then y, then z.
__device__ __forceinline__ float interp(const float* __restrict__ f, const Cell& c, float wx0,
                                        float wy0, float wz0) {
    const int i = c.base;
    const float f000 = __ldg(f + i), f100 = __ldg(f + i + c.dx);
    const float f010 = __ldg(f + i + c.dy), f110 = __ldg(f + i + c.dy + c.dx);
    const float f001 = __ldg(f + i + c.dz), f101 = __ldg(f + i + c.dz + c.dx);
    const float f011 = __ldg(f + i + c.dz + c.dy), f111 = __ldg(f + i + c.dz + c.dy + c.dx);
    const float c00 = __fmaf_rn(c.fx, f100, __fmul_rn(wx0, f000));
    const float c10 = __fmaf_rn(c.fx, f110, __fmul_rn(wx0, f010));
    const float c01 = __fmaf_rn(c.fx, f101, __fmul_rn(wx0, f001));
    const float c11 = __fmaf_rn(c.fx, f111, __fmul_rn(wx0, f011));
    const float c0 = __fmaf_rn(c.fy, c10, __fmul_rn(wy0, c00));
    const float c1 = __fmaf_rn(c.fy, c11, __fmul_rn(wy0, c01));
    return __fmaf_rn(c.fz, c1, __fmul_rn(wz0, c0));
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

struct Fields {
    const float* gx;
    const float* gy;
    const float* gz;
    const float* w;
};

// Euler-Maruyama push (Eq. u_hat_update) in grid units:
// s <- s + (chi tau / h) grad v_H + (sqrt(2 Du tau) / h) z, then wrap.
__device__ __forceinline__ void push(const PushArgs& a, const Fields& F, const Cell& c,
                                     uint32_t id, float& x, float& y, float& z, int* bad) {
    const float wx0 = __fsub_rn(1.0f, c.fx), wy0 = __fsub_rn(1.0f, c.fy),
                wz0 = __fsub_rn(1.0f, c.fz);
    const float g0 = interp(F.gx, c, wx0, wy0, wz0);
    const float g1 = interp(F.gy, c, wx0, wy0, wz0);
    const float g2 = interp(F.gz, c, wx0, wy0, wz0);
    const float3 nz = brownian(id, a.n, a.k0, a.k1);
    const float Hf = __int2float_rn(a.H);
    x = wrap(__fmaf_rn(a.noise, nz.x, __fmaf_rn(a.drift, g0, x)), Hf, bad);
    y = wrap(__fmaf_rn(a.noise, nz.y, __fmaf_rn(a.drift, g1, y)), Hf, bad);
    z = wrap(__fmaf_rn(a.noise, nz.z, __fmaf_rn(a.drift, g2, z)), Hf, bad);
}

// ------------------------------------------------------------------ kernels

// Pass 1: count particles per cell of X^n (or of X^(n-1) when a.push == 0).
__global__ void __launch_bounds__(kNT) k_count(PushArgs a, Fields F, const float* __restrict__ sx,
                                               const float* __restrict__ sy,
                                               const float* __restrict__ sz,
                                               const uint32_t* __restrict__ ids, int N,
                                               int* __restrict__ count) {
    const int i = blockIdx.x * kNT + threadIdx.x;
    const bool valid = i < N;
    uint32_t key = 0xffffffffu;
    if (valid) {
        float x = sx[i], y = sy[i], z = sz[i];
        if (a.push) {
            int bad = 0;
            const Cell c = locate(x, y, z, a.H);
            push(a, F, c, ids[i], x, y, z, &bad);
        }
        key = key_of(x, y, z, a.H);
    }
    const unsigned peers = __match_any_sync(kFull, key);
    const int lane = threadIdx.x & 31;
    if (valid && lane == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
}

struct Store {
    float* sx;
    float* sy;
    float* sz;
    double* loga;
    uint32_t* id;
};

// Pass 2: deposit u_bar^(n-1) (Alg. 1) from X^(n-1), then push, update the
// log-mass and write the particle into its new cell's run.
__global__ void __launch_bounds__(kNT)
    k_scatter(PushArgs a, DepositArgs d, Fields F, Store src, Store dst, int N, int do_deposit,
              int do_scatter, int* __restrict__ count, const int* __restrict__ cell_start,
              unsigned long long* __restrict__ acc, int* __restrict__ status) {
    const int i = blockIdx.x * kNT + threadIdx.x;
    const bool valid = i < N;
    const int lane = threadIdx.x & 31;
    float x = 0.f, y = 0.f, z = 0.f;
    double la = 0.0;
    uint32_t id = 0;
    Cell c{};
    if (valid) {
        x = src.sx[i];
        y = src.sy[i];
        z = src.sz[i];
        la = src.loga[i];
        id = src.id[i];
        c = locate(x, y, z, a.H);
    }
    const float wx0 = __fsub_rn(1.0f, c.fx), wy0 = __fsub_rn(1.0f, c.fy),
                wz0 = __fsub_rn(1.0f, c.fz);

    if (do_deposit) {
        // a_p * R_h(X_p, node) * h^3 in units of exp(logref) 2^-S.
        long long q[8];
        {
            const float ea = valid ? __fmul_rn(expf(static_cast<float>(la - d.logref)), d.scale)
                                   : 0.0f;
            const float e0 = __fmul_rn(ea, wz0), e1 = __fmul_rn(ea, c.fz);
            const float xy00 = __fmul_rn(wx0, wy0), xy10 = __fmul_rn(c.fx, wy0);
            const float xy01 = __fmul_rn(wx0, c.fy), xy11 = __fmul_rn(c.fx, c.fy);
            q[0] = __float2ll_rn(__fmul_rn(e0, xy00));
            q[1] = __float2ll_rn(__fmul_rn(e0, xy10));
            q[2] = __float2ll_rn(__fmul_rn(e0, xy01));
            q[3] = __float2ll_rn(__fmul_rn(e0, xy11));
            q[4] = __float2ll_rn(__fmul_rn(e1, xy00));
            q[5] = __float2ll_rn(__fmul_rn(e1, xy10));
            q[6] = __float2ll_rn(__fmul_rn(e1, xy01));
            q[7] = __float2ll_rn(__fmul_rn(e1, xy11));
        }
        const uint32_t key0 = __shfl_sync(kFull, c.key, 0);
        const bool uniform = __all_sync(kFull, valid && c.key == key0);
        const int node[8] = {c.base,
                             c.base + c.dx,
                             c.base + c.dy,
                             c.base + c.dy + c.dx,
                             c.base + c.dz,
                             c.base + c.dz + c.dx,
                             c.base + c.dz + c.dy,
                             c.base + c.dz + c.dy + c.dx};
        if (uniform) {
            // whole warp in one cell: integer butterfly sum, one atomic per corner
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int j = 0; j < 8; ++j) q[j] += __shfl_xor_sync(kFull, q[j], off);
            }
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    atomicAdd(acc + node[j], static_cast<unsigned long long>(q[j]));
            }
        } else if (valid) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (q[j]) atomicAdd(acc + node[j], static_cast<unsigned long long>(q[j]));
        }
    }

    if (!do_scatter) return;
    int bad = 0;
    if (valid && a.push) {
        // mass factor 1 + tau (rho(w_H) - 1), rho(w) = 2w/(1+w) (Eq. u_hat_update)
        const float wH = interp(F.w, c, wx0, wy0, wz0);
        const float rho = __fdiv_rn(2.0f * wH, __fadd_rn(1.0f, wH));
        const float inc = log1pf(__fmul_rn(a.tau, __fsub_rn(rho, 1.0f)));
        la += static_cast<double>(inc);
        push(a, F, c, id, x, y, z, &bad);
    }
    const uint32_t key = valid ? key_of(x, y, z, a.H) : 0xffffffffu;
    const unsigned peers = __match_any_sync(kFull, key);
    const int leader = __ffs(peers) - 1;
    int old = 0;
    if (valid && lane == leader) old = atomicSub(count + key, __popc(peers));
    old = __shfl_sync(kFull, old, leader);
    if (!valid) return;
    if (bad) atomicOr(status, kStatusNonfinite);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int slot = old - 1 - rank;
    const int start = cell_start[key], end = cell_start[key + 1];
    const int dest = start + slot;
    if (slot < 0 || dest >= end) {
        atomicOr(status, kStatusSlot);
        return;
    }
    dst.sx[dest] = x;
    dst.sy[dest] = y;
    dst.sz[dest] = z;
    dst.loga[dest] = la;
    dst.id[dest] = id;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of the per-cell counts in three phases with fixed
// tiles (no inter-block waits): tile sums, a one-block scan of the tile
// sums, then the per-tile scan plus its offset.
constexpr int kScanNT = 1024;
constexpr int kScanIPT = 8;
constexpr int kScanTile = kScanNT * kScanIPT;

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
                                                            int* __restrict__ cell_start, int n,
                                                            int N, int* __restrict__ status) {
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
    if (threadIdx.x == 0) {
        cell_start[n] = carry;
        if (carry != N) atomicOr(status, kStatusTotal);
    }
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

// ------------------------------------------------------------------ misc
__global__ void k_wrap_positions(const float* __restrict__ x, int N, float o0, float o1, float o2,
                                 float h, int H, float* sx, float* sy, float* sz,
                                 int* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float Hf = __int2float_rn(H);
    int bad = 0;
    sx[i] = wrap(__fdiv_rn(__fsub_rn(x[i], o0), h), Hf, &bad);
    sy[i] = wrap(__fdiv_rn(__fsub_rn(x[N + i], o1), h), Hf, &bad);
    sz[i] = wrap(__fdiv_rn(__fsub_rn(x[2 * N + i], o2), h), Hf, &bad);
    if (bad) atomicOr(status, kStatusNonfinite);
}

__global__ void k_log_mass(const double* __restrict__ mass, int N, double* loga) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) loga[i] = log(mass[i]);
}

__global__ void k_iota(uint32_t* id, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) id[i] = static_cast<uint32_t>(i);
}

__global__ void k_export_positions(const float* __restrict__ sx, const float* __restrict__ sy,
                                   const float* __restrict__ sz, int N, float o0, float o1,
                                   float o2, float h, float* x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    x[i] = __fmaf_rn(sx[i], h, o0);
    x[N + i] = __fmaf_rn(sy[i], h, o1);
    x[2 * N + i] = __fmaf_rn(sz[i], h, o2);
}

__global__ void k_export_mass(const double* __restrict__ loga, int N, double* mass) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) mass[i] = exp(loga[i]);
}

// u_bar = acc * scale; the accumulator is cleared for the next deposit.
__global__ void k_acc_to_float(unsigned long long* __restrict__ acc, int n, float scale,
                               float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long q = static_cast<long long>(acc[i]);
    acc[i] = 0ull;
    out[i] = __fmul_rn(__ll2float_rn(q), scale);
}

// Diagnostics: deterministic two-level reduction (fixed grid, fixed trees).
constexpr int kDiagBlocks = 304;
constexpr int kDiagNT = 256;

struct DiagPart {
    double mass;      // sum exp(loga)
    double minv, minm, minw;
    double nonfinite;
    long long accsum; // fixed-point sum of u_bar
    long long accmin;
};

__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }

__global__ void __launch_bounds__(kDiagNT)
    k_diag_partials(const double* __restrict__ loga, const float* __restrict__ sx,
                    const float* __restrict__ sy, const float* __restrict__ sz, int N,
                    const float* __restrict__ v, const float* __restrict__ m,
                    const float* __restrict__ w, const unsigned long long* __restrict__ acc,
                    int ncell, double* __restrict__ part_d, long long* __restrict__ part_l) {
    double mass = 0.0, mv = INFINITY, mm = INFINITY, mw = INFINITY, nf = 0.0;
    long long as = 0, amin = LLONG_MAX;
    const int stride = kDiagBlocks * kDiagNT;
    for (int i = blockIdx.x * kDiagNT + threadIdx.x; i < N; i += stride) {
        mass += exp(loga[i]);
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
    sd[0][threadIdx.x] = mass;
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
            sd[0][threadIdx.x] += sd[0][j];
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
        part_l[blockIdx.x * 2] = sl[0][0];
        part_l[blockIdx.x * 2 + 1] = sl[1][0];
    }
}

__global__ void k_diag_final(const double* __restrict__ part_d, const long long* __restrict__ part_l,
                             double acc_to_u, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double mass = 0, mv = INFINITY, mm = INFINITY, mw = INFINITY, nf = 0;
    long long as = 0, amin = LLONG_MAX;
    for (int b = 0; b < kDiagBlocks; ++b) {
        mass += part_d[b * 5];
        mv = dmin(mv, part_d[b * 5 + 1]);
        mm = dmin(mm, part_d[b * 5 + 2]);
        mw = dmin(mw, part_d[b * 5 + 3]);
        nf += part_d[b * 5 + 4];
        as += part_l[b * 2];
        amin = part_l[b * 2 + 1] < amin ? part_l[b * 2 + 1] : amin;
    }
    out[0] = mass;
    out[1] = static_cast<double>(as) * acc_to_u;   // sum of u_bar (times h^3 on the host)
    out[2] = static_cast<double>(amin) * acc_to_u;
    out[3] = mv;
    out[4] = mm;
    out[5] = mw;
    out[6] = nf;
}

__global__ void k_normals(const uint32_t* __restrict__ ids, int N, uint32_t n, uint32_t k0,
                          uint32_t k1, float* __restrict__ z, uint32_t* __restrict__ bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
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

inline Fields fields_of(sipf_ctx* c) { return Fields{c->gx, c->gy, c->gz, c->w}; }

inline Store store_of(sipf_ctx* c, int b) {
    return Store{c->sx[b], c->sy[b], c->sz[b], c->loga[b], c->id[b]};
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_count(sipf_ctx* c, const PushArgs& a) {
    const int b = c->cur;
    k_count<<<blocks_for(c->N, kNT), kNT, 0, c->stream>>>(a, fields_of(c), c->sx[b], c->sy[b],
                                                           c->sz[b], c->id[b],
                                                           static_cast<int>(c->N), c->count);
    return cudaGetLastError();
}

cudaError_t launch_scan(sipf_ctx* c) {
    const int n = c->H * c->H * c->H;
    const int ntiles = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<ntiles, kScanNT, 0, c->stream>>>(c->count, n, c->scan_tmp);
    k_scan_tile_sums<<<1, kScanNT, 0, c->stream>>>(c->scan_tmp, ntiles, c->cell_start, n,
                                                   static_cast<int>(c->N), c->status);
    k_scan_apply<<<ntiles, kScanNT, 0, c->stream>>>(c->count, n, c->scan_tmp, c->cell_start);
    return cudaGetLastError();
}

cudaError_t launch_scatter(sipf_ctx* c, const PushArgs& a, const DepositArgs& d, int deposit,
                           int scatter) {
    const int b = c->cur;
    k_scatter<<<blocks_for(c->N, kNT), kNT, 0, c->stream>>>(
        a, d, fields_of(c), store_of(c, b), store_of(c, b ^ 1), static_cast<int>(c->N), deposit,
        scatter, c->count, c->cell_start, reinterpret_cast<unsigned long long*>(c->acc),
        c->status);
    return cudaGetLastError();
}

cudaError_t launch_wrap_positions(sipf_ctx* c, const float* x, int buf) {
    const int N = static_cast<int>(c->N);
    k_wrap_positions<<<blocks_for(N, 256), 256, 0, c->stream>>>(
        x, N, static_cast<float>(c->origin[0]), static_cast<float>(c->origin[1]),
        static_cast<float>(c->origin[2]), static_cast<float>(c->h), c->H, c->sx[buf], c->sy[buf],
        c->sz[buf], c->status);
    return cudaGetLastError();
}

cudaError_t launch_log_mass(sipf_ctx* c, const double* mass, int buf) {
    const int N = static_cast<int>(c->N);
    k_log_mass<<<blocks_for(N, 256), 256, 0, c->stream>>>(mass, N, c->loga[buf]);
    return cudaGetLastError();
}

cudaError_t launch_iota(sipf_ctx* c, int buf) {
    const int N = static_cast<int>(c->N);
    k_iota<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->id[buf], N);
    return cudaGetLastError();
}

cudaError_t launch_export_positions(sipf_ctx* c, float* x) {
    const int N = static_cast<int>(c->N), b = c->cur;
    k_export_positions<<<blocks_for(N, 256), 256, 0, c->stream>>>(
        c->sx[b], c->sy[b], c->sz[b], N, static_cast<float>(c->origin[0]),
        static_cast<float>(c->origin[1]), static_cast<float>(c->origin[2]),
        static_cast<float>(c->h), x);
    return cudaGetLastError();
}

cudaError_t launch_export_mass(sipf_ctx* c, double* mass) {
    const int N = static_cast<int>(c->N);
    k_export_mass<<<blocks_for(N, 256), 256, 0, c->stream>>>(c->loga[c->cur], N, mass);
    return cudaGetLastError();
}

cudaError_t launch_acc_to_float(sipf_ctx* c, float* dst, float scale) {
    const int n = c->H * c->H * c->H;
    k_acc_to_float<<<blocks_for(n, 256), 256, 0, c->stream>>>(
        reinterpret_cast<unsigned long long*>(c->acc), n, scale, dst);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(sipf_ctx* c, float acc_to_u) {
    const int b = c->cur;
    k_diag_partials<<<kDiagBlocks, kDiagNT, 0, c->stream>>>(
        c->loga[b], c->sx[b], c->sy[b], c->sz[b], static_cast<int>(c->N), c->v, c->m, c->w,
        reinterpret_cast<const unsigned long long*>(c->acc), c->H * c->H * c->H, c->diag_tmp,
        c->diag_ll);
    k_diag_final<<<1, 32, 0, c->stream>>>(c->diag_tmp, c->diag_ll, static_cast<double>(acc_to_u),
                                          c->diag_out);
    return cudaGetLastError();
}

cudaError_t launch_normals(const uint32_t* ids, int64_t N, uint32_t n, uint64_t seed, float* z,
                           uint32_t* bits, cudaStream_t s) {
    k_normals<<<blocks_for(N, 256), 256, 0, s>>>(ids, static_cast<int>(N), n,
                                                 static_cast<uint32_t>(seed),
                                                 static_cast<uint32_t>(seed >> 32), z, bits);
    return cudaGetLastError();
}

size_t diag_scratch_doubles() { return static_cast<size_t>(kDiagBlocks) * 5; }
size_t diag_scratch_ll() { return static_cast<size_t>(kDiagBlocks) * 2; }
int scan_tiles(int n) { return (n + kScanTile - 1) / kScanTile; }

}  // namespace sipf
