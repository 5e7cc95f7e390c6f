// Kernel templates of the spectral passes (see fft.cu for the pass
// structure): the three fused plane/column passes for H <= 128, the per-axis
// passes for H > 128, and their launch templates.  Each translation unit that
// launches them includes this header (internal linkage) and instantiates the
// grid sizes and radix plans it serves, so that the instantiations compile in
// parallel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fft_stages.cuh"
#include "sipf_internal.cuh"

namespace sipf {
namespace {


using namespace fftk;

// (H - k) mod H for 0 <= k <= H: the index of the mode -k.
template <int H>
__device__ __forceinline__ int neg_mod(int k) {
    if constexpr ((H & (H - 1)) == 0) return (H - k) & (H - 1);
    else return k == 0 ? 0 : H - k;
}

// Threads of the three fused passes (H <= 128) or of the z pass (H > 128),
// chosen so that the radix-16 or radix-8 stages hold at most two butterflies
// per thread.
template <int H> struct Cfg;
template <> struct Cfg<8> { static constexpr int NT1 = 64, NT2 = 64, NT3 = 64; };
template <> struct Cfg<16> { static constexpr int NT1 = 256, NT2 = 256, NT3 = 256; };
template <> struct Cfg<24> { static constexpr int NT1 = 256, NT2 = 128, NT3 = 256; };
template <> struct Cfg<32> { static constexpr int NT1 = 256, NT2 = 256, NT3 = 256; };
template <> struct Cfg<48> { static constexpr int NT1 = 256, NT2 = 256, NT3 = 256; };
template <> struct Cfg<64> { static constexpr int NT1 = 512, NT2 = 512, NT3 = 512; };
template <> struct Cfg<72> { static constexpr int NT1 = 512, NT2 = 352, NT3 = 512; };
template <> struct Cfg<96> { static constexpr int NT1 = 768, NT2 = 608, NT3 = 768; };
// 544 = 17 warps: one radix-16 butterfly per thread for the 65 z-transforms
template <> struct Cfg<128> { static constexpr int NT1 = 1024, NT2 = 544, NT3 = 1024; };
// H > 128 runs the per-axis pipeline; only the z pass (over 32-column tiles)
// takes its threads from here
template <> struct Cfg<144> { static constexpr int NT2 = 288; };
template <> struct Cfg<192> { static constexpr int NT2 = 384; };
template <> struct Cfg<216> { static constexpr int NT2 = 896; };
template <> struct Cfg<256> { static constexpr int NT2 = 512; };
template <> struct Cfg<288> { static constexpr int NT2 = 576; };
template <> struct Cfg<384> { static constexpr int NT2 = 768; };
template <> struct Cfg<432> { static constexpr int NT2 = 896; };
template <> struct Cfg<512> { static constexpr int NT2 = 1024; };

// kx columns per block of the z pass: the whole padded row up to H = 128
template <int H> constexpr int zcols() { return H <= 128 ? H / 2 + 2 : 32; }

template <int H> constexpr int kxp() { return H / 2 + 2; }
// shared-memory pitch (float2) of half-spectrum rows in the inverse pass: odd,
// so that lanes reading one element of consecutive rows hit distinct banks
template <int H> constexpr int kxs() { return H / 2 + 1; }
// shared-memory pitch (float2) of rows that are transformed along the row
template <int H> constexpr int rowp() { return H + 1; }

__device__ __forceinline__ int signed_mode(int k, int H) { return k < H / 2 ? k : k - H; }

// ---------------------------------------------------------------- I/O helpers
// int64 (two's complement) deposit accumulator -> float, via the signed high
// and the unsigned low 32-bit halves (the single 64-bit conversion would run
// on the FP64 pipe).
__device__ __forceinline__ float acc_to_float(unsigned long long q) {
    const float hi = __int2float_rn(static_cast<int>(static_cast<unsigned>(q >> 32)));
    const float lo = __uint2float_rn(static_cast<unsigned>(q));
    return fmaf(hi, 4294967296.0f, lo);
}

// R_tau at one node: (m*, w*) and v^n.
// um is the u of the m source: u itself, or K_sigma * u (Eq. m_reg).
// The quotients use the hardware reciprocal (within 2 ulp): the
// denominators are at least 1.
__device__ __forceinline__ void react(const SpectralArgs& a, float vv, float mm, float ww, float u,
                                      float um, float& ms, float& ws, float& vn) {
    ms = mm;
    ws = ww;
    if (a.do_mw) {
        // explicit Euler of S = (-alpha m v; u; gamma v - eta(u) w), eta(u) = 2u/(1+u)
        const float eta = __fdividef(2.0f * u, 1.0f + u);
        ms = mm + a.tau * um;
        ws = ww + a.tau * (a.gamma * vv - eta * ww);
    }
    vn = (a.v_update == SIPF_V_IMPLICIT) ? __fdividef(vv, 1.0f + a.alpha * a.tau * mm)
                                         : vv * (1.0f - a.alpha * a.tau * mm);
}

// ---------------------------------------------------------------- pass 1
// Launch-parameter batches: NB = 1 for one context's step, kMaxBatch for an
// ensemble's runs of one grid size (the run index is a grid dimension).
template <int H, int NB, int V>
__global__ void __launch_bounds__(Cfg<H>::NT1)
    k_forward_xy(const __grid_constant__ SpecBatch<NB> batch) {
    const SpecRun& R = batch.run[NB == 1 ? 0 : blockIdx.y];
    const SpectralArgs& a = R.a;
    const float* v = R.v;
    const float* __restrict__ m = R.m;
    const float* __restrict__ w = R.w;
    unsigned long long* __restrict__ acc = R.acc;
    float* v_out = R.v_out;
    float2* __restrict__ gM = R.specM;
    float2* __restrict__ gW = R.specW;
    float2* __restrict__ gV = R.specV;
    const float2* __restrict__ twg = R.twiddle;
    const float* __restrict__ voff = R.voff;
    const StepScalars* __restrict__ sc = R.sc;
    const float* __restrict__ us = R.us;
    constexpr int NT = Cfg<H>::NT1, KXP = kxp<H>(), HK = H / 2 + 1, RP = rowp<H>();
    pdl_trigger();
    extern __shared__ float2 sm[];
    float2* Z = sm;               // [H][RP]: m* + i w*
    float2* Vb = Z + H * RP;      // v^n: [H/2][RP] row pairs, then [H][KXP] half rows
    float2* tw = Vb + H * KXP;    // [H]
    const int z = blockIdx.x;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    pdl_wait();   // the deposit, fields and step scalars of the kernels before
    const float u_scale = sc->u_scale;   // u_bar per accumulator unit
    const size_t plane = static_cast<size_t>(z) * H * H;
    const float c0 = *voff;   // the v spectrum only feeds derivatives: remove a constant
    {
        // node pairs (p, x), (p + H/2, x): consecutive lanes take consecutive x,
        // so the rows of Z and the row pairs of Vb are written without bank
        // conflicts; all loads of a batch are issued first
        constexpr int HH = H / 2, NPR = HH * H, ITER = (NPR + NT - 1) / NT;
        constexpr int CH = ITER < 2 ? ITER : 2;
        const float* vp = v + plane;
        const float* mp = m + plane;
        const float* wp = w + plane;
        unsigned long long* ap = acc + plane;
        float* vo = v_out + plane;
#pragma unroll 1
        for (int i0 = 0; i0 < ITER; i0 += CH) {
            float rv[CH][2], rm[CH][2], rw[CH][2], ru[CH][2];
            unsigned long long ra[CH][2];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int q = threadIdx.x + (i0 + c) * NT;
                if (i0 + c < ITER && q < NPR) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int o = q + h * NPR;   // (p + h H/2) H + x
                        rv[c][h] = vp[o];
                        rm[c][h] = mp[o];
                        rw[c][h] = wp[o];
                        ra[c][h] = ap[o];
                        ru[c][h] = us ? us[plane + o] : 0.f;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int q = threadIdx.x + (i0 + c) * NT;
                if (!(i0 + c < ITER && q < NPR)) continue;
                const int pr = q / H, x = q % H;
                float vn[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int o = q + h * NPR;
                    ap[o] = 0ull;
                    float ms, ws;
                    const float u = acc_to_float(ra[c][h]) * u_scale;
                    react(a, rv[c][h], rm[c][h], rw[c][h], u, us ? ru[c][h] : u, ms, ws, vn[h]);
                    Z[(pr + h * HH) * RP + x] = make_float2(ms, ws);
                    if (a.write_v) vo[o] = vn[h];
                }
                Vb[pr * RP + x] = make_float2(vn[0] - c0, vn[1] - c0);
            }
        }
    }
    __syncthreads();
    if (a.do_mw) fft_axis<H, V, H, 1, RP, NT, -1>(Z, tw);
    fft_axis<H, V, H / 2, 1, RP, NT, -1>(Vb, tw);
    {
        // split each transformed row pair z = x1 + i x2 (rows p, p + H/2) into
        // the half rows X1, X2 (kx <= H/2).  X(0) and X(H/2) of a real row are
        // real: column 0 holds X(0) + i X(H/2), so H/2 columns remain
        constexpr int HH = H / 2, NS = HH * HH, SPT = (NS + NT - 1) / NT;
        float2 x1[SPT], x2[SPT];
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NS) {
                const int p = idx / HH, k = idx % HH;
                const float2 zp = Vb[p * RP + k];
                const float2 zm = Vb[p * RP + (k == 0 ? HH : H - k)];
                if (k == 0) {
                    // zm is z(H/2) here: X1(0) = Re z(0), X1(H/2) = Re z(H/2), X2 from Im
                    x1[s] = make_float2(zp.x, zm.x);
                    x2[s] = make_float2(zp.y, zm.y);
                } else {
                    x1[s] = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
                    x2[s] = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NS) {
                const int p = idx / HH, k = idx % HH;
                Vb[p * KXP + k] = x1[s];
                Vb[(p + HH) * KXP + k] = x2[s];
            }
        }
        __syncthreads();
    }
    if (a.do_mw) fft_axis<H, V, H, RP, 1, NT, -1>(Z, tw);
    fft_axis<H, V, H / 2, KXP, 1, NT, -1>(Vb, tw);
    // half spectra, rows of KXP (the last slot, kx = H/2 + 1, is zero); M, W
    // separated from the 2D spectrum of m* + i w*; one mode per thread
    constexpr int NP = H * KXP;
    const size_t sbase = static_cast<size_t>(z) * H * KXP;
    for (int idx = threadIdx.x; idx < NP; idx += NT) {
        const int ky = idx / KXP, k = idx % KXP;
        float2 M = make_float2(0.f, 0.f), W = M, Vk = M;
        if (k < HK) {
            const float2 zk = Z[ky * RP + k];
            const float2 zc = Z[neg_mod<H>(ky) * RP + neg_mod<H>(k)];
            M = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
            W = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
            if (k == 0 || k == H / 2) {
                // the packed column P = V(0, .) + i V(H/2, .): V(0, ky) =
                // (P(ky) + conj P(-ky))/2, V(H/2, ky) = (P(ky) - conj P(-ky))/(2i)
                const float2 pk = Vb[ky * KXP], pc = Vb[neg_mod<H>(ky) * KXP];
                Vk = k == 0 ? make_float2(0.5f * (pk.x + pc.x), 0.5f * (pk.y - pc.y))
                            : make_float2(0.5f * (pk.y + pc.y), -0.5f * (pk.x - pc.x));
            } else {
                Vk = Vb[ky * KXP + k];
            }
        }
        if (a.do_mw) {
            gM[sbase + idx] = M;
            gW[sbase + idx] = W;
        }
        gV[sbase + idx] = Vk;
    }
}

// ---------------------------------------------------------------- pass 2
// Block (ky, field, kx tile): forward DFT along z of the KB columns
// [k0, k0 + KB) of the (z, ky) rows, the per-mode multiplier, inverse DFT.
template <int H, int NB, int V>
__global__ void __launch_bounds__(Cfg<H>::NT2)
    k_z_multiply(const __grid_constant__ SpecBatch<NB> batch) {
    constexpr int NT = Cfg<H>::NT2, KXP = kxp<H>(), HK = H / 2 + 1, KB = zcols<H>();
    // batches (H <= 128: one kx tile per row) take the run from grid dimension z
    static_assert(NB == 1 || KB >= KXP, "batched z pass needs one kx tile");
    const SpecRun& R = batch.run[NB == 1 ? 0 : blockIdx.z];
    const SpectralArgs& a = R.a;
    float2* __restrict__ gM = R.specM;
    float2* __restrict__ gW = R.specW;
    const float2* __restrict__ gV = R.specV;
    float2* __restrict__ gB = R.specB;
    float2* __restrict__ gA = R.specA;
    const float2* __restrict__ twg = R.twiddle;
    float* __restrict__ voff = R.voff;
    extern __shared__ float2 sm[];
    float2* buf = sm;             // [H (z)][KB (kx)]
    float2* tw = buf + H * KB;
    const int ky = blockIdx.x, field = blockIdx.y;   // 0 m, 1 w, 2 v -> i k_z V, 3 v -> filtered V
    const int k0 = NB == 1 ? blockIdx.z * KB : 0;
    pdl_trigger();
    if (field < 2 && !a.do_mw) return;
    if (field == 3 && !a.filter) return;
    const float2* src = field == 0 ? gM : field == 1 ? gW : gV;
    float2* dst = field == 0 ? gM : field == 1 ? gW : field == 2 ? gB : gA;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    pdl_wait();   // the forward pass's spectra
    constexpr int R1 = Radix<H, V>::R1;
    // element (column t, z) of the block's tile in a [z][ky][KXP] half spectrum
    auto at = [ky, k0](int t, int zz) -> size_t {
        return (static_cast<size_t>(zz) * H + ky) * KXP + k0 + t;
    };
    // forward z DFT, its first stage loading the columns from global memory
    stage1_from<H, R1, KB, KB, 1, NT, -1>(buf, [=](int t, int zz) {
        return k0 + t < KXP ? src[at(t, zz)] : make_float2(0.f, 0.f);
    });
    // its last stage applies the per-mode factor on the way back to shared memory
    const int qy = signed_mode(ky, H);
    fft_rest_sink<H, V, KB, KB, 1, NT, -1>(buf, tw, [=](int t, int kz, float2 val) {
        const int qx = k0 + t;
        if (qx < HK) {
            if (field == 2 && ky == 0 && qx == 0 && kz == 0) {
                // DC of (v^n - c0): move the offset to the mean of v^n for the next step
                *voff = *voff + val.x * a.out_scale;
            }
            const int qz = signed_mode(kz, H);
            const float q2 = static_cast<float>(qx * qx + qy * qy + qz * qz);
            float f = 1.0f;
            if (field == 2) {
                const float kz_phys =
                    (qz == -H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(qz);
                val = make_float2(-kz_phys * val.y, kz_phys * val.x);
            } else if (field < 2) {
                const float c = field == 0 ? a.m_c : a.w_c;
                f = a.diffusion == SIPF_DIFFUSION_IMPLICIT ? __fdividef(1.0f, 1.0f + c * q2)
                                                           : expf(-c * q2);
            }
            if (a.filter) f *= expf(-a.inv_H0sq_2pi2 * q2);
            val = make_float2(f * val.x, f * val.y);
            if (field < 2) {
                // times r0 = hi + lo: the float32 rounding of r0 itself is compensated
                const float hi = field == 0 ? a.m_r0_hi : a.w_r0_hi;
                const float lo = field == 0 ? a.m_r0_lo : a.w_r0_lo;
                val = make_float2(fmaf(val.x, lo, val.x * hi), fmaf(val.y, lo, val.y * hi));
            }
        }
        buf[kz * KB + t] = val;
    });
    // inverse z DFT, its last stage storing the columns to global memory
    stage<H, R1, 1, KB, KB, 1, NT, +1>(buf, tw);
    fft_rest_sink<H, V, KB, KB, 1, NT, +1>(buf, tw, [=](int t, int zz, float2 val) {
        if (k0 + t < KXP) dst[at(t, zz)] = val;
    });
}

// Shapes of the lane-group transforms of the warp pipeline (below): P lanes
// per line; exchange tiles of PITCH float2 per row and TILE float2 per group,
// chosen so that the exchanges are free of bank conflicts.
template <int H> struct LaneShape;
template <> struct LaneShape<64> { static constexpr int P = 8, PITCH = 9, TILE = 72; };
template <> struct LaneShape<128> { static constexpr int P = 8, PITCH = 18, TILE = 145; };
template <> struct LaneShape<256> { static constexpr int P = 16, PITCH = 17, TILE = 272; };
constexpr int kLaneWarps = 8;   // warps per block of the warp pipeline

// ---------------------------------------------------------------- pass 3
// Build the full-length complex row Z[kx] = X1[kx] + i X2[kx] of two real
// signals from their half spectra (Hermitian extension, C2R semantics at
// kx = 0 and kx = H/2).
template <int H>
__device__ __forceinline__ float2 pack_two(const float2* r1, const float2* r2, int kx) {
    float2 a, b;
    if (kx <= H / 2) {
        a = r1[kx];
        b = r2[kx];
        if (kx == 0 || kx == H / 2) {
            a.y = 0.f;
            b.y = 0.f;
        }
    } else {
        a = conjf2(r1[H - kx]);
        b = conjf2(r2[H - kx]);
    }
    return make_float2(a.x - b.y, a.y + b.x);
}

// Loaders for the fused first stages of the inverse pass.
struct PlaneLoad {      // half-spectrum plane from global memory, optionally times i k
    const float2* p;
    int kxp;
    float kx_scale, ky_scale;   // 2 pi / L, or 0 for "no multiplier"
    int H, dir;                 // dir 0: plain, 1: i k_x, 2: i k_y
    __device__ __forceinline__ float2 operator()(int kx, int ky) const {
        const float2 val = __ldg(p + static_cast<size_t>(ky) * kxp + kx);
        if (dir == 0) return val;
        float k;
        if (dir == 1) {
            k = (kx >= H / 2) ? 0.0f : kx_scale * static_cast<float>(kx);
        } else {
            const int qy = ky < H / 2 ? ky : ky - H;
            k = (qy == -H / 2) ? 0.0f : ky_scale * static_cast<float>(qy);
        }
        return make_float2(-k * val.y, k * val.x);
    }
};

template <int H>
struct PackLoad {       // complex row of two real signals from their half spectra
    const float2* r1;
    const float2* r2;
    int pitch1, pitch2;         // row pitch (float2) of the two sources
    __device__ __forceinline__ float2 operator()(int row, int kx) const {
        return pack_two<H>(r1 + row * pitch1, r2 + row * pitch2, kx);
    }
};

// group 1: (i k_x V, i k_y V, B) -> grad v^n; group 0: (m, w) -> m^n, w^n.
// The first inverse-y stage reads the planes straight from global memory and
// the first inverse-x stage reads the packed rows straight from the y output.
template <int H, int NB, int V>
__global__ void __launch_bounds__(Cfg<H>::NT3)
    k_inverse_xy(const __grid_constant__ SpecBatch<NB> batch) {
    const SpecRun& R = batch.run[NB == 1 ? 0 : blockIdx.z];
    const SpectralArgs& a = R.a;
    const float2* __restrict__ gM = R.specM;
    const float2* __restrict__ gW = R.specW;
    const float2* __restrict__ gV = a.filter ? R.specA : R.specV;
    const float2* __restrict__ gB = R.specB;
    float* __restrict__ m_out = R.m_out;
    float* __restrict__ w_out = R.w_out;
    float* __restrict__ G = R.G;
    const float2* __restrict__ twg = R.twiddle;
    constexpr int NT = Cfg<H>::NT3, KXP = kxp<H>(), KXS = kxs<H>(), HK = H / 2 + 1;
    constexpr int RP = rowp<H>(), R1 = Radix<H, V>::R1;
    static_assert(H * RP <= 2 * H * KXS, "packed rows must fit in B0/B1");
    static_assert((H / 2) * RP <= H * KXS, "packed row pairs must fit in B2");
    extern __shared__ float2 sm[];
    float2* B0 = sm;              // [H][KXS]
    float2* B1 = B0 + H * KXS;    // [H][KXS]
    float2* B2 = B1 + H * KXS;    // [H][KXS] (group 1)
    float2* tw = B2 + H * KXS;
    float2* Z = sm;               // [H][RP] packed rows (aliases B0/B1)
    float2* Z2 = B2;              // [H/2][RP] rows y, y + H/2 of B2 packed (aliases B2)
    // the two groups of a plane are neighbouring blocks: their partial writes
    // of the gather array's nodes (x, y, z components, then w) follow each
    // other closely, while the lines are still in L2
    const int z = blockIdx.x >> 1, group = 1 - static_cast<int>(blockIdx.x & 1);
    pdl_trigger();
    if (group == 0 && !a.do_mw) return;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    __syncthreads();
    pdl_wait();   // the z pass's spectra
    const size_t pbase = static_cast<size_t>(z) * H * KXP;
    // inverse y: first stage from global, second in shared memory
    if (group == 0) {
        stage1_from<H, R1, HK, KXS, 1, NT, +1>(B0, PlaneLoad{gM + pbase, KXP, 0.f, 0.f, H, 0});
        stage1_from<H, R1, HK, KXS, 1, NT, +1>(B1, PlaneLoad{gW + pbase, KXP, 0.f, 0.f, H, 0});
    } else {
        const float k = a.two_pi_over_L;
        stage1_from<H, R1, HK, KXS, 1, NT, +1>(B0, PlaneLoad{gV + pbase, KXP, k, k, H, 1});
        stage1_from<H, R1, HK, KXS, 1, NT, +1>(B1, PlaneLoad{gV + pbase, KXP, k, k, H, 2});
        stage1_from<H, R1, HK, KXS, 1, NT, +1>(B2, PlaneLoad{gB + pbase, KXP, 0.f, 0.f, H, 0});
    }
    fft_rest<H, V, HK, KXS, 1, NT, +1>(B0, tw);
    fft_rest<H, V, HK, KXS, 1, NT, +1>(B1, tw);
    if (group == 1) fft_rest<H, V, HK, KXS, 1, NT, +1>(B2, tw);
    // inverse x: first stage from the packed half spectra (in place), second stage
    if (group == 1) {
        // B2's rows y and y + H/2 as one complex row -> Z2 (B2's own space); done
        // first, B0/B1 are still intact
        stage1_from<H, R1, H / 2, 1, RP, NT, +1>(Z2,
                                                  PackLoad<H>{B2, B2 + (H / 2) * KXS, KXS, KXS});
    }
    stage1_from<H, R1, H, 1, RP, NT, +1>(Z, PackLoad<H>{B0, B1, KXS, KXS});
    fft_rest<H, V, H, 1, RP, NT, +1>(Z, tw);
    if (group == 1) fft_rest<H, V, H / 2, 1, RP, NT, +1>(Z2, tw);
    const size_t plane = static_cast<size_t>(z) * H * H;
    float* Gp = G + 4 * plane;
    if (group == 0) {
        // m^n, w^n, and w^n again as the fourth component of the gather array
        // (consecutive lanes read consecutive x: no bank conflicts)
        const float sc = a.out_scale;
        float* p1 = m_out + plane;
        float* p2 = w_out + plane;
        for (int i = threadIdx.x; i < H * H; i += NT) {
            const int y = i / H, x = i % H;
            const float2 e = Z[y * RP + x];
            const float wv = e.y * sc;
            p1[i] = e.x * sc;
            p2[i] = wv;
            Gp[4 * i + 3] = wv;
        }
    } else {
        // (dv/dx, dv/dy, dv/dz) into components 0..2 of the gather array
        const float sxy = a.out_scale_xy, sz_ = a.out_scale;
        for (int i = threadIdx.x; i < H * H; i += NT) {
            const int y = i / H, x = i % H;
            const float2 e = Z[y * RP + x];
            const bool upper = y >= H / 2;
            const float2 f = Z2[(upper ? y - H / 2 : y) * RP + x];
            *reinterpret_cast<float2*>(Gp + 4 * i) = make_float2(e.x * sxy, e.y * sxy);
            Gp[4 * i + 2] = (upper ? f.y : f.x) * sz_;
        }
    }
}

// ---------------------------------------------------------------- warp per-axis pipeline
// For the grid sizes with a LaneShape the whole spectral step can run as
// five passes over lines held in registers by groups of P lanes (WarpFFT),
// with the half spectra in global memory (L2) between them and no block
// barrier inside a transform:
//   wx_forward: row pairs (z, y), (z, y + H/2): reaction; m* + i w* per row
//               and v^n of the two rows as one complex row, x DFT, split into
//               half rows -> M, W, V
//   wy (SIGN -1): columns (z, kx) of M, W, V: y DFT in place
//   z:          the block z pass (k_z_multiply; its tiles read whole rows)
//   wy (SIGN +1): columns of M, W, B in place, V (or its filtered copy) ->
//               i k_x V, i k_y V
//   wx_inverse: rows: (m, w), (dv/dx, dv/dy), and dv/dz row pairs, packed
//               two real outputs per complex row, inverse x DFT; a block
//               writes whole rows of the gather array.
// Lines are assigned to groups in a flat order, so that a warp's groups read
// and write neighbouring memory.

// Split a transformed complex row X = X1 + i X2 of two real rows, held in
// the spectral layout, into their half rows (kx < H/2 + 2, the last one the
// zero padding): X1(k) = (X(k) + conj X(-k))/2, X2(k) = (X(k) - conj X(-k))/(2i).
template <int H, class F>
__device__ __forceinline__ void split_store(const float2 (&v)[F::Q], int l, float2* ex,
                                            float2* d1, float2* d2) {
    constexpr int P = F::Q / F::S, S = F::S, Q = F::Q, KXP = kxp<H>(), HK = H / 2 + 1;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) ex[S * l + s + Q * k2] = v[s * P + k2];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < (KXP + P - 1) / P; ++j) {
        const int k = l + P * j;
        if (k < KXP) {
            float2 a1 = make_float2(0.f, 0.f), a2 = a1;
            if (k < HK) {
                const float2 zp = ex[k], zm = ex[neg_mod<H>(k)];
                a1 = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
                a2 = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
            }
            d1[k] = a1;
            if (d2) d2[k] = a2;
        }
    }
}

template <int H, int NB>
__global__ void __launch_bounds__(32 * kLaneWarps)
    k_wx_forward(const __grid_constant__ SpecBatch<NB> batch) {
    using C = LaneShape<H>;
    using F = WarpFFT<H, C::P, C::PITCH>;
    constexpr int P = C::P, Q = F::Q, G = 32 / P, KXP = kxp<H>(), HH = H / 2;
    __shared__ float2 tw[H];
    __shared__ float2 exch[kLaneWarps][G * C::TILE];
    const SpecRun& R = batch.run[NB == 1 ? 0 : blockIdx.z];
    const SpectralArgs& a = R.a;
    for (int i = threadIdx.x; i < H; i += blockDim.x) tw[i] = R.twiddle[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / P, l = lane % P;
    const int task = (blockIdx.x * kLaneWarps + warp) * G + g;   // (z, y < H/2)
    if (task >= H * HH) return;    // whole groups; H * H/2 is a multiple of every group count
    const int z = task / HH, y = task % HH;
    float2* ex = &exch[warp][g * C::TILE];
    const float u_scale = R.sc->u_scale;   // u_bar per accumulator unit
    const float c0 = *R.voff;   // the v spectrum only feeds derivatives: remove a constant
    const size_t row0 = (static_cast<size_t>(z) * H + y) * H;
    const size_t row1 = row0 + static_cast<size_t>(HH) * H;
    const float gamma_v = a.alpha * a.tau;
    {
        // v^n of the two rows as one complex row (reads v and m only)
        float2 zv[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const int x = l + P * m;
            float vn[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const size_t o = (h ? row1 : row0) + x;
                const float vv = R.v[o], mm = R.m[o];
                vn[h] = (a.v_update == SIPF_V_IMPLICIT) ? __fdividef(vv, 1.0f + gamma_v * mm)
                                                        : vv * (1.0f - gamma_v * mm);
            }
            zv[m] = make_float2(vn[0] - c0, vn[1] - c0);
        }
        F::template to_spectral<-1>(zv, l, ex, tw);
        const size_t s0 = (static_cast<size_t>(z) * H + y) * KXP;
        split_store<H, F>(zv, l, ex, R.specV + s0, R.specV + s0 + static_cast<size_t>(HH) * KXP);
    }
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        // the reaction on row y + h H/2: m* + i w*, v^n, the accumulator cleared
        const size_t row = h ? row1 : row0;
        float2 zr[Q];
        // chunks of CH elements: all loads of a chunk before its stores (the
        // stores may alias later loads, so they would otherwise wait)
        constexpr int CH = 4;
#pragma unroll
        for (int m0 = 0; m0 < Q; m0 += CH) {
            float vv[CH], mm[CH], ww[CH], uu[CH];
            unsigned long long qq[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const size_t o = row + l + P * (m0 + c);
                vv[c] = R.v[o];
                mm[c] = R.m[o];
                ww[c] = R.w[o];
                qq[c] = R.acc[o];
                uu[c] = R.us ? R.us[o] : 0.f;
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const size_t o = row + l + P * (m0 + c);
                R.acc[o] = 0ull;
                const float u = acc_to_float(qq[c]) * u_scale;
                float ms, ws, vn;
                react(a, vv[c], mm[c], ww[c], u, R.us ? uu[c] : u, ms, ws, vn);
                zr[m0 + c] = make_float2(ms, ws);
                if (a.write_v) R.v_out[o] = vn;
            }
        }
        if (a.do_mw) {
            F::template to_spectral<-1>(zr, l, ex, tw);
            const size_t s = (static_cast<size_t>(z) * H + y + h * HH) * KXP;
            split_store<H, F>(zr, l, ex, R.specM + s, R.specW + s);
        }
    }
}

// y DFT of columns (z, kx) of the half spectra.  SIGN -1: M, W, V in place
// (spatial layout in, spectral out).  SIGN +1: M, W, B in place, and V (or
// its filtered copy) -> i k_x V, i k_y V (spectral layout in, spatial out).
template <int H, int SIGN, int NB>
__global__ void __launch_bounds__(32 * kLaneWarps) k_wy(const __grid_constant__ SpecBatch<NB> batch) {
    using C = LaneShape<H>;
    using F = WarpFFT<H, C::P, C::PITCH>;
    constexpr int P = C::P, Q = F::Q, S = F::S, G = 32 / P, KXP = kxp<H>();
    __shared__ float2 tw[H];
    __shared__ float2 exch[kLaneWarps][G * C::TILE];
    const SpecRun& R = batch.run[NB == 1 ? 0 : blockIdx.z];
    const SpectralArgs& a = R.a;
    const int field = blockIdx.y;   // 0 M, 1 W, 2 V or B, 3 -> i k_x V, 4 -> i k_y V
    if (field < 2 && !a.do_mw) return;
    for (int i = threadIdx.x; i < H; i += blockDim.x) tw[i] = R.twiddle[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / P, l = lane % P;
    const int col = (blockIdx.x * kLaneWarps + warp) * G + g;   // (z, kx)
    if (col >= H * KXP) return;    // whole groups
    const int z = col / KXP, kx = col % KXP;
    float2* ex = &exch[warp][g * C::TILE];
    const float2* vsrc = a.filter ? R.specA : R.specV;
    const float2* src = field == 0 ? R.specM : field == 1 ? R.specW
                      : field == 2 ? (SIGN < 0 ? R.specV : R.specB) : vsrc;
    float2* dst = field == 0 ? R.specM : field == 1 ? R.specW
                : field == 2 ? (SIGN < 0 ? R.specV : R.specB) : field == 3 ? R.specDx : R.specDy;
    const size_t base = static_cast<size_t>(z) * H * KXP + kx;
    float2 v[Q];
    if constexpr (SIGN < 0) {
#pragma unroll
        for (int m = 0; m < Q; ++m) v[m] = src[base + static_cast<size_t>(l + P * m) * KXP];
        F::template to_spectral<-1>(v, l, ex, tw);
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2)
                dst[base + static_cast<size_t>(S * l + s + Q * k2) * KXP] = v[s * P + k2];
        }
    } else {
        const float kxs_ = (kx >= H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(kx);
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) {
                const int ky = S * l + s + Q * k2;
                float2 val = src[base + static_cast<size_t>(ky) * KXP];
                if (field >= 3) {
                    float k;
                    if (field == 3) {
                        k = kxs_;
                    } else {
                        const int qy = signed_mode(ky, H);
                        k = (qy == -H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(qy);
                    }
                    val = make_float2(-k * val.y, k * val.x);
                }
                v[s * P + k2] = val;
            }
        }
        F::template to_spatial<+1>(v, l, ex, tw);
#pragma unroll
        for (int m = 0; m < Q; ++m) dst[base + static_cast<size_t>(l + P * m) * KXP] = v[m];
    }
}

// Inverse x DFT of packed rows: (m, w) rows, (dv/dx, dv/dy) rows and dv/dz
// row pairs (y, y + H/2); scaled outputs.  A block takes PB row pairs
// (y0 + t, y0 + t + H/2), t < PB, of one plane: 2 PB (m, w) rows, 2 PB
// (dv/dx, dv/dy) rows and PB dv/dz pairs, each warp of one kind, so that the
// four components of each node of the gather array are written close
// together in time (they are written by three kinds of tasks).
template <int H> struct WxInv {
    static constexpr int G = 32 / LaneShape<H>::P;          // lines per warp
    static constexpr int PB = 2 * G;                        // row pairs per block
    static constexpr int WMW = 2 * PB / G, WD = 2 * PB / G, WB = PB / G;
    static constexpr int WARPS = WMW + WD + WB;             // 10
};

template <int H, int NB>
__global__ void __launch_bounds__(32 * WxInv<H>::WARPS)
    k_wx_inverse(const __grid_constant__ SpecBatch<NB> batch) {
    using C = LaneShape<H>;
    using F = WarpFFT<H, C::P, C::PITCH>;
    using X = WxInv<H>;
    constexpr int P = C::P, Q = F::Q, S = F::S, G = X::G, PB = X::PB, KXP = kxp<H>(), HH = H / 2;
    static_assert(HH % PB == 0, "whole blocks of row pairs");
    __shared__ float2 tw[H];
    __shared__ float2 exch[X::WARPS][G * C::TILE];
    const SpecRun& R = batch.run[NB == 1 ? 0 : blockIdx.z];
    const SpectralArgs& a = R.a;
    for (int i = threadIdx.x; i < H; i += blockDim.x) tw[i] = R.twiddle[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / P, l = lane % P;
    constexpr int YB = HH / PB;                     // blocks of PB row pairs per plane
    const int z = blockIdx.x / YB, y0 = (blockIdx.x % YB) * PB;
    int kind, y;
    if (warp < X::WMW) {
        kind = 0;
        const int t = warp * G + g;                 // 0 .. 2 PB - 1
        y = y0 + (t % PB) + (t / PB) * HH;
    } else if (warp < X::WMW + X::WD) {
        kind = 1;
        const int t = (warp - X::WMW) * G + g;
        y = y0 + (t % PB) + (t / PB) * HH;
    } else {
        kind = 2;
        y = y0 + (warp - X::WMW - X::WD) * G + g;   // pair (y, y + H/2)
    }
    if (kind == 0 && !a.do_mw) return;              // whole warps
    float2* ex = &exch[warp][g * C::TILE];
    const size_t r0 = (static_cast<size_t>(z) * H + y) * KXP;
    const float2* p1;
    const float2* p2;
    if (kind == 0) {
        p1 = R.specM + r0;
        p2 = R.specW + r0;
    } else if (kind == 1) {
        p1 = R.specDx + r0;
        p2 = R.specDy + r0;
    } else {
        p1 = R.specB + r0;
        p2 = R.specB + r0 + static_cast<size_t>(HH) * KXP;
    }
    float2 v[Q];
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) v[s * P + k2] = pack_two<H>(p1, p2, S * l + s + Q * k2);
    }
    F::template to_spatial<+1>(v, l, ex, tw);
    const size_t node0 = (static_cast<size_t>(z) * H + y) * H;
    if (kind == 0) {
        const float sc = a.out_scale;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const size_t node = node0 + l + P * m;
            const float wv = v[m].y * sc;
            R.m_out[node] = v[m].x * sc;
            R.w_out[node] = wv;
            R.G[4 * node + 3] = wv;
        }
    } else if (kind == 1) {
        const float sxy = a.out_scale_xy;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const size_t node = node0 + l + P * m;
            *reinterpret_cast<float2*>(R.G + 4 * node) = make_float2(v[m].x * sxy, v[m].y * sxy);
        }
    } else {
        const float sc = a.out_scale;
        const size_t node1 = node0 + static_cast<size_t>(HH) * H;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            R.G[4 * (node0 + l + P * m) + 2] = v[m].x * sc;
            R.G[4 * (node1 + l + P * m) + 2] = v[m].y * sc;
        }
    }
}

// Blocks covering n lines (groups of 32 / P lanes in kLaneWarps warps).
template <int H> constexpr int warp_blocks(int n) {
    constexpr int per_block = kLaneWarps * (32 / LaneShape<H>::P);
    return (n + per_block - 1) / per_block;
}

// The warp pipeline's passes, grouped like the fused ones.
template <int H, int NB>
cudaError_t warp_pass(const SpecBatch<NB>& batch, int nb, int pass, int device, cudaStream_t s) {
    constexpr int KXP = kxp<H>(), NT = 32 * kLaneWarps, KB = zcols<H>();
    constexpr size_t smz = (static_cast<size_t>(H) * KB + H) * sizeof(float2);
    static int configured_device = -1;
    if (configured_device != device) {
        cudaFuncSetAttribute(k_z_multiply<H, NB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smz));
        configured_device = device;
    }
    if (pass == 0) {
        k_wx_forward<H, NB><<<dim3(warp_blocks<H>(H * (H / 2)), 1, nb), NT, 0, s>>>(batch);
        k_wy<H, -1, NB><<<dim3(warp_blocks<H>(H * KXP), 3, nb), NT, 0, s>>>(batch);
    } else if (pass == 1) {
        k_z_multiply<H, NB, 0><<<dim3(H, 4, NB == 1 ? (KXP + KB - 1) / KB : nb), Cfg<H>::NT2, smz,
                                 s>>>(batch);
    } else {
        k_wy<H, +1, NB><<<dim3(warp_blocks<H>(H * KXP), 5, nb), NT, 0, s>>>(batch);
        k_wx_inverse<H, NB><<<dim3(H * (H / 2 / WxInv<H>::PB), 1, nb), 32 * WxInv<H>::WARPS, 0,
                              s>>>(batch);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- per-axis passes (H > 128)
// A plane above 128^2 does not fit in shared memory, so for H > 128 each
// axis is transformed by its own kernel over small blocks of lines:
//   sx_forward: rows of RB lines: reaction, x DFT (row pairs) -> half spectra
//   sx_columns: columns (KB kx at a time) of one plane: y DFT, forward or
//               inverse; in the inverse, V becomes i k_x V and i k_y V
//   k_z_multiply (32-column tiles) between them, then
//   sx_inverse: rows: pack two real outputs per complex row, inverse x DFT.
constexpr int kSxRows = 8;     // rows per block of the x passes
constexpr int kSxCols = 16;    // kx columns per block of the y passes
constexpr int kSxNT = 256;

template <int H, int V>
__global__ void __launch_bounds__(kSxNT)
    k_sx_forward(SpectralArgs a, const float* v, const float* __restrict__ m,
                 const float* __restrict__ w, unsigned long long* __restrict__ acc, float* v_out,
                 float2* __restrict__ gM, float2* __restrict__ gW, float2* __restrict__ gV,
                 const float2* __restrict__ twg, const float* __restrict__ voff,
                 const StepScalars* __restrict__ sc, const float* __restrict__ us) {
    constexpr int RB = kSxRows, NT = kSxNT, KXP = kxp<H>(), HK = H / 2 + 1, RP = rowp<H>();
    const float u_scale = sc->u_scale;   // u_bar per accumulator unit
    static_assert((RB / 2) * RP <= RB * KXP, "row pairs fit in the half-row space");
    extern __shared__ float2 sm[];
    float2* buf = sm;              // 3 fields: [RB/2][RP] row pairs, then [RB][KXP] half rows
    float2* tw = buf + 3 * RB * KXP;
    const int z = blockIdx.y, y0 = blockIdx.x * RB;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    const float c0 = *voff;
    const size_t row0 = (static_cast<size_t>(z) * H + y0) * H;
    for (int g = threadIdx.x; g < RB * H / 4; g += NT) {
        const size_t o = row0 + 4 * static_cast<size_t>(g);
        const float4 rv = *reinterpret_cast<const float4*>(v + o);
        const float4 rm = *reinterpret_cast<const float4*>(m + o);
        const float4 rw = *reinterpret_cast<const float4*>(w + o);
        const ulonglong2 q0 = *reinterpret_cast<const ulonglong2*>(acc + o);
        const ulonglong2 q1 = *reinterpret_cast<const ulonglong2*>(acc + o + 2);
        *reinterpret_cast<ulonglong2*>(acc + o) = make_ulonglong2(0ull, 0ull);
        *reinterpret_cast<ulonglong2*>(acc + o + 2) = make_ulonglong2(0ull, 0ull);
        const float vv[4] = {rv.x, rv.y, rv.z, rv.w}, mm[4] = {rm.x, rm.y, rm.z, rm.w};
        const float ww[4] = {rw.x, rw.y, rw.z, rw.w};
        const unsigned long long qq[4] = {q0.x, q0.y, q1.x, q1.y};
        const int r = (4 * g) / H, x0 = (4 * g) % H;
        float vn[4];
        float4 ru = make_float4(0.f, 0.f, 0.f, 0.f);
        if (us) ru = *reinterpret_cast<const float4*>(us + o);
        const float uu[4] = {ru.x, ru.y, ru.z, ru.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float ms, ws;
            const float u = acc_to_float(qq[e]) * u_scale;
            react(a, vv[e], mm[e], ww[e], u, us ? uu[e] : u, ms, ws, vn[e]);
            const float val[3] = {ms, ws, vn[e] - c0};
#pragma unroll
            for (int f = 0; f < 3; ++f)
                reinterpret_cast<float*>(buf + (f * (RB / 2) + (r >> 1)) * RP)[2 * (x0 + e) + (r & 1)] =
                    val[f];
        }
        if (a.write_v) *reinterpret_cast<float4*>(v_out + o) = make_float4(vn[0], vn[1], vn[2], vn[3]);
    }
    __syncthreads();
    fft_axis<H, V, 3 * (RB / 2), 1, RP, NT, -1>(buf, tw);
    {
        // split each transformed row pair into the two rows' half spectra
        constexpr int NS = 3 * (RB / 2) * HK, SPT = (NS + NT - 1) / NT;
        float2 x1[SPT], x2[SPT];
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const int idx = threadIdx.x + t * NT;
            if (idx < NS) {
                const int pr = idx / HK, k = idx % HK;
                const float2 zp = buf[pr * RP + k];
                const float2 zm = buf[pr * RP + neg_mod<H>(k)];
                x1[t] = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
                x2[t] = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
            const int idx = threadIdx.x + t * NT;
            if (idx < NS) {
                const int pr = idx / HK, k = idx % HK;
                const int f = pr / (RB / 2), p = pr % (RB / 2);
                buf[(f * RB + 2 * p) * KXP + k] = x1[t];
                buf[(f * RB + 2 * p + 1) * KXP + k] = x2[t];
            }
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < 3 * RB * (KXP / 2); q += NT) {
        const int f = q / (RB * (KXP / 2)), rem = q % (RB * (KXP / 2));
        const int r = rem / (KXP / 2), k = 2 * (rem % (KXP / 2));
        if (f < 2 && !a.do_mw) continue;
        float2* dst = f == 0 ? gM : f == 1 ? gW : gV;
        const float2 e0 = buf[(f * RB + r) * KXP + k];
        const float2 e1 = k + 1 < HK ? buf[(f * RB + r) * KXP + k + 1] : make_float2(0.f, 0.f);
        *reinterpret_cast<float4*>(dst + (static_cast<size_t>(z) * H + y0 + r) * KXP + k) =
            make_float4(e0.x, e0.y, e1.x, e1.y);
    }
}

// y DFT of KB kx columns of one plane of `field` (forward: M, W, V in place;
// inverse: M, W, B in place, and V (or its filtered copy) -> i k_x V, i k_y V).
template <int H, int SIGN, int V>
__global__ void __launch_bounds__(kSxNT)
    k_sx_columns(SpectralArgs a, float2* f0, float2* f1, float2* f2, float2* __restrict__ dx,
                 float2* __restrict__ dy,
                 const float2* __restrict__ twg, int plain) {
    constexpr int NT = kSxNT, KXP = kxp<H>(), KB = kSxCols, CP = KB + 1;
    extern __shared__ float2 sm[];
    float2* tw = sm;               // [H]
    float2* b0 = tw + H;           // [H (y)][CP]
    float2* b1 = b0 + H * CP;      // second buffer (derivatives; allocated only for them)
    const int k0 = blockIdx.x * KB, z = blockIdx.y, field = blockIdx.z;
    if (!plain && field < 2 && !a.do_mw) return;
    const bool deriv = !plain && SIGN > 0 && field == 2;
    float2* src = field == 0 ? f0 : field == 1 ? f1 : f2;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    const size_t plane = static_cast<size_t>(z) * H * KXP;
    for (int q = threadIdx.x; q < H * KB; q += NT) {
        const int y = q / KB, t = q % KB, k = k0 + t;
        float2 val = k < KXP ? src[plane + static_cast<size_t>(y) * KXP + k] : make_float2(0.f, 0.f);
        if (deriv) {
            const int qy = signed_mode(y, H);
            const float kxp_ = (k >= H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(k);
            const float kyp = (qy == -H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(qy);
            b1[y * CP + t] = make_float2(-kyp * val.y, kyp * val.x);
            val = make_float2(-kxp_ * val.y, kxp_ * val.x);
        }
        b0[y * CP + t] = val;
    }
    __syncthreads();
    fft_axis<H, V, KB, CP, 1, NT, SIGN>(b0, tw);
    if (deriv) fft_axis<H, V, KB, CP, 1, NT, SIGN>(b1, tw);
    float2* d0 = deriv ? dx : src;
    for (int q = threadIdx.x; q < H * KB; q += NT) {
        const int y = q / KB, t = q % KB, k = k0 + t;
        if (k >= KXP) continue;
        d0[plane + static_cast<size_t>(y) * KXP + k] = b0[y * CP + t];
        if (deriv) dy[plane + static_cast<size_t>(y) * KXP + k] = b1[y * CP + t];
    }
}

// Rows of the inverse: (m, w), (dv/dx, dv/dy) and dv/dz row pairs, packed
// two real outputs per complex row, inverse x DFT, scaled outputs.
template <int H, int V>
__global__ void __launch_bounds__(kSxNT)
    k_sx_inverse(SpectralArgs a, const float2* __restrict__ gM, const float2* __restrict__ gW,
                 const float2* __restrict__ gDx, const float2* __restrict__ gDy,
                 const float2* __restrict__ gB, float* __restrict__ m_out,
                 float* __restrict__ w_out, float* __restrict__ G, const float2* __restrict__ twg) {
    constexpr int RB = kSxRows, NT = kSxNT, KXP = kxp<H>(), RP = rowp<H>();
    constexpr int NZ = RB + RB + RB / 2;       // packed rows: (m, w), (dx, dy), dz pairs
    extern __shared__ float2 sm[];
    float2* Z = sm;                            // [NZ][RP]
    float2* tw = Z + NZ * RP;
    const int z = blockIdx.y, y0 = blockIdx.x * RB;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    // pack straight from the half spectra in global memory (consecutive lanes
    // read consecutive, or mirrored consecutive, kx), so that the block holds
    // only the packed rows and more blocks share an SM
    auto row = [z, y0](const float2* f, int r) {
        return f + (static_cast<size_t>(z) * H + y0 + r) * KXP;
    };
    for (int q = threadIdx.x; q < NZ * H; q += NT) {
        const int zr = q / H, kx = q % H;
        float2 val;
        if (zr < RB) {
            val = a.do_mw ? pack_two<H>(row(gM, zr), row(gW, zr), kx) : make_float2(0.f, 0.f);
        } else if (zr < 2 * RB) {
            const int r = zr - RB;
            val = pack_two<H>(row(gDx, r), row(gDy, r), kx);
        } else {
            const int p = zr - 2 * RB;
            val = pack_two<H>(row(gB, 2 * p), row(gB, 2 * p + 1), kx);
        }
        Z[zr * RP + kx] = val;
    }
    __syncthreads();
    fft_axis<H, V, NZ, 1, RP, NT, +1>(Z, tw);
    const float sc = a.out_scale, sxy = a.out_scale_xy;
    for (int q = threadIdx.x; q < RB * H; q += NT) {
        const int r = q / H, x = q % H;
        const size_t node = (static_cast<size_t>(z) * H + y0 + r) * H + x;
        const float2 mw = Z[r * RP + x];
        const float2 dxy = Z[(RB + r) * RP + x];
        const float2 bz = Z[(2 * RB + (r >> 1)) * RP + x];
        if (a.do_mw) {
            m_out[node] = mw.x * sc;
            w_out[node] = mw.y * sc;
            *reinterpret_cast<float4*>(G + 4 * node) =
                make_float4(dxy.x * sxy, dxy.y * sxy, ((r & 1) ? bz.y : bz.x) * sc, mw.y * sc);
        } else {
            *reinterpret_cast<float2*>(G + 4 * node) = make_float2(dxy.x * sxy, dxy.y * sxy);
            G[4 * node + 2] = ((r & 1) ? bz.y : bz.x) * sc;
        }
    }
}

// Passes of the per-axis pipeline, grouped like the fused ones:
// 0 forward (x, y), 1 z, 2 inverse (y, x).
template <int H, int V>
cudaError_t spectral_pass_split_v(sipf_ctx* c, const SpectralArgs& a, int pass) {
    constexpr int KXP = kxp<H>(), RB = kSxRows, KB = kSxCols, RP = rowp<H>();
    const size_t smx1 = (3 * static_cast<size_t>(RB) * KXP + H) * sizeof(float2);
    // the column passes: one buffer, or two where V becomes i k_x V and i k_y V
    const size_t smy1 = (static_cast<size_t>(H) * (KB + 1) + H) * sizeof(float2);
    const size_t smy2 = (2 * static_cast<size_t>(H) * (KB + 1) + H) * sizeof(float2);
    const size_t smz = (static_cast<size_t>(H) * zcols<H>() + H) * sizeof(float2);
    const size_t smx2 = (static_cast<size_t>(2 * RB + RB / 2) * RP + H) * sizeof(float2);
    static int configured_device = -1;
    if (configured_device != c->device) {
        cudaFuncSetAttribute(k_sx_forward<H, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smx1));
        cudaFuncSetAttribute(k_sx_columns<H, -1, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smy1));
        cudaFuncSetAttribute(k_sx_columns<H, +1, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smy2));
        cudaFuncSetAttribute(k_z_multiply<H, 1, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smz));
        cudaFuncSetAttribute(k_sx_inverse<H, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smx2));
        configured_device = c->device;
    }
    const dim3 gy((KXP + KB - 1) / KB, H, 3);
    if (pass == 0) {
        k_sx_forward<H, V><<<dim3(H / RB, H), kSxNT, smx1, c->stream>>>(
            a, c->v, c->m, c->w, reinterpret_cast<unsigned long long*>(c->acc), c->v, c->specM,
            c->specW, c->specV, c->twiddle, c->voff, c->dsc + c->cur, c->us);
        k_sx_columns<H, -1, V><<<gy, kSxNT, smy1, c->stream>>>(a, c->specM, c->specW, c->specV,
                                                              nullptr, nullptr, c->twiddle, 0);
    } else if (pass == 1) {
        SpecBatch<1> one;
        one.run[0] = spec_run(c, a);
        k_z_multiply<H, 1, V><<<dim3(H, 4, (KXP + zcols<H>() - 1) / zcols<H>()), Cfg<H>::NT2, smz,
                               c->stream>>>(one);
    } else {
        // inverse y: M, W and B in place; V (or its filtered copy) -> i k_x V, i k_y V
        k_sx_columns<H, +1, V><<<gy, kSxNT, smy2, c->stream>>>(
            a, c->specM, c->specW, a.filter ? c->specA : c->specV, c->specDx, c->specDy, c->twiddle,
            0);
        k_sx_columns<H, +1, V><<<dim3(gy.x, H, 1), kSxNT, smy1, c->stream>>>(
            a, c->specB, c->specB, c->specB, nullptr, nullptr, c->twiddle, 1);
        k_sx_inverse<H, V><<<dim3(H / RB, H), kSxNT, smx2, c->stream>>>(
            a, c->specM, c->specW, c->specDx, c->specDy, c->specB, c->m, c->w, c->G, c->twiddle);
    }
    return cudaGetLastError();
}

// Shared memory of the fused passes.
template <int H> struct FusedSmem {
    static constexpr size_t fwd = (static_cast<size_t>(H) * rowp<H>() + H * kxp<H>() + H) * sizeof(float2);
    static constexpr size_t z = (static_cast<size_t>(H) * zcols<H>() + H) * sizeof(float2);
    static constexpr size_t inv = (3 * static_cast<size_t>(H) * kxs<H>() + H) * sizeof(float2);
};

template <int H, int NB, int V>
void configure_fused(int device) {
    static int configured_device = -1;   // attributes are set once per process and device
    if (configured_device == device) return;
    cudaFuncSetAttribute(k_forward_xy<H, NB, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(FusedSmem<H>::fwd));
    cudaFuncSetAttribute(k_z_multiply<H, NB, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(FusedSmem<H>::z));
    cudaFuncSetAttribute(k_inverse_xy<H, NB, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(FusedSmem<H>::inv));
    configured_device = device;
}

// One fused pass over a batch of nb runs of grid size H.
template <int H, int NB, int V>
cudaError_t fused_pass(const SpecBatch<NB>& batch, int nb, int pass, int device, cudaStream_t s) {
    configure_fused<H, NB, V>(device);
    constexpr int KXP = kxp<H>();
    if (pass == 0) {
        return launch_pdl(k_forward_xy<H, NB, V>, dim3(H, nb), dim3(Cfg<H>::NT1),
                          FusedSmem<H>::fwd, s, batch);
    } else if (pass == 1) {
        const int kt = (KXP + zcols<H>() - 1) / zcols<H>();
        return launch_pdl(k_z_multiply<H, NB, V>, dim3(H, 4, NB == 1 ? kt : nb),
                          dim3(Cfg<H>::NT2), FusedSmem<H>::z, s, batch);
    } else {
        return launch_pdl(k_inverse_xy<H, NB, V>, dim3(2 * H, 1, nb), dim3(Cfg<H>::NT3),
                          FusedSmem<H>::inv, s, batch);
    }
}

// One fused pass over n runs (n = 1: the batch-of-one instantiation).
template <int H, int V>
cudaError_t fused_runs(const SpecRun* runs, int n, int pass, int device, cudaStream_t s) {
    if (n == 1) {
        SpecBatch<1> one;
        one.run[0] = runs[0];
        return fused_pass<H, 1, V>(one, 1, pass, device, s);
    }
    SpecBatch<kMaxBatch> batch;
    for (int i = 0; i < n; ++i) batch.run[i] = runs[i];
    return fused_pass<H, kMaxBatch, V>(batch, n, pass, device, s);
}

}  // namespace
}  // namespace sipf
