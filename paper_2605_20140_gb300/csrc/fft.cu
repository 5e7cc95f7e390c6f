// Grid side of the SIPF-W step on sm_103a: the explicit reaction R_tau, the
// spectral diffusion solve D_tau and the spectral gradient of v (paper
// Eq. g_hat_phy, Eq. k_q_update with the implicit multipliers of Sec. 4,
// Eq. gradv), as three passes over the grid with a hand-written FFT:
//
//  1. per z-plane: read v, m, w and the integer deposit accumulator, form
//     m* = m + tau u, w* = w + tau (gamma v - eta(u) w), v^n = v/(1 + alpha tau m),
//     store v^n, and transform m*, w*, v^n along x and y in shared memory
//     (m* + i w* as one complex plane; v^n as pairs of rows).  Writes three
//     half spectra [z][ky][kx], kx <= H/2.
//  2. per (ky, field) slab: forward FFT along z, multiply by
//     1/(1 + tau beta + tau Dm |k|^2) (m), 1/(1 + tau + tau Dw |k|^2) (w), or
//     i k_z (v -> B), inverse FFT along z; in place for m and w.
//  3. per (z-plane, group): inverse FFT along y and a packed complex inverse
//     along x: (m, w), (i k_x V, i k_y V) -> (dv/dx, dv/dy), and B in row
//     pairs -> dv/dz.  Writes m^n, w^n and grad v^n, scaled by 1/H^3.
//
// The FFT is a Stockham radix-R formulation (natural order in and out): each
// stage loads R strided elements per butterfly into registers, applies the
// stage twiddles from a table exp(-2 pi i j / H), does an R-point DFT in
// registers and writes the results in place after a block barrier.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sipf_internal.cuh"

namespace sipf {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// exp(-2 pi i t / 16) for t < 8.
__device__ __forceinline__ float2 root16(int t) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
    switch (t) {
        case 0: return make_float2(1.f, 0.f);
        case 1: return make_float2(c1, -s1);
        case 2: return make_float2(r2, -r2);
        case 3: return make_float2(s1, -c1);
        case 4: return make_float2(0.f, -1.f);
        case 5: return make_float2(-s1, -c1);
        case 6: return make_float2(-r2, -r2);
        default: return make_float2(-c1, -s1);
    }
}

template <int R>
__host__ __device__ constexpr int bitrev(int i) {
    return R == 1 ? 0 : ((i & 1) * (R / 2) + bitrev<(R > 1 ? R / 2 : 1)>(i >> 1));
}

// Bit-reversal permutation of a register array, resolved at compile time.
template <int R, int I>
struct BitRevSwap {
    static __device__ __forceinline__ void run(float2 (&v)[R]) {
        constexpr int J = bitrev<R>(I);
        if constexpr (J > I) {
            const float2 t = v[I];
            v[I] = v[J];
            v[J] = t;
        }
        BitRevSwap<R, I + 1>::run(v);
    }
};
template <int R>
struct BitRevSwap<R, R> {
    static __device__ __forceinline__ void run(float2 (&)[R]) {}
};

// One radix-2 level of the in-register DFT: butterflies of span LEN/2.
template <int R, int LEN, int SIGN>
struct DftLevel {
    static __device__ __forceinline__ void run(float2 (&v)[R]) {
#pragma unroll
        for (int i = 0; i < R; i += LEN) {
#pragma unroll
            for (int k = 0; k < LEN / 2; ++k) {
                constexpr int step = 16 / LEN;
                const int t = k * step;
                float2 b = v[i + k + LEN / 2];
                if (t == 4) {
                    b = SIGN < 0 ? make_float2(b.y, -b.x) : make_float2(-b.y, b.x);
                } else if (t != 0) {
                    float2 wv = root16(t);
                    if (SIGN > 0) wv.y = -wv.y;
                    b = cmul(b, wv);
                }
                const float2 a = v[i + k];
                v[i + k] = cadd(a, b);
                v[i + k + LEN / 2] = csub(a, b);
            }
        }
        if constexpr (2 * LEN <= R) DftLevel<R, 2 * LEN, SIGN>::run(v);
    }
};

// In-register R-point DFT (R = 2, 4, 8, 16), sign -1 forward, +1 inverse:
// bit-reversal permutation, then log2 R radix-2 levels (decimation in time).
template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    BitRevSwap<R, 0>::run(v);
    DftLevel<R, 2, SIGN>::run(v);
}

// One Stockham stage of radix R after NS points have been combined.
// Transform t, element j lives at buf[t * TS + j * ES].
template <int L, int R, int NS, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void stage(float2* buf, const float2* tw) {
    constexpr int NB = NTRANS * (L / R);
    constexpr int BPT = (NB + NT - 1) / NT;
    float2 v[BPT][R];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < NB) {
            const int t = (ES == 1) ? b / (L / R) : b % NTRANS;
            const int j = (ES == 1) ? b % (L / R) : b / NTRANS;
            const int k = j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 x = buf[t * TS + (j + r * (L / R)) * ES];
                if (NS > 1 && r > 0) {
                    float2 wv = tw[r * k * (L / (NS * R))];
                    if (SIGN > 0) wv.y = -wv.y;
                    x = cmul(x, wv);
                }
                v[i][r] = x;
            }
            dft<R, SIGN>(v[i]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < NB) {
            const int t = (ES == 1) ? b / (L / R) : b % NTRANS;
            const int j = (ES == 1) ? b % (L / R) : b / NTRANS;
            const int k = j % NS;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[t * TS + (base + r * NS) * ES] = v[i][r];
        }
    }
    __syncthreads();
}

template <int L> struct Radix;
template <> struct Radix<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Radix<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Radix<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Radix<128> { static constexpr int R1 = 16, R2 = 8; };

// Batched length-L FFT along one axis of a shared-memory array.
template <int L, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void fft_axis(float2* buf, const float2* tw) {
    constexpr int R1 = Radix<L>::R1, R2 = Radix<L>::R2;
    static_assert(R1 * R2 == L, "radix plan");
    stage<L, R1, 1, NTRANS, ES, TS, NT, SIGN>(buf, tw);
    stage<L, R2, R1, NTRANS, ES, TS, NT, SIGN>(buf, tw);
}

template <int H> struct Cfg;
template <> struct Cfg<16> { static constexpr int NT = 256; };
template <> struct Cfg<32> { static constexpr int NT = 256; };
template <> struct Cfg<64> { static constexpr int NT = 512; };
template <> struct Cfg<128> { static constexpr int NT = 512; };

template <int H> constexpr int kxp() { return H / 2 + 2; }

__device__ __forceinline__ int signed_mode(int k, int H) { return k < H / 2 ? k : k - H; }

// ---------------------------------------------------------------- pass 1
template <int H>
__global__ void __launch_bounds__(Cfg<H>::NT)
    k_forward_xy(SpectralArgs a, const float* v, const float* __restrict__ m,
                 const float* __restrict__ w, unsigned long long* __restrict__ acc,
                 float* v_out, float2* __restrict__ gM, float2* __restrict__ gW,
                 float2* __restrict__ gV, const float2* __restrict__ twg,
                 const float* __restrict__ voff) {
    constexpr int NT = Cfg<H>::NT, KXP = kxp<H>(), HK = H / 2 + 1;
    extern __shared__ float2 sm[];
    float2* Z = sm;               // [H][H]: m* + i w*
    float2* Vb = Z + H * H;       // [H][KXP]: v^n as pairs of rows, then half rows
    float2* tw = Vb + H * KXP;    // [H]
    const int z = blockIdx.x;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    const size_t plane = static_cast<size_t>(z) * H * H;
    const float c0 = *voff;   // the v spectrum only feeds derivatives: remove a constant
    for (int idx = threadIdx.x; idx < H * H; idx += NT) {
        const int y = idx / H, x = idx % H;
        const size_t node = plane + idx;
        const float vv = v[node], mm = m[node], ww = w[node];
        const long long q = static_cast<long long>(acc[node]);
        acc[node] = 0ull;
        const float u = __ll2float_rn(q) * a.react_scale;
        float ms = mm, ws = ww;
        if (a.do_mw) {
            // R_tau: explicit Euler of S = (-alpha m v; u; gamma v - eta(u) w)
            const float eta = 2.0f * u / (1.0f + u);
            ms = mm + a.tau * u;
            ws = ww + a.tau * (a.gamma * vv - eta * ww);
        }
        const float vn = (a.v_update == SIPF_V_IMPLICIT) ? vv / (1.0f + a.alpha * a.tau * mm)
                                                          : vv * (1.0f - a.alpha * a.tau * mm);
        if (a.write_v) v_out[node] = vn;
        Z[idx] = make_float2(ms, ws);
        reinterpret_cast<float*>(Vb + (y >> 1) * 2 * KXP)[2 * x + (y & 1)] = vn - c0;
    }
    __syncthreads();
    if (a.do_mw) fft_axis<H, H, 1, H, NT, -1>(Z, tw);
    fft_axis<H, H / 2, 1, 2 * KXP, NT, -1>(Vb, tw);
    {
        // split each transformed row pair z = x1 + i x2 into X1, X2 (kx <= H/2)
        constexpr int NS = (H / 2) * HK, SPT = (NS + NT - 1) / NT;
        float2 x1[SPT], x2[SPT];
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NS) {
                const int p = idx / HK, k = idx % HK;
                const float2 zp = Vb[p * 2 * KXP + k];
                const float2 zm = Vb[p * 2 * KXP + ((H - k) & (H - 1))];
                x1[s] = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
                x2[s] = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NS) {
                const int p = idx / HK, k = idx % HK;
                Vb[(2 * p) * KXP + k] = x1[s];
                Vb[(2 * p + 1) * KXP + k] = x2[s];
            }
        }
        __syncthreads();
    }
    if (a.do_mw) fft_axis<H, H, H, 1, NT, -1>(Z, tw);
    fft_axis<H, HK, KXP, 1, NT, -1>(Vb, tw);
    // write half spectra; M, W separated from the 2D spectrum of m* + i w*
    for (int idx = threadIdx.x; idx < H * HK; idx += NT) {
        const int ky = idx / HK, kx = idx % HK;
        const size_t o = (static_cast<size_t>(z) * H + ky) * KXP + kx;
        if (a.do_mw) {
            const float2 zk = Z[ky * H + kx];
            const float2 zc = Z[((H - ky) & (H - 1)) * H + ((H - kx) & (H - 1))];
            gM[o] = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
            gW[o] = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
        }
        gV[o] = Vb[ky * KXP + kx];
    }
}

// ---------------------------------------------------------------- pass 2
template <int H>
__global__ void __launch_bounds__(Cfg<H>::NT)
    k_z_multiply(SpectralArgs a, float2* __restrict__ gM, float2* __restrict__ gW,
                 const float2* __restrict__ gV, float2* __restrict__ gB, float2* __restrict__ gA,
                 const float2* __restrict__ twg, float* __restrict__ voff) {
    constexpr int NT = Cfg<H>::NT, KXP = kxp<H>(), HK = H / 2 + 1;
    extern __shared__ float2 sm[];
    float2* buf = sm;             // [H (z)][HK (kx)]
    float2* tw = buf + H * HK;
    const int ky = blockIdx.x, field = blockIdx.y;   // 0 m, 1 w, 2 v -> i k_z V, 3 v -> filtered V
    if (field < 2 && !a.do_mw) return;
    if (field == 3 && !a.filter) return;
    const float2* src = field == 0 ? gM : field == 1 ? gW : gV;
    float2* dst = field == 0 ? gM : field == 1 ? gW : field == 2 ? gB : gA;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    for (int idx = threadIdx.x; idx < H * HK; idx += NT) {
        const int zz = idx / HK, kx = idx % HK;
        buf[idx] = src[(static_cast<size_t>(zz) * H + ky) * KXP + kx];
    }
    __syncthreads();
    fft_axis<H, HK, HK, 1, NT, -1>(buf, tw);
    if (field == 2 && ky == 0 && threadIdx.x == 0) {
        // DC of (v^n - c0): move the offset to the mean of v^n for the next step
        *voff = *voff + buf[0].x * a.out_scale;
    }
    const int qy = signed_mode(ky, H);
    for (int idx = threadIdx.x; idx < H * HK; idx += NT) {
        const int kz = idx / HK, qx = idx % HK;
        const int qz = signed_mode(kz, H);
        const float q2 = static_cast<float>(qx * qx + qy * qy + qz * qz);
        float f = 1.0f;
        float2 val = buf[idx];
        if (field == 2) {
            const float kz_phys = (qz == -H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(qz);
            val = make_float2(-kz_phys * val.y, kz_phys * val.x);
        } else if (field < 2) {
            const float c = field == 0 ? a.m_c : a.w_c;
            f = a.diffusion == SIPF_DIFFUSION_IMPLICIT ? 1.0f / (1.0f + c * q2) : expf(-c * q2);
        }
        if (a.filter) f *= expf(-a.inv_H0sq_2pi2 * q2);
        val = make_float2(f * val.x, f * val.y);
        if (field < 2) {
            // times r0 = hi + lo: the float32 rounding of r0 itself is compensated
            const float hi = field == 0 ? a.m_r0_hi : a.w_r0_hi;
            const float lo = field == 0 ? a.m_r0_lo : a.w_r0_lo;
            val = make_float2(fmaf(val.x, lo, val.x * hi), fmaf(val.y, lo, val.y * hi));
        }
        buf[idx] = val;
    }
    __syncthreads();
    fft_axis<H, HK, HK, 1, NT, +1>(buf, tw);
    for (int idx = threadIdx.x; idx < H * HK; idx += NT) {
        const int zz = idx / HK, kx = idx % HK;
        dst[(static_cast<size_t>(zz) * H + ky) * KXP + kx] = buf[idx];
    }
}

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

template <int H>
__global__ void __launch_bounds__(Cfg<H>::NT)
    k_inverse_xy(SpectralArgs a, const float2* __restrict__ gM, const float2* __restrict__ gW,
                 const float2* __restrict__ gV, const float2* __restrict__ gB,
                 float* __restrict__ m_out, float* __restrict__ w_out, float* __restrict__ gx_out,
                 float* __restrict__ gy_out, float* __restrict__ gz_out,
                 const float2* __restrict__ twg) {
    constexpr int NT = Cfg<H>::NT, KXP = kxp<H>(), HK = H / 2 + 1;
    extern __shared__ float2 sm[];
    float2* B0 = sm;              // [H][KXP]
    float2* B1 = B0 + H * KXP;    // [H][KXP]
    float2* Z = sm;               // [H][H] packed rows (aliases B0/B1)
    float2* tw = B1 + H * KXP;
    const int z = blockIdx.x, group = blockIdx.y;   // 0 (m, w), 1 (dv/dx, dv/dy), 2 dv/dz
    if (group == 0 && !a.do_mw) return;
    for (int i = threadIdx.x; i < H; i += NT) tw[i] = twg[i];
    const size_t pbase = static_cast<size_t>(z) * H * KXP;
    for (int idx = threadIdx.x; idx < H * HK; idx += NT) {
        const int ky = idx / HK, kx = idx % HK;
        const size_t o = pbase + static_cast<size_t>(ky) * KXP + kx;
        if (group == 0) {
            B0[ky * KXP + kx] = gM[o];
            B1[ky * KXP + kx] = gW[o];
        } else if (group == 1) {
            const float2 val = gV[o];
            const float kxp_ = (kx == H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(kx);
            const int qy = signed_mode(ky, H);
            const float kyp = (qy == -H / 2) ? 0.0f : a.two_pi_over_L * static_cast<float>(qy);
            B0[ky * KXP + kx] = make_float2(-kxp_ * val.y, kxp_ * val.x);
            B1[ky * KXP + kx] = make_float2(-kyp * val.y, kyp * val.x);
        } else {
            B0[ky * KXP + kx] = gB[o];
        }
    }
    __syncthreads();
    fft_axis<H, HK, KXP, 1, NT, +1>(B0, tw);
    if (group < 2) {
        fft_axis<H, HK, KXP, 1, NT, +1>(B1, tw);
        constexpr int NE = H * H, EPT = (NE + NT - 1) / NT;
        float2 r[EPT];
#pragma unroll
        for (int s = 0; s < EPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NE) {
                const int y = idx / H, kx = idx % H;
                r[s] = pack_two<H>(B0 + y * KXP, B1 + y * KXP, kx);
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < EPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NE) Z[idx] = r[s];
        }
        __syncthreads();
        fft_axis<H, H, 1, H, NT, +1>(Z, tw);
        float* o1 = group == 0 ? m_out : gx_out;
        float* o2 = group == 0 ? w_out : gy_out;
        const float sc = group == 0 ? a.out_scale : a.out_scale_xy;
        const size_t plane = static_cast<size_t>(z) * H * H;
        for (int idx = threadIdx.x; idx < H * H; idx += NT) {
            const float2 val = Z[idx];
            o1[plane + idx] = val.x * sc;
            o2[plane + idx] = val.y * sc;
        }
    } else {
        constexpr int NE = (H / 2) * H, EPT = (NE + NT - 1) / NT;
        float2 r[EPT];
#pragma unroll
        for (int s = 0; s < EPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NE) {
                const int p = idx / H, kx = idx % H;
                r[s] = pack_two<H>(B0 + (2 * p) * KXP, B0 + (2 * p + 1) * KXP, kx);
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < EPT; ++s) {
            const int idx = threadIdx.x + s * NT;
            if (idx < NE) Z[idx] = r[s];
        }
        __syncthreads();
        fft_axis<H, H / 2, 1, H, NT, +1>(Z, tw);
        const size_t plane = static_cast<size_t>(z) * H * H;
        for (int idx = threadIdx.x; idx < NE; idx += NT) {
            const int p = idx / H, x = idx % H;
            const float2 val = Z[idx];
            gz_out[plane + (2 * p) * H + x] = val.x * a.out_scale;
            gz_out[plane + (2 * p + 1) * H + x] = val.y * a.out_scale;
        }
    }
}

template <int H>
cudaError_t spectral_step(sipf_ctx* c, const SpectralArgs& a) {
    constexpr int NT = Cfg<H>::NT, KXP = kxp<H>(), HK = H / 2 + 1;
    const size_t sm1 = (static_cast<size_t>(H) * H + H * KXP + H) * sizeof(float2);
    const size_t sm2 = (static_cast<size_t>(H) * HK + H) * sizeof(float2);
    const size_t sm3 = (2 * static_cast<size_t>(H) * KXP + H) * sizeof(float2);
    static bool configured = false;   // per process; attributes are per function
    if (!configured) {
        cudaFuncSetAttribute(k_forward_xy<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm1));
        cudaFuncSetAttribute(k_z_multiply<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm2));
        cudaFuncSetAttribute(k_inverse_xy<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm3));
        configured = true;
    }
    k_forward_xy<H><<<H, NT, sm1, c->stream>>>(
        a, c->v, c->m, c->w, reinterpret_cast<unsigned long long*>(c->acc), c->v, c->specM,
        c->specW, c->specV, c->twiddle, c->voff);
    k_z_multiply<H><<<dim3(H, 4), NT, sm2, c->stream>>>(a, c->specM, c->specW, c->specV,
                                                         c->specB, c->specA, c->twiddle, c->voff);
    k_inverse_xy<H><<<dim3(H, 3), NT, sm3, c->stream>>>(
        a, c->specM, c->specW, a.filter ? c->specA : c->specV, c->specB, c->m, c->w, c->gx,
        c->gy, c->gz, c->twiddle);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spectral_step(sipf_ctx* c, const SpectralArgs& a) {
    switch (c->H) {
        case 16: return spectral_step<16>(c, a);
        case 32: return spectral_step<32>(c, a);
        case 64: return spectral_step<64>(c, a);
        case 128: return spectral_step<128>(c, a);
        default: return cudaErrorInvalidValue;
    }
}

void fill_twiddles(int H, float2* out) {
    for (int j = 0; j < H; ++j) {
        const double ang = -2.0 * M_PI * static_cast<double>(j) / static_cast<double>(H);
        out[j] = make_float2(static_cast<float>(cos(ang)), static_cast<float>(sin(ang)));
    }
}

}  // namespace sipf
