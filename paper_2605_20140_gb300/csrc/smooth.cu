// Gaussian smoothing K_sigma * u_bar of the deposited density, the
// regularised source of the m equation (paper Eq. m_reg), K_sigma the density
// of N(0, sigma I_3).  Its Fourier multiplier exp(-sigma |k|^2 / 2) is a
// product over the three axes, so the 3D smoothing is one periodic 1D
// smoothing per axis.  Along an axis two real lines share one complex
// transform: the multiplier is real and even in k, so it keeps the real and
// imaginary parts apart.  Each line pair: forward DFT, times
// g_j = exp(-sigma k_j^2 / 2) / H, inverse DFT (Stockham stages in shared
// memory, as in the spectral passes).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fft_stages.cuh"
#include "sipf_internal.cuh"

namespace sipf {
namespace {

using namespace fftk;

constexpr int kPairsX = 4;   // row pairs per block along x
constexpr int kPairsYZ = 16; // column pairs per block along y and z

// Threads of a block transforming P line pairs of length H: at most two
// first-stage butterflies per thread, 64 to 512 threads.
template <int H, int P>
constexpr int smooth_threads() {
    constexpr int nb = P * (H / Radix<H>::R1);
    constexpr int t = ((nb + 1) / 2 + 31) / 32 * 32;
    return t < 64 ? 64 : (t > 512 ? 512 : t);
}

// u_bar = acc * u_scale (the scale of the current step, from device memory).
__global__ void k_acc_to_u(const unsigned long long* __restrict__ acc, int n,
                           const StepScalars* __restrict__ sc, float* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long q = acc[i];
    const float f = fmaf(__int2float_rn(static_cast<int>(static_cast<unsigned>(q >> 32))),
                         4294967296.0f, __uint2float_rn(static_cast<unsigned>(q)));
    u[i] = f * sc->u_scale;
}

// Along x: block (pair group, z) smooths rows y = 2p, 2p + 1 of plane z for
// kPairsX consecutive pairs p (H/2 is a multiple of kPairsX).
template <int H>
__global__ void __launch_bounds__(smooth_threads<H, kPairsX>())
    k_smooth_x(float* __restrict__ u, const float* __restrict__ g, const float2* __restrict__ twg) {
    constexpr int P = kPairsX, RP = H + 1, kSmNT = smooth_threads<H, kPairsX>();
    __shared__ float2 buf[P * RP];
    __shared__ float2 tw[H];
    __shared__ float gs[H];
    for (int i = threadIdx.x; i < H; i += kSmNT) {
        tw[i] = twg[i];
        gs[i] = g[i];
    }
    const int z = blockIdx.y, p0 = blockIdx.x * P;
    float* plane = u + static_cast<size_t>(z) * H * H;
    for (int q = threadIdx.x; q < P * H; q += kSmNT) {
        const int t = q / H, x = q % H, y = 2 * (p0 + t);
        buf[t * RP + x] = make_float2(plane[y * H + x], plane[(y + 1) * H + x]);
    }
    __syncthreads();
    fft_axis<H, 0, P, 1, RP, kSmNT, -1>(buf, tw);
    for (int q = threadIdx.x; q < P * H; q += kSmNT) {
        const int t = q / H, j = q % H;
        const float2 e = buf[t * RP + j];
        buf[t * RP + j] = make_float2(e.x * gs[j], e.y * gs[j]);
    }
    __syncthreads();
    fft_axis<H, 0, P, 1, RP, kSmNT, +1>(buf, tw);
    for (int q = threadIdx.x; q < P * H; q += kSmNT) {
        const int t = q / H, x = q % H, y = 2 * (p0 + t);
        const float2 e = buf[t * RP + x];
        plane[y * H + x] = e.x;
        plane[(y + 1) * H + x] = e.y;
    }
}

// Along y (AXIS 1, block (pair group, z)) or z (AXIS 2, block (pair group, y)):
// columns x = x0 + 2t, x0 + 2t + 1 for kPairsYZ pairs t, every element j of
// the axis; a column pair is one float2 in memory.
template <int H, int AXIS>
__global__ void __launch_bounds__(smooth_threads<H, kPairsYZ>())
    k_smooth_yz(float* __restrict__ u, const float* __restrict__ g, const float2* __restrict__ twg) {
    constexpr int P = kPairsYZ, PP = P + 1, kSmNT = smooth_threads<H, kPairsYZ>();
    extern __shared__ float2 sm[];
    float2* buf = sm;                                   // [H (j)][PP (t)]
    float2* tw = buf + H * PP;                          // [H]
    float* gs = reinterpret_cast<float*>(tw + H);       // [H]
    for (int i = threadIdx.x; i < H; i += kSmNT) {
        tw[i] = twg[i];
        gs[i] = g[i];
    }
    const int c = blockIdx.y, x0 = blockIdx.x * 2 * P;
    auto at = [c](int j, int x) -> size_t {
        return AXIS == 1 ? (static_cast<size_t>(c) * H + j) * H + x
                         : (static_cast<size_t>(j) * H + c) * H + x;
    };
    for (int q = threadIdx.x; q < H * P; q += kSmNT) {
        const int j = q / P, t = q % P, x = x0 + 2 * t;
        buf[j * PP + t] = x < H ? *reinterpret_cast<const float2*>(u + at(j, x))
                                : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_axis<H, 0, P, PP, 1, kSmNT, -1>(buf, tw);
    for (int q = threadIdx.x; q < H * P; q += kSmNT) {
        const int j = q / P, t = q % P;
        const float2 e = buf[j * PP + t];
        buf[j * PP + t] = make_float2(e.x * gs[j], e.y * gs[j]);
    }
    __syncthreads();
    fft_axis<H, 0, P, PP, 1, kSmNT, +1>(buf, tw);
    for (int q = threadIdx.x; q < H * P; q += kSmNT) {
        const int j = q / P, t = q % P, x = x0 + 2 * t;
        if (x < H) *reinterpret_cast<float2*>(u + at(j, x)) = buf[j * PP + t];
    }
}

template <int H>
cudaError_t smooth_h(sipf_ctx* c, float* us, cudaStream_t s) {
    constexpr int PP = kPairsYZ + 1;
    const size_t smyz = (static_cast<size_t>(H) * PP + H) * sizeof(float2) + H * sizeof(float);
    static int configured_device = -1;
    if (configured_device != c->device) {
        cudaFuncSetAttribute(k_smooth_yz<H, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smyz));
        cudaFuncSetAttribute(k_smooth_yz<H, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smyz));
        configured_device = c->device;
    }
    const int n = H * H * H;
    k_acc_to_u<<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(c->acc),
                                                n, c->dsc + c->cur, us);
    constexpr int NTX = smooth_threads<H, kPairsX>(), NTYZ = smooth_threads<H, kPairsYZ>();
    k_smooth_x<H><<<dim3(H / 2 / kPairsX, H), NTX, 0, s>>>(us, c->ksig, c->twiddle);
    const dim3 gyz((H / 2 + kPairsYZ - 1) / kPairsYZ, H);
    k_smooth_yz<H, 1><<<gyz, NTYZ, smyz, s>>>(us, c->ksig, c->twiddle);
    k_smooth_yz<H, 2><<<gyz, NTYZ, smyz, s>>>(us, c->ksig, c->twiddle);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_smooth(sipf_ctx* c, float* us, cudaStream_t s) {
    switch (c->H) {
        case 8: return smooth_h<8>(c, us, s);
        case 16: return smooth_h<16>(c, us, s);
        case 24: return smooth_h<24>(c, us, s);
        case 32: return smooth_h<32>(c, us, s);
        case 48: return smooth_h<48>(c, us, s);
        case 64: return smooth_h<64>(c, us, s);
        case 72: return smooth_h<72>(c, us, s);
        case 96: return smooth_h<96>(c, us, s);
        case 128: return smooth_h<128>(c, us, s);
        case 144: return smooth_h<144>(c, us, s);
        case 192: return smooth_h<192>(c, us, s);
        case 216: return smooth_h<216>(c, us, s);
        case 256: return smooth_h<256>(c, us, s);
        case 288: return smooth_h<288>(c, us, s);
        case 384: return smooth_h<384>(c, us, s);
        case 432: return smooth_h<432>(c, us, s);
        case 512: return smooth_h<512>(c, us, s);
        default: return cudaErrorInvalidValue;
    }
}

// g_j = exp(-sigma (2 pi q_j / L)^2 / 2) / H, q_j the signed mode of index j.
void fill_smoothing(int H, double L, double sigma, float* out) {
    for (int j = 0; j < H; ++j) {
        const double q = j < H / 2 ? j : j - H;
        const double k = 2.0 * M_PI * q / L;
        out[j] = static_cast<float>(exp(-0.5 * sigma * k * k) / H);
    }
}

}  // namespace sipf
