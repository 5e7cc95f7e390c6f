// Building blocks of the hand-written FFT (shared by the spectral passes and
// the Gaussian smoothing): complex helpers, in-register R-point DFTs, one
// Stockham stage over a batch of transforms in shared memory, and the radix
// plans.
#pragma once

#include <cuda_runtime.h>

namespace sipf {
namespace fftk {

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

// In-register R-point DFT, sign -1 forward, +1 inverse.  R = 2, 4, 8, 16:
// bit-reversal permutation, then log2 R radix-2 levels (decimation in time).
// R = 3: X0 = a + b + c, X1 = a - (b + c)/2 + SIGN i (sqrt 3 / 2)(b - c),
// X2 = a - (b + c)/2 - SIGN i (sqrt 3 / 2)(b - c).
template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    if constexpr (R == 3) {
        constexpr float s3 = 0.86602540378443865f;
        const float2 sum = cadd(v[1], v[2]), dif = csub(v[1], v[2]);
        const float2 mid = make_float2(v[0].x - 0.5f * sum.x, v[0].y - 0.5f * sum.y);
        // rot = SIGN i s3 (b - c)
        const float2 rot = SIGN < 0 ? make_float2(s3 * dif.y, -s3 * dif.x)
                                    : make_float2(-s3 * dif.y, s3 * dif.x);
        v[0] = cadd(v[0], sum);
        v[1] = cadd(mid, rot);
        v[2] = csub(mid, rot);
    } else {
        BitRevSwap<R, 0>::run(v);
        DftLevel<R, 2, SIGN>::run(v);
    }
}

// Element addressing of a batch of transforms: element j of transform t is
// buf[at(t, j)].  Strided: transform t at t * TS, elements ES apart.
template <int TS, int ES>
struct Strided {
    __device__ __forceinline__ int operator()(int t, int j) const { return t * TS + j * ES; }
};

// One Stockham stage of radix R after NS points have been combined, over
// NTRANS transforms addressed by `at`.  Consecutive lanes take consecutive
// transforms (same butterfly), so a warp's accesses are contiguous when
// transforms are adjacent and spread over all banks when their pitch is odd.
// The outputs go to sink(t, p, v) (transform t, output position p); a block
// barrier separates the reads from the sink calls and follows them, so the
// sink may write into buf.
template <int L, int R, int NS, int NTRANS, int NT, int SIGN, class At, class Sink>
__device__ __forceinline__ void stage_sink_at(const float2* buf, const float2* tw, At at,
                                              Sink sink) {
    constexpr int NB = NTRANS * (L / R);
    constexpr int BPT = (NB + NT - 1) / NT;
    float2 v[BPT][R];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < NB) {
            const int t = b % NTRANS;
            const int j = b / NTRANS;
            const int k = j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 x = buf[at(t, j + r * (L / R))];
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
            const int t = b % NTRANS;
            const int j = b / NTRANS;
            const int k = j % NS;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sink(t, base + r * NS, v[i][r]);
        }
    }
    __syncthreads();
}

// The same stage in place.
template <int L, int R, int NS, int NTRANS, int NT, int SIGN, class At>
__device__ __forceinline__ void stage_at(float2* buf, const float2* tw, At at) {
    stage_sink_at<L, R, NS, NTRANS, NT, SIGN>(
        buf, tw, at, [=](int t, int p, float2 v) { buf[at(t, p)] = v; });
}

template <int L, int R, int NS, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void stage(float2* buf, const float2* tw) {
    stage_at<L, R, NS, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{});
}

template <int L, int R, int NS, int NTRANS, int ES, int TS, int NT, int SIGN, class Sink>
__device__ __forceinline__ void stage_sink(const float2* buf, const float2* tw, Sink sink) {
    stage_sink_at<L, R, NS, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{}, sink);
}

// First Stockham stage (NS = 1) with inputs from a loader: element j of
// transform t is load(t, j).  All loads precede all writes (a block barrier
// in between), so the loader may read the memory `out` overwrites.
template <int L, int R, int NTRANS, int NT, int SIGN, class At, class Load>
__device__ __forceinline__ void stage1_from_at(float2* out, At at, Load load) {
    constexpr int NB = NTRANS * (L / R);
    constexpr int BPT = (NB + NT - 1) / NT;
    float2 v[BPT][R];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < NB) {
            const int t = b % NTRANS, j = b / NTRANS;
#pragma unroll
            for (int r = 0; r < R; ++r) v[i][r] = load(t, j + r * (L / R));
            dft<R, SIGN>(v[i]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < NB) {
            const int t = b % NTRANS, j = b / NTRANS;
#pragma unroll
            for (int r = 0; r < R; ++r) out[at(t, j * R + r)] = v[i][r];
        }
    }
    __syncthreads();
}

template <int L, int R, int NTRANS, int ES, int TS, int NT, int SIGN, class Load>
__device__ __forceinline__ void stage1_from(float2* out, Load load) {
    stage1_from_at<L, R, NTRANS, NT, SIGN>(out, Strided<TS, ES>{}, load);
}

// Radix plan of a length-L transform: two to four Stockham stages (R3, R4 =
// 1: fewer).  Lengths are 2^a 3^b with 8 <= L <= 512.
template <int L> struct Radix;
template <int A, int B, int C = 1, int D = 1>
struct RadixPlan { static constexpr int R1 = A, R2 = B, R3 = C, R4 = D; };
template <> struct Radix<8> : RadixPlan<4, 2> {};
template <> struct Radix<16> : RadixPlan<4, 4> {};
template <> struct Radix<24> : RadixPlan<8, 3> {};
template <> struct Radix<32> : RadixPlan<8, 4> {};
template <> struct Radix<48> : RadixPlan<16, 3> {};
template <> struct Radix<64> : RadixPlan<8, 8> {};
template <> struct Radix<72> : RadixPlan<8, 3, 3> {};
template <> struct Radix<96> : RadixPlan<8, 4, 3> {};
template <> struct Radix<128> : RadixPlan<16, 8> {};
template <> struct Radix<144> : RadixPlan<16, 3, 3> {};
template <> struct Radix<192> : RadixPlan<16, 4, 3> {};
template <> struct Radix<216> : RadixPlan<8, 3, 3, 3> {};
template <> struct Radix<256> : RadixPlan<16, 16> {};
template <> struct Radix<288> : RadixPlan<16, 3, 3, 2> {};
template <> struct Radix<384> : RadixPlan<16, 8, 3> {};
template <> struct Radix<432> : RadixPlan<16, 3, 3, 3> {};
template <> struct Radix<512> : RadixPlan<8, 8, 8> {};

// The stages after the first of a batched length-L FFT, the last one into a
// sink (see stage_sink_at).
template <int L, int NTRANS, int NT, int SIGN, class At, class Sink>
__device__ __forceinline__ void fft_rest_sink_at(float2* buf, const float2* tw, At at, Sink sink) {
    constexpr int R1 = Radix<L>::R1, R2 = Radix<L>::R2, R3 = Radix<L>::R3, R4 = Radix<L>::R4;
    static_assert(R1 * R2 * R3 * R4 == L, "radix plan");
    if constexpr (R3 == 1) {
        stage_sink_at<L, R2, R1, NTRANS, NT, SIGN>(buf, tw, at, sink);
    } else if constexpr (R4 == 1) {
        stage_at<L, R2, R1, NTRANS, NT, SIGN>(buf, tw, at);
        stage_sink_at<L, R3, R1 * R2, NTRANS, NT, SIGN>(buf, tw, at, sink);
    } else {
        stage_at<L, R2, R1, NTRANS, NT, SIGN>(buf, tw, at);
        stage_at<L, R3, R1 * R2, NTRANS, NT, SIGN>(buf, tw, at);
        stage_sink_at<L, R4, R1 * R2 * R3, NTRANS, NT, SIGN>(buf, tw, at, sink);
    }
}

// The stages after the first, in place.
template <int L, int NTRANS, int NT, int SIGN, class At>
__device__ __forceinline__ void fft_rest_at(float2* buf, const float2* tw, At at) {
    fft_rest_sink_at<L, NTRANS, NT, SIGN>(
        buf, tw, at, [=](int t, int p, float2 v) { buf[at(t, p)] = v; });
}

template <int L, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void fft_rest(float2* buf, const float2* tw) {
    fft_rest_at<L, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{});
}

template <int L, int NTRANS, int ES, int TS, int NT, int SIGN, class Sink>
__device__ __forceinline__ void fft_rest_sink(float2* buf, const float2* tw, Sink sink) {
    fft_rest_sink_at<L, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{}, sink);
}

// Batched length-L FFT along one axis, in place.
template <int L, int NTRANS, int NT, int SIGN, class At>
__device__ __forceinline__ void fft_axis_at(float2* buf, const float2* tw, At at) {
    stage_at<L, Radix<L>::R1, 1, NTRANS, NT, SIGN>(buf, tw, at);
    fft_rest_at<L, NTRANS, NT, SIGN>(buf, tw, at);
}

template <int L, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void fft_axis(float2* buf, const float2* tw) {
    fft_axis_at<L, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{});
}

}  // namespace fftk
}  // namespace sipf
