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

template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]);

// a^-1 mod m for coprime a, m (small, at compile time).
__host__ __device__ constexpr int modinv(int a, int m) {
    int x = 1;
    while ((a * x) % m != 1) ++x;
    return x;
}

// Prime-factor (Good-Thomas) DFT of length N = N1 N2 with gcd(N1, N2) = 1:
// the input index n = (N2 n1 + N1 n2) mod N and the output index
// k = (N2 (N2^-1 mod N1) k1 + N1 (N1^-1 mod N2) k2) mod N turn it into N2
// DFTs of length N1 followed by N1 DFTs of length N2, with no twiddle
// factors in between.
template <int N1, int N2, int SIGN>
__device__ __forceinline__ void dft_pfa(float2 (&v)[N1 * N2]) {
    constexpr int N = N1 * N2;
    constexpr int C1 = N2 * modinv(N2, N1), C2 = N1 * modinv(N1, N2);
    float2 y[N1][N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
        float2 t[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) t[n1] = v[(N2 * n1 + N1 * n2) % N];
        dft<N1, SIGN>(t);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) y[k1][n2] = t[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        float2 t[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) t[n2] = y[k1][n2];
        dft<N2, SIGN>(t);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[(C1 * k1 + C2 * k2) % N] = t[k2];
    }
}

// In-register R-point DFT, sign -1 forward, +1 inverse.  R = 2, 4, 8, 16:
// bit-reversal permutation, then log2 R radix-2 levels (decimation in time).
// R = 3: X0 = a + b + c, X1 = a - (b + c)/2 + SIGN i (sqrt 3 / 2)(b - c),
// X2 = a - (b + c)/2 - SIGN i (sqrt 3 / 2)(b - c).  R = 6 = 2 x 3 and
// R = 12 = 3 x 4: the prime-factor form above.
template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    if constexpr (R == 6) {
        dft_pfa<2, 3, SIGN>(v);
    } else if constexpr (R == 12) {
        dft_pfa<3, 4, SIGN>(v);
    } else if constexpr (R == 3) {
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

// Radix plans of a length-L transform: two to four Stockham stages (R3, R4 =
// 1: fewer).  Lengths are 2^a 3^b with 8 <= L <= 512.  Plan V = 0 and an
// alternative V = 1 (fewer stages through the radix-6 and radix-12 DFTs, or
// the stage order reversed); which one runs is a tuning choice per grid size.
template <int L, int V = 0> struct Radix;
template <int A, int B, int C = 1, int D = 1>
struct RadixPlan { static constexpr int R1 = A, R2 = B, R3 = C, R4 = D; };
template <> struct Radix<8, 0> : RadixPlan<4, 2> {};
template <> struct Radix<16, 0> : RadixPlan<4, 4> {};
template <> struct Radix<24, 0> : RadixPlan<8, 3> {};
template <> struct Radix<32, 0> : RadixPlan<8, 4> {};
template <> struct Radix<48, 0> : RadixPlan<16, 3> {};
template <> struct Radix<64, 0> : RadixPlan<8, 8> {};
template <> struct Radix<72, 0> : RadixPlan<8, 3, 3> {};
template <> struct Radix<96, 0> : RadixPlan<8, 4, 3> {};
template <> struct Radix<128, 0> : RadixPlan<16, 8> {};
template <> struct Radix<144, 0> : RadixPlan<16, 3, 3> {};
template <> struct Radix<192, 0> : RadixPlan<16, 4, 3> {};
template <> struct Radix<216, 0> : RadixPlan<8, 3, 3, 3> {};
template <> struct Radix<256, 0> : RadixPlan<16, 16> {};
template <> struct Radix<288, 0> : RadixPlan<16, 3, 3, 2> {};
template <> struct Radix<384, 0> : RadixPlan<16, 8, 3> {};
template <> struct Radix<432, 0> : RadixPlan<16, 3, 3, 3> {};
template <> struct Radix<512, 0> : RadixPlan<8, 8, 8> {};
template <> struct Radix<8, 1> : RadixPlan<2, 4> {};
template <> struct Radix<16, 1> : RadixPlan<8, 2> {};
template <> struct Radix<24, 1> : RadixPlan<12, 2> {};
template <> struct Radix<32, 1> : RadixPlan<4, 8> {};
template <> struct Radix<48, 1> : RadixPlan<12, 4> {};
template <> struct Radix<64, 1> : RadixPlan<16, 4> {};
template <> struct Radix<72, 1> : RadixPlan<12, 6> {};
template <> struct Radix<96, 1> : RadixPlan<12, 8> {};
template <> struct Radix<128, 1> : RadixPlan<8, 16> {};
template <> struct Radix<144, 1> : RadixPlan<12, 12> {};
template <> struct Radix<192, 1> : RadixPlan<16, 12> {};
template <> struct Radix<216, 1> : RadixPlan<6, 6, 6> {};
template <> struct Radix<256, 1> : RadixPlan<8, 8, 4> {};
template <> struct Radix<288, 1> : RadixPlan<8, 6, 6> {};
template <> struct Radix<384, 1> : RadixPlan<8, 8, 6> {};
template <> struct Radix<432, 1> : RadixPlan<12, 6, 6> {};
template <> struct Radix<512, 1> : RadixPlan<16, 8, 4> {};

// The stages after the first of a batched length-L FFT, the last one into a
// sink (see stage_sink_at).
template <int L, int V, int NTRANS, int NT, int SIGN, class At, class Sink>
__device__ __forceinline__ void fft_rest_sink_at(float2* buf, const float2* tw, At at, Sink sink) {
    using P = Radix<L, V>;
    constexpr int R1 = P::R1, R2 = P::R2, R3 = P::R3, R4 = P::R4;
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
template <int L, int V, int NTRANS, int NT, int SIGN, class At>
__device__ __forceinline__ void fft_rest_at(float2* buf, const float2* tw, At at) {
    fft_rest_sink_at<L, V, NTRANS, NT, SIGN>(
        buf, tw, at, [=](int t, int p, float2 v) { buf[at(t, p)] = v; });
}

template <int L, int V, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void fft_rest(float2* buf, const float2* tw) {
    fft_rest_at<L, V, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{});
}

template <int L, int V, int NTRANS, int ES, int TS, int NT, int SIGN, class Sink>
__device__ __forceinline__ void fft_rest_sink(float2* buf, const float2* tw, Sink sink) {
    fft_rest_sink_at<L, V, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{}, sink);
}

// Batched length-L FFT along one axis, in place (radix plan V).
template <int L, int V, int NTRANS, int NT, int SIGN, class At>
__device__ __forceinline__ void fft_axis_at(float2* buf, const float2* tw, At at) {
    stage_at<L, Radix<L, V>::R1, 1, NTRANS, NT, SIGN>(buf, tw, at);
    fft_rest_at<L, V, NTRANS, NT, SIGN>(buf, tw, at);
}

template <int L, int V, int NTRANS, int ES, int TS, int NT, int SIGN>
__device__ __forceinline__ void fft_axis(float2* buf, const float2* tw) {
    fft_axis_at<L, V, NTRANS, NT, SIGN>(buf, tw, Strided<TS, ES>{});
}

// A length-L DFT spread over a group of P lanes of one warp (Q = L / P
// elements per lane, S = Q / P), as the two factors of L = P Q
// (Cooley-Tukey) with one exchange through the group's shared-memory tile:
//  * spatial layout: lane l holds n = l + P m in v[m], m < Q;
//  * spectral layout: lane l holds k = k1 + Q k2 with k1 = S l + s in
//    v[s P + k2], s < S, k2 < P.
// to_spectral: DFT_Q over m, twiddle w_L^(l k1), exchange, DFT_P over l.
// to_spatial reverses it: DFT_P over k2, twiddle w_L^(n1 k1), exchange,
// DFT_Q over k1.  The tile holds P rows of PITCH float2; __syncwarp orders
// the exchange, so no block barrier is involved.
template <int L, int P, int PITCH>
struct WarpFFT {
    static constexpr int Q = L / P, S = Q / P;
    static_assert(Q % P == 0 && PITCH >= Q, "warp FFT shape");

    template <int SIGN>
    static __device__ __forceinline__ float2 twiddle(const float2* tw, int j) {
        float2 w = tw[j];
        if (SIGN > 0) w.y = -w.y;
        return w;
    }

    template <int SIGN>
    static __device__ __forceinline__ void to_spectral(float2 (&v)[Q], int l, float2* ex,
                                                       const float2* tw) {
        dft<Q, SIGN>(v);
#pragma unroll
        for (int k1 = 1; k1 < Q; ++k1) v[k1] = cmul(v[k1], twiddle<SIGN>(tw, l * k1));
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) ex[l * PITCH + k1] = v[k1];
        __syncwarp();
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float2 u[P];
#pragma unroll
            for (int j = 0; j < P; ++j) u[j] = ex[j * PITCH + S * l + s];
            dft<P, SIGN>(u);
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) v[s * P + k2] = u[k2];
        }
    }

    template <int SIGN>
    static __device__ __forceinline__ void to_spatial(float2 (&v)[Q], int l, float2* ex,
                                                      const float2* tw) {
        __syncwarp();
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float2 u[P];
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) u[k2] = v[s * P + k2];
            dft<P, SIGN>(u);
            const int k1 = S * l + s;
            ex[k1] = u[0];
#pragma unroll
            for (int j = 1; j < P; ++j) ex[j * PITCH + k1] = cmul(u[j], twiddle<SIGN>(tw, j * k1));
        }
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) v[k1] = ex[l * PITCH + k1];
        dft<Q, SIGN>(v);
    }
};

}  // namespace fftk
}  // namespace sipf
