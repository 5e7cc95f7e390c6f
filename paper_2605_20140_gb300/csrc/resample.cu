// Residual resampling of the particle store (paper Alg. 4) on the device.
//
// Input: the compacted particles of one buffer (slots [0, N)), whose ids must
// be a permutation of 0..N-1; the loop over p of Alg. 4 runs in id order.
// The integer decisions are taken on fixed-point weights so that they do not
// depend on summation order:
//   E   binary exponent of the largest mass (a_max < 2^E),
//   Q_p = floor(a_p 2^(31-E)) < 2^31,  S = sum_p Q_p < 2^62,
//   k_p = floor(Q_p N / S)            (the integer part floor(a_p / a_0)),
//   R_p = Q_p N - k_p S               (the residual a_p - k_p a_0, times N 2^(31-E)).
// N_stoch = N - sum k_p particles are drawn independently with probability
// R_p / C, C = sum R_p = S N_stoch: draw j takes U = b0 + 2^32 b1 of the
// Philox4x32-10 block of counter (n, 1, j, 0), the target
// t = floor(U C / 2^64) (exact, 128-bit) and the first p whose inclusive
// prefix sum of R exceeds t.  The new list is the k_p copies of each p in
// order of p, then the draws in order; new ids are the list positions and
// every new particle has the mass a_0 = T 2^(E-62) / N, T = sum_p
// round(a_p 2^(62-E)) (exact 128-bit total, rounded once).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "sipf_internal.cuh"

namespace sipf {
namespace {

using u128 = unsigned __int128;

constexpr int kRsNT = 256;
constexpr int kRsIPT = 8;                 // elements per thread of the scans
constexpr int kRsTile = kRsNT * kRsIPT;   // elements per scan block
constexpr int kRsBlocks = 304;            // blocks of the fixed-grid reductions

// Flags of k_rs_index.
constexpr int kRsBadId = 1;       // id >= N
constexpr int kRsDupId = 2;       // id seen twice
constexpr int kRsNonfinite = 4;   // mass NaN or infinite

struct RsScratch {
    int* perm;                // [N] compacted slot of id p
    double* a;                // [N] mass of id p
    int* seen;                // [N] id occurrence counts
    int* k;                   // [N] k_p, then its inclusive prefix sum
    u128* r;                  // [N] R_p, then its inclusive prefix sum
    int* tile_k;              // [tiles] scan block sums
    u128* tile_r;
    unsigned long long* part; // [kRsBlocks * 3] S, T lo, T hi per block
    unsigned long long* ext;  // [2] largest, smallest mass (bits)
    int* flag;
};

size_t align256(size_t b) { return (b + 255) & ~size_t{255}; }

size_t scratch_bytes(int64_t N, int tiles) {
    return align256(N * sizeof(int)) * 3 + align256(N * sizeof(double)) +
           align256(N * sizeof(u128)) + align256(tiles * sizeof(int)) +
           align256(tiles * sizeof(u128)) + align256(kRsBlocks * 3 * sizeof(unsigned long long)) +
           align256(2 * sizeof(unsigned long long)) + align256(sizeof(int));
}

RsScratch carve(void* base, int64_t N, int tiles) {
    char* p = static_cast<char*>(base);
    auto take = [&p](size_t bytes) {
        char* q = p;
        p += align256(bytes);
        return q;
    };
    RsScratch s;
    s.perm = reinterpret_cast<int*>(take(N * sizeof(int)));
    s.seen = reinterpret_cast<int*>(take(N * sizeof(int)));
    s.k = reinterpret_cast<int*>(take(N * sizeof(int)));
    s.a = reinterpret_cast<double*>(take(N * sizeof(double)));
    s.r = reinterpret_cast<u128*>(take(N * sizeof(u128)));
    s.tile_k = reinterpret_cast<int*>(take(tiles * sizeof(int)));
    s.tile_r = reinterpret_cast<u128*>(take(tiles * sizeof(u128)));
    s.part = reinterpret_cast<unsigned long long*>(take(kRsBlocks * 3 * sizeof(unsigned long long)));
    s.ext = reinterpret_cast<unsigned long long*>(take(2 * sizeof(unsigned long long)));
    s.flag = reinterpret_cast<int*>(take(sizeof(int)));
    return s;
}

__global__ void k_rs_init(unsigned long long* ext, int* flag) {
    ext[0] = 0ull;
    ext[1] = ~0ull;
    *flag = 0;
}

// Ids checked, masses a_p = exp(dl + logref) (as exported) in id order,
// largest and smallest mass (non-negative doubles order like their bits).
__global__ void k_rs_index(const uint32_t* __restrict__ id, const double* __restrict__ dl,
                           double logref, int N, int* __restrict__ perm, double* __restrict__ a,
                           int* seen, unsigned long long* ext, int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t q = id[i];
    if (q >= static_cast<uint32_t>(N)) {
        atomicOr(flag, kRsBadId);
        return;
    }
    if (atomicAdd(seen + q, 1) != 0) {
        atomicOr(flag, kRsDupId);
        return;
    }
    perm[q] = i;
    const double v = exp(dl[i] + logref);
    a[q] = v;
    if (!(v >= 0.0) || isinf(v)) {
        atomicOr(flag, kRsNonfinite);
        return;
    }
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    atomicMax(ext, b);
    atomicMin(ext + 1, b);
}

__device__ __forceinline__ uint64_t q_weight(double a, int E) {
    return static_cast<uint64_t>(floor(scalbn(a, 31 - E)));
}

// Per-block partial sums of Q_p (S) and of round(a_p 2^(62-E)) (T, 128-bit).
__global__ void __launch_bounds__(kRsNT)
    k_rs_sums(const double* __restrict__ a, int N, int E, unsigned long long* __restrict__ part) {
    __shared__ uint64_t ss[kRsNT];
    __shared__ u128 st[kRsNT];
    uint64_t S = 0;
    u128 T = 0;
    for (int p = blockIdx.x * kRsNT + threadIdx.x; p < N; p += kRsBlocks * kRsNT) {
        S += q_weight(a[p], E);
        T += __double2ull_rn(scalbn(a[p], 62 - E));
    }
    ss[threadIdx.x] = S;
    st[threadIdx.x] = T;
    __syncthreads();
    for (int h = kRsNT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            ss[threadIdx.x] += ss[threadIdx.x + h];
            st[threadIdx.x] += st[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = ss[0];
        part[3 * blockIdx.x + 1] = static_cast<uint64_t>(st[0]);
        part[3 * blockIdx.x + 2] = static_cast<uint64_t>(st[0] >> 64);
    }
}

// k_p = floor(Q_p N / S), R_p = Q_p N - k_p S.
__global__ void k_rs_split(const double* __restrict__ a, int N, int E, uint64_t S,
                           int* __restrict__ k, u128* __restrict__ r) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const uint64_t qn = q_weight(a[p], E) * static_cast<uint64_t>(N);
    const uint64_t kp = qn / S;
    k[p] = static_cast<int>(kp);
    r[p] = qn - kp * S;
}

// ---- inclusive prefix sums (three passes: block sums, their scan, apply)
template <class T>
__device__ T block_inclusive_scan(T v, T* sm) {
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kRsNT; off <<= 1) {
        const T t = threadIdx.x >= off ? sm[threadIdx.x - off] : T(0);
        __syncthreads();
        sm[threadIdx.x] += t;
        __syncthreads();
    }
    const T out = sm[threadIdx.x];
    __syncthreads();
    return out;
}

template <class T>
__global__ void __launch_bounds__(kRsNT) k_rs_tile_sums(const T* __restrict__ in, int n,
                                                        T* __restrict__ tile_sum) {
    __shared__ T sm[kRsNT];
    const int base = blockIdx.x * kRsTile + threadIdx.x * kRsIPT;
    T s = 0;
    for (int e = 0; e < kRsIPT; ++e)
        if (base + e < n) s += in[base + e];
    const T incl = block_inclusive_scan<T>(s, sm);
    if (threadIdx.x == kRsNT - 1) tile_sum[blockIdx.x] = incl;
}

template <class T>
__global__ void __launch_bounds__(kRsNT) k_rs_scan_tile_sums(T* tile_sum, int tiles) {
    __shared__ T sm[kRsNT];
    __shared__ T total;
    T carry = 0;
    for (int b0 = 0; b0 < tiles; b0 += kRsNT) {
        const int j = b0 + threadIdx.x;
        const T v = j < tiles ? tile_sum[j] : T(0);
        const T incl = block_inclusive_scan<T>(v, sm);
        if (j < tiles) tile_sum[j] = carry + incl - v;   // exclusive offset of block j
        if (threadIdx.x == kRsNT - 1) total = incl;
        __syncthreads();
        carry += total;
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kRsNT) k_rs_scan_apply(T* data, int n, const T* __restrict__ tile_off) {
    __shared__ T sm[kRsNT];
    const int base = blockIdx.x * kRsTile + threadIdx.x * kRsIPT;
    T v[kRsIPT];
    T s = 0;
    for (int e = 0; e < kRsIPT; ++e) {
        v[e] = base + e < n ? data[base + e] : T(0);
        s += v[e];
    }
    T run = block_inclusive_scan<T>(s, sm) - s + tile_off[blockIdx.x];
    for (int e = 0; e < kRsIPT; ++e) {
        run += v[e];
        if (base + e < n) data[base + e] = run;
    }
}

// Copies of the parents into the new list: slot j < Kdet is a deterministic
// copy (first p with prefix k > j), slot j >= Kdet is draw j - Kdet.
__global__ void k_rs_emit(int N, int Kdet, const int* __restrict__ kpre,
                          const u128* __restrict__ rpre, uint64_t C_lo, uint64_t C_hi, uint32_t n,
                          uint32_t k0, uint32_t k1, const int* __restrict__ perm,
                          const float* __restrict__ sx, const float* __restrict__ sy,
                          const float* __restrict__ sz, float* __restrict__ ox,
                          float* __restrict__ oy, float* __restrict__ oz, double* __restrict__ odl,
                          uint32_t* __restrict__ oid, double dl_new) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int lo = 0, hi = N - 1;   // the answer is in [lo, hi]: kpre[N-1] = Kdet > j, rpre[N-1] = C > t
    if (j < Kdet) {
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (kpre[mid] > j) hi = mid;
            else lo = mid + 1;
        }
    } else {
        const uint4 b = philox4x32_10(make_uint4(n, 1u, static_cast<uint32_t>(j - Kdet), 0u), k0, k1);
        const uint64_t U = static_cast<uint64_t>(b.x) | (static_cast<uint64_t>(b.y) << 32);
        const u128 t = static_cast<u128>(U) * C_hi + __umul64hi(U, C_lo);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rpre[mid] > t) hi = mid;
            else lo = mid + 1;
        }
    }
    const int src = perm[lo];
    ox[j] = sx[src];
    oy[j] = sy[src];
    oz[j] = sz[src];
    odl[j] = dl_new;
    oid[j] = static_cast<uint32_t>(j);
}

template <class T>
cudaError_t inclusive_scan(T* data, int n, T* tile_sum, cudaStream_t s) {
    const int tiles = (n + kRsTile - 1) / kRsTile;
    k_rs_tile_sums<T><<<tiles, kRsNT, 0, s>>>(data, n, tile_sum);
    k_rs_scan_tile_sums<T><<<1, kRsNT, 0, s>>>(tile_sum, tiles);
    k_rs_scan_apply<T><<<tiles, kRsNT, 0, s>>>(data, n, tile_sum);
    return cudaGetLastError();
}

}  // namespace

// Device part of sipf_resample: particles of buffer `src` ([0, N), compacted)
// -> unbinned buffer `dst` ([0, N)).  *done = 0 when the largest/smallest
// mass ratio is <= ratio (ratio > 0) and nothing was written.
int resample_device(sipf_ctx* c, int src, int dst, double ratio, int* done, std::string* err) {
    *done = 0;
    const int N = static_cast<int>(c->N);
    const int tiles = (N + kRsTile - 1) / kRsTile;
    const size_t need = scratch_bytes(N, tiles);
    if (c->rs_bytes < need) {
        if (c->rs_scratch) cudaFree(c->rs_scratch);
        c->rs_scratch = nullptr;
        c->rs_bytes = 0;
        if (cudaMalloc(&c->rs_scratch, need) != cudaSuccess) {
            cudaGetLastError();
            *err = "resampling scratch";
            return SIPF_ENOMEM;
        }
        c->rs_bytes = need;
    }
    const RsScratch s = carve(c->rs_scratch, N, tiles);
    cudaStream_t st = c->stream;
    const int nb = (N + 255) / 256;
    cudaError_t e = cudaMemsetAsync(s.seen, 0, sizeof(int) * N, st);
    if (e == cudaSuccess) {
        k_rs_init<<<1, 1, 0, st>>>(s.ext, s.flag);
        k_rs_index<<<nb, 256, 0, st>>>(c->id[src], c->dl[src], c->logref, N, s.perm, s.a, s.seen,
                                       s.ext, s.flag);
        e = cudaGetLastError();
    }
    unsigned long long ext[2] = {0, 0};
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ext, s.ext, sizeof(ext), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, s.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return SIPF_ECUDA;
    }
    if (flag & (kRsBadId | kRsDupId)) {
        *err = "resampling needs particle ids that are a permutation of 0..N-1";
        return SIPF_EINVAL;
    }
    if (flag & kRsNonfinite) {
        *err = "a particle mass is not finite";
        return SIPF_ENONFINITE;
    }
    double amax, amin;
    memcpy(&amax, &ext[0], sizeof(double));
    memcpy(&amin, &ext[1], sizeof(double));
    if (!(amax > 0.0)) {
        *err = "resampling needs a positive total mass";
        return SIPF_EINVAL;
    }
    if (ratio > 0.0 && amax <= ratio * amin) return SIPF_OK;
    int E = 0;
    frexp(amax, &E);

    // S and T (exact), then a_0
    std::vector<unsigned long long> part(3 * kRsBlocks);
    k_rs_sums<<<kRsBlocks, kRsNT, 0, st>>>(s.a, N, E, s.part);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(part.data(), s.part, part.size() * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return SIPF_ECUDA;
    }
    uint64_t S = 0;
    u128 T = 0;
    for (int b = 0; b < kRsBlocks; ++b) {
        S += part[3 * b];
        T += (static_cast<u128>(part[3 * b + 2]) << 64) | part[3 * b + 1];
    }
    const double a0 = ldexp(static_cast<double>(T), -(62 - E)) / static_cast<double>(N);

    // k_p, R_p and their prefix sums
    k_rs_split<<<nb, 256, 0, st>>>(s.a, N, E, S, s.k, s.r);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = inclusive_scan<int>(s.k, N, s.tile_k, st);
    if (e == cudaSuccess) e = inclusive_scan<u128>(s.r, N, s.tile_r, st);
    int Kdet = 0;
    u128 C = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&Kdet, s.k + (N - 1), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&C, s.r + (N - 1), sizeof(u128), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return SIPF_ECUDA;
    }
    if (Kdet < 0 || Kdet > N || C != static_cast<u128>(S) * static_cast<u128>(N - Kdet)) {
        *err = "resampling: inconsistent integer parts";
        return SIPF_EINTERNAL;
    }
    const double dl_new = log(a0) - c->logref;
    k_rs_emit<<<nb, 256, 0, st>>>(N, Kdet, s.k, s.r, static_cast<uint64_t>(C),
                                  static_cast<uint64_t>(C >> 64), static_cast<uint32_t>(c->step),
                                  static_cast<uint32_t>(c->p.seed),
                                  static_cast<uint32_t>(c->p.seed >> 32), s.perm, c->sx[src],
                                  c->sy[src], c->sz[src], c->sx[dst], c->sy[dst], c->sz[dst],
                                  c->dl[dst], c->id[dst], dl_new);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return SIPF_ECUDA;
    }
    *done = 1;
    return SIPF_OK;
}

}  // namespace sipf
