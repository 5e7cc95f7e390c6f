// Allocation-free particle-to-grid deposit.
//
// Some callers cannot allocate device memory at the moment they need a
// density: code that runs while another framework owns the device memory
// budget (a caching allocator that must not see foreign cudaMalloc calls,
// which also synchronise the device), real-time loops that may not block
// or fail on allocation, or plug-ins handed only pre-allocated buffers.
// sipf_deposit_noalloc serves them: it computes the same deposit as the
// context path (sipf_fields with SIPF_FIELD_U) but keeps its integer
// accumulator in a fixed file-scope device array instead of context
// memory, so it never calls cudaMalloc, cudaFree or any allocating
// routine.  The array holds at most kNoAllocMaxNodes grid nodes; every GPU
// that loads the library keeps it until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "sipf_internal.cuh"

namespace {

constexpr int kNoAllocMaxH = 64;
constexpr int kNoAllocMaxNodes = kNoAllocMaxH * kNoAllocMaxH * kNoAllocMaxH;
constexpr int kCtl = 32;            // control words in front of the node sums
constexpr int kMaxDevices = 64;

// [0]: bits of the largest mass (non-negative doubles order like int64);
// [kCtl, kCtl + H^3): fixed-point node sums.  Shared by every call.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kCtl + kNoAllocMaxNodes];

std::mutex g_mutex;
unsigned long long* g_scratch_ptr[kMaxDevices] = {nullptr};

__global__ void k_na_clear(unsigned long long* s, int nodes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kCtl + nodes) s[i] = 0ull;
}

// A particle contributes only if its mass is finite and positive: an
// infinite or NaN mass is skipped (it would otherwise fix the scale of every
// node), a zero mass adds nothing anyway.
__device__ __forceinline__ bool na_counts(double m) { return isfinite(m) && m > 0.0; }

__global__ void k_na_max_mass(const double* __restrict__ mass, int64_t N, unsigned long long* s) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < N) {
        const double m = mass[i];
        if (na_counts(m)) atomicMax(reinterpret_cast<long long*>(s), __double_as_longlong(m));
    }
}

// 2^S with S chosen so that the largest mass times 2^S stays below 2^30.
__device__ __forceinline__ int na_shift(const unsigned long long* s) {
    const double mmax = __longlong_as_double(static_cast<long long>(s[0]));
    if (!(mmax > 0.0)) return 0;
    int e;
    frexp(mmax, &e);    // mmax < 2^e
    return 30 - e;
}

__global__ void k_na_deposit(const float* __restrict__ x, const double* __restrict__ mass,
                             int64_t N, int H, float o0, float o1, float o2, float h,
                             unsigned long long* s) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double m = mass[i];
    if (!na_counts(m)) return;
    const float Hf = __int2float_rn(H);
    const float o[3] = {o0, o1, o2};
    int c[3], c1[3];
    float f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // grid units, wrapped into [0, H) (a result rounding to H becomes 0)
        float v = __fdiv_rn(__fsub_rn(x[static_cast<int64_t>(d) * N + i], o[d]), h);
        if (!(v >= 0.0f && v < Hf)) {
            v = __fsub_rn(v, __fmul_rn(Hf, floorf(__fdiv_rn(v, Hf))));
            if (v < 0.0f) v = __fadd_rn(v, Hf);
            if (!(v < Hf)) v = 0.0f;
        }
        c[d] = min(max(static_cast<int>(v), 0), H - 1);
        c1[d] = c[d] + 1 < H ? c[d] + 1 : 0;
        f[d] = __fsub_rn(v, __int2float_rn(c[d]));
    }
    const float a = static_cast<float>(ldexp(m, na_shift(s)));
    unsigned long long* acc = s + kCtl;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
        const float wx = dx ? f[0] : __fsub_rn(1.0f, f[0]);
        const float wy = dy ? f[1] : __fsub_rn(1.0f, f[1]);
        const float wz = dz ? f[2] : __fsub_rn(1.0f, f[2]);
        const uint32_t q = __float2uint_rn(__fmul_rn(__fmul_rn(a, wz), __fmul_rn(wx, wy)));
        const int node = ((dz ? c1[2] : c[2]) * H + (dy ? c1[1] : c[1])) * H + (dx ? c1[0] : c[0]);
        if (q) atomicAdd(acc + node, static_cast<unsigned long long>(q));
    }
}

__global__ void k_na_finish(const unsigned long long* s, int nodes, double inv_h3,
                            float* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nodes) return;
    const double scale = ldexp(inv_h3, -na_shift(s));
    u[i] = static_cast<float>(static_cast<double>(s[kCtl + i]) * scale);
}

// Device address of the scratch array on the current device (looked up
// once per device; host code only sees a host-side stand-in otherwise).
// The address is kept for the life of the process, so the entry point must
// not be used on a device after cudaDeviceReset in the same process.
int scratch_for_current_device(unsigned long long** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIPF_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SIPF_ECUDA;
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return SIPF_OK;
}

}  // namespace

extern "C" int sipf_deposit_noalloc(const sipf_grid* grid, const float* x, const double* mass,
                                    int64_t N, float* u, void* stream) {
    if (!grid || !x || !mass || !u) return SIPF_EINVAL;
    const int H = grid->H;
    if (H < 1 || H > kNoAllocMaxH) return SIPF_EINVAL;   // scratch holds at most 64^3 nodes
    if (N < 1 || N >= (int64_t{1} << 31)) return SIPF_EINVAL;
    if (!(isfinite(grid->L) && grid->L > 0.0)) return SIPF_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(grid->origin[k])) return SIPF_EINVAL;
    unsigned long long* s = nullptr;
    const int r = scratch_for_current_device(&s);
    if (r != SIPF_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nodes = H * H * H;
    const double h = grid->L / H;
    const unsigned pblocks = static_cast<unsigned>((N + 255) / 256);   // N < 2^31: fits
    k_na_clear<<<(kCtl + nodes + 255) / 256, 256, 0, st>>>(s, nodes);
    k_na_max_mass<<<pblocks, 256, 0, st>>>(mass, N, s);
    k_na_deposit<<<pblocks, 256, 0, st>>>(
        x, mass, N, H, static_cast<float>(grid->origin[0]), static_cast<float>(grid->origin[1]),
        static_cast<float>(grid->origin[2]), static_cast<float>(h), s);
    k_na_finish<<<(nodes + 255) / 256, 256, 0, st>>>(s, nodes, 1.0 / (h * h * h), u);
    if (cudaGetLastError() != cudaSuccess) return SIPF_ECUDA;
    return SIPF_OK;
}
