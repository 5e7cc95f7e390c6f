// Internal declarations of the SIPF-W CUDA path: context layout, device
// helpers shared by the particle kernels, kernel launch wrappers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/sipf.h"

namespace sipf {

constexpr int kTile = 8;            // cells per tile edge of the tile-major cell key
constexpr int kMaxH = 512;          // largest grid of this build

// Device status bits (ORed into ctx->status by kernels, read by sipf_sync).
constexpr int kStatusNonfinite = 1;   // a pushed position was NaN/inf (reset to 0)
constexpr int kStatusSlot = 2;        // overflow region full, or a bucket/position mismatch
constexpr int kStatusTotal = 4;       // particle counts inconsistent

// Kernel groups of a step, in launch order (tracing).
constexpr int kProfGroups = 4;
constexpr int kProfMaxSteps = 4096;

// ------------------------------------------------------------------ Philox
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with key mixing; the key advances by the Weyl
// constants between rounds.  Each product is one wide multiply.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
    return make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0, static_cast<uint32_t>(p1),
                      static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1, static_cast<uint32_t>(p0));
}

// Programmatic dependent launch.  A kernel launched with launch_pdl may
// begin while the kernel before it in the stream runs its last blocks:
// pdl_wait() returns once that kernel has completed and its writes are
// visible (a kernel reads nothing its predecessor writes before it), and
// pdl_trigger() lets the next kernel's blocks start launching.  Both are
// no-ops in kernels launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... Exp, class... Act>
cudaError_t launch_pdl(void (*kernel)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Act&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    // the legacy default stream (NULL or its explicit handle) keeps ordinary launches
    cfg.numAttrs = (s == nullptr || s == cudaStreamLegacy) ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Act>(args)...);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        c = philox_round(c, k0, k1);
    }
    return c;
}

// The same generator with the ten round keys given (rk[2r], rk[2r+1]).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, rk[2 * r], rk[2 * r + 1]);
    return c;
}

// Per-step scalars of the particle kernels.
struct PushArgs {
    int H;
    float drift;      // chi * tau / h      (grid units per unit grad v)
    float noise;      // sqrt(2 Du tau) / h (grid units per standard normal)
    float tau;
    uint32_t k0, k1;  // Philox key
    uint32_t rk[20];  // Philox round keys (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85), r = 0..9
    int push;         // 0: positions unchanged (pure binning)
};

// Per-step scalars, kept in device memory (one slot per buffer parity) so
// that the kernels of a step read them there rather than as launch
// arguments: the plan kernel of step n writes step n + 1's slot, and a
// captured sequence of steps can be replayed.
struct StepScalars {
    uint32_t n;            // the step being taken (Philox counter word 0), from 1
    int32_t deposit_shift; // S of deposit_scale = 2^S
    double time;           // t_{n-1}
    float deposit_scale;   // 2^S: contribution of a particle to a node is
                           // exp(log a - logref) * weight * 2^S, rounded to an integer
    float u_scale;         // u_bar per accumulator unit: 2^-S exp(logref) / h^3
};

// S for the deposit at time t: one contribution is at most
// max_p a_p / exp(logref) <= maxrel e^t (Lemma mass: a grows by at most
// 1 + tau <= e^tau per step) and must stay below 2^20 after scaling, so the
// sums of one 1024-particle item fit exactly in 32 bits.  Host and device
// evaluate the same expression (an explicit fma), so they agree bit for bit.
__host__ __device__ inline int deposit_shift_at(double log2_maxrel, double t) {
    const double bound = fma(t, 1.4426950408889634, log2_maxrel) + 0.5;
    int S = static_cast<int>(floor(20.0 - bound));
    if (S > 40) S = 40;
    if (S < -60) S = -60;
    return S;
}

__host__ __device__ inline void fill_step_scalars(StepScalars* s, uint32_t n, double t,
                                                  double log2_maxrel, double exp_logref,
                                                  double h3) {
    const int S = deposit_shift_at(log2_maxrel, t);
    s->n = n;
    s->deposit_shift = S;
    s->time = t;
    s->deposit_scale = static_cast<float>(ldexp(1.0, S));
    s->u_scale = static_cast<float>(ldexp(exp_logref, -S) / h3);
}

// A run of particles read by one block of the step kernel: [beg, end) of a
// buffer, all in bucket `tile` (or tile = -1 for the overflow region / an
// unbinned input), written at `out` in the compacted particle order.
struct Item {
    int tile;
    int beg;
    int end;
    int out;
    int tx, ty, tz;   // tile coordinates (0 for tile = -1)
    int pad;
};

// Spectral-step scalars.
struct SpectralArgs {
    float tau;
    float gamma, alpha;
    int v_update;          // SIPF_V_*
    int diffusion;         // SIPF_DIFFUSION_*
    float two_pi_over_L;
    // Per-mode factor of field f in {m, w}: r0_f * g_f(q^2) with
    //   implicit: r0 = 1/(1 + tau R), g = 1/(1 + c q^2), c = tau D (2 pi/L)^2 r0
    //   exp:      r0 = exp(-tau R),   g = exp(-c q^2),   c = tau D (2 pi/L)^2
    // r0 is carried as a float hi + lo pair so that the k = 0 mode (the mean,
    // multiplied by r0 every step) carries no systematic float32 rounding.
    float m_r0_hi, m_r0_lo, m_c;
    float w_r0_hi, w_r0_lo, w_c;
    float inv_H0sq_2pi2;   // 2 pi^2 / H0^2, 0 when the filter is off
    int filter;            // 1 when the low-pass filter is on
    float out_scale;       // 1 / H^3 (fields that went through all three transform pairs)
    float out_scale_xy;    // scale of dv/dx, dv/dy: 1 / H^2 when their spectrum skips the z pair
    int write_v;           // store v^n (0 in the grad-v-only initial transform)
    int do_mw;             // transform m and w (0 in the initial transform)
};

// One run's data for the fused spectral passes (H <= 128).  The passes take
// a batch of runs as a launch parameter: one run for a context's own step,
// up to kMaxBatch runs of one grid size for an ensemble's batched step (the
// run is then a grid dimension of the launch).
struct SpecRun {
    SpectralArgs a;
    const float* v;
    const float* m;
    const float* w;
    unsigned long long* acc;      // deposit accumulator (read and cleared by the forward pass)
    float* v_out;
    float* m_out;
    float* w_out;
    float* G;                     // gather array (dv/dx, dv/dy, dv/dz, w) per node
    float2* specM;
    float2* specW;
    float2* specV;
    float2* specB;
    float2* specA;                // filtered v spectrum (filter on only)
    float2* specDx;               // i k_x V and i k_y V after the inverse y pass
    float2* specDy;               // (per-axis pipelines only)
    const float2* twiddle;
    float* voff;
    const StepScalars* sc;        // scalars of the step (u_bar per accumulator unit)
    const float* us;              // K_sigma * u_bar (sigma > 0 only)
};
constexpr int kMaxBatch = 64;

// One ensemble member as the batched particle kernels see it (device table
// written when the ensemble captures its step graph; both buffer parities).
struct RunDesc {
    int H, ntiles, ovf_base, ovf_cap;
    float drift, noise, tau;            // push of this run's dt (grid units)
    uint32_t k0, k1;                    // Philox key
    float* sx[2];
    float* sy[2];
    float* sz[2];
    double* dl[2];
    uint32_t* id[2];
    int* bstart[2];
    int* cap[2];
    int* cnt[2];
    int* ovf[2];
    Item* items;
    int* n_items;
    unsigned long long* acc;
    const float* G;
    int* status;
    StepScalars* dsc;                   // [2], slot = parity of the source buffer
    double dt, log2_maxrel, exp_logref, h3;
    int slack_div, slack_add;           // bucket capacity count + count/slack_div + slack_add
};
constexpr int kMaxRuns = 256;           // runs of one batched particle launch
template <int NB> struct SpecBatch {
    SpecRun run[NB];
};

}  // namespace sipf

struct sipf_ctx {
    int H = 0;
    double L = 0, h = 0;
    double origin[3] = {0, 0, 0};
    int64_t N = 0;
    sipf_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;         // plan kernel, concurrent with the spectral passes
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join = nullptr;
    int device = 0;
    // tuning choices (sipf_set_tuning): radix plan of the spectral passes,
    // particle-step blocks per SM (0: occupancy limit), bucket slack
    int radix_plan = 0;
    int step_bps = 0;
    int slack_div = 8;
    int slack_add = 32;
    cudaMemPool_t pool = nullptr;        // stream-ordered allocation from this pool (null: cudaMalloc)

    // particle store, ping-pong; positions in grid units, log-mass relative
    // to logref, ids; tile buckets followed by an overflow region of N
    float* sx[2] = {nullptr, nullptr};
    float* sy[2] = {nullptr, nullptr};
    float* sz[2] = {nullptr, nullptr};
    double* dl[2] = {nullptr, nullptr};
    uint32_t* id[2] = {nullptr, nullptr};
    int cur = 0;
    int ntiles = 0;                      // (H/8)^3
    int ovf_base = 0;                    // first slot of the overflow region
    int64_t buf_slots = 0;               // slots per buffer
    size_t dev_bytes = 0;                // device memory allocated by sipf_create
    int* bstart[2] = {nullptr, nullptr}; // bucket layout per buffer
    int* cap[2] = {nullptr, nullptr};
    int* cnt[2] = {nullptr, nullptr};    // arrivals per bucket (incl. overflowed)
    int* ovf[2] = {nullptr, nullptr};    // particles in the overflow region
    sipf::Item* items = nullptr;         // items of the current buffer
    int* n_items = nullptr;
    int* work = nullptr;                 // work counter of the persistent step kernel
    int max_items = 0;
    int step_blocks = 0;

    // per-cell histogram (sipf_cell_start)
    int32_t* count = nullptr;        // H^3
    int32_t* cell_start = nullptr;   // H^3 + 1
    int32_t* scan_tmp = nullptr;

    // grid
    long long* acc = nullptr;        // H^3 fixed-point deposit accumulator, zero between steps
    float* us = nullptr;             // K_sigma * u_bar, the m source (sigma > 0 only)
    float* ksig = nullptr;           // [H] 1D smoothing multiplier exp(-sigma k_j^2 / 2) / H
    float* v = nullptr;
    float* m = nullptr;
    float* w = nullptr;
    float* G = nullptr;              // H^3 float4 (dv/dx, dv/dy, dv/dz, w) for the gather
    float2* specM = nullptr;         // half spectra [z][ky][kx], row pitch kxp
    float2* specW = nullptr;
    float2* specV = nullptr;
    float2* specB = nullptr;
    float2* specA = nullptr;         // filtered v spectrum (filter on only)
    float2* specDx = nullptr;        // i k_x V, i k_y V after the inverse y pass (H > 128 only)
    float2* specDy = nullptr;
    float2* twiddle = nullptr;       // exp(-2 pi i j / H), j < H
    float* voff = nullptr;           // device scalar: offset subtracted from v before its FFT
    int kxp = 0;

    void* rs_scratch = nullptr;      // residual resampling work space (allocated on first use)
    size_t rs_bytes = 0;

    sipf::StepScalars* dsc = nullptr;      // [2] per-step scalars, slot = parity of the source buffer
    double log2_maxrel = 0;          // log2(maxrel), exp(logref), h^3: constants of the scalars
    double exp_logref = 1;
    double h3 = 1;
    struct StepGraph {
        double dt;
        int parity;
        cudaGraphExec_t exec;
    };
    std::vector<StepGraph> graphs;   // captured two-step sequences, by (dt, parity)

    int* status = nullptr;           // device status word
    double* diag_tmp = nullptr;      // diagnostics partials
    double* diag_out = nullptr;      // 8 doubles
    long long* diag_ll = nullptr;    // fixed-point partial sums

    // tracing: CUDA events between the kernel groups of each step
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_events;      // kProfGroups + 1 per recorded step
    int64_t prof_steps = 0;

    int64_t step = 0;
    double time = 0;
    double logref = 0;               // log(M0 / N) of the initial state
    double maxrel = 1;               // max_p a_p(0) / exp(logref)
    float voff_host = 0;             // staging value for voff
    bool state_set = false;
    std::string last_error;
};

namespace sipf {

// ---------------------------------------------------------------- launchers
// particles.cu
int step_grid(sipf_ctx* c);
int item_size();
size_t diag_scratch_doubles();
size_t diag_scratch_ll();
int scan_tiles(int n);
cudaError_t launch_step_kernel(sipf_ctx* c, const PushArgs& a, int do_deposit, int do_move);
// Items of buffer b and, with next_layout, the layout of b ^ 1; with dt > 0
// also the scalars of the next step (slot b ^ 1) from those of slot b.
cudaError_t launch_plan(sipf_ctx* c, int b, int next_layout, cudaStream_t s, double dt);
cudaError_t launch_tile_count(sipf_ctx* c, int b, int* cnt);
cudaError_t launch_plan_flat(sipf_ctx* c);
cudaError_t launch_compact(sipf_ctx* c, int b, int out);
cudaError_t launch_cell_histogram(sipf_ctx* c, int b, int* count, int* tmp, int* cell_start);
// cell_start of buffer b and its ids in canonical (cell key, id) order, the
// latter into b's id array (b's log-masses are overwritten as work space)
cudaError_t launch_canonical_order(sipf_ctx* c, int b);
cudaError_t launch_wrap_positions(sipf_ctx* c, const float* x, const float* y, const float* z,
                                  int buf);
cudaError_t launch_export_positions_inplace(sipf_ctx* c, int b);
cudaError_t launch_rel_log_mass(sipf_ctx* c, const double* mass, int buf);
cudaError_t launch_iota(sipf_ctx* c, int buf);
cudaError_t launch_export_mass(sipf_ctx* c, int b, double* out, int as_log);
cudaError_t launch_acc_to_float(sipf_ctx* c, float* dst, float scale);
cudaError_t launch_component(sipf_ctx* c, int comp, float* dst);
cudaError_t launch_diagnostics(sipf_ctx* c, int b, double acc_to_u);
cudaError_t launch_normals(const uint32_t* ids, int64_t N, uint32_t n, uint64_t seed, float* z,
                           uint32_t* bits, cudaStream_t s);
// Batched particle kernels of an ensemble whose n <= kMaxRuns members all
// read buffer `parity`: the step over the concatenated items of all runs
// (one persistent launch), and the plan of every run (one block per run).
cudaError_t launch_step_multi(const RunDesc* runs, int n, int parity, cudaStream_t s);
cudaError_t launch_plan_multi(const RunDesc* runs, int n, int parity, cudaStream_t s);
RunDesc run_desc(const sipf_ctx* c, double dt);
// api.cu
int run_steps_for(sipf_ctx* c, double dt, int64_t k);
// sipf_create with every device array taken from `pool` on `stream`
// (cudaMallocFromPoolAsync; freed with cudaFreeAsync by sipf_destroy), so
// that creating and destroying contexts never calls cudaMalloc or cudaFree.
int create_in_pool(const sipf_grid* grid, int64_t N, const sipf_params* params,
                   cudaStream_t stream, cudaMemPool_t pool, sipf_ctx** out);
// smooth.cu
cudaError_t launch_smooth(sipf_ctx* c, float* us, cudaStream_t s);
void fill_smoothing(int H, double L, double sigma, float* host_out);
// resample.cu
int resample_device(sipf_ctx* c, int src, int dst, double ratio, int* done, std::string* err);
// fft.cu
cudaError_t launch_spectral_step(sipf_ctx* c, const SpectralArgs& a);
cudaError_t launch_spectral_pass(sipf_ctx* c, const SpectralArgs& a, int pass);
// The context's data for the fused spectral passes (its current buffer parity).
bool has_warp_pipeline(int H);
SpecRun spec_run(const sipf_ctx* c, const SpectralArgs& a);
// One fused spectral pass (0 forward, 1 z, 2 inverse) over n <= kMaxBatch
// runs of grid size H <= 128, in one launch.
cudaError_t launch_spectral_batch(int H, const SpecRun* runs, int n, int pass, int plan,
                                  int device, cudaStream_t s);
void fill_twiddles(int H, float2* host_out);

}  // namespace sipf
