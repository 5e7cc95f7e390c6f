// Internal declarations of the SIPF-W CUDA path: context layout, device
// helpers shared by the particle kernels, kernel launch wrappers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sipf.h"

namespace sipf {

constexpr int kTile = 8;            // cells per tile edge of the tile-major cell key
constexpr int kMaxH = 128;          // largest grid of this build

// Device status bits (ORed into ctx->status by kernels, read by sipf_sync).
constexpr int kStatusNonfinite = 1;   // a pushed position was NaN/inf (reset to 0)
constexpr int kStatusSlot = 2;        // scatter slot outside its cell's run
constexpr int kStatusTotal = 4;       // cell counts did not sum to N

// Kernel groups of a step, in launch order (tracing).
constexpr int kProfGroups = 6;
constexpr int kProfMaxSteps = 4096;

// Per-step scalars of the particle kernels.
struct PushArgs {
    int H;
    float drift;      // chi * tau / h      (grid units per unit grad v)
    float noise;      // sqrt(2 Du tau) / h (grid units per standard normal)
    float tau;
    uint32_t n;       // step index (Philox counter word 0)
    uint32_t k0, k1;  // Philox key
    int push;         // 0: positions unchanged (pure binning)
};

// Deposit scaling: contribution of a particle to a corner node is
// exp(loga - logref) * weight, stored as the integer round(value * 2^S).
struct DepositArgs {
    double logref;    // reference log-mass subtracted before the float exp
    float scale;      // 2^S
};

// Spectral-step scalars.
struct SpectralArgs {
    float tau;
    float react_scale;     // converts the integer deposit accumulator to u_bar
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

}  // namespace sipf

struct sipf_ctx {
    int H = 0;
    double L = 0, h = 0;
    double origin[3] = {0, 0, 0};
    int64_t N = 0;
    sipf_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;

    // particle store, ping-pong (storage order = bucketed by cell key)
    float* sx[2] = {nullptr, nullptr};
    float* sy[2] = {nullptr, nullptr};
    float* sz[2] = {nullptr, nullptr};
    double* loga[2] = {nullptr, nullptr};
    uint32_t* id[2] = {nullptr, nullptr};
    int cur = 0;

    // binning
    int32_t* count = nullptr;        // H^3, zero between steps
    int32_t* cell_start = nullptr;   // H^3 + 1, of the current store
    int32_t* scan_tmp = nullptr;     // block sums of the scan

    // grid
    long long* acc = nullptr;        // H^3 fixed-point deposit accumulator, zero between steps
    float* v = nullptr;
    float* m = nullptr;
    float* w = nullptr;
    float* gx = nullptr;
    float* gy = nullptr;
    float* gz = nullptr;
    float2* specM = nullptr;         // half spectra [z][ky][kx], row pitch kxp
    float2* specW = nullptr;
    float2* specV = nullptr;
    float2* specB = nullptr;
    float2* specA = nullptr;         // filtered v spectrum (filter on only)
    float2* twiddle = nullptr;       // exp(-2 pi i j / H), j < H
    float* voff = nullptr;           // device scalar: offset subtracted from v before its FFT
    int kxp = 0;

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
    float voff_host = 0;             // staging value for voff
    bool state_set = false;
    std::string last_error;
};

namespace sipf {

// ---------------------------------------------------------------- launchers
// particles.cu
cudaError_t launch_count(sipf_ctx* c, const PushArgs& a);
cudaError_t launch_scan(sipf_ctx* c);
cudaError_t launch_scatter(sipf_ctx* c, const PushArgs& a, const DepositArgs& d, int deposit,
                           int scatter);
cudaError_t launch_wrap_positions(sipf_ctx* c, const float* x, int buf);
cudaError_t launch_log_mass(sipf_ctx* c, const double* mass, int buf);
cudaError_t launch_export_positions(sipf_ctx* c, float* x);
cudaError_t launch_export_mass(sipf_ctx* c, double* mass);
cudaError_t launch_acc_to_float(sipf_ctx* c, float* dst, float scale);
cudaError_t launch_diagnostics(sipf_ctx* c, float acc_to_u);
cudaError_t launch_normals(const uint32_t* ids, int64_t N, uint32_t n, uint64_t seed, float* z,
                           uint32_t* bits, cudaStream_t s);
// fft.cu
cudaError_t launch_spectral_step(sipf_ctx* c, const SpectralArgs& a);
cudaError_t launch_spectral_pass(sipf_ctx* c, const SpectralArgs& a, int pass);
void fill_twiddles(int H, float2* host_out);

}  // namespace sipf
