// Grid side of the SIPF-W step on sm_103a: the explicit reaction R_tau, the
// spectral diffusion solve D_tau and the spectral gradient of v (paper
// Eq. g_hat_phy, Eq. k_q_update with the implicit multipliers of Sec. 4,
// Eq. gradv), as three passes over the grid with a hand-written FFT:
//
//  1. per z-plane: read v, m, w and the integer deposit accumulator, form
//     m* = m + tau u, w* = w + tau (gamma v - eta(u) w), v^n = v/(1 + alpha tau m),
//     store v^n, and transform m*, w*, v^n along x and y in shared memory
//     (m* + i w* as one complex plane; v^n as pairs of rows y, y + H/2).
//     Writes three half spectra [z][ky][kx], kx <= H/2.
//  2. per (ky, field) slab: forward FFT along z, multiply by
//     1/(1 + tau beta + tau Dm |k|^2) (m), 1/(1 + tau + tau Dw |k|^2) (w), or
//     i k_z (v -> B), inverse FFT along z; in place for m and w.  The load,
//     the multiply and the store ride on the first and last DFT stages.
//  3. per (z-plane, group): inverse FFT along y and a packed complex inverse
//     along x: (m, w), (i k_x V, i k_y V) -> (dv/dx, dv/dy), and B in rows
//     y, y + H/2 -> dv/dz.  Writes m^n, w^n and grad v^n, scaled by 1/H^3.
//
// Shared-memory layouts keep a warp's accesses free of bank conflicts: lanes
// take consecutive transforms, whose elements lie one float2 apart or at an
// odd pitch (H + 1 for rows, H/2 + 1 for the inverse pass's half spectra).
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

// Per-size dispatch, one translation unit per (pass family, radix plan).
cudaError_t fused_dispatch_p0(int H, const SpecRun* runs, int n, int pass, int device,
                              cudaStream_t s);
cudaError_t fused_dispatch_p1(int H, const SpecRun* runs, int n, int pass, int device,
                              cudaStream_t s);
cudaError_t split_dispatch_p0(sipf_ctx* c, const SpectralArgs& a, int pass);
cudaError_t split_dispatch_p1(sipf_ctx* c, const SpectralArgs& a, int pass);
cudaError_t warp_dispatch(int H, const SpecRun& run, int pass, int device, cudaStream_t s);

cudaError_t launch_spectral_pass(sipf_ctx* c, const SpectralArgs& a, int pass) {
    if (c->radix_plan == 2) return warp_dispatch(c->H, spec_run(c, a), pass, c->device, c->stream);
    if (c->H <= 128) {
        const SpecRun one = spec_run(c, a);
        return c->radix_plan ? fused_dispatch_p1(c->H, &one, 1, pass, c->device, c->stream)
                             : fused_dispatch_p0(c->H, &one, 1, pass, c->device, c->stream);
    }
    return c->radix_plan ? split_dispatch_p1(c, a, pass) : split_dispatch_p0(c, a, pass);
}

cudaError_t launch_spectral_batch(int H, const SpecRun* runs, int n, int pass, int plan,
                                  int device, cudaStream_t s) {
    if (n < 1 || n > kMaxBatch || H > 128) return cudaErrorInvalidValue;
    if (plan == 2) {
        // the warp pipeline's lines are independent of the run: one launch set per run
        for (int i = 0; i < n; ++i) {
            const cudaError_t e = warp_dispatch(H, runs[i], pass, device, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return plan == 1 ? fused_dispatch_p1(H, runs, n, pass, device, s)
                : fused_dispatch_p0(H, runs, n, pass, device, s);
}

SpecRun spec_run(const sipf_ctx* c, const SpectralArgs& a) {
    SpecRun r;
    r.a = a;
    r.v = c->v;
    r.m = c->m;
    r.w = c->w;
    r.acc = reinterpret_cast<unsigned long long*>(c->acc);
    r.v_out = c->v;
    r.m_out = c->m;
    r.w_out = c->w;
    r.G = c->G;
    r.specM = c->specM;
    r.specW = c->specW;
    r.specV = c->specV;
    r.specB = c->specB;
    r.specA = c->specA;
    r.specDx = c->specDx;
    r.specDy = c->specDy;
    r.twiddle = c->twiddle;
    r.voff = c->voff;
    r.sc = c->dsc + c->cur;
    r.us = c->us;
    return r;
}

cudaError_t launch_spectral_step(sipf_ctx* c, const SpectralArgs& a) {
    for (int pass = 0; pass < 3; ++pass) {
        const cudaError_t e = launch_spectral_pass(c, a, pass);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void fill_twiddles(int H, float2* out) {
    for (int j = 0; j < H; ++j) {
        const double ang = -2.0 * M_PI * static_cast<double>(j) / static_cast<double>(H);
        out[j] = make_float2(static_cast<float>(cos(ang)), static_cast<float>(sin(ang)));
    }
}

}  // namespace sipf
