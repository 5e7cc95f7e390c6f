// Per-axis spectral passes (H > 128) with radix plan 1.
#include "fft_kernels.cuh"

namespace sipf {

cudaError_t split_dispatch_p1(sipf_ctx* c, const SpectralArgs& a, int pass) {
    switch (c->H) {
        case 144: return spectral_pass_split_v<144, 1>(c, a, pass);
        case 192: return spectral_pass_split_v<192, 1>(c, a, pass);
        case 216: return spectral_pass_split_v<216, 1>(c, a, pass);
        case 256: return spectral_pass_split_v<256, 1>(c, a, pass);
        case 288: return spectral_pass_split_v<288, 1>(c, a, pass);
        case 384: return spectral_pass_split_v<384, 1>(c, a, pass);
        case 432: return spectral_pass_split_v<432, 1>(c, a, pass);
        case 512: return spectral_pass_split_v<512, 1>(c, a, pass);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sipf
