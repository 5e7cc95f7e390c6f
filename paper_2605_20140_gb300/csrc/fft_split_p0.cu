// Per-axis spectral passes (H > 128) with radix plan 0.
#include "fft_kernels.cuh"

namespace sipf {

cudaError_t split_dispatch_p0(sipf_ctx* c, const SpectralArgs& a, int pass) {
    switch (c->H) {
        case 144: return spectral_pass_split_v<144, 0>(c, a, pass);
        case 192: return spectral_pass_split_v<192, 0>(c, a, pass);
        case 216: return spectral_pass_split_v<216, 0>(c, a, pass);
        case 256: return spectral_pass_split_v<256, 0>(c, a, pass);
        case 288: return spectral_pass_split_v<288, 0>(c, a, pass);
        case 384: return spectral_pass_split_v<384, 0>(c, a, pass);
        case 432: return spectral_pass_split_v<432, 0>(c, a, pass);
        case 512: return spectral_pass_split_v<512, 0>(c, a, pass);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sipf
