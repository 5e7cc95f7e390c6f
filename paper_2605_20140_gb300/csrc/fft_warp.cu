// Spectral passes of the warp per-axis pipeline (radix plan 2) for the grid
// sizes that have a WarpZ shape.
#include "fft_kernels.cuh"

namespace sipf {

bool has_warp_pipeline(int H) { return H == 64 || H == 128 || H == 256; }

cudaError_t warp_dispatch(int H, const SpecRun& run, int pass, int device, cudaStream_t s) {
    SpecBatch<1> one;
    one.run[0] = run;
    switch (H) {
        case 64: return warp_pass<64, 1>(one, 1, pass, device, s);
        case 128: return warp_pass<128, 1>(one, 1, pass, device, s);
        case 256: return warp_pass<256, 1>(one, 1, pass, device, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sipf
