// Fused spectral passes (H <= 128) with radix plan 1.
#include "fft_kernels.cuh"

namespace sipf {

cudaError_t fused_dispatch_p1(int H, const SpecRun* runs, int n, int pass, int device,
                              cudaStream_t s) {
    switch (H) {
        case 8: return fused_runs<8, 1>(runs, n, pass, device, s);
        case 16: return fused_runs<16, 1>(runs, n, pass, device, s);
        case 24: return fused_runs<24, 1>(runs, n, pass, device, s);
        case 32: return fused_runs<32, 1>(runs, n, pass, device, s);
        case 48: return fused_runs<48, 1>(runs, n, pass, device, s);
        case 64: return fused_runs<64, 1>(runs, n, pass, device, s);
        case 72: return fused_runs<72, 1>(runs, n, pass, device, s);
        case 96: return fused_runs<96, 1>(runs, n, pass, device, s);
        case 128: return fused_runs<128, 1>(runs, n, pass, device, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sipf
