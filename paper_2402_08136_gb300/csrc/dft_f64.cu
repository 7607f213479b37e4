// Fourier-transform pass kernels for complex128 amplitudes (see dft_impl.cuh).
#include "dft_impl.cuh"

namespace qsim {
void dft_launch_f64(const dftk::DftArgs &a, int K, int sign, int kind, bool contig, int threads, size_t smem,
                   cudaStream_t st) {
    dftk::launch_dtype<double>(a, K, sign, kind, contig, threads, smem, st);
}
}  // namespace qsim
