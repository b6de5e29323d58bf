// Register FFT kernels of the inverse x pass (X1 -> output, cropped), lengths of
// part 1 of the size table (each part compiled on its own for build speed).
#include "fftreg_impl.cuh"
#include "passes.cuh"

namespace ztoep {
template ztoep_status_t launch_fft_reg_part<true, LdY1<float>, StYOut<float>, 1>(int, const float2 *, dim3, int,
                                                                   const LdY1<float> &, const StYOut<float> &,
                                                                   cudaStream_t);
}  // namespace ztoep
