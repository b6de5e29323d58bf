// Register FFT kernels of the inverse y pass (spectrum -> X1, cropped), lengths of
// part 1 of the size table (each part compiled on its own for build speed).
#include "fftreg_impl.cuh"
#include "passes.cuh"

namespace ztoep {
template ztoep_status_t launch_fft_reg_part<true, LdXh<float>, StY1<float>, 1>(int, const float2 *, dim3, int,
                                                                   const LdXh<float> &, const StY1<float> &,
                                                                   cudaStream_t);
}  // namespace ztoep
