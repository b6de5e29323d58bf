// Register FFT kernels of the forward y pass (X1 -> spectrum), lengths of
// part 0 of the size table (each part compiled on its own for build speed).
#include "fftreg_impl.cuh"
#include "passes.cuh"

namespace ztoep {
template ztoep_status_t launch_fft_reg_part<false, LdX1<float>, StXh<float>, 0>(int, const float2 *, dim3, int,
                                                                   const LdX1<float> &, const StXh<float> &,
                                                                   cudaStream_t);
}  // namespace ztoep
