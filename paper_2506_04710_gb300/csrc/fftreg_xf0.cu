// Register FFT kernels of the forward x pass (input -> X1), lengths of
// part 0 of the size table (each part compiled on its own for build speed).
#include "fftreg_impl.cuh"
#include "passes.cuh"

namespace ztoep {
template ztoep_status_t launch_fft_reg_part<false, LdXFwd<float>, StX1<float>, 0>(int, const float2 *, dim3, int,
                                                                   const LdXFwd<float> &, const StX1<float> &,
                                                                   cudaStream_t);
}  // namespace ztoep
