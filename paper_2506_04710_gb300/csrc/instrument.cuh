// Launch accounting shared by the translation units (see instrument.cu).
#pragma once

#include <cuda_runtime.h>

namespace ztoep {

// Kernel classes (bit positions of the ztoep_timing_enable mask).
enum KClass { K_FFT = 0, K_BLOCKPROD = 1, K_EDGE = 2, K_ARNOLDI = 3, K_MISC = 4, K_TENSOR = 5, K_TENSOR_PIPE = 6,
              K_NCLASS = 7 };

// Wraps `n` kernel launches of one class on one stream.
class KScope {
  public:
    KScope(KClass c, cudaStream_t s);
    ~KScope();
    void add(int n) { n_ += n - 1; }
    KScope(const KScope &) = delete;
    KScope &operator=(const KScope &) = delete;

  private:
    int cls_;
    cudaStream_t s_;
    cudaEvent_t a_;
    int n_ = 1;
    bool capturing_ = false;
};

// Launches made while a stream is being captured are added to *sink (on this
// thread) instead of the process counter; graph replays are counted with
// add_launches.
void capture_count_begin(uint64_t *sink);
void capture_count_end();
void add_launches(uint64_t n);

// ZTOEP_TIMING_SERIAL set: products serialise their branches on one stream.
bool timing_serial();

}  // namespace ztoep
