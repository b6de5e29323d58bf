// Register-resident FFT passes (FP32) of the product: host-side interface.
//
// A pass transforms, for each line (blockIdx.y, blockIdx.z) and channel pair,
// L points along the line with L = P1 * P2 factored into two small DFTs held
// in registers: each of T = gcd(P1, P2) threads per line loads its P1-point
// sub-sequences (stride P2) straight from global memory, transforms them,
// applies the twiddles w_L^(n2 k1) and writes them to shared memory once; after
// one barrier it reads P2-point columns back, transforms them and stores the
// results (the Cooley-Tukey split of the DFT of Sec. II-C's circulant
// products).  One thread owns a channel pair (16-byte accesses), consecutive
// threads own consecutive pairs, so every global access is contiguous across
// the CTA's channel batch.  Kernels live in fftreg_impl.cuh, instantiated for
// the four pass kinds in fftreg_*.cu.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace ztoep {

// (L, P1, P2): the sizes with a register kernel, P1 and P2 from {2,...,16}
// with factors 2, 3, 5 and as many threads per line (gcd) as the split allows.
#define ZT_REG_FFT_SIZES_0(X)                                                                         \
    X(8, 4, 2) X(9, 3, 3) X(10, 5, 2) X(12, 6, 2) X(15, 5, 3) X(16, 4, 4) X(18, 6, 3) X(20, 10, 2)     \
    X(24, 6, 4) X(25, 5, 5) X(27, 9, 3) X(30, 10, 3) X(32, 8, 4) X(36, 6, 6) X(40, 10, 4) X(45, 15, 3) \
    X(48, 12, 4) X(50, 10, 5) X(54, 9, 6) X(60, 10, 6) X(64, 8, 8)
#define ZT_REG_FFT_SIZES_1(X)                                                                         \
    X(72, 12, 6) X(75, 15, 5) X(80, 10, 8) X(81, 9, 9) X(90, 15, 6) X(96, 12, 8) X(100, 10, 10)        \
    X(120, 12, 10) X(128, 16, 8) X(135, 15, 9) X(144, 12, 12) X(256, 16, 16)
#define ZT_REG_FFT_SIZES(X) ZT_REG_FFT_SIZES_0(X) ZT_REG_FFT_SIZES_1(X)

__host__ __device__ constexpr int reg_gcd(int a, int b) { return b == 0 ? a : reg_gcd(b, a % b); }

struct RegShape {
    int p1 = 0, p2 = 0, t = 0;
};

inline bool reg_fft_shape(int L, RegShape *out) {
    switch (L) {
#define ZT_REG_CASE(LL, A, B)                       \
    case LL:                                        \
        if (out) *out = RegShape{A, B, reg_gcd(A, B)}; \
        return true;
        ZT_REG_FFT_SIZES(ZT_REG_CASE)
#undef ZT_REG_CASE
        default: return false;
    }
}

// Shared memory of one CTA: L points x cpb channel pairs x 16 bytes.
inline size_t reg_fft_smem(int L, int cpb) { return (size_t)L * cpb * 16; }

// Channel pairs per CTA (a power of two): the tuned channel count / 2 when
// given, else the largest of 16, 8, 4 that still gives two CTAs per SM.  The
// batch stops at the first power of two covering all channels, 256 threads
// and 64 KB of shared memory.
inline int reg_fft_cpb(int L, int channels, int lines, int nsm, int tuned_channels) {
    RegShape sh;
    if (!reg_fft_shape(L, &sh)) return 1;
    int cap = 1;
    while (2 * cap < channels && cap < 32 && 2 * cap * sh.t <= 256 && reg_fft_smem(L, 2 * cap) <= 64 * 1024) cap *= 2;
    if (tuned_channels >= 2) return std::max(1, std::min(cap, tuned_channels / 2));
    int cpb = std::min(cap, 16);
    while (cpb > 4 && (int64_t)((channels + 2 * cpb - 1) / (2 * cpb)) * lines < 2LL * nsm) cpb /= 2;
    return cpb;
}

// Launch of the register pass (L must satisfy reg_fft_shape).  grid.x covers
// the channels in batches of 2 cpb, and the functors' ib must be 2 cpb.  The
// sizes are split over two instantiation units (PART 0 / 1) for build speed.
template <bool INV, class Ld, class St, int PART>
ztoep_status_t launch_fft_reg_part(int L, const float2 *tw, dim3 grid, int cpb, const Ld &ld, const St &st,
                                   cudaStream_t s);

inline bool reg_fft_part0(int L) {
    switch (L) {
#define ZT_REG_CASE0(LL, A, B) case LL:
        ZT_REG_FFT_SIZES_0(ZT_REG_CASE0)
#undef ZT_REG_CASE0
        return true;
        default: return false;
    }
}

template <bool INV, class Ld, class St>
ztoep_status_t launch_fft_reg(int L, const float2 *tw, dim3 grid, int cpb, const Ld &ld, const St &st,
                              cudaStream_t s) {
    if (!reg_fft_shape(L, nullptr)) return ZTOEP_ERR_UNSUPPORTED;
    return reg_fft_part0(L) ? launch_fft_reg_part<INV, Ld, St, 0>(L, tw, grid, cpb, ld, st, s)
                            : launch_fft_reg_part<INV, Ld, St, 1>(L, tw, grid, cpb, ld, st, s);
}

}  // namespace ztoep
