// Register-resident FFT pass kernels (FP32, channel pairs as float4): the
// small DFTs, their compile-time constants and the two-phase pass kernel.
// Included only by the fftreg_*.cu translation units.
#pragma once
#include <type_traits>
#include <utility>

#include "fftreg.cuh"
#include "instrument.cuh"

namespace ztoep {
namespace rf {

// ---------------------------------------------------------------- constants
// cos and sin of 2 pi j / n, evaluated at compile time: the angle is reduced
// to (-pi, pi] in exact integer arithmetic, then summed from the Taylor series
// (30 terms; error below 1e-15, far under the FP32 rounding of the result).
__host__ __device__ constexpr double ct_angle(int j, int n) {
    int r = ((j % n) + n) % n;
    if (2 * r > n) r -= n;
    return 6.283185307179586476925286766559 * (double)r / (double)n;
}
__host__ __device__ constexpr double ct_cos(int j, int n) {
    const double x = ct_angle(j, n);
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_sin(int j, int n) {
    const double x = ct_angle(j, n);
    double term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1.
template <class F, int... Is>
__host__ __device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F> __host__ __device__ __forceinline__ void sfor(F &&f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// ------------------------------------------------------- channel-pair algebra
// A float4 holds two complex numbers (x + iy, z + iw): the same channel
// pair's values; every operation applies to both.
__host__ __device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__host__ __device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__host__ __device__ __forceinline__ float4 scl4(float4 a, float s) {
    return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__host__ __device__ __forceinline__ float4 mul_mi(float4 a) { return make_float4(a.y, -a.x, a.w, -a.z); }  // * (-i)
__host__ __device__ __forceinline__ float4 mul_pi(float4 a) { return make_float4(-a.y, a.x, -a.w, a.z); }  // * (+i)
__host__ __device__ __forceinline__ float4 cmul4(float4 a, float c, float s) {  // * (c + i s)
    return make_float4(a.x * c - a.y * s, a.x * s + a.y * c, a.z * c - a.w * s, a.z * s + a.w * c);
}

// a * w_N^J with w_N = exp(-2 pi i / N) (forward) or its conjugate (INV).
template <int N, int J, bool INV> __host__ __device__ __forceinline__ float4 twc(float4 a) {
    constexpr int r = ((J % N) + N) % N;
    if constexpr (r == 0) {
        return a;
    } else if constexpr (2 * r == N) {
        return make_float4(-a.x, -a.y, -a.z, -a.w);
    } else if constexpr (4 * r == N) {
        return INV ? mul_pi(a) : mul_mi(a);
    } else if constexpr (4 * r == 3 * N) {
        return INV ? mul_mi(a) : mul_pi(a);
    } else {
        constexpr float c = (float)ct_cos(r, N);
        constexpr float s = (float)(INV ? ct_sin(r, N) : -ct_sin(r, N));
        return cmul4(a, c, s);
    }
}

// ------------------------------------------------------------- small DFTs
// X[k] = sum_n v[n] w_P^(n k) in place (w_P = exp(-+2 pi i / P)).
template <int P, bool INV> struct Dft;

template <bool INV> struct Dft<1, INV> {
    __host__ __device__ __forceinline__ static void run(float4 (&)[1]) {}
};
template <bool INV> struct Dft<2, INV> {
    __host__ __device__ __forceinline__ static void run(float4 (&v)[2]) {
        const float4 a = v[0], b = v[1];
        v[0] = add4(a, b);
        v[1] = sub4(a, b);
    }
};
template <bool INV> struct Dft<4, INV> {
    __host__ __device__ __forceinline__ static void run(float4 (&v)[4]) {
        const float4 t0 = add4(v[0], v[2]), t1 = sub4(v[0], v[2]), t2 = add4(v[1], v[3]);
        const float4 d = sub4(v[1], v[3]);
        const float4 t3 = INV ? mul_pi(d) : mul_mi(d);  // (v1 - v3) w_4
        v[0] = add4(t0, t2);
        v[2] = sub4(t0, t2);
        v[1] = add4(t1, t3);
        v[3] = sub4(t1, t3);
    }
};

// Odd prime P: pairs n, P - n share cos(2 pi n k / P) and have opposite sines,
// so X_k and X_(P-k) come from a_n = v_n + v_(P-n) and b_n = v_n - v_(P-n).
template <int P, bool INV> struct DftOdd {
    __host__ __device__ __forceinline__ static void run(float4 (&v)[P]) {
        constexpr int H = (P - 1) / 2;
        float4 a[H], b[H];
        float4 s0 = v[0];
        sfor<H>([&](auto nI) {
            constexpr int n = decltype(nI)::value + 1;
            a[n - 1] = add4(v[n], v[P - n]);
            b[n - 1] = sub4(v[n], v[P - n]);
            s0 = add4(s0, a[n - 1]);
        });
        float4 out[P];
        out[0] = s0;
        sfor<H>([&](auto kI) {
            constexpr int k = decltype(kI)::value + 1;
            float4 re = v[0], im = make_float4(0.f, 0.f, 0.f, 0.f);
            sfor<H>([&](auto nI) {
                constexpr int n = decltype(nI)::value + 1;
                constexpr float c = (float)ct_cos(n * k, P), s = (float)ct_sin(n * k, P);
                re = add4(re, scl4(a[n - 1], c));
                im = add4(im, scl4(b[n - 1], s));
            });
            const float4 mi = mul_mi(im);  // -i * sum b_n sin
            out[k] = INV ? sub4(re, mi) : add4(re, mi);
            out[P - k] = INV ? add4(re, mi) : sub4(re, mi);
        });
        sfor<P>([&](auto iI) {
            constexpr int i = decltype(iI)::value;
            v[i] = out[i];
        });
    }
};
template <bool INV> struct Dft<3, INV> : DftOdd<3, INV> {};
template <bool INV> struct Dft<5, INV> : DftOdd<5, INV> {};

__host__ __device__ constexpr int first_radix(int P) {
    if (P % 4 == 0 && P > 4) return 4;
    for (int f = 2; f <= P; ++f)
        if (P % f == 0) return f;
    return P;
}

// Composite P = p q (Cooley-Tukey): DFT-p over n1 of v[q n1 + n2] for each
// n2, twiddles w_P^(n2 k1), DFT-q over n2 for each k1; X[k1 + p k2] ends in
// slot q k1 + k2 and is moved to slot k1 + p k2.
template <int P, bool INV> struct Dft {
    static constexpr int p = first_radix(P), q = P / p;
    static_assert(p > 1 && q > 1, "composite size expected");
    __host__ __device__ __forceinline__ static void run(float4 (&v)[P]) {
        sfor<q>([&](auto n2I) {
            constexpr int n2 = decltype(n2I)::value;
            float4 t[p];
            sfor<p>([&](auto n1I) {
                constexpr int n1 = decltype(n1I)::value;
                t[n1] = v[q * n1 + n2];
            });
            Dft<p, INV>::run(t);
            sfor<p>([&](auto k1I) {
                constexpr int k1 = decltype(k1I)::value;
                v[q * k1 + n2] = twc<P, n2 * k1, INV>(t[k1]);
            });
        });
        float4 out[P];
        sfor<p>([&](auto k1I) {
            constexpr int k1 = decltype(k1I)::value;
            float4 t[q];
            sfor<q>([&](auto n2I) {
                constexpr int n2 = decltype(n2I)::value;
                t[n2] = v[q * k1 + n2];
            });
            Dft<q, INV>::run(t);
            sfor<q>([&](auto k2I) {
                constexpr int k2 = decltype(k2I)::value;
                out[k1 + p * k2] = t[k2];
            });
        });
        sfor<P>([&](auto iI) {
            constexpr int i = decltype(iI)::value;
            v[i] = out[i];
        });
    }
};

}  // namespace rf

// ---------------------------------------------------------------- pass kernel
// CTA = cpb channel pairs x T threads per line (thread = cp + cpb t).
// Phase 1: thread t takes n2 = t, t + T, ... (< P2): loads v[n1] = x[P2 n1 + n2],
//   DFT-P1, multiplies output k1 by w_L^(n2 k1) (the plan's table, conjugated
//   for the inverse) and writes it to buf[k1 P2 + n2].
// Phase 2: thread t takes k1 = t, t + T, ... (< P1): reads buf[k1 P2 + n2] for
//   all n2, DFT-P2, stores output k1 + P1 k2.
template <int P1, int P2, bool INV, class Ld, class St>
__global__ void __launch_bounds__(256) k_fft_reg(const float2 *__restrict__ tw, Ld ld, St st, int cpb) {
    constexpr int T = reg_gcd(P1, P2);
    extern __shared__ __align__(16) unsigned char zt_smem[];
    float4 *buf = reinterpret_cast<float4 *>(zt_smem);
    const int cp = threadIdx.x % cpb, t = threadIdx.x / cpb;
    const int ch = 2 * cp;
#pragma unroll
    for (int a = 0; a < P2 / T; ++a) {
        const int n2 = t + T * a;
        float4 v[P1];
#pragma unroll
        for (int n1 = 0; n1 < P1; ++n1) v[n1] = ld.ld2(P2 * n1 + n2, ch);
        rf::Dft<P1, INV>::run(v);
#pragma unroll
        for (int k1 = 1; k1 < P1; ++k1) {
            const float2 w = __ldg(tw + n2 * k1);
            v[k1] = rf::cmul4(v[k1], w.x, INV ? -w.y : w.y);
        }
#pragma unroll
        for (int k1 = 0; k1 < P1; ++k1) buf[(k1 * P2 + n2) * cpb + cp] = v[k1];
    }
    __syncthreads();
#pragma unroll
    for (int bq = 0; bq < P1 / T; ++bq) {
        const int k1 = t + T * bq;
        float4 v[P2];
#pragma unroll
        for (int n2 = 0; n2 < P2; ++n2) v[n2] = buf[(k1 * P2 + n2) * cpb + cp];
        rf::Dft<P2, INV>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < P2; ++k2) st.st2(k1 + P1 * k2, ch, v[k2]);
    }
}

template <int P1, int P2, bool INV, class Ld, class St>
static ztoep_status_t launch_reg_shape(const float2 *tw, dim3 grid, int cpb, const Ld &ld, const St &st,
                                       cudaStream_t s) {
    constexpr int T = reg_gcd(P1, P2);
    const size_t smem = reg_fft_smem(P1 * P2, cpb);
    if (cpb < 1 || cpb * T > 256 || smem > 200 * 1024) return ZTOEP_ERR_UNSUPPORTED;
    static bool attr_set = false;
    if (!attr_set && smem > 48 * 1024) {
        ZT_CUDA(cudaFuncSetAttribute(k_fft_reg<P1, P2, INV, Ld, St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024));
        attr_set = true;
    }
    KScope ks(K_FFT, s);
    k_fft_reg<P1, P2, INV, Ld, St><<<grid, cpb * T, smem, s>>>(tw, ld, st, cpb);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

template <bool INV, class Ld, class St, int PART>
ztoep_status_t launch_fft_reg_part(int L, const float2 *tw, dim3 grid, int cpb, const Ld &ld, const St &st,
                                   cudaStream_t s) {
#define ZT_REG_LAUNCH(LL, A, B) \
    case LL: return launch_reg_shape<A, B, INV, Ld, St>(tw, grid, cpb, ld, st, s);
    if constexpr (PART == 0) {
        switch (L) {
            ZT_REG_FFT_SIZES_0(ZT_REG_LAUNCH)
            default: return ZTOEP_ERR_UNSUPPORTED;
        }
    } else {
        switch (L) {
            ZT_REG_FFT_SIZES_1(ZT_REG_LAUNCH)
            default: return ZTOEP_ERR_UNSUPPORTED;
        }
    }
#undef ZT_REG_LAUNCH
}

}  // namespace ztoep
