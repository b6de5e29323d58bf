// Batched 1-D complex FFT passes in shared memory (Stockham autosort, radices
// 2, 3, 4, 5).  One CTA transforms `ib` channels of one line of length L;
// loader/storer functors map (position, channel) to global memory, which is
// where the zero-padding of the circulant embedding, the crop, the 1/(LxLy)
// scale and the epilogue fusions live.
#pragma once

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {

// Radix-R DFT of a[0..R) in registers.  Forward: b_q = sum_r a_r e^{-2 pi i q r / R}.
template <typename C> __device__ __forceinline__ C mul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }  // -i*a
template <typename C> __device__ __forceinline__ C mul_pi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }  // +i*a

template <int RAD, typename C> __device__ __forceinline__ void dft_small(C *a, bool inv);

template <> __device__ __forceinline__ void dft_small<2, float2>(float2 *a, bool) {
    float2 t = a[0] - a[1]; a[0] = a[0] + a[1]; a[1] = t;
}
template <> __device__ __forceinline__ void dft_small<2, double2>(double2 *a, bool) {
    double2 t = a[0] - a[1]; a[0] = a[0] + a[1]; a[1] = t;
}

template <typename C> __device__ __forceinline__ void dft4(C *a, bool inv) {
    C t0 = a[0] + a[2], t1 = a[0] - a[2], t2 = a[1] + a[3], t3 = a[1] - a[3];
    a[0] = t0 + t2;
    a[2] = t0 - t2;
    C r = inv ? mul_pi(t3) : mul_mi(t3);
    a[1] = t1 + r;
    a[3] = t1 - r;
}
template <> __device__ __forceinline__ void dft_small<4, float2>(float2 *a, bool inv) { dft4(a, inv); }
template <> __device__ __forceinline__ void dft_small<4, double2>(double2 *a, bool inv) { dft4(a, inv); }

// sin(2 pi / 3), cos/sin of 2 pi/5 and 4 pi/5.
#define ZT_S3 0.86602540378443864676
#define ZT_C51 0.30901699437494742410
#define ZT_C52 (-0.80901699437494742410)
#define ZT_S51 0.95105651629515357212
#define ZT_S52 0.58778525229247312917

template <typename C, typename R> __device__ __forceinline__ void dft3(C *a, bool inv) {
    C t = a[1] + a[2], u = a[1] - a[2];
    C m = a[0] - cscale(t, (R)0.5);
    a[0] = a[0] + t;
    C su = cscale(u, (R)ZT_S3);
    C r = inv ? mul_pi(su) : mul_mi(su);  // -+ i s u
    a[1] = m + r;
    a[2] = m - r;
}
template <> __device__ __forceinline__ void dft_small<3, float2>(float2 *a, bool inv) { dft3<float2, float>(a, inv); }
template <> __device__ __forceinline__ void dft_small<3, double2>(double2 *a, bool inv) { dft3<double2, double>(a, inv); }

template <typename C, typename R> __device__ __forceinline__ void dft5(C *a, bool inv) {
    C t1 = a[1] + a[4], t2 = a[2] + a[3], t3 = a[1] - a[4], t4 = a[2] - a[3];
    C m1 = a[0] + cscale(t1, (R)ZT_C51) + cscale(t2, (R)ZT_C52);
    C m2 = a[0] + cscale(t1, (R)ZT_C52) + cscale(t2, (R)ZT_C51);
    C s1 = cscale(t3, (R)ZT_S51) + cscale(t4, (R)ZT_S52);
    C s2 = cscale(t3, (R)ZT_S52) - cscale(t4, (R)ZT_S51);
    C r1 = inv ? mul_pi(s1) : mul_mi(s1);
    C r2 = inv ? mul_pi(s2) : mul_mi(s2);
    a[0] = a[0] + t1 + t2;
    a[1] = m1 + r1;
    a[4] = m1 - r1;
    a[2] = m2 + r2;
    a[3] = m2 - r2;
}
template <> __device__ __forceinline__ void dft_small<5, float2>(float2 *a, bool inv) { dft5<float2, float>(a, inv); }
template <> __device__ __forceinline__ void dft_small<5, double2>(double2 *a, bool inv) { dft5<double2, double>(a, inv); }

// One Stockham stage: sub-transforms of length Ns are merged into length Ns*RAD.
// Layout in shared memory: element (pos, ch) at pos*ib + ch, ib = 1 << lib.
template <int RAD, typename C>
__device__ __forceinline__ void stockham_stage(const C *__restrict__ src, C *__restrict__ dst, int L,
                                               int Ns, int mag, int lib, const C *__restrict__ tws, bool inv) {
    const int nbf = L / RAD;
    const int span = L / (Ns * RAD);
    const int items = nbf << lib;
    const int mask = (1 << lib) - 1;
    for (int item = threadIdx.x; item < items; item += blockDim.x) {
        const int j = item >> lib, ch = item & mask;
        const int k = j - (int)(((unsigned)j * (unsigned)mag) >> 16) * Ns;  // j mod Ns (j < 256)
        C a[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) a[r] = src[((j + r * nbf) << lib) + ch];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                C w = tws[r * k * span];
                if (inv) w.y = -w.y;
                a[r] = cmul(a[r], w);
            }
        }
        dft_small<RAD>(a, inv);
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int q = 0; q < RAD; ++q) dst[((base + q * Ns) << lib) + ch] = a[q];
    }
}

// FP32 stage on channel pairs: element (pos, 2 c2), (pos, 2 c2 + 1) is one
// 16-byte value at pos * ib/2 + c2, so each item moves two channels with one
// load/store per point and shares the twiddle and index arithmetic.
template <int RAD>
__device__ __forceinline__ void stockham_stage_v2(const float4 *__restrict__ src, float4 *__restrict__ dst, int L,
                                                  int Ns, int mag, int lib1, const float2 *__restrict__ tws,
                                                  bool inv) {
    const int nbf = L / RAD;
    const int span = L / (Ns * RAD);
    const int items = nbf << lib1;
    const int mask = (1 << lib1) - 1;
    for (int item = threadIdx.x; item < items; item += blockDim.x) {
        const int j = item >> lib1, c2 = item & mask;
        const int k = j - (int)(((unsigned)j * (unsigned)mag) >> 16) * Ns;  // j mod Ns (j < 256)
        float2 a[RAD], c[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            const float4 v = src[((j + r * nbf) << lib1) + c2];
            a[r] = make_float2(v.x, v.y);
            c[r] = make_float2(v.z, v.w);
        }
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                float2 w = tws[r * k * span];
                if (inv) w.y = -w.y;
                a[r] = cmul(a[r], w);
                c[r] = cmul(c[r], w);
            }
        }
        dft_small<RAD>(a, inv);
        dft_small<RAD>(c, inv);
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int q = 0; q < RAD; ++q)
            dst[((base + q * Ns) << lib1) + c2] = make_float4(a[q].x, a[q].y, c[q].x, c[q].y);
    }
}

// Generic pass: load L x ib values, transform along the L axis, store.
// Shared memory: tw[L] (padded to an even count) + 2 buffers of L*ib.  FP32
// passes with ib >= 2 move channel pairs (functors' ld2/st2).
template <typename R, typename Ld, typename St>
__global__ void __launch_bounds__(256) k_fft_pass(Fft1D pl, const cplx_t<R> *__restrict__ tw, int lib,
                                                  int inv, Ld ld, St st) {
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char zt_smem[];
    C *tws = reinterpret_cast<C *>(zt_smem);
    const int L = pl.L;
    const int ib = 1 << lib;
    C *A = tws + ((L + 1) & ~1);
    C *Bf = A + (size_t)L * ib;
    for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = tw[t];
    const int n = L << lib;
    if constexpr (sizeof(C) == 8) {
        if (lib >= 1) {
            const int lib1 = lib - 1, mask2 = (ib >> 1) - 1, n2 = n >> 1;
            float4 *A4 = reinterpret_cast<float4 *>(A), *B4 = reinterpret_cast<float4 *>(Bf);
            for (int idx = threadIdx.x; idx < n2; idx += blockDim.x)
                A4[idx] = ld.ld2(idx >> lib1, (idx & mask2) << 1);
            __syncthreads();
            float4 *src = A4, *dst = B4;
            int Ns = 1;
            for (int s = 0; s < pl.nst; ++s) {
                const int rad = pl.rad[s], mag = pl.mag[s];
                switch (rad) {
                    case 4: stockham_stage_v2<4>(src, dst, L, Ns, mag, lib1, tws, inv != 0); break;
                    case 2: stockham_stage_v2<2>(src, dst, L, Ns, mag, lib1, tws, inv != 0); break;
                    case 3: stockham_stage_v2<3>(src, dst, L, Ns, mag, lib1, tws, inv != 0); break;
                    default: stockham_stage_v2<5>(src, dst, L, Ns, mag, lib1, tws, inv != 0); break;
                }
                __syncthreads();
                float4 *t = src; src = dst; dst = t;
                Ns *= rad;
            }
            for (int idx = threadIdx.x; idx < n2; idx += blockDim.x)
                st.st2(idx >> lib1, (idx & mask2) << 1, src[idx]);
            return;
        }
    }
    const int mask = ib - 1;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) A[idx] = ld(idx >> lib, idx & mask);
    __syncthreads();
    C *src = A, *dst = Bf;
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int rad = pl.rad[s], mag = pl.mag[s];
        switch (rad) {
            case 4: stockham_stage<4>(src, dst, L, Ns, mag, lib, tws, inv != 0); break;
            case 2: stockham_stage<2>(src, dst, L, Ns, mag, lib, tws, inv != 0); break;
            case 3: stockham_stage<3>(src, dst, L, Ns, mag, lib, tws, inv != 0); break;
            default: stockham_stage<5>(src, dst, L, Ns, mag, lib, tws, inv != 0); break;
        }
        __syncthreads();
        C *t = src; src = dst; dst = t;
        Ns *= rad;
    }
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) st(idx >> lib, idx & mask, src[idx]);
}

// Channel-batch size: the largest power of two <= min(channels, cap) whose
// shared-memory footprint fits `budget` bytes.
inline int pick_lib(int L, int channels, size_t csize, size_t budget, int cap = 64) {
    int lib = 0;
    while ((2 << lib) <= channels && (2 << lib) <= cap &&
           (size_t)(((L + 1) & ~1) + 2 * (size_t)L * (2 << lib)) * csize <= budget)
        ++lib;
    return lib;
}

inline size_t fft_smem_bytes(int L, int lib, size_t csize) {
    return (size_t)(((L + 1) & ~1) + 2 * (size_t)L * ((size_t)1 << lib)) * csize;
}

// Pass geometry: the channel batch is shrunk (down to 32-byte chunks per
// line) until the grid covers every SM twice, and the CTA gets about one
// thread per radix-4 butterfly.
struct PassCfg {
    int lib, threads;
};
inline PassCfg pass_cfg(int L, int channels, int lines, size_t csize, int nsm) {
    int lib = pick_lib(L, channels, csize, 64 * 1024);
    const int min_lib = csize == 8 ? 2 : 1;
    while (lib > min_lib && (int64_t)((channels + (1 << lib) - 1) >> lib) * lines < 2LL * nsm) --lib;
    int thr = ((L << lib) / 4 + 31) / 32 * 32;
    thr = thr < 64 ? 64 : (thr > 256 ? 256 : thr);
    return {lib, thr};
}

template <typename R, typename Ld, typename St>
ztoep_status_t launch_fft_pass(const Fft1D &pl, const cplx_t<R> *tw, int lib, bool inv, dim3 grid,
                               Ld ld, St st, cudaStream_t s, int threads = 256) {
    size_t smem = fft_smem_bytes(pl.L, lib, sizeof(cplx_t<R>));
    static bool attr_set = false;  // one instantiation per (R, Ld, St)
    if (!attr_set) {
        ZT_CUDA(cudaFuncSetAttribute(k_fft_pass<R, Ld, St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024));
        attr_set = true;
    }
    KScope ks(K_FFT, s);
    k_fft_pass<R, Ld, St><<<grid, threads, smem, s>>>(pl, tw, lib, inv ? 1 : 0, ld, st);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

}  // namespace ztoep
