// Warp-specialised persistent complex GEMM on tcgen05 tensor cores, 3xTF32
// with FP32 accumulation in tensor memory:
//
//   C_p[m][q] = sum_k A_p[m][k] X_p[q][k]      (complex, per problem p)
//
// Complex arithmetic as one real GEMM with the small operand expanded: A's
// complex row m, read as the interleaved real row (ar0, ai0, ar1, ai1, ...),
// is used as it is in memory, and X's complex row q becomes the two real
// rows 2q = (xr, -xi, ...) and 2q+1 = (xi, xr, ...), so real column 2q of D
// is Re C[m][q] and column 2q+1 is Im C[m][q].  Each real value v is split as
// hi = tf32(v), lo = tf32(v - hi) and D = Ahi Xhi + Ahi Xlo + Alo Xhi (the
// 3xTF32 scheme).  Ahi [Xhi; Xlo] is one MMA of width 4 rp (the two products
// land in separate accumulator columns, added in the epilogue) and Alo Xhi a
// second one of width 2 rp, so A is read twice per k-step instead of three
// times.
//
// CTA = 10 warps, one CTA per SM, persistent over work items (problem, RHS
// chunk of rp <= 64, K split, 128-row tile):
//   warp 0     TMA producer: A tile (128 rows x 32 floats, 128B swizzle) and
//              the raw X tile (rp rows x 32 floats) of each k-block into a ring
//              of NS stages (mbarrier full[s], transaction bytes);
//   warps 2-5  split A in place into hi and a lo tile, expand and split X into
//              [Xhi; Xlo] (swizzled), then arrive on ready[s];
//   warp 1     one thread issues the MMAs of a k-block and commits them to
//              empty[s] (stage free) and, at the end of an item, to accf[b];
//   warps 6-9  epilogue: tensor memory -> registers -> C, then acce[b]; the
//              accumulator is double-buffered, so an item's epilogue overlaps
//              the next item's MMAs.
// Every wait is bounded: a wait that gives up records an error bit, raises an
// abort flag the other roles poll, and the producer waits (bounded) for its
// copies in flight before the CTA frees its tensor memory and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "instrument.cuh"
#include "tcgemm.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace ztoep {

namespace {

constexpr int G2_THREADS = 320;
constexpr int G2_MAXRP = 64;
constexpr int G2_MAXST = 6;
constexpr uint32_t G2_WAIT = 1u << 22;
constexpr size_t G2_SMEM_CAP = 227 * 1024 - 1024;  // per-block limit minus static shared memory
enum { G2_ERRBIT = 4 };

struct G2Args {
    float2 *C;
    int64_t ldc_q, ldc_m, strideC, strideCk;
    int M, K, N;         // complex sizes
    int rp;              // RHS rows per chunk (multiple of 8, <= 64)
    int nchunk, ksplit, mtiles, nprob, kchunk;
    int nstage;
    uint32_t tmem_cols;
    int *err;
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

struct Item {
    int p, c, s, mt, k0, nkb;
};

__device__ __forceinline__ Item decode(const G2Args &g, int it) {
    Item r;
    r.mt = it % g.mtiles;
    int rest = it / g.mtiles;
    r.s = rest % g.ksplit;
    rest /= g.ksplit;
    r.c = rest % g.nchunk;
    r.p = rest / g.nchunk;
    r.k0 = r.s * g.kchunk;
    const int k1 = min(g.K, r.k0 + g.kchunk);
    r.nkb = (k1 - r.k0 + 15) / 16;
    return r;
}

}  // namespace

__global__ void __launch_bounds__(G2_THREADS, 1)
    k_cgemm_tc2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, G2Args g) {
    extern __shared__ __align__(1024) unsigned char g2_smem_raw[];
    __shared__ __align__(8) uint64_t full[G2_MAXST], ready[G2_MAXST], empty[G2_MAXST], accf[2], acce[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint32_t raw = smem_u32(g2_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *smem = g2_smem_raw + (base - raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = g.nstage, rp = g.rp;
    // stage: A hi (16 KB) | A lo (16 KB) | X expanded [4 rp][128 B] | X raw [rp][128 B]
    const uint32_t stage_bytes = 32768u + 640u * (uint32_t)rp;
    auto a_hi = [&](int s) { return base + (uint32_t)s * stage_bytes; };
    auto a_lo = [&](int s) { return a_hi(s) + 16384u; };
    auto x_exp = [&](int s) { return a_hi(s) + 32768u; };
    auto x_raw = [&](int s) { return a_hi(s) + 32768u + 512u * (uint32_t)rp; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], 4);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_fence_init();
        abort_flag = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const int items = g.nprob * g.nchunk * g.ksplit * g.mtiles;
    volatile int *abort_v = &abort_flag;
    auto fail = [&]() {
        *abort_v = 1;
        atomicOr(g.err, G2_ERRBIT);
    };

    if (warp == 0) {
        if (lane == 0) {  // ---------------- producer
            const uint32_t tx = 128u * 128u + (uint32_t)rp * 128u;
            uint32_t kbg = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
                const Item w = decode(g, it);
                for (int kb = 0; kb < w.nkb; ++kb) {
                    const int s = (int)(kbg % NS);
                    const uint32_t n = kbg / NS;
                    if (n > 0 && !mbar_wait_bounded(&empty[s], (n - 1) & 1, G2_WAIT)) {
                        ok = false;
                        break;
                    }
                    if (*abort_v) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], tx);
                    const int kx = 2 * (w.k0 + kb * 16);
                    tma_load_3d(a_hi(s), &tmA, kx, w.mt * 128, w.p, &full[s]);
                    tma_load_3d(x_raw(s), &tmX, kx, w.c * rp, w.p, &full[s]);
                    ++kbg;
                }
            }
            if (!ok && !*abort_v) fail();
            // no copy may still be landing when the CTA leaves
            for (int s = 0; s < NS; ++s) {
                if (kbg <= (uint32_t)s) continue;
                const uint32_t cnt = (kbg - (uint32_t)s + NS - 1) / NS;  // copies issued into stage s
                if (!mbar_wait_bounded(&full[s], (cnt - 1) & 1, G2_WAIT)) fail();
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------- MMA issuer
            const uint32_t id_wide = idesc_tf32(4 * rp), id_half = idesc_tf32(2 * rp);
            uint32_t kbg = 0, tc = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
                const Item w = decode(g, it);
                const int b = (int)(tc & 1);
                const uint32_t u = tc >> 1;
                if (u > 0 && !mbar_wait_bounded(&acce[b], (u - 1) & 1, G2_WAIT)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 4 * rp);
                for (int kb = 0; kb < w.nkb; ++kb) {
                    const int s = (int)(kbg % NS);
                    const uint32_t n = kbg / NS;
                    if (*abort_v || !mbar_wait_bounded(&ready[s], n & 1, G2_WAIT)) {
                        ok = false;
                        break;
                    }
                    fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {  // 4 x (K = 8 real = 32 bytes)
                        const uint32_t off = ks * 32;
                        const uint64_t xb = sdesc(x_exp(s) + off);
                        mma_tf32(d, sdesc(a_hi(s) + off), xb, id_wide, (kb > 0 || ks > 0) ? 1 : 0);
                        mma_tf32(d, sdesc(a_lo(s) + off), xb, id_half, 1);
                    }
                    mma_commit(&empty[s]);
                    ++kbg;
                }
                if (!ok) break;
                mma_commit(&accf[b]);
                ++tc;
            }
            if (!ok && !*abort_v) fail();
        }
    } else if (warp <= 5) {  // ---------------- operand split / expansion (128 threads)
        const int t = threadIdx.x - 64;
        uint32_t kbg = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const Item w = decode(g, it);
            for (int kb = 0; kb < w.nkb; ++kb) {
                const int s = (int)(kbg % NS);
                const uint32_t n = kbg / NS;
                if (*abort_v || !mbar_wait_bounded(&full[s], n & 1, G2_WAIT)) {
                    ok = false;
                    break;
                }
                float4 *ah = reinterpret_cast<float4 *>(smem + (a_hi(s) - base));
                float4 *al = reinterpret_cast<float4 *>(smem + (a_lo(s) - base));
#pragma unroll 4
                for (int i = t; i < 1024; i += 128) {  // elementwise: the swizzle is irrelevant
                    const float4 v = ah[i];
                    const float4 h = tf32x4(v);
                    ah[i] = h;
                    al[i] = tf32x4(sub4(v, h));
                }
                const float4 *xr = reinterpret_cast<const float4 *>(smem + (x_raw(s) - base));
                unsigned char *xe = smem + (x_exp(s) - base);
                for (int i = t; i < rp * 8; i += 128) {
                    const int q = i >> 3, ch = i & 7;
                    const float4 v = xr[i];  // (xr0, xi0, xr1, xi1)
                    const float4 re = make_float4(v.x, -v.y, v.z, -v.w);
                    const float4 im = make_float4(v.y, v.x, v.w, v.z);
                    const float4 rh = tf32x4(re), ih = tf32x4(im);
                    *reinterpret_cast<float4 *>(xe + sw128(2 * q, ch)) = rh;
                    *reinterpret_cast<float4 *>(xe + sw128(2 * q + 1, ch)) = ih;
                    *reinterpret_cast<float4 *>(xe + sw128(2 * rp + 2 * q, ch)) = tf32x4(sub4(re, rh));
                    *reinterpret_cast<float4 *>(xe + sw128(2 * rp + 2 * q + 1, ch)) = tf32x4(sub4(im, ih));
                }
                fence_proxy_async();  // generic-proxy stores -> visible to the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&ready[s]);
                ++kbg;
            }
        }
        if (!ok && !*abort_v) fail();
    } else {  // ---------------- epilogue (warps 6-9: TMEM lane quarters 2, 3, 0, 1)
        const int q4 = warp & 3;
        const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
        uint32_t tc = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const Item w = decode(g, it);
            const int b = (int)(tc & 1);
            const uint32_t u = tc >> 1;
            if (*abort_v || !mbar_wait_bounded(&accf[b], u & 1, G2_WAIT)) {
                ok = false;
                break;
            }
            fence_after();
            const int m = w.mt * 128 + 32 * q4 + lane;
            float *C = reinterpret_cast<float *>(g.C + (int64_t)w.p * g.strideC + (int64_t)w.s * g.strideCk);
            const uint32_t col0 = (uint32_t)(b * 4 * rp);
            for (int c0 = 0; c0 < 2 * rp; c0 += 16) {
                uint32_t hh[16], hl[16];
                tmem_ld16_nowait(tmem + lane_base + col0 + (uint32_t)c0, hh);
                tmem_ld16_nowait(tmem + lane_base + col0 + (uint32_t)(2 * rp + c0), hl);
                tmem_ld_wait();
                if (m < g.M) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int q = w.c * rp + c0 / 2 + j;
                        if (q < g.N) {
                            const int64_t o = 2 * ((int64_t)q * g.ldc_q + (int64_t)m * g.ldc_m);
                            C[o] = __uint_as_float(hh[2 * j]) + __uint_as_float(hl[2 * j]);
                            C[o + 1] = __uint_as_float(hh[2 * j + 1]) + __uint_as_float(hl[2 * j + 1]);
                        }
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
            ++tc;
        }
        if (!ok && !*abort_v) fail();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                     : "memory");
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

// 3-D FP32 view {2K floats, rows, problems} of a complex operand; box
// {32 floats, box_rows, 1}.
bool make_map(CUtensorMap *m, const float2 *base, int K, int rows, int64_t ld, int nprob, int64_t stride,
              int box_rows, bool swizzle) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * (int64_t)K), (cuuint64_t)rows, (cuuint64_t)nprob};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 8), (cuuint64_t)((nprob > 1 ? stride : ld * rows) * 8)};
    const cuuint32_t box[3] = {32u, (cuuint32_t)box_rows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// The pipelined GEMM when its operands suit TMA (16-byte aligned bases, even
// leading dimensions and problem strides), else UNSUPPORTED.
ztoep_status_t launch_cgemm_tc2(const CgemmArgs &a, int nprob, int nsm, cudaStream_t s) {
    if (a.N < 1 || a.N > 256 || a.M < 1 || a.K < 1 || nprob < 1) return ZTOEP_ERR_ARG;
    if (!aligned16(a.A) || !aligned16(a.X) || (a.lda & 1) || (a.ldx & 1)) return ZTOEP_ERR_UNSUPPORTED;
    if (nprob > 1 && ((a.strideA & 1) || (a.strideX & 1))) return ZTOEP_ERR_UNSUPPORTED;
    G2Args g{};
    g.C = a.C;
    g.ldc_q = a.ldc_q;
    g.ldc_m = a.ldc_m;
    g.strideC = a.strideC;
    g.strideCk = a.strideCk;
    g.M = a.M;
    g.K = a.K;
    g.N = a.N;
    g.err = a.err;
    g.rp = std::min(G2_MAXRP, (a.N + 7) / 8 * 8);
    g.nchunk = (a.N + g.rp - 1) / g.rp;
    int kc = a.kchunk > 0 ? a.kchunk : a.K;
    kc = (kc + 15) / 16 * 16;
    g.kchunk = kc;
    g.ksplit = (a.K + kc - 1) / kc;
    g.mtiles = (a.M + 127) / 128;
    g.nprob = nprob;
    const size_t stage = 32768 + 640 * (size_t)g.rp;
    g.nstage = (int)std::min<size_t>(G2_MAXST, (G2_SMEM_CAP - 1024) / stage);
    if (g.nstage < 2) return ZTOEP_ERR_UNSUPPORTED;
    uint32_t cols = 32;
    while (cols < (uint32_t)(8 * g.rp)) cols <<= 1;
    g.tmem_cols = cols;
    CUtensorMap ma, mx;
    if (!make_map(&ma, a.A, a.K, a.M, a.lda, nprob, a.strideA, 128, true)) return ZTOEP_ERR_UNSUPPORTED;
    if (!make_map(&mx, a.X, a.K, a.N, a.ldx, nprob, a.strideX, g.rp, false)) return ZTOEP_ERR_UNSUPPORTED;
    const size_t smem = (size_t)g.nstage * stage + 1024;
    static bool attr = false;
    if (!attr) {
        ZT_CUDA(cudaFuncSetAttribute(k_cgemm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G2_SMEM_CAP));
        attr = true;
    }
    const int64_t items = (int64_t)nprob * g.nchunk * g.ksplit * g.mtiles;
    const int grid = (int)std::min<int64_t>(items, nsm);
    KScope ks(K_TENSOR_PIPE, s);
    k_cgemm_tc2<<<grid, G2_THREADS, smem, s>>>(ma, mx, g);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

}  // namespace ztoep
