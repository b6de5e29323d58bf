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
// CTA = 14 warps, one CTA per SM, persistent over work items (problem, RHS
// chunk of rp <= 64, K split, 128-row tile):
//   warp 0     TMA producer: the A tile (128 rows x 32 floats per k-block,
//              128B-swizzled boxes) and the raw X tile (rp rows) of two
//              k-blocks into a raw ring of NR stages (mbarrier full[r],
//              transaction bytes); a raw stage is refilled as soon as it has
//              been converted (rfree[r]), so up to NR loads are in flight
//              whatever the MMAs are doing;
//   warps 2-9  split A into hi and lo and write them to tensor memory (warp w
//              owns TMEM lanes 32 (w mod 4) .. +31, i.e. its rows, and half of
//              the k-block's columns; the swizzled raw box lets its 32 rows be
//              read without bank conflicts), expand and split X into [Xhi;
//              Xlo] (swizzled, shared memory), in one of NO = 2-3 operand
//              stages (once the MMAs that last read it are done, ofree[o]),
//              then arrive on rfree[r] and ready[o];
//   warp 1     one thread issues the MMAs of a k-block (A from tensor memory,
//              X from shared memory) and commits them to ofree[o] and, at the
//              end of an item, to accf[b];
//   warps 10-13 epilogue: tensor memory -> registers -> C, then acce[b]; the
//              accumulator is double-buffered when two buffers fit beside the
//              A stages (so an item's epilogue overlaps the next item's MMAs).
// Tensor memory: accumulator buffers of 4 rp columns, then 64 columns (A hi,
// A lo) per operand stage.
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

constexpr int G2_THREADS = 448;  // 14 warps
constexpr int G2_TW = 8;         // warps converting operands
constexpr int G2_MAXRP = 64;
constexpr int G2_MAXRAW = 8;
constexpr int G2_KPR = 2;  // k-blocks per raw stage (one TMA box per operand)
constexpr uint32_t G2_WAIT = 1u << 22;
constexpr size_t G2_SMEM_CAP = 227 * 1024 - 1024;  // per-block limit minus static shared memory
enum { G2_ERRBIT = 4 };

struct G2Args {
    float2 *C;
    int64_t ldc_q, ldc_m, strideC, strideCk;
    int M, K, N;         // complex sizes
    int rp;              // RHS rows per chunk (multiple of 8, <= 64)
    int nchunk, ksplit, mtiles, nprob, kchunk;
    int nraw;            // stages of the raw ring
    int nop;             // stages of the operand ring (2 or 3)
    int nacc;            // accumulator buffers in tensor memory (2, or 1 when they would not fit beside A)
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

// Round to TF32 (10 mantissa bits), nearest with ties away from zero: add half
// a TF32 unit to the magnitude bits and clear the 13 low bits (the IEEE
// layout is sign-magnitude, so this rounds the magnitude; a carry into the
// exponent is the correct round-up to the next binade).  Integer ops, so the
// split runs at full issue rate instead of the conversion unit's.
__device__ __forceinline__ float tf32_near(float v) {
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ float4 tf32n4(float4 v) {
    return make_float4(tf32_near(v.x), tf32_near(v.y), tf32_near(v.z), tf32_near(v.w));
}

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
    __shared__ __align__(8) uint64_t full[G2_MAXRAW], rfree[G2_MAXRAW], ready[3], ofree[3], accf[2], acce[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint32_t raw = smem_u32(g2_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *smem = g2_smem_raw + (base - raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NR = g.nraw, NO = g.nop, rp = g.rp;
    // operand ring (NO stages, one k-block each): X expanded [4 rp][128 B]
    //   (128B-swizzled K-major) in shared memory; A hi and A lo [128 lanes][32
    //   columns] each in tensor memory after the accumulators
    // raw ring (NR stages, G2_KPR k-blocks each, as loaded): A as G2_KPR
    //   128B-swizzled [128][128 B] boxes | X [rp][G2_KPR x 128 B] row-major
    constexpr uint32_t RW = 128u * G2_KPR;  // bytes of a raw X row
    const uint32_t op_bytes = 512u * (uint32_t)rp, raw_bytes = (128u + (uint32_t)rp) * RW;
    auto x_exp = [&](int o) { return base + (uint32_t)o * op_bytes; };
    auto a_raw = [&](int r) { return base + (uint32_t)NO * op_bytes + (uint32_t)r * raw_bytes; };
    auto x_raw = [&](int r) { return a_raw(r) + 128u * RW; };
    const uint32_t acol0 = (uint32_t)(g.nacc * 4 * rp);                   // first A column in tensor memory
    auto a_col = [&](int o) { return acol0 + (uint32_t)o * 64u; };  // hi: +0..31, lo: +32..63

    if (threadIdx.x == 0) {
        for (int r = 0; r < NR; ++r) {
            mbar_init(&full[r], 1);
            mbar_init(&rfree[r], G2_TW);
        }
        for (int o = 0; o < NO; ++o) {
            mbar_init(&ready[o], G2_TW);
            mbar_init(&ofree[o], 1);
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
        if (lane == 0) {  // ---------------- producer: raw ring
            const uint32_t tx = raw_bytes;
            uint32_t kbg = 0;  // raw stages issued
            bool ok = true;
            for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
                const Item w = decode(g, it);
                for (int kb = 0; kb < w.nkb; kb += G2_KPR) {
                    const int r = (int)(kbg % NR);
                    const uint32_t n = kbg / NR;
                    if (n > 0 && !mbar_wait_bounded(&rfree[r], (n - 1) & 1, G2_WAIT)) {
                        ok = false;
                        break;
                    }
                    if (*abort_v) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[r], tx);
                    const int kx = 2 * (w.k0 + kb * 16);
                    for (int sb = 0; sb < G2_KPR; ++sb)
                        tma_load_3d(a_raw(r) + (uint32_t)sb * 16384u, &tmA, kx + 32 * sb, w.mt * 128, w.p, &full[r]);
                    tma_load_3d(x_raw(r), &tmX, kx, w.c * rp, w.p, &full[r]);
                    ++kbg;
                }
            }
            if (!ok && !*abort_v) fail();
            // no copy may still be landing when the CTA leaves
            for (int r = 0; r < NR; ++r) {
                if (kbg <= (uint32_t)r) continue;
                const uint32_t cnt = (kbg - (uint32_t)r + NR - 1) / NR;  // copies issued into stage r
                if (!mbar_wait_bounded(&full[r], (cnt - 1) & 1, G2_WAIT)) fail();
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------- MMA issuer: operand ring
            const uint32_t id_wide = idesc_tf32(4 * rp), id_half = idesc_tf32(2 * rp);
            uint32_t kbg = 0, tc = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
                const Item w = decode(g, it);
                const int b = (int)(tc % (uint32_t)g.nacc);
                const uint32_t u = tc / (uint32_t)g.nacc;
                if (u > 0 && !mbar_wait_bounded(&acce[b], (u - 1) & 1, G2_WAIT)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 4 * rp);
                for (int kb = 0; kb < w.nkb; ++kb) {
                    const int o = (int)(kbg % NO);
                    if (*abort_v || !mbar_wait_bounded(&ready[o], (kbg / NO) & 1, G2_WAIT)) {
                        ok = false;
                        break;
                    }
                    fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {  // 4 x (K = 8 real = 32 bytes, 8 columns)
                        const uint64_t xb = sdesc(x_exp(o) + ks * 32);
                        const uint32_t ac = tmem + a_col(o) + 8u * ks;
                        mma_tf32_ta(d, ac, xb, id_wide, (kb > 0 || ks > 0) ? 1 : 0);
                        mma_tf32_ta(d, ac + 32u, xb, id_half, 1);
                    }
                    mma_commit(&ofree[o]);
                    ++kbg;
                }
                if (!ok) break;
                mma_commit(&accf[b]);
                ++tc;
            }
            if (!ok && !*abort_v) fail();
        }
    } else if (warp < 2 + G2_TW) {  // ---------------- raw -> operands (G2_TW warps)
        constexpr int NT = 32 * G2_TW;
        const int t = threadIdx.x - 64;
        // A: this warp's lane quarter (its tensor-memory lanes) and half of the
        // k-block's 32 reals; the thread's row is read from the swizzled raw box
        // (16-byte chunk c of row a at chunk c ^ (a mod 8): a warp's 32 rows hit
        // distinct banks)
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int arow = 32 * quarter + lane;
        const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
        // X: this thread's (row, 16-byte chunk) pieces: offsets in the raw
        // row-major tile and in the swizzled operand tile, fixed for the kernel
        constexpr int XP = (G2_MAXRP * 8 + NT - 1) / NT;
        uint32_t xi[XP], xo[XP][4];
#pragma unroll
        for (int k = 0; k < XP; ++k) {
            const int i = t + k * NT, q = i >> 3, ch = i & 7;
            xi[k] = (uint32_t)q * RW + (uint32_t)ch * 16u;
            xo[k][0] = sw128(2 * q, ch);
            xo[k][1] = sw128(2 * q + 1, ch);
            xo[k][2] = sw128(2 * rp + 2 * q, ch);
            xo[k][3] = sw128(2 * rp + 2 * q + 1, ch);
        }
        uint32_t rg = 0, kbg = 0;  // raw stages and k-blocks consumed
        bool ok = true;
        for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const Item w = decode(g, it);
            for (int kb0 = 0; kb0 < w.nkb && ok; kb0 += G2_KPR) {
                const int r = (int)(rg % NR);
                if (*abort_v || !mbar_wait_bounded(&full[r], (rg / NR) & 1, G2_WAIT)) {
                    ok = false;
                    break;
                }
                const unsigned char *ar = smem + (a_raw(r) - base);
                const unsigned char *xr = smem + (x_raw(r) - base);
                for (int sub = 0; sub < G2_KPR && kb0 + sub < w.nkb; ++sub) {
                    const int o = (int)(kbg % NO);
                    const uint32_t no = kbg / NO;
                    if (no > 0 && !mbar_wait_bounded(&ofree[o], (no - 1) & 1, G2_WAIT)) {
                        ok = false;
                        break;
                    }
                    fence_after();  // the MMAs that read stage o are complete before it is rewritten
                    const uint32_t so = (uint32_t)sub * 128u;
                    {
                        const unsigned char *arow_p = ar + sub * 16384 + arow * 128;
                        uint32_t hi[16], lo[16];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int ch = 4 * half + c;
                            const float4 v = *reinterpret_cast<const float4 *>(arow_p + ((ch ^ (arow & 7)) << 4));
                            const float4 h = tf32n4(v), l = tf32n4(sub4(v, h));
                            hi[4 * c] = __float_as_uint(h.x);
                            hi[4 * c + 1] = __float_as_uint(h.y);
                            hi[4 * c + 2] = __float_as_uint(h.z);
                            hi[4 * c + 3] = __float_as_uint(h.w);
                            lo[4 * c] = __float_as_uint(l.x);
                            lo[4 * c + 1] = __float_as_uint(l.y);
                            lo[4 * c + 2] = __float_as_uint(l.z);
                            lo[4 * c + 3] = __float_as_uint(l.w);
                        }
                        const uint32_t ta = tmem + tlane + a_col(o) + 16u * half;
                        tmem_st16(ta, hi);
                        tmem_st16(ta + 32u, lo);
                    }
                    unsigned char *xe = smem + (x_exp(o) - base);
#pragma unroll
                    for (int k = 0; k < XP; ++k) {
                        if (t + k * NT < rp * 8) {
                            const float4 v = *reinterpret_cast<const float4 *>(xr + xi[k] + so);  // (xr0, xi0, xr1, xi1)
                            const float4 re = make_float4(v.x, -v.y, v.z, -v.w);
                            const float4 im = make_float4(v.y, v.x, v.w, v.z);
                            const float4 rh = tf32n4(re), ih = tf32n4(im);
                            *reinterpret_cast<float4 *>(xe + xo[k][0]) = rh;
                            *reinterpret_cast<float4 *>(xe + xo[k][1]) = ih;
                            *reinterpret_cast<float4 *>(xe + xo[k][2]) = tf32n4(sub4(re, rh));
                            *reinterpret_cast<float4 *>(xe + xo[k][3]) = tf32n4(sub4(im, ih));
                        }
                    }
                    fence_proxy_async();  // generic-proxy stores -> visible to the tensor core
                    tmem_st_wait();       // the warp's tensor-memory stores have landed
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ready[o]);
                    ++kbg;
                }
                if (!ok) break;
                __syncwarp();
                if (lane == 0) mbar_arrive(&rfree[r]);  // raw stage read (its values are in the stores above)
                ++rg;
            }
        }
        if (!ok && !*abort_v) fail();
    } else {  // ---------------- epilogue (4 warps: TMEM lane quarters warp % 4)
        const int q4 = warp & 3;
        const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
        uint32_t tc = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const Item w = decode(g, it);
            const int b = (int)(tc % (uint32_t)g.nacc);
            const uint32_t u = tc / (uint32_t)g.nacc;
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
// {box_inner floats, box_rows, 1}, 128B-swizzled or not.
bool make_map(CUtensorMap *m, const float2 *base, int K, int rows, int64_t ld, int nprob, int64_t stride,
              int box_inner, int box_rows, bool swizzle) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * (int64_t)K), (cuuint64_t)rows, (cuuint64_t)nprob};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 8), (cuuint64_t)((nprob > 1 ? stride : ld * rows) * 8)};
    const cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, 1u};
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
    const size_t op_bytes = 512 * (size_t)g.rp, raw_bytes = (128 + (size_t)g.rp) * 128 * G2_KPR;
    if (G2_SMEM_CAP < 1024 + 2 * op_bytes + 2 * raw_bytes) return ZTOEP_ERR_UNSUPPORTED;
    // three operand stages when four raw stages still fit beside them
    g.nop = G2_SMEM_CAP >= 1024 + 3 * op_bytes + 4 * raw_bytes ? 3 : 2;
    g.nraw = (int)std::min<size_t>(G2_MAXRAW, (G2_SMEM_CAP - 1024 - g.nop * op_bytes) / raw_bytes);
    // tensor memory: the accumulators (two buffers when A's stages still fit
    // beside them, so an item's epilogue overlaps the next item's MMAs), then
    // 64 columns (A hi, A lo) per operand stage
    g.nacc = 2 * 4 * g.rp + 64 * g.nop <= 512 ? 2 : 1;
    uint32_t cols = 32;
    while (cols < (uint32_t)(g.nacc * 4 * g.rp + 64 * g.nop)) cols <<= 1;
    if (cols > 512) return ZTOEP_ERR_UNSUPPORTED;
    g.tmem_cols = cols;
    CUtensorMap ma, mx;
    if (!make_map(&ma, a.A, a.K, a.M, a.lda, nprob, a.strideA, 32, 128, true)) return ZTOEP_ERR_UNSUPPORTED;
    if (!make_map(&mx, a.X, a.K, a.N, a.ldx, nprob, a.strideX, 32 * G2_KPR, g.rp, false))
        return ZTOEP_ERR_UNSUPPORTED;
    const size_t smem = (size_t)g.nop * op_bytes + (size_t)g.nraw * raw_bytes + 1024;
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
