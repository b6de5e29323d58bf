// Batched complex GEMM on the 5th-generation tensor cores (tcgen05, sm_100
// family) with 3xTF32 split products and FP32 accumulation in TMEM.
//
//   C_p[m][q] = sum_k A_p[m][k] X_p[q][k]      (complex, per problem p)
//
// A is the resident operand (row-major, k contiguous), X the batch operand
// ([q][k], k contiguous).  Complex arithmetic is mapped to one real GEMM: A's
// complex row i becomes the real rows 2i = (ar, -ai, ...) and 2i+1 =
// (ai, ar, ...) over the interleaved real k axis, X's complex row q is read as
// the real row (xr, xi, ...), so real row 2i of D is Re C[i][q] and row 2i+1
// is Im C[i][q].  Each real operand value v is split as hi = tf32(v),
// lo = tf32(v - hi) and D += Ahi Xhi + Ahi Xlo + Alo Xhi (the 3xTF32 scheme),
// which keeps the products close to FP32 accuracy.
//
// One CTA (4 warps) computes 64 complex rows (M = 128 real rows) x all N
// columns over a K range: every k-block of 16 complex (32 real, 128 bytes) is
// loaded by the threads, expanded, split and stored into 128-byte-swizzled
// K-major tiles in shared memory; one thread issues the MMAs and commits them
// to an mbarrier; the next k-block is staged while the MMAs run.  The
// accumulator (128 lanes x N columns FP32) lives in tensor memory and is read
// back with tcgen05.ld for the epilogue.
#include <algorithm>

#include "common.cuh"
#include "instrument.cuh"
#include "tcgemm.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace ztoep {

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_MC = 64;       // complex rows of A per CTA (128 real rows)
constexpr int TC_KC = 16;       // complex k per k-block (32 real = 128 bytes)
constexpr int TC_NST = 2;       // shared-memory stages
constexpr uint32_t TC_WAIT = 1u << 22;

// Stage layout (bytes, each tile 1024-aligned):
//   A_hi [128 rows][128 B], A_lo [128][128], X_hi [NP rows][128], X_lo [NP][128]
struct Stage {
    uint32_t a_hi, a_lo, x_hi, x_lo;
};

__device__ __forceinline__ Stage stage_at(uint32_t base, int s, int np) {
    const uint32_t a = 128 * 128, x = (uint32_t)np * 128;
    const uint32_t sz = 2 * a + 2 * x;
    Stage st;
    st.a_hi = base + s * sz;
    st.a_lo = st.a_hi + a;
    st.x_hi = st.a_lo + a;
    st.x_lo = st.x_hi + x;
    return st;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One 16-byte piece (two complex values at k, k+1) of row `row` of a complex
// matrix into shared memory; out-of-range values are zero-filled.
__device__ __forceinline__ void copy_pair(uint32_t dst, const float2 *rowp, bool row_ok, int k, int kend) {
    const float2 *src = rowp + k;
    const bool v0 = row_ok && k < kend, v1 = row_ok && k + 1 < kend;
    if (v0 && v1 && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
        cp_async16(dst, src, 16);
    } else {
        cp_async8(dst, v0 ? (const void *)src : (const void *)rowp, v0 ? 8u : 0u);
        cp_async8(dst + 8, v1 ? (const void *)(src + 1) : (const void *)rowp, v1 ? 8u : 0u);
    }
}

// Raw k-block (A: 64 complex rows x 16 complex k; X: np rows x 16 complex k)
// into a raw staging buffer, row-major, by asynchronous copies.
__device__ __forceinline__ void raw_issue(const CgemmArgs &g, const float2 *A, const float2 *X, int m0, int k0,
                                          int kend, uint32_t raw_a, uint32_t raw_x) {
    for (int idx = threadIdx.x; idx < TC_MC * 8; idx += blockDim.x) {
        const int i = idx >> 3, pr = idx & 7;
        const int m = m0 + i;
        const bool ok = m < g.M;
        copy_pair(raw_a + (uint32_t)(i * 128 + pr * 16), A + (int64_t)(ok ? m : 0) * g.lda, ok, k0 + 2 * pr, kend);
    }
    for (int idx = threadIdx.x; idx < g.np * 8; idx += blockDim.x) {
        const int q = idx >> 3, pr = idx & 7;
        const bool ok = q < g.N;
        copy_pair(raw_x + (uint32_t)(q * 128 + pr * 16), X + (int64_t)(ok ? q : 0) * g.ldx, ok, k0 + 2 * pr, kend);
    }
}

// Expand (complex row i -> real rows 2i = (ar, -ai), 2i+1 = (ai, ar)), split
// into TF32 hi/lo and store into the 128B-swizzled operand tiles.
__device__ __forceinline__ void stage_transform(const unsigned char *smem, uint32_t sbase, uint32_t raw_a,
                                                uint32_t raw_x, int np, const Stage &st) {
    unsigned char *sm = const_cast<unsigned char *>(smem);
    for (int idx = threadIdx.x; idx < TC_MC * 8; idx += blockDim.x) {
        const int i = idx >> 3, chunk = idx & 7;  // chunk = 2 complex = 4 real columns
        const float4 a = *reinterpret_cast<const float4 *>(sm + (raw_a - sbase) + i * 128 + chunk * 16);
        const float4 re = make_float4(a.x, -a.y, a.z, -a.w);
        const float4 im = make_float4(a.y, a.x, a.w, a.z);
        const float4 reh = tf32x4(re), imh = tf32x4(im);
        const float4 rel = tf32x4(sub4(re, reh)), iml = tf32x4(sub4(im, imh));
        const uint32_t o0 = sw128(2 * i, chunk), o1 = sw128(2 * i + 1, chunk);
        *reinterpret_cast<float4 *>(sm + (st.a_hi - sbase) + o0) = reh;
        *reinterpret_cast<float4 *>(sm + (st.a_lo - sbase) + o0) = rel;
        *reinterpret_cast<float4 *>(sm + (st.a_hi - sbase) + o1) = imh;
        *reinterpret_cast<float4 *>(sm + (st.a_lo - sbase) + o1) = iml;
    }
    for (int idx = threadIdx.x; idx < np * 8; idx += blockDim.x) {
        const int q = idx >> 3, chunk = idx & 7;
        const float4 v = *reinterpret_cast<const float4 *>(sm + (raw_x - sbase) + q * 128 + chunk * 16);
        const float4 h = tf32x4(v), l = tf32x4(sub4(v, h));
        const uint32_t o = sw128(q, chunk);
        *reinterpret_cast<float4 *>(sm + (st.x_hi - sbase) + o) = h;
        *reinterpret_cast<float4 *>(sm + (st.x_lo - sbase) + o) = l;
    }
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS) k_cgemm_tc(CgemmArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t done[TC_NST];
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    // 1024-byte aligned base for the swizzled tiles
    const uint32_t raw = smem_u32(tc_smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char *smem = tc_smem_raw + (sbase - raw);

    const int p = blockIdx.z;
    const int m0 = blockIdx.x * TC_MC;
    const int kbeg = blockIdx.y * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);
    const int nkb = (kend - kbeg + TC_KC - 1) / TC_KC;
    const int warp = threadIdx.x >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NST; ++s) mbar_init(&done[s], 1);
        mbar_fence_init();
        fail = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_tf32(g.np);

    const float2 *A = g.A + (int64_t)p * g.strideA;
    const float2 *X = g.X + (int64_t)p * g.strideX;
    const uint32_t opbytes = (uint32_t)TC_NST * (2 * 128 * 128 + 2 * (uint32_t)g.np * 128);
    const uint32_t rawa_sz = TC_MC * 128, rawx_sz = (uint32_t)g.np * 128;
    const uint32_t raw0 = sbase + opbytes;
    auto raw_a = [&](int r) { return raw0 + (uint32_t)r * (rawa_sz + rawx_sz); };
    const int nraw = g.nraw;
    for (int r = 0; r < nraw - 1; ++r) {  // prologue: k-blocks 0 .. nraw-2 in flight
        if (r < nkb) raw_issue(g, A, X, m0, kbeg + r * TC_KC, kend, raw_a(r), raw_a(r) + rawa_sz);
        cp_async_commit();
    }
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TC_NST;
        {  // keep nraw - 1 k-blocks ahead in flight
            const int kn = kb + nraw - 1;
            if (kn < nkb) {
                const int r = kn % nraw;
                raw_issue(g, A, X, m0, kbeg + kn * TC_KC, kend, raw_a(r), raw_a(r) + rawa_sz);
            }
            cp_async_commit();
        }
        if (nraw == 3) cp_async_wait<2>(); else cp_async_wait<1>();  // k-block kb has landed (this thread)
        if (kb >= TC_NST) {  // operand stage s is free once the MMAs of k-block kb - NST are done
            const bool ok = mbar_wait_bounded(&done[s], (uint32_t)(((kb / TC_NST) - 1) & 1), TC_WAIT);
            if (!ok) fail = 1;
        }
        if (__syncthreads_or(fail)) break;  // also makes every thread's raw copies visible
        const Stage st = stage_at(sbase, s, g.np);
        const int r = kb % nraw;
        stage_transform(smem, sbase, raw_a(r), raw_a(r) + rawa_sz, g.np, st);
        fence_proxy_async();  // generic-proxy stores -> visible to the tensor core
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {  // 4 x (K = 8 real = 32 bytes)
                const uint32_t off = ks * 32;
                const uint64_t ah = sdesc(st.a_hi + off), al = sdesc(st.a_lo + off);
                const uint64_t xh = sdesc(st.x_hi + off), xl = sdesc(st.x_lo + off);
                mma_tf32(tmem, ah, xh, idesc, (kb > 0 || ks > 0) ? 1 : 0);
                mma_tf32(tmem, ah, xl, idesc, 1);
                mma_tf32(tmem, al, xh, idesc, 1);
            }
            mma_commit(&done[s]);
        }
    }
    cp_async_wait<0>();
    // wait for the last commit (covers every earlier MMA)
    if (!fail && nkb > 0) {
        const int kb = nkb - 1;
        const bool ok = mbar_wait_bounded(&done[kb % TC_NST], (uint32_t)((kb / TC_NST) & 1), TC_WAIT);
        if (!ok) fail = 1;
    }
    const int failed = __syncthreads_or(fail);
    fence_after();
    if (failed) {
        if (threadIdx.x == 0) atomicOr(g.err, 2);
    } else {
        // epilogue: warp w holds real rows 32w..32w+31 (TMEM lanes), columns = q
        const int row = warp * 32 + (threadIdx.x & 31);
        const int i = row >> 1, c = row & 1;
        const int m = m0 + i;
        float *C = reinterpret_cast<float *>(g.C + (int64_t)p * g.strideC + (int64_t)blockIdx.y * g.strideCk);
        for (int q0 = 0; q0 < g.np; q0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)q0, r);
            if (m < g.M && nkb > 0) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int q = q0 + j;
                    if (q < g.N) C[2 * ((int64_t)q * g.ldc_q + (int64_t)m * g.ldc_m) + c] = __uint_as_float(r[j]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
}

static size_t op_bytes(int np) { return (size_t)TC_NST * (2 * 128 * 128 + 2 * (size_t)np * 128); }
static size_t raw_bytes(int np, int nraw) { return (size_t)nraw * ((size_t)TC_MC * 128 + (size_t)np * 128); }
constexpr size_t kSmemCap = 227 * 1024 - 2048;  // per-block limit minus static shared memory

size_t cgemm_smem_bytes(int np) { return op_bytes(np) + raw_bytes(np, 2) + 1024; }

bool cgemm_fits(int n) {
    int np = (n + 15) / 16 * 16;
    if (np < 32) np = 32;
    return n >= 1 && n <= 256 && cgemm_smem_bytes(np) <= kSmemCap;
}

ztoep_status_t launch_cgemm_tc(CgemmArgs g, int nprob, cudaStream_t s) {
    if (g.N < 1 || g.N > 256 || g.M < 1 || g.K < 1 || nprob < 1) return ZTOEP_ERR_ARG;
    g.np = (g.N + 15) / 16 * 16;  // N of the MMA: multiple of 16 for M = 128
    if (g.np < 32) g.np = 32;     // epilogue reads 32 columns at a time
    int cols = 32;
    while (cols < g.np) cols <<= 1;
    g.tmem_cols = cols;
    if (g.kchunk <= 0) g.kchunk = g.K;
    g.kchunk = (g.kchunk + TC_KC - 1) / TC_KC * TC_KC;
    g.nraw = op_bytes(g.np) + raw_bytes(g.np, 3) + 1024 <= kSmemCap ? 3 : 2;
    const size_t smem = op_bytes(g.np) + raw_bytes(g.np, g.nraw) + 1024;
    static bool attr = false;
    if (!attr) {
        ZT_CUDA(cudaFuncSetAttribute(k_cgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
        attr = true;
    }
    if (smem > kSmemCap) return ZTOEP_ERR_UNSUPPORTED;
    dim3 grid((g.M + TC_MC - 1) / TC_MC, (g.K + g.kchunk - 1) / g.kchunk, nprob);
    KScope ks(K_TENSOR, s);
    k_cgemm_tc<<<grid, TC_THREADS, smem, s>>>(g);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

}  // namespace ztoep
