// Batched restarted GMRES inside an FP64 iterative-refinement loop for
// Z' X = V (Sec. II, Eq. MoMMatrixEq; Sec. II-D names GMRES on the
// second-level Toeplitz structure of A, with the FFT product for Z').
//
// Outer sweep (FP64):  r = v - Z' x (FP64 product), ||r|| per RHS, stop test.
// Inner cycle:         GMRES(m) on Z' d = r, Arnoldi by classical
//                      Gram-Schmidt with one reorthogonalisation (CGS2,
//                      Giraud, Langou & Rozloznik 2005), Givens rotations,
//                      least squares R y = g, x <- x + V y.  The products inside
//                      the cycle are FP32 (MIXED) or FP64 (FP64); the Arnoldi,
//                      rotations and updates are always FP64.
// Every kernel is batched over the RHS (grid.y) and each RHS stops on its own
// flag.  Cross-CTA reductions use the last-CTA-done pattern (atomic ticket,
// no waiting), so the summation order is fixed and results are reproducible.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {

enum { ST_ACTIVE = 0, ST_JLEN = 1, ST_ITERS = 2, ST_STATUS = 3, ST_OUTER = 4, ST_PENDING = 5, ST_STRIDE = 8 };
enum { RS_RUNNING = 0, RS_CONVERGED = 1, RS_NONFINITE = 2, RS_MAXITER = 3 };
enum { NM_VNORM = 0, NM_BETA0 = 1, NM_TARGET = 2, NM_RNORM = 3, NM_BETA = 4, NM_STRIDE = 8 };
enum { CNT_STRIDE = 4 };

struct GArgs {
    double2 *Vb, *w, *r, *x;
    const double2 *v;
    float2 *x32;
    const float2 *y32;
    double2 *H, *cs, *sn, *g, *y, *h1, *h2, *part;
    double *nrm;
    int *st;
    unsigned *cnt;
    int64_t N;
    int cap, m, nchunk, pstride;
    int mixed;
    double tol, inner_tol;
    int max_iter;
};

constexpr int NT_ = 256;       // threads per CTA
constexpr int NW_ = NT_ / 32;  // warps per CTA
constexpr int KG = 8;          // basis vectors per register group

__device__ __forceinline__ double2 wsum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Sum v[0..K) over the CTA; the totals land in red[0..K).
template <int K> __device__ __forceinline__ void block_sum(double2 (&v)[K], double2 *red /*[NW_][K]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = wsum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
        double2 s = red[threadIdx.x];
        for (int w = 1; w < NW_; ++w) s = s + red[w * K + threadIdx.x];
        red[threadIdx.x] = s;  // each thread reads only column threadIdx.x, rows >= 1 already read
    }
    __syncthreads();
}

// Last-CTA-done ticket for the CTAs of one RHS (no waiting).
__device__ __forceinline__ bool last_cta(unsigned *cnt, unsigned total) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(cnt, 1u);
        s_last = (t == total - 1);
        if (s_last) *cnt = 0;  // reset for the next use; nobody else touches it in this launch
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// In the last CTA: out[k] = sum_c part[c][k] for k < K (one warp per k).
__device__ __forceinline__ void reduce_partials(const double2 *part, int nchunk, int pstride, int K,
                                                double2 *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < K; k += NW_) {
        double2 s = make_double2(0, 0);
        for (int c = lane; c < nchunk; c += 32) {
            const double2 pv = __ldcg(part + (int64_t)c * pstride + k);
            s = s + pv;
        }
        s = wsum(s);
        if (lane == 0) out[k] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double2 *basis(const GArgs &a, int k, int rr) {
    return a.Vb + ((int64_t)k * a.cap + rr) * a.N;
}

// ---------------------------------------------------------------- norms
// ||v|| per RHS -> nrm[VNORM].
template <int ELEM> __global__ void __launch_bounds__(NT_) k_vnorm(GArgs a) {
    __shared__ double2 red[NW_];
    const int rr = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
    double2 acc[1] = {make_double2(0, 0)};
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        if (idx < a.N) {
            const double2 t = a.v[(int64_t)rr * a.N + idx];
            acc[0].x += t.x * t.x + t.y * t.y;
        }
    }
    block_sum<1>(acc, red);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = red[0];
    if (last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) {
        __shared__ double2 tot[1];
        reduce_partials(part, a.nchunk, a.pstride, 1, tot);
        if (threadIdx.x == 0) a.nrm[rr * NM_STRIDE + NM_VNORM] = sqrt(tot[0].x);
    }
}

// r = v - r (r holds Z' x) or r = v (zero guess); ||r||, stop test, start of a cycle.
template <int ELEM> __global__ void __launch_bounds__(NT_) k_residual(GArgs a, int zero) {
    __shared__ double2 red[NW_];
    const int rr = blockIdx.y;
    int *st = a.st + rr * ST_STRIDE;
    if (st[ST_STATUS] != RS_RUNNING) return;
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
    double2 acc[1] = {make_double2(0, 0)};
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        if (idx < a.N) {
            const int64_t o = (int64_t)rr * a.N + idx;
            const double2 t = zero ? a.v[o] : a.v[o] - a.r[o];
            a.r[o] = t;
            acc[0].x += t.x * t.x + t.y * t.y;
        }
    }
    block_sum<1>(acc, red);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = red[0];
    if (last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) {
        __shared__ double2 tot[1];
        reduce_partials(part, a.nchunk, a.pstride, 1, tot);
        if (threadIdx.x == 0) {
            double *nm = a.nrm + rr * NM_STRIDE;
            const double vn = nm[NM_VNORM], rn = sqrt(tot[0].x);
            nm[NM_RNORM] = rn;
            st[ST_OUTER] += 1;
            st[ST_PENDING] = 0;
            st[ST_JLEN] = 0;
            st[ST_ACTIVE] = 0;
            if (!isfinite(vn) || !isfinite(rn)) {
                st[ST_STATUS] = RS_NONFINITE;
            } else if (rn <= a.tol * vn || rn == 0.0) {
                st[ST_STATUS] = RS_CONVERGED;
            } else if (st[ST_ITERS] >= a.max_iter) {
                st[ST_STATUS] = RS_MAXITER;
            } else {
                st[ST_ACTIVE] = 1;
                nm[NM_BETA0] = rn;
                const double floor_abs = 0.5 * a.tol * vn;
                nm[NM_TARGET] = a.mixed ? fmax(a.inner_tol * rn, floor_abs) : floor_abs;
                double2 *g = a.g + (int64_t)rr * (a.m + 1);
                g[0] = make_double2(rn, 0);
                for (int i = 1; i <= a.m; ++i) g[i] = make_double2(0, 0);
            }
        }
    }
}

// V[0] = r / beta0 (and its FP32 copy for the inner product).
template <int ELEM> __global__ void __launch_bounds__(NT_) k_start(GArgs a) {
    const int rr = blockIdx.y;
    if (!a.st[rr * ST_STRIDE + ST_ACTIVE]) return;
    const double inv = 1.0 / a.nrm[rr * NM_STRIDE + NM_BETA0];
    double2 *v0 = basis(a, 0, rr);
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        if (idx < a.N) {
            const double2 t = cscale(a.r[(int64_t)rr * a.N + idx], inv);
            v0[idx] = t;
            if (a.mixed) a.x32[(int64_t)rr * a.N + idx] = make_float2((float)t.x, (float)t.y);
        }
    }
}

// ---------------------------------------------------------------- Arnoldi
// Partial sums of conj(V_k) . w for k <= j over this CTA's elements -> part.
template <int ELEM>
__device__ __forceinline__ void dots_partial(const GArgs &a, int rr, int j, const double2 (&wv)[ELEM],
                                             int64_t base, double2 *part, double2 *red) {
    for (int k0 = 0; k0 <= j; k0 += KG) {
        double2 acc[KG];
#pragma unroll
        for (int kk = 0; kk < KG; ++kk) acc[kk] = make_double2(0, 0);
#pragma unroll
        for (int kk = 0; kk < KG; ++kk) {
            if (k0 + kk <= j) {
                const double2 *vk = basis(a, k0 + kk, rr);
#pragma unroll
                for (int e = 0; e < ELEM; ++e) {
                    const int64_t idx = base + e * NT_ + threadIdx.x;
                    if (idx < a.N) acc[kk] = cfmac(vk[idx], wv[e], acc[kk]);
                }
            }
        }
        block_sum<KG>(acc, red);
        if (threadIdx.x < KG && k0 + threadIdx.x <= j)
            part[(int64_t)blockIdx.x * a.pstride + k0 + threadIdx.x] = red[threadIdx.x];
        __syncthreads();
    }
}

// First Gram-Schmidt pass: w <- product output (widened), h1 = V^H w.
template <int ELEM> __global__ void __launch_bounds__(NT_) k_gs1(GArgs a, int j) {
    __shared__ double2 red[NW_ * KG];
    const int rr = blockIdx.y;
    if (!a.st[rr * ST_STRIDE + ST_ACTIVE]) return;
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
    double2 wv[ELEM];
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        wv[e] = make_double2(0, 0);
        if (idx < a.N) {
            const int64_t o = (int64_t)rr * a.N + idx;
            if (a.mixed) {
                const float2 t = a.y32[o];
                wv[e] = make_double2(t.x, t.y);
                a.w[o] = wv[e];
            } else {
                wv[e] = a.w[o];
            }
        }
    }
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    dots_partial<ELEM>(a, rr, j, wv, base, part, red);
    if (last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk))
        reduce_partials(part, a.nchunk, a.pstride, j + 1, a.h1 + (int64_t)rr * (a.m + 1));
}

// w <- w - V h (h from the previous pass); optionally h2 = V^H w (second pass)
// or the partial ||w||^2.
template <int ELEM, bool SECOND>
__global__ void __launch_bounds__(NT_) k_gs_update(GArgs a, int j) {
    __shared__ double2 red[NW_ * KG];
    __shared__ double2 hs[129];
    const int rr = blockIdx.y;
    if (!a.st[rr * ST_STRIDE + ST_ACTIVE]) return;
    const double2 *h = (SECOND ? a.h1 : a.h2) + (int64_t)rr * (a.m + 1);
    for (int k = threadIdx.x; k <= j; k += NT_) hs[k] = __ldcg(h + k);
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
    double2 wv[ELEM];
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        wv[e] = make_double2(0, 0);
        if (idx < a.N) wv[e] = a.w[(int64_t)rr * a.N + idx];
    }
    for (int k = 0; k <= j; ++k) {
        const double2 hk = hs[k];
        const double2 *vk = basis(a, k, rr);
#pragma unroll
        for (int e = 0; e < ELEM; ++e) {
            const int64_t idx = base + e * NT_ + threadIdx.x;
            if (idx < a.N) wv[e] = wv[e] - cmul(hk, vk[idx]);
        }
    }
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        if (idx < a.N) a.w[(int64_t)rr * a.N + idx] = wv[e];
    }
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (SECOND) {
        dots_partial<ELEM>(a, rr, j, wv, base, part, red);
        if (last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk))
            reduce_partials(part, a.nchunk, a.pstride, j + 1, a.h2 + (int64_t)rr * (a.m + 1));
        return;
    }
    double2 acc[1] = {make_double2(0, 0)};
#pragma unroll
    for (int e = 0; e < ELEM; ++e) acc[0].x += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
    block_sum<1>(acc, red);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = red[0];
    if (!last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) return;
    __shared__ double2 tot[1];
    reduce_partials(part, a.nchunk, a.pstride, 1, tot);
    if (threadIdx.x != 0) return;
    // Hessenberg column j, Givens rotations, residual estimate (one thread).
    const int m = a.m;
    int *st = a.st + rr * ST_STRIDE;
    double *nm = a.nrm + rr * NM_STRIDE;
    double2 *H = a.H + (int64_t)rr * (m + 1) * m;
    double2 *cs = a.cs + (int64_t)rr * m, *sn = a.sn + (int64_t)rr * m;
    double2 *g = a.g + (int64_t)rr * (m + 1);
    const double2 *h1 = a.h1 + (int64_t)rr * (m + 1), *h2 = a.h2 + (int64_t)rr * (m + 1);
    const double beta = sqrt(tot[0].x);
    nm[NM_BETA] = beta;
    for (int i = 0; i <= j; ++i) H[i * m + j] = __ldcg(h1 + i) + __ldcg(h2 + i);
    for (int i = 0; i < j; ++i) {
        const double2 p = H[i * m + j], q = H[(i + 1) * m + j];
        H[i * m + j] = cmulc(cs[i], p) + cmulc(sn[i], q);
        H[(i + 1) * m + j] = cmul(cs[i], q) - cmul(sn[i], p);
    }
    const double2 p = H[j * m + j];
    const double d = sqrt(cabs2(p) + beta * beta);
    if (d > 0) {
        cs[j] = cscale(p, 1.0 / d);
        sn[j] = make_double2(beta / d, 0);
    } else {
        cs[j] = make_double2(1, 0);
        sn[j] = make_double2(0, 0);
    }
    H[j * m + j] = make_double2(d, 0);
    const double2 gj = g[j];
    g[j + 1] = make_double2(-sn[j].x * gj.x, -sn[j].x * gj.y);
    g[j] = cmulc(cs[j], gj);
    st[ST_JLEN] = j + 1;
    st[ST_ITERS] += 1;
    const double res = sqrt(cabs2(g[j + 1]));
    const bool end = !(res > nm[NM_TARGET]) || !(beta > 0) || (j + 1 == m) || (st[ST_ITERS] >= a.max_iter);
    if (end) {
        // least squares: R y = g (R upper triangular, (j+1) x (j+1))
        double2 *y = a.y + (int64_t)rr * m;
        for (int i = j; i >= 0; --i) {
            double2 s = g[i];
            for (int l = i + 1; l <= j; ++l) s = s - cmul(H[i * m + l], y[l]);
            y[i] = (H[i * m + i].x != 0.0 || H[i * m + i].y != 0.0) ? cdiv(s, H[i * m + i]) : make_double2(0, 0);
        }
        st[ST_ACTIVE] = 0;
        st[ST_PENDING] = 1;
    }
}

// V[j+1] = w / beta (and its FP32 copy).
template <int ELEM> __global__ void __launch_bounds__(NT_) k_normalize(GArgs a, int j) {
    const int rr = blockIdx.y;
    if (!a.st[rr * ST_STRIDE + ST_ACTIVE]) return;
    const double inv = 1.0 / a.nrm[rr * NM_STRIDE + NM_BETA];
    double2 *vn = basis(a, j + 1, rr);
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        if (idx < a.N) {
            const double2 t = cscale(a.w[(int64_t)rr * a.N + idx], inv);
            vn[idx] = t;
            if (a.mixed) a.x32[(int64_t)rr * a.N + idx] = make_float2((float)t.x, (float)t.y);
        }
    }
}

// x <- x + V y for RHS whose cycle produced an update.
template <int ELEM> __global__ void __launch_bounds__(NT_) k_update_x(GArgs a) {
    __shared__ double2 ys[128];
    const int rr = blockIdx.y;
    const int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_PENDING]) return;
    const int jl = st[ST_JLEN];
    for (int k = threadIdx.x; k < jl; k += NT_) ys[k] = __ldcg(a.y + (int64_t)rr * a.m + k);
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * NT_ * ELEM;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + e * NT_ + threadIdx.x;
        if (idx < a.N) {
            double2 s = a.x[(int64_t)rr * a.N + idx];
            for (int k = 0; k < jl; ++k) s = cfma(ys[k], basis(a, k, rr)[idx], s);
            a.x[(int64_t)rr * a.N + idx] = s;
        }
    }
}

// ---------------------------------------------------------------- workspace
void free_solve_ws(ztoep_plan_t p) {
    SolveWs &w = p->sws;
    cudaFree(w.Vb); cudaFree(w.w); cudaFree(w.r); cudaFree(w.H); cudaFree(w.cs); cudaFree(w.sn);
    cudaFree(w.g); cudaFree(w.y); cudaFree(w.h1); cudaFree(w.h2); cudaFree(w.part); cudaFree(w.nrm);
    cudaFree(w.st); cudaFree(w.cnt);
    if (w.hst) cudaFreeHost(w.hst);
    if (w.hnrm) cudaFreeHost(w.hnrm);
    w = SolveWs{};
}

static int elem_for(int64_t N, int nsm) {
    // 1 element per thread for small systems, 4 for large ones.  Depends on N
    // only, so a RHS is summed in the same order alone and in any batch.
    const int64_t ctas1 = (N + NT_ - 1) / NT_;
    return ctas1 >= 8LL * nsm ? 4 : 1;
}

static ztoep_status_t ensure_solve_ws(ztoep_plan_t p, int nrhs, int m) {
    SolveWs &w = p->sws;
    if (w.cap >= nrhs && w.m >= m) return ZTOEP_OK;
    free_solve_ws(p);
    const int64_t N = p->N;
    const int nchunk = (int)((N + NT_ - 1) / NT_);  // upper bound (ELEM = 1)
    const int pstride = m + 2;
    size_t acc = 0;
    ZT_TRY(dalloc((void **)&w.Vb, sizeof(double2) * (size_t)(m + 1) * nrhs * N, &acc));
    ZT_TRY(dalloc((void **)&w.w, sizeof(double2) * (size_t)nrhs * N, &acc));
    ZT_TRY(dalloc((void **)&w.r, sizeof(double2) * (size_t)nrhs * N, &acc));
    ZT_TRY(dalloc((void **)&w.H, sizeof(double2) * (size_t)nrhs * (m + 1) * m, &acc));
    ZT_TRY(dalloc((void **)&w.cs, sizeof(double2) * (size_t)nrhs * m, &acc));
    ZT_TRY(dalloc((void **)&w.sn, sizeof(double2) * (size_t)nrhs * m, &acc));
    ZT_TRY(dalloc((void **)&w.g, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.y, sizeof(double2) * (size_t)nrhs * m, &acc));
    ZT_TRY(dalloc((void **)&w.h1, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.h2, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.part, sizeof(double2) * (size_t)nrhs * nchunk * pstride, &acc));
    ZT_TRY(dalloc((void **)&w.nrm, sizeof(double) * (size_t)nrhs * NM_STRIDE, &acc));
    ZT_TRY(dalloc((void **)&w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE, &acc));
    ZT_TRY(dalloc((void **)&w.cnt, sizeof(unsigned) * (size_t)nrhs * CNT_STRIDE, &acc));
    ZT_CUDA(cudaMemset(w.cnt, 0, sizeof(unsigned) * (size_t)nrhs * CNT_STRIDE));
    ZT_CUDA(cudaMallocHost((void **)&w.hst, sizeof(int) * (size_t)nrhs * ST_STRIDE));
    ZT_CUDA(cudaMallocHost((void **)&w.hnrm, sizeof(double) * (size_t)nrhs * NM_STRIDE));
    w.cap = nrhs;
    w.m = m;
    w.bytes = acc;
    return ZTOEP_OK;
}

template <int ELEM> struct Launch {
    static ztoep_status_t vnorm(const GArgs &a, dim3 g, cudaStream_t s) { KScope ks(K_MISC, s); k_vnorm<ELEM><<<g, NT_, 0, s>>>(a); return ok(); }
    static ztoep_status_t residual(const GArgs &a, dim3 g, int zero, cudaStream_t s) { KScope ks(K_MISC, s); k_residual<ELEM><<<g, NT_, 0, s>>>(a, zero); return ok(); }
    static ztoep_status_t start(const GArgs &a, dim3 g, cudaStream_t s) { KScope ks(K_MISC, s); k_start<ELEM><<<g, NT_, 0, s>>>(a); return ok(); }
    static ztoep_status_t arnoldi(const GArgs &a, dim3 g, int j, cudaStream_t s) {
        KScope ks(K_ARNOLDI, s);
        ks.add(4);
        k_gs1<ELEM><<<g, NT_, 0, s>>>(a, j);
        k_gs_update<ELEM, true><<<g, NT_, 0, s>>>(a, j);
        k_gs_update<ELEM, false><<<g, NT_, 0, s>>>(a, j);
        k_normalize<ELEM><<<g, NT_, 0, s>>>(a, j);
        return ok();
    }
    static ztoep_status_t update_x(const GArgs &a, dim3 g, cudaStream_t s) { KScope ks(K_MISC, s); k_update_x<ELEM><<<g, NT_, 0, s>>>(a); return ok(); }
    static ztoep_status_t ok() { ZT_CUDA(cudaGetLastError()); return ZTOEP_OK; }
};

struct Ops {
    int elem;
    dim3 grid;
    ztoep_status_t vnorm(const GArgs &a, cudaStream_t s) const { return elem == 4 ? Launch<4>::vnorm(a, grid, s) : Launch<1>::vnorm(a, grid, s); }
    ztoep_status_t residual(const GArgs &a, int zero, cudaStream_t s) const { return elem == 4 ? Launch<4>::residual(a, grid, zero, s) : Launch<1>::residual(a, grid, zero, s); }
    ztoep_status_t start(const GArgs &a, cudaStream_t s) const { return elem == 4 ? Launch<4>::start(a, grid, s) : Launch<1>::start(a, grid, s); }
    ztoep_status_t arnoldi(const GArgs &a, int j, cudaStream_t s) const { return elem == 4 ? Launch<4>::arnoldi(a, grid, j, s) : Launch<1>::arnoldi(a, grid, j, s); }
    ztoep_status_t update_x(const GArgs &a, cudaStream_t s) const { return elem == 4 ? Launch<4>::update_x(a, grid, s) : Launch<1>::update_x(a, grid, s); }
};

static ztoep_status_t solve_impl(ztoep_plan_t p, const ztoep_solve_opts_t *o, int nrhs, const double2 *V,
                                 double2 *X, ztoep_solve_info_t *info, cudaStream_t s) {
    const auto t_start = std::chrono::steady_clock::now();
    const int m = o->restart;
    const bool mixed = o->prec == ZTOEP_MIXED;
    ZT_TRY(ensure_solve_ws(p, nrhs, m));
    if (mixed) ZT_TRY(ensure_ws<float>(p, nrhs));
    ZT_TRY(ensure_ws<double>(p, nrhs));
    SolveWs &w = p->sws;
    const int elem = elem_for(p->N, p->nsm);
    const int nchunk = (int)((p->N + (int64_t)NT_ * elem - 1) / ((int64_t)NT_ * elem));
    GArgs a{};
    a.Vb = w.Vb; a.w = w.w; a.r = w.r; a.x = X; a.v = V;
    a.x32 = (float2 *)p->ws32.xin; a.y32 = (const float2 *)p->ws32.yout;
    a.H = w.H; a.cs = w.cs; a.sn = w.sn; a.g = w.g; a.y = w.y; a.h1 = w.h1; a.h2 = w.h2; a.part = w.part;
    a.nrm = w.nrm; a.st = w.st; a.cnt = w.cnt;
    a.N = p->N; a.cap = w.cap; a.m = m; a.nchunk = nchunk; a.pstride = w.m + 2;
    a.mixed = mixed ? 1 : 0;
    a.tol = o->tol; a.inner_tol = o->inner_tol; a.max_iter = o->max_iter;
    Ops ops{elem, dim3(nchunk, nrhs)};

    ZT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(int) * (size_t)w.cap * ST_STRIDE, s));
    ZT_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * (size_t)w.cap * CNT_STRIDE, s));
    const bool zero = (o->flags & ZTOEP_FLAG_ZERO_GUESS) != 0;
    if (zero) ZT_CUDA(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)nrhs * p->N, s));
    ZT_TRY(ops.vnorm(a, s));

    ztoep_status_t worst = ZTOEP_OK;
    bool timed_out = false;
    const int poll = 4;
    for (int outer = 0;; ++outer) {
        // true residual in FP64
        if (!(zero && outer == 0)) ZT_TRY(run_matvec<double>(p, nrhs, X, w.r, s));
        ZT_TRY(ops.residual(a, (zero && outer == 0) ? 1 : 0, s));
        ZT_CUDA(cudaMemcpyAsync(w.hst, w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE, cudaMemcpyDeviceToHost, s));
        ZT_CUDA(cudaStreamSynchronize(s));
        int nact = 0;
        for (int rr = 0; rr < nrhs; ++rr) nact += w.hst[rr * ST_STRIDE + ST_ACTIVE];
        if (nact == 0) break;
        if (outer + 1 >= o->max_outer) { worst = ZTOEP_ERR_NOCONV; break; }
        if (o->timeout_ns > 0) {
            const auto el = std::chrono::duration_cast<std::chrono::nanoseconds>(
                std::chrono::steady_clock::now() - t_start).count();
            if (el > o->timeout_ns) { timed_out = true; break; }
        }
        // one GMRES cycle
        ZT_TRY(ops.start(a, s));
        for (int j = 0; j < m; ++j) {
            if (mixed)
                ZT_TRY(run_matvec<float>(p, nrhs, a.x32, (float2 *)p->ws32.yout, s));
            else
                ZT_TRY(run_matvec<double>(p, nrhs, w.Vb + (int64_t)j * w.cap * p->N, w.w, s));
            ZT_TRY(ops.arnoldi(a, j, s));
            if ((j + 1) % poll == 0 && j + 1 < m) {
                ZT_CUDA(cudaMemcpyAsync(w.hst, w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE,
                                        cudaMemcpyDeviceToHost, s));
                ZT_CUDA(cudaStreamSynchronize(s));
                int na = 0;
                for (int rr = 0; rr < nrhs; ++rr) na += w.hst[rr * ST_STRIDE + ST_ACTIVE];
                if (na == 0) break;
            }
        }
        ZT_TRY(ops.update_x(a, s));
    }
    ZT_CUDA(cudaMemcpyAsync(w.hst, w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE, cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaMemcpyAsync(w.hnrm, w.nrm, sizeof(double) * (size_t)nrhs * NM_STRIDE, cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaStreamSynchronize(s));
    for (int rr = 0; rr < nrhs; ++rr) {
        const int *st = w.hst + rr * ST_STRIDE;
        const double *nm = w.hnrm + rr * NM_STRIDE;
        ztoep_status_t rs;
        switch (st[ST_STATUS]) {
            case RS_CONVERGED: rs = ZTOEP_OK; break;
            case RS_NONFINITE: rs = ZTOEP_ERR_NONFINITE; break;
            case RS_MAXITER: rs = ZTOEP_ERR_NOCONV; break;
            default: rs = timed_out ? ZTOEP_ERR_TIMEOUT : ZTOEP_ERR_NOCONV; break;
        }
        if (rs != ZTOEP_OK && (worst == ZTOEP_OK || rs == ZTOEP_ERR_NONFINITE || rs == ZTOEP_ERR_TIMEOUT))
            worst = rs;
        if (info) {
            info[rr].outer = st[ST_OUTER];
            info[rr].inner_iters = st[ST_ITERS];
            info[rr].status = rs;
            info[rr].rel_residual = nm[NM_VNORM] > 0 ? nm[NM_RNORM] / nm[NM_VNORM] : nm[NM_RNORM];
        }
    }
    if (timed_out && worst == ZTOEP_ERR_NOCONV) worst = ZTOEP_ERR_TIMEOUT;
    return worst;
}

}  // namespace ztoep

using namespace ztoep;

extern "C" {

static bool valid_opts(const ztoep_solve_opts_t *o) {
    return o && o->restart >= 1 && o->restart <= 128 && o->max_iter >= 1 && o->max_outer >= 1 &&
           (o->prec == ZTOEP_FP64 || o->prec == ZTOEP_MIXED) && o->tol > 0 && o->inner_tol > 0 &&
           o->inner_tol < 1 && o->timeout_ns >= 0;
}

ztoep_status_t ztoep_solve(ztoep_plan_t p, const ztoep_solve_opts_t *o, int32_t nrhs, const void *V, void *X,
                           ztoep_solve_info_t *info, void *stream) {
    if (!p || !valid_opts(o) || nrhs < 1 || !V || !X || V == X) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(p->mu);
    return solve_impl(p, o, nrhs, (const double2 *)V, (double2 *)X, info, (cudaStream_t)stream);
}

ztoep_status_t ztoep_solve_host(ztoep_plan_t p, const ztoep_solve_opts_t *o, int32_t nrhs, const void *Vh,
                                void *Xh, ztoep_solve_info_t *info, void *stream) {
    if (!p || !valid_opts(o) || nrhs < 1 || !Vh || !Xh) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStream_t s = (cudaStream_t)stream;
    ZT_TRY(ensure_ws<double>(p, nrhs));
    // the FP64 workspace in/out buffers hold V and X on the device
    double2 *Vd = (double2 *)p->ws64.xin, *Xd = (double2 *)p->ws64.yout;
    const size_t bytes = sizeof(double2) * (size_t)nrhs * p->N;
    ZT_CUDA(cudaMemcpyAsync(Vd, Vh, bytes, cudaMemcpyHostToDevice, s));
    if (!(o->flags & ZTOEP_FLAG_ZERO_GUESS)) ZT_CUDA(cudaMemcpyAsync(Xd, Xh, bytes, cudaMemcpyHostToDevice, s));
    ztoep_status_t st = solve_impl(p, o, nrhs, Vd, Xd, info, s);
    if (st == ZTOEP_ERR_ARG || st == ZTOEP_ERR_CUDA || st == ZTOEP_ERR_NOMEM) return st;
    ZT_CUDA(cudaMemcpyAsync(Xh, Xd, bytes, cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"
