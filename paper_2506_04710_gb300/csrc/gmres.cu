// Batched restarted GMRES inside an FP64 iterative-refinement loop for
// Z' X = V (Sec. II, Eq. MoMMatrixEq; Sec. II-D names GMRES on the
// second-level Toeplitz structure of A, with the FFT product for Z').
//
// Outer sweep (FP64):  r = v - Z' x (FP64 product), ||r|| per RHS, stop test.
// Inner cycle:         GMRES(m) on Z' d = r (Saad & Schultz 1986) with
//                      classical Gram-Schmidt and selective
//                      reorthogonalisation (a second pass only when the first
//                      one leaves less than eta ||w||, the criterion of
//                      Daniel, Gragg, Kaufman & Stewart 1976),
//                      Givens rotations, least squares R y = g, x <- x + V y.
//                      The products inside the cycle are FP32 (MIXED) or FP64
//                      (FP64); Arnoldi, rotations and updates are FP64.
// The basis is kept unnormalised: u_k with v_k = u_k / beta_k, so no kernel
// pass is spent on normalising; every use of v_k folds 1/beta_k into its
// coefficient.
// Every kernel is batched over the RHS (grid.y) and each RHS stops on its own
// flag.  Cross-CTA reductions use the last-CTA-done pattern (atomic ticket,
// no waiting), so the summation order is fixed and results do not depend on
// the batch.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {

enum { ST_ACTIVE = 0, ST_JLEN = 1, ST_ITERS = 2, ST_STATUS = 3, ST_OUTER = 4, ST_PENDING = 5, ST_REORTH = 6,
       ST_INNER = 7, ST_RESTARTS = 8, ST_END = 9, ST_STRIDE = 12 };
// ST_END: the column just finalised ends the cycle; the iteration control
// turns it into ACTIVE = 0, PENDING = 1 once every kernel of the step is done
// (the Arnoldi kernels of the step test ACTIVE, so it must not change under them).
enum { RS_RUNNING = 0, RS_CONVERGED = 1, RS_NONFINITE = 2, RS_MAXITER = 3 };
enum { NM_VNORM = 0, NM_TARGET = 2, NM_RNORM = 3, NM_W0 = 5, NM_RIN = 6, NM_STRIDE = 8 };
// Inner (FP32-residual) restarts of one sweep: at most this many, and they stop
// early when a restart reduces the inner residual by less than 10%.
constexpr int kMaxRestarts = 64;
constexpr double kStagnation = 0.9;
enum { CNT_STRIDE = 4 };
// Second Gram-Schmidt pass when ||w'|| < eta ||w||.  The orthogonality lost by
// one classical pass is about u ||w|| / ||w'||, so eta = 1/64 keeps it below
// 64 u (~7e-15), far under what the residual targets need, while skipping the
// pass in the usual case (the stricter 1/sqrt(2) of "twice is enough" asked
// for it at every step on these systems, doubling the FP64 work).
constexpr double kReorthEta = 1.0 / 64.0;

// Device-side control of one solve (written by the host before each launch of
// the solve graph; loop counters advanced by the control kernels).
struct SolveCtl {
    int j;               // current inner iteration of the running cycle
    int sweeps;          // true-residual evaluations so far
    int timed_out;       // the deadline passed while some RHS was unconverged
    int zero;            // first sweep starts from x = 0
    int max_iter, max_outer;
    int outer_bodies;    // executions of the sweep body (for launch accounting)
    int inner_bodies;    // executions of the iteration body
    int restart_bodies;  // executions of the restart body
    int reorth_bodies;   // executions of the second Gram-Schmidt pass
    int cond_first, cond_sweep, cond_restart, cond_iter;  // loop decisions (read by the host-driven mode)
    double tol, inner_tol;
    long long timeout_ns;
    unsigned long long deadline;  // %globaltimer value, 0 = none
};

struct GArgs {
    double2 *Vb;       // [(m+1)][cap][N] unnormalised basis u_k
    double2 *w;        // [cap][N] FP64 product output
    double2 *x;        // [nrhs][N] iterate (caller's buffer)
    const double2 *v;  // [nrhs][N] right-hand sides
    float2 *x32;       // [cap][N] FP32 copy of the next product input (MIXED)
    const float2 *y32; // [cap][N] FP32 product output (MIXED)
    double2 *H, *cs, *sn, *g, *y, *h1, *h2, *part;
    double *beta;      // [cap][m+1] ||u_k||
    double2 *xin64;    // [cap][N] FP64 copy of the next product input (FP64)
    double2 *rbuf;     // [cap][N] FP64 residual r of the sweep
    double2 *dbuf;     // [cap][N] correction d of the sweep
    double *nrm;
    int *st;
    unsigned *cnt;
    SolveCtl *ctl;
    int64_t N;
    int cap, m, nchunk, pstride, nrhs;
    int mixed;
    int graph;                             // running inside the solve graph
    int redund;                            // pass-1 partials reduced by every update CTA (else by the dots' last CTA)
    cudaGraphConditionalHandle h_reorth;   // second Gram-Schmidt pass needed by some RHS
};

__device__ __forceinline__ double2 shfl_xor2(double2 v, int o) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    return v;
}
__device__ __forceinline__ double2 shfl_idx2(double2 v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
    return v;
}

// Warp reduce-scatter of 8 values: afterwards v[0] holds the warp total of
// value ((lane>>4)&1)*4 + ((lane>>3)&1)*2 + ((lane>>2)&1).  9 exchanges instead
// of 40 for 8 separate butterflies.
__device__ __forceinline__ void warp_rs8(double2 (&v)[8]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 recv = shfl_xor2(b4 ? v[i] : v[i + 4], 16);
        v[i] = (b4 ? v[i + 4] : v[i]) + recv;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double2 recv = shfl_xor2(b3 ? v[i] : v[i + 2], 8);
        v[i] = (b3 ? v[i + 2] : v[i]) + recv;
    }
    {
        const double2 recv = shfl_xor2(b2 ? v[0] : v[1], 4);
        v[0] = (b2 ? v[1] : v[0]) + recv;
    }
    v[0] = v[0] + shfl_xor2(v[0], 2);
    v[0] = v[0] + shfl_xor2(v[0], 1);
}

// CTA totals of 8 values into red[0..8) (red holds >= 8 * warps entries).
__device__ __forceinline__ void block_sum8(double2 (&v)[8], double2 *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_rs8(v);
    if ((lane & 3) == 0) red[warp * 8 + (((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1))] = v[0];
    __syncthreads();
    if (threadIdx.x < 8) {
        double2 s = red[threadIdx.x];
        for (int w = 1; w < nw; ++w) s = s + red[w * 8 + threadIdx.x];
        red[threadIdx.x] = s;  // thread t only touches column t
    }
    __syncthreads();
}

// CTA total of one real value (valid in thread 0).
__device__ __forceinline__ double block_sum1(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Last-CTA-done ticket for the CTAs of one RHS (no waiting).
__device__ __forceinline__ bool last_cta(unsigned *cnt, unsigned total) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(cnt, 1u);
        s_last = (t == total - 1);
        if (s_last) *cnt = 0;  // reset for the next use; no other CTA touches it in this launch
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// In the last CTA: out[k] = sum_c part[c][k] for k < K.  The threads form G
// groups of KP (K rounded up to a power of two, at most blockDim); thread
// (g, kk) adds chunks g, g+G, g+2G, ... of column kb+kk in four independent
// accumulators (so several loads are in flight), and the G group sums are then
// added by a pairwise tree.  The order depends only on nchunk, K and blockDim,
// never on timing or on the other RHS of the batch.
__device__ void reduce_partials(const double2 *part, int nchunk, int pstride, int K, double2 *out) {
    __shared__ double2 red2[256];
    int KP = 1;
    while (KP < K && KP < (int)blockDim.x) KP <<= 1;
    const int G = blockDim.x / KP;
    const int kk = threadIdx.x % KP, g = threadIdx.x / KP;
    for (int kb = 0; kb < K; kb += KP) {
        const int k = kb + kk;
        double2 sa[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) sa[q] = make_double2(0, 0);
        if (k < K) {
            int c = g;
            for (; c + 7 * G < nchunk; c += 8 * G) {  // 8 loads in flight
                double2 av[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) av[q] = __ldcg(part + (int64_t)(c + q * G) * pstride + k);
#pragma unroll
                for (int q = 0; q < 8; ++q) sa[q] = sa[q] + av[q];
            }
            for (; c < nchunk; c += G) sa[0] = sa[0] + __ldcg(part + (int64_t)c * pstride + k);
        }
        red2[threadIdx.x] = ((sa[0] + sa[1]) + (sa[2] + sa[3])) + ((sa[4] + sa[5]) + (sa[6] + sa[7]));
        __syncthreads();
        for (int h = G >> 1; h > 0; h >>= 1) {
            if (g < h) red2[threadIdx.x] = red2[threadIdx.x] + red2[threadIdx.x + h * KP];
            __syncthreads();
        }
        if (threadIdx.x < KP && kb + (int)threadIdx.x < K) out[kb + threadIdx.x] = red2[threadIdx.x];
        __syncthreads();
    }
}

__device__ __forceinline__ double2 *basis(const GArgs &a, int k, int rr) {
    return a.Vb + ((int64_t)k * a.cap + rr) * a.N;
}

// ---------------------------------------------------------------- norms
template <int ELEM> __global__ void __launch_bounds__(256) k_vnorm(GArgs a) {
    __shared__ double red[8];
    __shared__ double2 tot[1];
    const int rr = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        if (idx < a.N) acc += cabs2(a.v[(int64_t)rr * a.N + idx]);
    }
    acc = block_sum1(acc, red);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = make_double2(acc, 0);
    if (last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) {
        reduce_partials(part, a.nchunk, a.pstride, 1, tot);
        if (threadIdx.x == 0) a.nrm[rr * NM_STRIDE + NM_VNORM] = sqrt(tot[0].x);
    }
}

// u_0 = v - Z'x (w holds Z'x) or v (zero guess), its FP32 copy, ||u_0||, stop
// test and the start of a cycle.
template <int ELEM> __global__ void __launch_bounds__(256) k_residual(GArgs a, int first) {
    __shared__ double red[8];
    __shared__ double2 tot[1];
    const int rr = blockIdx.y;
    int *st = a.st + rr * ST_STRIDE;
    if (st[ST_STATUS] != RS_RUNNING) return;
    const int zero = first && a.ctl->zero;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
    double2 *u0 = basis(a, 0, rr);
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        if (idx < a.N) {
            const int64_t o = (int64_t)rr * a.N + idx;
            const double2 t = zero ? a.v[o] : a.v[o] - a.w[o];
            u0[idx] = t;
            a.rbuf[o] = t;
            a.dbuf[o] = make_double2(0, 0);
            if (a.mixed)
                a.x32[o] = make_float2((float)t.x, (float)t.y);
            else
                a.xin64[o] = t;
            acc += cabs2(t);
        }
    }
    acc = block_sum1(acc, red);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = make_double2(acc, 0);
    if (!last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) return;
    reduce_partials(part, a.nchunk, a.pstride, 1, tot);
    if (threadIdx.x != 0) return;
    double *nm = a.nrm + rr * NM_STRIDE;
    const double vn = nm[NM_VNORM], rn = sqrt(tot[0].x);
    nm[NM_RNORM] = rn;
    st[ST_OUTER] += 1;
    st[ST_PENDING] = 0;
    st[ST_JLEN] = 0;
    st[ST_ACTIVE] = 0;
    st[ST_REORTH] = 0;
    st[ST_INNER] = 0;
    st[ST_RESTARTS] = 0;
    if (!isfinite(vn) || !isfinite(rn)) {
        st[ST_STATUS] = RS_NONFINITE;
    } else if (rn <= a.ctl->tol * vn || rn == 0.0) {
        st[ST_STATUS] = RS_CONVERGED;
    } else if (st[ST_ITERS] >= a.ctl->max_iter) {
        st[ST_STATUS] = RS_MAXITER;
    } else {
        st[ST_ACTIVE] = 1;
        st[ST_INNER] = 1;
        nm[NM_RIN] = rn;
        a.beta[(int64_t)rr * (a.m + 1)] = rn;
        const double floor_abs = 0.5 * a.ctl->tol * vn;
        nm[NM_TARGET] = a.mixed ? fmax(a.ctl->inner_tol * rn, floor_abs) : floor_abs;
        double2 *g = a.g + (int64_t)rr * (a.m + 1);
        g[0] = make_double2(rn, 0);
        for (int i = 1; i <= a.m; ++i) g[i] = make_double2(0, 0);
    }
}

// ---------------------------------------------------------------- Arnoldi
// Hessenberg column j from the Gram-Schmidt coefficients hs[0..j] (shared
// memory, rotated in place) and beta_{j+1}: the earlier Givens rotations, the
// new one, the residual estimate and the end-of-cycle decision.  Called by
// every thread of one CTA; the rotation chain runs in one thread on shared
// copies of (c_i, s_i).  The least squares R y = g is solved at the update
// (k_update_d).
__device__ void finalize_column(const GArgs &a, int rr, int j, double2 *hs, double beta) {
    __shared__ double2 s_cs[128], s_sn[128];
    const int m = a.m;
    int *st = a.st + rr * ST_STRIDE;
    double *nm = a.nrm + rr * NM_STRIDE;
    double2 *H = a.H + (int64_t)rr * (m + 1) * m;
    double2 *cs = a.cs + (int64_t)rr * m, *sn = a.sn + (int64_t)rr * m;
    double2 *g = a.g + (int64_t)rr * (m + 1);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        s_cs[i] = __ldcg(cs + i);
        s_sn[i] = __ldcg(sn + i);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.beta[(int64_t)rr * (m + 1) + j + 1] = beta;
        double2 p = hs[0];
        for (int i = 0; i < j; ++i) {
            const double2 q = hs[i + 1];
            hs[i] = cmulc(s_cs[i], p) + cmulc(s_sn[i], q);
            p = cmul(s_cs[i], q) - cmul(s_sn[i], p);
        }
        const double d = sqrt(cabs2(p) + beta * beta);
        double2 c, sj;
        if (d > 0) {
            c = cscale(p, 1.0 / d);
            sj = make_double2(beta / d, 0);
        } else {
            c = make_double2(1, 0);
            sj = make_double2(0, 0);
        }
        cs[j] = c;
        sn[j] = sj;
        hs[j] = make_double2(d, 0);
        const double2 gj = __ldcg(g + j);
        const double2 gn = make_double2(-sj.x * gj.x, -sj.x * gj.y);
        g[j + 1] = gn;
        g[j] = cmulc(c, gj);
        st[ST_JLEN] = j + 1;
        st[ST_ITERS] += 1;
        const double res = sqrt(cabs2(gn));
        const bool end =
            !(res > nm[NM_TARGET]) || !(beta > 0) || (j + 1 == m) || (st[ST_ITERS] >= a.ctl->max_iter);
        if (end) st[ST_END] = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) H[i * m + j] = hs[i];
}

// After the first Gram-Schmidt pass (hs[k] = h_k for k <= j, hs[j+1].x =
// ||w||^2, shared memory, whole CTA): ||w - V h||^2 = ||w||^2 - sum |h_k|^2
// (exact for orthonormal v_k up to rounding of order u ||w||^2 / ||w'||^2,
// below 4096 u when no second pass is taken); strong cancellation (or NaN)
// asks for the second pass, else the Hessenberg column is finalised now.
__device__ void column_decision(const GArgs &a, int rr, int j, double2 *hs) {
    __shared__ double s_wn2;
    __shared__ int s_again;
    int *st = a.st + rr * ST_STRIDE;
    if (threadIdx.x == 0) {
        const double w2 = hs[j + 1].x;
        double hsq = 0;
        for (int k = 0; k <= j; ++k) hsq += cabs2(hs[k]);
        const double wn2 = w2 - hsq;
        const int again = !(wn2 > kReorthEta * kReorthEta * w2);
        st[ST_REORTH] = again;
        if (again && a.graph) cudaGraphSetConditional(a.h_reorth, 1u);
        s_wn2 = wn2;
        s_again = again;
    }
    __syncthreads();
    if (!s_again) finalize_column(a, rr, j, hs, sqrt(s_wn2));
}

// Partial dot products <u_k, w> for k in [k0, k0+8) (k <= j) plus, when
// with_norm and k0 + kk == j + 1, ||w||^2 in that slot; CTA totals -> part.
template <int ELEM>
__device__ __forceinline__ void dots_group(const GArgs &a, int rr, int j, int k0, bool with_norm,
                                           const double2 (&wv)[ELEM], int64_t base, double2 *part, double2 *red) {
    double2 acc[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) acc[kk] = make_double2(0, 0);
    if (k0 + 7 <= j) {  // full group: the 8 loads of an element are in flight together
        const double2 *u0 = basis(a, k0, rr);
        const int64_t vstride = (int64_t)a.cap * a.N;
#pragma unroll
        for (int e = 0; e < ELEM; ++e) {
            const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
            if (idx < a.N) {
                double2 uv[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) uv[kk] = u0[kk * vstride + idx];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) acc[kk] = cfmac(uv[kk], wv[e], acc[kk]);
            }
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int k = k0 + kk;
            if (k <= j) {
                const double2 *uk = basis(a, k, rr);
#pragma unroll
                for (int e = 0; e < ELEM; ++e) {
                    const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
                    if (idx < a.N) acc[kk] = cfmac(uk[idx], wv[e], acc[kk]);
                }
            } else if (with_norm && k == j + 1) {
#pragma unroll
                for (int e = 0; e < ELEM; ++e) acc[kk].x += cabs2(wv[e]);
            }
        }
    }
    block_sum8(acc, red);
    const int K = j + 1 + (with_norm ? 1 : 0);
    if (threadIdx.x < 8 && k0 + (int)threadIdx.x < K)
        part[(int64_t)blockIdx.x * a.pstride + k0 + threadIdx.x] = red[threadIdx.x];
    __syncthreads();
}

// Lowest RHS index that asked for a second Gram-Schmidt pass (-1 if none).
__device__ __forceinline__ int first_reorth_rhs(const GArgs &a) {
    for (int rr = 0; rr < a.nrhs; ++rr)
        if (a.st[rr * ST_STRIDE + ST_ACTIVE] && a.st[rr * ST_STRIDE + ST_REORTH]) return rr;
    return -1;
}

// Gram-Schmidt dots.
// PASS 1: w = (product of u_j) / beta_j is formed (from the FP32 or FP64
//   product) and stored as u_{j+1}; per-CTA partial sums of <v_k, w> and ||w||^2.
//   With a.redund every CTA of the update kernel reduces them (no serial tail
//   on the path); else the last CTA per RHS reduces them, takes the second-pass
//   decision and finalises the column (column_decision).
// PASS 2 (flagged RHS only): h2_k = <v_k, u_{j+1}> (last CTA reduces).
template <int ELEM, int PASS> __global__ void __launch_bounds__(256) k_dots(GArgs a) {
    __shared__ double2 red[64];
    __shared__ double2 tot[130];
    const int rr = blockIdx.y;
    int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_ACTIVE]) return;
    if (PASS == 2 && !st[ST_REORTH]) return;
    const int j = a.ctl->j;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
    const double *beta = a.beta + (int64_t)rr * (a.m + 1);
    double2 *un = basis(a, j + 1, rr);
    double2 wv[ELEM];
    const double sc = 1.0 / beta[j];
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        wv[e] = make_double2(0, 0);
        if (idx < a.N) {
            if (PASS == 1) {
                const int64_t o = (int64_t)rr * a.N + idx;
                double2 t;
                if (a.mixed) {
                    const float2 f = a.y32[o];
                    t = make_double2(f.x, f.y);
                } else {
                    t = a.w[o];
                }
                wv[e] = cscale(t, sc);
                un[idx] = wv[e];
            } else {
                wv[e] = un[idx];
            }
        }
    }
    if (PASS == 2 && blockIdx.x == 0 && threadIdx.x == 0 && rr == first_reorth_rhs(a)) a.ctl->reorth_bodies += 1;
    const int K = j + 1 + (PASS == 1 ? 1 : 0);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    for (int k0 = 0; k0 < K; k0 += 8) dots_group<ELEM>(a, rr, j, k0, PASS == 1, wv, base, part, red);
    if (PASS == 1 && a.redund) return;  // the update kernel reduces these partial sums
    if (!last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) return;
    reduce_partials(part, a.nchunk, a.pstride, K, tot);
    double2 *h = (PASS == 1 ? a.h1 : a.h2) + (int64_t)rr * (a.m + 1);
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        const double2 hk = cscale(tot[k], 1.0 / beta[k]);
        h[k] = hk;
        tot[k] = hk;
    }
    __syncthreads();
    if (PASS == 2) return;
    column_decision(a, rr, j, tot);
}

// u_{j+1} <- u_{j+1} - sum_k (h_k / beta_k) u_k and its copy for the next
// product.  PASS 1 with a.redund: every CTA first reduces the dots' partial
// sums (same order everywhere, so the same h as the last-CTA reduction); one
// extra CTA (blockIdx.x == nchunk) takes the second-pass decision and, without
// one, finalises the Hessenberg column, alongside the update.  PASS 2 (after a
// second Gram-Schmidt pass) also forms ||u_{j+1}|| and finalises the column.
template <int ELEM, int PASS> __global__ void __launch_bounds__(256) k_upd(GArgs a) {
    __shared__ double red[8];
    __shared__ double2 cf[129];
    __shared__ double2 tot[130];
    const int rr = blockIdx.y;
    int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_ACTIVE]) return;
    if (PASS == 2 && !st[ST_REORTH]) return;
    const int j = a.ctl->j;
    const double *beta = a.beta + (int64_t)rr * (a.m + 1);
    if (PASS == 1 && a.redund) {
        // every CTA reduces the dots' partial sums in the same fixed order:
        // tot[k] = <u_k, w> (k <= j), tot[j+1].x = ||w||^2
        reduce_partials(a.part + (int64_t)rr * a.nchunk * a.pstride, a.nchunk, a.pstride, j + 2, tot);
        for (int k = threadIdx.x; k <= j; k += blockDim.x) {
            const double2 hk = cscale(tot[k], 1.0 / beta[k]);  // h_k = <v_k, w>
            cf[k] = cscale(hk, 1.0 / beta[k]);
            tot[k] = hk;
        }
        __syncthreads();
        if (blockIdx.x == a.nchunk) {  // one extra CTA: the step decision and Hessenberg column
            double2 *h1 = a.h1 + (int64_t)rr * (a.m + 1);
            for (int k = threadIdx.x; k <= j; k += blockDim.x) h1[k] = tot[k];
            column_decision(a, rr, j, tot);
            return;
        }
    } else {  // h from the dots' last CTA
        const double2 *h = (PASS == 1 ? a.h1 : a.h2) + (int64_t)rr * (a.m + 1);
        for (int k = threadIdx.x; k <= j; k += blockDim.x) cf[k] = cscale(__ldcg(h + k), 1.0 / beta[k]);
        __syncthreads();
    }
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
    double2 *un = basis(a, j + 1, rr);
    double2 wv[ELEM];
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        wv[e] = idx < a.N ? un[idx] : make_double2(0, 0);
    }
    int k = 0;
    const int64_t vstride = (int64_t)a.cap * a.N;
    constexpr int UNR = ELEM == 1 ? 8 : 4;  // basis vectors per step, loads first
    for (; k + UNR <= j + 1; k += UNR) {
        const double2 *u0 = basis(a, k, rr);
#pragma unroll
        for (int e = 0; e < ELEM; ++e) {
            const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
            if (idx < a.N) {
                double2 uv[UNR];
#pragma unroll
                for (int kk = 0; kk < UNR; ++kk) uv[kk] = u0[kk * vstride + idx];
#pragma unroll
                for (int kk = 0; kk < UNR; ++kk) wv[e] = wv[e] - cmul(cf[k + kk], uv[kk]);
            }
        }
    }
    for (; k <= j; ++k) {
        const double2 c = cf[k];
        const double2 *uk = basis(a, k, rr);
#pragma unroll
        for (int e = 0; e < ELEM; ++e) {
            const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
            if (idx < a.N) wv[e] = wv[e] - cmul(c, uk[idx]);
        }
    }
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        if (idx < a.N) {
            un[idx] = wv[e];
            if (a.mixed)
                a.x32[(int64_t)rr * a.N + idx] = make_float2((float)wv[e].x, (float)wv[e].y);
            else
                a.xin64[(int64_t)rr * a.N + idx] = wv[e];
            acc += cabs2(wv[e]);
        }
    }
    if (PASS == 1) return;
    acc = block_sum1(acc, red);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = make_double2(acc, 0);
    if (!last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) return;
    reduce_partials(part, a.nchunk, a.pstride, 1, tot);
    const double wn = sqrt(tot[0].x);
    const double2 *h1 = a.h1 + (int64_t)rr * (a.m + 1);
    const double2 *h2 = a.h2 + (int64_t)rr * (a.m + 1);
    for (int kk = threadIdx.x; kk <= j; kk += blockDim.x) cf[kk] = __ldcg(h1 + kk) + __ldcg(h2 + kk);  // totals
    if (threadIdx.x == 0) st[ST_REORTH] = 0;
    __syncthreads();
    finalize_column(a, rr, j, cf, wn);
}

// Least squares of a finished cycle: R y = g with R the leading jl x jl
// upper triangle of the rotated Hessenberg matrix; ys[k] = y_k / beta_k.
// Every CTA of the RHS solves it (the same arithmetic, so the same result):
// R is staged in shared memory by all threads and one warp runs the
// column-oriented back substitution (lane l keeps the running right-hand side
// of row l).  Cycles longer than 32 fall back to one thread reading R from
// global memory.
__device__ void cycle_least_squares(const GArgs &a, int rr, int jl, double2 *ys) {
    __shared__ double2 Rs[32 * 32];
    const int m = a.m;
    const double2 *H = a.H + (int64_t)rr * (m + 1) * m;
    const double2 *g = a.g + (int64_t)rr * (m + 1);
    const double *beta = a.beta + (int64_t)rr * (m + 1);
    if (jl <= 32) {
        for (int idx = threadIdx.x; idx < jl * jl; idx += blockDim.x) {
            const int i = idx / jl, l = idx - i * jl;
            if (l >= i) Rs[i * 32 + l] = __ldcg(H + i * m + l);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double2 sl = lane < jl ? __ldcg(g + lane) : make_double2(0, 0);
            for (int i = jl - 1; i >= 0; --i) {
                double2 yi = make_double2(0, 0);
                if (lane == i) {
                    const double2 rii = Rs[i * 32 + i];
                    yi = (rii.x != 0.0 || rii.y != 0.0) ? cdiv(sl, rii) : make_double2(0, 0);
                    ys[i] = cscale(yi, 1.0 / beta[i]);
                }
                yi = shfl_idx2(yi, i);
                if (lane < i) sl = sl - cmul(Rs[lane * 32 + i], yi);
            }
        }
    } else if (threadIdx.x == 0) {
        double2 *yv = Rs;  // unused by this path: y_l, l < jl <= 128
        for (int i = jl - 1; i >= 0; --i) {
            double2 sacc = __ldcg(g + i);
            for (int l = i + 1; l < jl; ++l) sacc = sacc - cmul(__ldcg(H + i * m + l), yv[l]);
            const double2 rii = __ldcg(H + i * m + i);
            yv[i] = (rii.x != 0.0 || rii.y != 0.0) ? cdiv(sacc, rii) : make_double2(0, 0);
            ys[i] = cscale(yv[i], 1.0 / beta[i]);
        }
    }
    __syncthreads();
}

// d <- d + sum_k (y_k / beta_k) u_k for RHS whose cycle produced an update.
template <int ELEM> __global__ void __launch_bounds__(256) k_update_d(GArgs a) {
    __shared__ double2 ys[128];
    const int rr = blockIdx.y;
    const int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_PENDING]) return;
    const int jl = st[ST_JLEN];
    cycle_least_squares(a, rr, jl, ys);
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        if (idx < a.N) {
            const int64_t o = (int64_t)rr * a.N + idx;
            double2 s = a.dbuf[o];
            for (int k = 0; k < jl; ++k) s = cfma(ys[k], basis(a, k, rr)[idx], s);
            a.dbuf[o] = s;
            if (a.mixed) a.x32[o] = make_float2((float)s.x, (float)s.y);  // input of the restart product
        }
    }
}

// x <- x + d at the end of a sweep.
template <int ELEM> __global__ void __launch_bounds__(256) k_apply_d(GArgs a) {
    const int rr = blockIdx.y;
    if (!a.st[rr * ST_STRIDE + ST_INNER]) return;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        if (idx < a.N) {
            const int64_t o = (int64_t)rr * a.N + idx;
            a.x[o] = a.x[o] + a.dbuf[o];
        }
    }
}

// Inner restart (MIXED): r_in = r - Z32 d with the FP32 product of d in y32;
// r_in becomes u_0 of a new cycle unless the inner target is met, the restart
// gained less than 10%, or a cap is reached.
template <int ELEM> __global__ void __launch_bounds__(256) k_inner_residual(GArgs a) {
    __shared__ double red[8];
    __shared__ double2 tot[1];
    const int rr = blockIdx.y;
    int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_INNER] || !st[ST_PENDING]) return;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * ELEM;
    double2 *u0 = basis(a, 0, rr);
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = base + (int64_t)e * blockDim.x + threadIdx.x;
        if (idx < a.N) {
            const int64_t o = (int64_t)rr * a.N + idx;
            const float2 f = a.y32[o];
            const double2 t = a.rbuf[o] - make_double2(f.x, f.y);
            u0[idx] = t;
            a.x32[o] = make_float2((float)t.x, (float)t.y);
            acc += cabs2(t);
        }
    }
    acc = block_sum1(acc, red);
    double2 *part = a.part + (int64_t)rr * a.nchunk * a.pstride;
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * a.pstride] = make_double2(acc, 0);
    if (!last_cta(a.cnt + rr * CNT_STRIDE, a.nchunk)) return;
    reduce_partials(part, a.nchunk, a.pstride, 1, tot);
    if (threadIdx.x != 0) return;
    double *nm = a.nrm + rr * NM_STRIDE;
    const double rin = sqrt(tot[0].x), prev = nm[NM_RIN];
    nm[NM_RIN] = rin;
    st[ST_PENDING] = 0;
    const bool more = (rin > nm[NM_TARGET]) && (rin < kStagnation * prev) && st[ST_ITERS] < a.ctl->max_iter &&
                      st[ST_RESTARTS] < kMaxRestarts;  // false for NaN
    if (!more) return;
    st[ST_RESTARTS] += 1;
    st[ST_ACTIVE] = 1;
    a.beta[(int64_t)rr * (a.m + 1)] = rin;
    double2 *g = a.g + (int64_t)rr * (a.m + 1);
    g[0] = make_double2(rin, 0);
    for (int i = 1; i <= a.m; ++i) g[i] = make_double2(0, 0);
}

// ---------------------------------------------------------------- loop control
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Start of a solve: counters, deadline, x = 0 for a zero guess, and whether the
// first true residual needs a product (it does not when x = 0).
__global__ void k_solve_begin(GArgs a, cudaGraphConditionalHandle h_first_product, int use_graph) {
    SolveCtl *c = a.ctl;
    const int64_t total = (int64_t)a.nrhs * a.N;
    if (c->zero)
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x)
            a.x[k] = make_double2(0, 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->j = 0;
        c->sweeps = 0;
        c->timed_out = 0;
        c->outer_bodies = 0;
        c->restart_bodies = 0;
        c->inner_bodies = 0;
        c->deadline = c->timeout_ns > 0 ? globaltimer_ns() + (unsigned long long)c->timeout_ns : 0ull;
        c->cond_first = c->zero ? 0 : 1;
        if (use_graph) cudaGraphSetConditional(h_first_product, c->zero ? 0u : 1u);
    }
}

__device__ __forceinline__ bool any_active(const GArgs &a) {
    int any = 0;
    for (int rr = threadIdx.x; rr < a.nrhs; rr += blockDim.x) any |= a.st[rr * ST_STRIDE + ST_ACTIVE];
    return __syncthreads_or(any) != 0;
}

__device__ __forceinline__ bool past_deadline(const SolveCtl *c) {
    return c->deadline != 0ull && globaltimer_ns() > c->deadline;
}

// After a true residual: another sweep while some RHS is active, within the
// sweep cap and the deadline.
__global__ void k_sweep_ctl(GArgs a, cudaGraphConditionalHandle h_sweep, int use_graph) {
    const bool any = any_active(a);
    if (threadIdx.x != 0) return;
    SolveCtl *c = a.ctl;
    c->sweeps += 1;
    const bool late = past_deadline(c);
    if (any && late) c->timed_out = 1;
    const unsigned cond = (any && c->sweeps < c->max_outer && !late) ? 1u : 0u;
    c->cond_sweep = (int)cond;
    if (use_graph) cudaGraphSetConditional(h_sweep, cond);
}

__global__ void k_restart_begin(GArgs a, cudaGraphConditionalHandle h_restart, int use_graph) {
    if (threadIdx.x != 0) return;
    a.ctl->outer_bodies += 1;
    a.ctl->cond_restart = 1;
    if (use_graph) cudaGraphSetConditional(h_restart, 1u);
}

// After a restart: another cycle while some RHS started one (MIXED only).
__global__ void k_restart_ctl(GArgs a, cudaGraphConditionalHandle h_restart, int use_graph) {
    const bool any = a.mixed && any_active(a);
    if (threadIdx.x != 0) return;
    SolveCtl *c = a.ctl;
    const bool late = past_deadline(c);
    if (any && late) c->timed_out = 1;
    const unsigned cond = (any && !late) ? 1u : 0u;
    c->cond_restart = (int)cond;
    if (use_graph) cudaGraphSetConditional(h_restart, cond);
}

__global__ void k_cycle_begin(GArgs a, cudaGraphConditionalHandle h_iter, int use_graph) {
    if (threadIdx.x != 0) return;
    a.ctl->j = 0;
    a.ctl->restart_bodies += 1;
    a.ctl->cond_iter = 1;
    if (use_graph) cudaGraphSetConditional(h_iter, 1u);
}

// After an Arnoldi step: cycles that ended in this step close (ACTIVE -> 0,
// PENDING -> 1), then the next iteration runs while some RHS is still in its
// cycle.
__global__ void k_iter_ctl(GArgs a, cudaGraphConditionalHandle h_iter, int use_graph) {
    for (int rr = threadIdx.x; rr < a.nrhs; rr += blockDim.x) {
        int *st = a.st + rr * ST_STRIDE;
        if (st[ST_END]) {
            st[ST_END] = 0;
            st[ST_ACTIVE] = 0;
            st[ST_PENDING] = 1;
        }
    }
    __syncthreads();
    const bool any = any_active(a);
    if (threadIdx.x != 0) return;
    SolveCtl *c = a.ctl;
    c->j += 1;
    c->inner_bodies += 1;
    const bool late = past_deadline(c);
    if (any && late) c->timed_out = 1;
    const unsigned cond = (any && c->j < a.m && !late) ? 1u : 0u;
    c->cond_iter = (int)cond;
    if (use_graph) {
        cudaGraphSetConditional(h_iter, cond);
        cudaGraphSetConditional(a.h_reorth, 0u);
    }
}

// ---------------------------------------------------------------- workspace
void free_solve_graphs(ztoep_plan_t p) {
    for (auto &g : p->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = SolveGraph{};
    }
    p->graph_next = 0;
}

void free_solve_ws(ztoep_plan_t p) {
    free_solve_graphs(p);
    SolveWs &w = p->sws;
    cudaFree(w.Vb); cudaFree(w.w); cudaFree(w.xin64); cudaFree(w.vbuf); cudaFree(w.xbuf); cudaFree(w.rbuf); cudaFree(w.dbuf); cudaFree(w.H);
    cudaFree(w.cs); cudaFree(w.sn); cudaFree(w.g); cudaFree(w.y); cudaFree(w.h1); cudaFree(w.h2);
    cudaFree(w.part); cudaFree(w.nrm); cudaFree(w.st); cudaFree(w.cnt); cudaFree(w.ctl);
    if (w.hst) cudaFreeHost(w.hst);
    if (w.hnrm) cudaFreeHost(w.hnrm);
    w = SolveWs{};
}

// Launch geometry: depends on N only, so a RHS is summed in the same order
// alone and in any batch.  Small systems: 128 threads x 1 element (enough
// CTAs to cover every SM while keeping the partial sums of the cross-CTA
// reductions few); large ones: 256 threads x 4 elements.
struct Geom {
    int threads, elem;
};
static Geom geom_for(int64_t N, int nsm) {
    const int64_t ctas_small = (N + 255) / 256;
    if (ctas_small >= 8LL * nsm) return {256, 4};
    return {256, 1};
}

constexpr int kHostCtlInts = 32;  // host mirror of SolveCtl after st

static ztoep_status_t ensure_solve_ws(ztoep_plan_t p, int nrhs, int m) {
    SolveWs &w = p->sws;
    if (w.cap >= nrhs && w.m >= m) return ZTOEP_OK;
    free_solve_ws(p);
    const int64_t N = p->N;
    const Geom gm = geom_for(N, p->nsm);
    const int nchunk = (int)((N + gm.threads * gm.elem - 1) / (gm.threads * gm.elem));
    const int pstride = m + 2;
    const size_t vec = sizeof(double2) * (size_t)nrhs * N;
    size_t acc = 0;
    ZT_TRY(dalloc((void **)&w.Vb, sizeof(double2) * (size_t)(m + 1) * nrhs * N, &acc));
    ZT_TRY(dalloc((void **)&w.w, vec, &acc));
    ZT_TRY(dalloc((void **)&w.xin64, vec, &acc));
    ZT_TRY(dalloc((void **)&w.vbuf, vec, &acc));
    ZT_TRY(dalloc((void **)&w.xbuf, vec, &acc));
    ZT_TRY(dalloc((void **)&w.rbuf, vec, &acc));
    ZT_TRY(dalloc((void **)&w.dbuf, vec, &acc));
    ZT_TRY(dalloc((void **)&w.H, sizeof(double2) * (size_t)nrhs * (m + 1) * m, &acc));
    ZT_TRY(dalloc((void **)&w.cs, sizeof(double2) * (size_t)nrhs * m, &acc));
    ZT_TRY(dalloc((void **)&w.sn, sizeof(double2) * (size_t)nrhs * m, &acc));
    ZT_TRY(dalloc((void **)&w.g, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.y, sizeof(double2) * (size_t)nrhs * m, &acc));
    ZT_TRY(dalloc((void **)&w.h1, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.h2, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.part, sizeof(double2) * (size_t)nrhs * nchunk * pstride, &acc));
    ZT_TRY(dalloc((void **)&w.nrm, sizeof(double) * (size_t)nrhs * (NM_STRIDE + m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE, &acc));
    ZT_TRY(dalloc((void **)&w.cnt, sizeof(unsigned) * (size_t)nrhs * CNT_STRIDE, &acc));
    ZT_TRY(dalloc((void **)&w.ctl, sizeof(SolveCtl), &acc));
    ZT_CUDA(cudaMemset(w.cnt, 0, sizeof(unsigned) * (size_t)nrhs * CNT_STRIDE));
    ZT_CUDA(cudaMallocHost((void **)&w.hst, sizeof(int) * (size_t)nrhs * ST_STRIDE + sizeof(SolveCtl) + 64));
    ZT_CUDA(cudaMallocHost((void **)&w.hnrm, sizeof(double) * (size_t)nrhs * NM_STRIDE));
    w.cap = nrhs;
    w.m = m;
    w.bytes = acc;
    return ZTOEP_OK;
}

static GArgs make_args(ztoep_plan_t p, int nrhs, int m, bool mixed, int nchunk) {
    SolveWs &w = p->sws;
    GArgs a{};
    a.Vb = w.Vb; a.w = w.w; a.x = w.xbuf; a.v = w.vbuf; a.xin64 = w.xin64; a.rbuf = w.rbuf; a.dbuf = w.dbuf;
    a.x32 = (float2 *)p->ws32.xin; a.y32 = (const float2 *)p->ws32.yout;
    a.H = w.H; a.cs = w.cs; a.sn = w.sn; a.g = w.g; a.y = w.y; a.h1 = w.h1; a.h2 = w.h2; a.part = w.part;
    a.nrm = w.nrm; a.beta = w.nrm + (size_t)w.cap * NM_STRIDE; a.st = w.st; a.cnt = w.cnt;
    a.ctl = (SolveCtl *)w.ctl;
    a.N = p->N; a.cap = w.cap; a.m = m; a.nchunk = nchunk; a.pstride = w.m + 2; a.nrhs = nrhs;
    // Redundant reduction of the pass-1 partials when its L2 traffic (every one
    // of the nchunk update CTAs reads nchunk partial rows) stays small against
    // the Arnoldi's own; else the dots' last CTA per RHS reduces once.
    a.redund = (int64_t)nrhs * nchunk * nchunk <= (1 << 18) ? 1 : 0;
    a.mixed = mixed ? 1 : 0;
    return a;
}

template <int ELEM> struct Launch {
    static ztoep_status_t vnorm(const GArgs &a, dim3 g, int t, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_vnorm<ELEM><<<g, t, 0, s>>>(a);
        return ok();
    }
    static ztoep_status_t residual(const GArgs &a, dim3 g, int t, int first, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_residual<ELEM><<<g, t, 0, s>>>(a, first);
        return ok();
    }
    static ztoep_status_t arnoldi(const GArgs &a, dim3 g, int t, int pass, cudaStream_t s) {
        KScope ks(K_ARNOLDI, s);
        ks.add(2);
        if (pass == 1) {
            k_dots<ELEM, 1><<<g, t, 0, s>>>(a);
            k_upd<ELEM, 1><<<dim3(g.x + (a.redund ? 1 : 0), g.y), t, 0, s>>>(a);  // (+ the column CTA)
        } else {
            k_dots<ELEM, 2><<<g, t, 0, s>>>(a);
            k_upd<ELEM, 2><<<g, t, 0, s>>>(a);
        }
        return ok();
    }
    static ztoep_status_t update_d(const GArgs &a, dim3 g, int t, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_update_d<ELEM><<<g, t, 0, s>>>(a);
        return ok();
    }
    static ztoep_status_t apply_d(const GArgs &a, dim3 g, int t, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_apply_d<ELEM><<<g, t, 0, s>>>(a);
        return ok();
    }
    static ztoep_status_t inner_residual(const GArgs &a, dim3 g, int t, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_inner_residual<ELEM><<<g, t, 0, s>>>(a);
        return ok();
    }
    static ztoep_status_t ok() {
        ZT_CUDA(cudaGetLastError());
        return ZTOEP_OK;
    }
};

struct Ops {
    Geom gm;
    dim3 grid;
    ztoep_status_t vnorm(const GArgs &a, cudaStream_t s) const {
        return gm.elem == 4 ? Launch<4>::vnorm(a, grid, gm.threads, s) : Launch<1>::vnorm(a, grid, gm.threads, s);
    }
    ztoep_status_t residual(const GArgs &a, int first, cudaStream_t s) const {
        return gm.elem == 4 ? Launch<4>::residual(a, grid, gm.threads, first, s)
                            : Launch<1>::residual(a, grid, gm.threads, first, s);
    }
    ztoep_status_t arnoldi(const GArgs &a, int pass, cudaStream_t s) const {
        return gm.elem == 4 ? Launch<4>::arnoldi(a, grid, gm.threads, pass, s)
                            : Launch<1>::arnoldi(a, grid, gm.threads, pass, s);
    }
    ztoep_status_t update_d(const GArgs &a, cudaStream_t s) const {
        return gm.elem == 4 ? Launch<4>::update_d(a, grid, gm.threads, s)
                            : Launch<1>::update_d(a, grid, gm.threads, s);
    }
    ztoep_status_t apply_d(const GArgs &a, cudaStream_t s) const {
        return gm.elem == 4 ? Launch<4>::apply_d(a, grid, gm.threads, s)
                            : Launch<1>::apply_d(a, grid, gm.threads, s);
    }
    ztoep_status_t inner_residual(const GArgs &a, cudaStream_t s) const {
        return gm.elem == 4 ? Launch<4>::inner_residual(a, grid, gm.threads, s)
                            : Launch<1>::inner_residual(a, grid, gm.threads, s);
    }
};

static ztoep_status_t launch_small(void (*k)(GArgs, cudaGraphConditionalHandle, int), int blocks, const GArgs &a,
                                   cudaGraphConditionalHandle h, cudaStream_t s, int use_graph = 1) {
    KScope ks(K_MISC, s);
    k<<<blocks, 256, 0, s>>>(a, h, use_graph);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// Add a conditional node after the work captured so far on `s`; returns its body.
static ztoep_status_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                      cudaGraph_t *body) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    ZT_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    if (cst != cudaStreamCaptureStatusActive) return ZTOEP_ERR_CUDA;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ZT_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
    *body = cp.conditional.phGraph_out[0];
    ZT_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return ZTOEP_OK;
}

static ztoep_status_t capture_begin(cudaStream_t s, cudaGraph_t g, uint64_t *count) {
    ZT_CUDA(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capture_count_begin(count);
    return ZTOEP_OK;
}
static ztoep_status_t capture_end(cudaStream_t s) {
    capture_count_end();
    cudaGraph_t out = nullptr;
    ZT_CUDA(cudaStreamEndCapture(s, &out));
    return ZTOEP_OK;
}

// Whole solve as one graph:
//   begin -> IF(x != 0){FP64 product} -> residual -> sweep control ->
//   WHILE(sweep){ restart begin ->
//                 WHILE(restart){ cycle begin -> WHILE(iter){product, Arnoldi, iteration control}
//                                 -> d += V y -> [MIXED: FP32 product of d, r_in = r - Z d]
//                                 -> restart control }
//                 -> x += d -> FP64 product -> residual -> sweep control }
static ztoep_status_t build_graph(ztoep_plan_t p, SolveGraph &sg, int prec, int nrhs, int m) {
    const bool mixed = prec == ZTOEP_MIXED;
    SolveWs &w = p->sws;
    const Geom gm = geom_for(p->N, p->nsm);
    const int per_cta = gm.threads * gm.elem;
    const int nchunk = (int)((p->N + per_cta - 1) / per_cta);
    GArgs a = make_args(p, nrhs, m, mixed, nchunk);
    const Ops ops{gm, dim3(nchunk, nrhs)};
    cudaStream_t s = p->cap;
    cudaGraph_t top = nullptr;
    ZT_CUDA(cudaGraphCreate(&top, 0));
    sg.graph = top;
    a.graph = 1;
    cudaGraphConditionalHandle h_first, h_sweep, h_iter;
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_first, top, 0, 0));
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_sweep, top, 0, 0));
    cudaGraph_t body_first = nullptr, body_sweep = nullptr, body_iter = nullptr;

    // top level
    ZT_TRY(capture_begin(s, top, &sg.k_fixed));
    ZT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(int) * (size_t)w.cap * ST_STRIDE, s));
    ZT_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * (size_t)w.cap * CNT_STRIDE, s));
    const int zblocks = (int)std::min<int64_t>(4 * p->nsm, ((int64_t)nrhs * p->N + 255) / 256);
    ZT_TRY(launch_small(k_solve_begin, std::max(1, zblocks), a, h_first, s));
    ZT_TRY(ops.vnorm(a, s));
    ZT_TRY(add_conditional(s, h_first, cudaGraphCondTypeIf, &body_first));
    ZT_TRY(ops.residual(a, 1, s));
    ZT_TRY(launch_small(k_sweep_ctl, 1, a, h_sweep, s));
    ZT_TRY(add_conditional(s, h_sweep, cudaGraphCondTypeWhile, &body_sweep));
    ZT_TRY(capture_end(s));

    // first product (skipped for a zero guess)
    ZT_TRY(capture_begin(s, body_first, &sg.k_first_product));
    ZT_TRY(run_matvec<double>(p, nrhs, w.xbuf, w.w, s));
    ZT_TRY(capture_end(s));

    // one sweep: inner restarts, x += d, FP64 residual
    cudaGraphConditionalHandle h_restart;
    cudaGraph_t body_restart = nullptr;
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_restart, body_sweep, 0, 0));
    ZT_TRY(capture_begin(s, body_sweep, &sg.k_sweep));
    ZT_TRY(launch_small(k_restart_begin, 1, a, h_restart, s));
    ZT_TRY(add_conditional(s, h_restart, cudaGraphCondTypeWhile, &body_restart));
    ZT_TRY(ops.apply_d(a, s));
    ZT_TRY(run_matvec<double>(p, nrhs, w.xbuf, w.w, s));
    ZT_TRY(ops.residual(a, 0, s));
    ZT_TRY(launch_small(k_sweep_ctl, 1, a, h_sweep, s));
    ZT_TRY(capture_end(s));

    // one restart: GMRES cycle, d += V y, FP32 inner residual (MIXED)
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_iter, body_restart, 0, 0));
    ZT_TRY(capture_begin(s, body_restart, &sg.k_restart));
    ZT_TRY(launch_small(k_cycle_begin, 1, a, h_iter, s));
    ZT_TRY(add_conditional(s, h_iter, cudaGraphCondTypeWhile, &body_iter));
    ZT_TRY(ops.update_d(a, s));
    if (mixed) {
        ZT_TRY(run_matvec<float>(p, nrhs, a.x32, (float2 *)p->ws32.yout, s));
        ZT_TRY(ops.inner_residual(a, s));
    }
    ZT_TRY(launch_small(k_restart_ctl, 1, a, h_restart, s));
    ZT_TRY(capture_end(s));

    // one iteration; the second Gram-Schmidt pass only when a RHS asked for it
    // (its condition starts at 0 and is reset by every iteration control)
    cudaGraph_t body_reorth = nullptr;
    ZT_CUDA(cudaGraphConditionalHandleCreate(&a.h_reorth, body_iter, 0, cudaGraphCondAssignDefault));
    ZT_TRY(capture_begin(s, body_iter, &sg.k_iter));
    if (mixed)
        ZT_TRY(run_matvec<float>(p, nrhs, a.x32, (float2 *)p->ws32.yout, s));
    else
        ZT_TRY(run_matvec<double>(p, nrhs, w.xin64, w.w, s));
    ZT_TRY(ops.arnoldi(a, 1, s));
    ZT_TRY(add_conditional(s, a.h_reorth, cudaGraphCondTypeIf, &body_reorth));
    ZT_TRY(launch_small(k_iter_ctl, 1, a, h_iter, s));
    ZT_TRY(capture_end(s));
    ZT_TRY(capture_begin(s, body_reorth, &sg.k_reorth));
    ZT_TRY(ops.arnoldi(a, 2, s));
    ZT_TRY(capture_end(s));

    ZT_CUDA(cudaGraphInstantiate(&sg.exec, top, 0));
    sg.prec = prec;
    sg.nrhs = nrhs;
    sg.m = m;
    return ZTOEP_OK;
}

static ztoep_status_t get_graph(ztoep_plan_t p, int prec, int nrhs, int m, SolveGraph **out) {
    for (auto &g : p->graphs)
        if (g.exec && g.prec == prec && g.nrhs == nrhs && g.m == m) {
            *out = &g;
            return ZTOEP_OK;
        }
    SolveGraph &slot = p->graphs[p->graph_next];
    p->graph_next = (p->graph_next + 1) % 4;
    if (slot.exec) cudaGraphExecDestroy(slot.exec);
    if (slot.graph) cudaGraphDestroy(slot.graph);
    slot = SolveGraph{};
    ztoep_status_t st = build_graph(p, slot, prec, nrhs, m);
    if (st != ZTOEP_OK) {
        capture_count_end();
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(p->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(p->cap, &junk);
        }
        cudaGetLastError();
        if (slot.exec) cudaGraphExecDestroy(slot.exec);
        if (slot.graph) cudaGraphDestroy(slot.graph);
        slot = SolveGraph{};
        return st;
    }
    *out = &slot;
    return ZTOEP_OK;
}

// The same solve with the loops driven from the host: every kernel is a
// separate launch (for profilers that cannot see inside conditional graphs).
// The loop decisions are read back from the control block.
static ztoep_status_t run_host_loop(ztoep_plan_t p, int prec, int nrhs, int m, cudaStream_t s) {
    const bool mixed = prec == ZTOEP_MIXED;
    SolveWs &w = p->sws;
    const Geom gm = geom_for(p->N, p->nsm);
    const int per_cta = gm.threads * gm.elem;
    const int nchunk = (int)((p->N + per_cta - 1) / per_cta);
    const GArgs a = make_args(p, nrhs, m, mixed, nchunk);
    const Ops ops{gm, dim3(nchunk, nrhs)};
    SolveCtl *hc = reinterpret_cast<SolveCtl *>(w.hst + (size_t)w.cap * ST_STRIDE);
    auto read_ctl = [&]() -> ztoep_status_t {
        ZT_CUDA(cudaMemcpyAsync(hc, w.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
        ZT_CUDA(cudaStreamSynchronize(s));
        return ZTOEP_OK;
    };
    const cudaGraphConditionalHandle none = 0;
    ZT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(int) * (size_t)w.cap * ST_STRIDE, s));
    ZT_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * (size_t)w.cap * CNT_STRIDE, s));
    const int zblocks = (int)std::min<int64_t>(4 * p->nsm, ((int64_t)nrhs * p->N + 255) / 256);
    ZT_TRY(launch_small(k_solve_begin, std::max(1, zblocks), a, none, s, 0));
    ZT_TRY(ops.vnorm(a, s));
    ZT_TRY(read_ctl());
    if (hc->cond_first) ZT_TRY(run_matvec<double>(p, nrhs, w.xbuf, w.w, s));
    ZT_TRY(ops.residual(a, 1, s));
    ZT_TRY(launch_small(k_sweep_ctl, 1, a, none, s, 0));
    ZT_TRY(read_ctl());
    while (hc->cond_sweep) {
        ZT_TRY(launch_small(k_restart_begin, 1, a, none, s, 0));
        for (;;) {
            ZT_TRY(launch_small(k_cycle_begin, 1, a, none, s, 0));
            for (int it = 0; it < m; ++it) {
                if (mixed)
                    ZT_TRY(run_matvec<float>(p, nrhs, a.x32, (float2 *)p->ws32.yout, s));
                else
                    ZT_TRY(run_matvec<double>(p, nrhs, w.xin64, w.w, s));
                ZT_TRY(ops.arnoldi(a, 1, s));
                ZT_TRY(ops.arnoldi(a, 2, s));
                ZT_TRY(launch_small(k_iter_ctl, 1, a, none, s, 0));
                ZT_TRY(read_ctl());
                if (!hc->cond_iter) break;
            }
            ZT_TRY(ops.update_d(a, s));
            if (mixed) {
                ZT_TRY(run_matvec<float>(p, nrhs, a.x32, (float2 *)p->ws32.yout, s));
                ZT_TRY(ops.inner_residual(a, s));
            }
            ZT_TRY(launch_small(k_restart_ctl, 1, a, none, s, 0));
            ZT_TRY(read_ctl());
            if (!hc->cond_restart) break;
        }
        ZT_TRY(ops.apply_d(a, s));
        ZT_TRY(run_matvec<double>(p, nrhs, w.xbuf, w.w, s));
        ZT_TRY(ops.residual(a, 0, s));
        ZT_TRY(launch_small(k_sweep_ctl, 1, a, none, s, 0));
        ZT_TRY(read_ctl());
    }
    return ZTOEP_OK;
}

// Prepare buffers and the graph; V/X must already be in vbuf/xbuf (X only when
// no zero guess).  Runs the solve graph on `s` and fetches the per-RHS state.
static ztoep_status_t solve_core(ztoep_plan_t p, const ztoep_solve_opts_t *o, int nrhs, ztoep_solve_info_t *info,
                                 cudaStream_t s) {
    const int m = o->restart;
    const bool host_loop = (o->flags & ZTOEP_FLAG_HOST_LOOP) != 0;
    SolveGraph *g = nullptr;
    if (!host_loop) ZT_TRY(get_graph(p, o->prec, nrhs, m, &g));
    SolveWs &w = p->sws;
    SolveCtl *hc = reinterpret_cast<SolveCtl *>(w.hst + (size_t)w.cap * ST_STRIDE);
    std::memset(hc, 0, sizeof(SolveCtl));
    hc->zero = (o->flags & ZTOEP_FLAG_ZERO_GUESS) ? 1 : 0;
    hc->max_iter = o->max_iter;
    hc->max_outer = o->max_outer;
    hc->tol = o->tol;
    hc->inner_tol = o->inner_tol;
    hc->timeout_ns = o->timeout_ns;
    ZT_CUDA(cudaMemcpyAsync(w.ctl, hc, sizeof(SolveCtl), cudaMemcpyHostToDevice, s));
    if (host_loop)
        ZT_TRY(run_host_loop(p, o->prec, nrhs, m, s));
    else
        ZT_CUDA(cudaGraphLaunch(g->exec, s));
    ZT_CUDA(cudaMemcpyAsync(w.hst, w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE, cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaMemcpyAsync(hc, w.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaMemcpyAsync(w.hnrm, w.nrm, sizeof(double) * (size_t)nrhs * NM_STRIDE, cudaMemcpyDeviceToHost, s));
    int dev_err = 0;
    ZT_CUDA(cudaMemcpyAsync(&dev_err, p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaStreamSynchronize(s));
    if (g)
        add_launches(g->k_fixed + (hc->zero ? 0 : g->k_first_product) + (uint64_t)hc->outer_bodies * g->k_sweep +
                     (uint64_t)hc->restart_bodies * g->k_restart + (uint64_t)hc->inner_bodies * g->k_iter +
                     (uint64_t)hc->reorth_bodies * g->k_reorth);
    bool timed_out = hc->timed_out != 0;
    if (dev_err != 0) {  // a bounded device-side wait gave up
        ZT_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), s));
        timed_out = true;
    }
    ztoep_status_t worst = ZTOEP_OK;
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
        if (dev_err != 0) rs = ZTOEP_ERR_TIMEOUT;
        if (rs != ZTOEP_OK && (worst == ZTOEP_OK || rs == ZTOEP_ERR_NONFINITE || rs == ZTOEP_ERR_TIMEOUT))
            worst = rs;
        if (info) {
            info[rr].outer = st[ST_OUTER];
            info[rr].inner_iters = st[ST_ITERS];
            info[rr].status = rs;
            info[rr].rel_residual = nm[NM_VNORM] > 0 ? nm[NM_RNORM] / nm[NM_VNORM] : nm[NM_RNORM];
        }
    }
    return worst;
}

static ztoep_status_t prepare(ztoep_plan_t p, const ztoep_solve_opts_t *o, int nrhs, cudaStream_t s) {
    ZT_TRY(ensure_solve_ws(p, nrhs, o->restart));
    if (o->prec == ZTOEP_MIXED) {
        ZT_TRY(ensure_ws<float>(p, nrhs));
        ZT_TRY(ensure_tensor_data(p, nrhs, s));
    }
    ZT_TRY(ensure_ws<double>(p, nrhs));
    return ZTOEP_OK;
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
    cudaStream_t s = (cudaStream_t)stream;
    ZT_TRY(prepare(p, o, nrhs, s));
    SolveWs &w = p->sws;
    const size_t bytes = sizeof(double2) * (size_t)nrhs * p->N;
    ZT_CUDA(cudaMemcpyAsync(w.vbuf, V, bytes, cudaMemcpyDeviceToDevice, s));
    if (!(o->flags & ZTOEP_FLAG_ZERO_GUESS)) ZT_CUDA(cudaMemcpyAsync(w.xbuf, X, bytes, cudaMemcpyDeviceToDevice, s));
    const ztoep_status_t st = solve_core(p, o, nrhs, info, s);
    if (st == ZTOEP_ERR_ARG || st == ZTOEP_ERR_CUDA || st == ZTOEP_ERR_NOMEM || st == ZTOEP_ERR_UNSUPPORTED)
        return st;
    ZT_CUDA(cudaMemcpyAsync(X, w.xbuf, bytes, cudaMemcpyDeviceToDevice, s));
    return st;
}

ztoep_status_t ztoep_solve_host(ztoep_plan_t p, const ztoep_solve_opts_t *o, int32_t nrhs, const void *Vh,
                                void *Xh, ztoep_solve_info_t *info, void *stream) {
    if (!p || !valid_opts(o) || nrhs < 1 || !Vh || !Xh) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStream_t s = (cudaStream_t)stream;
    ZT_TRY(prepare(p, o, nrhs, s));
    SolveWs &w = p->sws;
    const size_t bytes = sizeof(double2) * (size_t)nrhs * p->N;
    ZT_CUDA(cudaMemcpyAsync(w.vbuf, Vh, bytes, cudaMemcpyHostToDevice, s));
    if (!(o->flags & ZTOEP_FLAG_ZERO_GUESS)) ZT_CUDA(cudaMemcpyAsync(w.xbuf, Xh, bytes, cudaMemcpyHostToDevice, s));
    const ztoep_status_t st = solve_core(p, o, nrhs, info, s);
    if (st == ZTOEP_ERR_ARG || st == ZTOEP_ERR_CUDA || st == ZTOEP_ERR_NOMEM || st == ZTOEP_ERR_UNSUPPORTED)
        return st;
    ZT_CUDA(cudaMemcpyAsync(Xh, w.xbuf, bytes, cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"
