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
// Every step kernel runs over a work list: the RHS of one or several systems
// (a group of plans of any sizes, one launch per step for all of them), each
// RHS cut into chunks whose size depends only on its system.  Each RHS stops
// on its own flags.  Cross-CTA sums use last-arriver tickets (no waiting) and
// a fixed summation order, so a RHS is summed identically alone, in a batch
// and in a group.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {

enum { ST_ACTIVE = 0, ST_JLEN = 1, ST_ITERS = 2, ST_STATUS = 3, ST_OUTER = 4, ST_PENDING = 5, ST_REORTH = 6,
       ST_INNER = 7, ST_RESTARTS = 8, ST_END = 9, ST_COLUMN = 10, ST_PASSES2 = 11, ST_STRIDE = 12 };
// ST_END: the column just finalised ends the cycle; the iteration control
// turns it into ACTIVE = 0, PENDING = 1 once every kernel of the step is done
// (the Arnoldi kernels of the step test ACTIVE, so it must not change under them).
// ST_COLUMN: Hessenberg column ctl->j - 1 is orthogonalised (its entries and
// beta stored) and waits for its Givens rotations, which run beside the next
// step's product.
enum { RS_RUNNING = 0, RS_CONVERGED = 1, RS_NONFINITE = 2, RS_MAXITER = 3 };
enum { NM_VNORM = 0, NM_TARGET = 2, NM_RNORM = 3, NM_RIN = 6, NM_STRIDE = 8 };
// Inner (FP32-residual) restarts of one sweep: at most this many, and they stop
// early when a restart reduces the inner residual by less than 10%.
constexpr int kMaxRestarts = 64;
constexpr double kStagnation = 0.9;
// Second Gram-Schmidt pass when ||w'|| < eta ||w||.  The orthogonality lost by
// one classical pass is about u ||w|| / ||w'||, so eta = 1/64 keeps it below
// 64 u (~7e-15), far under what the residual targets need, while skipping the
// pass in the usual case (the stricter 1/sqrt(2) of "twice is enough" asked
// for it at every step on these systems, doubling the FP64 work).
constexpr double kReorthEta = 1.0 / 64.0;
// Chunks per first-level group of the cross-CTA reductions.
// Largest Gram-Schmidt column: j + 2 <= m + 1 with m <= 128.
constexpr int kMaxK = 130;
// Systems solved together in one group (one launch per step for all).
constexpr int kMaxMembers = 8;

// Device-side control of one solve (written by the host before each launch of
// the solve graph; loop counters advanced by the control kernels).  A group
// of systems shares one.
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
    int reorth_pending;  // the step's second Gram-Schmidt pass (and iteration control) is still to run
    unsigned tick;       // last-arriver ticket of the update kernel's grid
    int cycle_bodies;    // iteration bodies run in the current cycle (at most m + 1 in a correct run)
    int guard;           // the iteration guard stopped the loops (a body count beyond its bound)
    double tol, inner_tol;
    long long timeout_ns;
    unsigned long long deadline;  // %globaltimer value, 0 = none
};

// One system's view of its solve workspace.
struct GArgs {
    double2 *Vb;       // [(m+1)][cap][N] unnormalised basis u_k
    double2 *w;        // [cap][N] FP64 product output
    double2 *x;        // [nrhs][N] iterate
    const double2 *v;  // [nrhs][N] right-hand sides
    float2 *x32;       // [cap][N] FP32 copy of the next product input (MIXED)
    const float2 *y32; // [cap][N] FP32 product output (MIXED)
    double2 *H, *cs, *sn, *g, *h1, *h2;
    double2 *part;     // [cap][nrows][pstride] chunk partial sums and the reduction tree's inner nodes
    double *beta;      // [cap][m+1] ||u_k||
    double *ibeta;     // [cap][m+1] 1 / ||u_k||, stored with beta (no division on the step kernels)
    double2 *xin64;    // [cap][N] FP64 copy of the next product input (FP64)
    double2 *rbuf;     // [cap][N] FP64 residual r of the sweep
    double2 *dbuf;     // [cap][N] correction d of the sweep
    double *nrm;
    int *st;
    unsigned *cnt;     // [cap][cstride] reduction tickets
    SolveCtl *ctl;     // shared by the group
    int64_t N;
    int cap, m, nchunk, per_cta, nrows, cstride, pstride, nrhs;
    int mixed;
};

// A launch's work list: the member systems, all with the same elements per
// thread (ELEM of the kernel); member i owns (nchunk_i [+ 1]) * nrhs_i
// consecutive CTAs.
struct GroupArgs {
    int n;
    int graph;                                     // running inside a solve graph
    cudaGraphConditionalHandle h_iter, h_reorth;   // iteration loop, second Gram-Schmidt pass
    int prod_if;                                   // the members' iteration products sit in IF nodes
    cudaGraphConditionalHandle h_prod[kMaxMembers];
    GArgs m[kMaxMembers];
};

struct Loc {
    int mi, rr, cx;
};

// The CTA's member, RHS and chunk (extra: one more CTA per RHS after its chunks).
__device__ __forceinline__ Loc locate(const GroupArgs &g, bool extra) {
    int b = blockIdx.x;
    for (int i = 0; i < g.n; ++i) {
        const int per = g.m[i].nchunk + (extra ? 1 : 0);
        const int cnt = per * g.m[i].nrhs;
        if (b < cnt) {
            const int rr = b / per;
            return {i, rr, b - rr * per};
        }
        b -= cnt;
    }
    return {-1, 0, 0};
}

// Element e of this thread in chunk cx: its index, or -1 outside the chunk.
__device__ __forceinline__ int64_t elem_index(const GArgs &a, int cx, int e) {
    const int off = e * blockDim.x + threadIdx.x;
    const int64_t idx = (int64_t)cx * a.per_cta + off;
    return (off < a.per_cta && idx < a.N) ? idx : -1;
}

__device__ __forceinline__ double2 *part_rows(const GArgs &a, int rr) {
    return a.part + (int64_t)rr * a.nrows * a.pstride;
}

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

// Cross-CTA sums use one fixed tree over the chunks of a RHS: nodes of 16
// chunks at the first level and of 32 nodes above, each node the pairwise
// sum ((v0 + v1) + (v2 + v3)) + ... of its children, zero-padded to the full
// fan-in.  The tree depends only on the chunk count, so a RHS is summed in the
// same order alone, in any batch and in any group.
constexpr int kFan0 = 16, kFanUp = 32;
__host__ __device__ inline int tree_fan(int level) { return level == 0 ? kFan0 : kFanUp; }
// Stored rows per RHS (every level but the root) and tickets (every node above the chunks).
__host__ __device__ inline int tree_rows(int nchunk) {
    int n = nchunk, rows = 0, l = 0;
    while (true) {
        const int np = (n + tree_fan(l) - 1) / tree_fan(l);
        rows += n;
        if (np == 1) return rows;
        n = np;
        ++l;
    }
}
__host__ __device__ inline int tree_tickets(int nchunk) {
    int n = nchunk, t = 0, l = 0;
    while (true) {
        const int np = (n + tree_fan(l) - 1) / tree_fan(l);
        t += np;
        if (np == 1) return t;
        n = np;
        ++l;
    }
}

// One node: the pairwise tree over FAN values ld(i) (i < nch, zero beyond).
template <int FAN, typename Ld> __device__ __forceinline__ double2 fan_sum(int nch, Ld ld) {
    double2 v[FAN];
#pragma unroll
    for (int i = 0; i < FAN; ++i) v[i] = i < nch ? ld(i) : make_double2(0, 0);
#pragma unroll
    for (int w = 1; w < FAN; w *= 2)
#pragma unroll
        for (int i = 0; i < FAN; i += 2 * w) v[i] = v[i] + v[i + w];
    return v[0];
}
__device__ __forceinline__ double2 node_sum(int level, const double2 *src, int nch, int64_t stride, bool global) {
    if (global) {
        if (level == 0) return fan_sum<kFan0>(nch, [&](int i) { return __ldcg(src + i * stride); });
        return fan_sum<kFanUp>(nch, [&](int i) { return __ldcg(src + i * stride); });
    }
    if (level == 0) return fan_sum<kFan0>(nch, [&](int i) { return src[i * stride]; });
    return fan_sum<kFanUp>(nch, [&](int i) { return src[i * stride]; });
}

// Cross-CTA sum of one RHS's partial rows (chunk cx has written row cx,
// columns 0..K-1): the last CTA to finish among a node's children forms the
// node (a row of the next level), and so on up; the CTA that forms the root
// writes it to tot[0..K) (shared memory) and returns true (all threads).  The
// tickets are last-arriver counters that reset themselves; nothing waits.
__device__ bool reduce_rows(const GArgs &a, int rr, int cx, int K, double2 *tot) {
    __shared__ unsigned s_t;
    double2 *rows = part_rows(a, rr);
    unsigned *cnt = a.cnt + (int64_t)rr * a.cstride;
    int node = cx, n = a.nchunk, roff = 0, coff = 0;
    for (int level = 0;; ++level) {
        const int fan = tree_fan(level);
        const int parent = node / fan, first = parent * fan, nch = min(fan, n - first);
        const int np = (n + fan - 1) / fan;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(cnt + coff + parent, 1u);
        __syncthreads();
        if (s_t != (unsigned)nch - 1) return false;
        __threadfence();
        if (threadIdx.x == 0) cnt[coff + parent] = 0u;  // no other CTA of this launch touches it again
        const double2 *src = rows + (int64_t)(roff + first) * a.pstride;
        double2 *dst = np == 1 ? tot : rows + (int64_t)(roff + n + parent) * a.pstride;
        for (int k = threadIdx.x; k < K; k += blockDim.x) dst[k] = node_sum(level, src + k, nch, a.pstride, true);
        if (np == 1) {
            __syncthreads();
            return true;
        }
        roff += n;
        coff += np;
        node = parent;
        n = np;
    }
}

__device__ __forceinline__ double2 *basis(const GArgs &a, int k, int rr) {
    return a.Vb + ((int64_t)k * a.cap + rr) * a.N;
}

// acc - c * u with four fused multiply-adds
__device__ __forceinline__ double2 cfms(double2 c, double2 u, double2 acc) {
    acc.x = fma(-c.x, u.x, acc.x);
    acc.x = fma(c.y, u.y, acc.x);
    acc.y = fma(-c.x, u.y, acc.y);
    acc.y = fma(-c.y, u.x, acc.y);
    return acc;
}

// ---------------------------------------------------------------- norms
template <int ELEM> __global__ void __launch_bounds__(256) k_vnorm(const __grid_constant__ GroupArgs g) {
    __shared__ double red[8];
    __shared__ double2 tot[1];
    const Loc L = locate(g, false);
    if (L.mi < 0) return;
    const GArgs &a = g.m[L.mi];
    const int rr = L.rr;
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = elem_index(a, L.cx, e);
        if (idx >= 0) acc += cabs2(a.v[(int64_t)rr * a.N + idx]);
    }
    acc = block_sum1(acc, red);
    if (threadIdx.x == 0) part_rows(a, rr)[(int64_t)L.cx * a.pstride] = make_double2(acc, 0);
    if (reduce_rows(a, rr, L.cx, 1, tot) && threadIdx.x == 0) a.nrm[rr * NM_STRIDE + NM_VNORM] = sqrt(tot[0].x);
}

// u_0 = v - Z'x (w holds Z'x) or v (zero guess), its FP32 copy, ||u_0||, stop
// test and the start of a cycle.
template <int ELEM> __global__ void __launch_bounds__(256) k_residual(const __grid_constant__ GroupArgs g, int first) {
    __shared__ double red[8];
    __shared__ double2 tot[1];
    const Loc L = locate(g, false);
    if (L.mi < 0) return;
    const GArgs &a = g.m[L.mi];
    const int rr = L.rr;
    int *st = a.st + rr * ST_STRIDE;
    if (st[ST_STATUS] != RS_RUNNING) return;
    const int zero = first && a.ctl->zero;
    double2 *u0 = basis(a, 0, rr);
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = elem_index(a, L.cx, e);
        if (idx >= 0) {
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
    if (threadIdx.x == 0) part_rows(a, rr)[(int64_t)L.cx * a.pstride] = make_double2(acc, 0);
    if (!reduce_rows(a, rr, L.cx, 1, tot)) return;
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
    st[ST_COLUMN] = 0;
    st[ST_END] = 0;
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
        a.ibeta[(int64_t)rr * (a.m + 1)] = 1.0 / rn;
        const double floor_abs = 0.5 * a.ctl->tol * vn;
        nm[NM_TARGET] = a.mixed ? fmax(a.ctl->inner_tol * rn, floor_abs) : floor_abs;
        double2 *gg = a.g + (int64_t)rr * (a.m + 1);
        gg[0] = make_double2(rn, 0);
        for (int i = 1; i <= a.m; ++i) gg[i] = make_double2(0, 0);
    }
}

// ---------------------------------------------------------------- Arnoldi
// Givens rotations of Hessenberg column j (stored unrotated in H by the
// update kernel, with beta_{j+1}): the earlier rotations, the new one, the
// residual estimate and the end-of-cycle decision.  Called by every thread
// of one CTA; the rotation chain runs in one thread on shared copies.  It
// runs beside the next step's product (which does no FP64 work), off the
// Arnoldi kernels' path.  The least squares R y = g is solved at the update
// (k_update_d).
__device__ void givens_column(const GArgs &a, int rr, int j) {
    __shared__ double2 s_cs[128], s_sn[128], hs[129];
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
    for (int i = threadIdx.x; i <= j; i += blockDim.x) hs[i] = __ldcg(H + (int64_t)i * m + j);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double beta = a.beta[(int64_t)rr * (m + 1) + j + 1];
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
        st[ST_COLUMN] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) H[(int64_t)i * m + j] = hs[i];
}

// After the first Gram-Schmidt pass (hs[k] = h_k for k <= j, shared memory;
// w2 = ||w||^2): ||w - V h||^2 = ||w||^2 - sum |h_k|^2 (exact for orthonormal
// v_k up to rounding of order u ||w||^2 / ||w'||^2, below 4096 u when no
// second pass is taken); strong cancellation (or NaN) asks for the second
// pass.  The column h goes to H; without a second pass beta_{j+1} = ||w'|| is
// stored and the column waits for its rotations.  Whole CTA; the sum of
// |h_k|^2 is a fixed-order warp tree.
__device__ int column_decision(const GArgs &a, int rr, int j, const double2 *hs, double w2, bool store) {
    __shared__ double s_hsq;
    int *st = a.st + rr * ST_STRIDE;
    const int m = a.m;
    double2 *H = a.H + (int64_t)rr * (m + 1) * m;
    if (store)
        for (int i = threadIdx.x; i <= j; i += blockDim.x) H[(int64_t)i * m + j] = hs[i];
    if (threadIdx.x < 32) {
        double v = 0;
        for (int k = threadIdx.x; k <= j; k += 32) v += cabs2(hs[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_hsq = v;
    }
    __syncthreads();
    const double wn2 = w2 - s_hsq;
    const int again = !(wn2 > kReorthEta * kReorthEta * w2);
    if (store && threadIdx.x == 0) {
        st[ST_REORTH] = again;
        st[ST_PASSES2] += again;
        if (!again) {
            const double bn = sqrt(wn2);
            a.beta[(int64_t)rr * (m + 1) + j + 1] = bn;
            a.ibeta[(int64_t)rr * (m + 1) + j + 1] = 1.0 / bn;
            st[ST_COLUMN] = 1;
        }
    }
    __syncthreads();
    return again;
}

// Partial dot products <u_k, w> for k in [k0, k0+8) (k <= j) plus, when
// with_norm and k0 + kk == j + 1, ||w||^2 in that slot: per-thread sums,
// then one warp reduce-scatter; the warp's 8 totals go to wred[warp][k0..].
// No block barrier here: the warps are added once after all groups.
template <int ELEM>
__device__ __forceinline__ void dots_group(const GArgs &a, int rr, int j, int k0, int K, bool with_norm,
                                           const double2 (&wv)[ELEM], const int64_t (&ix)[ELEM],
                                           double2 (*wred)[kMaxK]) {
    double2 acc[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) acc[kk] = make_double2(0, 0);
    if (k0 + 7 <= j) {  // full group: the 8 loads of an element are in flight together
        const double2 *u0 = basis(a, k0, rr);
        const int64_t vstride = (int64_t)a.cap * a.N;
#pragma unroll
        for (int e = 0; e < ELEM; ++e) {
            if (ix[e] >= 0) {
                double2 uv[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) uv[kk] = u0[kk * vstride + ix[e]];
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
                for (int e = 0; e < ELEM; ++e)
                    if (ix[e] >= 0) acc[kk] = cfmac(uk[ix[e]], wv[e], acc[kk]);
            } else if (with_norm && k == j + 1) {
#pragma unroll
                for (int e = 0; e < ELEM; ++e) acc[kk].x += cabs2(wv[e]);
            }
        }
    }
    warp_rs8(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if ((lane & 3) == 0) {
        const int kk = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (k0 + kk < K) wred[warp][k0 + kk] = acc[0];
    }
}

// Guard: every iteration body advances j, so a cycle runs at most m + 1
// bodies (one after its end is seen); beyond that the loops are ended and the
// solve reports TIMEOUT rather than running on.  Block 0, thread 0 of the
// step's first kernel.
__device__ __forceinline__ void iteration_guard(const GroupArgs &g) {
    SolveCtl *c = g.m[0].ctl;
    if (++c->cycle_bodies > g.m[0].m + 2) {
        c->guard = 1;
        c->timed_out = 1;
        c->cond_iter = 0;
        if (g.graph) cudaGraphSetConditional(g.h_iter, 0u);
    }
}

// The chunk's partial row of the Gram-Schmidt sums (whole CTA).
// PASS 1: w = (product of u_j) / beta_j is formed (from the FP32 or FP64
//   product) and stored as u_{j+1}; row = <u_k, w> (k <= j) and ||w||^2.
// PASS 2: row = <u_k, u_{j+1}> (k <= j).  Returns the row length K.
template <int ELEM, int PASS>
__device__ int dots_row(const GArgs &a, int rr, int cx, int j, double2 (*wred)[kMaxK]) {
    double2 *un = basis(a, j + 1, rr);
    double2 wv[ELEM];
    int64_t ix[ELEM];
    const double sc = a.ibeta[(int64_t)rr * (a.m + 1) + j];
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        ix[e] = elem_index(a, cx, e);
        wv[e] = make_double2(0, 0);
        if (ix[e] >= 0) {
            if (PASS == 1) {
                const int64_t o = (int64_t)rr * a.N + ix[e];
                double2 t;
                if (a.mixed) {
                    const float2 f = a.y32[o];
                    t = make_double2(f.x, f.y);
                } else {
                    t = a.w[o];
                }
                wv[e] = cscale(t, sc);
                un[ix[e]] = wv[e];
            } else {
                wv[e] = un[ix[e]];
            }
        }
    }
    const int K = j + 1 + (PASS == 1 ? 1 : 0);
    for (int k0 = 0; k0 < K; k0 += 8) dots_group<ELEM>(a, rr, j, k0, K, PASS == 1, wv, ix, wred);
    __syncthreads();
    double2 *row = part_rows(a, rr) + (int64_t)cx * a.pstride;
    for (int k = threadIdx.x; k < K; k += blockDim.x)  // the 8 warps' sums, pairwise
        row[k] = ((wred[0][k] + wred[1][k]) + (wred[2][k] + wred[3][k])) +
                 ((wred[4][k] + wred[5][k]) + (wred[6][k] + wred[7][k]));
    return K;
}

// Gram-Schmidt dots: the chunk rows, then the last CTA stores the sums
// unscaled (PASS 1: h1_k = beta_k <v_k, w> and h1_{j+1} = ||w||^2, the update
// kernel scales, so no division sits on this kernel's serial tail; PASS 2
// (flagged RHS only): h2_k = beta_k <v_k, u_{j+1}>).
template <int ELEM, int PASS> __global__ void __launch_bounds__(256) k_dots(const __grid_constant__ GroupArgs g) {
    __shared__ double2 wred[8][kMaxK];
    __shared__ double2 tot[kMaxK];
    if (PASS == 1 && blockIdx.x == 0 && threadIdx.x == 0) iteration_guard(g);
    const Loc L = locate(g, false);
    if (L.mi < 0) return;
    const GArgs &a = g.m[L.mi];
    const int rr = L.rr;
    const int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_ACTIVE]) return;
    if (PASS == 2 && !st[ST_REORTH]) return;
    const int j = a.ctl->j;
    if (j >= a.m) return;
    const int K = dots_row<ELEM, PASS>(a, rr, L.cx, j, wred);
    if (!reduce_rows(a, rr, L.cx, K, tot)) return;
    double2 *h = (PASS == 1 ? a.h1 : a.h2) + (int64_t)rr * (a.m + 1);
    for (int k = threadIdx.x; k < K; k += blockDim.x) h[k] = tot[k];  // (PASS 1: ||w||^2 in slot j+1)
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool past_deadline(const SolveCtl *c) {
    return c->deadline != 0ull && globaltimer_ns() > c->deadline;
}

// Some RHS of some member with flag f set (whole CTA).
__device__ __forceinline__ bool any_flag(const GroupArgs &g, int f, int f2 = -1) {
    int any = 0;
    for (int i = 0; i < g.n; ++i)
        for (int rr = threadIdx.x; rr < g.m[i].nrhs; rr += blockDim.x) {
            const int *st = g.m[i].st + rr * ST_STRIDE;
            any |= st[f] && (f2 < 0 || st[f2]);
        }
    return __syncthreads_or(any) != 0;
}

// End of an Arnoldi step (one CTA): cycles that ended in this step close
// (ACTIVE -> 0, PENDING -> 1), then the next iteration runs while some RHS is
// still in its cycle; members with no RHS in a cycle skip their next product.
__device__ void iteration_control(const GroupArgs &g) {
    for (int i = 0; i < g.n; ++i)
        for (int rr = threadIdx.x; rr < g.m[i].nrhs; rr += blockDim.x) {
            int *st = g.m[i].st + rr * ST_STRIDE;
            if (st[ST_END]) {
                st[ST_END] = 0;
                st[ST_ACTIVE] = 0;
                st[ST_PENDING] = 1;
            }
        }
    __syncthreads();
    const bool any = any_flag(g, ST_ACTIVE);
    unsigned member_on[kMaxMembers];
    if (g.prod_if)
        for (int i = 0; i < g.n; ++i) {
            int on = 0;
            for (int rr = threadIdx.x; rr < g.m[i].nrhs; rr += blockDim.x) on |= g.m[i].st[rr * ST_STRIDE + ST_ACTIVE];
            member_on[i] = __syncthreads_or(on) ? 1u : 0u;
        }
    if (threadIdx.x != 0) return;
    SolveCtl *c = g.m[0].ctl;
    c->j += 1;
    c->inner_bodies += 1;
    c->reorth_pending = 0;
    const bool late = past_deadline(c);
    if (any && late) c->timed_out = 1;
    const unsigned cond = (any && c->j < g.m[0].m && !late && !c->guard) ? 1u : 0u;
    c->cond_iter = (int)cond;
    if (g.graph) {
        cudaGraphSetConditional(g.h_iter, cond);
        cudaGraphSetConditional(g.h_reorth, 0u);
        // next iteration's products: the members still in a cycle; when the
        // loop ends, all on again for the next cycle's first step
        if (g.prod_if)
            for (int i = 0; i < g.n; ++i) cudaGraphSetConditional(g.h_prod[i], cond ? member_on[i] : 1u);
    }
}

// u_{j+1} <- u_{j+1} - sum_k (h_k / beta_k) u_k and its copy for the next
// product, from the sums the dots kernel stored (h_k = that / beta_k).
// PASS 1: one extra CTA per RHS (cx == nchunk) takes the second-pass
//   decision and stores the column (and, without a second pass, beta_{j+1})
//   alongside the update; the last CTA of the whole grid then runs the
//   iteration control (or, when some RHS asked for a second pass, leaves it
//   to that pass).
// PASS 2 (after a second Gram-Schmidt pass): also forms ||u_{j+1}|| across
//   the chunks, adds h2 to the stored column and stores beta_{j+1}.
// hs_k = h_k / beta_k and the update coefficients cf_k = hs_k / beta_k
// (k <= j) from the step's sums h (whole CTA, ends with a barrier).
__device__ __forceinline__ void step_coefficients(const GArgs &a, int rr, int j, const double2 *h, bool global,
                                                  double2 *hs, double2 *cf) {
    const double *ibeta = a.ibeta + (int64_t)rr * (a.m + 1);
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        const double ib = ibeta[k];
        const double2 hk = cscale(global ? __ldcg(h + k) : h[k], ib);
        hs[k] = hk;
        cf[k] = cscale(hk, ib);
    }
    __syncthreads();
}

// The chunk's update u_{j+1} <- u_{j+1} - sum_k cf_k u_k, with its copy for
// the next product; returns the thread's share of ||u_{j+1}||^2.
template <int ELEM> __device__ double update_chunk(const GArgs &a, int rr, int cx, int j, const double2 *cf) {
    double2 *un = basis(a, j + 1, rr);
    double2 wv[ELEM];
    int64_t ix[ELEM];
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        ix[e] = elem_index(a, cx, e);
        wv[e] = ix[e] >= 0 ? un[ix[e]] : make_double2(0, 0);
    }
    int k = 0;
    const int64_t vstride = (int64_t)a.cap * a.N;
    constexpr int UNR = ELEM == 1 ? 8 : 4;  // basis vectors per step, loads first
    for (; k + UNR <= j + 1; k += UNR) {
        const double2 *u0 = basis(a, k, rr);
#pragma unroll
        for (int e = 0; e < ELEM; ++e) {
            if (ix[e] >= 0) {
                double2 uv[UNR];
#pragma unroll
                for (int kk = 0; kk < UNR; ++kk) uv[kk] = u0[kk * vstride + ix[e]];
#pragma unroll
                for (int kk = 0; kk < UNR; ++kk) wv[e] = cfms(cf[k + kk], uv[kk], wv[e]);
            }
        }
    }
    for (; k <= j; ++k) {
        const double2 c = cf[k];
        const double2 *uk = basis(a, k, rr);
#pragma unroll
        for (int e = 0; e < ELEM; ++e)
            if (ix[e] >= 0) wv[e] = cfms(c, uk[ix[e]], wv[e]);
    }
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        if (ix[e] >= 0) {
            un[ix[e]] = wv[e];
            if (a.mixed)
                a.x32[(int64_t)rr * a.N + ix[e]] = make_float2((float)wv[e].x, (float)wv[e].y);
            else
                a.xin64[(int64_t)rr * a.N + ix[e]] = wv[e];
            acc += cabs2(wv[e]);
        }
    }
    return acc;
}

// After the second pass (the CTA that formed ||u_{j+1}||^2 = n2): H gets
// h1 + h2 and beta_{j+1} is stored; the column waits for its rotations.
__device__ void second_pass_close(const GArgs &a, int rr, int j, const double2 *hs2, double n2) {
    int *st = a.st + rr * ST_STRIDE;
    const int m = a.m;
    double2 *H = a.H + (int64_t)rr * (m + 1) * m;
    for (int kk = threadIdx.x; kk <= j; kk += blockDim.x)
        H[(int64_t)kk * m + j] = __ldcg(H + (int64_t)kk * m + j) + hs2[kk];  // h1 + h2
    if (threadIdx.x == 0) {
        const double bn = sqrt(n2);
        a.beta[(int64_t)rr * (m + 1) + j + 1] = bn;
        a.ibeta[(int64_t)rr * (m + 1) + j + 1] = 1.0 / bn;
        st[ST_REORTH] = 0;
        st[ST_COLUMN] = 1;
    }
}

template <int ELEM, int PASS> __global__ void __launch_bounds__(256) k_upd(const __grid_constant__ GroupArgs g) {
    __shared__ double red[8];
    __shared__ double2 cf[kMaxK];
    __shared__ double2 hs[kMaxK];
    __shared__ double2 tot[1];
    __shared__ unsigned s_t;
    const Loc L = locate(g, PASS == 1);
    if (L.mi >= 0) {
        const GArgs &a = g.m[L.mi];
        const int rr = L.rr;
        int *st = a.st + rr * ST_STRIDE;
        const int j = a.ctl->j;
        const bool work = st[ST_ACTIVE] && (PASS == 1 || st[ST_REORTH]) && j < a.m;
        if (work) {
            const double2 *h = (PASS == 1 ? a.h1 : a.h2) + (int64_t)rr * (a.m + 1);
            step_coefficients(a, rr, j, h, true, hs, cf);
            if (PASS == 1 && L.cx == a.nchunk) {
                column_decision(a, rr, j, hs, __ldcg(h + j + 1).x, true);
            } else {
                double acc = update_chunk<ELEM>(a, rr, L.cx, j, cf);
                if (PASS == 2) {
                    acc = block_sum1(acc, red);
                    if (threadIdx.x == 0) part_rows(a, rr)[(int64_t)L.cx * a.pstride] = make_double2(acc, 0);
                    if (reduce_rows(a, rr, L.cx, 1, tot)) second_pass_close(a, rr, j, hs, tot[0].x);
                }
            }
        }
    }
    if (PASS != 1) return;
    // the last CTA of the grid: iteration control, unless a second pass is due
    SolveCtl *c = g.m[0].ctl;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_t = atomicAdd(&c->tick, 1u);
    __syncthreads();
    if (s_t != gridDim.x - 1) return;
    __threadfence();
    if (threadIdx.x == 0) c->tick = 0u;
    if (any_flag(g, ST_ACTIVE, ST_REORTH)) {
        if (threadIdx.x == 0) {
            c->reorth_pending = 1;
            c->reorth_bodies += 1;
            if (g.graph) cudaGraphSetConditional(g.h_reorth, 1u);
        }
        return;
    }
    iteration_control(g);
}

// Givens rotations of the stored column ctl->j - 1, one CTA per RHS (member
// i owns nrhs_i CTAs).  In the iteration loop it runs beside the product of
// the next step; FINAL (after the loop) also closes the cycle of every RHS
// still in one (it reached the restart length or the deadline).
template <bool FINAL> __global__ void __launch_bounds__(128) k_givens(const __grid_constant__ GroupArgs g) {
    int b = blockIdx.x, mi = 0;
    while (mi < g.n && b >= g.m[mi].nrhs) b -= g.m[mi++].nrhs;
    if (mi >= g.n) return;
    const GArgs &a = g.m[mi];
    int *st = a.st + b * ST_STRIDE;
    const int j = a.ctl->j - 1;
    if (!st[ST_ACTIVE]) return;
    if (j >= 0 && j < a.m && st[ST_COLUMN]) givens_column(a, b, j);
    if (FINAL && threadIdx.x == 0) {
        st[ST_END] = 0;
        st[ST_ACTIVE] = 0;
        st[ST_PENDING] = 1;
    }
}

// After a second Gram-Schmidt pass: the step's iteration control.
__global__ void k_iter_ctl(const __grid_constant__ GroupArgs g) { iteration_control(g); }

// Least squares of a finished cycle: R y = g with R the leading jl x jl
// upper triangle of the rotated Hessenberg matrix; ys[k] = y_k / beta_k.
// Every CTA of the RHS solves it (the same arithmetic, so the same result):
// R is staged in shared memory by all threads, the reciprocals of its
// diagonal are formed in parallel (so no division sits in the serial chain:
// a dependent FP64 operation costs hundreds of cycles on this GPU), and one
// warp runs the column-oriented back substitution (lane l keeps the running
// right-hand side of row l).  Cycles longer than 32 fall back to one thread
// reading R from global memory.
__device__ void cycle_least_squares(const GArgs &a, int rr, int jl, double2 *ys) {
    __shared__ double2 Rs[32 * 32];
    __shared__ double2 rinv[32];
    const int m = a.m;
    const double2 *H = a.H + (int64_t)rr * (m + 1) * m;
    const double2 *g = a.g + (int64_t)rr * (m + 1);
    const double *ibeta = a.ibeta + (int64_t)rr * (m + 1);
    if (jl <= 32) {
        for (int idx = threadIdx.x; idx < jl * jl; idx += blockDim.x) {
            const int i = idx / jl, l = idx - i * jl;
            if (l >= i) Rs[i * 32 + l] = __ldcg(H + i * m + l);
        }
        if (threadIdx.x < jl) {
            const double2 rii = __ldcg(H + threadIdx.x * m + threadIdx.x);
            rinv[threadIdx.x] = (rii.x != 0.0 || rii.y != 0.0) ? cdiv(make_double2(1, 0), rii) : make_double2(0, 0);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double2 sl = lane < jl ? __ldcg(g + lane) : make_double2(0, 0);
            for (int i = jl - 1; i >= 0; --i) {
                double2 yi = make_double2(0, 0);
                if (lane == i) {
                    yi = cmul(sl, rinv[i]);
                    ys[i] = cscale(yi, ibeta[i]);
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
            ys[i] = cscale(yv[i], ibeta[i]);
        }
    }
    __syncthreads();
}

// d <- d + sum_k (y_k / beta_k) u_k for RHS whose cycle produced an update.
template <int ELEM> __global__ void __launch_bounds__(256) k_update_d(const __grid_constant__ GroupArgs g) {
    __shared__ double2 ys[128];
    const Loc L = locate(g, false);
    if (L.mi < 0) return;
    const GArgs &a = g.m[L.mi];
    const int rr = L.rr;
    const int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_PENDING]) return;
    const int jl = st[ST_JLEN];
    cycle_least_squares(a, rr, jl, ys);
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = elem_index(a, L.cx, e);
        if (idx >= 0) {
            const int64_t o = (int64_t)rr * a.N + idx;
            double2 s = a.dbuf[o];
            for (int k = 0; k < jl; ++k) s = cfma(ys[k], basis(a, k, rr)[idx], s);
            a.dbuf[o] = s;
            if (a.mixed) a.x32[o] = make_float2((float)s.x, (float)s.y);  // input of the restart product
        }
    }
}

// x <- x + d at the end of a sweep.
template <int ELEM> __global__ void __launch_bounds__(256) k_apply_d(const __grid_constant__ GroupArgs g) {
    const Loc L = locate(g, false);
    if (L.mi < 0) return;
    const GArgs &a = g.m[L.mi];
    const int rr = L.rr;
    if (!a.st[rr * ST_STRIDE + ST_INNER]) return;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = elem_index(a, L.cx, e);
        if (idx >= 0) {
            const int64_t o = (int64_t)rr * a.N + idx;
            a.x[o] = a.x[o] + a.dbuf[o];
        }
    }
}

// Inner restart (MIXED): r_in = r - Z32 d with the FP32 product of d in y32;
// r_in becomes u_0 of a new cycle unless the inner target is met, the restart
// gained less than 10%, or a cap is reached.
template <int ELEM> __global__ void __launch_bounds__(256) k_inner_residual(const __grid_constant__ GroupArgs g) {
    __shared__ double red[8];
    __shared__ double2 tot[1];
    const Loc L = locate(g, false);
    if (L.mi < 0) return;
    const GArgs &a = g.m[L.mi];
    const int rr = L.rr;
    int *st = a.st + rr * ST_STRIDE;
    if (!st[ST_INNER] || !st[ST_PENDING]) return;
    double2 *u0 = basis(a, 0, rr);
    double acc = 0;
#pragma unroll
    for (int e = 0; e < ELEM; ++e) {
        const int64_t idx = elem_index(a, L.cx, e);
        if (idx >= 0) {
            const int64_t o = (int64_t)rr * a.N + idx;
            const float2 f = a.y32[o];
            const double2 t = a.rbuf[o] - make_double2(f.x, f.y);
            u0[idx] = t;
            a.x32[o] = make_float2((float)t.x, (float)t.y);
            acc += cabs2(t);
        }
    }
    acc = block_sum1(acc, red);
    if (threadIdx.x == 0) part_rows(a, rr)[(int64_t)L.cx * a.pstride] = make_double2(acc, 0);
    if (!reduce_rows(a, rr, L.cx, 1, tot)) return;
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
    st[ST_REORTH] = 0;
    st[ST_COLUMN] = 0;
    st[ST_END] = 0;
    a.beta[(int64_t)rr * (a.m + 1)] = rin;
    a.ibeta[(int64_t)rr * (a.m + 1)] = 1.0 / rin;
    double2 *gg = a.g + (int64_t)rr * (a.m + 1);
    gg[0] = make_double2(rin, 0);
    for (int i = 1; i <= a.m; ++i) gg[i] = make_double2(0, 0);
}

// ---------------------------------------------------------------- loop control
// Start of a solve: counters, deadline, x = 0 for a zero guess, and whether the
// first true residual needs a product (it does not when x = 0).
__global__ void k_solve_begin(const __grid_constant__ GroupArgs g, cudaGraphConditionalHandle h_first) {
    SolveCtl *c = g.m[0].ctl;
    if (c->zero)
        for (int i = 0; i < g.n; ++i) {
            const GArgs &a = g.m[i];
            const int64_t total = (int64_t)a.nrhs * a.N;
            for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
                 k += (int64_t)gridDim.x * blockDim.x)
                a.x[k] = make_double2(0, 0);
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->j = 0;
        c->sweeps = 0;
        c->timed_out = 0;
        c->outer_bodies = 0;
        c->restart_bodies = 0;
        c->inner_bodies = 0;
        c->reorth_bodies = 0;
        c->reorth_pending = 0;
        c->tick = 0u;
        c->cycle_bodies = 0;
        c->guard = 0;
        c->deadline = c->timeout_ns > 0 ? globaltimer_ns() + (unsigned long long)c->timeout_ns : 0ull;
        c->cond_first = c->zero ? 0 : 1;
        if (g.graph) cudaGraphSetConditional(h_first, c->zero ? 0u : 1u);
    }
}

// After a true residual: another sweep while some RHS is active, within the
// sweep cap and the deadline.
__global__ void k_sweep_ctl(const __grid_constant__ GroupArgs g, cudaGraphConditionalHandle h_sweep) {
    const bool any = any_flag(g, ST_ACTIVE);
    if (threadIdx.x != 0) return;
    SolveCtl *c = g.m[0].ctl;
    c->sweeps += 1;
    const bool late = past_deadline(c);
    if (any && late) c->timed_out = 1;
    const unsigned cond = (any && c->sweeps < c->max_outer && !late && !c->guard) ? 1u : 0u;
    c->cond_sweep = (int)cond;
    if (g.graph) cudaGraphSetConditional(h_sweep, cond);
}

__global__ void k_restart_begin(const __grid_constant__ GroupArgs g, cudaGraphConditionalHandle h_restart) {
    if (threadIdx.x != 0) return;
    SolveCtl *c = g.m[0].ctl;
    c->outer_bodies += 1;
    c->cond_restart = 1;
    if (g.graph) cudaGraphSetConditional(h_restart, 1u);
}

// After a restart: another cycle while some RHS started one (MIXED only).
__global__ void k_restart_ctl(const __grid_constant__ GroupArgs g, cudaGraphConditionalHandle h_restart) {
    const bool any = g.m[0].mixed && any_flag(g, ST_ACTIVE);
    if (threadIdx.x != 0) return;
    SolveCtl *c = g.m[0].ctl;
    const bool late = past_deadline(c);
    if (any && late) c->timed_out = 1;
    const unsigned cond = (any && !late && !c->guard) ? 1u : 0u;
    c->cond_restart = (int)cond;
    if (g.graph) cudaGraphSetConditional(h_restart, cond);
}

__global__ void k_cycle_begin(const __grid_constant__ GroupArgs g) {
    if (threadIdx.x != 0) return;
    SolveCtl *c = g.m[0].ctl;
    c->j = 0;
    c->cycle_bodies = 0;
    c->restart_bodies += 1;
    c->cond_iter = 1;
    if (g.graph) cudaGraphSetConditional(g.h_iter, 1u);
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
    cudaFree(w.cs); cudaFree(w.sn); cudaFree(w.g); cudaFree(w.h1); cudaFree(w.h2);
    cudaFree(w.part); cudaFree(w.nrm); cudaFree(w.st); cudaFree(w.cnt); cudaFree(w.ctl);
    if (w.hst) cudaFreeHost(w.hst);
    if (w.hnrm) cudaFreeHost(w.hnrm);
    w = SolveWs{};
}

// Chunks of a RHS: 256 threads x ELEM elements (ELEM = 4 for large systems),
// and, once there are at least half as many chunks as SMs, their count
// rounded up to a multiple of the SM count with the elements spread evenly,
// so every SM gets the same FP64 work.  Depends on N (and the device) only,
// so a RHS is summed in the same order alone, in any batch and in any group.
struct Geom {
    int threads, elem, per_cta, nchunk;
};
static Geom geom_for(int64_t N, int nsm) {
    const int elem = (N + 255) / 256 >= 8LL * nsm ? 4 : 1;
    const int64_t span = 256LL * elem;
    int64_t nchunk = (N + span - 1) / span;
    if (nchunk >= nsm / 2) nchunk = (nchunk + nsm - 1) / nsm * nsm;
    const int64_t per = (N + nchunk - 1) / nchunk;
    return {256, elem, (int)per, (int)((N + per - 1) / per)};
}


static ztoep_status_t ensure_solve_ws(ztoep_plan_t p, int nrhs, int m) {
    SolveWs &w = p->sws;
    if (w.cap >= nrhs && w.m >= m) return ZTOEP_OK;
    free_solve_ws(p);
    const int64_t N = p->N;
    const Geom gm = geom_for(N, p->nsm);
    const int nrows = tree_rows(gm.nchunk);
    const int cstride = tree_tickets(gm.nchunk);
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
    ZT_TRY(dalloc((void **)&w.h1, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.h2, sizeof(double2) * (size_t)nrhs * (m + 1), &acc));
    ZT_TRY(dalloc((void **)&w.part, sizeof(double2) * (size_t)nrhs * nrows * pstride, &acc));
    ZT_TRY(dalloc((void **)&w.nrm, sizeof(double) * (size_t)nrhs * (NM_STRIDE + 2 * (m + 1)), &acc));
    ZT_TRY(dalloc((void **)&w.st, sizeof(int) * (size_t)nrhs * ST_STRIDE, &acc));
    ZT_TRY(dalloc((void **)&w.cnt, sizeof(unsigned) * (size_t)nrhs * cstride, &acc));
    ZT_TRY(dalloc((void **)&w.ctl, sizeof(SolveCtl), &acc));
    ZT_CUDA(cudaMemset(w.cnt, 0, sizeof(unsigned) * (size_t)nrhs * cstride));
    ZT_CUDA(cudaMallocHost((void **)&w.hst, sizeof(int) * (size_t)nrhs * ST_STRIDE + sizeof(SolveCtl) + 64));
    ZT_CUDA(cudaMallocHost((void **)&w.hnrm, sizeof(double) * (size_t)nrhs * NM_STRIDE));
    w.cap = nrhs;
    w.m = m;
    w.cstride = cstride;
    w.bytes = acc;
    return ZTOEP_OK;
}

// One system of a solve: its plan and RHS count.
struct Member {
    ztoep_plan_t p;
    int nrhs;
};

static GArgs make_args(ztoep_plan_t p, int nrhs, int m, bool mixed, SolveCtl *ctl) {
    SolveWs &w = p->sws;
    const Geom gm = geom_for(p->N, p->nsm);
    GArgs a{};
    a.Vb = w.Vb; a.w = w.w; a.x = w.xbuf; a.v = w.vbuf; a.xin64 = w.xin64; a.rbuf = w.rbuf; a.dbuf = w.dbuf;
    a.x32 = (float2 *)p->ws32.xin; a.y32 = (const float2 *)p->ws32.yout;
    a.H = w.H; a.cs = w.cs; a.sn = w.sn; a.g = w.g; a.h1 = w.h1; a.h2 = w.h2; a.part = w.part;
    a.nrm = w.nrm; a.beta = w.nrm + (size_t)w.cap * NM_STRIDE; a.ibeta = a.beta + (size_t)w.cap * (w.m + 1);
    a.st = w.st; a.cnt = w.cnt;
    a.ctl = ctl;
    a.N = p->N; a.cap = w.cap; a.m = m; a.nchunk = gm.nchunk; a.per_cta = gm.per_cta;
    a.nrows = tree_rows(gm.nchunk); a.cstride = w.cstride; a.pstride = w.m + 2;
    a.nrhs = nrhs;
    a.mixed = mixed ? 1 : 0;
    return a;
}


// The work list of a solve of `n` members (the first member's control block
// is the group's).
static GroupArgs make_group(const Member *mem, int n, int m, bool mixed) {
    GroupArgs g{};
    g.n = n;
    SolveCtl *ctl = (SolveCtl *)mem[0].p->sws.ctl;
    for (int i = 0; i < n; ++i) g.m[i] = make_args(mem[i].p, mem[i].nrhs, m, mixed, ctl);
    return g;
}

static int group_elem(const Member *mem, int n) { return geom_for(mem[0].p->N, mem[0].p->nsm).elem; }

static unsigned group_ctas(const GroupArgs &g, bool extra) {
    unsigned t = 0;
    for (int i = 0; i < g.n; ++i) t += (unsigned)(g.m[i].nchunk + (extra ? 1 : 0)) * g.m[i].nrhs;
    return t;
}

template <int ELEM> struct Launch {
    static ztoep_status_t vnorm(const GroupArgs &g, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_vnorm<ELEM><<<group_ctas(g, false), 256, 0, s>>>(g);
        return ok();
    }
    static ztoep_status_t residual(const GroupArgs &g, int first, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_residual<ELEM><<<group_ctas(g, false), 256, 0, s>>>(g, first);
        return ok();
    }
    static ztoep_status_t arnoldi(const GroupArgs &g, int pass, cudaStream_t s) {
        KScope ks(K_ARNOLDI, s);
        ks.add(pass == 1 ? 2 : 3);
        if (pass == 1) {
            k_dots<ELEM, 1><<<group_ctas(g, false), 256, 0, s>>>(g);
            k_upd<ELEM, 1><<<group_ctas(g, true), 256, 0, s>>>(g);  // (+ one decision CTA per RHS)
        } else {
            k_dots<ELEM, 2><<<group_ctas(g, false), 256, 0, s>>>(g);
            k_upd<ELEM, 2><<<group_ctas(g, false), 256, 0, s>>>(g);
            k_iter_ctl<<<1, 256, 0, s>>>(g);
        }
        return ok();
    }
    static ztoep_status_t update_d(const GroupArgs &g, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_update_d<ELEM><<<group_ctas(g, false), 256, 0, s>>>(g);
        return ok();
    }
    static ztoep_status_t apply_d(const GroupArgs &g, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_apply_d<ELEM><<<group_ctas(g, false), 256, 0, s>>>(g);
        return ok();
    }
    static ztoep_status_t inner_residual(const GroupArgs &g, cudaStream_t s) {
        KScope ks(K_MISC, s);
        k_inner_residual<ELEM><<<group_ctas(g, false), 256, 0, s>>>(g);
        return ok();
    }
    static ztoep_status_t ok() {
        ZT_CUDA(cudaGetLastError());
        return ZTOEP_OK;
    }
};

static unsigned group_rhs(const GroupArgs &g) {
    unsigned t = 0;
    for (int i = 0; i < g.n; ++i) t += (unsigned)g.m[i].nrhs;
    return t;
}

static ztoep_status_t launch_givens(const GroupArgs &g, bool final_, cudaStream_t s) {
    KScope ks(K_ARNOLDI, s);
    if (final_)
        k_givens<true><<<group_rhs(g), 128, 0, s>>>(g);
    else
        k_givens<false><<<group_rhs(g), 128, 0, s>>>(g);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

struct Ops {
    int elem;
    ztoep_status_t vnorm(const GroupArgs &g, cudaStream_t s) const {
        return elem == 4 ? Launch<4>::vnorm(g, s) : Launch<1>::vnorm(g, s);
    }
    ztoep_status_t residual(const GroupArgs &g, int first, cudaStream_t s) const {
        return elem == 4 ? Launch<4>::residual(g, first, s) : Launch<1>::residual(g, first, s);
    }
    ztoep_status_t arnoldi(const GroupArgs &g, int pass, cudaStream_t s) const {
        return elem == 4 ? Launch<4>::arnoldi(g, pass, s) : Launch<1>::arnoldi(g, pass, s);
    }
    ztoep_status_t update_d(const GroupArgs &g, cudaStream_t s) const {
        return elem == 4 ? Launch<4>::update_d(g, s) : Launch<1>::update_d(g, s);
    }
    ztoep_status_t apply_d(const GroupArgs &g, cudaStream_t s) const {
        return elem == 4 ? Launch<4>::apply_d(g, s) : Launch<1>::apply_d(g, s);
    }
    ztoep_status_t inner_residual(const GroupArgs &g, cudaStream_t s) const {
        return elem == 4 ? Launch<4>::inner_residual(g, s) : Launch<1>::inner_residual(g, s);
    }
};

static ztoep_status_t launch_ctl(void (*k)(GroupArgs, cudaGraphConditionalHandle), int blocks, const GroupArgs &g,
                                 cudaGraphConditionalHandle h, cudaStream_t s) {
    KScope ks(K_MISC, s);
    k<<<blocks, 256, 0, s>>>(g, h);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}
static ztoep_status_t launch_ctl(void (*k)(GroupArgs), const GroupArgs &g, cudaStream_t s) {
    KScope ks(K_MISC, s);
    k<<<1, 256, 0, s>>>(g);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// Add conditional nodes after the work captured so far on `s`, all on the
// same dependencies (so they can run concurrently); returns their bodies.
static ztoep_status_t add_conditionals(cudaStream_t s, const cudaGraphConditionalHandle *h, int n,
                                       cudaGraphConditionalNodeType type, cudaGraph_t *bodies) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    ZT_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    if (cst != cudaStreamCaptureStatusActive) return ZTOEP_ERR_CUDA;
    std::vector<cudaGraphNode_t> dep(deps, deps + ndeps), nodes(n);
    for (int i = 0; i < n; ++i) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h[i];
        cp.conditional.type = type;
        cp.conditional.size = 1;
        ZT_CUDA(cudaGraphAddNode(&nodes[i], g, dep.data(), nullptr, dep.size(), &cp));
        bodies[i] = cp.conditional.phGraph_out[0];
    }
    ZT_CUDA(cudaStreamUpdateCaptureDependencies(s, nodes.data(), nullptr, n, cudaStreamSetCaptureDependencies));
    return ZTOEP_OK;
}
static ztoep_status_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                      cudaGraph_t *body) {
    return add_conditionals(s, &h, 1, type, body);
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

// Events of one graph capture (fork/join of the members' products).
struct CaptureEvents {
    std::vector<cudaEvent_t> ev;
    ~CaptureEvents() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    ztoep_status_t make(cudaEvent_t *out) {
        cudaEvent_t e = nullptr;
        ZT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ev.push_back(e);
        *out = e;
        return ZTOEP_OK;
    }
};

// Product of every member on its own buffers: FP32 (x32 -> y32) or FP64
// (in64 -> w), the members concurrently (member 0 on `s`, the others on their
// plans' capture streams, joined back to `s`).
static ztoep_status_t member_products(const Member *mem, int n, bool fp32, bool xbuf_in, cudaStream_t s,
                                      CaptureEvents &ce) {
    auto one = [&](int i, cudaStream_t si) -> ztoep_status_t {
        ztoep_plan_t p = mem[i].p;
        if (fp32) return run_matvec<float>(p, mem[i].nrhs, (const float2 *)p->ws32.xin, (float2 *)p->ws32.yout, si);
        return run_matvec<double>(p, mem[i].nrhs, xbuf_in ? p->sws.xbuf : p->sws.xin64, p->sws.w, si);
    };
    if (n == 1) return one(0, s);
    cudaEvent_t fork = nullptr;
    ZT_TRY(ce.make(&fork));
    ZT_CUDA(cudaEventRecord(fork, s));
    for (int i = 1; i < n; ++i) {
        cudaStream_t si = mem[i].p->cap;
        ZT_CUDA(cudaStreamWaitEvent(si, fork, 0));
        ZT_TRY(one(i, si));
        cudaEvent_t join = nullptr;
        ZT_TRY(ce.make(&join));
        ZT_CUDA(cudaEventRecord(join, si));
        ZT_CUDA(cudaStreamWaitEvent(s, join, 0));
    }
    return one(0, s);
}

// Whole solve as one graph:
//   begin -> IF(x != 0){FP64 products} -> residual -> sweep control ->
//   WHILE(sweep){ restart begin ->
//                 WHILE(restart){ cycle begin -> WHILE(iter){products, Arnoldi (+ iteration control)}
//                                 -> d += V y -> [MIXED: FP32 products of d, r_in = r - Z d]
//                                 -> restart control }
//                 -> x += d -> FP64 products -> residual -> sweep control }
// The Arnoldi step is k_dots + k_upd, whose last CTA runs the iteration
// control; a RHS that asks for a second Gram-Schmidt pass makes it set the IF
// node that runs k_dots<2>, k_upd<2> and the iteration control instead.  The
// Givens rotations of a step's column run in the next iteration (k_givens; for
// one system on a branch beside its product, for a group after the members'
// products) and after the loop for the last column, so the end of a cycle is
// seen one step late: that step's work is discarded.  In a
// group of several members, each member's iteration product sits in its own
// IF node (members with no RHS in a cycle skip it) and the members' products
// run concurrently; every other kernel is one launch for all members.
static ztoep_status_t build_graph(const Member *mem, int n, SolveGraph &sg, int prec, int m) {
    const bool mixed = prec == ZTOEP_MIXED;
    GroupArgs g = make_group(mem, n, m, mixed);
    const Ops ops{group_elem(mem, n)};
    ztoep_plan_t p0 = mem[0].p;
    cudaStream_t s = p0->cap;
    CaptureEvents ce;
    cudaGraph_t top = nullptr;
    ZT_CUDA(cudaGraphCreate(&top, 0));
    sg.graph = top;
    g.graph = 1;
    g.prod_if = n > 1 ? 1 : 0;
    cudaGraphConditionalHandle h_first, h_sweep;
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_first, top, 0, 0));
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_sweep, top, 0, 0));
    cudaGraph_t body_first = nullptr, body_sweep = nullptr, body_iter = nullptr;

    // top level.  GroupArgs is copied into every launch when it is captured,
    // so each loop handle is created before the first kernel that sets it is
    // captured (k_cycle_begin: h_iter; k_upd<1> and k_iter_ctl: h_iter,
    // h_reorth and the members' h_prod).
    ZT_TRY(capture_begin(s, top, &sg.k_fixed));
    for (int i = 0; i < n; ++i) {
        SolveWs &w = mem[i].p->sws;
        ZT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(int) * (size_t)w.cap * ST_STRIDE, s));
        ZT_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * (size_t)w.cap * w.cstride, s));
    }
    int64_t elems = 0;
    for (int i = 0; i < n; ++i) elems += (int64_t)mem[i].nrhs * mem[i].p->N;
    const int zblocks = (int)std::min<int64_t>(4 * p0->nsm, (elems + 255) / 256);
    ZT_TRY(launch_ctl(k_solve_begin, std::max(1, zblocks), g, h_first, s));
    ZT_TRY(ops.vnorm(g, s));
    ZT_TRY(add_conditional(s, h_first, cudaGraphCondTypeIf, &body_first));
    ZT_TRY(ops.residual(g, 1, s));
    ZT_TRY(launch_ctl(k_sweep_ctl, 1, g, h_sweep, s));
    ZT_TRY(add_conditional(s, h_sweep, cudaGraphCondTypeWhile, &body_sweep));
    ZT_TRY(capture_end(s));

    // first products (skipped for a zero guess)
    ZT_TRY(capture_begin(s, body_first, &sg.k_first_product));
    ZT_TRY(member_products(mem, n, false, true, s, ce));
    ZT_TRY(capture_end(s));

    // one sweep: inner restarts, x += d, FP64 residual
    cudaGraphConditionalHandle h_restart;
    cudaGraph_t body_restart = nullptr;
    ZT_CUDA(cudaGraphConditionalHandleCreate(&h_restart, body_sweep, 0, 0));
    ZT_TRY(capture_begin(s, body_sweep, &sg.k_sweep));
    ZT_TRY(launch_ctl(k_restart_begin, 1, g, h_restart, s));
    ZT_TRY(add_conditional(s, h_restart, cudaGraphCondTypeWhile, &body_restart));
    ZT_TRY(ops.apply_d(g, s));
    ZT_TRY(member_products(mem, n, false, true, s, ce));
    ZT_TRY(ops.residual(g, 0, s));
    ZT_TRY(launch_ctl(k_sweep_ctl, 1, g, h_sweep, s));
    ZT_TRY(capture_end(s));

    // one restart: GMRES cycle, d += V y, FP32 inner residual (MIXED)
    ZT_CUDA(cudaGraphConditionalHandleCreate(&g.h_iter, body_restart, 0, 0));
    ZT_TRY(capture_begin(s, body_restart, &sg.k_restart));
    ZT_TRY(launch_ctl(k_cycle_begin, g, s));
    ZT_TRY(add_conditional(s, g.h_iter, cudaGraphCondTypeWhile, &body_iter));
    ZT_TRY(launch_givens(g, true, s));
    ZT_TRY(ops.update_d(g, s));
    if (mixed) {
        ZT_TRY(member_products(mem, n, true, false, s, ce));
        ZT_TRY(ops.inner_residual(g, s));
    }
    ZT_TRY(launch_ctl(k_restart_ctl, 1, g, h_restart, s));
    ZT_TRY(capture_end(s));

    // one iteration; the second Gram-Schmidt pass only when a RHS asked for it
    // (its condition starts at 0 in every iteration)
    cudaGraph_t body_reorth = nullptr;
    ZT_CUDA(cudaGraphConditionalHandleCreate(&g.h_reorth, body_iter, 0, cudaGraphCondAssignDefault));
    cudaGraph_t body_prod[kMaxMembers] = {};
    if (g.prod_if)
        for (int i = 0; i < n; ++i)
            ZT_CUDA(cudaGraphConditionalHandleCreate(&g.h_prod[i], body_iter, 1, cudaGraphCondAssignDefault));
    ZT_TRY(capture_begin(s, body_iter, &sg.k_iter));
    if (g.prod_if) {
        // members' products in IF nodes (all roots of the body), then the
        // previous column's rotations: a kernel root beside several IF roots
        // stalled the graph on GB300 (5 members), this order did not
        ZT_TRY(add_conditionals(s, g.h_prod, n, cudaGraphCondTypeIf, body_prod));
        ZT_TRY(launch_givens(g, false, s));
    } else {
        // the previous column's rotations on a branch beside the product
        cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr;
        ZT_TRY(ce.make(&ev_g0));
        ZT_TRY(ce.make(&ev_g1));
        ZT_CUDA(cudaEventRecord(ev_g0, s));
        ZT_CUDA(cudaStreamWaitEvent(p0->aux, ev_g0, 0));
        ZT_TRY(launch_givens(g, false, p0->aux));
        ZT_CUDA(cudaEventRecord(ev_g1, p0->aux));
        if (mixed)
            ZT_TRY(run_matvec<float>(p0, mem[0].nrhs, (const float2 *)p0->ws32.xin, (float2 *)p0->ws32.yout, s));
        else
            ZT_TRY(run_matvec<double>(p0, mem[0].nrhs, p0->sws.xin64, p0->sws.w, s));
        ZT_CUDA(cudaStreamWaitEvent(s, ev_g1, 0));
    }
    ZT_TRY(ops.arnoldi(g, 1, s));
    ZT_TRY(add_conditional(s, g.h_reorth, cudaGraphCondTypeIf, &body_reorth));
    ZT_TRY(capture_end(s));
    ZT_TRY(capture_begin(s, body_reorth, &sg.k_reorth));
    ZT_TRY(ops.arnoldi(g, 2, s));
    ZT_TRY(capture_end(s));
    for (int i = 0; g.prod_if && i < n; ++i) {  // each member's iteration product
        ztoep_plan_t p = mem[i].p;
        uint64_t cnt = 0;
        ZT_TRY(capture_begin(p->cap, body_prod[i], &cnt));
        if (mixed)
            ZT_TRY(run_matvec<float>(p, mem[i].nrhs, (const float2 *)p->ws32.xin, (float2 *)p->ws32.yout, p->cap));
        else
            ZT_TRY(run_matvec<double>(p, mem[i].nrhs, p->sws.xin64, p->sws.w, p->cap));
        ZT_TRY(capture_end(p->cap));
        sg.k_iter += cnt;
    }

    ZT_CUDA(cudaGraphInstantiate(&sg.exec, top, 0));
    sg.prec = prec;
    sg.nrhs = mem[0].nrhs;
    sg.m = m;
    return ZTOEP_OK;
}

static void abandon_capture(const Member *mem, int n) {
    capture_count_end();
    for (int i = 0; i < n; ++i) {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(mem[i].p->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(mem[i].p->cap, &junk);
            if (junk) cudaGraphDestroy(junk);
        }
    }
    cudaGetLastError();
}

static void destroy_graph(SolveGraph &sg) {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (sg.graph) cudaGraphDestroy(sg.graph);
    sg = SolveGraph{};
}

// Cached graph of a single-system solve (instantiated once per precision, RHS
// count and restart length).
static ztoep_status_t get_graph(ztoep_plan_t p, int prec, int nrhs, int m, SolveGraph **out) {
    for (auto &g : p->graphs)
        if (g.exec && g.prec == prec && g.nrhs == nrhs && g.m == m) {
            *out = &g;
            return ZTOEP_OK;
        }
    SolveGraph &slot = p->graphs[p->graph_next];
    p->graph_next = (p->graph_next + 1) % 4;
    destroy_graph(slot);
    const Member mem{p, nrhs};
    ztoep_status_t st = build_graph(&mem, 1, slot, prec, m);
    if (st != ZTOEP_OK) {
        abandon_capture(&mem, 1);
        destroy_graph(slot);
        return st;
    }
    *out = &slot;
    return ZTOEP_OK;
}

// The same solve with the loops driven from the host: every kernel is a
// separate launch (for profilers that cannot look inside conditional graph
// nodes).  The loop decisions are read back from the control block.
static ztoep_status_t run_host_loop(const Member *mem, int n, int prec, int m, cudaStream_t s) {
    const bool mixed = prec == ZTOEP_MIXED;
    GroupArgs g = make_group(mem, n, m, mixed);
    const Ops ops{group_elem(mem, n)};
    SolveWs &w0 = mem[0].p->sws;
    SolveCtl *hc = reinterpret_cast<SolveCtl *>(w0.hst + (size_t)w0.cap * ST_STRIDE);
    CaptureEvents ce;
    auto read_ctl = [&]() -> ztoep_status_t {
        ZT_CUDA(cudaMemcpyAsync(hc, w0.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
        ZT_CUDA(cudaStreamSynchronize(s));
        return ZTOEP_OK;
    };
    const cudaGraphConditionalHandle none = 0;
    for (int i = 0; i < n; ++i) {
        SolveWs &w = mem[i].p->sws;
        ZT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(int) * (size_t)w.cap * ST_STRIDE, s));
        ZT_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * (size_t)w.cap * w.cstride, s));
    }
    int64_t elems = 0;
    for (int i = 0; i < n; ++i) elems += (int64_t)mem[i].nrhs * mem[i].p->N;
    const int zblocks = (int)std::min<int64_t>(4 * mem[0].p->nsm, (elems + 255) / 256);
    ZT_TRY(launch_ctl(k_solve_begin, std::max(1, zblocks), g, none, s));
    ZT_TRY(ops.vnorm(g, s));
    ZT_TRY(read_ctl());
    if (hc->cond_first) ZT_TRY(member_products(mem, n, false, true, s, ce));
    ZT_TRY(ops.residual(g, 1, s));
    ZT_TRY(launch_ctl(k_sweep_ctl, 1, g, none, s));
    ZT_TRY(read_ctl());
    while (hc->cond_sweep) {
        ZT_TRY(launch_ctl(k_restart_begin, 1, g, none, s));
        for (;;) {
            ZT_TRY(launch_ctl(k_cycle_begin, g, s));
            for (int it = 0; it < m; ++it) {
                ZT_TRY(launch_givens(g, false, s));
                ZT_TRY(member_products(mem, n, mixed, false, s, ce));
                ZT_TRY(ops.arnoldi(g, 1, s));
                ZT_TRY(read_ctl());
                if (hc->reorth_pending) {
                    ZT_TRY(ops.arnoldi(g, 2, s));
                    ZT_TRY(read_ctl());
                }
                if (!hc->cond_iter) break;
            }
            ZT_TRY(launch_givens(g, true, s));
            ZT_TRY(ops.update_d(g, s));
            if (mixed) {
                ZT_TRY(member_products(mem, n, true, false, s, ce));
                ZT_TRY(ops.inner_residual(g, s));
            }
            ZT_TRY(launch_ctl(k_restart_ctl, 1, g, none, s));
            ZT_TRY(read_ctl());
            if (!hc->cond_restart) break;
        }
        ZT_TRY(ops.apply_d(g, s));
        ZT_TRY(member_products(mem, n, false, true, s, ce));
        ZT_TRY(ops.residual(g, 0, s));
        ZT_TRY(launch_ctl(k_sweep_ctl, 1, g, none, s));
        ZT_TRY(read_ctl());
    }
    return ZTOEP_OK;
}

// Runs the solve of the members (V / X already in each member's vbuf / xbuf,
// X only without a zero guess) on `s` and fetches the per-RHS states.  `sg`:
// the graph to launch, or null for the host-driven loop.
static ztoep_status_t solve_core(const Member *mem, int n, const ztoep_solve_opts_t *o, SolveGraph *sg,
                                 ztoep_solve_info_t *const *info, cudaStream_t s) {
    const int m = o->restart;
    SolveWs &w0 = mem[0].p->sws;
    SolveCtl *hc = reinterpret_cast<SolveCtl *>(w0.hst + (size_t)w0.cap * ST_STRIDE);
    std::memset(hc, 0, sizeof(SolveCtl));
    hc->zero = (o->flags & ZTOEP_FLAG_ZERO_GUESS) ? 1 : 0;
    hc->max_iter = o->max_iter;
    hc->max_outer = o->max_outer;
    hc->tol = o->tol;
    hc->inner_tol = o->inner_tol;
    hc->timeout_ns = o->timeout_ns;
    ZT_CUDA(cudaMemcpyAsync(w0.ctl, hc, sizeof(SolveCtl), cudaMemcpyHostToDevice, s));
    if (!sg)
        ZT_TRY(run_host_loop(mem, n, o->prec, m, s));
    else
        ZT_CUDA(cudaGraphLaunch(sg->exec, s));
    std::vector<int> dev_err(n, 0);
    for (int i = 0; i < n; ++i) {
        SolveWs &w = mem[i].p->sws;
        ZT_CUDA(cudaMemcpyAsync(w.hst, w.st, sizeof(int) * (size_t)mem[i].nrhs * ST_STRIDE, cudaMemcpyDeviceToHost, s));
        ZT_CUDA(cudaMemcpyAsync(w.hnrm, w.nrm, sizeof(double) * (size_t)mem[i].nrhs * NM_STRIDE,
                                cudaMemcpyDeviceToHost, s));
        ZT_CUDA(cudaMemcpyAsync(&dev_err[i], mem[i].p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    ZT_CUDA(cudaMemcpyAsync(hc, w0.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaStreamSynchronize(s));
    if (sg)
        add_launches(sg->k_fixed + (hc->zero ? 0 : sg->k_first_product) + (uint64_t)hc->outer_bodies * sg->k_sweep +
                     (uint64_t)hc->restart_bodies * sg->k_restart + (uint64_t)hc->inner_bodies * sg->k_iter +
                     (uint64_t)hc->reorth_bodies * sg->k_reorth);
    const bool timed_out = hc->timed_out != 0;
    ztoep_status_t worst = ZTOEP_OK;
    for (int i = 0; i < n; ++i) {
        if (dev_err[i] != 0) ZT_CUDA(cudaMemsetAsync(mem[i].p->err, 0, sizeof(int), s));  // a bounded wait gave up
        for (int rr = 0; rr < mem[i].nrhs; ++rr) {
            const int *st = mem[i].p->sws.hst + rr * ST_STRIDE;
            const double *nm = mem[i].p->sws.hnrm + rr * NM_STRIDE;
            ztoep_status_t rs;
            switch (st[ST_STATUS]) {
                case RS_CONVERGED: rs = ZTOEP_OK; break;
                case RS_NONFINITE: rs = ZTOEP_ERR_NONFINITE; break;
                case RS_MAXITER: rs = ZTOEP_ERR_NOCONV; break;
                default: rs = timed_out ? ZTOEP_ERR_TIMEOUT : ZTOEP_ERR_NOCONV; break;
            }
            if (dev_err[i] != 0) rs = ZTOEP_ERR_TIMEOUT;
            if (rs != ZTOEP_OK && (worst == ZTOEP_OK || rs == ZTOEP_ERR_NONFINITE || rs == ZTOEP_ERR_TIMEOUT))
                worst = rs;
            if (info && info[i]) {
                info[i][rr].outer = st[ST_OUTER];
                info[i][rr].inner_iters = st[ST_ITERS];
                info[i][rr].status = rs;
                info[i][rr].rel_residual = nm[NM_VNORM] > 0 ? nm[NM_RNORM] / nm[NM_VNORM] : nm[NM_RNORM];
                info[i][rr].second_passes = st[ST_PASSES2];
            }
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

static bool hard_error(ztoep_status_t st) {
    return st == ZTOEP_ERR_ARG || st == ZTOEP_ERR_CUDA || st == ZTOEP_ERR_NOMEM || st == ZTOEP_ERR_UNSUPPORTED;
}

// One system: the plan's cached graph (or the host-driven loop).
static ztoep_status_t solve_single(ztoep_plan_t p, const ztoep_solve_opts_t *o, int nrhs, ztoep_solve_info_t *info,
                                   cudaStream_t s) {
    SolveGraph *g = nullptr;
    if (!(o->flags & ZTOEP_FLAG_HOST_LOOP)) ZT_TRY(get_graph(p, o->prec, nrhs, o->restart, &g));
    const Member mem{p, nrhs};
    ztoep_solve_info_t *const infos[1] = {info};
    return solve_core(&mem, 1, o, g, infos, s);
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
    const ztoep_status_t st = solve_single(p, o, nrhs, info, s);
    if (hard_error(st)) return st;
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
    const ztoep_status_t st = solve_single(p, o, nrhs, info, s);
    if (hard_error(st)) return st;
    ZT_CUDA(cudaMemcpyAsync(Xh, w.xbuf, bytes, cudaMemcpyDeviceToHost, s));
    ZT_CUDA(cudaStreamSynchronize(s));
    return st;
}

ztoep_status_t ztoep_solve_group(int32_t count, const ztoep_plan_t *plans, const ztoep_solve_opts_t *o,
                                 const int32_t *nrhs, const void *const *V, void *const *X,
                                 ztoep_solve_info_t *const *info, void *stream) {
    if (count < 1 || count > kMaxMembers || !plans || !valid_opts(o) || !nrhs || !V || !X) return ZTOEP_ERR_ARG;
    Member mem[kMaxMembers];
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || nrhs[i] < 1 || !V[i] || !X[i] || V[i] == X[i]) return ZTOEP_ERR_ARG;
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return ZTOEP_ERR_ARG;  // each member needs its own plan (workspace)
        if (plans[i]->device != plans[0]->device) return ZTOEP_ERR_ARG;
        mem[i] = Member{plans[i], nrhs[i]};
    }
    // one launch per step needs one chunk shape (elements per thread) for all
    for (int i = 1; i < count; ++i)
        if (geom_for(plans[i]->N, plans[i]->nsm).elem != geom_for(plans[0]->N, plans[0]->nsm).elem)
            return ZTOEP_ERR_UNSUPPORTED;
    // lock the plans in address order (no deadlock with other group calls)
    std::vector<ztoep_plan_t> order(plans, plans + count);
    std::sort(order.begin(), order.end());
    std::vector<std::unique_lock<std::mutex>> locks;
    for (ztoep_plan_t p : order) locks.emplace_back(p->mu);
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        ztoep_plan_t p = mem[i].p;
        ZT_TRY(prepare(p, o, mem[i].nrhs, s));
        const size_t bytes = sizeof(double2) * (size_t)mem[i].nrhs * p->N;
        ZT_CUDA(cudaMemcpyAsync(p->sws.vbuf, V[i], bytes, cudaMemcpyDeviceToDevice, s));
        if (!(o->flags & ZTOEP_FLAG_ZERO_GUESS))
            ZT_CUDA(cudaMemcpyAsync(p->sws.xbuf, X[i], bytes, cudaMemcpyDeviceToDevice, s));
    }
    ztoep_status_t st;
    if (count == 1) {
        st = solve_single(mem[0].p, o, mem[0].nrhs, info ? info[0] : nullptr, s);
    } else if (o->flags & ZTOEP_FLAG_HOST_LOOP) {
        st = solve_core(mem, count, o, nullptr, info, s);
    } else {
        // the members' copies of V and X above are ordered before the graph on s
        SolveGraph sg;
        st = build_graph(mem, count, sg, o->prec, o->restart);
        if (st != ZTOEP_OK) {
            abandon_capture(mem, count);
            destroy_graph(sg);
            return st;
        }
        st = solve_core(mem, count, o, &sg, info, s);
        if (hard_error(st)) cudaStreamSynchronize(s);
        destroy_graph(sg);  // the graph has finished (solve_core synchronised the stream)
    }
    if (hard_error(st)) return st;
    for (int i = 0; i < count; ++i) {
        ztoep_plan_t p = mem[i].p;
        ZT_CUDA(cudaMemcpyAsync(X[i], p->sws.xbuf, sizeof(double2) * (size_t)mem[i].nrhs * p->N,
                                cudaMemcpyDeviceToDevice, s));
    }
    return st;
}

}  // extern "C"
